"""Ball sets on the tensor-core sphere-set walker (|c|^2 - 2 x.c by tcgen05.mma, balls sorted by
radius into 16-ball chunks, or 32-ball ones from 128 tiles of 64 balls up in d <= 8, exact FP32
refinement of the best chunk, lower bound for the rest).

* the distance bound never exceeds the exact FP64 distance |x - c| - r (minus box) and is
  tight for most points;
* walks agree with the FP64 oracle and with the CUDA-core ball screen (same Philox streams),
  within 4 combined standard errors;
* with exponential boundary data the estimates match the exact solution u = exp(a.x).
"""
import ctypes
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle  # noqa: E402
from paper_2406_01713_gb300 import _lib, synth  # noqa: E402
from paper_2406_01713_gb300 import wos as W  # noqa: E402


def np_(t):
    return t.detach().cpu().numpy()


def within(a, se_a, b, se_b, k=4.0, atol=1e-4):
    return np.abs(a - b) <= k * np.sqrt(se_a ** 2 + se_b ** 2) + atol


def ball_problem(d, B, sigma, seed, n_queries):
    rng = np.random.default_rng(seed)
    c = rng.uniform(-1, 1, size=(B, d))
    r = np.exp(rng.uniform(math.log(0.01), math.log(0.2), size=B))
    a = rng.standard_normal(d)
    a *= math.sqrt(sigma) / np.linalg.norm(a)
    dom = {"d": d, "box_lo": -np.ones(d), "box_hi": np.ones(d), "ball_c": c, "ball_r": r,
           "exp_w": np.ones(1), "exp_a": a[None, :]}
    X = synth._free_points(rng, n_queries, -np.ones(d), np.ones(d), c, r, 0.01)
    return dom, X, rng


def exact_radius(dom, X, block=256):
    c, r = dom["ball_c"], dom["ball_r"]
    db = np.concatenate([(np.sqrt(((X[i:i + block, None, :] - c[None, :, :]) ** 2).sum(-1)) - r[None, :]).min(1)
                         for i in range(0, X.shape[0], block)])
    box = np.minimum(X - dom["box_lo"][None, :], dom["box_hi"][None, :] - X).min(1)
    return np.minimum(db, box)


def gpu_radius(D, X):
    L = _lib.load()
    x = torch.tensor(X, dtype=torch.float64, device="cuda")
    out = torch.full((X.shape[0],), float("nan"), dtype=torch.float64, device="cuda")
    _lib.check(L.wos_debug_pointcloud_radius(D.h, ctypes.c_void_p(x.data_ptr()), X.shape[0],
                                             ctypes.c_void_p(out.data_ptr()), None), "radius")
    torch.cuda.synchronize()
    return np_(out)


@pytest.mark.parametrize("d,B", [(3, 4096), (3, 8192), (7, 1000), (8, 9000), (10, 600), (12, 800), (12, 2048)])
def test_radius_bound_is_safe_and_tight(d, B):
    """Both chunk widths (32 columns for the 8192 and 9000 balls) and both contraction lengths."""
    dom, X, rng = ball_problem(d, B, 4.0, 11 + d, 2000)
    D = W.Domain(dom)
    # also points close to ball surfaces (outside them)
    idx = rng.integers(0, B, size=2000)
    v = rng.standard_normal((2000, d))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    near = dom["ball_c"][idx] + (dom["ball_r"][idx] + 10 ** rng.uniform(-4, -1.5, size=2000))[:, None] * v
    near = near[np.all(np.abs(near) < 0.999, axis=1)]
    want_near = exact_radius(dom, near)
    Y = np.vstack([X, near[want_near > 0]])
    want = exact_radius(dom, Y)
    got = gpu_radius(D, Y)
    assert np.all(np.isfinite(got))
    assert np.all(got <= want * (1 + 1e-5) + 2e-6), np.max(got - want)
    rel = (want - got) / np.maximum(want, 1e-12)
    assert np.mean(rel < 1e-3) > 0.9, np.mean(rel < 1e-3)
    assert np.mean(rel < 0.5) > 0.99


@pytest.mark.parametrize("d,B", [(3, 2048), (6, 512), (11, 600)])
def test_walks_match_oracle_and_cuda_core_screen(d, B):
    dom, X, _ = ball_problem(d, B, 9.0, 5 + d, 12)
    D = W.Domain(dom)
    N, eps, sigma, seed = 4096, 1e-3, 9.0, 3
    ref = oracle.solve(dom, X, N, eps, sigma, seed, grad=True, control_variate=True)
    tc = D.grad(X, N, eps, sigma, seed=seed, with_stats=True, control_variate=True)
    cc = D.grad(X, N, eps, sigma, seed=seed, with_stats=True, control_variate=True, cuda_core_balls=True)
    for got in (tc, cc):
        st = W.stats_dict(got["stats"])
        assert st["walks"] == 12 * N and st["outside"] == 0
        assert np.all(within(np_(got["u"]), np_(got["u_se"]), ref["u"], ref["u_se"]))
        assert np.all(within(np_(got["grad"]), np_(got["grad_se"]), ref["grad"], ref["grad_se"], atol=1e-4))
    # exact solution u = exp(a.x) (|a|^2 = sigma) on any domain
    a = dom["exp_a"][0]
    ex = np.exp(X @ a)
    u, se = np_(tc["u"]), np_(tc["u_se"])
    assert np.all(np.abs(u - ex) <= 4.5 * se + 3e-3 * ex)


def test_wide_chunks_match_oracle_alone_and_batched():
    """A set of 8192 balls (128 tiles: 32-column candidate chunks) in d = 5: the walks against the
    oracle, and the same problem in a batch beside a 16-column set takes the same walks."""
    dom, X, _ = ball_problem(5, 8192, 9.0, 41, 8)
    D = W.Domain(dom)
    assert D.info()["tensor_sphere_set"] and D.info()["sphere_tiles"] == 128
    N, eps, sigma, seed = 1024, 1e-3, 9.0, 6
    ref = oracle.solve(dom, X, N, eps, sigma, seed, grad=True, control_variate=True)
    got = D.grad(X, N, eps, sigma, seed=seed, with_stats=True, control_variate=True)
    st = W.stats_dict(got["stats"])
    assert st["walks"] == 8 * N and st["outside"] == 0
    assert np.all(within(np_(got["u"]), np_(got["u_se"]), ref["u"], ref["u_se"]))
    assert np.all(within(np_(got["grad"]), np_(got["grad_se"]), ref["grad"], ref["grad_se"]))
    a = dom["exp_a"][0]
    ex = np.exp(X @ a)
    assert np.all(np.abs(np_(got["u"]) - ex) <= 4.5 * np_(got["u_se"]) + 3e-3 * ex)
    dom2, X2, _ = ball_problem(5, 700, sigma, 42, 16)
    b = W.Batch([{"domain": D, "x": X, "n_walks": N, "eps": eps, "sigma": sigma, "grad": True},
                 {"domain": W.Domain(dom2), "x": X2, "n_walks": 256, "eps": eps, "sigma": sigma, "grad": True}],
                seed=seed, control_variate=True)
    out = b.run()
    torch.cuda.synchronize()
    assert np.array_equal(np_(out[0]["walk_steps"]).sum(), st["walk_steps"])
    for k in ("u", "grad"):
        assert np.allclose(np_(out[0][k]), np_(got[k]), rtol=1e-12, atol=1e-15), k
    b.close()


def test_large_problem_exact_solution():
    dom, X, _ = ball_problem(8, 4096, 16.0, 99, 64)
    D = W.Domain(dom)
    r = D.grad(X, 8192, 1e-3, 16.0, seed=1, with_stats=True, control_variate=True)
    st = W.stats_dict(r["stats"])
    assert st["walks"] == 64 * 8192 and st["outside"] == 0 and st["capped"] == 0
    a = dom["exp_a"][0]
    ex = np.exp(X @ a)
    u, se = np_(r["u"]), np_(r["u_se"])
    assert np.mean(np.abs(u - ex) <= 4.5 * se + 3e-3 * ex) > 0.98
    g, gse = np_(r["grad"]), np_(r["grad_se"])
    gx = a[None, :] * ex[:, None]
    assert np.mean(np.abs(g - gx) <= 4.5 * gse + 3e-2 * np.abs(gx).max(axis=1, keepdims=True)) > 0.97


def test_batch_mixes_tensor_and_cuda_core_problems():
    """A batch with large ball sets (tensor-core sphere walker, one launch per dimension), small
    ones (CUDA-core walker) and a point set, in one graph: every problem matches the oracle."""
    specs = [(3, 2048, 4.0), (5, 16, 9.0), (5, 700, 1.0), (7, 64, 0.0), (8, 1024, 16.0), (3, 600, 25.0), (12, 900, 9.0)]
    probs, refs, base, seed = [], [], 0, 11
    for i, (d, B, sigma) in enumerate(specs):
        dom, X, _ = ball_problem(d, B, sigma, 100 + i, 6)
        N = 2048
        probs.append({"domain": W.Domain(dom), "x": X, "n_walks": N, "eps": 1e-3, "sigma": sigma, "grad": True})
        refs.append(oracle.solve(dom, X, N, 1e-3, sigma, seed, walk_offset=base, grad=True, control_variate=True))
        base += X.shape[0] * N
    rng = np.random.default_rng(3)
    pts = synth.ellipsoid_cloud(rng, 6, 2, 300)
    a = rng.standard_normal(6)
    a *= 2.0 / np.linalg.norm(a)
    pdom = {"d": 6, "box_lo": -np.ones(6), "box_hi": np.ones(6), "points": pts, "exp_w": np.ones(1),
            "exp_a": a[None, :]}
    Xp = rng.uniform(-0.8, 0.8, size=(6, 6))
    probs.append({"domain": W.Domain(pdom), "x": Xp, "n_walks": 2048, "eps": 1e-3, "sigma": 4.0, "grad": True})
    refs.append(oracle.solve(pdom, Xp, 2048, 1e-3, 4.0, seed, walk_offset=base, grad=True, control_variate=True))
    B_ = W.Batch(probs, seed=seed, control_variate=True)
    out = B_.run()
    torch.cuda.synchronize()
    st = W.stats_dict(B_.stats)
    assert st["walks"] == sum(p["x"].shape[0] * p["n_walks"] for p in probs) and st["outside"] == 0
    for o, ref in zip(out, refs):
        assert np.all(within(np_(o["u"]), np_(o["u_se"]), ref["u"], ref["u_se"]))
        assert np.all(within(np_(o["grad"]), np_(o["grad_se"]), ref["grad"], ref["grad_se"], atol=1e-4))
    B_.close()


@pytest.mark.parametrize("B", [40, 2048])
def test_per_query_sums_equal_per_walk_means(B):
    """The per-query reduction (per-walk records summed per query in FP64, in a fixed order)
    gives the mean of the per-walk outputs exactly up to FP64 summation order, on the CUDA-core
    screen (40 balls) and the tensor-core sphere walker (2048 balls), alone and in a batch, with
    few walks per query over many queries; the integer counters are exact, and repeated runs
    agree bit for bit."""
    d, N, Q, eps, sigma, seed = 3, 5, 300, 1e-3, 9.0, 21
    dom, X, _ = ball_problem(d, B, sigma, 70 + B, Q)
    D = W.Domain(dom)
    assert D.info()["tensor_sphere_set"] == (B >= 2048)
    per = D.walks(X, N, eps, sigma, grad_mode=True, seed=seed, walk_offset=10)
    got = D.grad(X, N, eps, sigma, seed=seed, walk_offset=10, with_stats=True)
    st = W.stats_dict(got["stats"])
    assert st["walks"] == Q * N and st["outside"] == 0
    assert st["walk_steps"] == int(np_(per["jumps"]).sum()) + Q * N
    assert np.allclose(np_(got["u"]), np_(per["term"]).mean(1), rtol=1e-12, atol=1e-15)
    # the per-walk gradient and d/dsigma outputs are FP32 products (gt v0, term dsigma) where the
    # sums take them in FP64: agreement to FP32 rounding of each walk's term
    pg, pd = np_(per["grad"]), np_(per["dsigma"])
    assert np.all(np.abs(np_(got["grad"]) - pg.mean(1)) <= 2e-7 * np.abs(pg).mean(1) + 1e-12)
    assert np.all(np.abs(np_(got["du_dsigma"]) - pd.mean(1)) <= 2e-7 * np.abs(pd).mean(1) + 1e-12)
    again = D.grad(X, N, eps, sigma, seed=seed, walk_offset=10, control_variate=True)
    again2 = D.grad(X, N, eps, sigma, seed=seed, walk_offset=10, control_variate=True)
    for k in ("u", "u_se", "grad", "grad_se", "du_dsigma"):
        assert torch.equal(again[k], again2[k]), k
    # a batch of both kinds, same walks (walk indices follow the problems in order)
    dom2, X2, _ = ball_problem(d, 2048 if B < 2048 else 40, sigma, 90 + B, 200)
    D2 = W.Domain(dom2)
    b = W.Batch([{"domain": D, "x": X, "n_walks": N, "eps": eps, "sigma": sigma, "grad": True},
                 {"domain": D2, "x": X2, "n_walks": 3, "eps": eps, "sigma": sigma, "grad": True}], seed=seed)
    out = b.run()
    torch.cuda.synchronize()
    per2 = D2.walks(X2, 3, eps, sigma, grad_mode=True, seed=seed, walk_offset=Q * N)
    per1 = D.walks(X, N, eps, sigma, grad_mode=True, seed=seed, walk_offset=0)
    for o, p in ((out[0], per1), (out[1], per2)):
        assert np.allclose(np_(o["u"]), np_(p["term"]).mean(1), rtol=1e-12, atol=1e-15)
        pg = np_(p["grad"])
        assert np.all(np.abs(np_(o["grad"]) - pg.mean(1)) <= 2e-7 * np.abs(pg).mean(1) + 1e-12)
        assert np.array_equal(np_(o["walk_steps"]), np_(p["jumps"]).sum(1) + p["jumps"].shape[1])
    first = [{k: o[k].clone() for k in ("u", "u_se", "grad", "grad_se")} for o in out]
    b.run()
    torch.cuda.synchronize()
    for o, f in zip(b.out, first):
        for k in f:
            assert torch.equal(o[k], f[k]), k
    b.close()


def test_autotuner_covers_both_walkers_and_results_do_not_depend_on_the_shape(tmp_path):
    """The autotuner times the CUDA-core walker's shapes and then the tensor-core walker's (CTAs
    per SM, walks per item) and caches the best; every launch shape gives the same outputs bit for
    bit (walks are a function of their indices, the per-query sums are formed in a fixed order)."""
    probs = []
    for i, (d, B) in enumerate([(3, 40), (4, 600), (7, 900), (10, 500)]):
        dom, X, _ = ball_problem(d, B, 6.0, 300 + i, 8)
        probs.append((W.Domain(dom), X))
    items = [{"domain": D, "x": X, "n_walks": 1024, "eps": 1e-3, "sigma": 6.0, "grad": True} for D, X in probs]
    b = W.Batch(items, seed=4, control_variate=True)
    b.run()
    torch.cuda.synchronize()
    ref = [{k: o[k].clone() for k in ("u", "u_se", "grad", "grad_se", "walk_steps")} for o in b.out]
    cache = tmp_path / "tune.txt"
    best = b.autotune(str(cache))
    lines = [l.split() for l in open(cache) if l.startswith("#")]
    assert len({(int(l[5]), int(l[6])) for l in lines}) >= 4  # sphere CTAs per SM x walks per item
    assert best["sphere_ctas_per_sm"] in (2, 3, 4) and best["sphere_item_walks"] in (2048, 4096, 8192)
    for cfg in (best, {"threads": 256, "ctas_per_sm": 2, "item_work": 1 << 22, "sphere_ctas_per_sm": 2,
                       "sphere_item_walks": 256}):
        b2 = W.Batch(items, seed=4, control_variate=True, config=cfg)
        b2.run()
        torch.cuda.synchronize()
        for o, r in zip(b2.out, ref):
            for k in r:
                assert torch.equal(o[k], r[k]), (cfg, k)
        b2.close()
    b.close()
