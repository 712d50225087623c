"""Point-cloud obstacles (Sec. VII-A point-set distance) on the tensor-core walker.

* the distance bound the walker uses never exceeds the exact FP64 distance to the point set
  (BF16 contraction + FP32 refinement + error-bound shrink: no sphere leaves the domain) and
  stays close to it;
* walks through the tensor-core path agree with the FP64 oracle on the same random streams;
* the FP64 parity walker handles point sets walk by walk;
* the full-size workload (65536 points on 16 ellipsoid surfaces in 7D, 8192 queries x 4096
  walks) runs with exact counters and, with exponential boundary data, matches the exact
  solution u = exp(a.x) in aggregate.
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


def small_cloud(n_surfaces=4, per_surface=500, d=7, exp_data=True, sigma=25.0):
    rng = np.random.default_rng(77)
    pts = synth.ellipsoid_cloud(rng, d, n_surfaces, per_surface)  # 2000 points: a ragged last tile
    dom = {"d": d, "box_lo": -np.ones(d), "box_hi": np.ones(d), "points": pts}
    if exp_data:
        a = rng.standard_normal(d)
        a *= math.sqrt(sigma) / np.linalg.norm(a)
        dom["exp_w"] = np.array([math.exp(-2.0)])
        dom["exp_a"] = a[None, :]
    else:
        dom["goal_c"] = np.zeros(d)
        dom["goal_r"] = 0.05
    return dom, pts, rng


def exact_radius(dom, pts, X, block=256):
    dp = np.concatenate([np.sqrt(((X[i:i + block, None, :] - pts[None, :, :]) ** 2).sum(-1)).min(1)
                         for i in range(0, X.shape[0], block)])
    box = np.minimum(X - dom["box_lo"][None, :], dom["box_hi"][None, :] - X).min(1)
    r = np.minimum(dp, box)
    if dom.get("goal_r") is not None:
        r = np.minimum(r, np.linalg.norm(X - dom["goal_c"][None, :], axis=1) - dom["goal_r"])
    return r


def gpu_radius(dom_h, X):
    L = _lib.load()
    x = torch.tensor(X, dtype=torch.float64, device="cuda")
    out = torch.full((X.shape[0],), float("nan"), dtype=torch.float64, device="cuda")
    _lib.check(L.wos_debug_pointcloud_radius(dom_h.h, ctypes.c_void_p(x.data_ptr()), X.shape[0],
                                             ctypes.c_void_p(out.data_ptr()), None), "radius")
    torch.cuda.synchronize()
    return np_(out)


@pytest.mark.parametrize("n_surfaces,per_surface", [(4, 500), (16, 600)])
def test_radius_bound_is_safe_and_tight(n_surfaces, per_surface):
    """2000 points (32 tiles: 16-point chunks) and 9600 (150 tiles: 32-point chunks)."""
    dom, pts, rng = small_cloud(exp_data=False, n_surfaces=n_surfaces, per_surface=per_surface)
    D = W.Domain(dom)
    d = dom["d"]
    far = rng.uniform(-0.9, 0.9, size=(3000, d))
    idx = rng.integers(0, pts.shape[0], size=3000)
    off = rng.standard_normal((3000, d))
    off *= (10 ** rng.uniform(-3, -1.3, size=(3000, 1))) / np.linalg.norm(off, axis=1, keepdims=True)
    near = np.clip(pts[idx] + off, -0.99, 0.99)
    X = np.vstack([far, near])
    X = X[np.linalg.norm(X - dom["goal_c"][None, :], axis=1) > 0.06]
    want = exact_radius(dom, pts, X)
    got = gpu_radius(D, X)
    assert np.all(np.isfinite(got))
    # safety: never above the exact distance (FP32 rounding of the refinement aside)
    assert np.all(got <= want * (1 + 1e-5) + 2e-6), np.max(got - want)
    # tightness: the bound shrinks the radius only rarely and only a little
    rel = (want - got) / np.maximum(want, 1e-12)
    assert np.mean(rel < 1e-4) > 0.95, np.mean(rel < 1e-4)
    assert np.mean(rel < 0.5) > 0.999


def test_pointcloud_walks_match_oracle_and_closed_form():
    dom, pts, rng = small_cloud(exp_data=True)
    D = W.Domain(dom)
    X = rng.uniform(-0.8, 0.8, size=(16, dom["d"]))
    N, eps, sigma, seed = 2048, 1e-3, 25.0, 7
    ref = oracle.solve(dom, X, N, eps, sigma, seed, grad=True)
    got = D.grad(X, N, eps, sigma, precision="mixed", seed=seed, with_stats=True)
    u, se = np_(got["u"]), np_(got["u_se"])
    st = W.stats_dict(got["stats"])
    assert st["walks"] == 16 * N and st["outside"] == 0
    assert np.all(np.abs(u - ref["u"]) <= 4 * np.sqrt(se ** 2 + ref["u_se"] ** 2) + 1e-4)
    g, gse = np_(got["grad"]), np_(got["grad_se"])
    assert np.all(np.abs(g - ref["grad"]) <= 4 * np.sqrt(gse ** 2 + ref["grad_se"] ** 2) + 1e-4)
    # the exact solution (|a|^2 = sigma) on a domain bounded by the box and the point set
    a = dom["exp_a"][0]
    ex = dom["exp_w"][0] * np.exp(X @ a)
    assert np.mean(np.abs(u - ex) <= 5 * se + 3e-2 * ex) > 0.9


def test_pointcloud_fp64_walks_match_oracle_walk_by_walk():
    dom, pts, rng = small_cloud(exp_data=True, n_surfaces=2, per_surface=300)
    D = W.Domain(dom)
    X = rng.uniform(-0.8, 0.8, size=(4, dom["d"]))
    ref = oracle.solve(dom, X, 64, 1e-3, 25.0, 3, grad=True, per_walk=True)
    got = D.walks(X, 64, 1e-3, 25.0, grad_mode=True, precision="fp64", seed=3)
    t, to = np_(got["term"]), ref["walk_term"]
    assert np.mean(np.abs(t - to) <= 1e-12 * np.maximum(1, np.abs(to))) >= 0.999
    assert np.mean(np_(got["jumps"]) == ref["walk_jumps"]) >= 0.999


def test_full_size_pointcloud_exact_solution():
    """65536 points on 16 ellipsoid surfaces in [-1,1]^7, 8192 queries x 4096 walks through the
    tensor-core walker, with exponential data so that u = exp(a.x) holds exactly."""
    w = synth.c3()
    dom = dict(w["domain"])
    dom.pop("goal_c")
    dom.pop("goal_r")
    rng = np.random.default_rng(5)
    a = rng.standard_normal(7)
    a *= math.sqrt(w["sigma"]) / np.linalg.norm(a)
    dom["exp_w"] = np.array([math.exp(-2.0)])
    dom["exp_a"] = a[None, :]
    D = W.Domain(dom)
    r = D.solve(w["X"], w["n_walks"], w["eps"], w["sigma"], precision="mixed", seed=w["seed"], with_stats=True)
    st = W.stats_dict(r["stats"])
    assert st["walks"] == w["X"].shape[0] * w["n_walks"]
    assert st["outside"] == 0 and st["capped"] == 0
    u, se = np_(r["u"]), np_(r["u_se"])
    assert np.all(np.isfinite(u))
    ex = dom["exp_w"][0] * np.exp(w["X"] @ a)
    assert np.mean(np.abs(u - ex) <= 5 * se + 2e-2 * ex) > 0.98
    # and the goal-indicator workload itself: maximum principle, exact counters
    D2 = W.Domain(w["domain"])
    r2 = D2.solve(w["X"][:2048], w["n_walks"], w["eps"], w["sigma"], precision="mixed", seed=w["seed"],
                  with_stats=True)
    u2 = np_(r2["u"])
    assert np.all((u2 >= 0) & (u2 <= 1))
    assert W.stats_dict(r2["stats"])["walks"] == 2048 * w["n_walks"]
