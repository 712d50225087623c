"""Impulse source (the paper's unit impulse at the goal) on the GPU walkers against the oracle.

Laplace(u) - sigma u = -q delta_z: each step whose ball contains z adds q G_B(x_k, z) times the
walk's weight; the first-sphere gradient adds q grad_x G_B(x_0, z).

  * FP64 mode, same Philox streams: per-walk values within 1e-12 (relative to max(1, |t|)) on
    >= 99.9 % of walks, identical jump counts, per-walk gradients within 1e-10;
  * mixed and plain FP32: per query within 4 sqrt(se_gpu^2 + se_oracle^2) + 1e-4 (value and
    gradient, also with the control variate);
  * the centred source in a ball: the closed form u = G_Omega(|x|);
  * du/dsigma (each walk's derivative, including the source contributions'): FP64 per walk
    within 1e-10, mixed and FP32 per query within 4 sqrt(2) standard errors of the oracle's
    per-walk spread plus 1e-4 relative, and the centred-source closed form;
  * batches and the planner (the paper's two-disc environment) use it.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle  # noqa: E402
from scipy import special  # noqa: E402
from paper_2406_01713_gb300 import synth  # noqa: E402
from paper_2406_01713_gb300 import wos as W  # noqa: E402


def np_(t):
    return t.detach().cpu().numpy()


def within(a, se_a, b, se_b, k=4.0, atol=1e-4):
    return np.abs(a - b) <= k * np.sqrt(se_a ** 2 + se_b ** 2) + atol


def source_domain(d, seed=3, n_balls=4):
    rng = np.random.default_rng(seed)
    c = rng.uniform(0.15, 0.85, size=(n_balls, d))
    r = rng.uniform(0.05, 0.1, size=n_balls)
    z = np.full(d, 0.5)
    z[0] = 0.75
    while np.any(np.linalg.norm(c - z, axis=1) < r + 0.05):
        z = rng.uniform(0.2, 0.8, d)
    dom = {"d": d, "box_lo": np.zeros(d), "box_hi": np.ones(d), "ball_c": c, "ball_r": r, "source_z": z,
           "source_q": 1.0}
    X = synth._free_points(rng, 8, np.zeros(d), np.ones(d), c, r, 0.02,
                           extra=lambda x: np.linalg.norm(x - z[None, :], axis=1) > 0.05)
    return dom, X


@pytest.mark.parametrize("d,sigma", [(2, 4.0), (3, 0.0)])
def test_fp64_per_walk_parity(d, sigma):
    dom, X = source_domain(d)
    D = W.Domain(dom)
    for grad_mode in (False, True):
        ref = oracle.solve(dom, X, 1000, 1e-3, sigma, 5, grad=grad_mode, per_walk=True)
        got = D.walks(X, 1000, 1e-3, sigma, grad_mode=grad_mode, precision="fp64", seed=5)
        t, to = np_(got["term"]), ref["walk_term"]
        ok = np.abs(t - to) <= 1e-12 * np.maximum(1.0, np.abs(to))
        assert ok.mean() >= 0.999, ok.mean()
        assert (np_(got["jumps"]) == ref["walk_jumps"]).mean() >= 0.999
        if grad_mode:
            g, go = np_(got["grad"]), ref["walk_grad"]
            okg = np.all(np.abs(g - go) <= 1e-10 * np.maximum(1.0, np.abs(go)), axis=-1)
            assert okg.mean() >= 0.999, okg.mean()
        ds, dso = np_(got["dsigma"]), ref["walk_dsigma"]
        okd = np.abs(ds - dso) <= 1e-10 * np.maximum(1.0, np.abs(dso))
        assert okd.mean() >= 0.999, okd.mean()


@pytest.mark.parametrize("precision", ["fp64", "mixed", "fp32"])
@pytest.mark.parametrize("cv", [False, True])
def test_per_query_matches_oracle(precision, cv):
    dom, X = source_domain(2, seed=8)
    sigma = 4.0
    ref = oracle.solve(dom, X, 8000, 1e-3, sigma, 11, grad=True, control_variate=cv, per_walk=True)
    D = W.Domain(dom)
    got = D.grad(X, 8000, 1e-3, sigma, precision=precision, seed=11, control_variate=cv)
    assert np.all(within(np_(got["u"]), np_(got["u_se"]), ref["u"], ref["u_se"]))
    assert np.all(within(np_(got["grad"]), np_(got["grad_se"]), ref["grad"], ref["grad_se"], atol=1e-4))
    assert_dsigma(np_(got["du_dsigma"]), ref, precision)


def assert_dsigma(got, ref, precision):
    """du/dsigma against the oracle on the same walks: FP64 to rounding; mixed and plain FP32
    within 4 sqrt(2) standard errors (from the oracle's per-walk values) + 1e-4 relative."""
    want = ref["du_dsigma"]
    assert np.all(np.isfinite(got))
    if precision == "fp64":
        assert np.allclose(got, want, rtol=1e-9, atol=1e-12)
        return
    wd = ref["walk_dsigma"]
    se = wd.std(axis=1, ddof=1) / math.sqrt(wd.shape[1])
    assert np.all(np.abs(got - want) <= 4 * math.sqrt(2) * se + 1e-4 * np.abs(want))


@pytest.mark.parametrize("d,sigma", [(2, 0.0), (3, 9.0)])
def test_centred_source_closed_form(d, sigma):
    R = 1.0
    dom = {"d": d, "outer_c": np.zeros(d), "outer_r": R, "source_z": np.zeros(d)}
    rng = np.random.default_rng(2)
    X = np.array([0.3 * v / np.linalg.norm(v) for v in rng.standard_normal((4, d))])
    got = W.Domain(dom).grad(X, 32768, 1e-5, sigma, seed=1, control_variate=True)
    nu, k = d / 2 - 1, math.sqrt(sigma)
    omega = 2 * math.pi ** (d / 2) / math.gamma(d / 2)
    for q, x in enumerate(X):
        r = np.linalg.norm(x)
        if sigma == 0.0:
            u = math.log(R / r) / (2 * math.pi) if d == 2 else (r ** (2 - d) - R ** (2 - d)) / ((d - 2) * omega)
            du = -r ** (1 - d) / omega
        else:
            c0 = k ** nu / (2 * math.pi) ** (d / 2)
            u = c0 * r ** -nu * (special.kv(nu, k * r) - special.kv(nu, k * R) * special.iv(nu, k * r) / special.iv(nu, k * R))
            du = -c0 * k * r ** -nu * (special.kv(nu + 1, k * r) + special.kv(nu, k * R) * special.iv(nu + 1, k * r)
                                        / special.iv(nu, k * R))
        assert abs(np_(got["u"])[q] - u) <= 4.5 * np_(got["u_se"])[q] + 1e-4 * abs(u)
        g = du * x / r
        assert np.all(np.abs(np_(got["grad"])[q] - g) <= 4.5 * np_(got["grad_se"])[q] + 2e-3 * np.abs(g).max())
    # du/dsigma = d/dsigma G_Omega(|x|): scipy's form by central differences (one-sided at
    # sigma = 0); the standard error from the same walks' per-walk derivatives
    per = np_(W.Domain(dom).walks(X, 32768, 1e-5, sigma, grad_mode=True, seed=1)["dsigma"])
    se = per.std(axis=1, ddof=1) / math.sqrt(per.shape[1])
    h = 1e-4
    for q, x in enumerate(X):
        r = np.linalg.norm(x)

        def G(s):
            if s == 0.0:
                return math.log(R / r) / (2 * math.pi) if d == 2 else (r ** (2 - d) - R ** (2 - d)) / ((d - 2) * omega)
            kk = math.sqrt(s)
            c0 = kk ** nu / (2 * math.pi) ** (d / 2)
            return c0 * r ** -nu * (special.kv(nu, kk * r) - special.kv(nu, kk * R) * special.iv(nu, kk * r)
                                    / special.iv(nu, kk * R))

        want = (-3 * G(0.0) + 4 * G(h) - G(2 * h)) / (2 * h) if sigma == 0.0 else (G(sigma + h) - G(sigma - h)) / (2 * h)
        assert abs(np_(got["du_dsigma"])[q] - want) <= 4.5 * se[q] + 1e-4 * abs(want)


def test_batch_with_a_source_problem():
    dom, X = source_domain(3, seed=4)
    w = synth.c4(n_problems=3, n_queries=6, scale_walks=0.2, max_balls=200)
    probs = [{"domain": W.Domain(dom), "x": X, "n_walks": 4000, "eps": 1e-3, "sigma": 1.0, "grad": True}]
    specs = [(dom, X, 4000, 1e-3, 1.0)]
    for p in w["problems"]:
        probs.append({"domain": W.Domain(p["domain"]), "x": p["X"], "n_walks": p["n_walks"], "eps": p["eps"],
                      "sigma": p["sigma"], "grad": True})
        specs.append((p["domain"], p["X"], p["n_walks"], p["eps"], p["sigma"]))
    B = W.Batch(probs, seed=21, control_variate=True)
    out = B.run()
    torch.cuda.synchronize()
    base = 0
    for (dm, Xq, N, eps, sigma), o in zip(specs, out):
        ref = oracle.solve(dm, Xq, N, eps, sigma, 21, walk_offset=base, grad=True, control_variate=True)
        base += Xq.shape[0] * N
        assert np.all(within(np_(o["u"]), np_(o["u_se"]), ref["u"], ref["u_se"]))
        assert np.all(within(np_(o["grad"]), np_(o["grad_se"]), ref["grad"], ref["grad_se"], atol=1e-4))
    B.close()


def paper_environment(k_r=0.3, goal=(6.0, 0.0)):
    """Outer disc r_o = 10 at the origin; discs r_u = k_r r_o at (0, r_u) and r_l = r_u/2 at
    (0, -r_l), touching at the origin; a unit impulse at the goal (Sec. VI)."""
    r_o = 10.0
    r_u = k_r * r_o
    r_l = 0.5 * r_u
    return {"d": 2, "outer_c": np.zeros(2), "outer_r": r_o, "ball_c": np.array([[0.0, r_u], [0.0, -r_l]]),
            "ball_r": np.array([r_u, r_l]), "source_z": np.array(goal), "source_q": 1.0}


def test_planner_fp64_steps_match_oracle():
    dom = paper_environment()
    x0 = np.array([3.0, 1.0])
    ref_path, ref_flags, ref_grads = oracle.plan_path(dom, x0, 3, 2048, 0.01, 0.1, 0.1, seed=9)
    path, flags, grads = W.Domain(dom).plan_path(x0, 3, 2048, 0.01, 0.1, 0.1, precision="fp64", seed=9)
    assert np.array_equal(np_(flags), ref_flags)
    assert np.allclose(np_(path)[: len(ref_path)], ref_path, rtol=0, atol=1e-9)
    scale = np.abs(ref_grads).max()
    assert np.allclose(np_(grads), ref_grads, rtol=0, atol=1e-9 * scale)


def test_planner_reaches_the_source_goal():
    dom = paper_environment()
    x0 = np.array([3.0, 1.0])
    path, flags, _ = W.Domain(dom).plan_path(x0, 200, 4096, 0.01, 0.1, 0.1, seed=3, control_variate=True)
    f = np_(flags)
    assert (f == 1).any(), "goal not reached"
    p = np_(path)
    # the path never enters an obstacle or leaves the outer disc
    assert np.all(np.linalg.norm(p, axis=1) < 10.0)
    for c, r in zip(dom["ball_c"], dom["ball_r"]):
        assert np.all(np.linalg.norm(p - c[None, :], axis=1) > r)


@pytest.mark.parametrize("kind", ["points", "balls"])
@pytest.mark.parametrize("cv", [False, True])
def test_tensor_core_walker_with_a_source(kind, cv):
    """The impulse source on the tensor-core sphere-set walker (mixed precision): a point set
    (Sec. VII-A) and a large ball set, against the oracle on the same walks; the per-walk records
    carry the source part of the gradient."""
    rng = np.random.default_rng(31)
    d = 3
    z = np.array([0.7, 0.5, 0.5])
    if kind == "points":
        t = rng.uniform(0, 2 * np.pi, 800)
        p = np.stack([0.3 + 0.15 * np.cos(t), 0.5 + 0.15 * np.sin(t), rng.uniform(0.1, 0.9, 800)], 1)
        dom = {"d": d, "box_lo": np.zeros(d), "box_hi": np.ones(d), "points": p, "source_z": z, "source_q": 1.0}
        X = np.array([[0.6, 0.3, 0.4], [0.5, 0.7, 0.6], [0.85, 0.5, 0.2], [0.3, 0.5, 0.5]])
    else:
        c = rng.uniform(0.0, 1.0, (600, d))
        r = np.exp(rng.uniform(np.log(0.004), np.log(0.02), 600))
        keep = np.linalg.norm(c - z[None, :], axis=1) > r + 0.05
        dom = {"d": d, "box_lo": np.zeros(d), "box_hi": np.ones(d), "ball_c": c[keep], "ball_r": r[keep],
               "source_z": z, "source_q": 1.0}
        X = synth._free_points(rng, 6, np.zeros(d), np.ones(d), c[keep], r[keep], 0.02,
                               extra=lambda x: np.linalg.norm(x - z[None, :], axis=1) > 0.1)
    D = W.Domain(dom)
    assert D.info()["tensor_sphere_set"]
    sigma, N = 4.0, 8000
    ref = oracle.solve(dom, X, N, 2e-3, sigma, 13, grad=True, control_variate=cv, per_walk=True)
    got = D.grad(X, N, 2e-3, sigma, seed=13, control_variate=cv)
    assert np.all(within(np_(got["u"]), np_(got["u_se"]), ref["u"], ref["u_se"]))
    assert np.all(within(np_(got["grad"]), np_(got["grad_se"]), ref["grad"], ref["grad_se"]))
    assert_dsigma(np_(got["du_dsigma"]), ref, "mixed")
    if not cv:
        per = D.walks(X[:2], 512, 2e-3, sigma, grad_mode=True, seed=13)
        ro = oracle.solve(dom, X[:2], 512, 2e-3, sigma, 13, grad=True, per_walk=True)
        # the per-walk gradients include the (deterministic) source part q grad_x G_B(x0, z)
        assert np.allclose(np_(per["grad"]).mean(1), ro["walk_grad"].mean(1),
                           atol=4 * ro["grad_se"].max() + 1e-4)


@pytest.mark.parametrize("precision", ["fp64", "mixed", "fp32"])
def test_source_with_roulette_and_antithetic_pairs(precision):
    """The impulse source together with the Russian roulette (a killed walk keeps its source
    contributions and their sigma derivatives) and antithetic first directions."""
    dom, X = source_domain(3, seed=12)
    sigma, N, eps, seed, w_min = 16.0, 4000, 1e-3, 17, 0.3
    D = W.Domain(dom)
    ref = oracle.solve(dom, X, N, eps, sigma, seed, grad=True, roulette=w_min, antithetic=True, per_walk=True)
    assert int(ref["killed"].sum()) > 0
    if precision == "fp64":
        got = D.walks(X, N, eps, sigma, grad_mode=True, precision="fp64", seed=seed, roulette=w_min, antithetic=True)
        for k, kr in (("term", "walk_term"), ("dsigma", "walk_dsigma")):
            a, b = np_(got[k]), ref[kr]
            assert (np.abs(a - b) <= 1e-10 * np.maximum(1.0, np.abs(b))).mean() >= 0.999, k
    r = D.grad(X, N, eps, sigma, precision=precision, seed=seed, roulette=w_min, antithetic=True, with_stats=True)
    assert W.stats_dict(r["stats"])["killed"] > 0
    assert np.all(within(np_(r["u"]), np_(r["u_se"]), ref["u"], ref["u_se"]))
    assert np.all(within(np_(r["grad"]), np_(r["grad_se"]), ref["grad"], ref["grad_se"]))
    assert_dsigma(np_(r["du_dsigma"]), ref, precision)
