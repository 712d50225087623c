"""Control-variate gradient (WOS_FLAG_GRAD_CONTROL_VARIATE) on the GPU against the oracle.

grad^ = G/(N-1) sum_w (t_w - tbar) v_w, G = alpha(R0)/C(R0). The GPU forms it from one-pass
per-query sums (sum G t v, sum G v, sum G^2 t v^2, ...); the oracle by its two-pass definition.

  * FP64 mode, same walks: per-query estimates and SEs agree to rounding (the sums differ only
    in order) on >= 95 % of queries, and within 4 combined SE everywhere;
  * mixed and plain FP32: within 4 sqrt(se_gpu^2 + se_oracle^2) + 1e-4;
  * constant data at sigma = 0 (every walk returns 1): the estimate vanishes to rounding;
  * two-walk unbiasedness: the mean of 10^5 independent N = 2 estimates is the exact gradient;
  * exp data (u = g exactly): unbiased, and the SE is at most half the paper's estimator's;
  * the batched launch, the point-cloud walker and the planner use it too.
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


def ball_gradient(d, R, sigma, x):
    """grad u for Omega = B(0, R), g = 1: u = rho(|x|)/rho(R), rho(r) = r^-nu I_nu(sqrt(sigma) r)."""
    nu = d / 2 - 1
    k = math.sqrt(sigma)
    r = np.linalg.norm(x)
    rho = lambda t: t ** (-nu) * special.iv(nu, k * t)
    return k * r ** (-nu) * special.iv(nu + 1, k * r) / rho(R) * x / r


@pytest.fixture(scope="module")
def c1():
    w = synth.c1(n_queries=32)
    return w, W.Domain(w["domain"])


@pytest.fixture(scope="module")
def c1_oracle_cv(c1):
    w, _ = c1
    return oracle.solve(w["domain"], w["X"], 4000, w["eps"], w["sigma"], w["seed"], grad=True,
                        control_variate=True)


def test_fp64_matches_oracle_to_rounding(c1, c1_oracle_cv):
    w, dom = c1
    ref = c1_oracle_cv
    got = dom.grad(w["X"], 4000, w["eps"], w["sigma"], precision="fp64", seed=w["seed"], control_variate=True)
    g, se = np_(got["grad"]), np_(got["grad_se"])
    # u is unchanged by the option; the gradient sums differ from the two-pass oracle only in
    # summation order (relative 1e-9 of the per-walk scale leaves room for that, not for a
    # different estimator: the control-variate SE is ~1e-2 of that scale here)
    scale = np.sqrt(4000) * ref["grad_se"]
    tight = np.all(np.abs(g - ref["grad"]) <= 1e-9 * scale + 1e-13, axis=1)
    assert tight.mean() >= 0.95, tight.mean()
    se_ok = np.abs(se - ref["grad_se"]) <= 1e-6 * ref["grad_se"] + 1e-13
    assert np.all(se_ok[tight])
    assert np.all(within(g, se, ref["grad"], ref["grad_se"]))
    assert np.allclose(np_(got["u"]), ref["u"], rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("precision", ["mixed", "fp32"])
def test_single_precision_matches_oracle(c1, c1_oracle_cv, precision):
    w, dom = c1
    ref = c1_oracle_cv
    got = dom.grad(w["X"], 4000, w["eps"], w["sigma"], precision=precision, seed=w["seed"], control_variate=True)
    assert np.all(within(np_(got["grad"]), np_(got["grad_se"]), ref["grad"], ref["grad_se"]))


@pytest.mark.parametrize("n_walks", [4096, 3 * 4096 + 100])
@pytest.mark.parametrize("precision", ["fp64", "mixed", "fp32"])
def test_constant_data_gives_zero(precision, n_walks):
    # with g = 1 every walk has t = 1, so the estimate cancels to rounding only if the sum of
    # first directions matches the walkers' own; above 4096 walks a query's mixed-precision
    # prepass is split across warps (three full segments and a ragged one here)
    d = 3
    dom = W.Domain(synth.ball_domain(d, 1.0))
    X = np.array([[0.3, -0.2, 0.1], [0.0, 0.6, 0.0]])
    cv = dom.grad(X, n_walks, 1e-4, 0.0, precision=precision, seed=5, control_variate=True)
    plain = dom.grad(X, n_walks, 1e-4, 0.0, precision=precision, seed=5)
    G = d / (1.0 - np.linalg.norm(X, axis=1, keepdims=True))
    tol = 1e-10 if precision == "fp64" else 1e-5
    assert np.all(np.abs(np_(cv["grad"])) <= tol * G)
    assert np.all(np.abs(np_(plain["grad"])).max(axis=1) > 1e-3)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_two_walk_estimates_are_unbiased(precision):
    d, R, sigma = 2, 1.0, 4.0
    dom = W.Domain(synth.ball_domain(d, R))
    x = np.array([0.3, 0.4])
    Q = 100000
    got = dom.grad(np.tile(x, (Q, 1)), 2, 1e-5, sigma, precision=precision, seed=23, control_variate=True)
    g = np_(got["grad"])
    mean, se = g.mean(axis=0), g.std(axis=0, ddof=1) / math.sqrt(Q)
    exact = ball_gradient(d, R, sigma, x)
    assert np.all(np.abs(mean - exact) < 4.0 * se), (mean, exact, se)
    assert np.all(np.abs(0.5 * mean - exact) > 4.0 * se)  # a 1/N slip would be seen


def test_exp_data_exact_and_lower_variance():
    w = synth.c1(n_queries=32)
    dom = W.Domain(w["domain"])
    cv = dom.grad(w["X"], 16384, 1e-4, w["sigma"], seed=3, control_variate=True)
    plain = dom.grad(w["X"], 16384, 1e-4, w["sigma"], seed=3)
    a = w["domain"]["exp_a"][0]
    g = np.exp(w["X"] @ a)
    bias = 3e-4 * g * np.linalg.norm(a)
    gg = a[None, :] * g[:, None]
    assert np.all(np.abs(np_(cv["grad"]) - gg) < 4.5 * np_(cv["grad_se"]) + 10 * bias[:, None])
    assert np.mean(np_(cv["grad_se"])) < 0.5 * np.mean(np_(plain["grad_se"]))


def test_batch_matches_oracle():
    wl = synth.c4(n_problems=6, n_queries=8, scale_walks=0.25, max_balls=256)
    probs = []
    for p in wl["problems"]:
        probs.append({"domain": W.Domain(p["domain"]), "x": p["X"], "n_walks": p["n_walks"], "eps": p["eps"],
                      "sigma": p["sigma"], "grad": True})
    B = W.Batch(probs, seed=wl["seed"], control_variate=True)
    out = B.run()
    torch.cuda.synchronize()
    base = 0
    for p, o in zip(wl["problems"], out):
        ref = oracle.solve(p["domain"], p["X"], p["n_walks"], p["eps"], p["sigma"], wl["seed"], walk_offset=base,
                           grad=True, control_variate=True)
        base += p["X"].shape[0] * p["n_walks"]
        assert np.all(within(np_(o["u"]), np_(o["u_se"]), ref["u"], ref["u_se"]))
        assert np.all(within(np_(o["grad"]), np_(o["grad_se"]), ref["grad"], ref["grad_se"], atol=1e-4))


def test_pointcloud_matches_oracle():
    rng = np.random.default_rng(77)
    d, sigma = 7, 25.0
    pts = synth.ellipsoid_cloud(rng, d, 2, 400)
    a = rng.standard_normal(d)
    a *= math.sqrt(sigma) / np.linalg.norm(a)
    dom = {"d": d, "box_lo": -np.ones(d), "box_hi": np.ones(d), "points": pts,
           "exp_w": np.array([math.exp(-2.0)]), "exp_a": a[None, :]}
    D = W.Domain(dom)
    X = rng.uniform(-0.8, 0.8, size=(12, d))
    ref = oracle.solve(dom, X, 2048, 1e-3, sigma, 7, grad=True, control_variate=True)
    got = D.grad(X, 2048, 1e-3, sigma, seed=7, control_variate=True)
    assert np.all(within(np_(got["grad"]), np_(got["grad_se"]), ref["grad"], ref["grad_se"], atol=1e-4))


def test_planner_step_uses_it():
    dom_h = synth.annulus_domain(2, 0.2, 2.0)  # goal = inner sphere
    dom = W.Domain(dom_h)
    x0 = np.array([1.2, 0.3])
    x = torch.tensor(x0, dtype=torch.float64, device="cuda")
    flag, g = dom.plan_step(x, 2048, 1e-4, 1.0, 0.1, 0, precision="fp64", seed=8, control_variate=True)
    ref = oracle.solve(dom_h, x0[None, :], 2048, 1e-4, 1.0, 8, grad=True, control_variate=True)
    scale = np.sqrt(2048) * ref["grad_se"][0]
    assert int(np_(flag)[0]) == 0
    assert np.all(np.abs(np_(g) - ref["grad"][0]) <= 1e-9 * scale + 1e-13)
    # the step moved x by min(s_ub, R/2) along the estimated direction
    step = np_(x) - x0
    assert abs(np.linalg.norm(step) - 0.1) < 1e-12
    assert np.allclose(step / 0.1, ref["grad"][0] / np.linalg.norm(ref["grad"][0]), atol=1e-8)
