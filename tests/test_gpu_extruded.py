"""Extruded domains on the GPU (Sec. VI dimensionality study): the paper's two-disc environment
measured in its first two coordinates, free and unbounded in the others.

Bars:
  * FP64, same Philox streams as the oracle: per-walk terminals within 1e-12 (relative to
    max(1, |u|)) on >= 99.9 % of walks, identical jump counts on matched walks;
  * mixed and plain FP32: per query within 4 sqrt(se_gpu^2 + se_oracle^2) + 1e-4 of the oracle,
    and the exp closed form (exp(a.x) with |a|^2 = sigma solves the PDE in all of R^d);
  * the gradient angle error e = arccos(g^.g / (|g^| |g|)) against a many-walk reference falls
    like N^-1/2 (Fig. 10), in d = 2 and in the extruded d = 4 environment with the unit impulse,
    at (2, -6), a point with a direct line to the goal (behind the obstacle, at (-8, 0), the
    gradient is ~1e-10 and rare walks dominate its estimate).
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle  # noqa: E402
from paper_2406_01713_gb300 import synth  # noqa: E402
from paper_2406_01713_gb300 import wos as W  # noqa: E402


def np_(t):
    return t.detach().cpu().numpy()


def within(a, se_a, b, se_b, k=4.0, atol=1e-4):
    return np.abs(np.asarray(a) - b) <= k * np.sqrt(np.asarray(se_a) ** 2 + np.asarray(se_b) ** 2) + atol


@pytest.fixture(scope="module", autouse=True)
def built():
    W._lib.load()
    oracle.build()


def unit_env(d, sigma, seed):
    """The two-disc environment at unit scale, extruded, with g = exp(a.x), |a|^2 = sigma, a
    along every coordinate; queries in the free cross-section, free coordinates in [-2, 2]."""
    rng = np.random.default_rng(seed)
    dom = synth.paper_environment(d, goal=(0.8, 0.0), r_o=1.0)
    del dom["source_z"], dom["source_q"]
    a = rng.standard_normal(d)
    a *= math.sqrt(sigma) / np.linalg.norm(a)
    dom["exp_w"], dom["exp_a"] = np.ones(1), a[None, :]
    X = []
    while len(X) < 8:
        p = rng.uniform(-0.9, 0.9, size=2)
        if np.linalg.norm(p) > 0.9 or any(np.linalg.norm(p - c[:2]) < 1.1 * r
                                          for c, r in zip(dom["ball_c"], dom["ball_r"])):
            continue
        X.append(np.concatenate([p, rng.uniform(-2, 2, size=d - 2)]))
    return dom, np.array(X), a


@pytest.mark.parametrize("d,grad_mode", [(3, False), (3, True), (5, True)])
def test_fp64_per_walk_parity(d, grad_mode):
    dom, X, _ = unit_env(d, 1.0, 20 + d)
    N, eps, sigma, seed = 1024, 1e-3, 1.0, 7
    ref = oracle.solve(dom, X, N, eps, sigma, seed, grad=grad_mode, per_walk=True)
    got = W.Domain(dom).walks(X, N, eps, sigma, grad_mode=grad_mode, precision="fp64", seed=seed)
    t_g, t_o = np_(got["term"]), ref["walk_term"]
    assert (np.abs(t_g - t_o) <= 1e-12 * np.maximum(1.0, np.abs(t_o))).mean() >= 0.999
    assert (np_(got["jumps"]) == ref["walk_jumps"]).mean() >= 0.999
    if grad_mode:
        g_g, g_o = np_(got["grad"]), ref["walk_grad"]
        assert np.all(np.abs(g_g - g_o) <= 1e-12 * np.maximum(1.0, np.abs(g_o)), axis=2).mean() >= 0.999


@pytest.mark.parametrize("precision", ["mixed", "fp32"])
@pytest.mark.parametrize("d", [3, 4])
def test_per_query_and_exact_solution(d, precision):
    dom, X, a = unit_env(d, 1.0, 30 + d)
    N, eps, sigma, seed = 8192, 1e-3, 1.0, 11
    ref = oracle.solve(dom, X, N, eps, sigma, seed, grad=True)
    got = W.Domain(dom).grad(X, N, eps, sigma, precision=precision, seed=seed, with_stats=True)
    st = W.stats_dict(got["stats"])
    assert st["walks"] == X.shape[0] * N and st["outside"] == 0 and st["capped"] == 0
    u, se, g, gse = np_(got["u"]), np_(got["u_se"]), np_(got["grad"]), np_(got["grad_se"])
    assert np.all(within(u, se, ref["u"], ref["u_se"]))
    assert np.all(within(g, gse, ref["grad"], ref["grad_se"], atol=1e-4))
    ex = np.exp(X @ a)
    assert np.all(np.abs(u - ex) <= 4.5 * se + 3e-3 * ex)


def angle_deg(g, ref):
    c = np.sum(g * ref, axis=-1) / (np.linalg.norm(g, axis=-1) * np.linalg.norm(ref))
    return np.degrees(np.arccos(np.clip(c, -1.0, 1.0)))


@pytest.mark.parametrize("d", [2, 4])
def test_angle_error_falls_like_inverse_sqrt_n(d):
    # the paper's dimensionality study: unit impulse at the goal, c = 1, eps = 0.01, the point
    # (2, -6, 0, ...); the reference gradient from 2^24 walks
    dom = W.Domain(synth.paper_environment(d))
    x = np.zeros((1, d))
    x[0, :2] = (2.0, -6.0)
    eps, sigma = 0.01, 1.0
    ref = np_(dom.grad(x, 1 << 24, eps, sigma, seed=1, control_variate=True)["grad"])[0]
    assert np.linalg.norm(ref) > 0
    errs = {}
    for n in (1 << 12, 1 << 16):
        g = np.stack([np_(dom.grad(x, n, eps, sigma, seed=100 + s, control_variate=True)["grad"])[0]
                      for s in range(24)])
        errs[n] = angle_deg(g, ref).mean()
    # 16x the walks: the error shrinks about 4x (at least 2.5x), and is small at 2^16 walks
    assert errs[1 << 12] / errs[1 << 16] > 2.5, errs
    assert errs[1 << 16] < 10.0, errs
