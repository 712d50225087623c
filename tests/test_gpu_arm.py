"""Planar arm in configuration space (Sec. V-A: the safe-ball radius d_tau/K) and the RR
validation environment (Sec. VII, Table I) on the GPU walkers, through the C ABI, against the
FP64 oracle.

Bars: FP64 per-walk terminal values, jumps and gradients within 1e-12 on >= 99.9 % of walks;
mixed and plain FP32 per query within 4 sqrt(se_gpu^2 + se_oracle^2) + 1e-4; the exact solution
u = exp(a.q) (|a|^2 = sigma) on the RR space; FP64 planner steps equal to the oracle's at the GPU
path's points."""
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


def agree(a, se_a, b, se_b, k=4.0, atol=1e-4):
    return np.abs(np.asarray(a) - np.asarray(b)) <= k * np.sqrt(np.asarray(se_a) ** 2 + np.asarray(se_b) ** 2) + atol


def rr_exp_domain(sigma=4.0):
    """The RR configuration space (Lipschitz arm) with exp data |a|^2 = sigma instead of the source."""
    w = synth.rr_arm(0.0)
    dom = {k: v for k, v in w["domain"].items() if k not in ("source_z", "source_q")}
    a = np.array([1.2, -1.6]) * np.sqrt(sigma) / 2.0
    dom.update({"exp_w": np.ones(1), "exp_a": a[None, :]})
    X = np.array([w["start"], w["goal"], [1.2, 1.0], [2.6, -0.5], [0.3, 2.5], [3.9, 0.4]])
    return dom, X, a


def test_arm_fp64_per_walk_parity():
    for sigma in (0.0, 5.0):
        w = synth.rr_arm(sigma)
        X = np.array([w["start"], [1.2, 1.0], [3.0, -1.0]])
        D = W.Domain(w["domain"])
        ref = oracle.solve(w["domain"], X, 3000, w["eps"], sigma, 9, grad=True, per_walk=True)
        got = D.walks(X, 3000, w["eps"], sigma, grad_mode=True, precision="fp64", seed=9)
        t_g, t_o = np_(got["term"]), ref["walk_term"]
        assert (np.abs(t_g - t_o) <= 1e-12 * np.maximum(1.0, np.abs(t_o))).mean() >= 0.999
        assert (np_(got["jumps"]) == ref["walk_jumps"]).mean() >= 0.999
        okg = np.all(np.abs(np_(got["grad"]) - ref["walk_grad"]) <= 1e-12 * np.maximum(1.0, np.abs(ref["walk_grad"])),
                     axis=2)
        assert okg.mean() >= 0.999


@pytest.mark.parametrize("precision", ["mixed", "fp32"])
def test_arm_per_query_and_exact_solution(precision):
    dom, X, a = rr_exp_domain()
    D = W.Domain(dom)
    N, eps, sigma, seed = 20000, 1e-3, 4.0, 3
    ref = oracle.solve(dom, X, N, eps, sigma, seed, grad=True)
    r = D.grad(X, N, eps, sigma, precision=precision, seed=seed, with_stats=True)
    assert np.all(agree(np_(r["u"]), np_(r["u_se"]), ref["u"], ref["u_se"]))
    assert np.all(agree(np_(r["grad"]), np_(r["grad_se"]), ref["grad"], ref["grad_se"]))
    g = np.exp(X @ a)
    assert np.all(np.abs(np_(r["u"]) - g) <= 4.5 * np_(r["u_se"]) + 3 * eps * np.linalg.norm(a) * g)
    assert W.stats_dict(r["stats"])["walks"] == X.shape[0] * N


def test_rr_source_per_query_mixed():
    w = synth.rr_arm(5.0)
    D = W.Domain(w["domain"])
    X = np.array([w["start"], [1.2, 1.0], [3.0, -1.0], [1.8, 0.6]])
    ref = oracle.solve(w["domain"], X, 20000, w["eps"], 5.0, 4, grad=True)
    r = D.grad(X, 20000, w["eps"], 5.0, seed=4)
    assert np.all(agree(np_(r["u"]), np_(r["u_se"]), ref["u"], ref["u_se"]))
    assert np.all(agree(np_(r["grad"]), np_(r["grad_se"]), ref["grad"], ref["grad_se"]))


@pytest.mark.parametrize("method,precision", [("lipschitz", "fp64"), ("ik", "fp64"), ("lipschitz", "mixed")])
def test_rr_planner_paths(method, precision):
    """The RR validation (Sec. VII): paths from q_start toward the unit impulse at q_goal; the FP64
    steps equal the oracle's at the GPU path's points (same walks); every path reaches the goal."""
    w = synth.rr_arm(0.0, method=method)
    D = W.Domain(w["domain"])
    N, steps = 4096, 200
    path, flags, grads = D.plan_path(w["start"], steps, N, w["eps"], w["sigma"], w["s_ub"], precision=precision,
                                     seed=w["seed"])
    path, flags, grads = np_(path), np_(flags), np_(grads)
    assert 1 in flags, "the path reaches the goal"
    last = int(np.argmax(flags == 1))
    assert np.linalg.norm(path[last] - w["goal"]) < w["s_ub"]
    for i in range(last):
        R = oracle.distance(w["domain"], path[i])[0]
        assert R > 0  # the path stays in the free configuration space
    if precision == "fp64":
        for i in range(0, last, 9):
            ref = oracle.solve(w["domain"], path[i][None, :], N, w["eps"], w["sigma"], w["seed"], walk_offset=i * N,
                               grad=True)
            assert np.allclose(grads[i], ref["grad"][0], rtol=1e-8, atol=1e-12)


def test_arm_argument_checks():
    w = synth.rr_arm(0.0)
    bad = dict(w["domain"])
    bad["link_l"] = np.array([1.0, -1.0])
    with pytest.raises(_lib.WoSError):
        W.Domain(bad)
    many = dict(w["domain"])
    many["arm_obs"] = np.random.default_rng(0).uniform(-2, 2, (40, 2))
    D = W.Domain(many)  # FP64 and FP32 take any number of obstacle points
    D.solve(np.array([w["start"]]), 64, w["eps"], 0.0, precision="fp64")
    with pytest.raises(_lib.WoSError):
        D.solve(np.array([w["start"]]), 64, w["eps"], 0.0)  # mixed: at most 32
