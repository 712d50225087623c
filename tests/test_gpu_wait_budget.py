"""Failure detection in the tensor-core sphere-set walker: every wait on its shared-memory
barriers is bounded, and a wait that runs out of its budget ends the launch cleanly.

A budget of one clock cycle (wos_options.wait_cycles) makes a healthy launch give up at its
first wait that is not already complete. The tests check that such a call ends, that its
outputs are NaN and wos_stats.timeouts is set (asynchronous calls), that the synchronous planner
calls return WOS_ERR_TIMEOUT, and that the next call on the same device runs normally and gives
the same outputs as before, bit for bit. No test faults, traps or hangs the GPU: the give-up path
is the kernel's own bounded wait, and its teardown waits (with the full budget) for the products
and copies already issued before it frees the tensor memory.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2406_01713_gb300 import _lib, synth  # noqa: E402
from paper_2406_01713_gb300 import wos as W  # noqa: E402

WOS_ERR_TIMEOUT = 5


def ball_field(d=4, B=512, seed=3):
    """[-1,1]^d with B balls (the tensor-core walker) and exp data |a|^2 = 4."""
    rng = np.random.default_rng(seed)
    c = rng.uniform(-1, 1, size=(B, d))
    r = np.exp(rng.uniform(math.log(0.01), math.log(0.06), size=B))
    a = rng.standard_normal(d)
    a *= 2.0 / np.linalg.norm(a)
    dom = {"d": d, "box_lo": -np.ones(d), "box_hi": np.ones(d), "ball_c": c, "ball_r": r,
           "exp_w": np.ones(1), "exp_a": a[None, :]}
    X = synth._free_points(rng, 16, -np.ones(d), np.ones(d), c, r, 0.02)
    return dom, X


def test_budget_runs_out_then_next_call_is_clean():
    dom, X = ball_field()
    D = W.Domain(dom)
    assert D.info()["tensor_sphere_set"]
    ref = D.grad(X, 2048, 1e-3, 4.0, seed=5, with_stats=True)
    torch.cuda.synchronize()
    assert np.all(np.isfinite(ref["u"].cpu().numpy()))
    assert W.stats_dict(ref["stats"])["timeouts"] == 0
    bad = D.grad(X, 2048, 1e-3, 4.0, seed=5, with_stats=True, wait_cycles=1)
    torch.cuda.synchronize()
    st = W.stats_dict(bad["stats"])
    assert st["timeouts"] != 0
    for k in ("u", "u_se", "grad", "grad_se", "du_dw"):
        assert torch.isnan(bad[k]).all(), k
    again = D.grad(X, 2048, 1e-3, 4.0, seed=5, with_stats=True)
    torch.cuda.synchronize()
    assert W.stats_dict(again["stats"])["timeouts"] == 0
    for k in ("u", "u_se", "grad", "grad_se", "du_dw"):
        assert torch.equal(again[k], ref[k]), k


def test_batch_budget_runs_out_then_clean():
    dom, X = ball_field(d=5, B=640, seed=8)
    dom2, X2 = ball_field(d=3, B=16, seed=9)  # CUDA-core walker beside it
    D, D2 = W.Domain(dom), W.Domain(dom2)
    probs = [{"domain": D, "x": X, "n_walks": 1024, "eps": 1e-3, "sigma": 4.0, "grad": True},
             {"domain": D2, "x": X2, "n_walks": 1024, "eps": 1e-3, "sigma": 4.0, "grad": True}]
    b = W.Batch(probs, seed=2, wait_cycles=1)
    out = b.run()
    torch.cuda.synchronize()
    assert W.stats_dict(b.stats)["timeouts"] != 0
    assert all(torch.isnan(o["u"]).all() for o in out)
    b.close()
    b = W.Batch(probs, seed=2)
    out = b.run()
    torch.cuda.synchronize()
    assert W.stats_dict(b.stats)["timeouts"] == 0
    assert all(torch.isfinite(o["u"]).all() and torch.isfinite(o["grad"]).all() for o in out)
    b.close()


def test_planner_calls_return_timeout():
    dom, X = ball_field(d=3, B=400, seed=11)
    dom = {k: v for k, v in dom.items() if k not in ("exp_w", "exp_a")}
    dom["goal_c"] = X[0]
    dom["goal_r"] = 0.05
    D = W.Domain(dom)
    assert D.info()["tensor_sphere_set"]
    with pytest.raises(_lib.WoSError) as e:
        D.plan_path(X[1], 20, 512, 1e-3, 4.0, 0.05, seed=1, wait_cycles=1)
    assert e.value.status == WOS_ERR_TIMEOUT
    items = [{"domain": D, "x0": X[2], "n_walks": 512, "eps": 1e-3, "sigma": 4.0, "s_ub": 0.05}]
    with pytest.raises(_lib.WoSError) as e:
        W.plan_paths(items, 20, seed=1, wait_cycles=1)
    assert e.value.status == WOS_ERR_TIMEOUT
    # the same calls with the default budget run to the end; the single path equals the batched one
    p1, f1, g1 = D.plan_path(X[2], 20, 512, 1e-3, 4.0, 0.05, seed=1)
    (p2, f2, g2), = W.plan_paths(items, 20, seed=1)
    torch.cuda.synchronize()
    assert not (f1 == 16).any()
    assert torch.equal(p1, p2) and torch.equal(f1, f2) and torch.equal(g1, g2)
