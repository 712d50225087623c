"""Many planner paths in one batched graph (wos_plan_paths) against the same paths one at a time
(wos_plan_path): the multistart set of the paper's evaluation environment (Sec. VI, Fig. 5) and
paths in other domains and dimensions, including one on the tensor-core sphere-set walker. The
paths draw the same walks and form the same per-query sums in the same order, so points, flags
and gradients must be equal bit for bit."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2406_01713_gb300 import synth  # noqa: E402
from paper_2406_01713_gb300 import wos as W  # noqa: E402


def _ball_field(d, B, seed):
    """[-1,1]^d with B balls and a goal ball (g = 1 there): B = 400 runs on the tensor cores."""
    rng = np.random.default_rng(seed)
    c = rng.uniform(-1, 1, size=(B, d))
    r = np.exp(rng.uniform(math.log(0.01), math.log(0.06), size=B))
    lo, hi = -np.ones(d), np.ones(d)
    goal = synth._free_points(rng, 1, lo, hi, c, r, 0.2)[0]
    dom = {"d": d, "box_lo": lo, "box_hi": hi, "ball_c": c, "ball_r": r, "goal_c": goal, "goal_r": 0.1}
    start = synth._free_points(rng, 1, lo, hi, c, r, 0.05, extra=lambda x: np.linalg.norm(x - goal, axis=1) > 1.0)[0]
    return dom, start


@pytest.mark.parametrize("control_variate", [True, False])
def test_batched_paths_equal_single_paths(control_variate):
    env = W.Domain(synth.paper_environment(2, k_r=0.2))
    env3 = W.Domain(synth.paper_environment(3, k_r=0.3))
    dball, sball = _ball_field(3, 400, 5)
    ball = W.Domain(dball)
    assert ball.info()["tensor_sphere_set"]
    items = []
    for deg in (90, 135, 180, 225, 270, 315):
        x0 = 8.0 * np.array([math.cos(math.radians(deg)), math.sin(math.radians(deg))])
        items.append({"domain": env, "x0": x0, "n_walks": 1024, "eps": 0.01, "sigma": 1.0, "s_ub": 0.1})
    items.append({"domain": env3, "x0": np.array([-8.0, 0.0, 0.3]), "n_walks": 2048, "eps": 0.01, "sigma": 1.0,
                  "s_ub": 0.1})
    items.append({"domain": ball, "x0": sball, "n_walks": 512, "eps": 1e-3, "sigma": 4.0, "s_ub": 0.05})
    steps, seed = 120, 17
    got = W.plan_paths(items, steps, seed=seed, control_variate=control_variate)
    torch.cuda.synchronize()
    reached = 0
    for it, (path, flags, grads) in zip(items, got):
        p1, f1, g1 = it["domain"].plan_path(it["x0"], steps, it["n_walks"], it["eps"], it["sigma"], it["s_ub"],
                                            seed=seed, control_variate=control_variate)
        torch.cuda.synchronize()
        assert torch.equal(flags, f1)
        assert torch.equal(path, p1)
        assert torch.equal(grads, g1)
        reached += int((flags == 1).any())
        assert float(torch.linalg.norm(path[-1] - path[0])) > 0.05  # every path moves
    assert reached >= 2  # some paths reach the goal within the steps and stop (flag 8 after)


def test_paths_with_roulette_and_antithetic_pairs():
    env = W.Domain(synth.paper_environment(2, k_r=0.3))
    items = [{"domain": env, "x0": np.array([-8.0, 0.0]), "n_walks": 1024, "eps": 0.01, "sigma": 1.0, "s_ub": 0.1},
             {"domain": env, "x0": np.array([0.0, -8.0]), "n_walks": 2048, "eps": 0.01, "sigma": 1.0, "s_ub": 0.1}]
    got = W.plan_paths(items, 60, seed=3, roulette=0.05, antithetic=True)
    for it, (path, flags, grads) in zip(items, got):
        p1, f1, g1 = it["domain"].plan_path(it["x0"], 60, it["n_walks"], it["eps"], it["sigma"], it["s_ub"], seed=3,
                                            roulette=0.05, antithetic=True)
        assert torch.equal(path, p1) and torch.equal(flags, f1) and torch.equal(grads, g1)
