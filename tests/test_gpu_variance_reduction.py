"""Russian roulette on the walk weight and antithetic first directions (the closing discussion's
variance reductions, Sec. IX) in every GPU walker, through the C ABI, against the FP64 oracle.

Bars (as for the plain estimators):
  * FP64 walker, same Philox streams: per-walk terminal values, jumps and gradients within 1e-12
    on >= 99.9 % of walks; per-query outputs and standard errors to rounding; the counters
    (walk-steps, walks ended by the roulette) equal the oracle's exactly;
  * mixed (CUDA-core screen and tensor-core sphere set) and plain FP32 walkers: per query within
    4 sqrt(se_gpu^2 + se_oracle^2) + 1e-4, on the same walk indices; antithetic standard errors
    (from the pair means) within 10 % of the oracle's;
  * the exact solution u = exp(a.x) (|a|^2 = sigma) still holds.
"""
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


def agree(a, se_a, b, se_b, k=4.0, atol=1e-4):
    return np.abs(np.asarray(a) - np.asarray(b)) <= k * np.sqrt(np.asarray(se_a) ** 2 + np.asarray(se_b) ** 2) + atol


def roulette_domain(sigma=16.0, n_balls=2, d=3, seed=4):
    """Unit ball with ball obstacles and exp data (|a|^2 = sigma): at sigma = 16 a third of the
    walks' later steps carry weights below 0.3, so the roulette acts often. With many balls
    (1024) the mixed walker runs the domain on the tensor cores."""
    rng = np.random.default_rng(seed)
    a = rng.standard_normal(d)
    a *= math.sqrt(sigma) / np.linalg.norm(a)
    if n_balls == 2:
        c = np.array([[0.5, 0.0, 0.0], [-0.4, 0.3, 0.1]])[:, :d]
        r = np.array([0.2, 0.15])
    else:
        v = rng.standard_normal((n_balls, d))
        c = v / np.linalg.norm(v, axis=1, keepdims=True) * rng.uniform(0.0, 0.9, (n_balls, 1))
        r = np.exp(rng.uniform(math.log(0.005), math.log(0.05), n_balls))
    dom = {"d": d, "outer_c": np.zeros(d), "outer_r": 1.0, "ball_c": c, "ball_r": r,
           "exp_w": np.ones(1), "exp_a": a[None, :]}
    X = []
    while len(X) < 12:
        p = rng.uniform(-0.7, 0.7, size=d)
        if np.linalg.norm(p) < 0.7 and np.all(np.linalg.norm(c - p[None, :], axis=1) > r + 0.02):
            X.append(p)
    return dom, np.array(X), a, sigma


ROULETTE_W, EPS = 0.3, 1e-4


def test_roulette_fp64_per_walk_parity_and_counters():
    dom, X, a, sigma = roulette_domain()
    D = W.Domain(dom)
    N, seed = 4000, 3
    ref = oracle.solve(dom, X, N, EPS, sigma, seed, grad=True, roulette=ROULETTE_W, per_walk=True)
    got = D.walks(X, N, EPS, sigma, grad_mode=True, precision="fp64", seed=seed, roulette=ROULETTE_W)
    t_g, t_o = np_(got["term"]), ref["walk_term"]
    assert (np.abs(t_g - t_o) <= 1e-12 * np.maximum(1.0, np.abs(t_o))).mean() >= 0.999
    assert (np_(got["jumps"]) == ref["walk_jumps"]).mean() >= 0.999
    okg = np.all(np.abs(np_(got["grad"]) - ref["walk_grad"]) <= 1e-12 * np.maximum(1.0, np.abs(ref["walk_grad"])), axis=2)
    assert okg.mean() >= 0.999
    r = D.grad(X, N, EPS, sigma, precision="fp64", seed=seed, roulette=ROULETTE_W, with_stats=True)
    st = W.stats_dict(r["stats"])
    assert st["killed"] == int(ref["killed"].sum()) > 0
    assert st["walk_steps"] == int(ref["walk_steps"].sum())
    assert np.allclose(np_(r["u"]), ref["u"], rtol=1e-10, atol=1e-13)
    assert np.allclose(np_(r["grad"]), ref["grad"], rtol=1e-9, atol=1e-12)
    assert np.allclose(np_(r["du_dsigma"]), ref["du_dsigma"], rtol=1e-9, atol=1e-12)


@pytest.mark.parametrize("precision,n_balls,sigma", [("mixed", 2, 16.0), ("fp32", 2, 16.0), ("mixed", 1024, 64.0)])
def test_roulette_per_query_against_oracle(precision, n_balls, sigma):
    # (1024 small balls end walks early: sigma = 64 makes their weights small enough for the roulette)
    dom, X, a, sigma = roulette_domain(sigma=sigma, n_balls=n_balls)
    D = W.Domain(dom)
    assert D.info()["tensor_sphere_set"] == (n_balls >= 1024)
    N, seed = 8000, 5
    ref = oracle.solve(dom, X, N, EPS, sigma, seed, grad=True, roulette=ROULETTE_W)
    r = D.grad(X, N, EPS, sigma, precision=precision, seed=seed, roulette=ROULETTE_W, with_stats=True)
    plain = D.grad(X, N, EPS, sigma, precision=precision, seed=seed, with_stats=True)
    st, stp = W.stats_dict(r["stats"]), W.stats_dict(plain["stats"])
    assert st["killed"] > 0 and stp["killed"] == 0
    assert st["walk_steps"] < 0.97 * stp["walk_steps"]  # the roulette shortens the walks
    assert np.all(agree(np_(r["u"]), np_(r["u_se"]), ref["u"], ref["u_se"]))
    assert np.all(agree(np_(r["grad"]), np_(r["grad_se"]), ref["grad"], ref["grad_se"]))
    g = np.exp(X @ a)
    assert np.all(np.abs(np_(r["u"]) - g) <= 4.5 * np_(r["u_se"]) + 3e-4 * g * np.linalg.norm(a))


def test_antithetic_fp64_matches_oracle_with_pair_standard_errors():
    w = synth.c1(n_queries=16)
    D = W.Domain(w["domain"])
    N = 2000
    ref = oracle.solve(w["domain"], w["X"], N, w["eps"], w["sigma"], w["seed"], grad=True, antithetic=True,
                       per_walk=True)
    got = D.walks(w["X"], N, w["eps"], w["sigma"], grad_mode=True, precision="fp64", seed=w["seed"],
                  antithetic=True)
    assert (np.abs(np_(got["term"]) - ref["walk_term"]) <= 1e-12 * np.maximum(1.0, np.abs(ref["walk_term"]))).mean() >= 0.999
    okg = np.all(np.abs(np_(got["grad"]) - ref["walk_grad"]) <= 1e-12 * np.maximum(1.0, np.abs(ref["walk_grad"])), axis=2)
    assert okg.mean() >= 0.999
    r = D.grad(w["X"], N, w["eps"], w["sigma"], precision="fp64", seed=w["seed"], antithetic=True)
    for k in ("u", "u_se", "grad", "grad_se"):
        assert np.allclose(np_(r[k]), ref[k], rtol=1e-8, atol=1e-12), k


@pytest.mark.parametrize("precision,n_balls", [("mixed", 2), ("fp32", 2), ("mixed", 1024)])
def test_antithetic_per_query_against_oracle(precision, n_balls):
    dom, X, a, sigma = roulette_domain(sigma=4.0, n_balls=n_balls, seed=9)
    D = W.Domain(dom)
    N, seed = 8000, 7
    ref = oracle.solve(dom, X, N, EPS, sigma, seed, grad=True, antithetic=True)
    plain = oracle.solve(dom, X, N, EPS, sigma, seed, grad=True)
    r = D.grad(X, N, EPS, sigma, precision=precision, seed=seed, antithetic=True)
    assert np.all(agree(np_(r["u"]), np_(r["u_se"]), ref["u"], ref["u_se"]))
    assert np.all(agree(np_(r["grad"]), np_(r["grad_se"]), ref["grad"], ref["grad_se"]))
    # the same walks give the same pair spread: standard errors within 10 %
    assert np.allclose(np_(r["u_se"]), ref["u_se"], rtol=0.1)
    assert np.allclose(np_(r["grad_se"]), ref["grad_se"], rtol=0.1)
    assert np_(r["grad_se"]).mean() < 0.8 * plain["grad_se"].mean()


def test_batch_with_roulette_and_antithetic_pairs():
    """A batch of a CUDA-core problem and a tensor-core problem with both options, against the
    oracle on the same walk indices (the batch numbers the walks problem after problem)."""
    probs = [roulette_domain(n_balls=2, seed=21), roulette_domain(sigma=64.0, n_balls=1024, seed=22)]
    doms = [W.Domain(p[0]) for p in probs]
    Ns = [2000, 1000]
    b = W.Batch([{"domain": D, "x": p[1], "n_walks": n, "eps": EPS, "sigma": p[3], "grad": True}
                 for D, p, n in zip(doms, probs, Ns)], seed=11, roulette=ROULETTE_W, antithetic=True)
    out = b.run()
    torch.cuda.synchronize()
    base = 0
    for (dom, X, a, sigma), o, n in zip(probs, out, Ns):
        ref = oracle.solve(dom, X, n, EPS, sigma, 11, walk_offset=base, grad=True, roulette=ROULETTE_W,
                           antithetic=True)
        base += X.shape[0] * n
        assert np.all(agree(np_(o["u"]), np_(o["u_se"]), ref["u"], ref["u_se"]))
        assert np.all(agree(np_(o["grad"]), np_(o["grad_se"]), ref["grad"], ref["grad_se"]))
        assert np.array_equal(np_(o["walk_steps"]) > 0, np.ones(X.shape[0], bool))
    assert W.stats_dict(b.stats)["killed"] > 0
    b.close()


def test_option_checks():
    w = synth.c1(n_queries=2)
    D = W.Domain(w["domain"])
    for kw in ({"antithetic": True, "n": 101}, {"antithetic": True, "walk_offset": 1},
               {"antithetic": True, "control_variate": True}, {"roulette": -0.5}):
        n = kw.pop("n", 100)
        with pytest.raises(_lib.WoSError):
            D.grad(w["X"], n, w["eps"], w["sigma"], **kw)
