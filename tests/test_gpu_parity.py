"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle and closed forms.

Bars:
  * FP64 mode, same Philox streams: per-walk terminals within 1e-12 (relative to max(1, |u|))
    on >= 99.9 % of walks, identical jump counts on matched walks;
  * mixed (FP32 walkers, FP64 sums) and plain FP32: per query within
    4 sqrt(se_gpu^2 + se_oracle^2) + 1e-4;
  * integer counters (walks, walk-steps, capped, outside) bit-exact.
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
from paper_2406_01713_gb300 import _lib  # noqa: E402


def np_(t):
    return t.detach().cpu().numpy()


def agree(a, se_a, b, se_b, k=4.0, atol=1e-4):
    a, b = np.asarray(a), np.asarray(b)
    return np.abs(a - b) <= k * np.sqrt(np.asarray(se_a) ** 2 + np.asarray(se_b) ** 2) + atol


@pytest.fixture(scope="module", autouse=True)
def built():
    W._lib.load()
    oracle.build()


# --------------------------------------------------------------------------- RNG contract
def test_philox_bitwise_against_oracle():
    import ctypes

    L = _lib.load()
    n = 1 << 16
    walk0 = (1 << 32) - n // 2  # crosses the high word of the walk index
    for step, block in [(0, 0), (7, 1), (123456, 2)]:
        out = torch.empty(n * 4, dtype=torch.int32, device="cuda")
        _lib.check(L.wos_debug_philox(2406, walk0, n, step, block, ctypes.c_void_p(out.data_ptr()), None),
                   "philox")
        got = np_(out).view(np.uint32).reshape(n, 4)
        for i in list(range(0, n, 97)) + [n // 2 - 1, n // 2, n - 1]:
            w = walk0 + i
            want = oracle.philox4x32_10([2406, 0], [w & 0xFFFFFFFF, w >> 32, step, block])
            assert list(got[i]) == want, (i, step, block)


# --------------------------------------------------------------------------- c1, FP64
@pytest.fixture(scope="module")
def c1():
    w = synth.c1()
    dom = W.Domain(w["domain"])
    return w, dom


@pytest.mark.parametrize("grad_mode", [False, True])
def test_c1_fp64_per_walk_parity(c1, grad_mode):
    w, dom = c1
    N = w["n_walks"]
    ref = oracle.solve(w["domain"], w["X"], N, w["eps"], w["sigma"], w["seed"], grad=grad_mode,
                       per_walk=True)
    got = dom.walks(w["X"], N, w["eps"], w["sigma"], grad_mode=grad_mode, precision="fp64", seed=w["seed"])
    t_g, t_o = np_(got["term"]), ref["walk_term"]
    ok = np.abs(t_g - t_o) <= 1e-12 * np.maximum(1.0, np.abs(t_o))
    assert ok.mean() >= 0.999, ok.mean()
    same_jumps = np_(got["jumps"]) == ref["walk_jumps"]
    assert same_jumps.mean() >= 0.999
    if grad_mode:
        g_g, g_o = np_(got["grad"]), ref["walk_grad"]
        okg = np.all(np.abs(g_g - g_o) <= 1e-12 * np.maximum(1.0, np.abs(g_o)), axis=2)
        assert okg.mean() >= 0.999
    d_g, d_o = np_(got["dsigma"]), ref["walk_dsigma"]
    okd = np.abs(d_g - d_o) <= 1e-12 * np.maximum(1.0, np.abs(d_o))
    assert okd.mean() >= 0.999


@pytest.fixture(scope="module")
def c1_oracle(c1):
    w, _ = c1
    return oracle.solve(w["domain"], w["X"], w["n_walks"], w["eps"], w["sigma"], w["seed"], grad=True)


@pytest.mark.parametrize("precision", ["fp64", "mixed", "fp32"])
def test_c1_per_query(c1, c1_oracle, precision):
    w, dom = c1
    ref = c1_oracle
    got = dom.grad(w["X"], w["n_walks"], w["eps"], w["sigma"], precision=precision, seed=w["seed"],
                   with_stats=True)
    u, se = np_(got["u"]), np_(got["u_se"])
    g, gse = np_(got["grad"]), np_(got["grad_se"])
    st = W.stats_dict(got["stats"])
    assert st["walks"] == w["X"].shape[0] * w["n_walks"]
    assert st["outside"] == 0 and st["capped"] == 0
    if precision == "fp64":
        assert np.allclose(u, ref["u"], rtol=1e-10, atol=1e-12)
        assert np.allclose(g, ref["grad"], rtol=1e-9, atol=1e-10)
        assert np.allclose(np_(got["du_dsigma"]), ref["du_dsigma"], rtol=1e-9, atol=1e-12)
        assert st["walk_steps"] == int(ref["walk_steps"].sum())
    assert np.all(agree(u, se, ref["u"], ref["u_se"]))
    assert np.all(agree(g, gse, ref["grad"], ref["grad_se"]))
    # one term with w = 1: du/dw per walk equals the walk's value, so u's standard errors are its own
    assert np.all(agree(np_(got["du_dw"])[:, 0], se, ref["du_dw"][:, 0], ref["u_se"]))
    # the exact solution (|a|^2 = sigma): u = exp(a.x), grad u = a u; O(eps) shell bias allowed
    a = w["domain"]["exp_a"][0]
    gx = np.exp(w["X"] @ a)
    assert np.all(np.abs(u - gx) <= 4.5 * se + 3e-3 * gx)


def test_counters_match_per_walk_jumps(c1):
    w, dom = c1
    X = w["X"][:9]
    N = 777  # ragged: not a multiple of a warp or an item
    for precision in ["mixed", "fp32", "fp64"]:
        per = dom.walks(X, N, w["eps"], w["sigma"], precision=precision, seed=5)
        got = dom.solve(X, N, w["eps"], w["sigma"], precision=precision, seed=5, with_stats=True)
        st = W.stats_dict(got["stats"])
        assert st["walks"] == 9 * N
        assert st["walk_steps"] == int(np_(per["jumps"]).sum()) + 9 * N
        assert np.allclose(np_(got["u"]), np_(per["term"]).mean(axis=1), rtol=1e-6, atol=1e-9)


# --------------------------------------------------------------------------- normaliser
def test_weight_table_against_oracle():
    import ctypes

    L = _lib.load()
    for d in [2, 3, 7, 12]:
        n = 2049
        zmax = 30.0
        lc = np.zeros(n)
        ra = np.zeros(n)
        P = ctypes.POINTER(ctypes.c_double)
        _lib.check(L.wos_debug_weight_table(d, zmax, n, lc.ctypes.data_as(P), ra.ctypes.data_as(P)), "table")
        nu = d / 2 - 1
        for i in range(0, n, 16):
            z = zmax * i / (n - 1)
            want = oracle.log_C(nu, z)
            assert abs(lc[i] - want) <= 2e-7 * max(1.0, abs(want))
            want_r = oracle.series_S(nu + 1, z) / oracle.series_S(nu, z)
            assert abs(ra[i] - want_r) <= 2e-7 * want_r


@pytest.mark.parametrize("d", [2, 3, 5, 8, 12])
def test_ball_centre_deterministic(d):
    R, sigma = 1.3, 9.0
    dom = W.Domain(synth.ball_domain(d, R))
    x = np.zeros((1, d))
    want = math.exp(oracle.log_C(d / 2 - 1, R * math.sqrt(sigma)))
    for precision, tol in [("fp64", 1e-13), ("mixed", 2e-5), ("fp32", 2e-5)]:
        r = dom.walks(x, 256, 1e-6, sigma, grad_mode=True, precision=precision, seed=1)
        assert np.all(np_(r["jumps"]) == 1)
        assert np.max(np.abs(np_(r["term"]) - want)) <= tol * want
        alpha = (d / R) * math.exp(oracle.log_C(d / 2, R * math.sqrt(sigma)))
        gn = np.linalg.norm(np_(r["grad"])[0], axis=1)
        assert np.max(np.abs(gn - alpha)) <= max(tol, 1e-12) * alpha * 10


# --------------------------------------------------------------------------- edge cases
def test_edge_cases(c1):
    w, dom = c1
    # empty query set
    r = dom.solve(np.zeros((0, 2)), 10, 1e-3, 4.0, with_stats=True)
    assert r["u"].numel() == 0 and int(r["stats"][0]) == 0
    # one walk: standard error is 0
    r = dom.solve(w["X"][:3], 1, 1e-3, 4.0, precision="mixed")
    assert np.all(np_(r["u_se"]) == 0)
    # a query inside an obstacle: NaN and counted as outside, the others unaffected
    X = np.vstack([w["X"][:2], w["domain"]["ball_c"][:1]])
    for precision in ["fp64", "mixed", "fp32"]:
        r = dom.solve(X, 100, 1e-3, 4.0, precision=precision, with_stats=True)
        u = np_(r["u"])
        assert np.isnan(u[2]) and np.all(np.isfinite(u[:2]))
        assert int(r["stats"][3]) == 100
    # step cap: capped walks contribute 0 and are counted exactly (FP64 equals the oracle)
    ref = oracle.solve(w["domain"], w["X"][:4], 300, 1e-9, 4.0, 7, max_steps=3)
    got = dom.solve(w["X"][:4], 300, 1e-9, 4.0, precision="fp64", seed=7, max_steps=3, with_stats=True)
    assert int(got["stats"][2]) == int(ref["capped"].sum()) > 0
    # invalid arguments are rejected before launching
    with pytest.raises(_lib.WoSError):
        dom.solve(w["X"][:2], 0, 1e-3, 4.0)
    with pytest.raises(_lib.WoSError):
        dom.solve(w["X"][:2], 10, -1.0, 4.0)


# --------------------------------------------------------------------------- planner
@pytest.fixture(scope="module")
def c2():
    w = synth.c2()
    return w, W.Domain(w["domain"])


def test_planner_fp64_matches_oracle(c2):
    """FP64 planner, step by step: at every GPU path point the oracle (same walks, same point)
    gives the same grad u and the step follows s = min(s_ub, d/2) along grad/|grad|. Whole
    paths are compared loosely: last-bit differences of the summed gradient (atomics versus
    the oracle's ordered sums) are amplified by the walk dynamics (the jump map can double a
    perturbation per jump), so paths drift apart at the 1e-7 level without any step being wrong."""
    w, dom = c2
    steps = 60
    path, flags, grads = dom.plan_path(w["start"], steps, w["n_walks"], w["eps"], w["sigma"], w["s_ub"],
                                       precision="fp64", seed=w["seed"])
    path, flags, grads = np_(path), np_(flags), np_(grads)
    last = int(np.argmax(flags == 1)) if (flags == 1).any() else steps
    good = 0
    for i in range(last):
        ref = oracle.solve(w["domain"], path[i][None, :], w["n_walks"], w["eps"], w["sigma"], w["seed"],
                           walk_offset=i * w["n_walks"], grad=True)
        g = ref["grad"][0]
        good += bool(np.allclose(grads[i], g, rtol=1e-9, atol=1e-15))
        if flags[i] == 0:
            R = oracle.distance(w["domain"], path[i])[0]
            s = min(w["s_ub"], 0.5 * R)
            gn = np.linalg.norm(grads[i])
            assert np.allclose(path[i + 1], path[i] + s * (grads[i] / gn), rtol=0, atol=1e-13)
        elif flags[i] == 2:
            assert np.all(grads[i] == 0) and np.array_equal(path[i + 1], path[i])
    assert good >= 0.98 * last, (good, last)
    pref, fref, _ = oracle.plan_path(w["domain"], w["start"], steps, w["n_walks"], w["eps"], w["sigma"],
                                     w["s_ub"], w["seed"])
    n = min(len(pref), last + 1)
    assert np.max(np.abs(path[:n] - pref[:n])) < 1e-4


def test_planner_mixed_teacher_forced(c2):
    w, dom = c2
    steps = w["n_steps"]
    path, flags, grads = dom.plan_path(w["start"], steps, w["n_walks"], w["eps"], w["sigma"], w["s_ub"],
                                       precision="mixed", seed=w["seed"])
    path, flags, grads = np_(path), np_(flags), np_(grads)
    assert 1 in flags, "the 200-step path must reach the goal"
    last = int(np.argmax(flags == 1))
    g = w["domain"]["goal_c"]
    assert np.linalg.norm(path[last] - g) - 0.1 < w["eps"]
    # every step stays in the domain and moves by s = min(s_ub, d/2)
    for i in range(last):
        R = oracle.distance(w["domain"], path[i])[0]
        assert R > 0
        if flags[i] == 0:
            s = min(w["s_ub"], 0.5 * R)
            assert abs(np.linalg.norm(path[i + 1] - path[i]) - s) < 1e-9
    # teacher forcing: at GPU path points the oracle, with the same walks, gives the same grad u
    for i in range(0, last, 7):
        ref = oracle.solve(w["domain"], path[i][None, :], w["n_walks"], w["eps"], w["sigma"], w["seed"],
                           walk_offset=i * w["n_walks"], grad=True)
        assert np.all(agree(grads[i], 0 * grads[i], ref["grad"][0], ref["grad_se"][0], atol=1e-6))


def test_plan_step_matches_path(c2):
    w, dom = c2
    x = torch.tensor(w["start"], dtype=torch.float64, device="cuda")
    path, flags, _ = dom.plan_path(w["start"], 5, w["n_walks"], w["eps"], w["sigma"], w["s_ub"],
                                   precision="fp64", seed=w["seed"])
    for i in range(5):
        f, _ = dom.plan_step(x, w["n_walks"], w["eps"], w["sigma"], w["s_ub"], i, precision="fp64",
                             seed=w["seed"])
        assert int(f[0]) == int(flags[i])
        assert torch.allclose(x, path[i + 1], rtol=0, atol=1e-14)


# --------------------------------------------------------------------------- autograd
def test_autograd_c5_small():
    w = synth.c5(n_queries=48, n_walks=2048)
    dom = W.Domain(w["domain"])
    X = torch.tensor(w["X"], dtype=torch.float64, device="cuda", requires_grad=True)
    wt = torch.tensor(w["domain"]["exp_w"], dtype=torch.float64, device="cuda", requires_grad=True)
    sig = torch.tensor(w["sigma"], dtype=torch.float64, requires_grad=True)
    for precision, rtol in [("fp64", 1e-9), ("mixed", 2e-4)]:
        X.grad = wt.grad = sig.grad = None
        u = W.WoSFunction.apply(X, sig, wt, dom, w["n_walks"], w["eps"], w["seed"], precision)
        gout = torch.linspace(0.5, 1.5, u.numel(), dtype=torch.float64, device="cuda")
        (u * gout).sum().backward()
        ref = oracle.solve(w["domain"], w["X"], w["n_walks"], w["eps"], w["sigma"], w["seed"], grad=True)
        go = np_(gout)
        # d/dx = gout * grad u (the oracle's FP64 gradient estimate from the same walks)
        gx = np_(X.grad)
        if precision == "fp64":
            assert np.allclose(gx, go[:, None] * ref["grad"], rtol=1e-9, atol=1e-12)
        else:
            assert np.all(agree(gx, 0, go[:, None] * ref["grad"], go[:, None] * ref["grad_se"], atol=1e-4))
        # d/dsigma against common-random-number central differences (same walks, h = 1e-3)
        h = w["fd_h"]
        up = dom.solve(w["X"], w["n_walks"], w["eps"], w["sigma"] + h, precision=precision, seed=w["seed"])
        um = dom.solve(w["X"], w["n_walks"], w["eps"], w["sigma"] - h, precision=precision, seed=w["seed"])
        # value walks and gradient walks coincide here (no query starts in the eps shell)
        fd_s = float(((np_(up["u"]) - np_(um["u"])) / (2 * h) * go).sum())
        assert abs(float(sig.grad) - fd_s) <= rtol * abs(fd_s) + 1e-6 * abs(fd_s)
        # d/dw: u is linear in w, so central differences are exact up to rounding
        for k in [0, 3, 7]:
            wp = w["domain"]["exp_w"].copy()
            wm = wp.copy()
            wp[k] += h
            wm[k] -= h
            dom.set_exp_w(wp)
            a = np_(dom.solve(w["X"], w["n_walks"], w["eps"], w["sigma"], precision=precision, seed=w["seed"])["u"])
            dom.set_exp_w(wm)
            b = np_(dom.solve(w["X"], w["n_walks"], w["eps"], w["sigma"], precision=precision, seed=w["seed"])["u"])
            dom.set_exp_w(w["domain"]["exp_w"])
            fd_w = float(((a - b) / (2 * h) * go).sum())
            assert abs(float(wt.grad[k]) - fd_w) <= max(rtol, 1e-6) * abs(fd_w) + 1e-9
        # and the FP64 oracle's du/dw
        assert abs(float(wt.grad[0]) - float((ref["du_dw"][:, 0] * go).sum())) <= (
            1e-9 if precision == "fp64" else 5e-3) * abs(float(wt.grad[0]))


# --------------------------------------------------------------------------- batched
def _batch(problems, seed, grad=True):
    """A batch with the benchmark's launch configuration (cached autotuner choice if any)."""
    doms = [W.Domain(p["domain"]) for p in problems]
    b = W.Batch([{"domain": d, "x": p["X"], "n_walks": p["n_walks"], "eps": p["eps"], "sigma": p["sigma"],
                  "grad": grad} for d, p in zip(doms, problems)], seed=seed)
    return doms, b


def test_batch_subsample_matches_oracle():
    w = synth.c4(n_problems=24, n_queries=5, scale_walks=1 / 16)
    probs = w["problems"]
    doms, b = _batch(probs, w["seed"])
    out = b.run()
    torch.cuda.synchronize()
    st = W.stats_dict(b.stats)
    assert st["walks"] == sum(p["X"].shape[0] * p["n_walks"] for p in probs)
    base = 0
    for p, o in zip(probs, out):
        ref = oracle.solve(p["domain"], p["X"], p["n_walks"], p["eps"], p["sigma"], w["seed"],
                           walk_offset=base, grad=True)
        base += p["X"].shape[0] * p["n_walks"]
        assert np.all(agree(np_(o["u"]), np_(o["u_se"]), ref["u"], ref["u_se"]))
        assert np.all(agree(np_(o["grad"]), np_(o["grad_se"]), ref["grad"], ref["grad_se"], atol=1e-4))


@pytest.fixture(scope="module")
def c4_full():
    w = synth.c4()  # about 10 s of input generation
    doms, b = _batch(w["problems"], w["seed"], grad=True)
    out = b.run()
    torch.cuda.synchronize()
    return w, doms, b, out


def test_batch_full_size_counters_and_properties(c4_full):
    """The full 256-problem batch in the launch configuration the benchmark times: exact
    counters, the maximum principle on indicator problems, and the exact solution
    u = exp(a.x) on exponential-data problems in aggregate (their terminal values are
    heavy-tailed, so a per-query SE test is not a valid bar)."""
    w, doms, b, out = c4_full
    probs = w["problems"]
    st = W.stats_dict(b.stats)
    assert st["walks"] == sum(p["X"].shape[0] * p["n_walks"] for p in probs)
    assert st["outside"] == 0
    assert st["walk_steps"] == sum(int(np_(o["walk_steps"]).sum()) for o in out)
    oks = []
    for i, (p, o) in enumerate(zip(probs, out)):
        u, se = np_(o["u"]), np_(o["u_se"])
        if i % 2 == 1:
            assert np.all((u >= 0) & (u <= 1))
        else:
            g = np.exp(p["X"] @ p["domain"]["exp_a"][0])
            oks.append(np.abs(u - g) <= 5 * se + 2e-2 * g)
    assert np.concatenate(oks).mean() > 0.98


def test_batch_full_size_sampled_oracle_parity(c4_full):
    """Sampled outputs of the full batch recomputed one by one by the oracle on the same walk
    indices: one query from each of 40 problems (seeded choice, cost-capped)."""
    w, doms, b, out = c4_full
    probs = w["problems"]
    bases = np.cumsum([0] + [p["X"].shape[0] * p["n_walks"] for p in probs])
    rng = np.random.default_rng(11)
    picked = 0
    for i in rng.permutation(len(probs)):
        p = probs[i]
        cost = p["n_walks"] * (p["domain"]["ball_r"].size + 8) * p["domain"]["d"]
        if cost > 4e7:
            continue
        q = int(rng.integers(p["X"].shape[0]))
        ref = oracle.solve(p["domain"], p["X"][q:q + 1], p["n_walks"], p["eps"], p["sigma"], w["seed"],
                           walk_offset=int(bases[i]) + q * p["n_walks"], grad=True)
        o = out[i]
        assert agree(np_(o["u"])[q], np_(o["u_se"])[q], ref["u"][0], ref["u_se"][0]), (i, q)
        assert np.all(agree(np_(o["grad"])[q], np_(o["grad_se"])[q], ref["grad"][0], ref["grad_se"][0])), (i, q)
        picked += 1
        if picked == 40:
            break
    assert picked == 40


def test_c5_full_size_closed_form():
    w = synth.c5()
    dom = W.Domain(w["domain"])
    r = dom.grad(w["X"], w["n_walks"], w["eps"], w["sigma"], precision="mixed", seed=w["seed"], with_stats=True)
    st = W.stats_dict(r["stats"])
    assert st["walks"] == w["X"].shape[0] * w["n_walks"]
    E = np.exp(w["X"] @ w["domain"]["exp_a"].T)  # Q x K
    g = E @ w["domain"]["exp_w"]
    u, se = np_(r["u"]), np_(r["u_se"])
    assert (np.abs(u - g) <= 4.5 * se + 5e-3 * g).mean() > 0.995
    dw = np_(r["du_dw"])
    assert (np.abs(dw - E) <= 0.05 * E + 1e-3).mean() > 0.99


def test_batch_full_size_tensor_core_queries_match_oracle(c4_full):
    """The problems the tensor-core sphere-set walker runs in the full batch (most of the
    headline's device time): one query from a problem of every dimension 3..12, plus the
    problems with the largest ball set and the most walks, against the oracle on the same walk
    indices, u and every component of grad u at 4 combined SE + 1e-4."""
    w, doms, b, out = c4_full
    probs = w["problems"]
    bases = np.cumsum([0] + [p["X"].shape[0] * p["n_walks"] for p in probs])
    tens = [i for i, d in enumerate(doms) if d.info()["tensor_sphere_set"]]
    rng = np.random.default_rng(23)
    pick = []
    for d in range(3, 13):
        of_d = [i for i in tens if probs[i]["domain"]["d"] == d]
        assert of_d, d
        pick.append(int(rng.choice(of_d)))
    pick.append(max(tens, key=lambda i: probs[i]["domain"]["ball_r"].size * probs[i]["domain"]["d"]))
    pick.append(max(tens, key=lambda i: probs[i]["n_walks"] * probs[i]["domain"]["ball_r"].size))
    for i in dict.fromkeys(pick):
        p, o = probs[i], out[i]
        q = int(rng.integers(p["X"].shape[0]))
        ref = oracle.solve(p["domain"], p["X"][q:q + 1], p["n_walks"], p["eps"], p["sigma"], w["seed"],
                           walk_offset=int(bases[i]) + q * p["n_walks"], grad=True)
        assert agree(np_(o["u"])[q], np_(o["u_se"])[q], ref["u"][0], ref["u_se"][0]), (i, q)
        assert np.all(agree(np_(o["grad"])[q], np_(o["grad_se"])[q], ref["grad"][0], ref["grad_se"][0])), (i, q)
        assert int(np_(o["walk_steps"])[q]) > 0
