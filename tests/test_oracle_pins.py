"""Pins for the FP64 CPU oracle: checks against what the paper and the mathematics fix,
never against the oracle itself.

  * Philox4x32-10 known-answer vectors (Salmon et al., SC'11)           -> RNG contract
  * Box-Muller normals / sphere directions: moments, KS test              -> sphere sampling
  * log C_nu against scipy's exponentially scaled Bessel I and the odd-d
    closed forms (d = 3: z / sinh z; d = 5: z^3 / (3 (z cosh z - sinh z)))  -> normaliser C
  * ball centre (P1): one jump, u^ = C_nu(R sqrt(sigma)) exactly, |grad^| = (d/R) C_{nu+1}
  * ball off-centre (P2): u = rho(r)/rho(R), grad u radial (scipy), within 4.5 SE
  * exp boundary data with |a|^2 = sigma (P3): u = g, grad u = a g, du/dw = exp(a.x)
  * annulus with g = 1 on the inner sphere: closed forms with I_nu, K_nu (sigma > 0) and
    log / power laws (sigma = 0)
  * derivative in sigma: closed form at the ball centre, common-random-number FD (P8)
  * derivative in w: linear, FD exact (P9); max principle (P6); SE ~ N^-1/2 (P7)
  * planner: adaptive step s = min(s_ub, d/2) and radial descent in the annulus
  * extruded domains (Sec. VI dimensionality study): nearest-point geometry against sampled
    cylinder surfaces, and the exp closed form with a along all or only the free coordinates
  * Russian roulette on the weight: the exp closed form with shorter walks, du/dsigma against
    the plain estimator, and a planted mistake (survivors not reweighted) that must fail
  * antithetic first directions: paired walks' first directions are exact negatives, the exp
    closed form with a lower gradient SE, and the pair-based SE against the spread of repeated
    estimates (a per-walk SE would be ~3.7x too large)
  * point sets (Sec. VII-A): the distance, component and closest point against numpy
    enumeration (plain and extruded, with every other component kind present), exact ties
    between a point and the components before and after it in the tie order, and the exp closed
    form on a box-plus-points domain (extruded: with a along the free coordinate)
  * sigma = 0 with harmonic polynomial data on a ball (P4): u = g, grad u = grad g
  * the unit square with g = 1 on the top edge (P5): u and grad u against the
    separation-of-variables series, itself checked against a Richardson-extrapolated 5-point
    finite-difference solve on 65^2 and 129^2 grids
and one planted mistake (the paper's literal d/R gradient factor at sigma > 0), which the
off-centre ball pin must reject.
"""
import math
import os

import numpy as np
import pytest
from scipy import special, stats

from paper_2406_01713_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def log_C_scipy(nu, z):
    """log[(z/2)^nu / (Gamma(nu+1) I_nu(z))] from scipy's ive (I_nu(z) = ive(nu, z) e^z)."""
    z = np.asarray(z, float)
    return nu * np.log(z / 2.0) - special.gammaln(nu + 1.0) - (np.log(special.ive(nu, z)) + z)


# --------------------------------------------------------------------------- RNG
def test_philox_known_answers(oracle_mod):
    n = 0
    for line in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        v = [int(t, 16) for t in line.split()]
        assert oracle_mod.philox4x32_10(v[4:6], v[0:4]) == v[6:10]
        n += 1
    assert n == 3


def test_normals_are_standard_gaussian(oracle_mod):
    d = 4
    samples = np.array([oracle_mod.normals(2406, w, 3, d) for w in range(20000)]).ravel()
    assert abs(samples.mean()) < 5 / math.sqrt(samples.size)
    assert abs(samples.var() - 1.0) < 5 * math.sqrt(2.0 / samples.size)
    assert stats.kstest(samples, "norm").pvalue > 1e-3


@pytest.mark.parametrize("d", [2, 3, 7])
def test_directions_uniform_on_sphere(oracle_mod, d):
    n = 20000
    v = np.array([oracle_mod.direction(7, w, 0, d) for w in range(n)])
    assert np.allclose(np.linalg.norm(v, axis=1), 1.0, atol=1e-14)
    assert np.all(np.abs(v.mean(axis=0)) < 5 / math.sqrt(n))
    cov = v.T @ v / n
    assert np.all(np.abs(cov - np.eye(d) / d) < 6 * math.sqrt(2.0 / n) / d + 1e-3)


def test_counter_layout_distinguishes_walk_step_block(oracle_mod):
    base = oracle_mod.normals(1, 5, 2, 8)
    assert not np.allclose(base, oracle_mod.normals(1, 6, 2, 8))
    assert not np.allclose(base, oracle_mod.normals(1, 5, 3, 8))
    assert not np.allclose(base, oracle_mod.normals(2, 5, 2, 8))
    # walk index high word is part of the counter
    assert not np.allclose(oracle_mod.normals(1, 5, 2, 4), oracle_mod.normals(1, 5 + (1 << 32), 2, 4))
    # blocks: normals 4..7 come from block 1, not a repeat of block 0
    assert not np.allclose(base[:4], base[4:])


# --------------------------------------------------------------------------- normaliser
@pytest.mark.parametrize("nu", [0.0, 0.5, 1.0, 1.5, 2.0, 2.5, 3.5, 5.0, 6.0])
def test_log_C_matches_scipy(oracle_mod, nu):
    for z in np.concatenate([np.logspace(-4, 1.9, 60), [0.0]]):
        got = oracle_mod.log_C(nu, z)
        if z == 0.0:
            assert got == 0.0
            continue
        want = log_C_scipy(nu, z)
        assert abs(got - want) <= 1e-13 * max(1.0, abs(want)), (nu, z, got, want)


def test_log_C_odd_dimension_closed_forms(oracle_mod):
    for z in [1e-3, 0.1, 0.7, 1.0, 3.3, 9.0, 25.0]:
        # d = 3 (nu = 1/2): C = z / sinh z
        assert abs(oracle_mod.log_C(0.5, z) - math.log(z / math.sinh(z))) < 1e-13 * max(1, z)
        # d = 5 (nu = 3/2): C = z^3 / (3 (z cosh z - sinh z)); series for tiny z avoids cancellation
        if z > 0.05:
            c5 = z ** 3 / (3.0 * (z * math.cosh(z) - math.sinh(z)))
            assert abs(oracle_mod.log_C(1.5, z) - math.log(c5)) < 1e-12 * max(1, z)


def test_dsigma_log_C(oracle_mod):
    for nu in [0.0, 0.5, 2.0, 4.0]:
        d = 2 * nu + 2
        for R, sigma in [(0.3, 4.0), (1.0, 25.0), (0.05, 0.5), (2.0, 10.0)]:
            z = R * math.sqrt(sigma)
            # d/dsigma log C = -(R / (2 sqrt(sigma))) I_{nu+1}(z) / I_nu(z)
            want = -(R / (2 * math.sqrt(sigma))) * special.ive(nu + 1, z) / special.ive(nu, z)
            got = oracle_mod.dsigma_log_C(nu, R, sigma)
            assert abs(got - want) < 1e-12 * abs(want)
        # sigma -> 0 limit: -R^2 / (2d)
        assert abs(oracle_mod.dsigma_log_C(nu, 0.7, 0.0) + 0.49 / (2 * d)) < 1e-15


# --------------------------------------------------------------------------- distance
def test_distance_invariants(oracle_mod):
    w = synth.c1()
    dom = w["domain"]
    rng = np.random.default_rng(0)
    for x in rng.uniform(0, 1, size=(200, 2)):
        R, kind, idx, xbar = oracle_mod.distance(dom, x)
        if R <= 0:
            continue  # not in the open domain (inside a disc)
        # closest point is at distance |R| and lies on the boundary
        assert abs(np.linalg.norm(x - xbar) - abs(R)) < 1e-12
        R2, _, _, _ = oracle_mod.distance(dom, xbar)
        assert abs(R2) < 1e-12
        # no boundary point of any component is closer: sample each component densely
        for c, r in zip(dom["ball_c"], dom["ball_r"]):
            t = np.linspace(0, 2 * math.pi, 721)
            ring = c[None, :] + r * np.stack([np.cos(t), np.sin(t)], 1)
            assert np.min(np.linalg.norm(ring - x[None, :], axis=1)) >= R - 1e-12
        for j in range(2):
            assert x[j] - 0.0 >= R - 1e-15 and 1.0 - x[j] >= R - 1e-15


# --------------------------------------------------------------------------- P1, P2
@pytest.mark.parametrize("d", [2, 3, 4, 7, 12, 14])
def test_ball_centre_is_deterministic(oracle_mod, d):
    R, sigma = 1.3, 9.0
    dom = synth.ball_domain(d, R)
    res = oracle_mod.solve(dom, np.zeros((1, d)), 64, 1e-6, sigma, seed=11, grad=True, per_walk=True)
    nu = d / 2 - 1
    z = R * math.sqrt(sigma)
    C = math.exp(log_C_scipy(nu, z))
    assert np.all(res["walk_jumps"] == 1)
    assert np.max(np.abs(res["walk_term"] - C)) < 1e-13 * C
    # |grad^| per walk = (d/R) C_{nu+1}(z): pins the first-sphere factor alpha
    gn = np.linalg.norm(res["walk_grad"][0], axis=1)
    alpha = (d / R) * math.exp(log_C_scipy(nu + 1, z))
    assert np.max(np.abs(gn - alpha)) < 1e-12 * alpha
    # d/dsigma of C at the centre, against a central difference of the scipy closed form
    h = 1e-5
    dC = (math.exp(log_C_scipy(nu, R * math.sqrt(sigma + h))) -
          math.exp(log_C_scipy(nu, R * math.sqrt(sigma - h)))) / (2 * h)
    assert np.max(np.abs(res["walk_dsigma"] - dC)) < 1e-7 * abs(dC)


def ball_solution(d, R, sigma, x):
    """u = rho(|x|)/rho(R), rho(r) = r^-nu I_nu(k r); grad u = k r^-nu I_{nu+1}(k r)/rho(R) x/r."""
    if sigma == 0.0:
        return 1.0, np.zeros(d)  # g = 1 is harmonic: u = 1
    nu = d / 2 - 1
    k = math.sqrt(sigma)
    r = np.linalg.norm(x)
    rho = lambda s: s ** (-nu) * special.iv(nu, k * s)
    u = rho(r) / rho(R)
    du = k * r ** (-nu) * special.iv(nu + 1, k * r) / rho(R)
    return u, du * x / r


def _ball_case(oracle_mod, d, sigma, laplace_factor=False, n=40000):
    R = 1.0
    dom = synth.ball_domain(d, R)
    rng = np.random.default_rng(d)
    X = []
    for rad in [0.25, 0.5, 0.7]:
        v = rng.standard_normal(d)
        X.append(rad * v / np.linalg.norm(v))
    X = np.array(X)
    res = oracle_mod.solve(dom, X, n, 1e-6, sigma, seed=99 + d, grad=True,
                           laplace_factor=laplace_factor)
    ok_u, ok_g = True, True
    for q in range(len(X)):
        u, g = ball_solution(d, R, sigma, X[q])
        ok_u &= abs(res["u"][q] - u) < 4.5 * res["u_se"][q] + 1e-5
        ok_g &= bool(np.all(np.abs(res["grad"][q] - g) < 4.5 * res["grad_se"][q] + 1e-4))
    return ok_u, ok_g


@pytest.mark.parametrize("d,sigma", [(2, 4.0), (3, 16.0), (6, 9.0), (3, 0.0)])
def test_ball_off_centre(oracle_mod, d, sigma):
    ok_u, ok_g = _ball_case(oracle_mod, d, sigma)
    assert ok_u and ok_g


def test_planted_laplace_factor_is_rejected(oracle_mod):
    # The paper's printed factor n/R is the Laplace one; at sigma > 0 it overestimates |grad u|.
    ok_u, ok_g = _ball_case(oracle_mod, 3, 16.0, laplace_factor=True)
    assert ok_u and not ok_g


# --------------------------------------------------------------------------- P3
def test_exp_data_exact_solution_c1(oracle_mod):
    w = synth.c1(n_queries=16)
    dom = w["domain"]
    res = oracle_mod.solve(dom, w["X"], 20000, 1e-4, w["sigma"], w["seed"], grad=True)
    a = dom["exp_a"][0]
    g = np.exp(w["X"] @ a)
    bias = 3e-4 * np.abs(g) * np.linalg.norm(a)  # O(eps) shell bias
    assert np.all(np.abs(res["u"] - g) < 4.5 * res["u_se"] + bias)
    gg = a[None, :] * g[:, None]
    assert np.all(np.abs(res["grad"] - gg) < 4.5 * res["grad_se"] + 10 * bias[:, None])
    assert np.all(res["capped"] == 0)


def test_du_dw_is_exp_and_fd_exact(oracle_mod):
    w = synth.c5(n_queries=4, n_walks=2000, n_balls=8, n_terms=3)
    dom = w["domain"]
    base = oracle_mod.solve(dom, w["X"], w["n_walks"], w["eps"], w["sigma"], w["seed"])
    h = 1e-3
    for k in range(3):
        dp = dict(dom)
        dm = dict(dom)
        dp["exp_w"] = dom["exp_w"].copy()
        dm["exp_w"] = dom["exp_w"].copy()
        dp["exp_w"][k] += h
        dm["exp_w"][k] -= h
        up = oracle_mod.solve(dp, w["X"], w["n_walks"], w["eps"], w["sigma"], w["seed"])["u"]
        um = oracle_mod.solve(dm, w["X"], w["n_walks"], w["eps"], w["sigma"], w["seed"])["u"]
        fd = (up - um) / (2 * h)
        assert np.allclose(fd, base["du_dw"][:, k], rtol=1e-9, atol=1e-12)
        # and du/dw_k estimates exp(a_k . x) (the exact solution's derivative)
        e = np.exp(w["X"] @ dom["exp_a"][k])
        assert np.all(np.abs(base["du_dw"][:, k] - e) < 0.1 * e)


def test_dsigma_crn_finite_difference(oracle_mod):
    w = synth.c5(n_queries=4, n_walks=2000, n_balls=8, n_terms=2)
    dom = w["domain"]
    s, h = w["sigma"], 1e-3
    base = oracle_mod.solve(dom, w["X"], w["n_walks"], w["eps"], s, w["seed"])
    up = oracle_mod.solve(dom, w["X"], w["n_walks"], w["eps"], s + h, w["seed"])["u"]
    um = oracle_mod.solve(dom, w["X"], w["n_walks"], w["eps"], s - h, w["seed"])["u"]
    fd = (up - um) / (2 * h)
    assert np.allclose(fd, base["du_dsigma"], rtol=1e-5, atol=1e-9)
    assert np.all(base["du_dsigma"] < 0)  # more screening, smaller u for positive data


# --------------------------------------------------------------------------- annulus
def annulus_solution(d, r1, r2, sigma, x):
    r = np.linalg.norm(x)
    if sigma == 0.0:
        if d == 2:
            u = math.log(r2 / r) / math.log(r2 / r1)
            du = -1.0 / (r * math.log(r2 / r1))
        else:
            p = 2 - d
            u = (r ** p - r2 ** p) / (r1 ** p - r2 ** p)
            du = p * r ** (p - 1) / (r1 ** p - r2 ** p)
    else:
        nu, k = d / 2 - 1, math.sqrt(sigma)
        f = lambda s: s ** (-nu) * (special.iv(nu, k * s) * special.kv(nu, k * r2) -
                                    special.kv(nu, k * s) * special.iv(nu, k * r2))
        fp = lambda s: k * s ** (-nu) * (special.iv(nu + 1, k * s) * special.kv(nu, k * r2) +
                                         special.kv(nu + 1, k * s) * special.iv(nu, k * r2))
        u = f(r) / f(r1)
        du = fp(r) / f(r1)
    return u, du * x / r


@pytest.mark.parametrize("d,sigma", [(2, 0.0), (2, 4.0), (3, 0.0), (3, 9.0), (5, 2.0)])
def test_annulus_goal_indicator(oracle_mod, d, sigma):
    r1, r2 = 0.3, 1.0
    dom = synth.annulus_domain(d, r1, r2)
    rng = np.random.default_rng(5)
    X = []
    for rad in [0.4, 0.6, 0.85]:
        v = rng.standard_normal(d)
        X.append(rad * v / np.linalg.norm(v))
    X = np.array(X)
    eps = 1e-5
    res = oracle_mod.solve(dom, X, 40000, eps, sigma, seed=3 + d, grad=True, per_walk=True)
    assert np.all((res["walk_term"] >= 0) & (res["walk_term"] <= 1))  # max principle, P6
    for q in range(len(X)):
        u, g = annulus_solution(d, r1, r2, sigma, X[q])
        assert abs(res["u"][q] - u) < 4.5 * res["u_se"][q] + 1e-4
        assert np.all(np.abs(res["grad"][q] - g) < 4.5 * res["grad_se"][q] + 1e-3)


# --------------------------------------------------------------------------- statistics
def test_standard_error_scaling(oracle_mod):
    w = synth.c1(n_queries=6)
    dom, X = w["domain"], w["X"]
    s1 = oracle_mod.solve(dom, X, 4000, w["eps"], w["sigma"], 1)["u_se"]
    s4 = oracle_mod.solve(dom, X, 16000, w["eps"], w["sigma"], 1)["u_se"]
    ratio = s1 / s4
    assert np.all((ratio > 1.8) & (ratio < 2.2)), ratio
    # spread of independent estimates matches the reported standard error
    us = np.array([oracle_mod.solve(dom, X[:2], 1000, w["eps"], w["sigma"], seed)["u"]
                   for seed in range(24)])
    se = oracle_mod.solve(dom, X[:2], 1000, w["eps"], w["sigma"], 100)["u_se"]
    emp = us.std(axis=0, ddof=1)
    assert np.all((emp / se > 0.6) & (emp / se < 1.5))


def test_max_principle_indicator_c2(oracle_mod):
    w = synth.c2()
    X = synth._free_points(np.random.default_rng(1), 8, w["domain"]["box_lo"], w["domain"]["box_hi"],
                           w["domain"]["ball_c"], w["domain"]["ball_r"], 0.05)
    res = oracle_mod.solve(w["domain"], X, 500, w["eps"], w["sigma"], w["seed"], per_walk=True)
    t = res["walk_term"]
    assert np.all((t >= 0) & (t <= 1))
    assert np.all((res["u"] >= 0) & (res["u"] <= 1))


def test_thread_count_does_not_change_results(oracle_mod):
    w = synth.c1(n_queries=5)
    a = oracle_mod.solve(w["domain"], w["X"], 3000, w["eps"], w["sigma"], 5, grad=True, threads=1)
    b = oracle_mod.solve(w["domain"], w["X"], 3000, w["eps"], w["sigma"], 5, grad=True, threads=7)
    for k in a:
        assert np.array_equal(a[k], b[k]), k


def test_cap_and_outside(oracle_mod):
    w = synth.c1(n_queries=3)
    res = oracle_mod.solve(w["domain"], w["X"], 500, 1e-9, w["sigma"], 1, max_steps=2, per_walk=True)
    # exp data is positive, so a zero terminal marks a capped walk; caps happen only at 2 jumps
    capped = res["walk_term"] == 0.0
    assert res["capped"].sum() == capped.sum() > 0
    assert np.all(res["walk_jumps"][capped] == 2)
    assert np.all(res["walk_steps"] == res["walk_jumps"].sum(axis=1) + 500)
    inside_disc = w["domain"]["ball_c"][:1]
    out = oracle_mod.solve(w["domain"], inside_disc, 10, 1e-3, 4.0, 1)
    assert out["outside"][0] == 10 and np.isnan(out["u"][0])


# --------------------------------------------------------------------------- planner
def test_planner_annulus_descends_radially(oracle_mod):
    d = 2
    dom = synth.annulus_domain(d, 0.2, 2.0)
    x0 = np.array([1.2, 0.3])
    s_ub = 0.1
    path, flags, grads = oracle_mod.plan_path(dom, x0, 60, 4000, 1e-4, 1.0, s_ub, seed=8)
    assert flags[len(path) - 1] == 1  # reached the goal
    r = np.linalg.norm(path, axis=1)
    for i in range(len(path) - 1):
        R = min(r[i] - 0.2, 2.0 - r[i])
        s = min(s_ub, 0.5 * R)
        assert abs(np.linalg.norm(path[i + 1] - path[i]) - s) < 1e-12
        if R > 0.05:
            # far from the goal the estimate is accurate: the step points at the centre.
            # (Close to the boundary the first-sphere estimator's variance grows like 1/R0^2.)
            radial = -path[i] / r[i]
            assert (path[i + 1] - path[i]) @ radial / s > math.cos(math.radians(25))
            assert r[i + 1] < r[i]


# --------------------------------------------------------------------------- control variate
# grad^ = G/(N-1) sum_w (t_w - tbar) v_w: G times the sample covariance of the walk values and
# the first directions; E[v] = 0 makes it unbiased for every N >= 2.
def test_control_variate_vanishes_for_constant_data(oracle_mod):
    # sigma = 0 and g = 1 on the whole boundary: every walk returns exactly 1 (C = 1), so the
    # deviations t_w - tbar are rounding-sized and so are the estimate and its standard error,
    # while the plain first-sphere estimate carries the full sampling noise of v.
    d = 3
    dom = synth.ball_domain(d, 1.0)
    X = np.array([[0.3, -0.2, 0.1], [0.0, 0.6, 0.0]])
    cv = oracle_mod.solve(dom, X, 2000, 1e-4, 0.0, 5, grad=True, control_variate=True, per_walk=True)
    plain = oracle_mod.solve(dom, X, 2000, 1e-4, 0.0, 5, grad=True)
    assert np.all(cv["walk_term"] == 1.0)
    G = d / (1.0 - np.linalg.norm(X, axis=1, keepdims=True))  # alpha(R0) / C(R0) = d / R0 at sigma = 0
    assert np.all(np.abs(cv["grad"]) <= 1e-12 * G)
    assert np.all(cv["grad_se"] <= 1e-12 * G)
    assert np.all(np.abs(plain["grad"]).max(axis=1) > 1e-3)
    # the per-query value outputs do not depend on the option
    assert np.array_equal(cv["u"], plain["u"]) and np.array_equal(cv["u_se"], plain["u_se"])


def _two_walk_replicas(oracle_mod, scale=1.0):
    # 20000 independent two-walk estimates at one point of the disc, sigma = 4: the mean of
    # the control-variate estimates must be the exact gradient (off-centre ball closed form)
    d, R, sigma = 2, 1.0, 4.0
    dom = synth.ball_domain(d, R)
    x = np.array([0.3, 0.4])
    Q = 20000
    res = oracle_mod.solve(dom, np.tile(x, (Q, 1)), 2, 1e-6, sigma, 17, grad=True, control_variate=True)
    g = scale * res["grad"]
    mean, se = g.mean(axis=0), g.std(axis=0, ddof=1) / math.sqrt(Q)
    _, exact = ball_solution(d, R, sigma, x)
    return np.abs(mean - exact) < 4.0 * se, se, exact


def test_control_variate_unbiased_with_two_walks(oracle_mod):
    ok, se, exact = _two_walk_replicas(oracle_mod)
    assert np.all(ok)
    assert np.all(se < 0.05 * np.linalg.norm(exact))  # the check has the power to see a bias


def test_planted_control_variate_normalisation_is_rejected(oracle_mod):
    # dividing by N instead of N - 1 (a plausible slip) halves the two-walk estimate
    ok, _, _ = _two_walk_replicas(oracle_mod, scale=0.5)
    assert not np.any(ok)


def test_control_variate_exp_data_exact_and_lower_variance(oracle_mod):
    w = synth.c1(n_queries=16)
    dom = w["domain"]
    cv = oracle_mod.solve(dom, w["X"], 20000, 1e-4, w["sigma"], w["seed"], grad=True, control_variate=True)
    plain = oracle_mod.solve(dom, w["X"], 20000, 1e-4, w["sigma"], w["seed"], grad=True)
    a = dom["exp_a"][0]
    g = np.exp(w["X"] @ a)
    bias = 3e-4 * np.abs(g) * np.linalg.norm(a)  # O(eps) shell bias
    gg = a[None, :] * g[:, None]
    assert np.all(np.abs(cv["grad"] - gg) < 4.5 * cv["grad_se"] + 10 * bias[:, None])
    assert np.mean(cv["grad_se"]) < 0.5 * np.mean(plain["grad_se"])


# --------------------------------------------------------------------------- impulse source
# Laplace(u) - sigma u = -q delta_z, u = 0 on the boundary: each step whose ball contains z
# adds q G_B(x_k, z) times the weight so far; the first-sphere gradient adds q grad_x G_B(x0, z).
def _c0(d, sigma):
    return math.sqrt(sigma) ** (d / 2 - 1) / (2 * math.pi) ** (d / 2)


def _omega(d):
    return 2 * math.pi ** (d / 2) / math.gamma(d / 2)


def test_bessel_K_matches_scipy(oracle_mod):
    worst = 0.0
    for nu in [0, 0.5, 1, 1.5, 2, 3.5, 5, 6, 7]:
        for x in [1e-6, 1e-3, 0.2, 1.0, 7.0, 30.0, 120.0, 400.0]:
            a, b = oracle_mod.bessel_K(nu, x), special.kv(nu, x)
            worst = max(worst, abs(a - b) / b)
    assert worst < 1e-13, worst


@pytest.mark.parametrize("d", [2, 3, 4, 7])
def test_ball_green_function(oracle_mod, d):
    R, sigma = 0.8, 4.0
    k, nu = 2.0, d / 2 - 1
    for r in [1e-3, 0.1, 0.5, 0.79]:
        G, F = oracle_mod.ball_green(d, sigma, r, R)
        # written with scipy's I and K (the oracle uses its own K integral and I series)
        G_ref = _c0(d, sigma) * r ** -nu * (special.kv(nu, k * r) - special.kv(nu, k * R) * special.iv(nu, k * r)
                                            / special.iv(nu, k * R))
        F_ref = _c0(d, sigma) * k * r ** -nu * (special.kv(nu + 1, k * r) - special.kv(nu + 1, k * R)
                                                * special.iv(nu + 1, k * r) / special.iv(nu + 1, k * R))
        assert abs(G - G_ref) <= 1e-10 * abs(G_ref) + 1e-14
        assert abs(F - F_ref) <= 1e-10 * abs(F_ref) + 1e-14
    # zero on the sphere; unit flux out of a small sphere around the source (a unit impulse)
    assert abs(oracle_mod.ball_green(d, sigma, R * (1 - 1e-9), R)[0]) < 1e-7
    r, h = 1e-4, 1e-7
    dG = (oracle_mod.ball_green(d, sigma, r + h, R)[0] - oracle_mod.ball_green(d, sigma, r - h, R)[0]) / (2 * h)
    assert abs(-_omega(d) * r ** (d - 1) * dG - 1.0) < 1e-5
    # sigma -> 0 is the Laplace form (closed, separate code path)
    for r in [0.05, 0.4]:
        G0, F0 = oracle_mod.ball_green(d, 0.0, r, R)
        Gs, Fs = oracle_mod.ball_green(d, 1e-9, r, R)
        assert abs(G0 - Gs) <= 1e-6 * abs(G0) and abs(F0 - Fs) <= 1e-6 * abs(F0)


def test_ball_green_three_dimensional_closed_form(oracle_mod):
    # d = 3: G = (e^{-kr} - e^{-kR} sinh(kr)/sinh(kR)) / (4 pi r); Laplace F = (r^-2 - r R^-3)/(4 pi)
    R, k = 1.3, 1.7
    for r in [0.01, 0.3, 1.0]:
        G, _ = oracle_mod.ball_green(3, k * k, r, R)
        want = (math.exp(-k * r) - math.exp(-k * R) * math.sinh(k * r) / math.sinh(k * R)) / (4 * math.pi * r)
        assert abs(G - want) < 1e-12 * want
        _, F0 = oracle_mod.ball_green(3, 0.0, r, R)
        assert abs(F0 - (r ** -2 - r / R ** 3) / (4 * math.pi)) < 1e-12 * F0


def _centred_source_solution(d, sigma, R, x):
    """u = G_Omega(x, 0) for Omega = B(0, R) and its gradient (radial)."""
    r = np.linalg.norm(x)
    nu = d / 2 - 1
    if sigma == 0.0:
        u = math.log(R / r) / (2 * math.pi) if d == 2 else (r ** (2 - d) - R ** (2 - d)) / ((d - 2) * _omega(d))
        du = -r ** (1 - d) / _omega(d)
    else:
        k = math.sqrt(sigma)
        c0 = _c0(d, sigma)
        u = c0 * r ** -nu * (special.kv(nu, k * r) - special.kv(nu, k * R) * special.iv(nu, k * r) / special.iv(nu, k * R))
        du = -c0 * k * r ** -nu * (special.kv(nu + 1, k * r) + special.kv(nu, k * R) * special.iv(nu + 1, k * r)
                                    / special.iv(nu, k * R))
    return u, du * x / r


def _source_case(oracle_mod, d, sigma, planted=False, control_variate=False):
    R = 1.0
    dom = {"d": d, "outer_c": np.zeros(d), "outer_r": R, "source_z": np.zeros(d), "source_q": 1.0}
    rng = np.random.default_rng(40 + d)
    X = []
    for rad in [0.3, 0.6]:
        v = rng.standard_normal(d)
        X.append(rad * v / np.linalg.norm(v))
    X = np.array(X)
    res = oracle_mod.solve(dom, X, 20000, 1e-6, sigma, seed=7 + d, grad=True, control_variate=control_variate,
                           plant_free_space_source_grad=planted)
    ok_u, ok_g = True, True
    for q in range(len(X)):
        u, g = _centred_source_solution(d, sigma, R, X[q])
        ok_u &= abs(res["u"][q] - u) < 4.5 * res["u_se"][q] + 1e-4 * abs(u)
        ok_g &= bool(np.all(np.abs(res["grad"][q] - g) < 4.5 * res["grad_se"][q] + 1e-3 * np.abs(g).max()))
    return ok_u, ok_g, res


@pytest.mark.parametrize("d,sigma", [(2, 0.0), (2, 4.0), (3, 0.0), (3, 9.0)])
def test_centred_impulse_source_in_a_ball(oracle_mod, d, sigma):
    ok_u, ok_g, res = _source_case(oracle_mod, d, sigma)
    assert ok_u and ok_g
    ok_u, ok_g, _ = _source_case(oracle_mod, d, sigma, control_variate=True)
    assert ok_u and ok_g


def _scipy_ball_green(d, sigma, r, R):
    """G_B between the centre and distance r, written with scipy's I and K (sigma > 0)."""
    k, nu = math.sqrt(sigma), d / 2 - 1
    return _c0(d, sigma) * r ** -nu * (special.kv(nu, k * r) - special.kv(nu, k * R) * special.iv(nu, k * r)
                                       / special.iv(nu, k * R))


def test_ball_green_dsigma(oracle_mod):
    # d = 3 closed form G = sinh(k (R - r)) / (4 pi r sinh(k R)), differentiated symbolically
    sp = pytest.importorskip("sympy")
    s_, r_, R_ = sp.symbols("s r R", positive=True)
    G3 = sp.sinh(sp.sqrt(s_) * (R_ - r_)) / (4 * sp.pi * r_ * sp.sinh(sp.sqrt(s_) * R_))
    dG3 = sp.lambdify((s_, r_, R_), sp.diff(G3, s_))
    for sigma in (0.3, 4.0, 25.0):
        for r in (0.05, 0.4, 0.9):
            want = dG3(sigma, r, 1.2)
            assert abs(oracle_mod.ball_green_dsigma(3, sigma, r, 1.2) - want) < 1e-12 * abs(want)
    # every d: central differences of scipy's form (sigma > 0) and one-sided ones at sigma = 0
    # against the Laplace limit (the first-order term of G_B in sigma)
    for d in range(2, 8):
        for r in (0.1, 0.6):
            for sigma in (2.0, 30.0):
                h = 1e-4 * sigma
                fd = (_scipy_ball_green(d, sigma + h, r, 1.0) - _scipy_ball_green(d, sigma - h, r, 1.0)) / (2 * h)
                assert abs(oracle_mod.ball_green_dsigma(d, sigma, r, 1.0) - fd) < 1e-6 * abs(fd)
            h = 1e-4
            fd = (-3 * oracle_mod.ball_green(d, 0.0, r, 1.0)[0] + 4 * _scipy_ball_green(d, h, r, 1.0)
                  - _scipy_ball_green(d, 2 * h, r, 1.0)) / (2 * h)
            assert abs(oracle_mod.ball_green_dsigma(d, 0.0, r, 1.0) - fd) < 1e-5 * abs(fd)


def _source_exp_domain(d):
    """Unit ball with two ball obstacles, exp data (|a|^2 = 4) on the whole boundary and an
    impulse source: u has a boundary part and a source part."""
    rng = np.random.default_rng(70 + d)
    a = rng.standard_normal(d)
    a *= 2.0 / np.linalg.norm(a)
    c = np.zeros((2, d))
    c[0, 0], c[1, 1] = 0.5, -0.45
    z = np.zeros(d)
    z[0] = -0.3
    return {"d": d, "outer_c": np.zeros(d), "outer_r": 1.0, "ball_c": c, "ball_r": np.array([0.15, 0.1]),
            "exp_w": np.ones(1), "exp_a": a[None, :], "source_z": z, "source_q": 0.7}


@pytest.mark.parametrize("d,sigma", [(2, 0.0), (2, 3.0), (3, 0.0), (3, 6.0), (5, 2.0)])
def test_source_dsigma_crn_finite_difference(oracle_mod, d, sigma):
    # the walk geometry does not depend on sigma, so each walk's value is a smooth function of
    # sigma and its estimated derivative must equal the difference quotient of the same walk
    dom = _source_exp_domain(d)
    X = np.array([[0.1] + [0.2] * (d - 1), [-0.5] + [0.0] * (d - 1)])
    N, eps, seed = 300, 1e-4, 11

    def term(s):
        return oracle_mod.solve(dom, X, N, eps, s, seed, per_walk=True)["walk_term"]

    ref = oracle_mod.solve(dom, X, N, eps, sigma, seed, per_walk=True)
    h = 1e-5
    if sigma == 0.0:
        fd = (-3 * ref["walk_term"] + 4 * term(h) - term(2 * h)) / (2 * h)
    else:
        fd = (term(sigma + h) - term(sigma - h)) / (2 * h)
    got = ref["walk_dsigma"]
    assert np.all(np.isfinite(got))
    assert np.abs(got - fd).max() <= 1e-5 * np.abs(fd).max()
    assert np.allclose(ref["du_dsigma"], got.mean(axis=1), rtol=1e-12, atol=1e-15)
    # the source part matters: without it the derivative is visibly different
    nosrc = {k: v for k, v in dom.items() if k not in ("source_z", "source_q")}
    base = oracle_mod.solve(nosrc, X, N, eps, sigma, seed)
    assert np.abs(ref["du_dsigma"] - base["du_dsigma"]).max() > 1e-3


@pytest.mark.parametrize("d,sigma", [(2, 4.0), (3, 0.0), (3, 9.0)])
def test_centred_source_dsigma_closed_form(oracle_mod, d, sigma):
    # Omega = B(0, 1), unit impulse at the centre: u = G_Omega(x, 0); du/dsigma from scipy's form
    # by central differences (one-sided at sigma = 0, from the Laplace value)
    dom = {"d": d, "outer_c": np.zeros(d), "outer_r": 1.0, "source_z": np.zeros(d), "source_q": 1.0}
    X = np.array([[0.3] + [0.0] * (d - 1), [0.0, 0.6] + [0.0] * (d - 2)])
    res = oracle_mod.solve(dom, X, 20000, 1e-6, sigma, seed=5 + d, per_walk=True)
    se = res["walk_dsigma"].std(axis=1, ddof=1) / math.sqrt(20000)
    for q in range(2):
        r = float(np.linalg.norm(X[q]))
        h = 1e-4
        if sigma == 0.0:
            want = (-3 * _centred_source_solution(d, 0.0, 1.0, X[q])[0] + 4 * _scipy_ball_green(d, h, r, 1.0)
                    - _scipy_ball_green(d, 2 * h, r, 1.0)) / (2 * h)
        else:
            want = (_scipy_ball_green(d, sigma + h, r, 1.0) - _scipy_ball_green(d, sigma - h, r, 1.0)) / (2 * h)
        assert abs(res["du_dsigma"][q] - want) < 4.5 * se[q] + 1e-4 * abs(want)


def test_planted_free_space_source_gradient_is_rejected(oracle_mod):
    # dropping the ball's image term from grad_x G_B biases the gradient wherever the source is
    # inside the first sphere
    ok_u, ok_g, _ = _source_case(oracle_mod, 3, 9.0, planted=True)
    assert ok_u and not ok_g


def test_off_centre_source_kelvin_image(oracle_mod):
    # sigma = 0, Omega = B(0, 1), source at z: u = (1/|x - z| - 1/(|z| |x - z*|)) / (4 pi), z* = z/|z|^2
    z = np.array([0.4, 0.0, 0.0])
    zs = z / np.dot(z, z)
    dom = {"d": 3, "outer_c": np.zeros(3), "outer_r": 1.0, "source_z": z}
    X = np.array([[-0.3, 0.2, 0.0], [0.6, 0.3, 0.1], [0.1, -0.5, 0.4]])
    res = oracle_mod.solve(dom, X, 20000, 1e-6, 0.0, seed=3, grad=True)
    for q, x in enumerate(X):
        a, b = x - z, x - zs
        u = (1 / np.linalg.norm(a) - 1 / (np.linalg.norm(z) * np.linalg.norm(b))) / (4 * math.pi)
        g = (-a / np.linalg.norm(a) ** 3 + b / (np.linalg.norm(z) * np.linalg.norm(b) ** 3)) / (4 * math.pi)
        assert abs(res["u"][q] - u) < 4.5 * res["u_se"][q] + 1e-4 * abs(u)
        assert np.all(np.abs(res["grad"][q] - g) < 4.5 * res["grad_se"][q] + 1e-3 * np.abs(g).max())


# --------------------------------------------------------------------------- extruded domains
def _extruded_env(d, scale=1.0, k_r=0.3):
    """The paper's two-disc environment (Sec. VI) with r_o = scale, extruded along coordinates
    3..d: every component is measured in the first two coordinates, the others are free."""
    r_o = scale
    r_u = k_r * r_o
    r_l = 0.5 * r_u
    c = np.zeros((2, d))
    c[0, 1], c[1, 1] = r_u, -r_l
    return {"d": d, "outer_c": np.zeros(d), "outer_r": r_o, "ball_c": c, "ball_r": np.array([r_u, r_l]),
            "proj_dims": 2}


def _free_cross_section(rng, n, dom):
    """n points of the free cross-section (first two coordinates), free coordinates in [-2, 2]."""
    out = []
    while len(out) < n:
        p = rng.uniform(-dom["outer_r"], dom["outer_r"], size=2)
        if np.linalg.norm(p) > 0.95 * dom["outer_r"]:
            continue
        if any(np.linalg.norm(p - c[:2]) < 1.05 * r for c, r in zip(dom["ball_c"], dom["ball_r"])):
            continue
        out.append(np.concatenate([p, rng.uniform(-2, 2, size=dom["d"] - 2)]))
    return np.array(out)


@pytest.mark.parametrize("d", [3, 5])
def test_extruded_distance_geometry(oracle_mod, d):
    # a component's surface is its cross-section circle times R^(d-2): the nearest point keeps
    # the free coordinates, lies on the boundary at distance R, and no sampled surface point is
    # nearer (with x's free coordinates or any others)
    dom = _extruded_env(d)
    rng = np.random.default_rng(d)
    t = np.linspace(0, 2 * math.pi, 721)
    circles = [(np.zeros(2), dom["outer_r"])] + [(c[:2], r) for c, r in zip(dom["ball_c"], dom["ball_r"])]
    for x in _free_cross_section(rng, 60, dom):
        R, kind, idx, xbar = oracle_mod.distance(dom, x)
        assert R > 0
        assert abs(np.linalg.norm(x - xbar) - R) < 1e-12
        assert np.array_equal(xbar[2:], x[2:])
        R2, _, _, _ = oracle_mod.distance(dom, xbar)
        assert abs(R2) < 1e-12
        for c, r in circles:
            ring = c[None, :] + r * np.stack([np.cos(t), np.sin(t)], 1)
            for free in (x[2:], rng.uniform(-3, 3, size=d - 2)):
                pts = np.concatenate([ring, np.repeat(free[None, :], len(t), 0)], 1)
                assert np.min(np.linalg.norm(pts - x[None, :], axis=1)) >= R - 1e-12


@pytest.mark.parametrize("d,free_only", [(3, False), (4, True)])
def test_extruded_exp_data_exact_solution(oracle_mod, d, free_only):
    # exp(a.x) with |a|^2 = sigma solves the PDE in all of R^d, so with g = exp(a.x) on the
    # extruded boundary it is the solution; a along the free coordinates only tests that the
    # nearest boundary point keeps them
    sigma = 1.0
    rng = np.random.default_rng(40 + d)
    a = np.zeros(d)
    if free_only:
        a[2:] = rng.standard_normal(d - 2)
    else:
        a = rng.standard_normal(d)
    a *= math.sqrt(sigma) / np.linalg.norm(a)
    dom = dict(_extruded_env(d), exp_w=np.ones(1), exp_a=a[None, :])
    X = _free_cross_section(rng, 4, dom)
    res = oracle_mod.solve(dom, X, 6000, 1e-4, sigma, seed=5, grad=True)
    g = np.exp(X @ a)
    bias = 3e-4 * g
    assert np.all(res["capped"] == 0) and np.all(res["outside"] == 0)
    assert np.all(np.abs(res["u"] - g) < 4.5 * res["u_se"] + bias)
    assert np.all(np.abs(res["grad"] - a[None, :] * g[:, None]) < 4.5 * res["grad_se"] + 10 * bias[:, None])


def test_full_projection_is_the_plain_domain(oracle_mod):
    # proj_dims = d measures every component in all coordinates: the same walks as without it
    w = synth.c1(n_queries=4)
    dom = dict(w["domain"])
    a = oracle_mod.solve(dom, w["X"], 500, 1e-3, w["sigma"], w["seed"], grad=True)
    b = oracle_mod.solve(dict(dom, proj_dims=2), w["X"], 500, 1e-3, w["sigma"], w["seed"], grad=True)
    assert np.array_equal(a["u"], b["u"]) and np.array_equal(a["grad"], b["grad"])


# --------------------------------------------------------------------------- Russian roulette
def _roulette_domain(sigma=16.0):
    """d = 3 unit ball with two ball obstacles and exp data (|a|^2 = sigma); 12 queries."""
    rng = np.random.default_rng(4)
    d = 3
    a = rng.standard_normal(d)
    a *= math.sqrt(sigma) / np.linalg.norm(a)
    dom = {"d": d, "outer_c": np.zeros(d), "outer_r": 1.0,
           "ball_c": np.array([[0.5, 0.0, 0.0], [-0.4, 0.3, 0.1]]), "ball_r": np.array([0.2, 0.15]),
           "exp_w": np.ones(1), "exp_a": a[None, :]}
    X = []
    while len(X) < 12:
        p = rng.uniform(-0.7, 0.7, size=d)
        if np.linalg.norm(p) < 0.7 and all(np.linalg.norm(p - c) > r + 0.05
                                           for c, r in zip(dom["ball_c"], dom["ball_r"])):
            X.append(p)
    return dom, np.array(X), a, sigma


def test_roulette_keeps_the_exp_solution_and_shortens_walks(oracle_mod):
    # roulette below w = 0.3 (a third of the walks' later steps have smaller weights at sigma = 16)
    dom, X, a, sigma = _roulette_domain()
    g = np.exp(X @ a)
    bias = 3e-4 * g * np.linalg.norm(a)
    plain = oracle_mod.solve(dom, X, 40000, 1e-4, sigma, 3, grad=True)
    for cv in (False, True):
        res = oracle_mod.solve(dom, X, 40000, 1e-4, sigma, 3, grad=True, roulette=0.3, control_variate=cv)
        assert np.all(np.abs(res["u"] - g) < 4.5 * res["u_se"] + bias)
        assert np.all(np.abs(res["grad"] - a[None, :] * g[:, None]) < 4.5 * res["grad_se"] + 10 * bias[:, None])
        assert res["walk_steps"].sum() < 0.9 * plain["walk_steps"].sum()


def test_roulette_dsigma_agrees_with_the_plain_estimator(oracle_mod):
    # the pathwise du/dsigma (term times the summed d log C / dsigma) stays unbiased under the
    # roulette; the plain estimator is pinned by the ball-centre closed form and the FD test
    dom, X, _, sigma = _roulette_domain()
    est = []
    for roulette, seed in ((0.0, 5), (0.3, 6)):
        r = oracle_mod.solve(dom, X, 40000, 1e-4, sigma, seed, per_walk=True, roulette=roulette)
        w = r["walk_dsigma"]
        est.append((w.mean(axis=1), w.std(axis=1, ddof=1) / math.sqrt(w.shape[1])))
        assert np.allclose(est[-1][0], r["du_dsigma"], rtol=1e-9, atol=1e-12)
    (m0, s0), (m1, s1) = est
    assert np.all(np.abs(m0 - m1) < 4.5 * np.sqrt(s0 ** 2 + s1 ** 2))


def test_roulette_killed_count_matches_the_walks(oracle_mod):
    # the per-query count of walks ended by the roulette is the number of single walks that say so
    dom, X, _, sigma = _roulette_domain()
    res = oracle_mod.solve(dom, X[:2], 300, 1e-4, sigma, 8, grad=True, roulette=0.3)
    for q in range(2):
        n = sum(oracle_mod.walk(dom, X[q], q * 300 + w, 1e-4, sigma, 8, grad=True, roulette=0.3)["killed"]
                for w in range(300))
        assert res["killed"][q] == n > 0
    assert oracle_mod.solve(dom, X[:2], 300, 1e-4, sigma, 8, grad=True)["killed"].sum() == 0


def test_planted_roulette_without_reweight_is_rejected(oracle_mod):
    # survivors that keep their small weight bias u low
    dom, X, a, sigma = _roulette_domain()
    res = oracle_mod.solve(dom, X, 40000, 1e-4, sigma, 3, roulette=0.3, plant_roulette_no_reweight=True)
    g = np.exp(X @ a)
    assert np.mean(np.abs(res["u"] - g) < 4.5 * res["u_se"] + 3e-4 * g * np.linalg.norm(a)) < 0.5


# --------------------------------------------------------------------------- antithetic pairs
def test_antithetic_pairs_take_opposite_first_directions(oracle_mod):
    w = synth.c1(n_queries=1)
    dom, x = w["domain"], w["X"][0]
    for m in (0, 5, 123):
        a = oracle_mod.walk(dom, x, 2 * m, 1e-4, w["sigma"], 7, grad=True, antithetic=True)
        b = oracle_mod.walk(dom, x, 2 * m + 1, 1e-4, w["sigma"], 7, grad=True, antithetic=True)
        assert np.array_equal(a["gv0"], -b["gv0"]) and np.any(a["gv0"] != 0)
        plain = oracle_mod.walk(dom, x, 2 * m, 1e-4, w["sigma"], 7, grad=True)
        assert np.array_equal(a["gv0"], plain["gv0"])  # the even walk is the plain walk


def test_antithetic_exp_solution_with_lower_gradient_se(oracle_mod):
    w = synth.c1(n_queries=16)
    dom = w["domain"]
    a = dom["exp_a"][0]
    g = np.exp(w["X"] @ a)
    bias = 3e-4 * np.abs(g) * np.linalg.norm(a)
    plain = oracle_mod.solve(dom, w["X"], 20000, 1e-4, w["sigma"], w["seed"], grad=True)
    anti = oracle_mod.solve(dom, w["X"], 20000, 1e-4, w["sigma"], w["seed"], grad=True, antithetic=True)
    assert np.all(np.abs(anti["u"] - g) < 4.5 * anti["u_se"] + bias)
    assert np.all(np.abs(anti["grad"] - a[None, :] * g[:, None]) < 4.5 * anti["grad_se"] + 10 * bias[:, None])
    # the pair cancels the part of the walk value even in the first direction
    assert anti["grad_se"].mean() < 0.5 * plain["grad_se"].mean()


def test_antithetic_se_matches_the_spread_of_estimates(oracle_mod):
    # pair means are independent, walks of a pair are not: the SE must come from the pairs
    w = synth.c1(n_queries=1)
    est = np.array([[r["grad"][0, 0], r["grad_se"][0, 0]] for r in
                    (oracle_mod.solve(w["domain"], w["X"], 2000, 1e-4, w["sigma"], 100 + s, grad=True,
                                      antithetic=True) for s in range(60))])
    ratio = est[:, 1].mean() / est[:, 0].std(ddof=1)
    assert 0.7 < ratio < 1.4, ratio


def test_antithetic_rejects_unpaired_layouts(oracle_mod):
    w = synth.c1(n_queries=1)
    for kw in ({"n_walks": 3}, {"walk_offset": 1}, {"control_variate": True}):
        args = dict(n_walks=4, walk_offset=0, control_variate=False)
        args.update(kw)
        with pytest.raises(ValueError):
            oracle_mod.solve(w["domain"], w["X"], args["n_walks"], 1e-4, w["sigma"], 1, grad=True,
                             walk_offset=args["walk_offset"], control_variate=args["control_variate"],
                             antithetic=True)


# --------------------------------------------------------------------------- point sets (Sec. VII-A)
_ORDER = {"goal": 0, "ball": 1, "point": 2, "outer": 3, "face": 4}


def _brute_distance(dom, x):
    """Distance, component and closest point by enumerating every component in numpy, in the
    tie order goal, balls, points, outer ball, box faces (lo_0, hi_0, lo_1, ...); the components
    are measured in the first proj_dims coordinates and the closest point keeps the others."""
    d = dom["d"]
    m = dom.get("proj_dims", 0) or d
    cands = []  # (distance, kind, index)
    if dom.get("goal_r") is not None:
        cands.append((np.linalg.norm(x[:m] - dom["goal_c"][:m]) - dom["goal_r"], 0, 0))
    for i, (c, r) in enumerate(zip(dom.get("ball_c", []), dom.get("ball_r", []))):
        cands.append((np.linalg.norm(x[:m] - c[:m]) - r, 1, i))
    pts = dom.get("points")
    if pts is not None:
        dist = np.linalg.norm(pts[:, :m] - x[None, :m], axis=1)
        for i in range(pts.shape[0]):
            cands.append((dist[i], 2, i))
    if dom.get("outer_r") is not None:
        cands.append((dom["outer_r"] - np.linalg.norm(x[:m] - dom["outer_c"][:m]), 3, 0))
    if dom.get("box_lo") is not None:
        for j in range(m):
            cands.append((x[j] - dom["box_lo"][j], 4, 2 * j))
            cands.append((dom["box_hi"][j] - x[j], 4, 2 * j + 1))
    best = min(range(len(cands)), key=lambda t: (cands[t][0], t))  # first of the minima
    R, kind, idx = cands[best]
    xbar = x.copy()
    if kind == 2:
        xbar[:m] = pts[idx, :m]
    elif kind == 4:
        xbar[idx // 2] = dom["box_lo"][idx // 2] if idx % 2 == 0 else dom["box_hi"][idx // 2]
    else:
        c = {0: dom.get("goal_c"), 1: None if kind != 1 else dom["ball_c"][idx], 3: dom.get("outer_c")}[kind]
        r = {0: dom.get("goal_r"), 1: None if kind != 1 else dom["ball_r"][idx], 3: dom.get("outer_r")}[kind]
        v = x[:m] - c[:m]
        xbar[:m] = c[:m] + r * v / np.linalg.norm(v)
    return R, kind, idx, xbar


@pytest.mark.parametrize("d,m", [(2, 2), (3, 3), (7, 7), (4, 2)])
def test_point_set_distance_brute_force(oracle_mod, d, m):
    """The point-set branch of the distance and its closest point, in a domain that also holds
    a goal, balls, an outer ball and a box, against numpy enumeration of every component."""
    rng = np.random.default_rng(40 + d + m)
    dom = {"d": d, "box_lo": -np.ones(d), "box_hi": np.ones(d), "outer_c": 0.1 * np.ones(d), "outer_r": 1.3,
           "goal_c": rng.uniform(-0.5, 0.5, d), "goal_r": 0.05,
           "ball_c": rng.uniform(-0.8, 0.8, (5, d)), "ball_r": rng.uniform(0.02, 0.08, 5),
           "points": rng.uniform(-0.9, 0.9, (300, d))}
    if m < d:
        dom["proj_dims"] = m
    kinds = set()
    for x in rng.uniform(-0.95, 0.95, (400, d)):
        R, kind, idx, xbar = oracle_mod.distance(dom, x)
        Rb, kb, ib, xb = _brute_distance(dom, x)
        assert abs(R - Rb) <= 1e-14 * max(1.0, abs(Rb))
        assert (kind, idx) == (kb, ib)
        assert np.allclose(xbar, xb, rtol=0, atol=1e-14)
        kinds.add(kind)
    assert 2 in kinds  # the point branch was taken


def test_point_set_ties_go_to_the_lower_component():
    """Exact ties (all values dyadic): a point beats the outer ball and a box face at the same
    distance, and a ball beats a point."""
    import oracle as oracle_mod

    dom = {"d": 2, "outer_c": np.zeros(2), "outer_r": 1.0, "points": np.array([[0.5, 0.5]])}
    R, kind, idx, xbar = oracle_mod.distance(dom, np.array([0.5, 0.0]))
    assert (R, kind, idx) == (0.5, oracle_mod.KIND_POINT, 0) and np.array_equal(xbar, [0.5, 0.5])
    dom = {"d": 2, "box_lo": np.zeros(2), "box_hi": np.ones(2), "points": np.array([[0.25, 0.75]])}
    R, kind, idx, xbar = oracle_mod.distance(dom, np.array([0.25, 0.5]))
    assert (R, kind) == (0.25, oracle_mod.KIND_POINT) and np.array_equal(xbar, [0.25, 0.75])
    dom["ball_c"], dom["ball_r"] = np.array([[0.75, 0.5]]), np.array([0.25])
    R, kind, idx, xbar = oracle_mod.distance(dom, np.array([0.25, 0.5]))
    assert (R, kind) == (0.25, oracle_mod.KIND_BALL) and np.allclose(xbar, [0.5, 0.5], atol=0)


def _ring_points(d, n, centre, radius, rng):
    """n points on a circle in the first two coordinates (other coordinates uniform in [-1, 1])."""
    t = 2 * math.pi * (np.arange(n) + 0.5) / n
    p = np.zeros((n, d))
    p[:, 0] = centre[0] + radius * np.cos(t)
    p[:, 1] = centre[1] + radius * np.sin(t)
    if d > 2:
        p[:, 2:] = rng.uniform(-1, 1, (n, d - 2))
    return p


@pytest.mark.parametrize("d,m", [(2, 2), (3, 2)])
def test_point_set_exp_data_exact_solution(oracle_mod, d, m):
    """g = exp(a.x) with |a|^2 = sigma is the exact solution on a box-plus-points domain: walks
    that end on a point read g at the point (and, extruded, at the walker's free coordinates).
    The point ring is denser than eps, so it acts as a wall and many walks end on it."""
    rng = np.random.default_rng(90 + d)
    sigma = 4.0
    a = rng.standard_normal(d)
    if m < d:
        a[m:] *= 3.0  # weight the free coordinate: a projection that dropped it would fail
    a *= math.sqrt(sigma) / np.linalg.norm(a)
    dom = {"d": d, "box_lo": np.zeros(d), "box_hi": np.ones(d),
           "points": _ring_points(d, 600, (0.5, 0.5), 0.2, rng), "exp_w": np.ones(1), "exp_a": a[None, :]}
    if m < d:
        dom["proj_dims"] = m
        dom["box_lo"][m:], dom["box_hi"][m:] = -5.0, 5.0
    X = np.array([[0.15, 0.5], [0.5, 0.85], [0.8, 0.2], [0.5, 0.5]])
    if d > 2:
        X = np.hstack([X, rng.uniform(-0.5, 0.5, (4, d - 2))])
    eps = 4e-3
    res = oracle_mod.solve(dom, X, 20000, eps, sigma, seed=5, grad=True)
    g = np.exp(X @ a)
    bias = eps * np.linalg.norm(a) * g  # O(eps) shell bias
    assert np.all(np.abs(res["u"] - g) < 4.5 * res["u_se"] + bias)
    assert np.all(np.abs(res["grad"] - a[None, :] * g[:, None]) < 4.5 * res["grad_se"] + 10 * bias[:, None])
    kinds = [oracle_mod.walk(dom, X[0], w, eps, sigma, 5)["comp_kind"] for w in range(400)]
    assert np.mean(np.array(kinds) == oracle_mod.KIND_POINT) > 0.3


# --------------------------------------------------------------------------- P4: sigma = 0, harmonic data
@pytest.mark.parametrize("d,poly", [(2, "x1^2-x2^2"), (3, "x1^2-x2^2"), (3, "x1x2x3")])
def test_laplace_harmonic_polynomial_on_a_ball(oracle_mod, d, poly):
    """sigma = 0 (C = 1 exactly, gradient factor d/R0) on the unit ball with harmonic
    polynomial data: u = g and grad u = grad g inside."""
    if poly == "x1^2-x2^2":
        c, p = np.array([1.0, -1.0]), np.zeros((2, d), np.int32)
        p[0, 0], p[1, 1] = 2, 2
        u_f = lambda x: x[0] ** 2 - x[1] ** 2
        g_f = lambda x: np.r_[2 * x[0], -2 * x[1], np.zeros(d - 2)]
    else:
        c, p = np.array([1.0]), np.ones((1, d), np.int32)
        u_f = lambda x: x[0] * x[1] * x[2]
        g_f = lambda x: np.array([x[1] * x[2], x[0] * x[2], x[0] * x[1]])
    dom = {"d": d, "outer_c": np.zeros(d), "outer_r": 1.0, "poly_c": c, "poly_p": p}
    rng = np.random.default_rng(7 + d)
    X = []
    for rad in [0.3, 0.55, 0.8]:
        v = rng.standard_normal(d)
        X.append(rad * v / np.linalg.norm(v))
    X = np.array(X)
    res = oracle_mod.solve(dom, X, 40000, 1e-5, 0.0, seed=31 + d, grad=True)
    for q in range(len(X)):
        assert abs(res["u"][q] - u_f(X[q])) < 4.5 * res["u_se"][q] + 1e-4
        assert np.all(np.abs(res["grad"][q] - g_f(X[q])) < 4.5 * res["grad_se"][q] + 1e-3)


# --------------------------------------------------------------------------- P5: unit square, g = 1 on the top edge
def square_series(x, y, sigma, terms=4000):
    """u = sum_{k odd} 4/(k pi) sin(k pi x) sinh(l_k y)/sinh(l_k), l_k = sqrt(k^2 pi^2 + sigma),
    and its gradient (separation of variables), for 0 < y < 1."""
    k = np.arange(1, 2 * terms, 2, dtype=float)
    lam = np.sqrt((k * math.pi) ** 2 + sigma)
    ratio = np.exp(lam * (y - 1.0)) * (1 - np.exp(-2 * lam * y)) / (1 - np.exp(-2 * lam))  # sinh(l y)/sinh(l)
    dratio = lam * np.exp(lam * (y - 1.0)) * (1 + np.exp(-2 * lam * y)) / (1 - np.exp(-2 * lam))
    c = 4.0 / (k * math.pi)
    u = np.sum(c * np.sin(k * math.pi * x) * ratio)
    ux = np.sum(c * k * math.pi * np.cos(k * math.pi * x) * ratio)
    uy = np.sum(c * np.sin(k * math.pi * x) * dratio)
    return u, np.array([ux, uy])


def square_fd(n, sigma):
    """5-point finite differences of Laplace(u) = sigma u on an (n+1)^2 grid of the unit square,
    u = 1 on the top edge (0.5 at its two corners), 0 on the other edges."""
    from scipy.sparse import diags, identity, kron
    from scipy.sparse.linalg import spsolve

    h = 1.0 / n
    m = n - 1
    T = diags([np.ones(m - 1), -2 * np.ones(m), np.ones(m - 1)], [-1, 0, 1]) / h ** 2
    I = identity(m)
    A = (kron(I, T) + kron(T, I) - sigma * kron(I, I)).tocsr()  # unknowns ordered (row y, col x)
    b = np.zeros(m * m)
    b[(m - 1) * m:] -= 1.0 / h ** 2  # the top row's neighbours on y = 1 carry u = 1
    U = np.zeros((n + 1, n + 1))
    U[1:n, 1:n] = spsolve(A, b).reshape(m, m)
    U[n, :] = 1.0
    U[n, 0] = U[n, n] = 0.5
    return U  # U[iy, ix]


@pytest.mark.parametrize("sigma", [0.0, 10.0])
def test_unit_square_top_edge_fd_and_series(oracle_mod, sigma):
    """Unit square, g = 1 on the top edge (face hi_1) and 0 elsewhere: the oracle's u and grad u
    against the separation-of-variables series, which is itself checked against a
    Richardson-extrapolated 5-point finite-difference solve on 65^2 and 129^2 grids."""
    pts = np.array([[0.5, 0.5], [0.25, 0.75], [0.75, 0.375], [0.5, 0.875], [0.125, 0.25]])
    U64, U128 = square_fd(64, sigma), square_fd(128, sigma)
    for x, y in pts:
        us, _ = square_series(x, y, sigma)
        u_rich = (4 * U128[int(round(128 * y)), int(round(128 * x))] - U64[int(round(64 * y)), int(round(64 * x))]) / 3
        assert abs(u_rich - us) < 2e-4, (x, y, u_rich, us)
    dom = {"d": 2, "box_lo": np.zeros(2), "box_hi": np.ones(2), "face_g": np.array([0.0, 0.0, 0.0, 1.0])}
    res = oracle_mod.solve(dom, pts, 40000, 1e-5, sigma, seed=17, grad=True)
    for q, (x, y) in enumerate(pts):
        us, gs = square_series(x, y, sigma)
        assert abs(res["u"][q] - us) < 4.5 * res["u_se"][q] + 1e-4, (q, res["u"][q], us)
        assert np.all(np.abs(res["grad"][q] - gs) < 4.5 * res["grad_se"][q] + 1e-3), (q, res["grad"][q], gs)


# --------------------------------------------------------------------------- planar arm (Sec. V, V-A, VII)
def _chain_points(link_l, q, per_link=4001):
    """Points along the links of a planar chain (base at the origin), densely sampled."""
    pts, p, ang = [], np.zeros(2), 0.0
    for l, qi in zip(link_l, q):
        ang += qi
        e = p + l * np.array([math.cos(ang), math.sin(ang)])
        t = np.linspace(0.0, 1.0, per_link)[:, None]
        pts.append(p[None, :] + t * (e - p)[None, :])
        p = e
    return np.concatenate(pts)


def _arm_domain(link_l, obs):
    n = len(link_l)
    return {"d": n, "box_lo": -math.pi * np.ones(n), "box_hi": math.pi * np.ones(n),
            "link_l": np.asarray(link_l, float), "arm_obs": np.asarray(obs, float)}


@pytest.mark.parametrize("link_l", [(1.0, 1.0), (0.7, 1.3, 0.5), (0.4, 0.3, 0.6, 0.2)])
def test_arm_task_distance_brute_force(oracle_mod, link_l):
    rng = np.random.default_rng(len(link_l))
    obs = rng.uniform(-1.5, 1.5, (6, 2))
    dom = _arm_domain(link_l, obs)
    for q in rng.uniform(-math.pi, math.pi, (50, len(link_l))):
        pts = _chain_points(link_l, q)
        brute = np.min(np.linalg.norm(pts[:, None, :] - obs[None, :, :], axis=2))
        got = oracle_mod.arm_task_distance(dom, q)
        assert got <= brute + 1e-12 and brute - got <= max(link_l) / 4000 + 1e-12


@pytest.mark.parametrize("link_l", [(1.0, 1.0), (0.7, 1.3, 0.5)])
def test_arm_lipschitz_constant_bounds_the_kinematics(oracle_mod, link_l):
    """K = sqrt(sum_n (sum_{i<=n} l_i)^2) bounds the spectral norm of the Jacobian of every
    point of the chain (finite differences), and is reached by the stretched chain when all
    links are equal."""
    n = len(link_l)
    K = oracle_mod.arm_lipschitz(_arm_domain(link_l, [[5.0, 5.0]]))
    assert abs(K - math.sqrt(sum(sum(link_l[:i + 1]) ** 2 for i in range(n)))) < 1e-14
    rng = np.random.default_rng(n + 10)
    h = 1e-6
    worst = 0.0
    for q in list(rng.uniform(-math.pi, math.pi, (40, n))) + [np.zeros(n)]:
        base = _chain_points(link_l, q, per_link=9)
        J = np.stack([(_chain_points(link_l, q + h * np.eye(n)[j], per_link=9) - base) / h for j in range(n)], axis=2)
        sv = np.linalg.norm(J, ord=2, axis=(1, 2))
        worst = max(worst, float(sv.max()))
        assert np.all(sv <= K * (1 + 1e-5))
    if len(set(link_l)) == 1:
        assert worst > K * (1 - 1e-5)  # tight for equal links (the stretched chain's tip)


def test_arm_safe_ball_is_collision_free(oracle_mod):
    """Eq. safe_ball: every configuration inside B(q, d_tau(q) / K) keeps the arm off the
    obstacles; the oracle's C-space distance of the arm component is that radius."""
    rng = np.random.default_rng(3)
    link_l, obs = (0.7, 1.3, 0.5), rng.uniform(-1.5, 1.5, (5, 2))
    dom = _arm_domain(link_l, obs)
    K = oracle_mod.arm_lipschitz(dom)
    checked = 0
    for q in rng.uniform(-2.5, 2.5, (60, 3)):
        dt = oracle_mod.arm_task_distance(dom, q)
        R, kind, _, xbar = oracle_mod.distance(dom, q)
        if kind != oracle_mod.KIND_ARM:
            continue
        assert abs(R - dt / K) < 1e-15 and np.array_equal(xbar, q)
        v = rng.standard_normal((300, 3))
        v /= np.linalg.norm(v, axis=1, keepdims=True)
        y = q[None, :] + (R * rng.uniform(0, 1, (300, 1)) ** (1 / 3)) * v
        assert all(oracle_mod.arm_task_distance(dom, yy) > 0.0 for yy in y)
        checked += 1
    assert checked > 20


def test_arm_domain_exp_data_exact_solution(oracle_mod):
    """g = exp(a.q) with |a|^2 = sigma is the exact solution on the RR configuration space; a walk
    ending in the arm's shell reads g at its own position, so only the box faces add an O(eps)
    shell bias."""
    w = synth.rr_arm(0.0)
    dom = dict(w["domain"])
    dom.pop("source_z")
    sigma = 4.0
    a = np.array([1.2, -1.6])
    dom.update({"exp_w": np.ones(1), "exp_a": a[None, :]})
    X = np.array([w["start"], w["goal"], [1.2, 1.0], [2.6, -0.5]])
    eps = 1e-3
    res = oracle_mod.solve(dom, X, 20000, eps, sigma, seed=7, grad=True)
    g = np.exp(X @ a)
    bias = 3 * eps * np.linalg.norm(a) * g
    assert np.all(np.abs(res["u"] - g) < 4.5 * res["u_se"] + bias)
    assert np.all(np.abs(res["grad"] - a[None, :] * g[:, None]) < 4.5 * res["grad_se"] + 10 * bias[:, None])


def test_rr_ik_collision_points_match_the_printed_spacing(oracle_mod):
    """Sec. VII-A: the 200 collision configurations of the RR arm (closed-form IK) touch the
    obstacle, and consecutive ones are 0.017..0.0235 apart, the range the paper prints (it
    supports the link lengths l1 = l2 = 1 read from the figure)."""
    w = synth.rr_arm(0.0, method="lipschitz")
    p = synth.rr_collision_points()
    assert p.shape == (200, 2)
    assert max(oracle_mod.arm_task_distance(w["domain"], q) for q in p) < 1e-12
    gap = np.linalg.norm(np.diff(p, axis=0), axis=1)
    assert gap.min() >= 0.017 and gap.max() <= 0.0235
    # every IK configuration lies in the joint box of Table I
    assert np.all(p >= w["domain"]["box_lo"]) and np.all(p <= w["domain"]["box_hi"])
