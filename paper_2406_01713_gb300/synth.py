"""Seeded synthetic workloads shaped like the paper's environments.

This module only draws inputs (obstacles, boundary data, query points). It holds none
of the Walk-on-Spheres arithmetic, and it serves both the CUDA path and the CPU oracle.
The paper's environments are analytic and synthetic (Sec. VI, Sec. VII); these
generators stand in for them:

  c1  plain FP64 check, d = 2: [0,1]^2 minus 4 discs, sigma = 4, g = exp(a.x), |a| = 2
  c2  2D planning field: [-pi,pi]^2, 32 discs, goal disc r = 0.1, sigma = 10, 200-step path
  c3  point-cloud C-space, d = 7: 16 random hyperellipsoid surfaces x 4096 points, goal r = 0.05
  c4  batched uneven: 256 problems, d in {3..12}, 16-4096 balls, sigma in [0, 50]
  c5  differentiable, d = 6: 64 balls, g = sum_k w_k exp(a_k.x), 8 terms, |a_k| = 2, sigma = 4

Seeds: workload i (c1 = 1, ...) draws geometry from 1713 + i and walks from 2406 + i.
  env the paper's evaluation environment (Sec. VI): outer disc r_o = 10, discs r_u = k_r r_o
      and r_l = r_u / 2 touching at the origin, a unit impulse at the goal; for d > 2 extruded
      along the added coordinates (free and unbounded), as in the dimensionality study

A domain is a dict of numpy arrays; every key is optional except d:
  d, box_lo, box_hi, outer_c, outer_r, goal_c, goal_r, ball_c (B x d), ball_r (B),
  points (M x d), exp_w (K), exp_a (K x d), source_z (d), source_q, proj_dims.
"""
import math

import numpy as np

GEOM_SEED0 = 1713
WALK_SEED0 = 2406


def _rng(i, salt=0):
    return np.random.default_rng([GEOM_SEED0 + i, salt])


def walk_seed(i):
    return WALK_SEED0 + i


def _clearance_ok(x, centres, radii, margin):
    """True where x (n x d) lies outside every ball by more than margin (input rejection)."""
    if centres is None or len(centres) == 0:
        return np.ones(x.shape[0], bool)
    try:
        from scipy.spatial import cKDTree
    except ImportError:
        cKDTree = None
    if cKDTree is not None and len(centres) > 64:
        # only balls whose centre lies within r_max + margin can violate the clearance
        tree = cKDTree(centres)
        near = tree.query_ball_point(x, float(np.max(radii)) + margin)
        ok = np.ones(x.shape[0], bool)
        for i, idx in enumerate(near):
            if idx:
                dd = np.linalg.norm(centres[idx] - x[i][None, :], axis=1)
                ok[i] = bool(np.all(dd > radii[idx] + margin))
        return ok
    ok = np.ones(x.shape[0], bool)
    for s in range(0, centres.shape[0], 512):
        c = centres[s:s + 512]
        r = radii[s:s + 512]
        diff = x[:, None, :] - c[None, :, :]
        dd = np.sqrt(np.einsum("nbd,nbd->nb", diff, diff))
        ok &= np.all(dd > r[None, :] + margin, axis=1)
    return ok


def _free_points(rng, n, lo, hi, centres, radii, margin, extra=None, max_draws=4_000_000):
    """n points uniform in the box [lo+margin, hi-margin] outside all balls (+margin).
    Raises RuntimeError after max_draws candidates (a region too crowded for the margin)."""
    lo = np.asarray(lo, float)
    hi = np.asarray(hi, float)
    out = []
    have = 0
    drawn = 0
    while have < n:
        if drawn > max_draws:
            raise RuntimeError("no free point with clearance %g after %d draws" % (margin, drawn))
        m = max(64, 2 * (n - have))
        drawn += m
        x = rng.uniform(lo + margin, hi - margin, size=(m, lo.size))
        ok = _clearance_ok(x, centres, radii, margin)
        if extra is not None:
            ok &= extra(x)
        x = x[ok]
        out.append(x)
        have += x.shape[0]
    return np.concatenate(out)[:n]


# ----------------------------------------------------------------------------- c1
def c1(n_queries=64, n_walks=10_000):
    """[0,1]^2 minus 4 discs (centres U[0.2,0.8]^2, r U[0.05,0.12]); sigma = 4;
    g = exp(a.x), a = 2(cos t, sin t) so |a|^2 = sigma and u = g is the exact solution."""
    rng = _rng(1)
    d = 2
    centres = rng.uniform(0.2, 0.8, size=(4, d))
    radii = rng.uniform(0.05, 0.12, size=4)
    theta = rng.uniform(0.0, 2.0 * math.pi)
    a = 2.0 * np.array([[math.cos(theta), math.sin(theta)]])
    dom = {"d": d, "box_lo": np.zeros(d), "box_hi": np.ones(d), "ball_c": centres, "ball_r": radii,
           "exp_w": np.ones(1), "exp_a": a}
    X = _free_points(rng, n_queries, dom["box_lo"], dom["box_hi"], centres, radii, 0.02)
    return {"name": "c1", "domain": dom, "X": X, "n_walks": n_walks, "eps": 1e-3, "sigma": 4.0,
            "seed": walk_seed(1)}


# ----------------------------------------------------------------------------- c2
def c2(n_obstacles=32, n_walks=1024, n_steps=200):
    """[-pi,pi]^2, 32 discs r U[0.1,0.4] (rejecting overlap with start and goal), goal disc
    r = 0.1 (g = 1 there, 0 elsewhere), sigma = 10, eps = 1e-4, s_ub = 0.1."""
    rng = _rng(2)
    d = 2
    lo, hi = -math.pi * np.ones(d), math.pi * np.ones(d)
    while True:
        start = rng.uniform(lo + 0.5, hi - 0.5)
        goal = rng.uniform(lo + 0.5, hi - 0.5)
        if 3.0 <= np.linalg.norm(start - goal) <= 5.0:
            break
    centres, radii = [], []
    while len(centres) < n_obstacles:
        c = rng.uniform(lo, hi)
        r = rng.uniform(0.1, 0.4)
        if np.linalg.norm(c - start) > r + 0.3 and np.linalg.norm(c - goal) > r + 0.3:
            centres.append(c)
            radii.append(r)
    dom = {"d": d, "box_lo": lo, "box_hi": hi, "ball_c": np.array(centres), "ball_r": np.array(radii),
           "goal_c": goal, "goal_r": 0.1}
    return {"name": "c2", "domain": dom, "start": start, "n_walks": n_walks, "n_steps": n_steps,
            "eps": 1e-4, "sigma": 10.0, "s_ub": 0.1, "seed": walk_seed(2)}


# ----------------------------------------------------------------------------- c3
def ellipsoid_cloud(rng, d, n_surfaces, per_surface, box=1.0):
    """Points on random hyperellipsoid surfaces: centre U[-0.6,0.6]^d, semi-axes U[0.1,0.3],
    rotation from the QR factor of a Gaussian matrix; points outside the box are redrawn."""
    pts = []
    for _ in range(n_surfaces):
        centre = rng.uniform(-0.6, 0.6, size=d)
        axes = rng.uniform(0.1, 0.3, size=d)
        q, r = np.linalg.qr(rng.standard_normal((d, d)))
        q = q * np.sign(np.diag(r))[None, :]
        got = []
        have = 0
        while have < per_surface:
            n = rng.standard_normal((per_surface, d))
            n /= np.linalg.norm(n, axis=1, keepdims=True)
            p = (n * axes[None, :]) @ q.T + centre[None, :]
            p = p[np.all(np.abs(p) < box, axis=1)]
            got.append(p)
            have += p.shape[0]
        pts.append(np.concatenate(got)[:per_surface])
    return np.concatenate(pts)


def c3(n_queries=8192, n_walks=4096, n_surfaces=16, per_surface=4096):
    """d = 7 point cloud (16 x 4096 points), box [-1,1]^7 (g = 0), goal ball r = 0.05 (g = 1),
    sigma = 25, eps = 1e-3. Queries uniform in [-0.9,0.9]^7 outside the goal ball."""
    rng = _rng(3)
    d = 7
    pts = ellipsoid_cloud(rng, d, n_surfaces, per_surface)
    while True:
        g = rng.uniform(-0.7, 0.7, size=d)
        if np.min(np.linalg.norm(pts - g[None, :], axis=1)) > 0.2:
            break
    goal_r = 0.05
    X = rng.uniform(-0.9, 0.9, size=(n_queries * 2, d))
    X = X[np.linalg.norm(X - g[None, :], axis=1) > goal_r + 0.01][:n_queries]
    dom = {"d": d, "box_lo": -np.ones(d), "box_hi": np.ones(d), "points": pts.astype(np.float32).astype(float),
           "goal_c": g, "goal_r": goal_r}
    return {"name": "c3", "domain": dom, "X": X, "n_walks": n_walks, "eps": 1e-3, "sigma": 25.0,
            "seed": walk_seed(3)}


# ----------------------------------------------------------------------------- c4
def c4_problem(rng, index, n_queries=64, d=None, n_balls=None, n_walks=None, sigma=None):
    """One problem of the batched workload: d U{3..12}, B log-U[16,4096] balls with radii
    log-U[0.01,0.2] and centres U[-1,1]^d, sigma U[0,50], N log-U[256,16384].
    Even index: g = exp(a.x), |a| = sqrt(sigma) (exact solution u = g).
    Odd index: goal ball r = 0.1 at a point with clearance 0.15 from every obstacle (0.1, 0.05,
    0.02 or 0.01 where the obstacles are too dense), g = 1 there and 0 elsewhere."""
    d = int(rng.integers(3, 13)) if d is None else d
    B = int(round(math.exp(rng.uniform(math.log(16), math.log(4096))))) if n_balls is None else n_balls
    N = int(round(math.exp(rng.uniform(math.log(256), math.log(16384))))) if n_walks is None else n_walks
    sig = float(rng.uniform(0.0, 50.0)) if sigma is None else sigma
    centres = rng.uniform(-1.0, 1.0, size=(B, d))
    radii = np.exp(rng.uniform(math.log(0.01), math.log(0.2), size=B))
    lo, hi = -np.ones(d), np.ones(d)
    dom = {"d": d, "box_lo": lo, "box_hi": hi, "ball_c": centres, "ball_r": radii}
    if index % 2 == 0:
        a = rng.standard_normal(d)
        a *= math.sqrt(sig) / np.linalg.norm(a)
        dom["exp_w"] = np.ones(1)
        dom["exp_a"] = a[None, :]
        X = _free_points(rng, n_queries, lo, hi, centres, radii, 0.01)
    else:
        goal = None
        for clearance in (0.15, 0.1, 0.05, 0.02, 0.01):
            try:
                goal = _free_points(rng, 1, lo, hi, centres, radii, clearance, max_draws=100_000)[0]
                break
            except RuntimeError:
                continue
        if goal is None:
            raise RuntimeError("no free goal position")
        dom["goal_c"] = goal
        dom["goal_r"] = 0.1
        far = lambda x: np.linalg.norm(x - goal[None, :], axis=1) > 0.11
        X = _free_points(rng, n_queries, lo, hi, centres, radii, 0.01, extra=far)
    return {"domain": dom, "X": X, "n_walks": N, "eps": 1e-3, "sigma": sig}


def c4(n_problems=256, n_queries=64, scale_walks=1.0, max_balls=None):
    rng = _rng(4)
    probs = []
    for p in range(n_problems):
        pr = c4_problem(rng, p, n_queries=n_queries)
        if scale_walks != 1.0:
            pr["n_walks"] = max(2, int(round(pr["n_walks"] * scale_walks)))
        if max_balls is not None and pr["domain"]["ball_r"].size > max_balls:
            pr["domain"]["ball_c"] = pr["domain"]["ball_c"][:max_balls]
            pr["domain"]["ball_r"] = pr["domain"]["ball_r"][:max_balls]
        probs.append(pr)
    return {"name": "c4", "problems": probs, "seed": walk_seed(4)}


# ----------------------------------------------------------------------------- c5
def c5(n_queries=4096, n_walks=2048, n_balls=64, n_terms=8):
    """d = 6, 64 balls (radii log-U[0.01,0.2], centres U[-1,1]^6), box [-1,1]^6, sigma = 4,
    g = sum_k w_k exp(a_k.x), |a_k| = 2 (so |a_k|^2 = sigma), w_k ~ U[0.1, 1]."""
    rng = _rng(5)
    d = 6
    centres = rng.uniform(-1.0, 1.0, size=(n_balls, d))
    radii = np.exp(rng.uniform(math.log(0.01), math.log(0.2), size=n_balls))
    a = rng.standard_normal((n_terms, d))
    a *= 2.0 / np.linalg.norm(a, axis=1, keepdims=True)
    w = rng.uniform(0.1, 1.0, size=n_terms)
    lo, hi = -np.ones(d), np.ones(d)
    dom = {"d": d, "box_lo": lo, "box_hi": hi, "ball_c": centres, "ball_r": radii, "exp_w": w, "exp_a": a}
    X = _free_points(rng, n_queries, lo, hi, centres, radii, 0.01)
    return {"name": "c5", "domain": dom, "X": X, "n_walks": n_walks, "eps": 1e-3, "sigma": 4.0,
            "seed": walk_seed(5), "fd_h": 1e-3}


# ----------------------------------------------------------------------------- pins
def ball_domain(d, radius=1.0, goal=None):
    """Omega = B(0, radius) (outer sphere only); g = 1 everywhere via exp data with a = 0."""
    dom = {"d": d, "outer_c": np.zeros(d), "outer_r": float(radius), "exp_w": np.ones(1),
           "exp_a": np.zeros((1, d))}
    return dom


def annulus_domain(d, r_in, r_out):
    """Omega = B(0, r_out) minus B(0, r_in); g = 1 on the inner sphere (goal), 0 outside."""
    return {"d": d, "outer_c": np.zeros(d), "outer_r": float(r_out), "goal_c": np.zeros(d),
            "goal_r": float(r_in)}


def paper_environment(d=2, k_r=0.3, goal=(8.0, 0.0), r_o=10.0):
    """The paper's evaluation environment (Sec. VI): outer disc r_o, upper disc r_u = k_r r_o
    centred at (0, r_u), lower disc r_l = r_u / 2 at (0, -r_l) (they touch at the origin), a
    unit impulse at the goal. The goal point is shown only in a figure; (8, 0) mirrors the
    paper's start (-8, 0). For d > 2 the components are measured in the first two coordinates
    (extruded along the others)."""
    r_u = k_r * r_o
    r_l = 0.5 * r_u
    c = np.zeros((2, d))
    c[0, 1], c[1, 1] = r_u, -r_l
    z = np.zeros(d)
    z[:2] = goal
    dom = {"d": d, "outer_c": np.zeros(d), "outer_r": r_o, "ball_c": c, "ball_r": np.array([r_u, r_l]),
           "source_z": z, "source_q": 1.0}
    if d > 2:
        dom["proj_dims"] = 2
    return dom


# ----------------------------------------------------------------------------- RR arm
RR_TABLE_I = {"q_ub": (1.5 * math.pi, math.pi), "q_start": (0.785, 0.800), "q_goal": (2.042, 0.200),
              "x_obs": (0.0, 1.3), "n_col": 200, "n_walks": 10 ** 5, "s_ub": 0.1, "c": (0.0, 5.0), "eps": 0.02}


def rr_collision_points(link_l=(1.0, 1.0), x_obs=RR_TABLE_I["x_obs"], n=RR_TABLE_I["n_col"]):
    """Configurations of a planar two-link arm whose second link touches the task-space point
    x_obs (closed-form inverse kinematics): the elbow lies on the circle of radius l1 at distance
    <= l2 from x_obs, and link 2 points from the elbow at x_obs. The curve is sampled at n points
    equidistant in arc length (angles wrapped to [-pi, pi) for joint 2)."""
    l1, l2 = link_l
    o = np.asarray(x_obs, float)
    ro = float(np.linalg.norm(o))
    # |o - e|^2 = ro^2 + l1^2 - 2 l1 (o . e) <= l2^2 with e = l1 (cos q1, sin q1)
    c = (ro ** 2 + l1 ** 2 - l2 ** 2) / (2.0 * l1 * ro)
    if not -1.0 <= c <= 1.0:
        raise ValueError("the point is not reachable by the second link only")
    base = math.atan2(o[1], o[0])
    half = math.acos(c)
    q1 = np.linspace(base - half, base + half, 200001)

    def pts(q1):
        e = l1 * np.stack([np.cos(q1), np.sin(q1)], 1)
        v = o[None, :] - e
        q2 = (np.arctan2(v[:, 1], v[:, 0]) - q1 + math.pi) % (2.0 * math.pi) - math.pi
        return np.stack([q1, q2], 1)

    p = pts(q1)
    s = np.concatenate([[0.0], np.cumsum(np.linalg.norm(np.diff(p, axis=0), axis=1))])
    return pts(np.interp(np.linspace(0.0, s[-1], n), s, q1))


def rr_arm(c=0.0, method="lipschitz", link_l=(1.0, 1.0), q_lb=(0.0, -math.pi)):
    """The RR validation environment (Sec. VII, Table I): joint limits q_lb..q_ub, the unit impulse
    at q_goal, zero boundary values, a task-space point obstacle at x_obs. The link lengths
    (l1 = l2 = 1) and the lower joint limits are this build's reading: the paper shows them only
    in a figure. method "lipschitz": the arm component (d_tau / K, Sec. V-A); "ik": the 200
    collision configurations from closed-form IK as a point set (Sec. VII-A)."""
    t = RR_TABLE_I
    dom = {"d": 2, "box_lo": np.asarray(q_lb, float), "box_hi": np.asarray(t["q_ub"], float),
           "source_z": np.asarray(t["q_goal"], float), "source_q": 1.0}
    if method == "lipschitz":
        dom["link_l"] = np.asarray(link_l, float)
        dom["arm_obs"] = np.asarray(t["x_obs"], float)[None, :]
    elif method == "ik":
        dom["points"] = rr_collision_points(link_l)
    else:
        raise ValueError(method)
    return {"name": "rr_" + method, "domain": dom, "start": np.asarray(t["q_start"], float),
            "goal": np.asarray(t["q_goal"], float), "n_walks": t["n_walks"], "eps": t["eps"], "sigma": float(c),
            "s_ub": t["s_ub"], "seed": walk_seed(6)}
