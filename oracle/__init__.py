"""Plain FP64 CPU oracle for Walk on Spheres (screened Poisson u and grad u).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference legs are the only callers. The product path
never imports this package, and this package never imports the product path.

The arithmetic lives in ``wos_oracle.c`` (plain C, FP64, pthreads). This module
compiles it with gcc when needed and marshals numpy arrays through ctypes.

Domains are plain dicts (see ``paper_2406_01713_gb300.synth``):
    d, box_lo/box_hi (optional), outer_c/outer_r (optional), goal_c/goal_r (optional),
    ball_c (B x d)/ball_r (B), points (M x d), exp_w (K)/exp_a (K x d).
  Planar arm (configuration-space domains, Sec. V): link_l (n links, joint angles q_0..q_{n-1})
  and arm_obs (M x 2 task-space obstacle points).
  Oracle-only boundary data for the closed-form pins: poly_c (n) / poly_p (n x d int
  exponents), g = sum_m c_m prod_j x_j^p_mj on the whole boundary; face_g (2d), a constant
  per box face in the order lo_0, hi_0, lo_1, ...
"""
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "wos_oracle.c")
_LIB = os.path.join(_HERE, "libwos_oracle.so")
MAXD = 16
MAXEXP = 16

KIND_GOAL, KIND_BALL, KIND_POINT, KIND_OUTER, KIND_FACE, KIND_ARM = 0, 1, 2, 3, 4, 5


def build(force=False):
    """Compile the oracle shared library with gcc (plain C11, no FP contraction)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", "-ffp-contract=off",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class _Domain(ctypes.Structure):
    _fields_ = [
        ("d", ctypes.c_int32),
        ("has_box", ctypes.c_int32),
        ("box_lo", ctypes.c_double * MAXD),
        ("box_hi", ctypes.c_double * MAXD),
        ("has_outer", ctypes.c_int32),
        ("outer_c", ctypes.c_double * MAXD),
        ("outer_r", ctypes.c_double),
        ("has_goal", ctypes.c_int32),
        ("goal_c", ctypes.c_double * MAXD),
        ("goal_r", ctypes.c_double),
        ("n_balls", ctypes.c_int32),
        ("ball_c", ctypes.POINTER(ctypes.c_double)),
        ("ball_r", ctypes.POINTER(ctypes.c_double)),
        ("n_points", ctypes.c_int64),
        ("points", ctypes.POINTER(ctypes.c_double)),
        ("n_exp", ctypes.c_int32),
        ("exp_w", ctypes.POINTER(ctypes.c_double)),
        ("exp_a", ctypes.POINTER(ctypes.c_double)),
        ("has_source", ctypes.c_int32),
        ("source_z", ctypes.c_double * MAXD),
        ("source_q", ctypes.c_double),
        ("proj_dims", ctypes.c_int32),
        ("n_poly", ctypes.c_int32),
        ("poly_c", ctypes.POINTER(ctypes.c_double)),
        ("poly_p", ctypes.POINTER(ctypes.c_int32)),
        ("has_face_g", ctypes.c_int32),
        ("face_g", ctypes.c_double * (2 * MAXD)),
        ("n_links", ctypes.c_int32),
        ("link_l", ctypes.c_double * MAXD),
        ("n_arm_obs", ctypes.c_int64),
        ("arm_obs", ctypes.POINTER(ctypes.c_double)),
    ]


class _Options(ctypes.Structure):
    _fields_ = [
        ("seed", ctypes.c_uint64),
        ("max_steps", ctypes.c_int64),
        ("grad", ctypes.c_int32),
        ("laplace_factor", ctypes.c_int32),
        ("control_variate", ctypes.c_int32),
        ("plant_free_space_source_grad", ctypes.c_int32),
        ("roulette_w", ctypes.c_double),
        ("plant_roulette_no_reweight", ctypes.c_int32),
        ("antithetic", ctypes.c_int32),
    ]


class _WalkOut(ctypes.Structure):
    _fields_ = [
        ("term", ctypes.c_double),
        ("jumps", ctypes.c_int64),
        ("capped", ctypes.c_int32),
        ("outside", ctypes.c_int32),
        ("killed", ctypes.c_int32),
        ("comp_kind", ctypes.c_int32),
        ("comp_index", ctypes.c_int64),
        ("grad", ctypes.c_double * MAXD),
        ("dsigma", ctypes.c_double),
        ("dw", ctypes.c_double * MAXEXP),
        ("gv0", ctypes.c_double * MAXD),
        ("gsrc", ctypes.c_double * MAXD),
    ]


_lib = None
_lock = threading.Lock()
_PD = ctypes.POINTER(ctypes.c_double)
_PI64 = ctypes.POINTER(ctypes.c_int64)
_PI32 = ctypes.POINTER(ctypes.c_int32)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            L.or_philox4x32_10.argtypes = [ctypes.POINTER(ctypes.c_uint32)] * 3
            L.or_normals.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int, _PD]
            L.or_direction.argtypes = L.or_normals.argtypes
            L.or_arm_task_distance.argtypes = [ctypes.POINTER(_Domain), _PD]
            L.or_arm_task_distance.restype = ctypes.c_double
            L.or_arm_lipschitz.argtypes = [ctypes.POINTER(_Domain)]
            L.or_arm_lipschitz.restype = ctypes.c_double
            L.or_series_S.argtypes = [ctypes.c_double, ctypes.c_double]
            L.or_series_S.restype = ctypes.c_double
            L.or_log_C.argtypes = [ctypes.c_double, ctypes.c_double]
            L.or_log_C.restype = ctypes.c_double
            L.or_dsigma_log_C.argtypes = [ctypes.c_double] * 3
            L.or_dsigma_log_C.restype = ctypes.c_double
            L.or_bessel_K.argtypes = [ctypes.c_double, ctypes.c_double]
            L.or_bessel_K.restype = ctypes.c_double
            L.or_ball_green.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_int, _PD, _PD]
            L.or_ball_green_dsigma.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double]
            L.or_ball_green_dsigma.restype = ctypes.c_double
            L.or_distance.argtypes = [ctypes.POINTER(_Domain), _PD, _PI32, _PI64, _PD]
            L.or_distance.restype = ctypes.c_double
            L.or_walk.argtypes = [ctypes.POINTER(_Domain), _PD, ctypes.c_uint64, ctypes.c_double,
                                  ctypes.c_double, ctypes.POINTER(_Options), ctypes.POINTER(_WalkOut)]
            L.or_solve.argtypes = [ctypes.POINTER(_Domain), _PD, ctypes.c_int64, ctypes.c_int64,
                                   ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                   ctypes.POINTER(_Options), ctypes.c_int, _PD, _PD, _PD, _PD, _PD,
                                   _PD, _PI64, _PI64, _PI64, _PI64, _PD, _PI64, _PD, _PD]
            L.or_solve.restype = ctypes.c_int
            L.or_plan_path.argtypes = [ctypes.POINTER(_Domain), _PD, ctypes.c_int64, ctypes.c_int64,
                                       ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                       ctypes.POINTER(_Options), ctypes.c_int, _PD, _PI32, _PD]
            L.or_plan_path.restype = ctypes.c_int64
            _lib = L
    return _lib


def _ptr(a, ctype=ctypes.c_double):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctype))


class Domain:
    """ctypes view of a domain dict; keeps the numpy buffers alive."""

    def __init__(self, dom):
        d = int(dom["d"])
        if not 1 <= d <= MAXD:
            raise ValueError("d out of range")
        s = _Domain()
        s.d = d
        self.d = d
        self._keep = []

        def arr(key, shape):
            v = dom.get(key)
            if v is None:
                return None
            a = np.ascontiguousarray(np.asarray(v, dtype=np.float64).reshape(shape))
            self._keep.append(a)
            return a

        if dom.get("box_lo") is not None:
            s.has_box = 1
            s.box_lo[:d] = list(np.asarray(dom["box_lo"], float))
            s.box_hi[:d] = list(np.asarray(dom["box_hi"], float))
        if dom.get("outer_r") is not None:
            s.has_outer = 1
            s.outer_c[:d] = list(np.asarray(dom["outer_c"], float))
            s.outer_r = float(dom["outer_r"])
        if dom.get("goal_r") is not None:
            s.has_goal = 1
            s.goal_c[:d] = list(np.asarray(dom["goal_c"], float))
            s.goal_r = float(dom["goal_r"])
        bc = arr("ball_c", (-1, d))
        if bc is not None and bc.shape[0] > 0:
            s.n_balls = bc.shape[0]
            s.ball_c = _ptr(bc)
            s.ball_r = _ptr(arr("ball_r", (-1,)))
        pts = arr("points", (-1, d))
        if pts is not None and pts.shape[0] > 0:
            s.n_points = pts.shape[0]
            s.points = _ptr(pts)
        ea = arr("exp_a", (-1, d))
        if ea is not None and ea.shape[0] > 0:
            if ea.shape[0] > MAXEXP:
                raise ValueError("too many exp terms")
            s.n_exp = ea.shape[0]
            s.exp_a = _ptr(ea)
            s.exp_w = _ptr(arr("exp_w", (-1,)))
        if dom.get("source_z") is not None:
            s.has_source = 1
            s.source_z[:d] = list(np.asarray(dom["source_z"], float))
            s.source_q = float(dom.get("source_q", 1.0))
        s.proj_dims = int(dom.get("proj_dims", 0))
        if dom.get("poly_c") is not None:
            pc = arr("poly_c", (-1,))
            pp = np.ascontiguousarray(np.asarray(dom["poly_p"], dtype=np.int32).reshape(-1, d))
            if pp.shape[0] != pc.shape[0] or np.any(pp < 0):
                raise ValueError("poly_p must be n_poly x d non-negative exponents")
            self._keep.append(pp)
            s.n_poly = pc.shape[0]
            s.poly_c = _ptr(pc)
            s.poly_p = _ptr(pp, ctypes.c_int32)
        if dom.get("link_l") is not None:
            ll = np.asarray(dom["link_l"], float).reshape(-1)
            if not 1 <= ll.size <= d:
                raise ValueError("the arm needs 1..d links")
            s.n_links = ll.size
            s.link_l[:ll.size] = list(ll)
            ob = arr("arm_obs", (-1, 2))
            s.n_arm_obs = ob.shape[0]
            s.arm_obs = _ptr(ob)
        if dom.get("face_g") is not None:
            s.has_face_g = 1
            s.face_g[:2 * d] = list(np.asarray(dom["face_g"], float).reshape(2 * d))
        self.n_exp = int(s.n_exp)
        self.s = s


def _opts(seed, max_steps, grad, laplace_factor, control_variate=False, plant_free_space_source_grad=False,
          roulette=0.0, plant_roulette_no_reweight=False, antithetic=False):
    o = _Options()
    o.antithetic = int(bool(antithetic))
    o.plant_free_space_source_grad = int(bool(plant_free_space_source_grad))
    o.roulette_w = float(roulette)
    o.plant_roulette_no_reweight = int(bool(plant_roulette_no_reweight))
    o.seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    o.max_steps = int(max_steps)
    o.grad = int(bool(grad))
    o.laplace_factor = int(bool(laplace_factor))
    o.control_variate = int(bool(control_variate))
    return o


def philox4x32_10(key, ctr):
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    o = (ctypes.c_uint32 * 4)()
    lib().or_philox4x32_10(k, c, o)
    return [int(v) for v in o]


def normals(seed, walk, step, d):
    out = np.zeros(d + 4)
    lib().or_normals(seed, walk, step, d, _ptr(out))
    return out[:d]


def direction(seed, walk, step, d):
    out = np.zeros(d + 4)
    lib().or_direction(seed, walk, step, d, _ptr(out))
    return out[:d]


def series_S(mu, z):
    return lib().or_series_S(float(mu), float(z))


def log_C(nu, z):
    return lib().or_log_C(float(nu), float(z))


def dsigma_log_C(nu, R, sigma):
    return lib().or_dsigma_log_C(float(nu), float(R), float(sigma))


def bessel_K(nu, x):
    return lib().or_bessel_K(float(nu), float(x))


def arm_task_distance(dom, q):
    D = dom if isinstance(dom, Domain) else Domain(dom)
    q = np.ascontiguousarray(np.asarray(q, float))
    return lib().or_arm_task_distance(ctypes.byref(D.s), _ptr(q))


def arm_lipschitz(dom):
    D = dom if isinstance(dom, Domain) else Domain(dom)
    return lib().or_arm_lipschitz(ctypes.byref(D.s))


def ball_green(d, sigma, r, R, free_space=False):
    """(G, F): the ball's Green's function between its centre and a point at distance r, and
    the factor F with grad_x G_B = F (y - x)/r at the centre."""
    G, F = ctypes.c_double(), ctypes.c_double()
    lib().or_ball_green(int(d), float(sigma), float(r), float(R), int(bool(free_space)), ctypes.byref(G),
                        ctypes.byref(F))
    return G.value, F.value


def ball_green_dsigma(d, sigma, r, R):
    """d/dsigma of the ball's Green's function between its centre and a point at distance r."""
    return lib().or_ball_green_dsigma(int(d), float(sigma), float(r), float(R))


def distance(dom, x):
    D = dom if isinstance(dom, Domain) else Domain(dom)
    x = np.ascontiguousarray(np.asarray(x, float))
    kind = ctypes.c_int32()
    idx = ctypes.c_int64()
    xbar = np.zeros(D.d)
    r = lib().or_distance(ctypes.byref(D.s), _ptr(x), ctypes.byref(kind), ctypes.byref(idx), _ptr(xbar))
    return r, int(kind.value), int(idx.value), xbar


def walk(dom, x0, walk_index, eps, sigma, seed, max_steps=10000, grad=False, laplace_factor=False,
         antithetic=False, roulette=0.0):
    D = dom if isinstance(dom, Domain) else Domain(dom)
    x0 = np.ascontiguousarray(np.asarray(x0, float))
    o = _WalkOut()
    opt = _opts(seed, max_steps, grad, laplace_factor, roulette=roulette, antithetic=antithetic)
    lib().or_walk(ctypes.byref(D.s), _ptr(x0), int(walk_index), float(eps), float(sigma),
                  ctypes.byref(opt), ctypes.byref(o))
    return {
        "term": o.term, "jumps": o.jumps, "capped": o.capped, "outside": o.outside, "killed": o.killed,
        "comp_kind": o.comp_kind, "comp_index": o.comp_index,
        "grad": np.array(o.grad[:D.d]), "dsigma": o.dsigma, "dw": np.array(o.dw[:D.n_exp]),
        "gv0": np.array(o.gv0[:D.d]), "gsrc": np.array(o.gsrc[:D.d]),
    }


def solve(dom, X, n_walks, eps, sigma, seed, walk_offset=0, max_steps=10000, grad=False,
          laplace_factor=False, threads=None, per_walk=False, control_variate=False,
          plant_free_space_source_grad=False, roulette=0.0, plant_roulette_no_reweight=False,
          antithetic=False):
    """Per-query estimates. Returns a dict of numpy arrays (u, u_se, grad, grad_se,
    du_dsigma, du_dw, walk_steps, capped, outside, killed; with per_walk also walk_term,
    walk_jumps, walk_grad, walk_dsigma). control_variate (with grad): grad and grad_se are
    the control-variate estimate G/(N-1) sum_w (t_w - tbar) v_w and its standard error.
    roulette > 0: Russian roulette on walk weights below it. antithetic: walk pairs (2m, 2m+1)
    with opposite first directions (n_walks and walk_offset even; not with control_variate)."""
    D = dom if isinstance(dom, Domain) else Domain(dom)
    d, K = D.d, D.n_exp
    X = np.ascontiguousarray(np.asarray(X, float).reshape(-1, d))
    Q, N = X.shape[0], int(n_walks)
    if threads is None:
        threads = os.cpu_count() or 1
    out = {
        "u": np.zeros(Q), "u_se": np.zeros(Q), "grad": np.zeros((Q, d)), "grad_se": np.zeros((Q, d)),
        "du_dsigma": np.zeros(Q), "du_dw": np.zeros((Q, max(K, 1))),
        "walk_steps": np.zeros(Q, np.int64), "capped": np.zeros(Q, np.int64),
        "outside": np.zeros(Q, np.int64), "killed": np.zeros(Q, np.int64),
    }
    pw = {}
    if per_walk:
        pw = {"walk_term": np.zeros((Q, N)), "walk_jumps": np.zeros((Q, N), np.int64),
              "walk_grad": np.zeros((Q, N, d)), "walk_dsigma": np.zeros((Q, N))}
    opt = _opts(seed, max_steps, grad, laplace_factor, control_variate, plant_free_space_source_grad,
                roulette, plant_roulette_no_reweight, antithetic)
    rc = lib().or_solve(
        ctypes.byref(D.s), _ptr(X), Q, N, int(walk_offset), float(eps), float(sigma), ctypes.byref(opt),
        int(threads), _ptr(out["u"]), _ptr(out["u_se"]), _ptr(out["grad"]), _ptr(out["grad_se"]),
        _ptr(out["du_dsigma"]), _ptr(out["du_dw"]) if K else None,
        _ptr(out["walk_steps"], ctypes.c_int64), _ptr(out["capped"], ctypes.c_int64),
        _ptr(out["outside"], ctypes.c_int64), _ptr(out["killed"], ctypes.c_int64),
        _ptr(pw.get("walk_term")), _ptr(pw.get("walk_jumps"), ctypes.c_int64),
        _ptr(pw.get("walk_grad")), _ptr(pw.get("walk_dsigma")))
    if rc != 0:
        raise ValueError("oracle or_solve rejected its arguments")
    out["du_dw"] = out["du_dw"][:, :K]
    out.update(pw)
    return out


def plan_path(dom, x0, n_steps, n_walks, eps, sigma, s_ub, seed, max_steps=10000, threads=None,
              laplace_factor=False, control_variate=False):
    """Screened-harmonic path; returns (path[n_points, d], flags[n_steps], grads[n_steps, d])."""
    D = dom if isinstance(dom, Domain) else Domain(dom)
    d = D.d
    if threads is None:
        threads = os.cpu_count() or 1
    x0 = np.ascontiguousarray(np.asarray(x0, float))
    path = np.zeros((n_steps + 1, d))
    flags = np.zeros(n_steps, np.int32)
    grads = np.zeros((n_steps, d))
    opt = _opts(seed, max_steps, True, laplace_factor, control_variate)
    n = lib().or_plan_path(ctypes.byref(D.s), _ptr(x0), int(n_steps), int(n_walks), float(eps),
                           float(sigma), float(s_ub), ctypes.byref(opt), int(threads), _ptr(path),
                           _ptr(flags, ctypes.c_int32), _ptr(grads))
    return path[:n], flags, grads
