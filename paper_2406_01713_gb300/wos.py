"""Thin Python binding of libwos.so: torch supplies device memory and the current stream;
every step of the estimators runs in the library's CUDA kernels.

    dom = Domain(domain_dict)                      # see synth.py for the dict layout
    r = dom.solve(x, n_walks, eps, sigma)          # u, u_se            (Sec. IV-A value estimator)
    r = dom.grad(x, n_walks, eps, sigma)           # + grad, grad_se, du_dsigma, du_dw
    path, flags, grads = dom.plan_path(x0, n_steps, n_walks, eps, sigma, s_ub)   (Sec. III, VII)
    u = WoSFunction.apply(x, sigma, w, dom, n_walks, eps, seed)   # autograd: d/dx, d/dsigma, d/dw
    b = Batch([...]); b.autotune(); b.run()        # uneven problems, one persistent launch + graph
"""
import ctypes

import numpy as np
import torch

from . import _lib

_VP = ctypes.c_void_p


def _ptr(t):
    return _VP(t.data_ptr()) if t is not None else _VP(0)


def _stream():
    return _VP(torch.cuda.current_stream().cuda_stream)


def _opts(precision="mixed", seed=0, walk_offset=0, max_steps=10000, laplace=False, control_variate=False,
          cuda_core_balls=False, roulette=0.0, antithetic=False, wait_cycles=0):
    o = _lib.Options()
    o.precision = _lib.PRECISION[precision] if isinstance(precision, str) else int(precision)
    o.flags = ((_lib.WOS_FLAG_LAPLACE_FACTOR if laplace else 0) |
               (_lib.WOS_FLAG_GRAD_CONTROL_VARIATE if control_variate else 0) |
               (_lib.WOS_FLAG_CUDA_CORE_BALLS if cuda_core_balls else 0) |
               (_lib.WOS_FLAG_ANTITHETIC if antithetic else 0))
    o.seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    o.walk_offset = int(walk_offset)
    o.max_steps = int(max_steps)
    o.roulette_w = float(roulette)
    o.wait_cycles = int(wait_cycles)
    return o


def _dev_f64(x, d=None):
    if not torch.cuda.is_available():
        raise RuntimeError("a CUDA device is required (the library has no CPU path)")
    t = torch.as_tensor(x, dtype=torch.float64)
    if t.device.type != "cuda":
        t = t.cuda()
    t = t.contiguous()
    if d is not None:
        t = t.reshape(-1, d)
    return t


def stats_dict(t):
    v = t.cpu().tolist()
    return dict(zip(_lib.STATS_FIELDS, v))


class Domain:
    """A domain on the device (wos_domain_create). See synth.py for the dict keys. sigma_max > 0
    builds the mixed-precision weight tables for every sigma up to it here, so that no later
    call allocates one."""

    def __init__(self, dom, sigma_max=None):
        L = _lib.load()
        d = int(dom["d"])
        self.d = d
        self._keep = []

        def arr(key, shape):
            v = dom.get(key)
            if v is None:
                return None
            a = np.ascontiguousarray(np.asarray(v, dtype=np.float64).reshape(shape))
            self._keep.append(a)
            return a

        def p(a):
            return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if a is not None else None

        s = _lib.DomainDesc()
        s.d = d
        s.box_lo = p(arr("box_lo", (d,)))
        s.box_hi = p(arr("box_hi", (d,)))
        if dom.get("outer_r") is not None:
            s.outer_c = p(arr("outer_c", (d,)))
            s.outer_r = float(dom["outer_r"])
        if dom.get("goal_r") is not None:
            s.goal_c = p(arr("goal_c", (d,)))
            s.goal_r = float(dom["goal_r"])
        bc = arr("ball_c", (-1, d))
        if bc is not None and bc.shape[0]:
            s.n_balls = bc.shape[0]
            s.ball_c = p(bc)
            s.ball_r = p(arr("ball_r", (-1,)))
        pts = arr("points", (-1, d))
        if pts is not None and pts.shape[0]:
            s.n_points = pts.shape[0]
            s.points = p(pts)
        ea = arr("exp_a", (-1, d))
        if ea is not None and ea.shape[0]:
            s.n_exp = ea.shape[0]
            s.exp_a = p(ea)
            s.exp_w = p(arr("exp_w", (-1,)))
        if dom.get("source_z") is not None:  # impulse source (strength source_q, default 1)
            s.source_z = p(arr("source_z", (d,)))
            s.source_q = float(dom.get("source_q", 1.0))
        self.has_source = dom.get("source_z") is not None
        # extruded domain: components measured in the first proj_dims coordinates only
        s.proj_dims = int(dom.get("proj_dims", 0))
        if dom.get("link_l") is not None:  # planar arm in configuration space (Sec. V-A)
            ll = arr("link_l", (-1,))
            s.n_links = ll.shape[0]
            s.link_l = p(ll)
            ob = arr("arm_obs", (-1, 2))
            s.n_arm_obs = ob.shape[0]
            s.arm_obs = p(ob)
        s.sigma_max = float(sigma_max if sigma_max is not None else dom.get("sigma_max", 0.0))
        self.n_exp = int(s.n_exp)
        self.n_balls = int(s.n_balls)
        self.n_points = int(s.n_points)
        h = _VP()
        _lib.check(L.wos_domain_create(ctypes.byref(s), ctypes.byref(h)), "wos_domain_create")
        self.h = h
        self._keep = None

    def close(self):
        if getattr(self, "h", None):
            _lib.load().wos_domain_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ----------------------------------------------------------------- estimators
    def solve(self, x, n_walks, eps, sigma, precision="mixed", seed=0, walk_offset=0,
              max_steps=10000, laplace=False, with_stats=False, cuda_core_balls=False, roulette=0.0,
              antithetic=False, wait_cycles=0):
        L = _lib.load()
        x = _dev_f64(x, self.d)
        Q = x.shape[0]
        u = torch.empty(Q, dtype=torch.float64, device=x.device)
        se = torch.empty_like(u)
        st = torch.zeros(len(_lib.STATS_FIELDS), dtype=torch.int64, device=x.device) if with_stats else None
        o = _opts(precision, seed, walk_offset, max_steps, laplace, cuda_core_balls=cuda_core_balls,
                  roulette=roulette, antithetic=antithetic, wait_cycles=wait_cycles)
        _lib.check(L.wos_solve(self.h, ctypes.byref(o), _ptr(x), Q, int(n_walks), float(eps),
                               float(sigma), _ptr(u), _ptr(se), _ptr(st), _stream()), "wos_solve")
        out = {"u": u, "u_se": se}
        if with_stats:
            out["stats"] = st
        return out

    def grad(self, x, n_walks, eps, sigma, precision="mixed", seed=0, walk_offset=0,
             max_steps=10000, laplace=False, with_stats=False, control_variate=False, cuda_core_balls=False,
             roulette=0.0, antithetic=False, wait_cycles=0):
        """u, grad u (first-sphere estimator; control_variate=True subtracts the walks' mean
        value, WOS_FLAG_GRAD_CONTROL_VARIATE), their SEs, du/dsigma and du/dw per query."""
        L = _lib.load()
        x = _dev_f64(x, self.d)
        Q, d = x.shape[0], self.d
        f = dict(dtype=torch.float64, device=x.device)
        out = {"u": torch.empty(Q, **f), "u_se": torch.empty(Q, **f), "grad": torch.empty(Q, d, **f),
               "grad_se": torch.empty(Q, d, **f), "du_dsigma": torch.empty(Q, **f),
               "du_dw": torch.empty(Q, self.n_exp, **f) if self.n_exp else None}
        st = torch.zeros(len(_lib.STATS_FIELDS), dtype=torch.int64, device=x.device) if with_stats else None
        o = _opts(precision, seed, walk_offset, max_steps, laplace, control_variate, cuda_core_balls, roulette,
                  antithetic, wait_cycles)
        _lib.check(L.wos_grad(self.h, ctypes.byref(o), _ptr(x), Q, int(n_walks), float(eps), float(sigma),
                              _ptr(out["u"]), _ptr(out["u_se"]), _ptr(out["grad"]), _ptr(out["grad_se"]),
                              _ptr(out["du_dsigma"]), _ptr(out["du_dw"]), _ptr(st), _stream()),
                   "wos_grad")
        if with_stats:
            out["stats"] = st
        return out

    def walks(self, x, n_walks, eps, sigma, grad_mode=False, precision="mixed", seed=0,
              walk_offset=0, max_steps=10000, laplace=False, cuda_core_balls=False, roulette=0.0,
              antithetic=False, wait_cycles=0):
        """Per-walk terminals, jump counts, gradient estimates and d/dsigma (parity checks)."""
        L = _lib.load()
        x = _dev_f64(x, self.d)
        Q, d, N = x.shape[0], self.d, int(n_walks)
        f = dict(dtype=torch.float64, device=x.device)
        out = {"term": torch.empty(Q, N, **f), "jumps": torch.empty(Q, N, dtype=torch.int64, device=x.device),
               "grad": torch.empty(Q, N, d, **f), "dsigma": torch.empty(Q, N, **f)}
        o = _opts(precision, seed, walk_offset, max_steps, laplace, cuda_core_balls=cuda_core_balls,
                  roulette=roulette, antithetic=antithetic, wait_cycles=wait_cycles)
        _lib.check(L.wos_walks(self.h, ctypes.byref(o), _ptr(x), Q, N, float(eps), float(sigma),
                               int(bool(grad_mode)), _ptr(out["term"]), _ptr(out["jumps"]),
                               _ptr(out["grad"]), _ptr(out["dsigma"]), _stream()), "wos_walks")
        return out

    # ----------------------------------------------------------------- planner
    def plan_step(self, x, n_walks, eps, sigma, s_ub, step_idx, precision="mixed", seed=0,
                  walk_offset=0, max_steps=10000, control_variate=False, roulette=0.0, antithetic=False,
                  wait_cycles=0):
        """One step in place on the device tensor x (d doubles); returns (flag, grad)."""
        L = _lib.load()
        assert x.dtype == torch.float64 and x.is_cuda and x.numel() == self.d and x.is_contiguous()
        flag = torch.zeros(1, dtype=torch.int32, device=x.device)
        g = torch.empty(self.d, dtype=torch.float64, device=x.device)
        o = _opts(precision, seed, walk_offset, max_steps, control_variate=control_variate, roulette=roulette,
                  antithetic=antithetic, wait_cycles=wait_cycles)
        _lib.check(L.wos_plan_step(self.h, ctypes.byref(o), _ptr(x), int(n_walks), float(eps), float(sigma),
                                   float(s_ub), int(step_idx), _ptr(flag), _ptr(g), _stream()),
                   "wos_plan_step")
        return flag, g

    def plan_path(self, x0, n_steps, n_walks, eps, sigma, s_ub, precision="mixed", seed=0,
                  walk_offset=0, max_steps=10000, control_variate=False, roulette=0.0, antithetic=False,
                  wait_cycles=0):
        """n_steps planner steps replayed as one CUDA graph: (path, flags, grads) on the device."""
        L = _lib.load()
        x0 = _dev_f64(x0).reshape(-1)
        d = self.d
        f = dict(dtype=torch.float64, device=x0.device)
        path = torch.empty(n_steps + 1, d, **f)
        flags = torch.zeros(n_steps, dtype=torch.int32, device=x0.device)
        grads = torch.zeros(n_steps, d, **f)
        o = _opts(precision, seed, walk_offset, max_steps, control_variate=control_variate, roulette=roulette,
                  antithetic=antithetic, wait_cycles=wait_cycles)
        _lib.check(L.wos_plan_path(self.h, ctypes.byref(o), _ptr(x0), int(n_steps), int(n_walks), float(eps),
                                   float(sigma), float(s_ub), _ptr(path), _ptr(flags), _ptr(grads),
                                   _stream()), "wos_plan_path")
        return path, flags, grads

    def info(self):
        """{'tensor_sphere_set': bool, 'sphere_tiles': int}: which mixed-precision walker runs it."""
        L = _lib.load()
        t, n = ctypes.c_int32(0), ctypes.c_int32(0)
        _lib.check(L.wos_domain_info(self.h, ctypes.byref(t), ctypes.byref(n)), "wos_domain_info")
        return {"tensor_sphere_set": bool(t.value), "sphere_tiles": int(n.value)}

    def set_exp_w(self, w):
        L = _lib.load()
        w = _dev_f64(w).reshape(-1)
        _lib.check(L.wos_domain_set_exp_w(self.h, _ptr(w), w.numel(), _stream()), "wos_domain_set_exp_w")
        self._w_keep = w


def backward(gout, grad, du_dsigma=None, du_dw=None):
    """gx = gout * grad, gsigma = sum gout du_dsigma, gw = sum gout du_dw (wos_backward)."""
    L = _lib.load()
    Q, d = grad.shape
    K = du_dw.shape[1] if du_dw is not None else 0
    f = dict(dtype=torch.float64, device=grad.device)
    gx = torch.empty(Q, d, **f)
    gs = torch.zeros(1, **f)
    gw = torch.zeros(max(K, 1), **f)
    gout = gout.to(torch.float64).contiguous()
    _lib.check(L.wos_backward(_ptr(gout), _ptr(grad.contiguous()),
                              _ptr(du_dsigma.contiguous()) if du_dsigma is not None else _VP(0),
                              _ptr(du_dw.contiguous()) if du_dw is not None else _VP(0), Q, d, K,
                              _ptr(gx), _ptr(gs), _ptr(gw) if K else _VP(0), _stream()), "wos_backward")
    return gx, gs[0], gw[:K]


def plan_paths(paths, n_steps, seed=0, walk_offset=0, max_steps=10000, control_variate=False, roulette=0.0,
               antithetic=False, wait_cycles=0):
    """Many planner paths in one CUDA graph (wos_plan_paths): paths is a list of dicts
    {domain: Domain, x0, n_walks, eps, sigma, s_ub}; returns [(path, flags, grads)] on the device,
    each equal to Domain.plan_path with the same arguments (mixed precision)."""
    L = _lib.load()
    arr = (_lib.PathProblem * len(paths))()
    out = []
    for i, p in enumerate(paths):
        dom = p["domain"]
        d = dom.d
        x0 = _dev_f64(p["x0"]).reshape(-1)
        f = dict(dtype=torch.float64, device=x0.device)
        path = torch.empty(n_steps + 1, d, **f)
        flags = torch.zeros(n_steps, dtype=torch.int32, device=x0.device)
        grads = torch.zeros(n_steps, d, **f)
        out.append((path, flags, grads, x0))
        a = arr[i]
        a.domain = dom.h
        a.x0 = x0.data_ptr()
        a.n_walks = int(p["n_walks"])
        a.eps = float(p["eps"])
        a.sigma = float(p["sigma"])
        a.s_ub = float(p["s_ub"])
        a.path = path.data_ptr()
        a.flags = flags.data_ptr()
        a.grads = grads.data_ptr()
    o = _opts("mixed", seed, walk_offset, max_steps, control_variate=control_variate, roulette=roulette,
              antithetic=antithetic, wait_cycles=wait_cycles)
    _lib.check(L.wos_plan_paths(arr, len(paths), int(n_steps), ctypes.byref(o), _stream()), "wos_plan_paths")
    return [(p, f, g) for p, f, g, _ in out]


class WoSFunction(torch.autograd.Function):
    """u(x; sigma, w) by Walk on Spheres with a hand-written backward.

    forward: one gradient-walk pass (wos_grad) gives u, grad u, du/dsigma and du/dw from the
    same walks; backward: wos_backward contracts the upstream gradient with them. The walk
    geometry does not depend on sigma or w, so du/dsigma and du/dw are exact per walk.
    """

    @staticmethod
    def forward(ctx, x, sigma, w, domain, n_walks, eps, seed=0, precision="mixed", control_variate=False):
        if w is not None:
            domain.set_exp_w(w.detach())
        r = domain.grad(x.detach(), n_walks, eps, float(sigma), precision=precision, seed=seed,
                        control_variate=control_variate)
        ctx.save_for_backward(r["grad"], r["du_dsigma"],
                              r["du_dw"] if r["du_dw"] is not None else torch.zeros(0, device=x.device))
        ctx.has_w = w is not None
        ctx.sigma_is_tensor = torch.is_tensor(sigma)
        return r["u"].to(x.dtype)

    @staticmethod
    def backward(ctx, gout):
        grad, dsig, dw = ctx.saved_tensors
        gx, gs, gw = backward(gout, grad, dsig, dw if dw.numel() else None)
        return (gx, gs if ctx.sigma_is_tensor else None, gw if ctx.has_w else None,
                None, None, None, None, None, None)


class Batch:
    """Uneven problems in one persistent launch recorded as a CUDA graph (wos_batch_*).

    problems: list of dicts {domain: Domain, x: (Q, d) array, n_walks, eps, sigma, grad: bool}.
    Inputs and outputs live in contiguous device buffers (x_buf, u_buf, se_buf, grad_buf,
    gse_buf, steps_buf) so that a whole batch moves with one copy each way;
    self.out[i] = {u, u_se, grad, grad_se, walk_steps} are views of them.
    """

    def __init__(self, problems, seed=0, max_steps=10000, config=None, control_variate=False, roulette=0.0,
                 antithetic=False, wait_cycles=0):
        L = _lib.load()
        self.problems = problems
        f = dict(dtype=torch.float64, device="cuda")
        qs = [int(np.asarray(p["x"]).reshape(-1, p["domain"].d).shape[0]) if not torch.is_tensor(p["x"])
              else int(p["x"].reshape(-1, p["domain"].d).shape[0]) for p in problems]
        xd = sum(q * p["domain"].d for q, p in zip(qs, problems))
        gd = sum(q * p["domain"].d for q, p in zip(qs, problems) if p.get("grad"))
        self.x_buf = torch.empty(max(xd, 1), **f)
        self.u_buf = torch.empty(max(sum(qs), 1), **f)
        self.se_buf = torch.empty_like(self.u_buf)
        self.steps_buf = torch.zeros(max(sum(qs), 1), dtype=torch.int64, device="cuda")
        self.grad_buf = torch.empty(max(gd, 1), **f)
        self.gse_buf = torch.empty_like(self.grad_buf)
        self.out = []
        arr = (_lib.Problem * len(problems))()
        ox = oq = og = 0
        for i, (p, Q) in enumerate(zip(problems, qs)):
            dom = p["domain"]
            d = dom.d
            xv = self.x_buf[ox:ox + Q * d].view(Q, d)
            xv.copy_(torch.as_tensor(p["x"], dtype=torch.float64).reshape(Q, d))
            o = {"x": xv, "u": self.u_buf[oq:oq + Q], "u_se": self.se_buf[oq:oq + Q],
                 "walk_steps": self.steps_buf[oq:oq + Q]}
            if p.get("grad"):
                o["grad"] = self.grad_buf[og:og + Q * d].view(Q, d)
                o["grad_se"] = self.gse_buf[og:og + Q * d].view(Q, d)
                og += Q * d
            ox += Q * d
            oq += Q
            self.out.append(o)
            a = arr[i]
            a.domain = dom.h
            a.x = xv.data_ptr()
            a.n_queries = Q
            a.n_walks = int(p["n_walks"])
            a.eps = float(p["eps"])
            a.sigma = float(p["sigma"])
            a.u = o["u"].data_ptr()
            a.u_se = o["u_se"].data_ptr()
            a.grad = o["grad"].data_ptr() if "grad" in o else None
            a.grad_se = o["grad_se"].data_ptr() if "grad_se" in o else None
            a.walk_steps = o["walk_steps"].data_ptr()
        self.n_x, self.n_q, self.n_g = ox, oq, og
        self._arr = arr
        opts = _opts("mixed", seed, 0, max_steps, control_variate=control_variate, roulette=roulette,
                     antithetic=antithetic, wait_cycles=wait_cycles)
        cfg = None
        if config is not None:
            cfg = _lib.BatchConfig(int(config["threads"]), int(config["ctas_per_sm"]), int(config["item_work"]),
                                   int(config.get("sphere_ctas_per_sm", 4)), 0,
                                   int(config.get("sphere_item_walks", 4096)))
        h = _VP()
        _lib.check(L.wos_batch_create(arr, len(problems), ctypes.byref(opts),
                                      ctypes.byref(cfg) if cfg is not None else None, ctypes.byref(h)),
                   "wos_batch_create")
        self.h = h
        self.stats = torch.zeros(len(_lib.STATS_FIELDS), dtype=torch.int64, device="cuda")

    def run(self, with_stats=True):
        L = _lib.load()
        _lib.check(L.wos_batch_run(self.h, _ptr(self.stats) if with_stats else _VP(0), _stream()),
                   "wos_batch_run")
        return self.out

    def autotune(self, cache_path=None):
        L = _lib.load()
        best = _lib.BatchConfig()
        _lib.check(L.wos_batch_autotune(self.h, cache_path.encode() if cache_path else None,
                                        ctypes.byref(best)), "wos_batch_autotune")
        return {"threads": best.threads, "ctas_per_sm": best.ctas_per_sm, "item_work": best.item_work,
                "sphere_ctas_per_sm": best.sphere_ctas_per_sm, "sphere_item_walks": best.sphere_item_walks}

    def config(self):
        L = _lib.load()
        c = _lib.BatchConfig()
        _lib.check(L.wos_batch_get_config(self.h, ctypes.byref(c)), "wos_batch_get_config")
        return {"threads": c.threads, "ctas_per_sm": c.ctas_per_sm, "item_work": c.item_work,
                "sphere_ctas_per_sm": c.sphere_ctas_per_sm, "sphere_item_walks": c.sphere_item_walks}

    def close(self):
        if getattr(self, "h", None):
            _lib.load().wos_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def set_autotune_cache(path):
    _lib.check(_lib.load().wos_set_autotune_cache(path.encode() if path else None), "wos_set_autotune_cache")
