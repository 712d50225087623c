"""ctypes declarations of the C ABI in include/wos.h (argument marshalling only)."""
import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libwos.so")

WOS_OK = 0
WOS_FP64, WOS_FP32_PLAIN, WOS_MIXED = 0, 1, 2
WOS_FLAG_LAPLACE_FACTOR = 1
WOS_FLAG_GRAD_CONTROL_VARIATE = 2
WOS_FLAG_CUDA_CORE_BALLS = 4
WOS_FLAG_ANTITHETIC = 8
WOS_MAX_D = 12
WOS_MAX_EXP = 8

PRECISION = {"fp64": WOS_FP64, "fp32": WOS_FP32_PLAIN, "plain": WOS_FP32_PLAIN, "mixed": WOS_MIXED}

_PD = ctypes.POINTER(ctypes.c_double)
_VP = ctypes.c_void_p


class DomainDesc(ctypes.Structure):
    _fields_ = [
        ("d", ctypes.c_int32),
        ("box_lo", _PD), ("box_hi", _PD),
        ("outer_c", _PD), ("outer_r", ctypes.c_double),
        ("goal_c", _PD), ("goal_r", ctypes.c_double),
        ("n_balls", ctypes.c_int32), ("ball_c", _PD), ("ball_r", _PD),
        ("n_points", ctypes.c_int64), ("points", _PD),
        ("n_exp", ctypes.c_int32), ("exp_w", _PD), ("exp_a", _PD),
        ("source_z", _PD), ("source_q", ctypes.c_double),
        ("proj_dims", ctypes.c_int32),
        ("n_links", ctypes.c_int32), ("link_l", _PD),
        ("n_arm_obs", ctypes.c_int64), ("arm_obs", _PD),
        ("sigma_max", ctypes.c_double),
    ]


class Options(ctypes.Structure):
    _fields_ = [
        ("precision", ctypes.c_int32),
        ("flags", ctypes.c_int32),
        ("seed", ctypes.c_uint64),
        ("walk_offset", ctypes.c_int64),
        ("max_steps", ctypes.c_int64),
        ("roulette_w", ctypes.c_double),
        ("wait_cycles", ctypes.c_int64),
    ]


class Stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in
                ("walks", "walk_steps", "capped", "outside", "shrinks", "killed", "timeouts")]


STATS_FIELDS = [f[0] for f in Stats._fields_]


class Problem(ctypes.Structure):
    _fields_ = [
        ("domain", _VP),
        ("x", _VP),
        ("n_queries", ctypes.c_int64),
        ("n_walks", ctypes.c_int64),
        ("eps", ctypes.c_double),
        ("sigma", ctypes.c_double),
        ("u", _VP), ("u_se", _VP), ("grad", _VP), ("grad_se", _VP),
        ("walk_steps", _VP),
    ]


class PathProblem(ctypes.Structure):
    _fields_ = [
        ("domain", _VP),
        ("x0", _VP),
        ("n_walks", ctypes.c_int64),
        ("eps", ctypes.c_double),
        ("sigma", ctypes.c_double),
        ("s_ub", ctypes.c_double),
        ("path", _VP), ("flags", _VP), ("grads", _VP),
    ]


class BatchConfig(ctypes.Structure):
    _fields_ = [("threads", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("item_work", ctypes.c_int64), ("sphere_ctas_per_sm", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("sphere_item_walks", ctypes.c_int64)]


# name -> (restype, argtypes); every entry point declared in include/wos.h
SIGNATURES = {
    "wos_domain_create": (ctypes.c_int, [ctypes.POINTER(DomainDesc), ctypes.POINTER(_VP)]),
    "wos_domain_destroy": (ctypes.c_int, [_VP]),
    "wos_domain_set_exp_w": (ctypes.c_int, [_VP, _VP, ctypes.c_int32, _VP]),
    "wos_domain_info": (ctypes.c_int, [_VP, _VP, _VP]),
    "wos_solve": (ctypes.c_int, [_VP, ctypes.POINTER(Options), _VP, ctypes.c_int64, ctypes.c_int64,
                                 ctypes.c_double, ctypes.c_double, _VP, _VP, _VP, _VP]),
    "wos_grad": (ctypes.c_int, [_VP, ctypes.POINTER(Options), _VP, ctypes.c_int64, ctypes.c_int64,
                                ctypes.c_double, ctypes.c_double, _VP, _VP, _VP, _VP, _VP, _VP, _VP,
                                _VP]),
    "wos_walks": (ctypes.c_int, [_VP, ctypes.POINTER(Options), _VP, ctypes.c_int64, ctypes.c_int64,
                                 ctypes.c_double, ctypes.c_double, ctypes.c_int32, _VP, _VP, _VP, _VP,
                                 _VP]),
    "wos_plan_step": (ctypes.c_int, [_VP, ctypes.POINTER(Options), _VP, ctypes.c_int64, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_double, ctypes.c_int64, _VP, _VP, _VP]),
    "wos_plan_path": (ctypes.c_int, [_VP, ctypes.POINTER(Options), _VP, ctypes.c_int64, ctypes.c_int64,
                                     ctypes.c_double, ctypes.c_double, ctypes.c_double, _VP, _VP, _VP,
                                     _VP]),
    "wos_plan_paths": (ctypes.c_int, [_VP, ctypes.c_int32, ctypes.c_int64, _VP, _VP]),
    "wos_backward": (ctypes.c_int, [_VP, _VP, _VP, _VP, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                    _VP, _VP, _VP, _VP]),
    "wos_batch_create": (ctypes.c_int, [ctypes.POINTER(Problem), ctypes.c_int32, ctypes.POINTER(Options),
                                        ctypes.POINTER(BatchConfig), ctypes.POINTER(_VP)]),
    "wos_batch_run": (ctypes.c_int, [_VP, _VP, _VP]),
    "wos_batch_get_config": (ctypes.c_int, [_VP, ctypes.POINTER(BatchConfig)]),
    "wos_batch_destroy": (ctypes.c_int, [_VP]),
    "wos_solve_batch": (ctypes.c_int, [ctypes.POINTER(Problem), ctypes.c_int32, ctypes.POINTER(Options),
                                       _VP, _VP]),
    "wos_batch_autotune": (ctypes.c_int, [_VP, ctypes.c_char_p, ctypes.POINTER(BatchConfig)]),
    "wos_set_autotune_cache": (ctypes.c_int, [ctypes.c_char_p]),
    "wos_solve_noalloc": (ctypes.c_int, [_VP, ctypes.POINTER(Options), _VP, ctypes.c_int64, ctypes.c_int64,
                                         ctypes.c_double, ctypes.c_double, _VP, _VP, _VP, _VP]),
    "wos_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "wos_last_error": (ctypes.c_char_p, []),
    "wos_debug_weight_table": (ctypes.c_int, [ctypes.c_int32, ctypes.c_double, ctypes.c_int32, _PD, _PD]),
    "wos_debug_pointcloud_radius": (ctypes.c_int, [_VP, _VP, ctypes.c_int64, _VP, _VP]),
    "wos_debug_philox": (ctypes.c_int, [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int64, ctypes.c_uint32,
                                        ctypes.c_uint32, _VP, _VP]),
}

_lib = None
_lock = threading.Lock()


class WoSError(RuntimeError):
    def __init__(self, status, where, detail):
        super().__init__("%s: %s (%s)" % (where, detail, status))
        self.status = status


def load():
    """Loads libwos.so; raises if it has not been built (there is no fallback path)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError("libwos.so is not built: run paper_2406_01713_gb300.build.build() "
                                   "(nvcc, sm_103a); the library has no CPU fallback")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def check(status, where):
    if status != WOS_OK:
        L = load()
        detail = L.wos_last_error().decode(errors="replace")
        raise WoSError(status, where, detail or L.wos_status_string(status).decode())
