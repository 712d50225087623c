"""GB300-native Walk on Spheres for screened-Poisson path planning (arXiv 2406.01713).

The estimators run in libwos.so (hand-written sm_103a CUDA behind the C ABI in
include/wos.h); this package is the thin binding. `build()` compiles the library in-tree.
Importing the package does not load CUDA; the binding loads libwos.so on first use and
raises if it has not been built -- there is no CPU fallback.
"""
from . import synth  # noqa: F401  (input generators only)

__all__ = ["build", "Domain", "Batch", "WoSFunction", "backward", "set_autotune_cache", "synth"]


def build(force=False, verbose=False):
    from .build import build as _build

    return _build(force=force, verbose=verbose)


def __getattr__(name):
    if name in ("Domain", "Batch", "WoSFunction", "backward", "set_autotune_cache", "stats_dict", "plan_paths"):
        from . import wos

        return getattr(wos, name)
    raise AttributeError(name)
