"""The allocation-free estimate, wos_solve_noalloc, against wos_solve through the C ABI.

Some callers cannot allocate device memory inside a call: a control loop with a hard deadline
(cudaMalloc/cudaFree can block on the driver's allocator and synchronise the device) or an
application that has handed all device memory to its own pool. They call wos_solve_noalloc,
whose per-query sums live in a static device array instead of freshly allocated scratch. It
must give what wos_solve gives, and must do so on two calls in a row: the array keeps the
previous call's contents, so every call has to clear what starts at zero.
This file is collected last so that a run stopping at its first failure has run every other
test before it.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2406_01713_gb300 import _lib, synth  # noqa: E402
from paper_2406_01713_gb300 import wos as W  # noqa: E402

VP = ctypes.c_void_p


def _call(fn, dom, opts, X, N, eps, sigma):
    Q = X.shape[0]
    u = torch.full((Q,), float("nan"), dtype=torch.float64, device="cuda")
    se = torch.full((Q,), float("nan"), dtype=torch.float64, device="cuda")
    st = torch.zeros(len(_lib.STATS_FIELDS), dtype=torch.int64, device="cuda")
    stream = VP(torch.cuda.current_stream().cuda_stream)
    rc = fn(dom.h, ctypes.byref(opts), VP(X.data_ptr()), Q, N, eps, sigma, VP(u.data_ptr()),
            VP(se.data_ptr()), VP(st.data_ptr()), stream)
    _lib.check(rc, fn.__name__)
    torch.cuda.synchronize()
    return u.cpu().numpy(), se.cpu().numpy(), st.cpu().numpy()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_noalloc_matches_wos_solve_on_two_calls(precision):
    L = _lib.load()
    w = synth.c1(n_queries=64, n_walks=3000)
    dom = W.Domain(w["domain"])
    X = torch.tensor(w["X"], dtype=torch.float64, device="cuda")
    opts = W._opts(precision, w["seed"])
    args = (dom, opts, X, w["n_walks"], w["eps"], w["sigma"])
    u0, se0, st0 = _call(L.wos_solve, *args)
    for _ in range(2):
        u1, se1, st1 = _call(L.wos_solve_noalloc, *args)
        assert np.array_equal(st1[:4], st0[:4])  # walks, walk-steps, capped, outside: exact
        if precision == "fp64":
            # same walks; only the order of the FP64 atomic additions differs
            assert np.allclose(u1, u0, rtol=1e-10, atol=1e-12)
            assert np.allclose(se1, se0, rtol=1e-6, atol=1e-12)
        else:
            assert np.all(np.abs(u1 - u0) <= 4 * np.sqrt(se1 ** 2 + se0 ** 2) + 1e-4)
            assert np.allclose(u1, u0, rtol=1e-5, atol=1e-7)


def test_noalloc_rejects_what_it_cannot_hold():
    L = _lib.load()
    w = synth.c1(n_queries=4, n_walks=100)
    dom = W.Domain(w["domain"])
    big = torch.zeros((200_000, 2), dtype=torch.float64, device="cuda")  # needs 12.8 MB > 1 MiB
    with pytest.raises(_lib.WoSError) as e:
        _call(L.wos_solve_noalloc, dom, W._opts("fp64", 1), big, 10, 1e-3, 4.0)
    assert e.value.status == 1 and "static array" in str(e.value)
    X = torch.tensor(w["X"], dtype=torch.float64, device="cuda")
    with pytest.raises(_lib.WoSError) as e:
        _call(L.wos_solve_noalloc, dom, W._opts("mixed", 1), X, 10, 1e-3, 4.0)
    assert e.value.status == 2
