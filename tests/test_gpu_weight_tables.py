"""The mixed-precision walkers' weight tables (log C_nu(z) and S_{nu+1}/S_nu(z), Sec. IV-A) sit on
one fixed grid in z, so a call's outputs depend on (domain, sigma, walks) only: not on which
tables earlier calls built, nor on whether the domain built them at creation (sigma_max)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2406_01713_gb300 import _lib, synth  # noqa: E402
from paper_2406_01713_gb300 import wos as W  # noqa: E402

KEYS = ("u", "u_se", "grad", "grad_se", "du_dsigma")


def _grad(D, w, sigma):
    r = D.grad(w["X"], 1024, w["eps"], sigma, seed=w["seed"])
    torch.cuda.synchronize()
    return r


@pytest.mark.parametrize("make", [synth.c1, lambda: synth.c5(n_queries=32, n_walks=1024)])
def test_outputs_do_not_depend_on_table_history(make):
    w = make()
    fresh = W.Domain(w["domain"])
    a = _grad(fresh, w, w["sigma"])
    used = W.Domain(w["domain"])
    _grad(used, w, 400.0 * w["sigma"] + 100.0)  # builds a larger table first
    b = _grad(used, w, w["sigma"])
    pre = W.Domain(w["domain"], sigma_max=1000.0)
    c = _grad(pre, w, w["sigma"])
    for k in KEYS:
        assert torch.equal(a[k], b[k]), k
        assert torch.equal(a[k], c[k]), k


def test_tables_on_other_streams_and_limits():
    w = synth.c1()
    D = W.Domain(w["domain"])
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):  # the table is built on this stream
        a = D.grad(w["X"], 512, w["eps"], w["sigma"], seed=1)
    b = D.grad(w["X"], 512, w["eps"], w["sigma"], seed=1)  # default stream: waits for that build
    torch.cuda.synchronize()
    for k in KEYS:
        assert torch.equal(a[k], b[k]), k
    with pytest.raises(_lib.WoSError):
        D.grad(w["X"], 16, w["eps"], 1e9)  # z beyond the largest table
    with pytest.raises(_lib.WoSError):
        W.Domain(w["domain"], sigma_max=-1.0)
    assert np.isfinite(D.grad(w["X"], 16, w["eps"], w["sigma"])["u"].cpu().numpy()).all()
