"""Failure detection without a GPU fault: a bounded device wait that runs out
(an mbarrier nothing completes, waited on with the deadline logic of the
tensor-core M2L kernels) is reported to the host as QBX_ERR_TIMEOUT, by
qbx_sync and by the next evaluation with host buffers, and the handle and the
CUDA context stay usable: the evaluations after it give the same bits."""
import numpy as np
import pytest

from qbx_workloads import discretise_curve, starfish
from qbx_workloads.configs import grid_targets

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qbxmod():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1602_05301_gb300 import build as b
    b.build()
    from paper_1602_05301_gb300 import qbx
    return qbx


def test_wait_timeout_reaches_the_host(qbxmod):
    g = discretise_curve(*starfish(0.3, 5), 64, 16, k=10.0)
    rng = np.random.default_rng(2)
    sig = rng.standard_normal(g.n) + 1j * rng.standard_normal(g.n)
    lp = qbxmod.LayerPotential(g.as_dict(), 8, sides=2)
    lp.build(grid_targets(40, -2.0, 2.0), mode=qbxmod.QBX_FMM, p_fmm=20, n_max=32)
    u0 = lp.eval(sigma_S=sig, cS=1.0)
    lp.sync()                                   # nothing pending
    lp.selftest_wait_timeout(2000)              # a 2 ms wait that runs out
    with pytest.raises(qbxmod.QBXError) as ei:
        lp.sync()
    assert ei.value.status == qbxmod.QBX_ERR_TIMEOUT
    lp.sync()                                   # the flag was cleared
    assert np.array_equal(lp.eval(sigma_S=sig, cS=1.0), u0)
    lp.selftest_wait_timeout(500)
    with pytest.raises(qbxmod.QBXError) as ei:  # a synchronous evaluation reports it
        lp.eval(sigma_S=sig, cS=1.0)
    assert ei.value.status == qbxmod.QBX_ERR_TIMEOUT
    assert np.array_equal(lp.eval(sigma_S=sig, cS=1.0), u0)
    lp.close()
