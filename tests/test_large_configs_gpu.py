"""The two large workloads at full size, FMM on the GPU, checked against the
FP64 oracle on sampled targets (each sample summed over all sources):
starfish k=50 (131 072 nodes, p=16, box order 70 on the finest level) and 200
ellipses in [0,100]^2 (2^20 nodes, k=20, 1e6 targets, double layer, p=16),
whose coarse boxes span hundreds of wavelengths and need the level-dependent
box orders. FP64 within 1e-10, mixed precision within 1e-6 of FP64 on every
target."""
import numpy as np
import pytest

from qbx_workloads import make_config

pytestmark = pytest.mark.gpu


def rel_l2(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b)))


@pytest.fixture(scope="module")
def qbxmod():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1602_05301_gb300 import build as b
    b.build()
    from paper_1602_05301_gb300 import qbx
    return qbx


@pytest.mark.parametrize("num,n_q,n_d", [(3, 12, 48), (5, 4, 16)])
def test_large_workload_sampled_parity(qbxmod, oracle, num, n_q, n_d):
    w = make_config(num)
    g = w["geom"]
    lp = qbxmod.LayerPotential(g.as_dict(), w["p"], sides=w["sides"])
    assoc = lp.build(w["tgt_xy"], w["on_surface_node"], w["on_surface_side"],
                     mode=qbxmod.QBX_FMM, p_fmm=w["p_fmm"])
    st = lp.stats()
    assert st["p_box"] == 70
    args = dict(sigma_S=w["sigma_S"], sigma_D=w["sigma_D"], cS=w["cS"], cD=w["cD"])
    u64 = lp.eval(precision=qbxmod.QBX_FP64, **args)
    u32 = lp.eval(precision=qbxmod.QBX_MIXED, **args)
    err_mixed = rel_l2(u32, u64)
    print("%s: boxes %d depth %d, mixed vs fp64 %.3e" % (w["name"], st["n_boxes"], st["depth"],
                                                        err_mixed))
    assert np.all(np.isfinite(u64)) and err_mixed < 1e-6
    rng = np.random.default_rng(num)
    qt = np.nonzero(assoc >= 0)[0]
    dt = np.nonzero(assoc < 0)[0]
    sample = np.concatenate([rng.choice(qt, n_q, replace=False),
                             rng.choice(dt, n_d, replace=False)])
    u_ref, _ = oracle.layer_potential(g.as_dict(), w["tgt_xy"][sample], w["p"], w["sigma_S"],
                                      w["sigma_D"], w["cS"], w["cD"], sides=w["sides"],
                                      centre_of_target=assoc[sample])
    err = rel_l2(u64[sample], u_ref)
    print("%s: fp64 vs oracle on %d samples %.3e" % (w["name"], sample.size, err))
    assert err < 1e-10
    lp.close()
