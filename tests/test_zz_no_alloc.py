"""The allocation-free entry point qbx_direct_qbx_eval_noalloc, called through the C ABI.

It serves callers that cannot allocate device memory (their HBM is owned by
their own pool allocator, or their loop cannot take the synchronisation a
cudaMalloc may bring). Its result must match qbx_layer_potential_eval in
QBX_DIRECT mode on the same targets and centres, on two calls in a row (the
second call reuses the static scratch that the first one left behind). This
file is collected last so that a failure here never hides another test.
"""
import ctypes

import numpy as np
import pytest

from qbx_workloads import discretise_curve, starfish

pytestmark = pytest.mark.gpu


def _setup():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1602_05301_gb300 import build as b
    b.build()
    from paper_1602_05301_gb300 import qbx
    lib = qbx.library()
    f = lib.qbx_direct_qbx_eval_noalloc
    f.restype = ctypes.c_int
    vp, d, i64 = ctypes.c_void_p, ctypes.c_double, ctypes.c_int64
    f.argtypes = [i64, vp, vp, vp, d, d, d, vp, d, d, vp, i64, vp, ctypes.c_int32, i64, vp, vp,
                  vp, vp]
    return torch, qbx, lib


def test_noalloc_matches_direct_eval_twice():
    torch, qbx, lib = _setup()
    k, p = 6.0, 10
    g = discretise_curve(*starfish(0.25, 4), 40, 12, k=k)     # 480 nodes, 960 centres
    rng = np.random.default_rng(21)
    n = g.n
    # every node on both sides plus a few off-surface targets near exterior centres
    tgt = np.concatenate([g.node_xy, g.node_xy])
    on_node = np.concatenate([np.arange(n), np.arange(n)])
    on_side = np.concatenate([np.ones(n, np.int8), -np.ones(n, np.int8)])
    lp = qbx.LayerPotential(g.as_dict(), p, sides=2)
    assoc = lp.build(tgt, on_node, on_side, mode=qbx.QBX_DIRECT)
    assert np.all(assoc >= 0)
    dev = torch.device("cuda")
    t64 = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(dev)
    sxy, snr, sw = t64(g.node_xy), t64(g.normal_xy), t64(g.weight)
    cxy_h = np.concatenate([g.node_xy + 0.5 * g.panel_h[g.panel_of_node, None] * g.normal_xy,
                            g.node_xy - 0.5 * g.panel_h[g.panel_of_node, None] * g.normal_xy])
    cxy = t64(cxy_h)
    txy = t64(tgt)
    tc = torch.from_numpy(assoc.astype(np.int32)).to(dev)
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        sS = rng.standard_normal(n) + 1j * rng.standard_normal(n)
        sD = rng.standard_normal(n) + 1j * rng.standard_normal(n)
        cS, cD = complex(0.3 + call, -0.7), complex(1.0, 0.25 * call)
        ref = lp.eval(sigma_S=sS, sigma_D=sD, cS=cS, cD=cD)
        dS = torch.from_numpy(sS).to(dev)
        dD = torch.from_numpy(sD).to(dev)
        out = torch.full((tgt.shape[0],), complex("nan"), dtype=torch.complex128, device=dev)
        st = lib.qbx_direct_qbx_eval_noalloc(
            n, sxy.data_ptr(), snr.data_ptr(), sw.data_ptr(), k, cS.real, cS.imag,
            dS.data_ptr(), cD.real, cD.imag, dD.data_ptr(), 2 * n, cxy.data_ptr(), p,
            tgt.shape[0], txy.data_ptr(), tc.data_ptr(), out.data_ptr(), stream)
        assert st == 0, lib.qbx_last_error()
        torch.cuda.synchronize()
        u = out.cpu().numpy()
        assert np.linalg.norm(u - ref) / np.linalg.norm(ref) < 1e-10
    lp.close()


def test_noalloc_rejects_oversize_and_host_memory():
    torch, qbx, lib = _setup()
    dev = torch.device("cuda")
    x = torch.zeros(16, dtype=torch.float64, device=dev)
    c = torch.zeros(8, dtype=torch.complex128, device=dev)
    big = 1 << 19
    st = lib.qbx_direct_qbx_eval_noalloc(big, x.data_ptr(), x.data_ptr(), x.data_ptr(), 1.0, 1.0,
                                         0.0, c.data_ptr(), 0.0, 0.0, None, 4, x.data_ptr(), 4, 0,
                                         None, None, None, None)
    assert st == qbx.QBX_ERR_ARG
    assert b"scratch" in lib.qbx_last_error()
    h = np.zeros(16)
    st = lib.qbx_direct_qbx_eval_noalloc(4, h.ctypes.data, x.data_ptr(), x.data_ptr(), 1.0, 1.0,
                                         0.0, c.data_ptr(), 0.0, 0.0, None, 2, x.data_ptr(), 2, 0,
                                         None, None, None, None)
    assert st == qbx.QBX_ERR_ARG
    assert b"device memory" in lib.qbx_last_error()
