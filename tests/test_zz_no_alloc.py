"""The allocation-free entry point qbx_direct_qbx_eval_noalloc, called through the C ABI.

It serves callers that cannot allocate device memory: applications whose GPU
memory is all handed out in advance by their own pool allocator, or loops that
cannot take the device-wide synchronisation a cudaMalloc may bring. Its result
must match the FP64 oracle and qbx_layer_potential_eval in QBX_DIRECT mode on
the same targets and centres, on two calls in a row (the second call reuses
the static scratch that the first one left behind). This file is collected last
so that a failure here never hides another test.
"""
import ctypes

import numpy as np
import pytest

from qbx_workloads import discretise_curve, starfish

pytestmark = pytest.mark.gpu

TOL64 = 1e-10


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


def _problem(torch, k=6.0):
    g = discretise_curve(*starfish(0.25, 4), 40, 12, k=k)     # 480 nodes, 960 centres
    n = g.n
    # every node on both sides (its own centre on each side)
    tgt = np.concatenate([g.node_xy, g.node_xy])
    on_node = np.concatenate([np.arange(n), np.arange(n)])
    on_side = np.concatenate([np.ones(n, np.int8), -np.ones(n, np.int8)])
    cxy_h = np.concatenate([g.node_xy + 0.5 * g.panel_h[g.panel_of_node, None] * g.normal_xy,
                            g.node_xy - 0.5 * g.panel_h[g.panel_of_node, None] * g.normal_xy])
    dev = torch.device("cuda")
    t64 = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(dev)
    bufs = dict(sxy=t64(g.node_xy), snr=t64(g.normal_xy), sw=t64(g.weight), cxy=t64(cxy_h),
                txy=t64(tgt))
    return g, tgt, on_node, on_side, bufs


def _call(lib, torch, g, bufs, k, p, cS, cD, dS, dD, n_tgt, tc):
    out = torch.full((n_tgt,), complex("nan"), dtype=torch.complex128, device="cuda")
    st = lib.qbx_direct_qbx_eval_noalloc(
        g.n, bufs["sxy"].data_ptr(), bufs["snr"].data_ptr(), bufs["sw"].data_ptr(), k,
        cS.real, cS.imag, None if dS is None else dS.data_ptr(), cD.real, cD.imag,
        None if dD is None else dD.data_ptr(), 2 * g.n, bufs["cxy"].data_ptr(), p, n_tgt,
        bufs["txy"].data_ptr(), tc.data_ptr(), out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert st == 0, lib.qbx_last_error()
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_noalloc_matches_oracle_and_direct_eval_twice(oracle):
    torch, qbx, lib = _setup()
    k, p = 6.0, 10
    g, tgt, on_node, on_side, bufs = _problem(torch, k)
    n = g.n
    rng = np.random.default_rng(21)
    lp = qbx.LayerPotential(g.as_dict(), p, sides=2)
    assoc = lp.build(tgt, on_node, on_side, mode=qbx.QBX_DIRECT)
    assert np.all(assoc >= 0)
    tc = torch.from_numpy(assoc.astype(np.int32)).cuda()
    for call in range(2):
        sS = rng.standard_normal(n) + 1j * rng.standard_normal(n)
        sD = rng.standard_normal(n) + 1j * rng.standard_normal(n)
        cS, cD = complex(0.3 + call, -0.7), complex(1.0, 0.25 * call)
        ref = lp.eval(sigma_S=sS, sigma_D=sD, cS=cS, cD=cD)
        u_ref, _ = oracle.layer_potential(g.as_dict(), tgt, p, sS, sD, cS, cD, sides=2,
                                          centre_of_target=assoc)
        u = _call(lib, torch, g, bufs, k, p, cS, cD, torch.from_numpy(sS).cuda(),
                  torch.from_numpy(sD).cuda(), tgt.shape[0], tc)
        assert np.linalg.norm(u - ref) / np.linalg.norm(ref) < TOL64
        assert np.linalg.norm(u - u_ref) / np.linalg.norm(u_ref) < TOL64
        assert np.max(np.abs(u - u_ref)) < TOL64 * np.max(np.abs(u_ref))
    lp.close()


@pytest.mark.parametrize("p", [4, 16])
@pytest.mark.parametrize("layer", ["S", "D"])
def test_noalloc_single_layer_vs_oracle(oracle, p, layer):
    torch, qbx, lib = _setup()
    k = 6.0
    g, tgt, on_node, on_side, bufs = _problem(torch, k)
    n = g.n
    rng = np.random.default_rng(22 + p)
    sig = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    assoc = np.concatenate([np.arange(n), n + np.arange(n)]).astype(np.int32)
    # targets with an out-of-range centre index (past the end, or -1) come back NaN
    bad = np.array([17, 18])
    tc_h = assoc.copy()
    tc_h[bad] = [2 * n, -1]
    tc = torch.from_numpy(tc_h).cuda()
    sS = torch.from_numpy(sig).cuda() if layer == "S" else None
    sD = torch.from_numpy(sig).cuda() if layer == "D" else None
    cS, cD = complex(0.0, k), complex(1.0, 0.0)
    u = _call(lib, torch, g, bufs, k, p, cS, cD, sS, sD, tgt.shape[0], tc)
    assert np.all(np.isnan(u[bad].real)) and np.all(np.isnan(u[bad].imag))
    ok = ~np.isin(np.arange(tgt.shape[0]), bad)
    u_ref, _ = oracle.layer_potential(g.as_dict(), tgt[ok], p,
                                      sig if layer == "S" else None,
                                      sig if layer == "D" else None, cS, cD, sides=2,
                                      centre_of_target=assoc[ok])
    assert np.linalg.norm(u[ok] - u_ref) / np.linalg.norm(u_ref) < TOL64
    assert np.max(np.abs(u[ok] - u_ref)) < TOL64 * np.max(np.abs(u_ref))


def test_noalloc_rejects_oversize_and_foreign_memory():
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
    # sizes whose product would overflow a signed 64-bit count are refused too
    st = lib.qbx_direct_qbx_eval_noalloc(4, x.data_ptr(), x.data_ptr(), x.data_ptr(), 1.0, 1.0,
                                         0.0, c.data_ptr(), 0.0, 0.0, None, (1 << 62) // 3,
                                         x.data_ptr(), 16, 0, None, None, None, None)
    assert st == qbx.QBX_ERR_ARG
    assert b"scratch" in lib.qbx_last_error()
    h = np.zeros(16)
    st = lib.qbx_direct_qbx_eval_noalloc(4, h.ctypes.data, x.data_ptr(), x.data_ptr(), 1.0, 1.0,
                                         0.0, c.data_ptr(), 0.0, 0.0, None, 2, x.data_ptr(), 2, 0,
                                         None, None, None, None)
    assert st == qbx.QBX_ERR_ARG
    assert b"src_xy must be device memory" in lib.qbx_last_error()
    if torch.cuda.device_count() > 1:
        # memory of another GPU is refused before any launch
        y = torch.zeros(16, dtype=torch.float64, device=torch.device("cuda", 1))
        st = lib.qbx_direct_qbx_eval_noalloc(4, x.data_ptr(), y.data_ptr(), x.data_ptr(), 1.0,
                                             1.0, 0.0, c.data_ptr(), 0.0, 0.0, None, 2,
                                             x.data_ptr(), 2, 0, None, None, None, None)
        assert st == qbx.QBX_ERR_ARG
        assert b"src_normal_xy must be device memory on the current device" in \
            lib.qbx_last_error()
