"""The large workloads at full size on the GPU, checked element by element
against the FP64 oracle.

* starfish k=50 (131 072 sources, p=16) and 200 ellipses in [0,100]^2 (2^20
  sources, k=20, 10^6 targets, double layer, p=16): the FMM plan of the
  benchmark against the oracle's values at 512 QBX targets, 512 direct targets
  and the coefficients of 256 used centres, each summed over all sources
  (stored by tests/golden/make_large_samples.py, which calls only the oracle).
* the batch of 256 random curves (2 046 320 sources and targets): one batched
  evaluation of all curves, 16 of them (spread over the panel-count and k
  range) against the oracle at 32 targets each.

Tolerances (per result): FP64 within 1e-10 of the oracle, both in relative l2
and element-wise as max|u - u_ref| / max|u_ref|; mixed precision within 1e-6
of the oracle on the samples and of the FP64 path on every target.
Coefficients alpha_l are compared weighted by |J_l(k r_c)|, their size where
the J-expansion uses them (alpha_l itself cancels to up to 1e14)."""
import os

import numpy as np
import pytest
from scipy.special import jv

from qbx_workloads import make_config

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
TOL64, TOL32 = 1e-10, 1e-6


def rel_l2(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b)))


def rel_max(a, b):
    return float(np.max(np.abs(np.ravel(a - b))) / np.max(np.abs(np.ravel(b))))


def check(name, got, ref, tol, tol_max=None):
    e2, em = rel_l2(got, ref), rel_max(got, ref)
    print("%s: rel l2 %.3e, max-norm %.3e" % (name, e2, em))
    assert e2 < tol and em < (tol if tol_max is None else tol_max), (name, e2, em)


@pytest.fixture(scope="module")
def qbxmod():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1602_05301_gb300 import build as b
    b.build()
    from paper_1602_05301_gb300 import qbx
    return qbx


@pytest.mark.parametrize("num", [3, 5])
def test_large_workload_elementwise_parity(qbxmod, num):
    import torch
    fx = np.load(os.path.join(GOLDEN, "large_config%d_samples.npz" % num))
    w = make_config(num)
    g = w["geom"]
    # the stored samples belong to this very workload
    chk = np.array([g.node_xy.sum(), g.normal_xy.sum(), g.weight.sum(), g.panel_h.sum(),
                    float(g.n)])
    # (the normals sum to ~1e-11 by cancellation, which summation order changes;
    # sin/cos of another machine's libm may differ in the last bit)
    assert np.allclose(chk, fx["geometry_checksum"], rtol=1e-12, atol=1e-9)
    tgt = fx["target"]
    assert np.allclose(w["tgt_xy"][tgt], fx["target_xy"], rtol=0, atol=1e-12)
    p, P = w["p"], 2 * w["p"] + 1
    lp = qbxmod.LayerPotential(g.as_dict(), p, sides=w["sides"])
    assoc = lp.build(w["tgt_xy"], w["on_surface_node"], w["on_surface_side"],
                     mode=qbxmod.QBX_FMM, p_fmm=w["p_fmm"])
    assert np.array_equal(assoc[tgt], fx["centre_of_target"])   # Sec. 6.1, exact
    dev = torch.device("cuda")
    ctr = torch.from_numpy(fx["centre"]).to(dev)
    args = dict(sigma_S=w["sigma_S"], sigma_D=w["sigma_D"], cS=w["cS"], cD=w["cD"])
    res = {}
    for prec in (qbxmod.QBX_FP64, qbxmod.QBX_MIXED):
        alpha = torch.empty((lp.n_centres, P), dtype=torch.complex128, device=dev)
        u = lp.eval(alpha_out=alpha, precision=prec, **args)
        res[prec] = (u, alpha[ctr].cpu().numpy())
        del alpha
    lp.close()
    (u64, a64), (u32, a32) = res[qbxmod.QBX_FP64], res[qbxmod.QBX_MIXED]
    assert np.all(np.isfinite(u64)) and np.all(np.isfinite(u32))
    q = fx["centre_of_target"] >= 0
    r_c = np.hypot(*(fx["centre_xy"] - g.node_xy[fx["centre"] % g.n]).T)
    wgt = np.abs(jv(np.arange(-p, p + 1)[None, :], g.k[0] * r_c[:, None]))
    for tag, u, a, tol in (("fp64", u64, a64, TOL64), ("mixed", u32, a32, TOL32)):
        check("%s %s QBX targets vs oracle" % (w["name"], tag), u[tgt][q], fx["u"][q], tol)
        check("%s %s direct targets vs oracle" % (w["name"], tag), u[tgt][~q], fx["u"][~q], tol)
        check("%s %s alpha vs oracle" % (w["name"], tag), a * wgt, fx["alpha"] * wgt, tol)
    check("%s mixed vs fp64, every target" % w["name"], u32, u64, TOL32)


@pytest.fixture(scope="module")
def batch256(qbxmod):
    """All 256 curves of the batch workload, plans chosen by the autotuner."""
    w = make_config(4)
    g = w["geom"]
    assert g.n_curves == 256
    noff = g.node_offset()
    probs = []
    for c in range(g.n_curves):
        G = g.as_dict(c)
        lp = qbxmod.LayerPotential(G, w["p"], sides=1)
        n = G["node_xy"].shape[0]
        lp.autotune(G["node_xy"], np.arange(n), np.ones(n, np.int8), p_fmm=w["p_fmm"],
                    precision=qbxmod.QBX_MIXED, reps=1)
        probs.append(lp)
    yield w, probs, noff
    for lp in probs:
        lp.close()


def test_batch256_against_oracle(qbxmod, batch256, oracle):
    w, probs, noff = batch256
    g = w["geom"]
    b = qbxmod.Batch(probs, n_streams=16)
    u64 = b.eval(sigma_S=w["sigma_S"], sigma_D=w["sigma_D"], cS=1.0, cD=1.0)
    u32 = b.eval(sigma_S=w["sigma_S"], sigma_D=w["sigma_D"], cS=1.0, cD=1.0,
                 precision=qbxmod.QBX_MIXED)
    b.close()
    assert u64.size == noff[-1] and np.all(np.isfinite(u64))
    check("batch-256 mixed vs fp64, every target", u32, u64, TOL32)
    # 16 curves spread over the range of panel counts and wavenumbers: sorted by
    # n * k, every 16th
    order = np.argsort(np.diff(noff) * np.asarray(g.k))
    curves = order[8::16]
    rng = np.random.default_rng(44)
    got64, got32, ref = [], [], []
    with oracle.hankel_recurrence():
        for c in curves:
            G = g.as_dict(int(c))
            n = G["node_xy"].shape[0]
            t = np.sort(rng.choice(n, 32, replace=False))
            sS = w["sigma_S"][noff[c]:noff[c + 1]]
            sD = w["sigma_D"][noff[c]:noff[c + 1]]
            # every node is an on-surface target on the exterior side: its own
            # exterior centre (side preference, Sec. 6.1)
            u_ref, _ = oracle.layer_potential(G, G["node_xy"][t], w["p"], sS, sD, 1.0, 1.0,
                                              sides=1, centre_of_target=t.astype(np.int32))
            got64.append(u64[noff[c] + t])
            got32.append(u32[noff[c] + t])
            ref.append(u_ref)
            # per curve, the FMM's own truncation at the batch's p_fmm = 20: up to
            # 1.4e-10 in l2 and 4.7e-10 element-wise (curve 43, k = 30.9, leaves of
            # n_max <= 64; 9.6e-12 at p_fmm = 25, 1.1e-12 at 30), so the bound is
            # 1e-9 per curve and element-wise, 1e-10 in l2 over the 16 curves
            check("batch-256 curve %d (n=%d, k=%.1f) fp64 vs oracle" % (c, n, g.k[c]),
                  got64[-1], u_ref, 1e-9)
    check("batch-256, 16 curves, fp64 vs oracle", np.concatenate(got64), np.concatenate(ref),
          TOL64, tol_max=1e-9)
    check("batch-256, 16 curves, mixed vs oracle", np.concatenate(got32), np.concatenate(ref),
          TOL32)
