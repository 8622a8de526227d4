"""The library-made source grid (Sec. 2.2: density values on an oversampled
source grid by polynomial interpolation, q_src from Table 1) and the two-sided
on-surface operator (the mean of the two one-sided QBX limits, Sec. 2,
Eq. (oneside)), on the GPU:

* the source grid against the oracle's interpolation, element by element;
* the on-surface values of S and D on a circle against their closed forms,
  with no source grid supplied by the caller;
* Green's identity in its on-surface form D[u] - S[du/dn] = u/2, against the
  exact field and against the oracle's two-sided value, in direct and FMM plans.
Tolerance: 1e-10 relative (max-norm) in FP64."""
import numpy as np
import pytest
from scipy.special import h1vp, hankel1, jv, jvp

from qbx_workloads import circle, discretise_curve, starfish
from tests.fields import PointSourceField

pytestmark = pytest.mark.gpu

TOL64 = 1e-10


def rel_max(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.fixture(scope="module")
def qbxmod():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1602_05301_gb300 import build as b
    b.build()
    from paper_1602_05301_gb300 import qbx
    return qbx


def test_library_source_grid_matches_oracle(qbxmod, oracle):
    g = discretise_curve(*starfish(0.3, 5), 40, 16, k=5.0)
    q_src = qbxmod.qbx_table1_q_src(16, 1e-12)
    assert q_src == 64
    lp = qbxmod.LayerPotential(g.as_dict(), 8, sides=2, q_src=q_src)
    xy, nr, w = lp.source_grid()
    lp.close()
    oxy, onr, ow = oracle.source_grid(g.node_xy, g.normal_xy, 16, q_src)
    # positions are sums of O(1) terms; tangents (normals, weights) come from the
    # differentiated interpolant, whose entries reach ~q^2 and cancel down to the
    # panel half-length |dx/du| ~ 1e-2 here: rounding up to ~1e-12 relative
    assert np.abs(xy - oxy).max() < 1e-13
    assert np.abs(nr - onr).max() < 1e-10
    assert np.abs(w - ow).max() < 1e-10 * ow.max()


@pytest.mark.parametrize("mode", ["direct", "fmm"])
def test_circle_on_surface_closed_forms(qbxmod, mode):
    """S[e^{3it}] and D[e^{3it}] at the nodes of the unit circle (k = 1, 32 panels
    x 16 nodes): the two-sided value is (i pi R/2) J_3(kR) H_3(kR) for S and the
    mean of the exterior and interior limits, (i pi k R/4)(J_3'(kR) H_3(kR) +
    J_3(kR) H_3'(kR)), for D; the library makes the 64-node source grid."""
    k, R, n = 1.0, 1.0, 3
    g = discretise_curve(*circle(R), 32, 16, k=k)
    sig = np.exp(1j * n * g.param_t)
    tgt = g.node_xy
    on_node = np.arange(g.n)
    on_side = np.zeros(g.n, np.int8)                      # on-surface value
    lp = qbxmod.LayerPotential(g.as_dict(), 12, sides=2, q_src=64)
    m = qbxmod.QBX_FMM if mode == "fmm" else qbxmod.QBX_DIRECT
    assoc = lp.build(tgt, on_node, on_side, mode=m, p_fmm=30, n_max=32)
    assert np.array_equal(assoc, on_node)                 # the exterior centre is reported
    uS = lp.eval(sigma_S=sig, cS=1.0)
    uD = lp.eval(sigma_D=sig, cS=0.0, cD=1.0)
    lp.close()
    S_exact = 1j * np.pi * R / 2 * jv(n, k * R) * hankel1(n, k * R) * sig
    D_exact = 1j * np.pi * k * R / 4 * (jvp(n, k * R) * hankel1(n, k * R)
                                        + jv(n, k * R) * h1vp(n, k * R)) * sig
    print(mode, "S", rel_max(uS, S_exact), "D", rel_max(uD, D_exact))
    assert rel_max(uS, S_exact) < TOL64
    assert rel_max(uD, D_exact) < TOL64


@pytest.mark.parametrize("mode", ["direct", "fmm"])
def test_greens_identity_on_surface_half(qbxmod, oracle, mode):
    """D[u] - S[du/dn] = u/2 on the curve for u radiated by two points inside a
    starfish (k = 5, 48 panels x 16), densities given on the density grid."""
    k = 5.0
    f = PointSourceField(k, [[0.1, 0.2], [-0.3, -0.1]], [1.0 + 0.5j, -0.7 + 0.2j])
    g = discretise_curve(*starfish(0.3, 5), 48, 16, k=k)
    sD = f.u(g.node_xy)
    sS = f.dudn(g.node_xy, g.normal_xy)
    tgt = g.node_xy
    on_node = np.arange(g.n)
    lp = qbxmod.LayerPotential(g.as_dict(), 12, sides=2, q_src=64)
    m = qbxmod.QBX_FMM if mode == "fmm" else qbxmod.QBX_DIRECT
    lp.build(tgt, on_node, np.zeros(g.n, np.int8), mode=m, p_fmm=30, n_max=32)
    u = lp.eval(sigma_S=sS, sigma_D=sD, cS=-1.0, cD=1.0)
    # the one-sided limits on the same plan: exterior u, interior 0
    lp.build(np.concatenate([tgt, tgt]), np.concatenate([on_node, on_node]),
             np.concatenate([np.ones(g.n, np.int8), -np.ones(g.n, np.int8)]), mode=m,
             p_fmm=30, n_max=32)
    u2 = lp.eval(sigma_S=sS, sigma_D=sD, cS=-1.0, cD=1.0)
    lp.close()
    ue = f.u(tgt)
    assert rel_max(u, 0.5 * ue) < TOL64
    assert rel_max(u2[:g.n], ue) < TOL64
    assert np.max(np.abs(u2[g.n:])) < TOL64 * np.max(np.abs(ue))
    assert rel_max(u, 0.5 * (u2[:g.n] + u2[g.n:])) < 1e-13
    # the oracle's two-sided value on its own interpolated source grid
    oxy, onr, ow = oracle.source_grid(g.node_xy, g.normal_xy, 16, 64)
    oS = oracle.interpolate_panels(sS, 16, 64)
    oD = oracle.interpolate_panels(sD, 16, 64)
    cxy, _ = oracle.centres(g.node_xy, g.normal_xy, g.panel_of_node, g.panel_h, 2)
    with oracle.hankel_recurrence():
        al = oracle.qbx_coefficients(oxy, onr, ow, k, cxy, 12, oS, oD, -1.0, 1.0)
    ext = oracle.qbx_evaluate(tgt, on_node.astype(np.int32), cxy, al, 12, k)
    inn = oracle.qbx_evaluate(tgt, (g.n + on_node).astype(np.int32), cxy, al, 12, k)
    assert rel_max(u, 0.5 * (ext + inn)) < TOL64


def test_two_sided_needs_both_centre_sides(qbxmod):
    g = discretise_curve(*circle(1.0), 16, 16, k=1.0)
    lp = qbxmod.LayerPotential(g.as_dict(), 6, sides=1, q_src=32)
    with pytest.raises(qbxmod.QBXError):
        lp.build(g.node_xy[:4], np.arange(4), np.zeros(4, np.int8))
    lp.close()
