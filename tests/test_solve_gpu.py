"""The sound-soft scattering problem of Sec. 8.3 solved with qbx_solve_dirichlet
(GMRES on (1/2) sigma + D* sigma + i k S* sigma = -u_inc, Global QBX for the
operator): against the Fourier-series solution on a circle, and on a starfish
against the FP64 oracle's own operator (the residual of the GPU's density)."""
import numpy as np
import pytest
from scipy.special import h1vp, hankel1, jv, jvp

from qbx_workloads import circle, discretise_curve, starfish
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


def plane_wave(k, phi, xy):
    return np.exp(1j * k * (xy[:, 0] * np.cos(phi) + xy[:, 1] * np.sin(phi)))


@pytest.mark.parametrize("mode,prec,tol", [("fmm", "fp64", 1e-11), ("direct", "fp64", 1e-11),
                                           ("fmm", "mixed", 1e-6)])
def test_circle_scattering_against_fourier_series(qbxmod, mode, prec, tol):
    """Unit circle, k = 5, plane wave from angle phi. Mode n of the density:
    sigma_n = -i^n J_n(k) e^{-in phi} / lam_n, lam_n = (i pi k/2) J_n'(k) H_n(k) +
    i k (i pi / 2) J_n(k) H_n(k) (exterior limit of D plus i k S on e^{int});
    the scattered field is -sum_n i^n J_n(k) H_n(kr) / H_n(k) e^{in(t - phi)}."""
    k, phi = 5.0, 0.3
    g = discretise_curve(*circle(1.0), 48, 16, k=k)
    lp = qbxmod.LayerPotential(g.as_dict(), 12, sides=1, q_src=64)
    m = qbxmod.QBX_FMM if mode == "fmm" else qbxmod.QBX_DIRECT
    pr = qbxmod.QBX_MIXED if prec == "mixed" else qbxmod.QBX_FP64
    sig, its, res = lp.solve_dirichlet(-plane_wave(k, phi, g.node_xy), mode=m, p_fmm=30,
                                       precision=pr, tol=tol, restart=60)
    print(mode, prec, "iterations", its, "residual %.2e" % res)
    assert res <= tol
    n = np.arange(-60, 61)
    lam = (1j * np.pi * k / 2) * jvp(n, k) * hankel1(n, k) + 1j * k * (1j * np.pi / 2) * jv(n, k) * hankel1(n, k)
    sn = -(1j ** n) * jv(n, k) * np.exp(-1j * n * phi) / lam
    t = g.param_t
    sig_exact = (sn[None, :] * np.exp(1j * n[None, :] * t[:, None])).sum(1)
    err = np.max(np.abs(sig - sig_exact)) / np.max(np.abs(sig_exact))
    print("density error %.2e" % err)
    assert err < (1e-9 if prec == "fp64" else 1e-5)
    # the scattered field off the curve from the solved density
    tg = np.array([[1.3, 0.2], [-2.0, 1.0], [0.1, -1.05], [3.0, 3.0]])
    lp.build(tg, mode=m, p_fmm=30)
    u = lp.eval(sigma_S=sig, sigma_D=sig, cS=1j * k, cD=1.0)
    lp.close()
    r, th = np.hypot(*tg.T), np.arctan2(tg[:, 1], tg[:, 0])
    u_exact = -((1j ** n)[None, :] * jv(n, k)[None, :] * hankel1(n[None, :], k * r[:, None])
                / hankel1(n, k)[None, :] * np.exp(1j * n[None, :] * (th[:, None] - phi))).sum(1)
    err_u = np.max(np.abs(u - u_exact)) / np.max(np.abs(u_exact))
    print("scattered field error %.2e" % err_u)
    assert err_u < (1e-9 if prec == "fp64" else 1e-5)


def test_starfish_solution_solves_the_oracle_operator(qbxmod, oracle):
    """GMRES with the direct and the FMM operator on a starfish (k = 10); the FP64
    oracle's own operator (direct Global QBX on its own 64-node source grid)
    applied to the GPU's density leaves the residual that the GPU reports (how
    fast GMRES converges is a property of the discretised operator; the
    residual of a given density is what the two must agree on)."""
    k, phi = 10.0, -0.7
    g = discretise_curve(*starfish(0.3, 5), 96, 16, k=k)
    f = -plane_wave(k, phi, g.node_xy)
    oxy, onr, ow = oracle.source_grid(g.node_xy, g.normal_xy, 16, 64)
    cxy, _ = oracle.centres(g.node_xy, g.normal_xy, g.panel_of_node, g.panel_h, 1)
    sols = []
    for mode in (qbxmod.QBX_DIRECT, qbxmod.QBX_FMM):
        lp = qbxmod.LayerPotential(g.as_dict(), 12, sides=1, q_src=64)
        sig, its, res = lp.solve_dirichlet(f, mode=mode, p_fmm=30, tol=1e-10, restart=100,
                                           max_iter=300)
        lp.close()
        os_ = oracle.interpolate_panels(sig, 16, 64)
        with oracle.hankel_recurrence():
            al = oracle.qbx_coefficients(oxy, onr, ow, k, cxy, 12, os_, os_, 1j * k, 1.0)
        Asig = oracle.qbx_evaluate(g.node_xy, np.arange(g.n, dtype=np.int32), cxy, al, 12, k)
        r = np.linalg.norm(Asig - f) / np.linalg.norm(f)
        print("starfish, mode %d: %d iterations, GPU residual %.3e, oracle residual %.3e"
              % (mode, its, res, r))
        assert res < 1e-6
        assert abs(r - res) < 1e-10 + 1e-3 * res
        sols.append(sig)
    # the two operators agree, so their GMRES iterates agree to the residual level
    assert np.linalg.norm(sols[0] - sols[1]) / np.linalg.norm(sols[0]) < 1e-6
