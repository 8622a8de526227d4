"""Pins for the FP64 CPU oracle: checks against closed forms, Green's identity,
mpmath brute force, Graf's addition theorem and invariants. None of these
re-types the oracle's own formulas; each would fail on a dropped term, a wrong
sign or index, or a transposed operand in the oracle."""
import numpy as np
import pytest
from scipy.special import hankel1 as sp_hankel1
from scipy.special import jv as sp_jv

from qbx_workloads import circle, discretise_curve, make_config, starfish
from tests.fields import PointSourceField, circle_dlp_mode, circle_slp_mode


def _rel(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


# ---------------------------------------------------------------- special functions
def test_library_bessel_vs_scipy(oracle):
    x = np.concatenate([np.linspace(0.05, 3, 25), np.linspace(3.5, 60, 25)])
    for l in list(range(-20, 21)):
        j = oracle.bessel_j(l, x)
        h = oracle.hankel1(l, x)
        habs = np.abs(sp_hankel1(l, x))
        # both libraries carry ~1e-15 absolute error near the zeros of J at large x
        assert np.all(np.abs(j - sp_jv(l, x)) <= 1e-13 * habs + 1e-12 * np.abs(sp_jv(l, x)))
        assert np.all(np.abs(h - sp_hankel1(l, x)) <= 1e-12 * habs)


def test_library_bessel_vs_mpmath(oracle):
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 30
    for l, x in [(0, 0.01), (1, 0.3), (-3, 1.0), (7, 2.5), (-12, 0.8), (16, 40.0), (25, 5.0)]:
        hj = complex(mpmath.hankel1(l, x))
        jj = float(mpmath.besselj(l, x))
        assert abs(oracle.hankel1(l, [x])[0] - hj) <= 1e-13 * abs(hj)
        # J is checked against the scale |H_l(x)|: ~1e-15 absolute error near J's zeros
        assert abs(oracle.bessel_j(l, [x])[0] - jj) <= 1e-13 * abs(hj)


def test_hankel_recurrence_vs_mpmath_and_library(oracle):
    """The optional Hankel tables of the QBX coefficients (H_0, H_1 from the library,
    then the upward recurrence) against mpmath at 30 digits, from tiny to large
    arguments, and the coefficients they give against the per-order library calls."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 30
    x = np.array([1e-3, 0.05, 0.7, 3.0, 17.3, 250.0, 2900.0])
    with oracle.hankel_recurrence():
        h = oracle.hankel_table(18, x)
    for i, xi in enumerate(x):
        ref = np.array([complex(mpmath.hankel1(m, mpmath.mpf(xi))) for m in range(19)])
        # libstdc++'s H_0, H_1 carry ~2e-13 relative error at x in the hundreds
        assert np.max(np.abs(h[i] - ref) / np.abs(ref)) < 1e-12, xi
    h_lib = oracle.hankel_table(18, x)          # default: one library call per order
    assert np.max(np.abs(h - h_lib) / np.abs(h_lib)) < 1e-12
    g = discretise_curve(*starfish(0.3, 5), 24, 16, k=10.0)
    rng = np.random.default_rng(30)
    sS = rng.standard_normal(g.n) + 1j * rng.standard_normal(g.n)
    sD = rng.standard_normal(g.n) + 1j * rng.standard_normal(g.n)
    cxy, crad = oracle.centres(g.node_xy, g.normal_xy, g.panel_of_node, g.panel_h, 2)
    cs = cxy[::37]
    a0 = oracle.qbx_coefficients(g.node_xy, g.normal_xy, g.weight, 10.0, cs, 12, sS, sD, 1j, 1.0)
    with oracle.hankel_recurrence():
        a1 = oracle.qbx_coefficients(g.node_xy, g.normal_xy, g.weight, 10.0, cs, 12, sS, sD,
                                     1j, 1.0)
    assert not oracle._load().oracle_hankel_recurrence()   # the context restored the default
    wgt = np.abs(sp_jv(np.arange(-12, 13)[None, :], 10.0 * crad[::37][:, None]))
    assert _rel(a1 * wgt, a0 * wgt) < 1e-12


# ---------------------------------------------------------------- source grid (Sec. 2.2)
def test_source_grid_interpolation_matches_the_curve(oracle):
    """The source grid made from the density grid alone (positions, normals and
    weights by per-panel polynomial interpolation) equals the curve's own
    discretisation with q_src nodes, and interpolated densities equal the density
    sampled there (a smooth curve: exact to rounding)."""
    g = discretise_curve(*starfish(0.3, 5), 48, 16, k=5.0)
    gs = discretise_curve(*starfish(0.3, 5), 48, 64, k=5.0)
    xy, nr, w = oracle.source_grid(g.node_xy, g.normal_xy, 16, 64)
    assert np.abs(xy - gs.node_xy).max() < 1e-13
    assert np.abs(nr - gs.normal_xy).max() < 1e-11
    assert np.abs(w - gs.weight).max() < 1e-12 * gs.weight.max()
    assert abs(w.sum() - gs.weight.sum()) < 1e-12 * gs.weight.sum()
    f = lambda t: np.exp(3j * t) + 0.5 * np.cos(7 * t)
    assert np.abs(oracle.interpolate_panels(f(g.param_t), 16, 64) - f(gs.param_t)).max() < 1e-13
    # a polynomial of degree < q in the panel variable is reproduced exactly on a
    # straight panel (the interpolation is exact there)
    x16, _ = np.polynomial.legendre.leggauss(16)
    x64, _ = np.polynomial.legendre.leggauss(64)
    poly = lambda u: 1 - 2 * u + 3 * u ** 5 - u ** 15
    assert np.abs(oracle.interpolate_panels(poly(x16), 16, 64) - poly(x64)).max() < 1e-12


# ---------------------------------------------------------------- Graf / conventions
def test_graf_expansion_single_source_slp(oracle):
    """alpha of one unit source, evaluated inside the disk, equals (i/4) H_0(k|x-y|)."""
    k = 3.0
    y = np.array([[0.9, -0.4]])
    c = np.array([[0.1, 0.2]])
    rng = np.random.default_rng(1)
    ang = rng.uniform(0, 2 * np.pi, 40)
    rad = rng.uniform(0, 0.35, 40)
    x = c + np.stack([rad * np.cos(ang), rad * np.sin(ang)], -1)
    al = oracle.qbx_coefficients(y, np.array([[1.0, 0.0]]), np.ones(1), k, c, 40,
                                 sigma_S=np.ones(1))
    u = oracle.qbx_evaluate(x, np.zeros(40, np.int32), c, al, 40, k)
    r = np.hypot(*(x - y).T)
    ref = 0.25j * sp_hankel1(0, k * r)
    assert _rel(u, ref) < 1e-13


def test_graf_expansion_single_source_dlp(oracle):
    """alpha of one unit dipole (normal n) equals (i/4) k H_1(kr) n.(x-y)/r inside the disk."""
    k = 2.0
    y = np.array([[-0.7, 0.5]])
    nrm = np.array([[0.6, 0.8]])
    c = np.array([[0.0, 0.0]])
    rng = np.random.default_rng(2)
    ang = rng.uniform(0, 2 * np.pi, 40)
    rad = rng.uniform(0, 0.3, 40)
    x = np.stack([rad * np.cos(ang), rad * np.sin(ang)], -1)
    al = oracle.qbx_coefficients(y, nrm, np.ones(1), k, c, 40, sigma_D=np.ones(1), cS=0, cD=1)
    u = oracle.qbx_evaluate(x, np.zeros(40, np.int32), c, al, 40, k)
    d = x - y
    r = np.hypot(*d.T)
    ref = 0.25j * k * sp_hankel1(1, k * r) * (d @ nrm[0]) / r
    assert _rel(u, ref) < 1e-12
    ud = oracle.direct_potential(y, nrm, np.ones(1), k, x, sigma_D=np.ones(1), cS=0, cD=1)
    assert _rel(ud, ref) < 1e-13


def test_alpha_tiny_vs_mpmath(oracle):
    """Brute-force alpha for 5 sources / 2 centres at 30 digits; the double-layer part
    differentiates the Graf kernel numerically along the normal (mpmath.diff)."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 30
    rng = np.random.default_rng(3)
    k, p = 4.0, 4
    src = rng.uniform(-1, 1, (5, 2))
    th = rng.uniform(0, 2 * np.pi, 5)
    nrm = np.stack([np.cos(th), np.sin(th)], -1)
    w = rng.uniform(0.1, 0.3, 5)
    sS = rng.standard_normal(5) + 1j * rng.standard_normal(5)
    sD = rng.standard_normal(5) + 1j * rng.standard_normal(5)
    cS, cD = 0.3 - 1.1j, 0.7 + 0.2j
    ctr = np.array([[1.6, 1.5], [-1.7, 1.4]])
    got = oracle.qbx_coefficients(src, nrm, w, k, ctr, p, sigma_S=sS, sigma_D=sD, cS=cS, cD=cD)

    def wave(l, sx, sy, cx, cy):
        dx, dy = sx - cx, sy - cy
        r = mpmath.sqrt(dx * dx + dy * dy)
        return mpmath.hankel1(l, k * r) * mpmath.expj(l * mpmath.atan2(dy, dx))

    for ci in range(2):
        for l in range(-p, p + 1):
            acc = mpmath.mpc(0)
            for j in range(5):
                sx, sy = mpmath.mpf(src[j, 0]), mpmath.mpf(src[j, 1])
                cx, cy = mpmath.mpf(ctr[ci, 0]), mpmath.mpf(ctr[ci, 1])
                s_term = wave(l, sx, sy, cx, cy)
                d_term = mpmath.diff(lambda e: wave(l, sx + e * nrm[j, 0], sy + e * nrm[j, 1],
                                                    cx, cy), 0)
                acc += w[j] * (cS * sS[j] * s_term + cD * sD[j] * d_term)
            ref = complex(0.25j * acc)
            assert abs(got[ci, l + p] - ref) <= 1e-12 * abs(ref) + 1e-15


def test_direct_tiny_vs_mpmath(oracle):
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 30
    rng = np.random.default_rng(4)
    k = 7.0
    src = rng.uniform(-1, 1, (4, 2))
    th = rng.uniform(0, 2 * np.pi, 4)
    nrm = np.stack([np.cos(th), np.sin(th)], -1)
    w = rng.uniform(0.1, 0.3, 4)
    sS = rng.standard_normal(4) + 1j * rng.standard_normal(4)
    sD = rng.standard_normal(4) + 1j * rng.standard_normal(4)
    tgt = rng.uniform(2, 3, (3, 2))
    got = oracle.direct_potential(src, nrm, w, k, tgt, sigma_S=sS, sigma_D=sD, cS=1.5, cD=-0.5j)
    for t in range(3):
        acc = mpmath.mpc(0)
        for j in range(4):
            def G(sx, sy):
                r = mpmath.sqrt((tgt[t, 0] - sx) ** 2 + (tgt[t, 1] - sy) ** 2)
                return mpmath.hankel1(0, k * r)
            sx, sy = mpmath.mpf(src[j, 0]), mpmath.mpf(src[j, 1])
            dG = mpmath.diff(lambda e: G(sx + e * nrm[j, 0], sy + e * nrm[j, 1]), 0)
            acc += w[j] * (1.5 * sS[j] * G(sx, sy) + (-0.5j) * sD[j] * dG)
        ref = complex(0.25j * acc)
        assert abs(got[t] - ref) <= 1e-13 * abs(ref)


# ---------------------------------------------------------------- closed forms on the circle
def test_circle_slp_closed_form(oracle):
    """S[cos 3t] on the unit circle (k=1): direct quadrature off the curve and the
    on-surface QBX limit (oversampled sources), converging geometrically in p."""
    w = make_config(1)
    g = w["geom"]
    G = g.as_dict()
    exact = 0.5 * (circle_slp_mode(3, 1.0, 1.0, w["tgt_xy"])
                   + circle_slp_mode(-3, 1.0, 1.0, w["tgt_xy"]))
    u, cot = oracle.layer_potential(G, w["tgt_xy"], 8, sigma_S=w["sigma_S"], cS=1.0, sides=2,
                                    on_surface_node=w["on_surface_node"],
                                    on_surface_side=w["on_surface_side"])
    assert np.all(cot[:1024] >= 0) and np.all(cot[1024:] == -1)
    scale = np.abs(exact).max()
    assert np.abs(u[1024:] - exact[1024:]).max() / scale < 1e-13
    assert np.abs(u[:1024] - exact[:1024]).max() / scale < 1e-6
    gf = discretise_curve(*circle(1.0), 32, 64, k=1.0)
    cxy, _ = oracle.centres(g.node_xy, g.normal_xy, g.panel_of_node, g.panel_h, 2)
    errs = []
    for p in (6, 8, 10, 12):
        al = oracle.qbx_coefficients(gf.node_xy, gf.normal_xy, gf.weight, 1.0, cxy, p,
                                     sigma_S=np.cos(3 * gf.param_t))
        uq = oracle.qbx_evaluate(w["tgt_xy"][:1024], cot[:1024], cxy, al, p, 1.0)
        errs.append(np.abs(uq - exact[:1024]).max() / scale)
    assert errs[-1] < 1e-10
    assert all(errs[i + 1] < 0.05 * errs[i] for i in range(3))


def test_circle_dlp_closed_form_and_jump(oracle):
    g = discretise_curve(*circle(1.0), 32, 16, k=1.0)
    gf = discretise_curve(*circle(1.0), 32, 64, k=1.0)
    cxy, _ = oracle.centres(g.node_xy, g.normal_xy, g.panel_of_node, g.panel_h, 2)
    n = g.n
    al = oracle.qbx_coefficients(gf.node_xy, gf.normal_xy, gf.weight, 1.0, cxy, 10,
                                 sigma_D=np.exp(3j * gf.param_t), cS=0, cD=1)
    tg = np.concatenate([g.node_xy, g.node_xy])
    cot = np.arange(2 * n, dtype=np.int32)
    uq = oracle.qbx_evaluate(tg, cot, cxy, al, 10, 1.0)
    side = np.concatenate([np.ones(n), -np.ones(n)])
    exact = circle_dlp_mode(3, 1.0, 1.0, tg, side)
    assert np.abs(uq - exact).max() / np.abs(exact).max() < 1e-9
    # exterior limit minus interior limit is the density itself (outward normal)
    assert np.abs(uq[:n] - uq[n:] - np.exp(3j * g.param_t)).max() < 1e-9
    off = np.array([[0.5, 0.0], [0.0, -0.4], [2.0, 1.0], [-1.5, -1.5]])
    ud = oracle.direct_potential(g.node_xy, g.normal_xy, g.weight, 1.0, off,
                                 sigma_D=np.exp(3j * g.param_t), cS=0, cD=1)
    side_off = np.where(np.hypot(*off.T) > 1, 1, -1)
    assert _rel(ud, circle_dlp_mode(3, 1.0, 1.0, off, side_off)) < 1e-13


# ---------------------------------------------------------------- Green's identity
@pytest.fixture(scope="module")
def green_setup(oracle):
    k = 5.0
    f = PointSourceField(k, [[0.1, 0.2], [-0.3, -0.1]], [1.0 + 0.5j, -0.7 + 0.2j])
    gd = discretise_curve(*starfish(0.3, 5), 48, 16, k=k)
    gs = discretise_curve(*starfish(0.3, 5), 48, 64, k=k)
    cxy, crad = oracle.centres(gd.node_xy, gd.normal_xy, gd.panel_of_node, gd.panel_h, 2)
    sD = f.u(gs.node_xy)
    sS = f.dudn(gs.node_xy, gs.normal_xy)
    al = oracle.qbx_coefficients(gs.node_xy, gs.normal_xy, gs.weight, k, cxy, 12,
                                 sigma_S=sS, sigma_D=sD, cS=-1.0, cD=1.0)
    return dict(k=k, f=f, gd=gd, gs=gs, cxy=cxy, crad=crad, sS=sS, sD=sD, al=al)


def test_greens_identity_on_surface(oracle, green_setup):
    s = green_setup
    gd, n = s["gd"], s["gd"].n
    tg = np.concatenate([gd.node_xy, gd.node_xy])
    uq = oracle.qbx_evaluate(tg, np.arange(2 * n, dtype=np.int32), s["cxy"], s["al"], 12, s["k"])
    ue = s["f"].u(gd.node_xy)
    scale = np.abs(ue).max()
    assert np.abs(uq[:n] - ue).max() / scale < 1e-10           # exterior limit = u
    assert np.abs(uq[n:]).max() / scale < 1e-10                # interior limit = 0
    assert np.abs(0.5 * (uq[:n] + uq[n:]) - 0.5 * ue).max() / scale < 1e-10


def test_greens_identity_volume(oracle, green_setup):
    s = green_setup
    gd, gs = s["gd"], s["gs"]
    rng = np.random.default_rng(0)
    tt = rng.uniform(-1.6, 1.6, (2000, 2))
    cot, fails = oracle.associate(tt, gd.node_xy, gd.panel_of_node, gd.panel_h, s["cxy"],
                                  s["crad"], 0.1)
    assert fails == 0 and (cot >= 0).sum() > 100
    u = np.zeros(len(tt), complex)
    dm = cot == -1
    u[dm] = oracle.direct_potential(gs.node_xy, gs.normal_xy, gs.weight, s["k"], tt[dm],
                                    sigma_S=s["sS"], sigma_D=s["sD"], cS=-1, cD=1)
    qm = cot >= 0
    u[qm] = oracle.qbx_evaluate(tt[qm], cot[qm], s["cxy"], s["al"], 12, s["k"])
    th = np.arctan2(tt[:, 1], tt[:, 0])
    inside = np.hypot(tt[:, 0], tt[:, 1]) < 1 + 0.3 * np.cos(5 * th)
    ue = s["f"].u(tt)
    ref = np.where(inside, 0, ue)
    assert np.abs(u - ref).max() / np.abs(ue).max() < 1e-10


# ---------------------------------------------------------------- association
def test_association_rules(oracle):
    # two panels (q=2) along the x axis, h=1 each, nodes at x=0.25,0.75,1.25,1.75
    node = np.array([[0.25, 0], [0.75, 0], [1.25, 0], [1.75, 0]], float)
    nrm = np.tile([0.0, 1.0], (4, 1))
    pon = np.array([0, 0, 1, 1])
    h = np.array([1.0, 1.0])
    cxy, crad = oracle.centres(node, nrm, pon, h, 2)
    assert np.allclose(cxy[:4, 1], 0.5) and np.allclose(cxy[4:, 1], -0.5)
    tgt = np.array([
        [0.3, 0.6],     # nearest exterior centre 0
        [0.74, -0.2],   # nearest interior centre of node 1 -> 5
        [0.5, 0.5],     # equidistant to centres 0 and 1 -> smaller index 0
        [5.0, 5.0],     # far: direct
        [3.0, 0.2],     # outside every disk, 1.25 from nodes: direct
        [0.75, 0.0],    # on-surface node 1, interior side
        [1.99, 0.0],    # outside all disks (d=0.5546 > 0.55) but within h/4 of node 3: failure
    ])
    osn = np.array([-1, -1, -1, -1, -1, 1, -1])
    oss = np.array([0, 0, 0, 0, 0, -1, 0], np.int8)
    cot, fails = oracle.associate(tgt, node, pon, h, cxy, crad, 0.1, osn, oss)
    assert list(cot) == [0, 5, 0, -1, -1, 5, -2]
    assert fails == 1


# ---------------------------------------------------------------- invariants
def test_rotation_and_linearity(oracle):
    k = 6.0
    g = discretise_curve(*starfish(0.2, 3), 24, 8, k=k)
    rng = np.random.default_rng(5)
    s1 = rng.standard_normal(g.n) + 1j * rng.standard_normal(g.n)
    s2 = rng.standard_normal(g.n) + 1j * rng.standard_normal(g.n)
    cxy, _ = oracle.centres(g.node_xy, g.normal_xy, g.panel_of_node, g.panel_h, 1)
    idx = np.arange(0, g.n, 17)
    p = 6
    a = oracle.qbx_coefficients(g.node_xy, g.normal_xy, g.weight, k, cxy[idx], p, s1, s2,
                                cS=2.0, cD=1.0)
    phi = 0.7
    R = np.array([[np.cos(phi), -np.sin(phi)], [np.sin(phi), np.cos(phi)]])
    ar = oracle.qbx_coefficients(g.node_xy @ R.T, g.normal_xy @ R.T, g.weight, k,
                                 cxy[idx] @ R.T, p, s1, s2, cS=2.0, cD=1.0)
    ell = np.arange(-p, p + 1)
    assert _rel(ar, a * np.exp(1j * ell * phi)[None, :]) < 1e-12
    # linearity in the density and in (cS, cD)
    a1 = oracle.qbx_coefficients(g.node_xy, g.normal_xy, g.weight, k, cxy[idx], p, s1, None,
                                 cS=2.0)
    a2 = oracle.qbx_coefficients(g.node_xy, g.normal_xy, g.weight, k, cxy[idx], p, None, s2,
                                 cS=0.0, cD=1.0)
    assert _rel(a1 + a2, a) < 1e-13
    # translation invariance of the potential
    t = np.array([[3.0, 1.0], [-2.5, 0.4]])
    u = oracle.direct_potential(g.node_xy, g.normal_xy, g.weight, k, t, s1, s2)
    ut = oracle.direct_potential(g.node_xy + 10.0, g.normal_xy, g.weight, k, t + 10.0, s1, s2)
    assert _rel(ut, u) < 1e-11


# ---------------------------------------------------------------- Conditions 1-4 (Sec. 3.3)
def test_condition_flags_two_circles_closed_form(oracle):
    """Two unit circles 0.05 apart: the oracle's brute-force flags equal those of
    the closed-form distance to circular arcs (Conditions 1 and 3), for equal
    and for very different panel sizes on the two circles."""
    from tests.condition_geoms import expected_two_circles, two_circles
    for n1, n2 in ((24, 24), (48, 12)):
        g = two_circles(0.05, n1, n2)
        got = oracle.conditions(g.as_dict(), sides=2)
        exp = expected_two_circles(g, n1, n2, 0.05)
        assert np.array_equal(got & 5, exp), (n1, n2, np.nonzero(got != exp))
        assert (got & 1).any()
    g = two_circles(0.05, 48, 12)
    assert (oracle.conditions(g.as_dict()) & 4).any()     # coarse arcs near fine centres
    g = two_circles(1.0, 24, 24)                           # far apart: nothing
    assert not oracle.conditions(g.as_dict()).any()


def test_condition_flags_two_to_one_and_wavelength(oracle):
    from tests.condition_geoms import uneven_circle
    g = uneven_circle(3.0)
    f = oracle.conditions(g.as_dict())
    assert np.nonzero(f & 2)[0].tolist() == [5]            # the long panel only
    g = uneven_circle(1.9)
    assert not (oracle.conditions(g.as_dict()) & 2).any()
    g = discretise_curve(*starfish(0.3, 5), 16, 16, k=12.0)  # k h about 6 > 5
    f = oracle.conditions(g.as_dict())
    assert np.array_equal((f & 8) != 0, 12.0 * g.panel_h > 5.0)
    assert (f & 8).any()
