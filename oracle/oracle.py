"""ctypes wrapper of the FP64 CPU oracle (``qbx_oracle.cpp``).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU-baseline leg are the only callers. It shares no code with the CUDA path
and never imports it.

Every function computes the plain definition of a quantity of the paper
(Rachh, Kloeckner, O'Neil, Fast algorithms for QBX I), FP64:

* ``centres``                Sec. 2.2, c = s + side (h_k/2) n.
* ``qbx_coefficients``       Sec. 7 Eq. (localexpcoeffs): alpha at centres over all sources.
* ``direct_potential``       Sec. 3.2 Eq. (gauss-layerpot): smooth Gauss quadrature.
* ``qbx_evaluate``           Sec. 2.1 Eq. (phiapprox): truncated J-expansion.
* ``associate``              Sec. 6.1 target association, brute force over all centres.
* ``layer_potential``        Sec. 2.4 steps 2-3 without acceleration: associate,
                             then QBX where associated and direct quadrature elsewhere.
* ``source_grid``,           Sec. 2.2: the source discretisation of the same panels and
  ``interpolate_panels``     the density values on it by polynomial interpolation.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qbx_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_D = ctypes.POINTER(ctypes.c_double)
_I64 = ctypes.POINTER(ctypes.c_int64)
_I32 = ctypes.POINTER(ctypes.c_int32)
_I8 = ctypes.POINTER(ctypes.c_int8)


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (FP64, OpenMP, no fast-math, no FMA contraction)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-fopenmp",
           "-fno-fast-math", "-ffp-contract=off", _SRC, "-o", tmp]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.oracle_num_threads.restype = ctypes.c_int
            lib.oracle_set_num_threads.argtypes = [ctypes.c_int]
            lib.oracle_bessel.argtypes = [ctypes.c_int, ctypes.c_int64, _D, _D, _D]
            lib.oracle_set_hankel_recurrence.argtypes = [ctypes.c_int]
            lib.oracle_hankel_recurrence.restype = ctypes.c_int
            lib.oracle_hankel_table.argtypes = [ctypes.c_int, ctypes.c_int64, _D, _D]
            lib.oracle_centres.argtypes = [ctypes.c_int64, _D, _D, _I64, _D, ctypes.c_int, _D, _D]
            lib.oracle_qbx_coefficients.argtypes = [
                ctypes.c_int64, _D, _D, _D, _D, _D,
                ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                ctypes.c_int64, _D, ctypes.c_int, _D]
            lib.oracle_direct_potential.argtypes = [
                ctypes.c_int64, _D, _D, _D, _D, _D,
                ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                ctypes.c_int64, _D, _D]
            lib.oracle_qbx_evaluate.argtypes = [ctypes.c_int64, _D, _I32, _D, _D, ctypes.c_int,
                                                ctypes.c_double, _D]
            lib.oracle_associate.restype = ctypes.c_int64
            lib.oracle_associate.argtypes = [
                ctypes.c_int64, _D, _I64, _I8, ctypes.c_int64, _D, _I64, _D,
                ctypes.c_int64, _D, _D, ctypes.c_double, _I32]
            _lib = lib
    return _lib


def _p(a, ptype):
    if a is None:
        return ctypes.cast(None, ptype)
    return a.ctypes.data_as(ptype)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def _c128(a):
    if a is None:
        return None
    return np.ascontiguousarray(np.asarray(a, dtype=np.complex128)).view(np.float64)


def num_threads() -> int:
    return _load().oracle_num_threads()


def set_num_threads(n: int) -> None:
    _load().oracle_set_num_threads(int(n))


def set_hankel_recurrence(on: bool) -> None:
    """Hankel tables of the QBX coefficients: per-order library calls (False,
    the default) or H_0, H_1 and the upward recurrence (True), the affordable
    route at 2^20 sources per centre."""
    _load().oracle_set_hankel_recurrence(1 if on else 0)


class hankel_recurrence:
    """Context manager: QBX coefficients use the Hankel recurrence inside."""

    def __enter__(self):
        self.prev = _load().oracle_hankel_recurrence()
        set_hankel_recurrence(True)
        return self

    def __exit__(self, *a):
        set_hankel_recurrence(bool(self.prev))


def hankel_table(M: int, x) -> np.ndarray:
    """H_m(x), m = 0..M, as the QBX coefficients form them: [n][M+1] complex."""
    x = _f64(np.atleast_1d(x))
    out = np.empty(2 * x.size * (M + 1))
    _load().oracle_hankel_table(int(M), x.size, _p(x, _D), _p(out, _D))
    return out.view(np.complex128).reshape(x.size, M + 1)


def bessel_j(order: int, x) -> np.ndarray:
    x = _f64(np.atleast_1d(x))
    out = np.empty_like(x)
    _load().oracle_bessel(int(order), x.size, _p(x, _D), _p(out, _D), _p(None, _D))
    return out


def hankel1(order: int, x) -> np.ndarray:
    x = _f64(np.atleast_1d(x))
    out = np.empty(2 * x.size)
    _load().oracle_bessel(int(order), x.size, _p(x, _D), _p(None, _D), _p(out, _D))
    return out.view(np.complex128)


def centres(node_xy, normal_xy, panel_of_node, panel_h, sides: int):
    node_xy = _f64(node_xy)
    normal_xy = _f64(normal_xy)
    panel_of_node = np.ascontiguousarray(panel_of_node, dtype=np.int64)
    panel_h = _f64(panel_h)
    n = node_xy.shape[0]
    cxy = np.empty((n * sides, 2))
    crad = np.empty(n * sides)
    _load().oracle_centres(n, _p(node_xy, _D), _p(normal_xy, _D), _p(panel_of_node, _I64),
                           _p(panel_h, _D), int(sides), _p(cxy, _D), _p(crad, _D))
    return cxy, crad


def qbx_coefficients(src_xy, src_normal, weight, k, ctr_xy, p, sigma_S=None, sigma_D=None,
                     cS=1.0, cD=1.0) -> np.ndarray:
    src_xy, src_normal, weight, ctr_xy = map(_f64, (src_xy, src_normal, weight, ctr_xy))
    sS, sD = _c128(sigma_S), _c128(sigma_D)
    n_ctr = ctr_xy.shape[0]
    P = 2 * p + 1
    out = np.empty(2 * n_ctr * P)
    cS, cD = complex(cS), complex(cD)
    _load().oracle_qbx_coefficients(src_xy.shape[0], _p(src_xy, _D), _p(src_normal, _D),
                                    _p(weight, _D), _p(sS, _D), _p(sD, _D),
                                    cS.real, cS.imag, cD.real, cD.imag, float(k),
                                    n_ctr, _p(ctr_xy, _D), int(p), _p(out, _D))
    return out.view(np.complex128).reshape(n_ctr, P)


def direct_potential(src_xy, src_normal, weight, k, tgt_xy, sigma_S=None, sigma_D=None,
                     cS=1.0, cD=1.0) -> np.ndarray:
    src_xy, src_normal, weight, tgt_xy = map(_f64, (src_xy, src_normal, weight, tgt_xy))
    sS, sD = _c128(sigma_S), _c128(sigma_D)
    n_tgt = tgt_xy.shape[0]
    out = np.empty(2 * n_tgt)
    cS, cD = complex(cS), complex(cD)
    _load().oracle_direct_potential(src_xy.shape[0], _p(src_xy, _D), _p(src_normal, _D),
                                    _p(weight, _D), _p(sS, _D), _p(sD, _D),
                                    cS.real, cS.imag, cD.real, cD.imag, float(k),
                                    n_tgt, _p(tgt_xy, _D), _p(out, _D))
    return out.view(np.complex128)


def qbx_evaluate(tgt_xy, centre_of_target, ctr_xy, alpha, p, k) -> np.ndarray:
    tgt_xy, ctr_xy = _f64(tgt_xy), _f64(ctr_xy)
    cot = np.ascontiguousarray(centre_of_target, dtype=np.int32)
    al = _c128(alpha)
    out = np.zeros(2 * tgt_xy.shape[0])
    _load().oracle_qbx_evaluate(tgt_xy.shape[0], _p(tgt_xy, _D), _p(cot, _I32), _p(ctr_xy, _D),
                                _p(al, _D), int(p), float(k), _p(out, _D))
    return out.view(np.complex128)


def associate(tgt_xy, node_xy, panel_of_node, panel_h, ctr_xy, ctr_radius, eps_assoc,
              on_surface_node=None, on_surface_side=None):
    """Returns (centre_of_target int32 [-1 direct, -2 failure], n_failures)."""
    tgt_xy, node_xy, panel_h, ctr_xy, ctr_radius = map(
        _f64, (tgt_xy, node_xy, panel_h, ctr_xy, ctr_radius))
    pon = np.ascontiguousarray(panel_of_node, dtype=np.int64)
    osn = None if on_surface_node is None else np.ascontiguousarray(on_surface_node, np.int64)
    oss = None if on_surface_side is None else np.ascontiguousarray(on_surface_side, np.int8)
    out = np.empty(tgt_xy.shape[0], dtype=np.int32)
    fails = _load().oracle_associate(tgt_xy.shape[0], _p(tgt_xy, _D), _p(osn, _I64),
                                     _p(oss, _I8), node_xy.shape[0], _p(node_xy, _D),
                                     _p(pon, _I64), _p(panel_h, _D), ctr_xy.shape[0],
                                     _p(ctr_xy, _D), _p(ctr_radius, _D), float(eps_assoc),
                                     _p(out, _I32))
    return out, int(fails)


def layer_potential(geom, tgt_xy, p, sigma_S=None, sigma_D=None, cS=1.0, cD=1.0, sides=2,
                    eps_assoc=0.1, on_surface_node=None, on_surface_side=None,
                    centre_of_target=None):
    """Global QBX evaluation without acceleration (Sec. 2.4, steps 2-3 done directly).

    ``geom`` is a dict with node_xy, normal_xy, weight, panel_of_node, panel_h, k.
    If ``centre_of_target`` is given it replaces the oracle's own association
    (used to evaluate on a shared association where several answers are correct).
    Returns (u, centre_of_target, alpha_at_used_centres dict)."""
    cxy, crad = centres(geom["node_xy"], geom["normal_xy"], geom["panel_of_node"],
                        geom["panel_h"], sides)
    if centre_of_target is None:
        centre_of_target, fails = associate(tgt_xy, geom["node_xy"], geom["panel_of_node"],
                                            geom["panel_h"], cxy, crad, eps_assoc,
                                            on_surface_node, on_surface_side)
        if fails:
            raise RuntimeError("oracle: target association failed for %d targets" % fails)
    centre_of_target = np.asarray(centre_of_target, dtype=np.int32)
    tgt_xy = _f64(tgt_xy)
    u = np.zeros(tgt_xy.shape[0], dtype=np.complex128)
    direct = np.nonzero(centre_of_target < 0)[0]
    if direct.size:
        u[direct] = direct_potential(geom["node_xy"], geom["normal_xy"], geom["weight"],
                                     geom["k"], tgt_xy[direct], sigma_S, sigma_D, cS, cD)
    qbx = np.nonzero(centre_of_target >= 0)[0]
    if qbx.size:
        used, inv = np.unique(centre_of_target[qbx], return_inverse=True)
        alpha = qbx_coefficients(geom["node_xy"], geom["normal_xy"], geom["weight"], geom["k"],
                                 cxy[used], p, sigma_S, sigma_D, cS, cD)
        u[qbx] = qbx_evaluate(tgt_xy[qbx], inv.astype(np.int32), cxy[used], alpha, p, geom["k"])
    return u, centre_of_target


# ---------------------------------------------------------------- source grid (Sec. 2.2)
def _lagrange(q, q_src):
    """Lagrange basis of the q Gauss-Legendre nodes on [-1, 1] and its derivative,
    evaluated at the q_src Gauss-Legendre nodes: L, D [q_src][q]; and the q_src weights.
    Written out from the product formula l_i(u) = prod_{r != i} (u - x_r) / (x_i - x_r)."""
    xq, _ = np.polynomial.legendre.leggauss(q)
    xs, ws = np.polynomial.legendre.leggauss(q_src)
    L = np.ones((q_src, q))
    D = np.zeros((q_src, q))
    for i in range(q):
        for r in range(q):
            if r != i:
                L[:, i] *= (xs - xq[r]) / (xq[i] - xq[r])
        for s in range(q):
            if s == i:
                continue
            t = np.full(q_src, 1.0 / (xq[i] - xq[s]))
            for r in range(q):
                if r != i and r != s:
                    t *= (xs - xq[r]) / (xq[i] - xq[r])
            D[:, i] += t
    return L, D, ws


def interpolate_panels(values, q, q_src):
    """Values at the q density nodes of every panel (panels contiguous) -> values
    at q_src Gauss-Legendre nodes of the same panels, by the interpolating
    polynomial of each panel (Sec. 2.2). values: [n_panels * q, ...]."""
    L, _, _ = _lagrange(q, q_src)
    v = np.asarray(values)
    vp = v.reshape((-1, q) + v.shape[1:])
    out = np.einsum("ji,pi...->pj...", L, vp)
    return out.reshape((-1,) + v.shape[1:])


def source_grid(node_xy, normal_xy, q, q_src):
    """Source nodes, unit normals and weights of the panels of a density grid
    (Sec. 2.2): positions interpolated at q_src Gauss-Legendre nodes of each
    panel's reference variable u, normals the unit tangent dx/du turned by
    -90 degrees (sign of the interpolated normals), weights w_j |dx/du|."""
    L, D, ws = _lagrange(q, q_src)
    xy = np.asarray(node_xy, dtype=np.float64).reshape(-1, q, 2)
    nr = np.asarray(normal_xy, dtype=np.float64).reshape(-1, q, 2)
    pos = np.einsum("ji,pic->pjc", L, xy)
    tan = np.einsum("ji,pic->pjc", D, xy)
    nin = np.einsum("ji,pic->pjc", L, nr)
    speed = np.hypot(tan[..., 0], tan[..., 1])
    nrm = np.stack([tan[..., 1], -tan[..., 0]], -1) / speed[..., None]
    flip = np.sum(nrm * nin, axis=-1) < 0
    nrm[flip] *= -1.0
    w = ws[None, :] * speed
    return pos.reshape(-1, 2), nrm.reshape(-1, 2), w.reshape(-1)


# ---------------------------------------------------------------- Conditions 1-4 (Sec. 3.3)
def panel_distances(node_xy, q, points, n_samples=257, refine_rel=0.05, thresholds=None,
                    skip=None):
    """Distance from every point to every panel (the curve through the panel's q
    nodes, the interpolating polynomial in u in [-1, 1]): dense sampling, then a
    golden-section search on the curve around the nearest sample for the pairs
    whose sampled distance lies within refine_rel of a threshold (thresholds
    [n_points, n_panels], or None: refine none; pairs where skip is True are
    not refined). [n_points, n_panels]."""
    xq, _ = np.polynomial.legendre.leggauss(q)
    us = np.linspace(-1.0, 1.0, n_samples)

    def lagrange(u):
        L = np.ones((u.size, q))
        for i in range(q):
            for r in range(q):
                if r != i:
                    L[:, i] *= (u - xq[r]) / (xq[i] - xq[r])
        return L
    xy = np.asarray(node_xy, dtype=np.float64).reshape(-1, q, 2)
    samp = np.einsum("si,pic->psc", lagrange(us), xy)              # [panels, samples, 2]
    pts = np.asarray(points, dtype=np.float64)
    npan = xy.shape[0]
    dist = np.empty((pts.shape[0], npan))
    best = np.empty((pts.shape[0], npan), np.int64)
    chunk = max(1, int(2e7 // (npan * n_samples)))
    for i0 in range(0, pts.shape[0], chunk):
        d2 = ((pts[i0:i0 + chunk, None, None, :] - samp[None]) ** 2).sum(-1)
        bi = d2.argmin(-1)
        best[i0:i0 + chunk] = bi
        dist[i0:i0 + chunk] = np.sqrt(np.take_along_axis(d2, bi[..., None], -1)[..., 0])
    if thresholds is None:
        return dist
    near = np.abs(dist - thresholds) < refine_rel * thresholds
    if skip is not None:
        near &= ~skip
    ii, mm = np.nonzero(near)
    if ii.size == 0:
        return dist
    hs = 2.0 / (n_samples - 1)
    a = np.maximum(-1.0, us[best[ii, mm]] - hs)
    b = np.minimum(1.0, us[best[ii, mm]] + hs)
    P = pts[ii]

    def f(u):
        x = np.einsum("ni,nic->nc", lagrange(u), xy[mm])
        return np.hypot(*(x - P).T)
    g = (np.sqrt(5.0) - 1.0) / 2.0
    c, e = b - g * (b - a), a + g * (b - a)
    fc, fe = f(c), f(e)
    for _ in range(60):   # golden-section search, all pairs at once
        left = fc < fe
        b = np.where(left, e, b)
        a = np.where(left, a, c)
        c_new = np.where(left, b - g * (b - a), e)
        e_new = np.where(left, c, a + g * (b - a))
        fc_new = np.where(left, f(c_new), fe)
        fe_new = np.where(left, fc, f(e_new))
        c, e, fc, fe = c_new, e_new, fc_new, fe_new
    dist[ii, mm] = np.minimum(dist[ii, mm], np.minimum(fc, fe))
    return dist


def conditions(geom, sides=2):
    """Flags of Conditions 1-4 (Sec. 3.3) per panel, by brute force over every
    (centre, panel) pair, with the panel attribution of Sec. 5: Condition 1
    flags the panel of a centre closer than h_n/2 to another panel; Condition 2
    the longer of two adjacent panels whose lengths differ by more than 2;
    Condition 3 a panel m closer than h_m/4 to a centre of a panel that is
    neither m nor adjacent to m; Condition 4 a panel with k h > 5. geom: dict
    with node_xy, normal_xy, panel_h, q, k and panel_offset (curves). Returns
    int32 [n_panels] of bits 1, 2, 4, 8."""
    q = int(geom["q"])
    h = np.asarray(geom["panel_h"], dtype=np.float64)
    npan = h.size
    po = np.asarray(geom.get("panel_offset", [0, npan]), dtype=np.int64)
    curve = np.repeat(np.arange(po.size - 1), np.diff(po))
    pon = np.repeat(np.arange(npan), q)
    cxy, _ = centres(geom["node_xy"], geom["normal_xy"], pon, h, sides)
    cpan = np.tile(pon, sides)
    r1 = 0.5 * h[cpan][:, None] * np.ones((1, npan))
    r3 = 0.25 * h[None, :] * np.ones((cpan.size, 1))
    own = cpan[:, None] == np.arange(npan)[None, :]
    # refine near either threshold: run twice, keep the smaller distance
    d = np.minimum(panel_distances(geom["node_xy"], q, cxy, thresholds=r1, skip=own),
                   panel_distances(geom["node_xy"], q, cxy, thresholds=r3, skip=own))
    flags = np.zeros(npan, np.int32)
    n_in = np.diff(po)[curve]
    diff = (cpan[:, None] - np.arange(npan)[None, :]) % n_in[None, :]
    same = curve[cpan][:, None] == curve[None, :]
    adj = same & ((diff == 1) | (diff == n_in[None, :] - 1)) & (n_in[None, :] > 1)
    c1 = (d < r1) & ~own
    flags[np.unique(cpan[c1.any(1)])] |= 1
    c3 = (d < r3) & ~own & ~adj
    flags[np.nonzero(c3.any(0))[0]] |= 4
    for c in range(po.size - 1):
        ids = np.arange(po[c], po[c + 1])
        if ids.size < 2:
            continue
        nxt = np.roll(ids, -1)
        flags[ids[h[ids] > 2.0 * h[nxt]]] |= 2
        flags[nxt[h[nxt] > 2.0 * h[ids]]] |= 2
    flags[float(geom["k"]) * h > 5.0] |= 8
    return flags
