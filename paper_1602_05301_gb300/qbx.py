"""Thin Python binding of the C ABI in include/qbx.h (argument marshalling only).

The functions keep the ABI's names (qbx_geometry_create, qbx_tree_build,
qbx_layer_potential_eval, qbx_destroy, ...). Arrays may be numpy arrays (host)
or torch tensors (host, pinned host or CUDA); the library decides by pointer.
Nothing here computes any part of the layer potential: without the compiled
CUDA library every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libqbx_gb300.so")

QBX_OK, QBX_ERR_ARG, QBX_ERR_OOM, QBX_ERR_CUDA, QBX_ERR_CONDITION = 0, 1, 2, 3, 4
QBX_ERR_ASSOCIATION, QBX_ERR_TIMEOUT, QBX_ERR_STATE = 5, 6, 7
QBX_FP64, QBX_MIXED = 0, 1
QBX_DIRECT, QBX_FMM = 0, 1
QBX_COND1, QBX_COND2, QBX_COND3, QBX_COND4 = 1, 2, 4, 8
QBX_MAX_P = 16
STAGES = ["strengths", "p2m", "m2m", "p2p", "p2qbxl", "m2l", "m2p", "m2qbxl", "p2l", "l2l",
          "l2p", "l2qbxl", "qbxl2p"]
STATUS_NAMES = {0: "QBX_OK", 1: "QBX_ERR_ARG", 2: "QBX_ERR_OOM", 3: "QBX_ERR_CUDA",
                4: "QBX_ERR_CONDITION", 5: "QBX_ERR_ASSOCIATION", 6: "QBX_ERR_TIMEOUT",
                7: "QBX_ERR_STATE"}

_vp = ctypes.c_void_p


class qbx_geometry_desc(ctypes.Structure):
    _fields_ = [("n_panels", ctypes.c_int64), ("q", ctypes.c_int32),
                ("node_xy", _vp), ("normal_xy", _vp), ("weight", _vp), ("panel_h", _vp),
                ("q_src", ctypes.c_int32), ("src_xy", _vp), ("src_normal_xy", _vp),
                ("src_weight", _vp), ("k", ctypes.c_double), ("p_qbx", ctypes.c_int32),
                ("center_sides", ctypes.c_int32), ("n_curves", ctypes.c_int32),
                ("curve_panel_offset", _vp), ("defer_conditions", ctypes.c_int32)]


class qbx_tree_desc(ctypes.Structure):
    _fields_ = [("n_targets", ctypes.c_int64), ("target_xy", _vp), ("on_surface_node", _vp),
                ("on_surface_side", _vp), ("mode", ctypes.c_int32), ("p_fmm", ctypes.c_int32),
                ("p_add", ctypes.c_int32), ("n_max", ctypes.c_int32),
                ("eps_assoc", ctypes.c_double), ("assoc_out", _vp), ("m2l_engine", ctypes.c_int32)]


class QBXError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


_lib = None
_lock = threading.Lock()


def library() -> ctypes.CDLL:
    """Loads libqbx_gb300.so; raises if it has not been built (no fallback exists)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError("CUDA library %s is missing: run __graft_entry__.build() "
                                   "(or paper_1602_05301_gb300/build.py) first" % LIB_PATH)
            lib = ctypes.CDLL(LIB_PATH)
            lib.qbx_geometry_create.restype = ctypes.c_int
            lib.qbx_geometry_create.argtypes = [ctypes.POINTER(qbx_geometry_desc),
                                                ctypes.POINTER(_vp)]
            lib.qbx_tree_build.restype = ctypes.c_int
            lib.qbx_tree_build.argtypes = [_vp, ctypes.POINTER(qbx_tree_desc)]
            lib.qbx_layer_potential_eval.restype = ctypes.c_int
            lib.qbx_layer_potential_eval.argtypes = [
                _vp, ctypes.c_double, ctypes.c_double, _vp, ctypes.c_double, ctypes.c_double,
                _vp, _vp, _vp, ctypes.c_int32, _vp]
            lib.qbx_destroy.restype = None
            lib.qbx_destroy.argtypes = [_vp]
            lib.qbx_last_error.restype = ctypes.c_char_p
            lib.qbx_last_error.argtypes = []
            lib.qbx_get_stats.restype = ctypes.c_int
            lib.qbx_get_stats.argtypes = [_vp, ctypes.POINTER(ctypes.c_int64), ctypes.c_int32]
            lib.qbx_set_timing.restype = ctypes.c_int
            lib.qbx_set_timing.argtypes = [_vp, ctypes.c_int32]
            lib.qbx_get_stage_times.restype = ctypes.c_int32
            lib.qbx_get_stage_times.argtypes = [_vp, ctypes.POINTER(ctypes.c_double),
                                                ctypes.c_int32]
            lib.qbx_export_tree.restype = ctypes.c_int
            lib.qbx_export_tree.argtypes = [_vp] + [_vp] * 11
            lib.qbx_autotune.restype = ctypes.c_int
            lib.qbx_autotune.argtypes = [_vp, ctypes.POINTER(qbx_tree_desc), ctypes.c_int32,
                                         ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _vp,
                                         _vp]
            lib.qbx_batch_create.restype = ctypes.c_int
            lib.qbx_batch_create.argtypes = [ctypes.c_int32, _vp, ctypes.c_int32,
                                             ctypes.POINTER(_vp)]
            lib.qbx_batch_eval.restype = ctypes.c_int
            lib.qbx_batch_eval.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp, ctypes.c_int32, _vp]
            lib.qbx_batch_destroy.restype = None
            lib.qbx_batch_destroy.argtypes = [_vp]
            lib.qbx_get_box_orders.restype = ctypes.c_int
            lib.qbx_get_box_orders.argtypes = [_vp, _vp, ctypes.c_int32]
            lib.qbx_fmm_level_orders.restype = ctypes.c_int
            lib.qbx_fmm_level_orders.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_int32,
                                                 ctypes.c_int32, ctypes.c_int32, _vp]
            lib.qbx_default_p_add.restype = ctypes.c_int32
            lib.qbx_default_p_add.argtypes = [ctypes.c_int32]
            lib.qbx_get_source_grid.restype = ctypes.c_int
            lib.qbx_get_source_grid.argtypes = [_vp, _vp, _vp, _vp]
            lib.qbx_table1_q_src.restype = ctypes.c_int32
            lib.qbx_table1_q_src.argtypes = [ctypes.c_int32, ctypes.c_double]
            lib.qbx_check_conditions.restype = ctypes.c_int
            lib.qbx_check_conditions.argtypes = [_vp, _vp, _vp]
            lib.qbx_refine.restype = ctypes.c_int
            lib.qbx_refine.argtypes = [_vp, ctypes.c_int32, _vp, _vp]
            lib.qbx_get_geometry.restype = ctypes.c_int
            lib.qbx_get_geometry.argtypes = [_vp] + [_vp] * 8
            lib.qbx_autotune_tol.restype = ctypes.c_int
            lib.qbx_autotune_tol.argtypes = [_vp, ctypes.POINTER(qbx_tree_desc), ctypes.c_int32,
                                             ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                             ctypes.c_int32, _vp, _vp]
            lib.qbx_solve_dirichlet.restype = ctypes.c_int
            lib.qbx_solve_dirichlet.argtypes = [_vp, _vp, _vp, ctypes.c_int32, ctypes.c_int32,
                                                ctypes.c_int32, ctypes.c_double, ctypes.c_int32,
                                                ctypes.c_int32, _vp, _vp, _vp]
            lib.qbx_sync.restype = ctypes.c_int
            lib.qbx_sync.argtypes = [_vp]
            lib.qbx_selftest_wait_timeout.restype = ctypes.c_int
            lib.qbx_selftest_wait_timeout.argtypes = [_vp, ctypes.c_int32]
            lib.qbx_f32_from_f64.restype = ctypes.c_int
            lib.qbx_f32_from_f64.argtypes = [_vp, ctypes.c_int64, _vp]
            lib.qbx_measure_fma_rates.restype = ctypes.c_int
            lib.qbx_measure_fma_rates.argtypes = [_vp, _vp]
            lib.qbx_hankel01.restype = ctypes.c_int
            lib.qbx_hankel01.argtypes = [_vp, ctypes.c_int64, ctypes.c_int32, _vp]
            _lib = lib
    return _lib


def _check(status):
    if status != QBX_OK:
        raise QBXError(status, library().qbx_last_error().decode())


def ptr(a):
    """Raw address of a numpy array or torch tensor (None -> NULL)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    assert isinstance(a, np.ndarray) and a.flags["C_CONTIGUOUS"], "contiguous array expected"
    return a.ctypes.data


# ---------------------------------------------------------------- ABI-named wrappers
def qbx_geometry_create(desc: qbx_geometry_desc):
    h = _vp()
    _check(library().qbx_geometry_create(ctypes.byref(desc), ctypes.byref(h)))
    return h


def qbx_tree_build(handle, desc: qbx_tree_desc):
    _check(library().qbx_tree_build(handle, ctypes.byref(desc)))


def qbx_layer_potential_eval(handle, cS, sigma_S, cD, sigma_D, out, alpha_out=None,
                             precision=QBX_FP64, cuda_stream=None):
    cS, cD = complex(cS), complex(cD)
    _check(library().qbx_layer_potential_eval(handle, cS.real, cS.imag, ptr(sigma_S), cD.real,
                                              cD.imag, ptr(sigma_D), ptr(out), ptr(alpha_out),
                                              int(precision), cuda_stream))


def qbx_destroy(handle):
    if handle:
        library().qbx_destroy(handle)


def qbx_get_stats(handle):
    st = (ctypes.c_int64 * 20)()
    _check(library().qbx_get_stats(handle, st, 20))
    return list(st)


def qbx_set_timing(handle, enable: bool):
    _check(library().qbx_set_timing(handle, 1 if enable else 0))


def qbx_get_stage_times(handle):
    t = (ctypes.c_double * len(STAGES))()
    n = library().qbx_get_stage_times(handle, t, len(STAGES))
    return {STAGES[i]: t[i] for i in range(n)}


def qbx_export_tree(handle, n_src, n_ctr, n_tgt):
    """Copies the FMM tree and lists to numpy arrays (see include/qbx.h)."""
    lib = library()
    info = np.zeros(8, np.int64)
    root = np.zeros(3)
    _check(lib.qbx_export_tree(handle, ptr(info), ptr(root), None, None, None, None, None, None,
                               None, None, None))
    nb = int(info[0])
    out = dict(info=info, root=root, level=np.zeros(nb, np.int32),
               ij=np.zeros((nb, 2), np.int32), child=np.zeros((nb, 4), np.int32),
               range=np.zeros((nb, 4, 2), np.int32), off=np.zeros((4, nb + 1), np.int32),
               idx=np.zeros(max(1, int(info[2:6].sum())), np.int32),
               perm_src=np.zeros(max(1, n_src), np.int32),
               perm_ctr=np.zeros(max(1, n_ctr), np.int32),
               perm_tgt=np.zeros(max(1, n_tgt), np.int32))
    _check(lib.qbx_export_tree(handle, ptr(info), ptr(root), ptr(out["level"]), ptr(out["ij"]),
                               ptr(out["child"]), ptr(out["range"]), ptr(out["off"]),
                               ptr(out["idx"]), ptr(out["perm_src"]), ptr(out["perm_ctr"]),
                               ptr(out["perm_tgt"])))
    lists = {}
    pos = 0
    for i, name in enumerate("UVWX"):
        n = int(info[2 + i])
        seg = out["idx"][pos:pos + n]
        lists[name] = [seg[out["off"][i][b]:out["off"][i][b + 1]] for b in range(nb)]
        pos += n
    out["lists"] = lists
    return out


def qbx_hankel01(x, variant=0) -> np.ndarray:
    """(H_0(x), H_1(x)) as complex [n][2], evaluated by the library's device code."""
    xx = np.ascontiguousarray(x, dtype=np.float64)
    out = np.zeros((xx.size, 4))
    _check(library().qbx_hankel01(ptr(xx), int(xx.size), int(variant), ptr(out)))
    return out[:, 0::2] + 1j * out[:, 1::2]


def qbx_f32_from_f64(x) -> np.ndarray:
    """The mixed kernels' FP64 -> FP32 rounding, evaluated on the device."""
    xx = np.ascontiguousarray(x, dtype=np.float64)
    out = np.zeros(xx.size, np.float32)
    _check(library().qbx_f32_from_f64(ptr(xx), int(xx.size), ptr(out)))
    return out


def qbx_measure_fma_rates():
    """(FP64, FP32) FMA rates of the current GPU in TFLOP/s (qbx_measure_fma_rates)."""
    out = np.zeros(2)
    _check(library().qbx_measure_fma_rates(ptr(out[0:1]), ptr(out[1:2])))
    return float(out[0]), float(out[1])


def qbx_default_p_add(p: int) -> int:
    """p_add chosen for QBX order p when a plan is built with p_add < 0."""
    return int(library().qbx_default_p_add(int(p)))


def qbx_fmm_level_orders(k: float, root_side: float, n_levels: int, p_fmm: int,
                         p_add: int) -> np.ndarray:
    """Box expansion order of every tree level (0 on levels 0 and 1)."""
    out = np.zeros(n_levels, dtype=np.int32)
    _check(library().qbx_fmm_level_orders(float(k), float(root_side), int(n_levels), int(p_fmm),
                                          int(p_add), out.ctypes.data))
    return out


def qbx_table1_q_src(q: int, eps: float) -> int:
    """Source nodes per panel from Table 1 (-1 outside the table's range)."""
    return int(library().qbx_table1_q_src(int(q), float(eps)))


def qbx_last_error() -> str:
    return library().qbx_last_error().decode()


# ---------------------------------------------------------------- convenience object
def _host_f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class LayerPotential:
    """Owns one handle: geometry -> plan -> evaluations.

    geom: object with node_xy, normal_xy, weight, panel_h (numpy), q, k (scalar or [1]).
    src:  optional oversampled source grid (same panels): dict with q, node_xy,
          normal_xy, weight; densities then live on that grid.
    q_src: instead of src, the number of source nodes per panel of a grid that
          the library makes by interpolation; densities then live on the
          density grid (n_nodes values).
    """

    def __init__(self, geom, p, sides=2, src=None, q_src=0, defer_conditions=False):
        self._keep = []
        k = float(np.atleast_1d(geom.k)[0]) if hasattr(geom, "k") else float(geom["k"])
        g = geom if isinstance(geom, dict) else geom.__dict__
        node_xy, normal_xy = _host_f64(g["node_xy"]), _host_f64(g["normal_xy"])
        weight, panel_h = _host_f64(g["weight"]), _host_f64(g["panel_h"])
        self._keep += [node_xy, normal_xy, weight, panel_h]
        d = qbx_geometry_desc()
        d.n_panels = panel_h.shape[0]
        d.q = int(g["q"])
        d.node_xy, d.normal_xy, d.weight, d.panel_h = map(ptr, (node_xy, normal_xy, weight,
                                                               panel_h))
        if src is not None:
            sxy, snr, sw = (_host_f64(src["node_xy"]), _host_f64(src["normal_xy"]),
                            _host_f64(src["weight"]))
            self._keep += [sxy, snr, sw]
            d.q_src = int(src["q"])
            d.src_xy, d.src_normal_xy, d.src_weight = ptr(sxy), ptr(snr), ptr(sw)
        elif q_src:
            d.q_src = int(q_src)
        d.k = k
        d.p_qbx = int(p)
        d.center_sides = int(sides)
        po = g.get("panel_offset") if isinstance(g, dict) else None
        if po is not None:
            po = np.ascontiguousarray(po, dtype=np.int64)
            self._keep.append(po)
            d.n_curves = po.shape[0] - 1
            d.curve_panel_offset = ptr(po)
        d.defer_conditions = 1 if defer_conditions else 0
        self.k, self.p, self.sides = k, int(p), int(sides)
        self.n_nodes = node_xy.shape[0]
        self.n_src = (d.n_panels * d.q_src) if d.q_src else self.n_nodes
        self.n_density = self.n_nodes if (q_src and src is None) else self.n_src
        self.q, self.q_src = int(g["q"]), int(d.q_src)
        self._upsample = bool(q_src and src is None)
        self.n_curves = int(d.n_curves) if d.n_curves > 0 else 1
        self.n_centres = self.n_nodes * self.sides
        self.handle = qbx_geometry_create(d)
        self._keep = []
        self.n_targets = 0

    def build(self, target_xy, on_surface_node=None, on_surface_side=None, mode=QBX_DIRECT,
              p_fmm=0, p_add=-1, n_max=0, eps_assoc=0.1, m2l_engine=0):
        txy = _host_f64(target_xy)
        n = txy.shape[0]
        osn = None if on_surface_node is None else np.ascontiguousarray(on_surface_node,
                                                                        np.int64)
        oss = None if on_surface_side is None else np.ascontiguousarray(on_surface_side,
                                                                        np.int8)
        assoc = np.empty(n, dtype=np.int32)
        d = qbx_tree_desc(n, ptr(txy), ptr(osn), ptr(oss), int(mode), int(p_fmm), int(p_add),
                          int(n_max), float(eps_assoc), ptr(assoc), int(m2l_engine))
        qbx_tree_build(self.handle, d)
        self.n_targets = n
        return assoc

    def eval(self, sigma_S=None, sigma_D=None, cS=1.0, cD=1.0, out=None, alpha_out=None,
             precision=QBX_FP64, stream=None):
        """Densities / outputs: complex128 numpy arrays or torch tensors (host or CUDA)."""
        def prep(a):
            if a is None or hasattr(a, "data_ptr"):
                return a
            return np.ascontiguousarray(a, dtype=np.complex128)
        sigma_S, sigma_D = prep(sigma_S), prep(sigma_D)
        if out is None:
            out = np.empty(self.n_targets, dtype=np.complex128)
        qbx_layer_potential_eval(self.handle, cS, sigma_S, cD, sigma_D, out, alpha_out,
                                 precision, stream)
        return out

    def stats(self):
        names = ["n_sources", "n_centres", "n_targets", "n_qbx_targets", "n_boxes", "n_leaves",
                 "depth", "p_box", "u_pairs", "v_pairs", "w_pairs", "x_pairs",
                 "p2qbxl_pairs", "p2p_pairs", "m2qbxl_pairs", "m2p_pairs", "launches",
                 "p2l_pairs", "m2m_l2l", "p_box_max"]
        return dict(zip(names, qbx_get_stats(self.handle)))

    def box_orders(self):
        """Box expansion order of every tree level of the FMM plan."""
        out = np.zeros(25, dtype=np.int32)
        _check(library().qbx_get_box_orders(self.handle, out.ctypes.data, 25))
        depth = int(self.stats()["depth"])
        return out[:depth + 1]

    def check_conditions(self):
        """(panel flags [n_panels] int32 of QBX_COND* bits, counts [4]) -- Sec. 3.3."""
        n = self.geometry_size()
        flags = np.zeros(n, np.int32)
        counts = np.zeros(4, np.int64)
        _check(library().qbx_check_conditions(self.handle, ptr(flags), ptr(counts)))
        return flags, counts

    def refine(self, max_rounds=20):
        """Bisects flagged panels until Conditions 1-4 hold (qbx_refine); returns
        (rounds, n_panels). The plan is dropped: build it again."""
        r = np.zeros(1, np.int32)
        npan = np.zeros(1, np.int64)
        _check(library().qbx_refine(self.handle, int(max_rounds), ptr(r), ptr(npan)))
        self.n_nodes = int(npan[0]) * self.q
        self.n_src = int(npan[0]) * self.q_src if self.q_src else self.n_nodes
        self.n_density = self.n_nodes if self._upsample else self.n_src
        self.n_centres = self.n_nodes * self.sides
        self.n_targets = 0
        return int(r[0]), int(npan[0])

    def solve_dirichlet(self, rhs, mode=QBX_FMM, p_fmm=20, precision=QBX_FP64, tol=1e-10,
                        max_iter=500, restart=50, stream=None):
        """sigma of (1/2) sigma + D* sigma + i k S* sigma = rhs (qbx_solve_dirichlet);
        returns (sigma, iterations, relative residual). The handle's plan is
        replaced by the solver's (targets: the nodes, exterior side)."""
        b = np.ascontiguousarray(rhs, dtype=np.complex128) if not hasattr(rhs, "data_ptr") else rhs
        sig = np.empty(self.n_nodes, np.complex128)
        it = np.zeros(1, np.int32)
        res = np.zeros(1)
        _check(library().qbx_solve_dirichlet(self.handle, ptr(b), ptr(sig), int(mode), int(p_fmm),
                                             int(precision), float(tol), int(max_iter),
                                             int(restart), ptr(it), ptr(res), stream))
        self.n_targets = self.n_nodes
        return sig, int(it[0]), float(res[0])

    def geometry_size(self):
        n = np.zeros(1, np.int64)
        _check(library().qbx_get_geometry(self.handle, ptr(n), None, None, None, None, None,
                                          None, None))
        return int(n[0])

    def geometry(self):
        """The handle's density geometry: dict with node_xy, normal_xy, weight,
        panel_h, panel_origin, panel_interval, panel_offset (numpy)."""
        n = self.geometry_size()
        nn = n * self.q
        out = dict(node_xy=np.empty((nn, 2)), normal_xy=np.empty((nn, 2)),
                   weight=np.empty(nn), panel_h=np.empty(n),
                   panel_origin=np.empty(n, np.int64), panel_interval=np.empty((n, 2)),
                   panel_offset=np.empty(self.n_curves + 1, np.int64))
        m = np.zeros(1, np.int64)
        _check(library().qbx_get_geometry(
            self.handle, ptr(m), ptr(out["node_xy"]), ptr(out["normal_xy"]), ptr(out["weight"]),
            ptr(out["panel_h"]), ptr(out["panel_origin"]), ptr(out["panel_interval"]),
            ptr(out["panel_offset"])))
        out["q"] = self.q
        out["k"] = self.k
        out["panel_of_node"] = np.repeat(np.arange(n, dtype=np.int64), self.q)
        return out

    def source_grid(self):
        """(src_xy [n_src][2], src_normal_xy [n_src][2], src_weight [n_src])."""
        xy, nr, w = np.empty((self.n_src, 2)), np.empty((self.n_src, 2)), np.empty(self.n_src)
        _check(library().qbx_get_source_grid(self.handle, ptr(xy), ptr(nr), ptr(w)))
        return xy, nr, w

    def export_tree(self):
        return qbx_export_tree(self.handle, self.n_src, self.n_centres, self.n_targets)

    def autotune(self, target_xy, on_surface_node=None, on_surface_side=None, p_fmm=0,
                 p_add=-1, eps_assoc=0.1, precision=QBX_FP64, has_S=True, has_D=True, reps=3):
        """Times direct and FMM plans (qbx_autotune) and keeps the fastest built."""
        txy = _host_f64(target_xy)
        n = txy.shape[0]
        osn = None if on_surface_node is None else np.ascontiguousarray(on_surface_node,
                                                                        np.int64)
        oss = None if on_surface_side is None else np.ascontiguousarray(on_surface_side,
                                                                        np.int8)
        assoc = np.empty(n, dtype=np.int32)
        d = qbx_tree_desc(n, ptr(txy), ptr(osn), ptr(oss), QBX_DIRECT, int(p_fmm), int(p_add),
                          0, float(eps_assoc), ptr(assoc))
        times = np.zeros(4)
        chosen = np.zeros(1, np.int32)
        _check(library().qbx_autotune(self.handle, ctypes.byref(d), int(precision),
                                      int(bool(has_S)), int(bool(has_D)), int(reps), ptr(times),
                                      ptr(chosen)))
        self.n_targets = n
        return assoc, times, int(chosen[0])

    def autotune_tol(self, target_xy, on_surface_node=None, on_surface_side=None, p_fmm=20,
                     tol=1e-6, eps_assoc=0.1, precision=QBX_MIXED, has_S=True, has_D=True,
                     reps=2):
        """qbx_autotune_tol: the fastest plan within tol of the most accurate one.
        Returns (assoc, plan dict, report dict)."""
        txy = _host_f64(target_xy)
        n = txy.shape[0]
        osn = None if on_surface_node is None else np.ascontiguousarray(on_surface_node,
                                                                        np.int64)
        oss = None if on_surface_side is None else np.ascontiguousarray(on_surface_side,
                                                                        np.int8)
        assoc = np.empty(n, dtype=np.int32)
        d = qbx_tree_desc(n, ptr(txy), ptr(osn), ptr(oss), QBX_FMM, int(p_fmm), -1, 0,
                          float(eps_assoc), ptr(assoc))
        plan = np.zeros(5, np.int32)
        rep = np.zeros(3)
        _check(library().qbx_autotune_tol(self.handle, ctypes.byref(d), int(precision),
                                          int(bool(has_S)), int(bool(has_D)), float(tol),
                                          int(reps), ptr(plan), ptr(rep)))
        self.n_targets = n
        return assoc, dict(zip(("mode", "n_max", "p_fmm", "engine", "g"), map(int, plan))), \
            dict(ms=float(rep[0]), err=float(rep[1]), tried=int(rep[2]))

    def sync(self):
        """Waits for the device work; raises QBXError(QBX_ERR_TIMEOUT) if a
        bounded device wait gave up since the last check (qbx_sync)."""
        _check(library().qbx_sync(self.handle))

    def selftest_wait_timeout(self, limit_us=2000):
        _check(library().qbx_selftest_wait_timeout(self.handle, int(limit_us)))

    def set_timing(self, on=True):
        qbx_set_timing(self.handle, on)

    def stage_times(self):
        return qbx_get_stage_times(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            qbx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many planned LayerPotential objects evaluated together (qbx_batch_*): one
    CUDA graph with concurrent branches. Densities / outputs are concatenated in
    the order of `problems`."""

    def __init__(self, problems, n_streams=16):
        self.problems = list(problems)
        arr = (_vp * len(self.problems))(*[p.handle for p in self.problems])
        self._arr = arr
        b = _vp()
        _check(library().qbx_batch_create(len(self.problems), ctypes.cast(arr, _vp),
                                          int(n_streams), ctypes.byref(b)))
        self.handle = b
        self.n_src = sum(p.n_density for p in self.problems)   # density values per batch
        self.n_targets = sum(p.n_targets for p in self.problems)

    def eval(self, sigma_S=None, sigma_D=None, cS=None, cD=None, out=None,
             precision=QBX_FP64, stream=None):
        def prep(a):
            if a is None or hasattr(a, "data_ptr"):
                return a
            return np.ascontiguousarray(a, dtype=np.complex128)
        n = len(self.problems)
        cs = None if cS is None else np.ascontiguousarray(
            np.broadcast_to(np.asarray(cS, np.complex128), (n,))).view(np.float64)
        cd = None if cD is None else np.ascontiguousarray(
            np.broadcast_to(np.asarray(cD, np.complex128), (n,))).view(np.float64)
        sigma_S, sigma_D = prep(sigma_S), prep(sigma_D)
        if out is None:
            out = np.empty(self.n_targets, dtype=np.complex128)
        _check(library().qbx_batch_eval(self.handle, ptr(cs), ptr(sigma_S), ptr(cd),
                                        ptr(sigma_D), ptr(out), int(precision), stream))
        return out

    def close(self):
        if getattr(self, "handle", None):
            library().qbx_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
