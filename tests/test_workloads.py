"""The synthetic workloads (qbx_workloads): seeded, with the sizes and
structure their recipe states, and obeying Condition 4 of Sec. 5
(k * max panel length <= 5) that the method's accuracy rests on."""
import numpy as np
import pytest

from qbx_workloads.configs import make_config


@pytest.fixture(scope="module")
def cfg():
    cache = {}

    def get(n):
        if n not in cache:
            cache[n] = make_config(n)
        return cache[n]
    return get


def _kh(w):
    g = w["geom"]
    curve = np.repeat(np.arange(g.n_curves), np.diff(g.panel_offset))
    return g.k[curve] * g.panel_h


def test_seeded_and_reproducible():
    a, b = make_config(2), make_config(2)
    for key in ("tgt_xy", "sigma_S", "sigma_D"):
        assert np.array_equal(a[key], b[key])
    assert np.array_equal(a["geom"].node_xy, b["geom"].node_xy)
    assert not np.array_equal(a["sigma_D"], make_config(3)["sigma_D"][: a["sigma_D"].size])


@pytest.mark.parametrize("num,name,nodes,targets,k,p,p_fmm", [
    (1, "circle-k1", 32 * 16, 2 * 512 + 1000, 1.0, 8, None),
    (2, "starfish-k10", 512 * 16, 316 * 316, 10.0, 12, 20),
    (3, "starfish-k50", 8192 * 16, 316 * 316, 50.0, 16, 30),
    (5, "ellipses-200", 2 ** 20, 10 ** 6, 20.0, 16, 30),
])
def test_sizes_and_orders(cfg, num, name, nodes, targets, k, p, p_fmm):
    w = cfg(num)
    g = w["geom"]
    assert w["name"] == name
    assert g.n == nodes and g.q == 16
    assert w["tgt_xy"].shape == (targets, 2)
    assert np.all(g.k == k)
    assert w["p"] == p
    if p_fmm is not None:
        assert w["p_fmm"] == p_fmm


def test_batch_curves(cfg):
    w = cfg(4)
    g = w["geom"]
    assert g.n_curves == 256
    assert np.all((g.k >= 1.0) & (g.k <= 40.0))
    panels = np.diff(g.panel_offset)
    assert panels.min() >= 16
    # every node is an exterior on-surface target
    assert w["tgt_xy"].shape[0] == g.n
    assert np.array_equal(w["on_surface_node"], np.arange(g.n))
    assert np.all(w["on_surface_side"] == 1)
    assert (w["p"], w["p_fmm"]) == (12, 20)


@pytest.mark.parametrize("num", [1, 2, 3, 4, 5])
def test_condition_4(cfg, num):
    assert _kh(cfg(num)).max() <= 5.0


def test_circle_quadrature_and_normals(cfg):
    g = cfg(1)["geom"]
    assert abs(g.weight.sum() - 2 * np.pi) < 1e-12
    assert np.allclose(np.hypot(*g.normal_xy.T), 1.0)
    assert np.allclose(g.normal_xy, g.node_xy)  # outward on the unit circle


def test_ellipses_apart_and_inside_the_square(cfg):
    w = cfg(5)
    g = w["geom"]
    assert g.n_curves == 200
    assert np.all((g.node_xy >= 0.0) & (g.node_xy <= 100.0))
    # the ellipses sit in disjoint discs whose boundaries are at least 1 apart,
    # so nodes of different curves are too (checked where bounding boxes are
    # closer than that)
    off = g.node_offset()
    lo = np.array([g.node_xy[off[c]:off[c + 1]].min(axis=0) for c in range(200)])
    hi = np.array([g.node_xy[off[c]:off[c + 1]].max(axis=0) for c in range(200)])
    gap = np.maximum(lo[:, None, :] - hi[None, :, :], lo[None, :, :] - hi[:, None, :]).max(axis=2)
    np.fill_diagonal(gap, np.inf)
    for i, j in zip(*np.nonzero(gap < 1.0)):
        if i < j:
            a, b = g.node_xy[off[i]:off[i + 1]], g.node_xy[off[j]:off[j + 1]]
            d = np.sqrt(((a[:, None, :] - b[None, :, :]) ** 2).sum(-1)).min()
            assert d >= 1.0, (i, j, d)
    # double layer only; the last 10^5 targets lie within half a panel of a node
    assert w["sigma_S"] is None and w["cS"] == 0
    spatial = pytest.importorskip("scipy.spatial")
    dist, _ = spatial.cKDTree(g.node_xy).query(w["tgt_xy"][-100_000:])
    assert dist.max() <= 0.5 * g.panel_h.max() * (1 + 1e-12)
