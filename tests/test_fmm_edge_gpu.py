"""Degenerate and ragged inputs of the FMM plan (Sec. 7) in both precisions,
against the FP64 oracle on a shared association: no targets at all, only
on-surface targets (every target a QBX target, no direct target), only far
targets (no QBX target), QBX order p = 0 (the expansion is alpha_0 alone), a
geometry small enough to be one leaf, targets far outside the curve's
bounding box (a tree that is mostly empty), and leaf sizes down to 4
particles (many levels, ragged leaves)."""
import numpy as np
import pytest

from qbx_workloads import circle, discretise_curve, starfish
from qbx_workloads.configs import grid_targets

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "mixed": 1e-6}


def errs(u, ref):
    d = np.abs(u - ref)
    return (float(np.linalg.norm(d) / np.linalg.norm(ref)), float(d.max() / np.abs(ref).max()))


@pytest.fixture(scope="module")
def qbxmod():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1602_05301_gb300 import build as b
    b.build()
    from paper_1602_05301_gb300 import qbx
    return qbx


def check(qbxmod, oracle, g, tgt, p, on_node=None, on_side=None, n_max=0, sides=2, seed=0,
          p_fmm=20):
    rng = np.random.default_rng(seed)
    sS = rng.standard_normal(g.n) + 1j * rng.standard_normal(g.n)
    sD = rng.standard_normal(g.n) + 1j * rng.standard_normal(g.n)
    cS, cD = 1j * g.k[0], 1.0
    lp = qbxmod.LayerPotential(g.as_dict(), p, sides=sides)
    assoc = lp.build(tgt, on_node, on_side, mode=qbxmod.QBX_FMM, p_fmm=p_fmm, n_max=n_max)
    res = {}
    for name, prec in (("fp64", qbxmod.QBX_FP64), ("mixed", qbxmod.QBX_MIXED)):
        res[name] = lp.eval(sigma_S=sS, sigma_D=sD, cS=cS, cD=cD, precision=prec)
    lp.close()
    if len(tgt) == 0:
        assert all(r.shape == (0,) for r in res.values())
        return assoc
    u_ref, _ = oracle.layer_potential(g.as_dict(), tgt, p, sS, sD, cS, cD, sides=sides,
                                      centre_of_target=assoc)
    for name, u in res.items():
        e2, em = errs(u, u_ref)
        print("%s: rel l2 %.2e, max-norm %.2e" % (name, e2, em))
        assert e2 < TOL[name] and em < TOL[name], (name, e2, em)
    return assoc


def test_no_targets(qbxmod, oracle):
    g = discretise_curve(*starfish(0.3, 5), 32, 16, k=5.0)
    check(qbxmod, oracle, g, np.zeros((0, 2)), 8)


def test_only_on_surface_targets(qbxmod, oracle):
    g = discretise_curve(*starfish(0.3, 5), 48, 16, k=8.0)
    nodes = np.arange(0, g.n, 3)
    side = np.where(nodes % 2 == 0, 1, -1).astype(np.int8)
    assoc = check(qbxmod, oracle, g, g.node_xy[nodes], 10, nodes, side)
    assert np.all(assoc >= 0)


def test_only_far_targets(qbxmod, oracle):
    g = discretise_curve(*starfish(0.3, 5), 48, 16, k=8.0)
    t = np.linspace(0, 2 * np.pi, 300, endpoint=False)
    tgt = np.stack([3.0 * np.cos(t), 3.0 * np.sin(t)], 1)
    assoc = check(qbxmod, oracle, g, tgt, 10)
    assert np.all(assoc < 0)


def test_qbx_order_zero(qbxmod, oracle):
    # p_add(0) = 0: the box orders are p_fmm alone, so p_fmm = 30 keeps the
    # FMM's own truncation at the centres (1.1e-9 at p_fmm = 20 here) below 1e-10
    g = discretise_curve(*circle(1.0), 64, 16, k=3.0)
    check(qbxmod, oracle, g, grid_targets(25, -1.6, 1.6), 0, p_fmm=30)


def test_direct_targets_at_leaf_centres(qbxmod, oracle):
    """Grid targets that fall (to rounding) on the centres of leaf boxes: L2P at
    k r of order 1e-9, where J_1 still contributes O(k r) of the result."""
    g = discretise_curve(*circle(1.0), 64, 16, k=3.0)
    check(qbxmod, oracle, g, grid_targets(25, -1.6, 1.6), 4, p_fmm=30)


def test_single_leaf_geometry(qbxmod, oracle):
    g = discretise_curve(*circle(0.5), 2, 4, k=1.0)
    tgt = np.array([[0.0, 0.0], [0.3, 0.1], [0.52, 0.0], [2.0, 2.0]])
    check(qbxmod, oracle, g, tgt, 4, n_max=64)


def test_targets_far_outside_the_curve(qbxmod, oracle):
    g = discretise_curve(*starfish(0.3, 5), 48, 16, k=6.0)
    tgt = np.concatenate([grid_targets(12, -1.5, 1.5), [[50.0, -40.0], [-30.0, 80.0]]])
    check(qbxmod, oracle, g, tgt, 8)


@pytest.mark.parametrize("n_max", [4, 13])
def test_small_ragged_leaves(qbxmod, oracle, n_max):
    g = discretise_curve(*starfish(0.25, 3), 37, 16, k=7.0)
    rng = np.random.default_rng(n_max)
    tgt = np.concatenate([grid_targets(17, -1.5, 1.5), rng.uniform(-1.4, 1.4, (333, 2))])
    check(qbxmod, oracle, g, tgt, 6, n_max=n_max, seed=n_max)
