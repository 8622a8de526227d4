"""Conditions 1-4 of Sec. 3.3 checked on the GPU (qbx_check_conditions) against
the oracle's brute-force flags, and source refinement (qbx_refine, Sec. 5):
after it every condition holds (on the GPU and in the oracle), the new panels
lie on the original curves, and Green's identity near two nearly touching
curves comes out accurate on the refined geometry."""
import numpy as np
import pytest

from qbx_workloads import circle, discretise_curve, starfish
from tests.condition_geoms import two_circles, uneven_circle
from tests.fields import PointSourceField

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


CASES = {
    "two-circles-equal": lambda: two_circles(0.05, 24, 24),
    "two-circles-fine-coarse": lambda: two_circles(0.05, 48, 12),
    "two-circles-apart": lambda: two_circles(1.0, 24, 24),
    "uneven-circle": lambda: uneven_circle(3.0),
    "starfish-high-k": lambda: discretise_curve(*starfish(0.3, 5), 16, 16, k=12.0),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_flags_match_oracle(qbxmod, oracle, name):
    g = CASES[name]()
    lp = qbxmod.LayerPotential(g.as_dict(), 8, sides=2, defer_conditions=True)
    flags, counts = lp.check_conditions()
    lp.close()
    ref = oracle.conditions(g.as_dict(), sides=2)
    assert np.array_equal(flags, ref), (name, np.nonzero(flags != ref), flags[flags != ref],
                                        ref[flags != ref])
    assert list(counts) == [int(np.count_nonzero(ref & b)) for b in (1, 2, 4, 8)]


def test_refinement_meets_every_condition(qbxmod, oracle):
    g = two_circles(0.05, 24, 16, k=40.0)      # Conditions 1, 3 and 4 all broken
    lp = qbxmod.LayerPotential(g.as_dict(), 8, sides=2, defer_conditions=True)
    f0, c0 = lp.check_conditions()
    assert c0[0] > 0 and c0[2] > 0 and c0[3] > 0
    with pytest.raises(qbxmod.QBXError):        # Condition 4: no plan before refinement
        lp.build(g.node_xy[:4])
    rounds, n_pan = lp.refine(max_rounds=30)
    assert rounds >= 1 and n_pan > g.n_panels
    f1, c1 = lp.check_conditions()
    assert not f1.any() and not c1.any()
    G = lp.geometry()
    assert G["panel_h"].shape[0] == n_pan and G["panel_offset"][-1] == n_pan
    assert not oracle.conditions(G, sides=2).any()
    # the new nodes lie on the original circles, with outward unit normals
    ctr = np.where(np.repeat(G["panel_origin"] < 24, 16)[:, None], [[0.0, 0.0]], [[2.05, 0.0]])
    r = np.hypot(*(G["node_xy"] - ctr).T)
    assert np.max(np.abs(r - 1.0)) < 1e-12
    assert np.max(np.abs(G["normal_xy"] - (G["node_xy"] - ctr))) < 1e-9
    # panel lengths add up to the circumferences; the intervals cover each original panel
    assert abs(G["panel_h"].sum() - 4 * np.pi) < 1e-10
    for o in range(g.n_panels):
        iv = G["panel_interval"][G["panel_origin"] == o]
        iv = iv[np.argsort(iv[:, 0])]
        assert abs(iv[0, 0] + 1.0) < 1e-15 and abs(iv[-1, 1] - 1.0) < 1e-15
        assert np.all(np.abs(iv[1:, 0] - iv[:-1, 1]) < 1e-15)
    lp.close()


def test_refined_geometry_is_accurate_near_the_gap(qbxmod):
    """Green's identity D[u] - S[du/dn] = u at exterior targets in the narrow gap
    between two circles: the unrefined panels break Conditions 1 and 3 there and
    the identity fails; after qbx_refine it holds to 1e-9."""
    k = 2.0
    f = PointSourceField(k, [[0.2, 0.1], [2.3, -0.2]], [1.0 + 0.3j, -0.6 + 0.4j])
    g = two_circles(0.02, 24, 24, k=k)
    tgt = np.stack([np.full(41, 1.01), np.linspace(-0.1, 0.1, 41)], -1)  # mid-gap
    errs = []
    for refine in (False, True):
        lp = qbxmod.LayerPotential(g.as_dict(), 12, sides=2, q_src=64)
        if refine:
            lp.refine(max_rounds=30)
        G = lp.geometry()
        sD = f.u(G["node_xy"])
        sS = f.dudn(G["node_xy"], G["normal_xy"])
        lp.build(tgt, mode=qbxmod.QBX_DIRECT)
        u = lp.eval(sigma_S=sS, sigma_D=sD, cS=-1.0, cD=1.0)
        lp.close()
        ue = f.u(tgt)
        errs.append(np.max(np.abs(u - ue)) / np.max(np.abs(ue)))
    print("Green's identity in the gap: unrefined %.2e, refined %.2e" % tuple(errs))
    assert errs[1] < 1e-9 and errs[0] > 100 * errs[1]
