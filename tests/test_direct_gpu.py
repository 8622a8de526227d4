"""GPU parity of the direct (all-pairs) Global QBX path against the FP64 oracle.

Tolerance (FP64 path): relative l2 error <= 1e-10 over every compared set
(potentials, and QBX coefficients order by order); association indices equal.
"""
import numpy as np
import pytest

from qbx_workloads import circle, discretise_curve, make_config, starfish
from tests.fields import PointSourceField

pytestmark = pytest.mark.gpu

TOL64 = 1e-10


def rel_l2(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b)))


def check_alpha(alpha, a_ref, k, radius, tol_rim=TOL64, tol_order=1e-8):
    """QBX coefficients: every order weighted by |J_l(k r_c)| (its size at the rim of
    the expansion disk, where u = sum alpha_l J_l e^{-il th} is evaluated) within
    tol_rim; each order on its own within tol_order (a wrong index or sign gives O(1))."""
    from scipy.special import jv
    P = alpha.shape[1]
    p = (P - 1) // 2
    wgt = np.abs(jv(np.arange(-p, p + 1)[None, :], k * np.asarray(radius)[:, None]))
    assert rel_l2(alpha * wgt, a_ref * wgt) < tol_rim
    for l in range(P):
        assert rel_l2(alpha[:, l], a_ref[:, l]) < tol_order, l


@pytest.fixture(scope="module")
def qbxmod():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1602_05301_gb300 import build as b
    b.build()
    from paper_1602_05301_gb300 import qbx
    return qbx


def _assoc_oracle(oracle, w, sides):
    g = w["geom"]
    cxy, crad = oracle.centres(g.node_xy, g.normal_xy, g.panel_of_node, g.panel_h, sides)
    cot, fails = oracle.associate(w["tgt_xy"], g.node_xy, g.panel_of_node, g.panel_h, cxy,
                                  crad, w["eps_assoc"], w["on_surface_node"],
                                  w["on_surface_side"])
    return cot, fails, cxy


def test_circle_config_parity(qbxmod, oracle):
    w = make_config(1)
    g = w["geom"]
    lp = qbxmod.LayerPotential(g.as_dict(), w["p"], sides=2)
    assoc = lp.build(w["tgt_xy"], w["on_surface_node"], w["on_surface_side"],
                     mode=qbxmod.QBX_DIRECT)
    cot, fails, cxy = _assoc_oracle(oracle, w, 2)
    assert fails == 0
    assert np.array_equal(assoc, cot)
    alpha = np.empty((lp.n_centres, 2 * w["p"] + 1), np.complex128)
    u = lp.eval(sigma_S=w["sigma_S"], cS=w["cS"], alpha_out=alpha)
    u_ref, _ = oracle.layer_potential(g.as_dict(), w["tgt_xy"], w["p"], sigma_S=w["sigma_S"],
                                      cS=w["cS"], sides=2, centre_of_target=cot)
    assert rel_l2(u, u_ref) < TOL64
    a_ref = oracle.qbx_coefficients(g.node_xy, g.normal_xy, g.weight, g.k[0], cxy, w["p"],
                                    sigma_S=w["sigma_S"], cS=w["cS"])
    _, crad = oracle.centres(g.node_xy, g.normal_xy, g.panel_of_node, g.panel_h, 2)
    check_alpha(alpha, a_ref, g.k[0], crad)
    lp.close()


@pytest.mark.parametrize("layers", ["S", "D", "SD"])
@pytest.mark.parametrize("p", [0, 5, 12, 16])
def test_ragged_starfish_layers_and_orders(qbxmod, oracle, layers, p):
    """Sizes that are not multiples of the 128-wide tiles; every order template."""
    k = 7.0
    g = discretise_curve(*starfish(0.25, 3), 37, 7, k=k)  # 259 nodes, 518 centres
    rng = np.random.default_rng(10 + p)
    s1 = rng.standard_normal(g.n) + 1j * rng.standard_normal(g.n)
    s2 = rng.standard_normal(g.n) + 1j * rng.standard_normal(g.n)
    sS = s1 if "S" in layers else None
    sD = s2 if "D" in layers else None
    cS, cD = 0.5 - 0.25j, 1.5 + 0.5j
    tgt = np.concatenate([rng.uniform(-1.6, 1.6, (301, 2)), g.node_xy[::5]])
    n_on = g.node_xy[::5].shape[0]
    on_node = np.concatenate([np.full(301, -1), np.arange(0, g.n, 5)])
    on_side = np.concatenate([np.zeros(301, np.int8),
                              np.where(np.arange(n_on) % 2 == 0, 1, -1).astype(np.int8)])
    lp = qbxmod.LayerPotential(g.as_dict(), p, sides=2)
    assoc = lp.build(tgt, on_node, on_side, mode=qbxmod.QBX_DIRECT, eps_assoc=0.5)
    alpha = np.empty((lp.n_centres, 2 * p + 1), np.complex128)
    u = lp.eval(sigma_S=sS, sigma_D=sD, cS=cS, cD=cD, alpha_out=alpha)
    u_ref, cot = oracle.layer_potential(g.as_dict(), tgt, p, sS, sD, cS, cD, sides=2,
                                        eps_assoc=0.5, on_surface_node=on_node,
                                        on_surface_side=on_side)
    assert np.array_equal(assoc, cot)
    assert rel_l2(u, u_ref) < TOL64
    cxy, crad = oracle.centres(g.node_xy, g.normal_xy, g.panel_of_node, g.panel_h, 2)
    idx = np.arange(0, lp.n_centres, 3)
    a_ref = oracle.qbx_coefficients(g.node_xy, g.normal_xy, g.weight, k, cxy[idx], p, sS, sD,
                                    cS, cD)
    check_alpha(alpha[idx], a_ref, k, crad[idx])
    lp.close()


def test_device_and_host_buffers_agree(qbxmod):
    torch = pytest.importorskip("torch")
    w = make_config(1)
    g = w["geom"]
    lp = qbxmod.LayerPotential(g.as_dict(), w["p"], sides=2)
    lp.build(w["tgt_xy"], w["on_surface_node"], w["on_surface_side"])
    u_host = lp.eval(sigma_S=w["sigma_S"], cS=1.0)
    sig = torch.from_numpy(w["sigma_S"]).cuda()
    out = torch.empty(lp.n_targets, dtype=torch.complex128, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    lp.eval(sigma_S=sig, cS=1.0, out=out, stream=stream)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), u_host)
    pinned = torch.from_numpy(w["sigma_S"]).pin_memory()
    out_p = torch.empty(lp.n_targets, dtype=torch.complex128).pin_memory()
    lp.eval(sigma_S=pinned, cS=1.0, out=out_p, stream=stream)
    assert np.array_equal(out_p.numpy(), u_host)
    lp.close()


def test_greens_identity_oversampled(qbxmod):
    """D[u] - S[du/dn] = u outside, 0 inside, on-surface limits u (ext) and 0 (int)."""
    k = 5.0
    f = PointSourceField(k, [[0.1, 0.2], [-0.3, -0.1]], [1.0 + 0.5j, -0.7 + 0.2j])
    gd = discretise_curve(*starfish(0.3, 5), 48, 16, k=k)
    gs = discretise_curve(*starfish(0.3, 5), 48, 64, k=k)
    src = dict(q=64, node_xy=gs.node_xy, normal_xy=gs.normal_xy, weight=gs.weight)
    lp = qbxmod.LayerPotential(gd.as_dict(), 12, sides=2, src=src)
    rng = np.random.default_rng(0)
    vol = rng.uniform(-1.6, 1.6, (1500, 2))
    n = gd.n
    tgt = np.concatenate([vol, gd.node_xy, gd.node_xy])
    on_node = np.concatenate([np.full(1500, -1), np.arange(n), np.arange(n)])
    on_side = np.concatenate([np.zeros(1500, np.int8), np.ones(n, np.int8),
                              -np.ones(n, np.int8)])
    lp.build(tgt, on_node, on_side)
    u = lp.eval(sigma_S=f.dudn(gs.node_xy, gs.normal_xy), sigma_D=f.u(gs.node_xy), cS=-1.0,
                cD=1.0)
    th = np.arctan2(vol[:, 1], vol[:, 0])
    inside = np.hypot(vol[:, 0], vol[:, 1]) < 1 + 0.3 * np.cos(5 * th)
    ue = f.u(tgt)
    ref = np.concatenate([np.where(inside, 0, ue[:1500]), ue[1500:1500 + n], np.zeros(n)])
    scale = np.abs(ue).max()
    assert np.abs(u - ref).max() / scale < 1e-10
    lp.close()


def test_starfish_config_sampled_parity(qbxmod, oracle):
    """Full-size starfish workload (8192 nodes, 99 856 grid targets), direct mode on the
    GPU; the oracle checks a sample of targets and centres one by one."""
    w = make_config(2)
    g = w["geom"]
    lp = qbxmod.LayerPotential(g.as_dict(), w["p"], sides=2)
    assoc = lp.build(w["tgt_xy"], mode=qbxmod.QBX_DIRECT)
    alpha = np.empty((lp.n_centres, 2 * w["p"] + 1), np.complex128)
    u = lp.eval(sigma_S=w["sigma_S"], sigma_D=w["sigma_D"], cS=w["cS"], cD=w["cD"],
                alpha_out=alpha)
    rng = np.random.default_rng(7)
    qbx_t = np.nonzero(assoc >= 0)[0]
    dir_t = np.nonzero(assoc < 0)[0]
    assert qbx_t.size > 100
    sample = np.concatenate([rng.choice(qbx_t, 96, replace=False),
                             rng.choice(dir_t, 96, replace=False)])
    cxy, crad = oracle.centres(g.node_xy, g.normal_xy, g.panel_of_node, g.panel_h, 2)
    cot, fails = oracle.associate(w["tgt_xy"][sample], g.node_xy, g.panel_of_node, g.panel_h,
                                  cxy, crad, w["eps_assoc"])
    assert fails == 0 and np.array_equal(cot, assoc[sample])
    u_ref, _ = oracle.layer_potential(g.as_dict(), w["tgt_xy"][sample], w["p"], w["sigma_S"],
                                      w["sigma_D"], w["cS"], w["cD"], sides=2,
                                      centre_of_target=cot)
    assert rel_l2(u[sample], u_ref) < TOL64
    cs = rng.choice(lp.n_centres, 64, replace=False)
    a_ref = oracle.qbx_coefficients(g.node_xy, g.normal_xy, g.weight, g.k[0], cxy[cs], w["p"],
                                    w["sigma_S"], w["sigma_D"], w["cS"], w["cD"])
    check_alpha(alpha[cs], a_ref, g.k[0], crad[cs])
    lp.close()


def test_edge_cases_and_statuses(qbxmod):
    g = discretise_curve(*circle(1.0), 8, 4, k=1.0)
    lp = qbxmod.LayerPotential(g.as_dict(), 3, sides=1)
    with pytest.raises(qbxmod.QBXError) as e:
        lp.eval(sigma_S=np.ones(g.n))
    assert e.value.status == qbxmod.QBX_ERR_STATE
    lp.build(np.zeros((0, 2)))                       # no targets at all
    out = lp.eval(sigma_S=np.ones(g.n))
    assert out.shape == (0,)
    with pytest.raises(qbxmod.QBXError) as e:         # interior side without interior centres
        lp.build(g.node_xy[:1], np.array([0]), np.array([-1], np.int8))
    assert e.value.status == qbxmod.QBX_ERR_ARG
    # association failure: inside h/4 of a node but in no disk (tiny eps_assoc)
    h = g.panel_h[0]
    t = g.node_xy[0] - 0.2 * h * g.normal_xy[0]
    with pytest.raises(qbxmod.QBXError) as e:
        lp.build(t[None, :], eps_assoc=1e-6)
    assert e.value.status == qbxmod.QBX_ERR_ASSOCIATION
    lp.close()
    # Condition 4: k * max h > 5
    big = discretise_curve(*circle(1.0), 4, 4, k=10.0).as_dict()
    with pytest.raises(qbxmod.QBXError) as e:
        qbxmod.LayerPotential(big, 4)
    assert e.value.status == qbxmod.QBX_ERR_CONDITION
