"""GPU FMM-accelerated Global QBX (Sec. 7): tree and interaction lists against the
brute-force definitions, and layer potentials / QBX coefficients against the
validated direct path and the FP64 oracle (relative l2 <= 1e-10)."""
import numpy as np
import pytest

from qbx_workloads import discretise_curve, make_config, starfish
from qbx_workloads.configs import grid_targets
from tests.listcheck import brute_lists, check_tree

pytestmark = pytest.mark.gpu

TOL64 = 1e-10


def rel_l2(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b)))


@pytest.fixture(scope="module")
def qbxmod():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1602_05301_gb300 import build as b
    b.build()
    from paper_1602_05301_gb300 import qbx
    return qbx


def _starfish(n_panels=64, k=10.0, grid=40, q=16):
    g = discretise_curve(*starfish(0.3, 5), n_panels, q, k=k)
    rng = np.random.default_rng(n_panels + grid)
    sigma = rng.standard_normal(g.n) + 1j * rng.standard_normal(g.n)
    tgt = grid_targets(grid, -2.0, 2.0)
    return g, sigma, tgt


@pytest.mark.parametrize("n_max", [8, 32, 64])
def test_tree_and_lists_match_definitions(qbxmod, n_max):
    g, sigma, tgt = _starfish(64, 10.0, 50)
    lp = qbxmod.LayerPotential(g.as_dict(), 6, sides=2)
    lp.build(tgt, mode=qbxmod.QBX_FMM, p_fmm=10, n_max=n_max)
    tree = lp.export_tree()
    cxy = np.concatenate([g.node_xy + 0.5 * g.panel_h[g.panel_of_node, None] * g.normal_xy,
                          g.node_xy - 0.5 * g.panel_h[g.panel_of_node, None] * g.normal_xy])
    crad = np.concatenate([0.5 * g.panel_h[g.panel_of_node]] * 2)
    check_tree(tree, [g.node_xy, cxy, tgt], n_max, crad)
    ref = brute_lists(tree)
    nb = tree["level"].shape[0]
    for name in "UVWX":
        for b in range(nb):
            assert sorted(tree["lists"][name][b].tolist()) == ref[name][b], (name, b)
    assert int(tree["info"][3]) > 0                        # V lists exist
    if n_max <= 8:
        assert int(tree["info"][4]) > 0 and int(tree["info"][5]) > 0   # W and X lists exist
    lp.close()


@pytest.mark.parametrize("layers", ["S", "D", "SD"])
@pytest.mark.parametrize("p", [4, 12])
def test_fmm_matches_direct(qbxmod, oracle, layers, p):
    """FMM and direct plans, each layer alone and combined, against each other and
    against the FP64 oracle (every target; coefficients at a sample of centres)."""
    g, sigma, tgt = _starfish(64, 10.0, 45)
    n = g.n
    tgt = np.concatenate([tgt, g.node_xy[::7], g.node_xy[3::11]])
    n_on = len(g.node_xy[::7]) + len(g.node_xy[3::11])
    on_node = np.concatenate([np.full(45 * 45, -1), np.arange(0, n, 7), np.arange(3, n, 11)])
    on_side = np.concatenate([np.zeros(45 * 45, np.int8),
                              np.where(np.arange(n_on) % 2 == 0, 1, -1).astype(np.int8)])
    sS = sigma if "S" in layers else None
    sD = np.conj(sigma) if "D" in layers else None
    res = {}
    for mode in (qbxmod.QBX_DIRECT, qbxmod.QBX_FMM):
        lp = qbxmod.LayerPotential(g.as_dict(), p, sides=2)
        assoc = lp.build(tgt, on_node, on_side, mode=mode, p_fmm=50, p_add=0, n_max=32)
        alpha = np.empty((lp.n_centres, 2 * p + 1), np.complex128)
        u = lp.eval(sigma_S=sS, sigma_D=sD, cS=10j, cD=1.0, alpha_out=alpha)
        res[mode] = (assoc, u, alpha)
        lp.close()
    a0, u0, al0 = res[qbxmod.QBX_DIRECT]
    a1, u1, al1 = res[qbxmod.QBX_FMM]
    assert np.array_equal(a0, a1)
    assert rel_l2(u1, u0) < TOL64
    r = 0.5 * g.panel_h[g.panel_of_node]
    from scipy.special import jv
    wgt = np.abs(jv(np.arange(-p, p + 1)[None, :], 10.0 * np.concatenate([r, r])[:, None]))
    assert rel_l2(al1 * wgt, al0 * wgt) < TOL64
    # the oracle, on the shared association
    with oracle.hankel_recurrence():
        u_ref, _ = oracle.layer_potential(g.as_dict(), tgt, p, sS, sD, 10j, 1.0, sides=2,
                                          centre_of_target=a1)
        cxy, _ = oracle.centres(g.node_xy, g.normal_xy, g.panel_of_node, g.panel_h, 2)
        cs = np.arange(0, lp_centres(g), 29)
        al_ref = oracle.qbx_coefficients(g.node_xy, g.normal_xy, g.weight, 10.0, cxy[cs], p,
                                         sS, sD, 10j, 1.0)
    for u in (u0, u1):
        assert rel_l2(u, u_ref) < TOL64
        assert np.max(np.abs(u - u_ref)) < TOL64 * np.max(np.abs(u_ref))
    for al in (al0, al1):
        assert rel_l2(al[cs] * wgt[cs], al_ref * wgt[cs]) < TOL64


def lp_centres(g):
    return 2 * g.n


def test_fmm_error_falls_with_box_order(qbxmod):
    g, sigma, tgt = _starfish(64, 10.0, 30)
    lp = qbxmod.LayerPotential(g.as_dict(), 8, sides=2)
    lp.build(tgt, mode=qbxmod.QBX_DIRECT)
    u0 = lp.eval(sigma_S=sigma, sigma_D=sigma, cS=10j, cD=1.0)
    lp.close()
    errs = []
    for pb in (10, 20, 30, 40):
        lp = qbxmod.LayerPotential(g.as_dict(), 8, sides=2)
        lp.build(tgt, mode=qbxmod.QBX_FMM, p_fmm=pb, p_add=0, n_max=32)
        u = lp.eval(sigma_S=sigma, sigma_D=sigma, cS=10j, cD=1.0)
        errs.append(rel_l2(u, u0))
        lp.close()
    assert errs[-1] < 1e-11, errs
    # geometric decay until the rounding floor (~1e-12) is reached
    assert all(errs[i + 1] < 0.25 * errs[i] or errs[i + 1] < 1e-12
               for i in range(len(errs) - 1)), errs


def test_fmm_circle_config(qbxmod, oracle):
    w = make_config(1)
    g = w["geom"]
    lp = qbxmod.LayerPotential(g.as_dict(), w["p"], sides=2)
    assoc = lp.build(w["tgt_xy"], w["on_surface_node"], w["on_surface_side"],
                     mode=qbxmod.QBX_FMM, p_fmm=20, n_max=32)
    u = lp.eval(sigma_S=w["sigma_S"], cS=1.0)
    u_ref, cot = oracle.layer_potential(g.as_dict(), w["tgt_xy"], w["p"], sigma_S=w["sigma_S"],
                                        cS=1.0, sides=2, on_surface_node=w["on_surface_node"],
                                        on_surface_side=w["on_surface_side"])
    assert np.array_equal(assoc, cot)
    assert rel_l2(u, u_ref) < TOL64
    lp.close()


def test_fmm_starfish_config_sampled_parity(qbxmod, oracle):
    """Full-size starfish workload (bench configuration) in FMM mode; the oracle
    checks a sample of targets and centres one by one."""
    w = make_config(2)
    g = w["geom"]
    lp = qbxmod.LayerPotential(g.as_dict(), w["p"], sides=2)
    assoc = lp.build(w["tgt_xy"], mode=qbxmod.QBX_FMM, p_fmm=w["p_fmm"])
    st = lp.stats()
    assert st["p_box"] == w["p_fmm"] + qbxmod.qbx_default_p_add(w["p"]) and st["n_boxes"] > 100
    alpha = np.empty((lp.n_centres, 2 * w["p"] + 1), np.complex128)
    u = lp.eval(sigma_S=w["sigma_S"], sigma_D=w["sigma_D"], cS=w["cS"], cD=w["cD"],
                alpha_out=alpha)
    rng = np.random.default_rng(8)
    qbx_t = np.nonzero(assoc >= 0)[0]
    dir_t = np.nonzero(assoc < 0)[0]
    sample = np.concatenate([rng.choice(qbx_t, 64, replace=False),
                             rng.choice(dir_t, 128, replace=False)])
    cxy, crad = oracle.centres(g.node_xy, g.normal_xy, g.panel_of_node, g.panel_h, 2)
    cot, fails = oracle.associate(w["tgt_xy"][sample], g.node_xy, g.panel_of_node, g.panel_h,
                                  cxy, crad, w["eps_assoc"])
    assert fails == 0 and np.array_equal(cot, assoc[sample])
    u_ref, _ = oracle.layer_potential(g.as_dict(), w["tgt_xy"][sample], w["p"], w["sigma_S"],
                                      w["sigma_D"], w["cS"], w["cD"], sides=2,
                                      centre_of_target=cot)
    assert rel_l2(u[sample], u_ref) < TOL64
    cs = rng.choice(lp.n_centres, 48, replace=False)
    a_ref = oracle.qbx_coefficients(g.node_xy, g.normal_xy, g.weight, g.k[0], cxy[cs], w["p"],
                                    w["sigma_S"], w["sigma_D"], w["cS"], w["cD"])
    from scipy.special import jv
    wgt = np.abs(jv(np.arange(-w["p"], w["p"] + 1)[None, :], g.k[0] * crad[cs][:, None]))
    assert rel_l2(alpha[cs] * wgt, a_ref * wgt) < TOL64
    lp.close()


def test_mixed_precision_starfish_config(qbxmod, oracle):
    """QBX_MIXED (FP32 translations with compensated sums, FP64 special functions and
    final sums) on the full starfish workload: relative l2 error <= 1e-6 against the
    FP64 path on every target and against the oracle on a sample; the error of each
    result (near targets, far targets, QBX coefficients) is reported."""
    w = make_config(2)
    g = w["geom"]
    lp = qbxmod.LayerPotential(g.as_dict(), w["p"], sides=2)
    assoc = lp.build(w["tgt_xy"], mode=qbxmod.QBX_FMM, p_fmm=w["p_fmm"])
    P = 2 * w["p"] + 1
    a64 = np.empty((lp.n_centres, P), np.complex128)
    a32 = np.empty((lp.n_centres, P), np.complex128)
    args = dict(sigma_S=w["sigma_S"], sigma_D=w["sigma_D"], cS=w["cS"], cD=w["cD"])
    u64 = lp.eval(alpha_out=a64, precision=qbxmod.QBX_FP64, **args)
    u32 = lp.eval(alpha_out=a32, precision=qbxmod.QBX_MIXED, **args)
    near = assoc >= 0
    from scipy.special import jv
    crad = np.concatenate([0.5 * g.panel_h[g.panel_of_node]] * 2)
    wgt = np.abs(jv(np.arange(-w["p"], w["p"] + 1)[None, :], g.k[0] * crad[:, None]))
    errs = dict(all=rel_l2(u32, u64), near=rel_l2(u32[near], u64[near]),
                far=rel_l2(u32[~near], u64[~near]), alpha=rel_l2(a32 * wgt, a64 * wgt))
    print("mixed vs fp64:", errs)
    assert max(errs.values()) < 1e-6, errs
    rng = np.random.default_rng(9)
    sample = np.concatenate([rng.choice(np.nonzero(near)[0], 32, replace=False),
                             rng.choice(np.nonzero(~near)[0], 64, replace=False)])
    u_ref, _ = oracle.layer_potential(g.as_dict(), w["tgt_xy"][sample], w["p"], w["sigma_S"],
                                      w["sigma_D"], w["cS"], w["cD"], sides=2,
                                      centre_of_target=assoc[sample])
    assert rel_l2(u32[sample], u_ref) < 1e-6
    lp.close()


def test_schedules_give_identical_fp64_results(qbxmod):
    """The evaluation's two-stream schedule, the single-stream order used while
    stage timing is on, and the throughput mode of a batched handle add the
    same terms in the same order into every output: FP64 results agree bit for
    bit (with and without the coefficients of every centre)."""
    w = make_config(2)
    g = w["geom"]
    lp = qbxmod.LayerPotential(g.as_dict(), w["p"], sides=w["sides"])
    lp.build(w["tgt_xy"], w["on_surface_node"], w["on_surface_side"], mode=qbxmod.QBX_FMM,
             p_fmm=w["p_fmm"])
    args = dict(sigma_S=w["sigma_S"], sigma_D=w["sigma_D"], cS=w["cS"], cD=w["cD"])
    u_fork = lp.eval(**args)
    a_fork = np.empty((lp.n_centres, 2 * w["p"] + 1), np.complex128)
    u_fork_all = lp.eval(alpha_out=a_fork, **args)
    assert np.array_equal(u_fork, u_fork_all)   # used centres only vs every centre
    lp.set_timing(True)
    u_serial = lp.eval(**args)
    lp.set_timing(False)
    assert np.array_equal(u_fork, u_serial)
    b = qbxmod.Batch([lp], n_streams=1)          # the handle is now in throughput mode
    u_batched = lp.eval(**args)
    a_batched = np.empty_like(a_fork)
    lp.eval(alpha_out=a_batched, **args)
    b.close()
    assert np.array_equal(u_fork, u_batched)
    assert np.array_equal(a_fork, a_batched)
    u_after = lp.eval(**args)                     # back to the single-problem schedule
    assert np.array_equal(u_fork, u_after)
    lp.close()


@pytest.mark.parametrize("engine", [0, 1, 2])
def test_m2l_engines_against_oracle(qbxmod, oracle, engine):
    """Every M2L engine (0: FP64 on tensor cores, mixed on the FP32 CUDA-core
    GEMM; 1: tensor cores in both precisions; 2: CUDA cores in both) meets the
    precision's tolerance against the oracle on a sample of the starfish
    workload, element-wise as well as in l2."""
    w = make_config(2)
    g = w["geom"]
    lp = qbxmod.LayerPotential(g.as_dict(), w["p"], sides=2)
    assoc = lp.build(w["tgt_xy"], mode=qbxmod.QBX_FMM, p_fmm=w["p_fmm"], m2l_engine=engine)
    args = dict(sigma_S=w["sigma_S"], sigma_D=w["sigma_D"], cS=w["cS"], cD=w["cD"])
    u64 = lp.eval(precision=qbxmod.QBX_FP64, **args)
    u32 = lp.eval(precision=qbxmod.QBX_MIXED, **args)
    lp.close()
    rng = np.random.default_rng(10)
    sample = np.concatenate([rng.choice(np.nonzero(assoc >= 0)[0], 48, replace=False),
                             rng.choice(np.nonzero(assoc < 0)[0], 96, replace=False)])
    u_ref, _ = oracle.layer_potential(g.as_dict(), w["tgt_xy"][sample], w["p"], w["sigma_S"],
                                      w["sigma_D"], w["cS"], w["cD"], sides=2,
                                      centre_of_target=assoc[sample])
    for u, tol in ((u64, TOL64), (u32, 1e-6)):
        d = u[sample] - u_ref
        e2 = rel_l2(u[sample], u_ref)
        em = float(np.max(np.abs(d)) / np.max(np.abs(u_ref)))
        print("engine %d: rel l2 %.3e, max-norm %.3e" % (engine, e2, em))
        assert e2 < tol and em < tol
    with pytest.raises(qbxmod.QBXError):
        lp2 = qbxmod.LayerPotential(g.as_dict(), w["p"], sides=2)
        try:
            lp2.build(w["tgt_xy"], mode=qbxmod.QBX_FMM, p_fmm=w["p_fmm"], m2l_engine=3)
        finally:
            lp2.close()
