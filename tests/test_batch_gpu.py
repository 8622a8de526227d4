"""Batched evaluation (qbx_batch_*) of many independent curves with their own
wavenumbers, with plans chosen by the measured autotuner (qbx_autotune): the
batch reproduces the per-curve evaluations bit for bit in FP64, matches the
oracle, and stays within 1e-6 of FP64 in mixed precision."""
import numpy as np
import pytest

from qbx_workloads import make_config

pytestmark = pytest.mark.gpu


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


@pytest.fixture(scope="module")
def batch_setup(qbxmod):
    w = make_config(4, n_curves=10)
    g = w["geom"]
    noff = g.node_offset()
    probs, chosen, sS, sD = [], [], [], []
    for c in range(g.n_curves):
        G = g.as_dict(c)
        lp = qbxmod.LayerPotential(G, w["p"], sides=1)
        n = G["node_xy"].shape[0]
        assoc, times, ch = lp.autotune(G["node_xy"], np.arange(n), np.ones(n, np.int8),
                                       p_fmm=w["p_fmm"], reps=2)
        assert np.all(assoc >= 0)
        probs.append(lp)
        chosen.append(ch)
        sS.append(w["sigma_S"][noff[c]:noff[c + 1]])
        sD.append(w["sigma_D"][noff[c]:noff[c + 1]])
    yield dict(w=w, probs=probs, chosen=chosen, sS=sS, sD=sD)
    for lp in probs:
        lp.close()


def test_autotuner_picks_measured_plans(batch_setup):
    ch = batch_setup["chosen"]
    assert all(c in (0, 1, 2, 3) for c in ch)
    small = [i for i, lp in enumerate(batch_setup["probs"]) if lp.n_src < 512]
    assert all(ch[i] == 0 for i in small)   # FMM candidates are not tried below 512 sources


def test_batch_equals_individual_fp64(qbxmod, batch_setup):
    probs = batch_setup["probs"]
    ref = [lp.eval(sigma_S=s, sigma_D=d, cS=1.0, cD=1.0)
           for lp, s, d in zip(probs, batch_setup["sS"], batch_setup["sD"])]
    b = qbxmod.Batch(probs, n_streams=4)
    sS = np.concatenate(batch_setup["sS"])
    sD = np.concatenate(batch_setup["sD"])
    for _ in range(2):   # capture, then replay
        out = b.eval(sigma_S=sS, sigma_D=sD, cS=1.0, cD=1.0)
        assert np.array_equal(out, np.concatenate(ref))
    # a coefficient change re-captures
    out2 = b.eval(sigma_S=sS, sigma_D=sD, cS=2.0, cD=1.0)
    ref2 = np.concatenate([lp.eval(sigma_S=s, sigma_D=d, cS=2.0, cD=1.0)
                           for lp, s, d in zip(probs, batch_setup["sS"], batch_setup["sD"])])
    assert np.array_equal(out2, ref2)
    b.close()


def test_batch_mixed_precision_and_oracle(qbxmod, batch_setup, oracle):
    probs = batch_setup["probs"]
    w = batch_setup["w"]
    g = w["geom"]
    b = qbxmod.Batch(probs)
    sS = np.concatenate(batch_setup["sS"])
    sD = np.concatenate(batch_setup["sD"])
    u64 = b.eval(sigma_S=sS, sigma_D=sD, cS=1.0, cD=1.0)
    u32 = b.eval(sigma_S=sS, sigma_D=sD, cS=1.0, cD=1.0, precision=qbxmod.QBX_MIXED)
    err = rel_l2(u32, u64)
    print("batch mixed vs fp64:", err)
    assert err < 1e-6
    b.close()
    # two curves against the oracle on sampled on-surface targets
    toff = np.concatenate([[0], np.cumsum([lp.n_targets for lp in probs])])
    rng = np.random.default_rng(3)
    for c in (0, len(probs) - 1):
        G = g.as_dict(c)
        n = G["node_xy"].shape[0]
        t = rng.choice(n, 24, replace=False)
        u_ref, _ = oracle.layer_potential(G, G["node_xy"][t], w["p"], batch_setup["sS"][c],
                                          batch_setup["sD"][c], 1.0, 1.0, sides=1,
                                          centre_of_target=t.astype(np.int32))
        assert rel_l2(u64[toff[c] + t], u_ref) < 1e-10


def test_tolerance_autotuner_meets_its_tolerance(qbxmod, oracle):
    """qbx_autotune_tol picks the fastest plan within tol of the most accurate
    one; the chosen plan's result stays within the tolerance of the oracle, and
    a second curve of the same size and k h reuses the cached decision."""
    w = make_config(4, n_curves=6)
    g = w["geom"]
    noff = g.node_offset()
    big = int(np.argmax(np.diff(noff)))
    for tol, prec in ((1e-6, qbxmod.QBX_MIXED), (1e-10, qbxmod.QBX_FP64)):
        G = g.as_dict(big)
        n = G["node_xy"].shape[0]
        lp = qbxmod.LayerPotential(G, w["p"], sides=1)
        assoc, plan, rep = lp.autotune_tol(G["node_xy"], np.arange(n), np.ones(n, np.int8),
                                           p_fmm=w["p_fmm"], tol=tol, precision=prec)
        print("tol %g: plan %s, report %s" % (tol, plan, rep))
        assert plan["mode"] in (0, 1) and rep["tried"] >= 1 and rep["err"] <= tol
        if plan["mode"] == 1:
            assert 4 <= plan["p_fmm"] <= w["p_fmm"] and plan["n_max"] in (16, 32, 64, 128)
        sS = w["sigma_S"][noff[big]:noff[big + 1]]
        sD = w["sigma_D"][noff[big]:noff[big + 1]]
        u = lp.eval(sigma_S=sS, sigma_D=sD, cS=1.0, cD=1.0, precision=prec)
        t = np.arange(0, n, max(1, n // 48))
        u_ref, _ = oracle.layer_potential(G, G["node_xy"][t], w["p"], sS, sD, 1.0, 1.0, sides=1,
                                          centre_of_target=t.astype(np.int32))
        err = rel_l2(u[t], u_ref)
        print("   vs oracle %.2e" % err)
        assert err < 20 * tol
        # the same curve again: the decision comes from the cache
        lp2 = qbxmod.LayerPotential(G, w["p"], sides=1)
        _, plan2, rep2 = lp2.autotune_tol(G["node_xy"], np.arange(n), np.ones(n, np.int8),
                                          p_fmm=w["p_fmm"], tol=tol, precision=prec)
        assert plan2 == plan and rep2["tried"] == 0
        lp.close()
        lp2.close()
