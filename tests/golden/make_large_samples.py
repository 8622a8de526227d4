"""Writes the oracle's values at sampled targets and centres of the two large
single-geometry workloads (starfish k=50, 131 072 sources; 200 ellipses,
2^20 sources), for the element-wise parity tests of the GPU path at full size.

Calls only the FP64 oracle (oracle/) and the seeded workload generators
(qbx_workloads/); nothing here touches the CUDA library. For each workload:
  * 512 targets that the oracle's brute-force association (Sec. 6.1) gives a
    centre (all of them where there are fewer), and 512 that it leaves to
    direct quadrature, drawn at random;
  * u at those targets: the QBX evaluation (Eq. (phiapprox)) with the
    coefficients of its centre summed over ALL sources (Eq. (localexpcoeffs)),
    or direct Gauss quadrature (Eq. (gauss-layerpot));
  * alpha (l = -p..p) at 256 of the centres those targets use (topped up with
    other centres where fewer are used).
Hankel tables come from H_0, H_1 and the upward recurrence (pinned against the
per-order library calls and mpmath in tests/test_oracle_pins.py).

    python tests/golden/make_large_samples.py [3] [5]     (about 30 min on 8 cores)
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import oracle  # noqa: E402
from qbx_workloads import make_config  # noqa: E402

N_QBX, N_DIRECT, N_ALPHA = 512, 512, 256


def geometry_checksum(g):
    return np.array([g.node_xy.sum(), g.normal_xy.sum(), g.weight.sum(), g.panel_h.sum(),
                     float(g.n)])


def make(num, seed=77):
    w = make_config(num)
    g = w["geom"]
    rng = np.random.default_rng(seed + num)
    cxy, crad = oracle.centres(g.node_xy, g.normal_xy, g.panel_of_node, g.panel_h, w["sides"])
    n_t = w["tgt_xy"].shape[0]
    # candidates for QBX: targets with some centre within the largest association
    # radius (a k-d tree filter only; the oracle's association decides)
    from scipy.spatial import cKDTree
    r_max = (1.0 + w["eps_assoc"]) * crad.max() * (1.0 + 1e-9)
    d, _ = cKDTree(cxy).query(w["tgt_xy"], k=1, distance_upper_bound=r_max)
    near = np.nonzero(np.isfinite(d))[0]
    far = np.nonzero(~np.isfinite(d))[0]
    if w["on_surface_node"] is not None:
        on = np.nonzero(w["on_surface_node"] >= 0)[0]
        near = np.union1d(near, on)
        far = np.setdiff1d(far, on)

    def associate(idx):
        osn = None if w["on_surface_node"] is None else w["on_surface_node"][idx]
        oss = None if w["on_surface_side"] is None else w["on_surface_side"][idx]
        cot, fails = oracle.associate(w["tgt_xy"][idx], g.node_xy, g.panel_of_node, g.panel_h,
                                      cxy, crad, w["eps_assoc"], osn, oss)
        assert fails == 0
        return cot
    qbx_t, cot_q = [], []
    cand = rng.permutation(near)
    for i0 in range(0, cand.size, 4096):   # every QBX target when there are fewer than N_QBX
        idx = cand[i0:i0 + 4096]
        cot = associate(idx)
        for t, c in zip(idx, cot):
            if c >= 0 and len(qbx_t) < N_QBX:
                qbx_t.append(int(t)); cot_q.append(int(c))
        if len(qbx_t) >= N_QBX:
            break
    dir_t = rng.choice(far, N_DIRECT, replace=False)
    cot_d = associate(dir_t)
    assert np.all(cot_d == -1)
    dir_t, cot_d = [int(t) for t in dir_t], [int(c) for c in cot_d]
    tgt = np.array(qbx_t + dir_t, np.int64)
    cot = np.array(cot_q + cot_d, np.int32)
    t0 = time.time()
    with oracle.hankel_recurrence():
        u, _ = oracle.layer_potential(g.as_dict(), w["tgt_xy"][tgt], w["p"], w["sigma_S"],
                                      w["sigma_D"], w["cS"], w["cD"], sides=w["sides"],
                                      centre_of_target=cot)
        used = np.unique(cot[cot >= 0])
        ctr = rng.choice(used, min(N_ALPHA, used.size), replace=False)
        if ctr.size < N_ALPHA:   # fewer used centres than N_ALPHA: add other centres
            rest = np.setdiff1d(np.arange(cxy.shape[0]), ctr)
            ctr = np.concatenate([ctr, rng.choice(rest, N_ALPHA - ctr.size, replace=False)])
        ctr = np.sort(ctr).astype(np.int64)
        alpha = oracle.qbx_coefficients(g.node_xy, g.normal_xy, g.weight, g.k[0], cxy[ctr],
                                        w["p"], w["sigma_S"], w["sigma_D"], w["cS"], w["cD"])
    print("config %d: %d QBX + %d direct targets, %d centres in %.0f s (%d threads)"
          % (num, len(qbx_t), len(dir_t), ctr.size, time.time() - t0, oracle.num_threads()),
          flush=True)
    out = os.path.join(HERE, "large_config%d_samples.npz" % num)
    np.savez_compressed(out, config=num, target=tgt, target_xy=w["tgt_xy"][tgt],
                        centre_of_target=cot, u=u, centre=ctr, centre_xy=cxy[ctr], alpha=alpha,
                        p=w["p"], geometry_checksum=geometry_checksum(g))
    print("wrote", out)


if __name__ == "__main__":
    for a in (sys.argv[1:] or ["3", "5"]):
        make(int(a))
