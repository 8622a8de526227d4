"""Calibrates p_add, the extra box order of FMM-accelerated QBX, on the GPU
(Sec. 7.1, "Maintaining Expansion Accuracy", and its Table 2).

The box order of tree level l is p_FMM^l + p_add, where p_FMM^l is the order a
plain point FMM needs on that level for a precision eps (the truncation
criterion of Sec. 7.1, as qbx_fmm_level_orders applies it). The paper finds
p_add by experiment, as a function of the QBX order p; this script repeats the
experiment with this library:

* random test curves r(t) = 5 + sum_{j=1..12} delta_j sin(j t), delta_j uniform
  in [-0.2, 0.2], Helmholtz parameter omega = k = 5;
* a known field u(x) = sum_m q_m H_0(k|x - x_m|) radiated by two point sources
  inside the curve, so that D[u] - S[du/dn] = u outside (Green's identity,
  Sec. 8.1);
* targets close to the boundary on the exterior side: every fourth node (the
  exterior one-sided limit) and as many points at distances up to h/2 along the
  outward normal of random nodes, all evaluated by QBX;
* the geometry refined (panel count) and oversampled (64 source nodes per
  16-node panel, Table 1 at eps = 1e-12) until the direct QBX evaluation has
  Green's-identity error at most eps / 2;
* for each eps, p_FMM from the criterion at the tree's finest level, and the
  smallest p' for which the FMM-accelerated evaluation has Green's-identity
  error below eps; p_add(p) is the largest such p' over all curves and all eps.

The errors are relative max-norm errors over the test targets. The result is
written to csrc/p_add_table.h (compiled into qbx_default_p_add) and a summary
to p_add_calibration.txt beside this file:

    python -m paper_1602_05301_gb300.calibrate_p_add [--curves 100] [--seed 2016]
"""
from __future__ import annotations

import argparse
import math
import os
import time

import numpy as np
from scipy.special import hankel1

HERE = os.path.dirname(os.path.abspath(__file__))
K = 5.0
EPS_LIST = [10.0 ** -e for e in range(3, 13)]
PANELS = [64, 128, 256, 512]
P_LIST = [2, 4, 6, 8, 10, 12, 14, 16]
P_ADD_MAX = 40


def random_curve(rng):
    from qbx_workloads.geometry import fourier_radial
    delta = rng.uniform(-0.2, 0.2, 12)
    # sin(j t) = cos(j t - pi/2)
    return fourier_radial(delta, np.full(12, -0.5 * np.pi), base=5.0)


_P_FMM_CACHE = {}


def p_fmm_for_eps(eps, kR):
    """Smallest p with max_{n > p} |H_n(3kR)| max_{y <= sqrt2 kR} |J_n(y)| <= eps
    (J_n increases on [0, sqrt2 kR] once n > sqrt2 kR; below that the bound 1
    is used), in log form through mpmath so that no order overflows."""
    import mpmath
    key = (eps, round(kR, 9))
    if key in _P_FMM_CACHE:
        return _P_FMM_CACHE[key]
    mpmath.mp.dps = 20
    b = math.sqrt(2.0) * kR
    lb = []
    for n in range(0, 161):
        v = mpmath.log(abs(mpmath.hankel1(n, 3.0 * kR)))
        if n > b:
            v += mpmath.log(abs(mpmath.besselj(n, b)))
        lb.append(float(v))
    suffix = np.maximum.accumulate(np.array(lb)[::-1])[::-1]   # max over orders >= n
    for p in range(1, 150):
        if suffix[p + 1] <= math.log(eps):
            _P_FMM_CACHE[key] = p
            return p
    raise ValueError("eps %g out of range at kR %g" % (eps, kR))


class PointField:
    """u(x) = sum_m q_m H_0(k|x - x_m|) and its normal derivative."""

    def __init__(self, points, charges):
        self.points, self.charges = np.asarray(points), np.asarray(charges)

    def u(self, x):
        r = np.hypot(*(x[:, None, :] - self.points[None]).transpose(2, 0, 1))
        return (self.charges * hankel1(0, K * r)).sum(axis=1)

    def dudn(self, x, n):
        d = x[:, None, :] - self.points[None]
        r = np.hypot(d[..., 0], d[..., 1])
        nd = d[..., 0] * n[:, None, 0] + d[..., 1] * n[:, None, 1]
        return (self.charges * (-K) * hankel1(1, K * r) * nd / r).sum(axis=1)


class Case:
    """One random curve at one panel count: geometry, targets, exact field."""

    def __init__(self, qbx, gamma, dgamma, n_panels, p, charges, points, rng):
        from qbx_workloads.geometry import discretise_curve
        f = PointField(points, charges)
        gd = discretise_curve(gamma, dgamma, n_panels, 16, k=K)
        gs = discretise_curve(gamma, dgamma, n_panels, 64, k=K)
        n = gd.n
        on = np.arange(0, n, 4)
        pick = rng.choice(n, on.size, replace=True)
        off = rng.uniform(0.02, 0.5, on.size) * gd.panel_h[gd.panel_of_node[pick]]
        near = gd.node_xy[pick] + off[:, None] * gd.normal_xy[pick]
        self.tgt = np.concatenate([gd.node_xy[on], near])
        self.on_node = np.concatenate([on, np.full(near.shape[0], -1)])
        self.on_side = np.ones(self.tgt.shape[0], np.int8)
        self.u_exact = f.u(self.tgt)
        self.sD = f.u(gs.node_xy)
        self.sS = f.dudn(gs.node_xy, gs.normal_xy)
        self.gd, self.gs, self.p, self.qbx = gd, gs, p, qbx
        self.src = dict(q=64, node_xy=gs.node_xy, normal_xy=gs.normal_xy, weight=gs.weight)

    def error(self, mode, p_fmm=0, p_add=0):
        qbx = self.qbx
        lp = qbx.LayerPotential(self.gd.as_dict(), self.p, sides=1, src=self.src)
        try:
            assoc = lp.build(self.tgt, self.on_node, self.on_side, mode=mode, p_fmm=p_fmm,
                             p_add=p_add, n_max=64)
            assert np.all(assoc >= 0), "a test target was not associated with a centre"
            u = lp.eval(sigma_S=self.sS, sigma_D=self.sD, cS=-1.0, cD=1.0)
            kR = None
            if mode == qbx.QBX_FMM:
                t = lp.export_tree()
                kR = 0.5 * K * t["root"][2] / 2 ** (int(t["info"][1]) - 1)
        finally:
            lp.close()
        err = float(np.max(np.abs(u - self.u_exact)) / np.max(np.abs(self.u_exact)))
        return err, kR


def calibrate(n_curves, seed, log):
    from paper_1602_05301_gb300 import build as b
    b.build()
    from paper_1602_05301_gb300 import qbx
    rng = np.random.default_rng(seed)
    curves = []
    for _ in range(n_curves):
        gamma, dgamma = random_curve(rng)
        ang = rng.uniform(0, 2 * np.pi, 2)
        rad = rng.uniform(0.0, 1.5, 2)
        points = np.stack([rad * np.cos(ang), rad * np.sin(ang)], -1)
        charges = (rng.standard_normal(2) + 1j * rng.standard_normal(2)) / np.sqrt(2)
        curves.append((gamma, dgamma, points, charges, int(rng.integers(1 << 30))))
    table = {}
    for p in P_LIST:
        worst, hist, n_meas, t0 = 0, {}, 0, time.time()
        by_eps = {}
        for ci, (gamma, dgamma, points, charges, cseed) in enumerate(curves):
            cases, e_dir = {}, {}
            for eps in EPS_LIST:
                # the coarsest panel count whose direct QBX error is at most eps / 2
                chosen = None
                for npan in PANELS:
                    if npan not in e_dir:
                        cases[npan] = Case(qbx, gamma, dgamma, npan, p, charges, points,
                                               np.random.default_rng(cseed))
                        e_dir[npan] = cases[npan].error(qbx.QBX_DIRECT)[0]
                    if e_dir[npan] <= 0.5 * eps:
                        chosen = npan
                        break
                    if npan == PANELS[-1]:
                        break
                if chosen is None:
                    continue
                case = cases[chosen]
                _, kR = case.error(qbx.QBX_FMM, p_fmm=1, p_add=0)   # tree geometry only
                p_fmm = p_fmm_for_eps(eps, min(kR, 1.0))
                for pa in range(0, P_ADD_MAX + 1):
                    e, _ = case.error(qbx.QBX_FMM, p_fmm=p_fmm, p_add=pa)
                    if e < eps:
                        break
                else:
                    raise RuntimeError("p=%d eps=%g curve %d: no p_add <= %d reaches eps"
                                       % (p, eps, ci, P_ADD_MAX))
                worst = max(worst, pa)
                hist[pa] = hist.get(pa, 0) + 1
                by_eps[eps] = max(by_eps.get(eps, 0), pa)
                n_meas += 1
        table[p] = worst
        log("p = %2d: p_add = %2d  (%d (curve, eps) cases; p' histogram %s; largest p' per "
            "eps %s; %.0f s)" % (p, worst, n_meas, dict(sorted(hist.items())),
                                 {"%.0e" % e: v for e, v in sorted(by_eps.items())},
                                 time.time() - t0))
    return table


def write_outputs(table, n_curves, seed, lines):
    """table: the largest p' measured per calibrated p. The library's table is
    its non-decreasing envelope in p (a larger QBX order never gets a smaller
    p_add; single outliers make the raw maxima non-monotone), and an order
    between calibrated ones takes the value of the next calibrated order."""
    env, run = {}, 0
    for p in sorted(table):
        run = max(run, table[p])
        env[p] = run
    full = []
    for p in range(0, 17):
        nxt = min(q for q in env if q >= max(p, min(env)))
        full.append(env[nxt])
    hdr = os.path.join(HERE, "csrc", "p_add_table.h")
    with open(hdr, "w") as f:
        f.write("// p_add against the QBX order p = 0..16, measured by calibrate_p_add.py\n"
                "// (the experiment of Sec. 7.1: %d random curves r = 5 + sum_j delta_j sin jt,\n"
                "// k = 5, Green's identity at targets near the boundary, seed %d): the\n"
                "// non-decreasing envelope of the largest p' found per calibrated p; orders\n"
                "// between calibrated ones take the value of the next calibrated order.\n"
                "// Generated file: rerun the script instead of editing it.\n" % (n_curves, seed))
        f.write("#pragma once\n")
        f.write("constexpr int kPAddCalibrated[17] = {%s};\n" % ", ".join(str(v) for v in full))
    with open(os.path.join(HERE, "p_add_calibration.txt"), "w") as f:
        f.write("# python -m paper_1602_05301_gb300.calibrate_p_add --curves %d --seed %d\n"
                % (n_curves, seed))
        for ln in lines:
            f.write(ln + "\n")
        f.write("table p=0..16: %s\n" % full)
    return full


def read_summary(path):
    """The per-p maxima and the run's parameters from a summary this script wrote."""
    import re
    table, lines, n_curves, seed = {}, [], None, None
    for ln in open(path):
        ln = ln.rstrip("\n")
        m = re.match(r"# python -m \S+ --curves (\d+) --seed (\d+)", ln)
        if m:
            n_curves, seed = int(m.group(1)), int(m.group(2))
            continue
        m = re.match(r"p = +(\d+): p_add = +(\d+)", ln)
        if m:
            table[int(m.group(1))] = int(m.group(2))
            lines.append(ln)
    return table, n_curves, seed, lines


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--curves", type=int, default=100)
    ap.add_argument("--seed", type=int, default=2016)
    ap.add_argument("--dry", action="store_true", help="print, write nothing")
    ap.add_argument("--from-summary", help="rewrite the outputs from a summary of an earlier run")
    a = ap.parse_args()
    if a.from_summary:
        table, n_curves, seed, lines = read_summary(a.from_summary)
        print("table:", write_outputs(table, n_curves, seed, lines))
        return
    lines = []

    def log(s):
        print(s, flush=True)
        lines.append(s)
    table = calibrate(a.curves, a.seed, log)
    if not a.dry:
        print("table:", write_outputs(table, a.curves, a.seed, lines))


if __name__ == "__main__":
    main()
