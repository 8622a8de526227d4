"""Geometries for the tests of Conditions 1-4 (Sec. 3.3) and of refinement,
with the flags that the paper's definitions give in closed form."""
from __future__ import annotations

import numpy as np

from qbx_workloads import circle, concat_geometries, discretise_breaks, discretise_curve


def two_circles(gap, n1, n2, k=1.0, q=16):
    """Unit circles centred at (0, 0) and (2 + gap, 0), n1 and n2 equal panels."""
    g1 = discretise_curve(*circle(1.0), n1, q, k=k)
    g2 = discretise_curve(*circle(1.0, (2.0 + gap, 0.0)), n2, q, k=k)
    return concat_geometries([g1, g2])


def expected_two_circles(geom, n1, n2, gap, sides=2):
    """Flags of two circles (unit radius, centres (0,0) and (2+gap, 0)) from the
    closed-form distance of a point to a circular arc: Condition 1 for panels of
    either circle whose centres come within h/2 of the other circle; Condition 3
    for arcs within h_m/4 of a centre of the other circle (a circle's own
    centres keep their distance h/2 from it)."""
    q = geom.q
    h = geom.panel_h
    C = [np.array([0.0, 0.0]), np.array([2.0 + gap, 0.0])]
    n_p = [n1, n2]
    off = [0, n1]
    flags = np.zeros(n1 + n2, np.int32)
    for a in range(2):
        b = 1 - a
        P = np.arange(off[a], off[a] + n_p[a])
        idx = (P[:, None] * q + np.arange(q)[None, :]).ravel()
        hh = np.repeat(h[P], q)
        for s in ((1.0, -1.0) if sides == 2 else (1.0,)):
            c = geom.node_xy[idx] + s * 0.5 * hh[:, None] * geom.normal_xy[idx]
            d = c - C[b]
            r = np.hypot(d[:, 0], d[:, 1])
            hit1 = r - 1.0 < 0.5 * hh
            flags[np.unique(idx[hit1] // q)] |= 1
            ang = np.arctan2(d[:, 1], d[:, 0])
            for pb in range(n_p[b]):
                Q = off[b] + pb
                t0 = 2 * np.pi * pb / n_p[b]
                t1 = 2 * np.pi * (pb + 1) / n_p[b]
                inside = (ang - t0) % (2 * np.pi) <= (t1 - t0)
                e0 = C[b] + np.array([np.cos(t0), np.sin(t0)])
                e1 = C[b] + np.array([np.cos(t1), np.sin(t1)])
                dd = np.where(inside, np.abs(r - 1.0),
                              np.minimum(np.hypot(*(c - e0).T), np.hypot(*(c - e1).T)))
                if np.any(dd < 0.25 * h[Q]):
                    flags[Q] |= 4
    return flags


def uneven_circle(ratio=3.0, n=24, q=16, k=1.0):
    """A unit circle with equal panels except that panel 5 is `ratio` times as
    long as its neighbours (it takes the angle of several)."""
    base = 2 * np.pi / (n + ratio - 1)
    lens = np.full(n, base)
    lens[5] = ratio * base
    tb = np.concatenate([[0.0], np.cumsum(lens)])
    return discretise_breaks(*circle(1.0), tb, q, k=k)
