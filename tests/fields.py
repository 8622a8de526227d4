"""Known Helmholtz fields for the pins (closed forms and Green's identity data).

Computed with scipy.special, independently of the oracle's special functions.
"""
from __future__ import annotations

import numpy as np
from scipy.special import h1vp, hankel1, jv, jvp


def circle_slp_mode(n, k, R, xy):
    """S[e^{i n t}] on the circle of radius R: (i pi R / 2) J_n(k r<) H_n(k r>) e^{i n th}.

    (Graf's expansion of H_0 integrated against a single Fourier mode.) Targets
    on the circle (r == R) give the continuous on-surface value."""
    r = np.hypot(xy[:, 0], xy[:, 1])
    th = np.arctan2(xy[:, 1], xy[:, 0])
    rl, rg = np.minimum(r, R), np.maximum(r, R)
    return 1j * np.pi * R / 2 * jv(n, k * rl) * hankel1(n, k * rg) * np.exp(1j * n * th)


def circle_dlp_mode(n, k, R, xy, side):
    """D[e^{i n t}] on the circle: exterior (i pi k R/2) J_n'(kR) H_n(kr) e^{inth},
    interior (i pi k R/2) J_n(kr) H_n'(kR) e^{inth}; ``side`` (+1/-1) selects the
    one-sided limit for targets on the circle."""
    r = np.hypot(xy[:, 0], xy[:, 1])
    th = np.arctan2(xy[:, 1], xy[:, 0])
    ext = 1j * np.pi * k * R / 2 * jvp(n, k * R) * hankel1(n, k * r) * np.exp(1j * n * th)
    inn = 1j * np.pi * k * R / 2 * jv(n, k * r) * h1vp(n, k * R) * np.exp(1j * n * th)
    return np.where(side > 0, ext, inn)


class PointSourceField:
    """u(x) = sum_m q_m H_0(k |x - x_m|), radiating, for Green's identity
    u = D[u] - S[du/dn] outside the curve and 0 inside (Sec. 8.1 of the paper)."""

    def __init__(self, k, points, charges):
        self.k = float(k)
        self.points = np.asarray(points, dtype=float)
        self.charges = np.asarray(charges, dtype=complex)

    def u(self, x):
        d = x[:, None, :] - self.points[None]
        r = np.hypot(d[..., 0], d[..., 1])
        return (self.charges * hankel1(0, self.k * r)).sum(axis=1)

    def dudn(self, x, n):
        d = x[:, None, :] - self.points[None]
        r = np.hypot(d[..., 0], d[..., 1])
        nd = d[..., 0] * n[:, None, 0] + d[..., 1] * n[:, None, 1]
        return (self.charges * (-self.k) * hankel1(1, self.k * r) * nd / r).sum(axis=1)
