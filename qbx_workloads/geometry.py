"""Gauss-Legendre panel discretisation of parametrised closed curves.

Each curve gamma(t), t in [0, 2 pi), counter-clockwise, is cut into panels of
equal parameter length; every panel carries the q-point Gauss-Legendre rule
mapped to its parameter interval. The quadrature weight of node j of panel k
is w_j (dt/2) |gamma'(t_j)| (an arclength quadrature rule on the panel), the
panel length h_k is the sum of its weights, and the unit normal
(gamma_y', -gamma_x') / |gamma'| points out of the enclosed region.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Callable, List

import numpy as np


def gauss_legendre(q: int):
    """Nodes and weights of the q-point Gauss-Legendre rule on [-1, 1]."""
    x, w = np.polynomial.legendre.leggauss(q)
    return x, w


@dataclass
class Geometry:
    node_xy: np.ndarray          # [n, 2]
    normal_xy: np.ndarray        # [n, 2] outward unit normals
    weight: np.ndarray           # [n] arclength quadrature weights
    panel_of_node: np.ndarray    # [n] int64
    panel_h: np.ndarray          # [n_panels] panel arclengths
    param_t: np.ndarray          # [n] curve parameter of each node
    q: int
    panel_offset: np.ndarray     # [n_curves + 1] int64, panels of curve c are [off[c], off[c+1])
    k: np.ndarray = field(default_factory=lambda: np.ones(1))  # [n_curves] wavenumbers

    @property
    def n(self) -> int:
        return self.node_xy.shape[0]

    @property
    def n_panels(self) -> int:
        return self.panel_h.shape[0]

    @property
    def n_curves(self) -> int:
        return self.panel_offset.shape[0] - 1

    def node_offset(self) -> np.ndarray:
        return self.panel_offset * self.q

    def as_dict(self, curve: int | None = None) -> dict:
        """Plain arrays (optionally one curve of a batch) with that curve's k."""
        if curve is None:
            assert self.n_curves == 1 or np.all(self.k == self.k[0])
            return dict(node_xy=self.node_xy, normal_xy=self.normal_xy, weight=self.weight,
                        panel_of_node=self.panel_of_node, panel_h=self.panel_h,
                        k=float(self.k[0]), q=self.q, panel_offset=self.panel_offset)
        p0, p1 = int(self.panel_offset[curve]), int(self.panel_offset[curve + 1])
        n0, n1 = p0 * self.q, p1 * self.q
        return dict(node_xy=self.node_xy[n0:n1], normal_xy=self.normal_xy[n0:n1],
                    weight=self.weight[n0:n1], panel_of_node=self.panel_of_node[n0:n1] - p0,
                    panel_h=self.panel_h[p0:p1], k=float(self.k[curve]), q=self.q,
                    panel_offset=np.array([0, p1 - p0], dtype=np.int64))


def discretise_curve(gamma: Callable, dgamma: Callable, n_panels: int, q: int,
                     k: float = 1.0) -> Geometry:
    x, w = gauss_legendre(q)
    dt = 2.0 * np.pi / n_panels
    t0 = np.arange(n_panels) * dt
    t = (t0[:, None] + (x[None, :] + 1.0) * 0.5 * dt).reshape(-1)
    xy = np.stack(gamma(t), axis=-1)
    d = np.stack(dgamma(t), axis=-1)
    speed = np.hypot(d[:, 0], d[:, 1])
    normal = np.stack([d[:, 1] / speed, -d[:, 0] / speed], axis=-1)
    weight = (np.tile(w, n_panels) * 0.5 * dt) * speed
    panel_of_node = np.repeat(np.arange(n_panels, dtype=np.int64), q)
    panel_h = weight.reshape(n_panels, q).sum(axis=1)
    return Geometry(node_xy=np.ascontiguousarray(xy), normal_xy=np.ascontiguousarray(normal),
                    weight=weight, panel_of_node=panel_of_node, panel_h=panel_h, param_t=t, q=q,
                    panel_offset=np.array([0, n_panels], dtype=np.int64),
                    k=np.array([float(k)]))


def discretise_breaks(gamma: Callable, dgamma: Callable, t_breaks, q: int,
                      k: float = 1.0) -> Geometry:
    """Like discretise_curve, with the panels between the given parameter values
    t_breaks[0] < ... < t_breaks[n] (t_breaks[n] = t_breaks[0] + 2 pi)."""
    x, w = gauss_legendre(q)
    tb = np.asarray(t_breaks, dtype=np.float64)
    dt = np.diff(tb)
    n_panels = dt.size
    t = (tb[:-1, None] + (x[None, :] + 1.0) * 0.5 * dt[:, None]).reshape(-1)
    xy = np.stack(gamma(t), axis=-1)
    d = np.stack(dgamma(t), axis=-1)
    speed = np.hypot(d[:, 0], d[:, 1])
    normal = np.stack([d[:, 1] / speed, -d[:, 0] / speed], axis=-1)
    weight = (np.tile(w, n_panels) * 0.5 * np.repeat(dt, q)) * speed
    panel_of_node = np.repeat(np.arange(n_panels, dtype=np.int64), q)
    panel_h = weight.reshape(n_panels, q).sum(axis=1)
    return Geometry(node_xy=np.ascontiguousarray(xy), normal_xy=np.ascontiguousarray(normal),
                    weight=weight, panel_of_node=panel_of_node, panel_h=panel_h, param_t=t, q=q,
                    panel_offset=np.array([0, n_panels], dtype=np.int64),
                    k=np.array([float(k)]))


def circle(radius: float = 1.0, centre=(0.0, 0.0)):
    cx, cy = centre

    def g(t):
        return cx + radius * np.cos(t), cy + radius * np.sin(t)

    def dg(t):
        return -radius * np.sin(t), radius * np.cos(t)
    return g, dg


def fourier_radial(a, phi, base: float = 1.0, centre=(0.0, 0.0)):
    """r(t) = base + sum_m a_m cos(m t + phi_m), m = 1..len(a)."""
    a = np.asarray(a, dtype=float)
    phi = np.asarray(phi, dtype=float)
    m = np.arange(1, a.size + 1)
    cx, cy = centre

    def r(t):
        return base + np.sum(a[:, None] * np.cos(m[:, None] * t[None, :] + phi[:, None]), axis=0)

    def dr(t):
        return -np.sum(a[:, None] * m[:, None] * np.sin(m[:, None] * t[None, :] + phi[:, None]),
                       axis=0)

    def g(t):
        rr = r(t)
        return cx + rr * np.cos(t), cy + rr * np.sin(t)

    def dg(t):
        rr, d = r(t), dr(t)
        return d * np.cos(t) - rr * np.sin(t), d * np.sin(t) + rr * np.cos(t)
    return g, dg


def starfish(amplitude: float = 0.3, arms: int = 5, base: float = 1.0):
    """r(t) = base + amplitude cos(arms t)."""
    a = np.zeros(arms)
    a[arms - 1] = amplitude
    return fourier_radial(a, np.zeros(arms), base)


def ellipse(a: float, b: float, rotation: float = 0.0, centre=(0.0, 0.0)):
    ca, sa = np.cos(rotation), np.sin(rotation)
    cx, cy = centre

    def g(t):
        x, y = a * np.cos(t), b * np.sin(t)
        return cx + ca * x - sa * y, cy + sa * x + ca * y

    def dg(t):
        x, y = -a * np.sin(t), b * np.cos(t)
        return ca * x - sa * y, sa * x + ca * y
    return g, dg


def concat_geometries(parts: List[Geometry]) -> Geometry:
    q = parts[0].q
    assert all(g.q == q for g in parts)
    offs = [0]
    pon = []
    for g in parts:
        pon.append(g.panel_of_node + offs[-1])
        offs.append(offs[-1] + g.n_panels)
    return Geometry(node_xy=np.concatenate([g.node_xy for g in parts]),
                    normal_xy=np.concatenate([g.normal_xy for g in parts]),
                    weight=np.concatenate([g.weight for g in parts]),
                    panel_of_node=np.concatenate(pon),
                    panel_h=np.concatenate([g.panel_h for g in parts]),
                    param_t=np.concatenate([g.param_t for g in parts]), q=q,
                    panel_offset=np.array(offs, dtype=np.int64),
                    k=np.concatenate([g.k for g in parts]))
