"""The five synthetic workloads (seeded with numpy PCG64, seed = 1000 + config number).

1. circle-k1      : circle R=1, k=1, 32 panels x 16 nodes, single layer, sigma = cos(3 t),
                    p=8, centres on both sides; targets: every node on both sides
                    (on-surface limits) + 500 points on r=0.5 + 500 on r=2. Direct QBX.
2. starfish-k10   : r(t)=1+0.3cos(5t), k=10, 512 panels x 16 (8192 nodes), combined field
                    D[s] + i k S[s], s = random complex Fourier modes |n|<=20, p=12,
                    p_fmm=20, 316x316 grid on [-2,2]^2 (99 856 targets), both sides.
3. starfish-k50   : as 2 with k=50, 8192 panels x 16 (131 072 nodes), p=16, p_fmm=30.
4. batch-256      : 256 curves r(t)=1+sum_{m<=5} a_m cos(m t + phi_m), a_m~U(0,0.05),
                    panels U{16..1024} raised to ceil(k L / 5), k~U(1,40), combined field,
                    random densities, targets = every node (exterior limit), p=12, p_fmm=20.
5. ellipses-200   : 200 non-overlapping ellipses in [0,100]^2, 2^20 nodes, k=20, double
                    layer, p=16, p_fmm=30, 9e5 uniform + 1e5 near-surface targets.
"""
from __future__ import annotations

import math

import numpy as np

from .geometry import (Geometry, circle, concat_geometries, discretise_curve, ellipse,
                       fourier_radial, starfish)

CONFIG_NAMES = {1: "circle-k1", 2: "starfish-k10", 3: "starfish-k50", 4: "batch-256",
                5: "ellipses-200"}


def _fourier_density(t, rng, modes=20):
    n = np.arange(-modes, modes + 1)
    c = (rng.standard_normal(n.size) + 1j * rng.standard_normal(n.size)) / math.sqrt(2.0)
    return (c[None, :] * np.exp(1j * n[None, :] * t[:, None])).sum(axis=1)


def grid_targets(m: int, lo: float, hi: float) -> np.ndarray:
    g = np.linspace(lo, hi, m)
    X, Y = np.meshgrid(g, g, indexing="xy")
    return np.stack([X.ravel(), Y.ravel()], axis=-1)


def on_surface_targets(geom: Geometry, sides=(1, -1)):
    """Every node as an on-surface target, once per requested side."""
    n = geom.n
    xy = np.concatenate([geom.node_xy for _ in sides])
    node = np.concatenate([np.arange(n, dtype=np.int64) for _ in sides])
    side = np.concatenate([np.full(n, s, dtype=np.int8) for s in sides])
    return xy, node, side


def _workload(name, geom, p, p_fmm, sigma_S, sigma_D, cS, cD, tgt_xy, on_node=None,
              on_side=None, sides=2, mode="fmm", eps_assoc=0.1, **extra):
    n_t = tgt_xy.shape[0]
    if on_node is None:
        on_node = np.full(n_t, -1, dtype=np.int64)
        on_side = np.zeros(n_t, dtype=np.int8)
    w = dict(name=name, geom=geom, p=p, p_fmm=p_fmm, sigma_S=sigma_S, sigma_D=sigma_D,
             cS=complex(cS), cD=complex(cD), tgt_xy=np.ascontiguousarray(tgt_xy, dtype=float),
             on_surface_node=on_node, on_surface_side=on_side, sides=sides, mode=mode,
             eps_assoc=eps_assoc)
    w.update(extra)
    return w


def config1(rng):
    g, dg = circle(1.0)
    geom = discretise_curve(g, dg, 32, 16, k=1.0)
    sigma = np.cos(3.0 * geom.param_t).astype(np.complex128)
    on_xy, on_node, on_side = on_surface_targets(geom)
    th = 2.0 * np.pi * np.arange(500) / 500.0
    ring = lambda r: np.stack([r * np.cos(th), r * np.sin(th)], axis=-1)
    tgt = np.concatenate([on_xy, ring(0.5), ring(2.0)])
    node = np.concatenate([on_node, np.full(1000, -1, dtype=np.int64)])
    side = np.concatenate([on_side, np.zeros(1000, dtype=np.int8)])
    return _workload(CONFIG_NAMES[1], geom, 8, 0, sigma, None, 1.0, 0.0, tgt, node, side,
                     mode="direct")


def _starfish_config(num, rng, k, n_panels, p, p_fmm, grid=316):
    g, dg = starfish(0.3, 5)
    geom = discretise_curve(g, dg, n_panels, 16, k=k)
    sigma = _fourier_density(geom.param_t, rng)
    tgt = grid_targets(grid, -2.0, 2.0)
    return _workload(CONFIG_NAMES[num], geom, p, p_fmm, sigma, sigma, 1j * k, 1.0, tgt)


def config2(rng, grid=316):
    return _starfish_config(2, rng, 10.0, 512, 12, 20, grid)


def config3(rng, grid=316):
    return _starfish_config(3, rng, 50.0, 8192, 16, 30, grid)


def config4(rng, n_curves=256):
    parts, dens = [], []
    raised = 0
    for _ in range(n_curves):
        a = rng.uniform(0.0, 0.05, 5)
        phi = rng.uniform(0.0, 2.0 * np.pi, 5)
        k = rng.uniform(1.0, 40.0)
        n_panels = int(rng.integers(16, 1025))
        g, dg = fourier_radial(a, phi)
        # panel size bounded by the wavelength (Condition 4: k * max h <= 5); the
        # panels are equal in the parameter, so their lengths differ slightly
        geom = discretise_curve(g, dg, n_panels, 16, k=k)
        if k * geom.panel_h.max() > 5.0:
            raised += 1
            while k * geom.panel_h.max() > 5.0:
                n_panels = int(math.ceil(n_panels * k * geom.panel_h.max() / 5.0)) + 1
                geom = discretise_curve(g, dg, n_panels, 16, k=k)
        parts.append(geom)
        dens.append(_fourier_density(geom.param_t, rng))
    geom = concat_geometries(parts)
    sigma = np.concatenate(dens)
    # combined field D[s] + i k_c S[s] per curve: the factor i k_c is folded into sigma_S
    ik = np.repeat(1j * geom.k, np.diff(geom.panel_offset) * geom.q)
    xy, node, side = on_surface_targets(geom, sides=(1,))
    return _workload(CONFIG_NAMES[4], geom, 12, 20, ik * sigma, sigma, 1.0, 1.0, xy, node, side,
                     sides=1, panels_raised=raised)


def config5(rng, n_ellipses=200, total_panels=65536, n_uniform=900_000, n_near=100_000):
    axes = rng.uniform(0.5, 2.0, (n_ellipses, 2))
    rot = rng.uniform(0.0, np.pi, n_ellipses)
    rad = axes.max(axis=1)
    ctr = []
    for i in range(n_ellipses):
        while True:
            c = rng.uniform(rad[i], 100.0 - rad[i], 2)
            if all(np.hypot(*(c - ctr[j])) >= rad[i] + rad[j] + 1.0 for j in range(len(ctr))):
                ctr.append(c)
                break
    # Ramanujan's perimeter approximation, then panels by largest remainder
    a, b = axes[:, 0], axes[:, 1]
    hh = ((a - b) / (a + b)) ** 2
    per = np.pi * (a + b) * (1 + 3 * hh / (10 + np.sqrt(4 - 3 * hh)))
    share = total_panels * per / per.sum()
    npan = np.floor(share).astype(int)
    rem = total_panels - npan.sum()
    npan[np.argsort(-(share - npan))[:rem]] += 1
    parts = []
    for i in range(n_ellipses):
        g, dg = ellipse(a[i], b[i], rot[i], ctr[i])
        parts.append(discretise_curve(g, dg, int(npan[i]), 16, k=20.0))
    geom = concat_geometries(parts)
    dens = []
    for gpart in parts:
        dens.append(_fourier_density(gpart.param_t, rng))
    sigma = np.concatenate(dens)
    uni = rng.uniform(0.0, 100.0, (n_uniform, 2))
    nodes = rng.integers(0, geom.n, n_near)
    off = rng.uniform(0.0, 0.5, n_near) * geom.panel_h[geom.panel_of_node[nodes]]
    sgn = np.where(rng.random(n_near) < 0.5, 1.0, -1.0)
    near = geom.node_xy[nodes] + (sgn * off)[:, None] * geom.normal_xy[nodes]
    tgt = np.concatenate([uni, near])
    return _workload(CONFIG_NAMES[5], geom, 16, 30, None, sigma, 0.0, 1.0, tgt)


def make_config(num: int, **kw) -> dict:
    rng = np.random.Generator(np.random.PCG64(1000 + num))
    return {1: config1, 2: config2, 3: config3, 4: config4, 5: config5}[num](rng, **kw)
