"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module holds geometry discretisation (Gauss-Legendre panels on
parametrised closed curves), densities and target sets only. It contains
none of the layer-potential arithmetic, and neither the CUDA path nor the
oracle is imported here.
"""
from .geometry import (Geometry, gauss_legendre, discretise_curve, discretise_breaks, circle,
                       starfish, fourier_radial, ellipse, concat_geometries)
from .configs import make_config, CONFIG_NAMES

__all__ = ["Geometry", "gauss_legendre", "discretise_curve", "discretise_breaks", "circle",
           "starfish",
           "fourier_radial", "ellipse", "concat_geometries", "make_config", "CONFIG_NAMES"]
