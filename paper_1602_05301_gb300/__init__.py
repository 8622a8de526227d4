"""GB300 (sm_103a) FMM-accelerated Global QBX for 2D Helmholtz layer potentials.

The compute path is the CUDA library libqbx_gb300.so (C ABI in include/qbx.h);
this package holds its build script and a ctypes binding.
"""
from .qbx import (LayerPotential, QBXError, QBX_DIRECT, QBX_FMM, QBX_FP64, QBX_MIXED,
                  qbx_destroy, qbx_geometry_create, qbx_layer_potential_eval, qbx_tree_build)

__all__ = ["LayerPotential", "QBXError", "QBX_DIRECT", "QBX_FMM", "QBX_FP64", "QBX_MIXED",
           "qbx_destroy", "qbx_geometry_create", "qbx_layer_potential_eval", "qbx_tree_build"]
