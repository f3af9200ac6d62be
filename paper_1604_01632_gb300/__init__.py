"""GB300 (sm_103a) free-surface lattice Boltzmann method with the enhanced bubble
model of Anderl et al. (arXiv:1604.01632).

The compute path is the CUDA library libfsl.so (C ABI in include/fsl.h); the
module `fsl` is its Python binding and `scenarios` builds seeded synthetic
inputs shaped like the paper's workloads.
"""
from . import scenarios  # noqa: F401

__all__ = ["scenarios", "fsl", "build"]
