"""GB300 (sm_103a) implementation of DAMAS on a wavelet-compressed computational grid.

The computation lives in libdamas.so (CUDA kernels behind the C ABI of
include/damas.h); `damas` is its Python binding.
"""
from . import damas  # noqa: F401
from .damas import (Context, Geometry, System, das_map, damas_build_psf, damas_build_psf_dr, damas_divide,  # noqa: F401
                    damas_gather, damas_lda,
                    damas_scatter_power, damas_solve, solve_bin, wavelet_compress_grid)
