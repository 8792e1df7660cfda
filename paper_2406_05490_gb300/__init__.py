"""GB300 (sm_103a) implementation of the Z-Model interface-velocity hot path exercised by the
Beatnik mini-application (arXiv:2406.05490): stencils, the exact all-pairs Birkhoff-Rott sum,
the FFT Riesz-transform velocity and SSP-RK3, behind the C ABI in include/zm.h.

Importing the package does not load the CUDA library; ``paper_2406_05490_gb300.zm`` does on
first use and raises if it has not been built.
"""
__all__ = ["inputs", "zm", "build"]
