"""GB300-native nonrigid SENSE operator (image-space gridding + NUFFT).

Implements the nonrigid SENSE operator A_j = G_j S T_j of Jang, Malave &
Nishimura, "Image-Space Gridding for Nonrigid Motion-Corrected MR Image
Reconstruction" (arXiv 2501.16713) as hand-written sm_103a CUDA kernels plus
cuFFT, behind the C ABI declared in include/nrsense.h.  This package holds the
CUDA sources (csrc/), the nvcc build (_build.py) and a thin ctypes binding
(nrsense.py, including the wavelet-FISTA solver calls), and the host-side
training loop of the CG preconditioner
(precond.py).  Importing the package does not load the library; creating a
Plan does, and raises if the library has not been built.
"""

from .nrsense import (Cnn, Plan, NrsenseError, load, exported_symbols,  # noqa: F401
                      wavelet_forward, wavelet_inverse, wavelet_shrink, translation_xcorr,
                      phase_ramp, kmeans)


def build(verbose: bool = False, force: bool = False) -> str:
    from ._build import build as _b
    return _b(verbose=verbose, force=force)
