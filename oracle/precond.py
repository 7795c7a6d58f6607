"""Circulant (Fourier-diagonal) preconditioner of the normal equations
(oracle; test infrastructure: only the tests, the smoke check and the
benchmark's CPU baseline use this module).

Not in the paper, which solves its problem without a preconditioner; it
serves the Tikhonov CG solve of the reconstruction problem.  Readings:

  * The point-spread function of the normal operator is its response to a
    unit impulse at the image centre c = (N0/2, N1/2, N2/2): h = E0 delta_c,
    E0 = sum_j A_j^H A_j.  A shift-invariant operator would be the circular
    convolution with h rolled so that c moves to the origin; its eigenvalues
    are the DFT of that kernel, hhat[k] = sum_n h[n] exp(-2 pi i k.(n - c)/N).
  * The preconditioner is the inverse of that circulant approximation of
    E0 + lambda I, kept Hermitian and positive: d[k] = 1 / (max(Re hhat[k], 0)
    + lambda), and M r = IDFT(d . DFT(r)).
"""

from __future__ import annotations

import numpy as np


def psf(apply_E0, shape):
    """h = E0 delta at the image centre."""
    d = np.zeros(shape, dtype=np.complex128)
    d[tuple(s // 2 for s in shape)] = 1.0
    return apply_E0(d)


def circulant_diag(apply_E0, shape, lam):
    """d[k] = 1 / (max(Re hhat[k], 0) + lam), hhat the DFT of h with the
    image centre moved to the origin."""
    h = psf(apply_E0, shape)
    hc = np.roll(h, tuple(-(s // 2) for s in shape), axis=(0, 1, 2))
    hhat = np.fft.fftn(hc)
    return 1.0 / (np.maximum(hhat.real, 0.0) + lam)


def apply_circulant(d, r):
    """M r = IDFT(d . DFT(r))."""
    return np.fft.ifftn(d * np.fft.fftn(np.asarray(r, dtype=np.complex128)))
