"""Conjugate gradients on the normal equations (oracle; test infrastructure).

The paper states the motion-corrected reconstruction as a regularised least
squares problem over the stacked nonrigid SENSE operators (the
reconstruction optimisation equation; wavelet-FISTA in the in-vivo study).
The solver here replaces the wavelet L1 term by a Tikhonov term lambda ||x||^2,
whose minimiser solves (sum_j A_j^H A_j + lambda I) x = sum_j A_j^H y_j, and
applies textbook conjugate gradients (Hestenes-Stiefel) to that Hermitian
positive-definite system, with x0 = 0 and the recursive residual relative to
||b|| as the stopping test.
"""

from __future__ import annotations

import numpy as np


def cg(apply_E, b, tol: float = 1e-4, maxit: int = 100, x0=None):
    """Solve E x = b.  Returns (x, iterations, relative residual history)."""
    b = np.asarray(b, dtype=np.complex128)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.complex128)
    r = b - apply_E(x) if x0 is not None else b.copy()
    p = r.copy()
    rr = np.vdot(r, r).real
    bnorm = np.sqrt(np.vdot(b, b).real)
    hist = [np.sqrt(rr) / bnorm if bnorm > 0 else 0.0]
    it = 0
    while it < maxit and hist[-1] > tol:
        Ep = apply_E(p)
        alpha = rr / np.vdot(p, Ep).real
        x = x + alpha * p
        r = r - alpha * Ep
        rr_new = np.vdot(r, r).real
        p = r + (rr_new / rr) * p
        rr = rr_new
        it += 1
        hist.append(np.sqrt(rr) / bnorm)
    return x, it, np.asarray(hist)
