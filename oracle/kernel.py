"""Interpolation kernel of the oracle (FP64).

The paper uses one interpolation kernel c(x) for the Projection/Backprojection
Cores and its Fourier transform C for deapodization (Notations table;
"k-space Gridding": the deapodization divides by the inverse Fourier transform
of the interpolation kernel).  The kernel family is Kaiser-Bessel, the kernel
of Beatty et al. whose notation the paper adapts.

Reading (the paper names the family, not its exact form): the Kaiser-Bessel shape minus its edge value,

    c(u) = I0(beta * sqrt(1 - (2u/W)^2)) - 1   for |u| <= W/2,   0 otherwise,

with u in oversampled-grid units.  Subtracting the edge value makes c
continuous at +-W/2, so the tap rule (< or <=) never matters and the aliasing
sum of its transform converges absolutely.  Its transform has the closed form

    C(nu) = W * [ sinh(z)/z - sin(pi W nu)/(pi W nu) ],  z = sqrt(beta^2 - (pi W nu)^2)

(sinh(z)/z becomes sin(y)/y, y = sqrt((pi W nu)^2 - beta^2), past the knee).
"""

from __future__ import annotations

import math

import numpy as np


def bessel_i0m1(z):
    """I0(z) - 1 from the power series sum_{k>=1} (z/2)^(2k) / (k!)^2.

    Summing from k = 1 avoids the cancellation of I0(z) - 1 near z = 0."""
    z = np.asarray(z, dtype=np.float64)
    q = 0.25 * z * z
    term = q.copy()
    total = q.copy()
    k = 1
    while True:
        k += 1
        term = term * q / float(k * k)
        total = total + term
        if np.all(term <= 1e-18 * np.maximum(total, 1e-300)) or k > 400:
            break
    return total


def bessel_i0(z):
    """Modified Bessel function of the first kind, order 0 (power series)."""
    return 1.0 + bessel_i0m1(z)


def beatty_beta(width: float, osf: float) -> float:
    """Kaiser-Bessel shape parameter of Beatty et al. (2005) for a kernel of
    `width` oversampled-grid units and oversampling ratio `osf`."""
    return math.pi * math.sqrt((width / osf) ** 2 * (osf - 0.5) ** 2 - 0.8)


def kb_kernel(u, width: float, beta: float):
    """c(u): edge-subtracted Kaiser-Bessel kernel, zero for |u| >= W/2."""
    u = np.asarray(u, dtype=np.float64)
    x = 2.0 * u / width
    inside = np.abs(x) < 1.0
    arg = np.where(inside, 1.0 - x * x, 0.0)
    val = bessel_i0m1(beta * np.sqrt(arg))
    return np.where(inside, val, 0.0)


def kb_kernel_ft(nu, width: float, beta: float):
    """C(nu) = integral c(u) exp(-2 pi i nu u) du (real, even), closed form."""
    nu = np.asarray(nu, dtype=np.float64)
    a = math.pi * width * nu
    z2 = beta * beta - a * a
    out = np.empty_like(nu)
    pos = z2 > 0
    zp = np.sqrt(np.where(pos, z2, 1.0))
    zn = np.sqrt(np.where(pos, 1.0, -z2))
    first = np.where(pos, np.sinh(zp) / zp, np.where(zn > 0, np.sin(zn) / np.where(zn > 0, zn, 1.0), 1.0))
    first = np.where(z2 == 0, 1.0, first)
    with np.errstate(invalid="ignore", divide="ignore"):
        second = np.where(a == 0, 1.0, np.sin(a) / np.where(a == 0, 1.0, a))
    out[...] = width * (first - second)
    return out
