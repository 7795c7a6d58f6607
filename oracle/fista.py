"""Wavelet-FISTA for the L1-regularised reconstruction problem (oracle; test
infrastructure: only the tests, the smoke check and the benchmark's CPU
baseline use this module).

The reconstruction problem (reconstruction optimisation equation) is

    minimise  F(x) = f(x) + g(x),   f(x) = sum_j ||y_j - A_j x||_2^2,
                                    g(x) = lambda ||W x||_1,

with W a sparsifying transform; the paper solves it with wavelet-FISTA
(Beck and Teboulle's fast iterative shrinkage-thresholding), in the in-vivo
study and in Appendix 1 (400 iterations, lambda = 1e-6, for a warp-only
operator q = T p).  The paper does not name the wavelet.  Readings taken here:

  * W is the orthonormal separable 3D Haar transform with `levels` levels of
    the standard (Mallat) pyramid: each level splits the current
    approximation cube along all three axes into eight sub-bands, low-pass
    (a + b)/sqrt(2) in the first half of each axis and high-pass
    (a - b)/sqrt(2) in the second half.  Every axis length must be divisible
    by 2^levels; levels = 0 is the identity.  W is real and applied to the
    real and imaginary parts alike, so W^H = W^T = W^{-1}.
  * ||c||_1 sums the moduli of the complex coefficients, every coefficient
    (the coarsest approximation included); its proximal map with weight tau
    is the complex soft threshold c max(0, 1 - tau / |c|).
  * f carries no factor 1/2 (as printed), so grad f(x) = 2 (E0 x - b) with
    E0 = sum_j A_j^H A_j and b = sum_j A_j^H y_j, and its Lipschitz constant
    is L = 2 lambda_max(E0).
  * FISTA with constant step 1/L (Beck and Teboulle's constant-step
    variant): z_1 = x_0, t_1 = 1;  x_k = prox_{g/L}(z_k - grad f(z_k) / L),
    t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2,
    z_{k+1} = x_k + ((t_k - 1) / t_{k+1}) (x_k - x_{k-1}).
    With W orthonormal, prox_{g/L}(v) = W^H soft(W v, lambda / L).
  * lambda_max(E0) is estimated by power iteration from a caller-given start
    vector (the Rayleigh quotient of the last iterate).
"""

from __future__ import annotations

import numpy as np

SQRT_HALF = np.sqrt(0.5)


def _check_levels(shape, levels):
    if levels < 0:
        raise ValueError("levels must be >= 0")
    for n in shape:
        if n % (1 << levels):
            raise ValueError(f"axis length {n} not divisible by 2^{levels}")


def haar_forward(x, levels):
    """W x: the orthonormal 3D Haar pyramid, coefficients in Mallat layout
    (level-1 details fill all but the first half-cube, the level-2 details
    the next, and the last approximation sits in the corner cube)."""
    c = np.array(x, dtype=np.complex128)
    _check_levels(c.shape, levels)
    m = list(c.shape)
    for _ in range(levels):
        cube = c[:m[0], :m[1], :m[2]]
        for ax in range(3):
            even = np.take(cube, np.arange(0, m[ax], 2), axis=ax)
            odd = np.take(cube, np.arange(1, m[ax], 2), axis=ax)
            cube = np.concatenate(((even + odd) * SQRT_HALF, (even - odd) * SQRT_HALF), axis=ax)
        c[:m[0], :m[1], :m[2]] = cube
        m = [v // 2 for v in m]
    return c


def haar_inverse(c, levels):
    """W^H c = W^{-1} c: undo the pyramid from the coarsest level out."""
    x = np.array(c, dtype=np.complex128)
    _check_levels(x.shape, levels)
    for lev in range(levels, 0, -1):
        m = [v >> (lev - 1) for v in x.shape]
        cube = x[:m[0], :m[1], :m[2]]
        for ax in range(3):
            h = m[ax] // 2
            low = np.take(cube, np.arange(0, h), axis=ax)
            high = np.take(cube, np.arange(h, m[ax]), axis=ax)
            out = np.empty_like(cube)
            idx_e = [slice(None)] * 3
            idx_o = [slice(None)] * 3
            idx_e[ax] = slice(0, m[ax], 2)
            idx_o[ax] = slice(1, m[ax], 2)
            out[tuple(idx_e)] = (low + high) * SQRT_HALF
            out[tuple(idx_o)] = (low - high) * SQRT_HALF
            cube = out
        x[:m[0], :m[1], :m[2]] = cube
    return x


def soft_threshold(c, tau):
    """Proximal map of tau |.| on complex numbers: shrink the modulus by tau,
    keep the phase, zero below tau."""
    c = np.asarray(c, dtype=np.complex128)
    mag = np.abs(c)
    scale = np.where(mag > tau, 1.0 - tau / np.where(mag > 0, mag, 1.0), 0.0)
    return c * scale


def wavelet_l1(x, levels):
    """||W x||_1 (sum of coefficient moduli)."""
    return float(np.abs(haar_forward(x, levels)).sum())


def prox_wavelet_l1(v, tau, levels):
    """argmin_u 1/2 ||u - v||^2 + tau ||W u||_1 = W^H soft(W v, tau) (W orthonormal)."""
    return haar_inverse(soft_threshold(haar_forward(v, levels), tau), levels)


def objective(residual_sq, x, lam, levels):
    """F(x) from ||y - A x||^2 (computed by the caller) and x."""
    return float(residual_sq) + lam * wavelet_l1(x, levels)


def momentum(maxit):
    """(t_k) for k = 1 .. maxit + 1 and mu_k = (t_k - 1) / t_{k+1}, k = 1 .. maxit."""
    t = [1.0]
    for _ in range(maxit):
        t.append((1.0 + np.sqrt(1.0 + 4.0 * t[-1] * t[-1])) / 2.0)
    t = np.asarray(t)
    return t, (t[:-1] - 1.0) / t[1:]


def fista(apply_E0, b, lam, L, levels, maxit, x0=None, callback=None):
    """Constant-step FISTA on F(x) = ||y - A x||^2 + lam ||W x||_1.

    apply_E0: x -> sum_j A_j^H A_j x;  b = sum_j A_j^H y_j;  L >= 2 lambda_max(E0).
    Returns (x_maxit, history of ||x_k - x_{k-1}|| / ||x_k|| for k = 1..maxit).
    callback(k, x_k), if given, is called after every iteration."""
    b = np.asarray(b, dtype=np.complex128)
    x_prev = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.complex128)
    z = x_prev.copy()
    _, mu = momentum(maxit)
    tau = lam / L
    hist = []
    for k in range(maxit):
        grad = 2.0 * (apply_E0(z) - b)
        x = prox_wavelet_l1(z - grad / L, tau, levels)
        z = x + mu[k] * (x - x_prev)
        nx = np.linalg.norm(x)
        hist.append(np.linalg.norm(x - x_prev) / nx if nx > 0 else 0.0)
        x_prev = x
        if callback is not None:
            callback(k + 1, x)
    return x_prev, np.asarray(hist)


def max_eig(apply_E0, v0, iters):
    """Power iteration on the Hermitian positive semi-definite E0 from v0;
    returns the Rayleigh quotient <v, E0 v> / <v, v> of the last normalised
    iterate and that iterate."""
    v = np.array(v0, dtype=np.complex128)
    v /= np.linalg.norm(v)
    rq = 0.0
    for _ in range(iters):
        w = apply_E0(v)
        rq = float(np.vdot(v, w).real)
        nw = np.linalg.norm(w)
        if nw == 0:
            return 0.0, v
        v = w / nw
    return rq, v
