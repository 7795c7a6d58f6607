"""Exact references, closed forms and dense matrices (oracle; test infra).

These pin the step-by-step operators of operators.py to things other than
themselves:

* warp_exact:   the displacement-field warp m_j[r] = m(r + d[r]) (section
                "Displacement Fields") evaluated exactly by trigonometric
                interpolation of m, i.e. the continuous band-limited image the
                NUFFT view of the warp samples (same section: voxel locations
                of the warped image are non-Cartesian points on m's grid).
* nudft:        the non-uniform DFT that inverse k-space gridding approximates.
* warp_eigs_constant: for a spatially constant displacement the gridded T is
                shift invariant; its Fourier multiplier in closed form.
* alias_eps:    the rigorous aliasing bound of the gridded operators against
                the exact ones (Poisson summation of the kernel).
* dense_*:      each factor of the process diagrams as an explicit matrix built
                from its formula, composed by matrix products, on tiny grids.
"""

from __future__ import annotations

import numpy as np

from .kernel import kb_kernel, kb_kernel_ft
from .operators import Geometry


def _axis_phase(freqs, pos, n):
    """exp(+2 pi i k p / n) as (P, K)."""
    return np.exp(2j * np.pi * np.outer(pos, freqs) / n)


def warp_exact(geo: Geometry, x, d):
    """T_exact x[n] = (1/N^3) sum_{k in K_N^3} X[k] exp(2 pi i k.(n + d[n]) / N).

    Brute force O(N^3 * N^3) but factorised per axis; for N <= 16."""
    x = np.asarray(x, dtype=np.complex128).reshape(geo.shape)
    X = np.fft.fftn(x)
    n = np.stack(np.meshgrid(*[np.arange(s, dtype=np.float64) for s in geo.shape],
                             indexing="ij")).reshape(3, -1)
    p = n + np.asarray(d, dtype=np.float64).reshape(3, -1)
    E = [_axis_phase(geo.kspace_freqs(a), p[a], geo.shape[a]) for a in range(3)]
    out = np.einsum("abc,pa,pb,pc->p", X, E[0], E[1], E[2], optimize=True)
    return (out / np.prod(geo.shape)).reshape(geo.shape)


def nudft(geo: Geometry, v, omega):
    """y_s = sum_{n' in K_N^3} v[n'] exp(-i omega_s . n'), n' = n - N/2."""
    v = np.asarray(v, dtype=np.complex128).reshape(geo.shape)
    om = np.asarray(omega, dtype=np.float64).reshape(-1, 3)
    E = [np.exp(-1j * np.outer(om[:, a], geo.centred_index(a).astype(np.float64)))
         for a in range(3)]
    return np.einsum("abc,pa,pb,pc->p", v, E[0], E[1], E[2], optimize=True)


def _shifted_kernel_sum(k, phi, geo: Geometry, axis):
    """sum_{t in phi + Z, |t| < W/2} c(t) exp(-2 pi i k t / G)."""
    W = geo.width
    js = np.arange(-W, W + 1)
    t = phi + js
    keep = np.abs(t) < W / 2
    t = t[keep]
    ct = kb_kernel(t, W, geo.beta)
    return np.exp(-2j * np.pi * np.outer(k, t) / geo.grid[axis]) @ ct


def warp_eigs_constant(geo: Geometry, dvec):
    """Fourier multiplier lambda_k of T for the constant displacement dvec:
    T x = ifftn(fftn(x) * lambda).  Per axis
      lambda_k(d) = exp(2 pi i k d / N) * [sum_{t in phi+Z} c(t) e^{-2 pi i k t/G}] / C(k/G),
    phi = frac(sigma d); the 3D multiplier is the product over axes."""
    lam = np.ones(geo.shape, dtype=np.complex128)
    for a in range(3):
        k = geo.kspace_freqs(a).astype(np.float64)
        sd = geo.osf * float(dvec[a])
        phi = sd - np.floor(sd)
        s = _shifted_kernel_sum(k, phi, geo, a)
        la = np.exp(2j * np.pi * k * float(dvec[a]) / geo.shape[a]) * s / kb_kernel_ft(
            k / geo.grid[a], geo.width, geo.beta)
        shp = [1, 1, 1]
        shp[a] = -1
        lam = lam * la.reshape(shp)
    return lam


def alias_eps(geo: Geometry, lmax: int = 10000):
    """eps1 = max_{|nu| <= 1/(2 sigma)} sum_{l != 0} |C(nu + l)| / C(nu), per
    axis (same for all axes), plus a tail estimate for |l| > lmax (the kernel
    is continuous with a kink at +-W/2, so |C| decays like 1/nu^2).
    Returns (eps1, eps3 = (1 + eps1)^3 - 1)."""
    nus = np.linspace(-0.5 / geo.osf, 0.5 / geo.osf, 201)
    ls = np.concatenate([np.arange(-lmax, 0), np.arange(1, lmax + 1)]).astype(np.float64)
    worst = 0.0
    for nu in nus:
        vals = np.abs(kb_kernel_ft(nu + ls, geo.width, geo.beta))
        # tail: bound |C(nu+l)| <= K / (|l| - 1/2)^2 with K fitted on the last
        # 100 terms on each side, summed in closed form beyond lmax
        edge = np.concatenate([vals[:100], vals[-100:]])
        ledge = np.concatenate([ls[:100], ls[-100:]])
        K = np.max(edge * (np.abs(ledge) - 0.5) ** 2)
        tail = 2.0 * K / (lmax - 0.5)
        e = (np.sum(vals) + tail) / kb_kernel_ft(nu, geo.width, geo.beta)
        worst = max(worst, float(e))
    return worst, (1.0 + worst) ** 3 - 1.0


# --------------------------------------------------------------------------
# Dense matrices (tiny grids only)
# --------------------------------------------------------------------------

def _kron3(a, b, c):
    return np.kron(np.kron(a, b), c)


def _interp_matrix(geo: Geometry, q):
    """Dense B (P x G^3): B[p, g] = c3(q_p - g) summed over all periodic
    images g + G*m with |q_p - g - G m| < W/2, built by explicit loops."""
    gs = geo.grid
    W = geo.width
    P = q.shape[1]
    B = np.zeros((P, gs[0] * gs[1] * gs[2]), dtype=np.float64)
    for p in range(P):
        taps = []
        for a in range(3):
            lo = int(np.ceil(q[a, p] - W / 2))
            hi = int(np.floor(q[a, p] + W / 2))
            ga = np.arange(lo, hi + 1)
            taps.append((np.mod(ga, gs[a]), kb_kernel(q[a, p] - ga, W, geo.beta)))
        for i0, w0 in zip(*taps[0]):
            for i1, w1 in zip(*taps[1]):
                for i2, w2 in zip(*taps[2]):
                    B[p, (i0 * gs[1] + i1) * gs[2] + i2] += w0 * w1 * w2
    return B


def dense_warp(geo: Geometry, d):
    """Dense T (N^3 x N^3) = B_j^(i) . [per-axis F^H_scaled Z (1/C) F]."""
    facs = []
    for a in range(3):
        n, g = geo.shape[a], geo.grid[a]
        k = geo.kspace_freqs(a)
        nn = np.arange(n)
        F = np.exp(-2j * np.pi * np.outer(k, nn) / n)                      # rows k (numpy order)
        D = np.diag(1.0 / kb_kernel_ft(k / g, geo.width, geo.beta))
        Z = np.zeros((g, n))
        Z[np.mod(k, g), np.arange(n)] = 1.0                                 # row = k mod G
        kg = np.rint(np.fft.fftfreq(g, 1.0 / g)).astype(np.int64)          # frequency of G-row
        gg = np.arange(g)
        Finv = np.exp(2j * np.pi * np.outer(gg, kg) / g) / n               # (1/N) e^{+}
        facs.append(Finv @ Z @ D @ F)
    L = _kron3(*facs)
    n = np.stack(np.meshgrid(*[np.arange(s, dtype=np.float64) for s in geo.shape],
                             indexing="ij")).reshape(3, -1)
    q = geo.osf * (n + np.asarray(d, dtype=np.float64).reshape(3, -1))
    return _interp_matrix(geo, q) @ L


def dense_kspace(geo: Geometry, omega):
    """Dense G (M x N^3) = B^(k) . [per-axis F Z (1/c*)] with centred n'."""
    facs = []
    for a in range(3):
        n, g = geo.shape[a], geo.grid[a]
        npr = geo.centred_index(a)
        gg = np.arange(g)
        K = np.exp(-2j * np.pi * np.outer(gg, npr) / g) / kb_kernel_ft(npr / g, geo.width, geo.beta)[None, :]
        facs.append(K)
    L = _kron3(*facs)
    om = np.asarray(omega, dtype=np.float64).reshape(-1, 3)
    q = om.T * np.asarray(geo.grid, dtype=np.float64)[:, None] / (2 * np.pi)
    return _interp_matrix(geo, q) @ L


def dense_sense(geo: Geometry, d, smaps, omega):
    """Dense A_j ((M*C) x N^3), rows ordered (sample, coil) with coil fastest."""
    Gm = dense_kspace(geo, omega)
    T = np.eye(int(np.prod(geo.shape))) if d is None else dense_warp(geo, d)
    S = np.asarray(smaps, dtype=np.complex128).reshape(np.shape(smaps)[0], -1)
    A = np.einsum("sm,cm,mn->scn", Gm, S, T)
    return A.reshape(-1, T.shape[1])
