"""Step-by-step FP64 operators of the method (oracle; test infrastructure).

Notation (per axis; 3D is the tensor product of the three axes):
  N      image size, sigma oversampling (integer), G = sigma * N
  W      kernel width in oversampled-grid units, beta its shape parameter
  K_N    the frequency set {-N/2, ..., N/2 - 1} (numpy FFT order in memory)
  c, C   interpolation kernel and its Fourier transform (kernel.py)

Image-space gridding (section "Image-space Gridding"):
  forward T_j  (process diagram ending in B_j^(i)):
    1. X[k]  = sum_n x[n] exp(-2 pi i k n / N)                 (F)
    2. U[k]  = X[k] / C(k/G) for k in K_N                      (1/C*[k])
    3. zero-pad K_N into K_G                                   (Z)
    4. u[g]  = (1/N) sum_{k in K_G} U[k] exp(+2 pi i k g / G)  (F^H)
    5. m_j[n] = sum_g c(q_n - g) u[g mod G],  q_n = sigma (n + d_j[n])
                                                               (B_j^(i))
  adjoint T_j^H (process diagram starting with P_j^(i)): the conjugate
    transpose of the above, i.e. spread, forward DFT of size G scaled by 1/N,
    crop to K_N, divide by C(k/G), unnormalised inverse DFT of size N.

Readings of the paper where it is silent: forward DFT uses exp(-2 pi i ...); the
inverse DFT of size G is scaled by 1/N so that T_j with zero displacement is
the identity up to the kernel's aliasing error; the -N/2 bin of K_N maps to
frequency -N/2 of the G grid; boundaries are periodic (positions mod N, taps
mod G); displacements pull (m_j[r] = m(r + d[r])) and are in N-grid voxels.

k-space gridding (section "k-space Gridding"): with the centred image index
n' = n - N/2,
  inverse gridding G_j (Type-2, process diagram 1/c* -> Z -> F -> B^(k)):
    v'[n'] = v[n'] / C(n'/G);  X[g] = sum_{n'} v'[n'] exp(-2 pi i g n'/G);
    y_s = sum_g c(q_s - g) X[g mod G],  q_s = omega_s G / (2 pi)
  gridding G_j^H (Type-1, P^(k) -> F^H -> Z^H -> 1/c): spread, unnormalised
    inverse DFT of size G, crop to K_N, divide by C(n'/G).
No density compensation is applied inside G^H: it is the exact adjoint.

Nonrigid SENSE (section "Nonrigid SENSE Operators"): A_j = G_j S T_j and
A_j^H = T_j^H S^H G_j^H, stacked over phases (stacked SENSE equation); the
normal operator is E x = sum_j A_j^H A_j x + lambda x.

Array layouts: image (N0, N1, N2); displacement (3, N0, N1, N2) with component
a along axis a; coil maps (C, N0, N1, N2); k-space coordinates (M, 3) radians;
k-space data of one phase (M, C) (coil index fastest).
"""

from __future__ import annotations

import numpy as np
import scipy.fft as sfft

from .kernel import beatty_beta, kb_kernel, kb_kernel_ft

FFT_WORKERS = 1


class Geometry:
    """Image size, oversampling and kernel parameters of one operator."""

    def __init__(self, shape, osf: float = 2, width: int = 4, beta: float | None = None):
        self.shape = tuple(int(s) for s in shape)
        if len(self.shape) != 3 or any(s % 2 for s in self.shape):
            raise ValueError("image dimensions must be three even integers")
        # sigma need not be an integer (the oversampled grid G = sigma N only
        # has to be a whole number of points per axis)
        self.osf = int(osf) if float(osf).is_integer() else float(osf)
        self.width = int(width)
        self.beta = float(beta_or_default(beta, width, self.osf))
        grid = [self.osf * s for s in self.shape]
        if any(abs(gv - round(gv)) > 1e-9 for gv in grid):
            raise ValueError("sigma * N must be an integer on every axis")
        self.grid = tuple(int(round(gv)) for gv in grid)

    def kspace_freqs(self, axis):
        """k in K_N, in numpy FFT order, as integers."""
        n = self.shape[axis]
        return np.rint(np.fft.fftfreq(n, 1.0 / n)).astype(np.int64)

    def centred_index(self, axis):
        """n' = n - N/2 for n = 0..N-1."""
        n = self.shape[axis]
        return np.arange(n, dtype=np.int64) - n // 2


def beta_or_default(beta, width, osf):
    return beatty_beta(width, osf) if (beta is None or beta == 0) else beta


# --------------------------------------------------------------------------
# Projection / Backprojection Cores on an arbitrary set of points
# --------------------------------------------------------------------------

def _axis_taps(q, g_size, width, beta):
    """For positions q (M,) on a periodic grid of g_size points: the candidate
    taps g = floor(q) + o, o in [-W/2, W/2], their indices mod g_size and the
    weights c(q - g).  Taps at distance >= W/2 get weight exactly 0."""
    base = np.floor(q).astype(np.int64)
    off = np.arange(-(width // 2), width // 2 + 1, dtype=np.int64)
    g = base[:, None] + off[None, :]
    w = kb_kernel(q[:, None] - g, width, beta)
    return np.mod(g, g_size), w


def backprojection_core(grid, q, width, beta):
    """B: y[p] = sum_g c3(q_p - g) grid[g mod G] (interpolation).

    grid: (G0, G1, G2) or (G0, G1, G2, C) complex; q: (3, M) float64.
    Returns (M,) or (M, C)."""
    gs = grid.shape[:3]
    idx, wts = zip(*[_axis_taps(q[a], gs[a], width, beta) for a in range(3)])
    ntap = wts[0].shape[1]
    out = np.zeros((q.shape[1],) + grid.shape[3:], dtype=np.complex128)
    for t0 in range(ntap):
        for t1 in range(ntap):
            w01 = wts[0][:, t0] * wts[1][:, t1]
            for t2 in range(ntap):
                w = w01 * wts[2][:, t2]
                vals = grid[idx[0][:, t0], idx[1][:, t1], idx[2][:, t2]]
                if vals.ndim == 2:
                    out += w[:, None] * vals
                else:
                    out += w * vals
    return out


def projection_core(vals, q, grid_shape, width, beta):
    """P: grid[g] = sum_p c3(q_p - g) vals[p] (spreading), the exact transpose
    of backprojection_core.  vals: (M,) or (M, C).  Scatter-add by np.add.at,
    one call per tap."""
    gs = tuple(grid_shape)
    idx, wts = zip(*[_axis_taps(q[a], gs[a], width, beta) for a in range(3)])
    ntap = wts[0].shape[1]
    vals = np.asarray(vals, dtype=np.complex128)
    out = np.zeros((gs[0] * gs[1] * gs[2],) + vals.shape[1:], dtype=np.complex128)
    for t0 in range(ntap):
        for t1 in range(ntap):
            w01 = wts[0][:, t0] * wts[1][:, t1]
            lin01 = idx[0][:, t0] * gs[1] + idx[1][:, t1]
            for t2 in range(ntap):
                w = w01 * wts[2][:, t2]
                lin = lin01 * gs[2] + idx[2][:, t2]
                np.add.at(out, lin, (w[:, None] * vals) if vals.ndim == 2 else w * vals)
    return out.reshape(gs + vals.shape[1:])


# --------------------------------------------------------------------------
# Image-space gridding T_j and T_j^H
# --------------------------------------------------------------------------

def warp_positions(geo: Geometry, d):
    """q = sigma * (n + d[n]) on the oversampled grid, shape (3, N^3)."""
    d = np.asarray(d, dtype=np.float64).reshape(3, -1)
    n = np.stack(np.meshgrid(*[np.arange(s, dtype=np.float64) for s in geo.shape],
                             indexing="ij")).reshape(3, -1)
    return geo.osf * (n + d)


def _deapod_table(geo: Geometry, axis, freqs):
    return 1.0 / kb_kernel_ft(freqs / geo.grid[axis], geo.width, geo.beta)


def _upsample_scale(geo: Geometry):
    """prod(G) / prod(N): turns ifftn's 1/prod(G) into the 1/prod(N) of step 4."""
    return float(np.prod(geo.grid)) / float(np.prod(geo.shape))


def _pad_index(geo: Geometry, axis):
    """Position of k in K_N (numpy order) on the G grid: k mod G."""
    return np.mod(geo.kspace_freqs(axis), geo.grid[axis])


def warp_forward(geo: Geometry, x, d):
    """T_j x: image-space gridding forward (F, 1/C*, Z, F^H, B_j^(i))."""
    x = np.asarray(x, dtype=np.complex128).reshape(geo.shape)
    X = sfft.fftn(x, workers=FFT_WORKERS)
    for a in range(3):
        shp = [1, 1, 1]
        shp[a] = -1
        X = X * _deapod_table(geo, a, geo.kspace_freqs(a)).reshape(shp)
    U = np.zeros(geo.grid, dtype=np.complex128)
    U[np.ix_(*[_pad_index(geo, a) for a in range(3)])] = X
    # (1/N) sum_k U[k] exp(+2 pi i k g / G): ifftn carries 1/prod(G)
    u = sfft.ifftn(U, workers=FFT_WORKERS) * _upsample_scale(geo)
    q = warp_positions(geo, d)
    return backprojection_core(u, q, geo.width, geo.beta).reshape(geo.shape)


def warp_adjoint(geo: Geometry, w, d):
    """T_j^H w: image-space gridding adjoint (P_j^(i), F, Z^H, 1/C, F^H)."""
    w = np.asarray(w, dtype=np.complex128).reshape(-1)
    nvox = float(np.prod(geo.shape))
    q = warp_positions(geo, d)
    ut = projection_core(w, q, geo.grid, geo.width, geo.beta)
    Ut = sfft.fftn(ut, workers=FFT_WORKERS)[np.ix_(*[_pad_index(geo, a) for a in range(3)])] * (
        _upsample_scale(geo) / float(np.prod(geo.grid)))
    for a in range(3):
        shp = [1, 1, 1]
        shp[a] = -1
        Ut = Ut * _deapod_table(geo, a, geo.kspace_freqs(a)).reshape(shp)
    # unnormalised inverse DFT of size N: ifftn carries 1/prod(N)
    return sfft.ifftn(Ut, workers=FFT_WORKERS) * nvox


# --------------------------------------------------------------------------
# k-space gridding G_j (Type 2) and G_j^H (Type 1)
# --------------------------------------------------------------------------

def kspace_positions(geo: Geometry, omega):
    """q_s = omega_s * G / (2 pi), shape (3, M)."""
    om = np.asarray(omega, dtype=np.float64).reshape(-1, 3)
    g = np.asarray(geo.grid, dtype=np.float64)[:, None]
    return om.T * g / (2.0 * np.pi)


def _centred_deapod(geo: Geometry, axis):
    return 1.0 / kb_kernel_ft(geo.centred_index(axis) / geo.grid[axis], geo.width, geo.beta)


def kspace_forward(geo: Geometry, v, omega):
    """G_j v (inverse k-space gridding).  v: (N0,N1,N2) or (C,N0,N1,N2).
    Returns (M,) or (M, C)."""
    v = np.asarray(v, dtype=np.complex128)
    single = v.ndim == 3
    if single:
        v = v[None]
    q = kspace_positions(geo, omega)
    out = np.zeros((q.shape[1], v.shape[0]), dtype=np.complex128)
    pidx = np.ix_(*[np.mod(geo.centred_index(a), geo.grid[a]) for a in range(3)])
    for c in range(v.shape[0]):
        vc = v[c]
        for a in range(3):
            shp = [1, 1, 1]
            shp[a] = -1
            vc = vc * _centred_deapod(geo, a).reshape(shp)
        pad = np.zeros(geo.grid, dtype=np.complex128)
        pad[pidx] = vc
        X = sfft.fftn(pad, workers=FFT_WORKERS)
        out[:, c] = backprojection_core(X, q, geo.width, geo.beta)
    return out[:, 0] if single else out


def kspace_adjoint(geo: Geometry, y, omega):
    """G_j^H y (k-space gridding).  y: (M,) or (M, C).
    Returns (N0,N1,N2) or (C,N0,N1,N2)."""
    y = np.asarray(y, dtype=np.complex128)
    single = y.ndim == 1
    if single:
        y = y[:, None]
    q = kspace_positions(geo, omega)
    pidx = np.ix_(*[np.mod(geo.centred_index(a), geo.grid[a]) for a in range(3)])
    out = np.zeros((y.shape[1],) + geo.shape, dtype=np.complex128)
    for c in range(y.shape[1]):
        Xt = projection_core(y[:, c], q, geo.grid, geo.width, geo.beta)
        v = sfft.ifftn(Xt, workers=FFT_WORKERS)[pidx] * float(np.prod(geo.grid))
        for a in range(3):
            shp = [1, 1, 1]
            shp[a] = -1
            v = v * _centred_deapod(geo, a).reshape(shp)
        out[c] = v
    return out[0] if single else out


# --------------------------------------------------------------------------
# Coil sensitivities and the nonrigid SENSE operator
# --------------------------------------------------------------------------

def coil_forward(smaps, m):
    """S m: (C, N0, N1, N2)."""
    return np.asarray(smaps, dtype=np.complex128) * np.asarray(m, dtype=np.complex128)[None]


def coil_adjoint(smaps, v):
    """S^H v = sum_c conj(S_c) v_c."""
    return np.sum(np.conj(np.asarray(smaps, dtype=np.complex128)) * v, axis=0)


def sense_forward(geo: Geometry, x, disp, smaps, omega):
    """A_j x = G_j S T_j x for one phase; disp None means T_j = I."""
    m = np.asarray(x, dtype=np.complex128) if disp is None else warp_forward(geo, x, disp)
    return kspace_forward(geo, coil_forward(smaps, m), omega)


def sense_adjoint(geo: Geometry, y, disp, smaps, omega):
    """A_j^H y = T_j^H S^H G_j^H y for one phase."""
    w = coil_adjoint(smaps, kspace_adjoint(geo, y, omega))
    return w if disp is None else warp_adjoint(geo, w, disp)


def stacked_forward(geo: Geometry, x, disps, smaps, omegas):
    """[A_0; ...; A_{P-1}] x as a list of (M_j, C) arrays."""
    return [sense_forward(geo, x, d, smaps, om) for d, om in zip(disps, omegas)]


def stacked_adjoint(geo: Geometry, ys, disps, smaps, omegas):
    """sum_j A_j^H y_j."""
    out = np.zeros(geo.shape, dtype=np.complex128)
    for y, d, om in zip(ys, disps, omegas):
        out += sense_adjoint(geo, y, d, smaps, om)
    return out


def normal(geo: Geometry, x, disps, smaps, omegas, lam: float = 0.0):
    """E x = sum_j A_j^H A_j x + lambda x."""
    out = lam * np.asarray(x, dtype=np.complex128)
    for d, om in zip(disps, omegas):
        out = out + sense_adjoint(geo, sense_forward(geo, x, d, smaps, om), d, smaps, om)
    return out


def warp_normal(geo: Geometry, x, disps, lam: float = 0.0):
    """sum_j T_j^H T_j x + lambda x (image-space-only model, no coils)."""
    out = lam * np.asarray(x, dtype=np.complex128)
    for d in disps:
        out = out + warp_adjoint(geo, warp_forward(geo, x, d), d)
    return out
