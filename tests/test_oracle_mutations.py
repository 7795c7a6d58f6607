"""Plant plausible mistakes in the oracle (CPU only) and require that the pins
catch every one of them.

Each mutant replaces one internal step of oracle/operators.py; the pins below
are the same kinds of checks as test_oracle_pins.py (dense factor-by-factor
construction, the constant-displacement closed form, the exact-warp and NUDFT
error bounds, the dot test).  A mutant that no pin catches fails this test.
"""

import numpy as np
import pytest

from oracle import operators as O
from oracle import references as R


def _crandn(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _rel(a, b):
    return np.linalg.norm(np.ravel(a - b)) / max(np.linalg.norm(np.ravel(b)), 1e-300)


def _pins_hold():
    """True if every pin holds for the (possibly mutated) oracle."""
    rng = np.random.Generator(np.random.PCG64(7))
    shape = (4, 6, 8)
    geo = O.Geometry(shape)
    ok = True
    # dense brute force of T, G and A (independent formulas)
    d = 1.3 * rng.uniform(-1, 1, (3,) + shape)
    x = _crandn(rng, shape)
    w = _crandn(rng, shape)
    T = R.dense_warp(geo, d)
    ok &= _rel(O.warp_forward(geo, x, d).ravel(), T @ x.ravel()) < 1e-12
    ok &= _rel(O.warp_adjoint(geo, w, d).ravel(), T.conj().T @ w.ravel()) < 1e-12
    om = rng.uniform(-np.pi, np.pi, (80, 3))
    smaps = _crandn(rng, (2,) + shape)
    A = R.dense_sense(geo, d, smaps, om)
    y = _crandn(rng, (80, 2))
    ok &= _rel(O.sense_forward(geo, x, d, smaps, om).ravel(), A @ x.ravel()) < 1e-12
    ok &= _rel(O.sense_adjoint(geo, y, d, smaps, om).ravel(), A.conj().T @ y.ravel()) < 1e-12
    # constant displacement closed form
    shape2 = (8, 12, 10)
    geo2 = O.Geometry(shape2)
    x2 = _crandn(rng, shape2)
    dv = (0.3, -1.7, 2.45)
    dc = np.broadcast_to(np.asarray(dv)[:, None, None, None], (3,) + shape2)
    ref = np.fft.ifftn(np.fft.fftn(x2) * R.warp_eigs_constant(geo2, dv))
    ok &= _rel(O.warp_forward(geo2, x2, dc), ref) < 1e-13
    # exact warp and NUDFT bounds
    eps1, eps3 = R.alias_eps(geo2, lmax=2000)
    dn = 1.5 * np.sin(np.linspace(0, 6, x2.size)).reshape(shape2)[None] * np.array([1.0, -0.5, 0.7])[:, None, None, None]
    bound = eps3 * np.sum(np.abs(np.fft.fftn(x2))) / x2.size
    ok &= np.max(np.abs(O.warp_forward(geo2, x2, dn) - R.warp_exact(geo2, x2, dn))) <= bound
    om2 = rng.uniform(-np.pi, np.pi, (200, 3))
    ok &= np.max(np.abs(O.kspace_forward(geo2, x2, om2) - R.nudft(geo2, x2, om2))) <= eps3 * np.sum(np.abs(x2))
    # dot test of the coil-combined adjoint
    s2 = _crandn(rng, (3,) + shape2)
    y2 = _crandn(rng, (200, 3))
    lhs = np.vdot(y2, O.sense_forward(geo2, x2, dn, s2, om2))
    rhs = np.vdot(O.sense_adjoint(geo2, y2, dn, s2, om2), x2)
    ok &= abs(lhs - rhs) <= 1e-12 * abs(lhs)
    return bool(ok)


def test_unmutated_oracle_passes_pins():
    assert _pins_hold()


def _mut_deapod_uses_N(geo, axis, freqs):
    return 1.0 / O.kb_kernel_ft(freqs / geo.shape[axis], geo.width, geo.beta)


def _mut_push_warp(geo, d):
    d = np.asarray(d, dtype=np.float64).reshape(3, -1)
    n = np.stack(np.meshgrid(*[np.arange(s, dtype=np.float64) for s in geo.shape],
                             indexing="ij")).reshape(3, -1)
    return geo.osf * (n - d)


def _mut_axes_swapped(geo, d):
    d = np.asarray(d, dtype=np.float64).reshape(3, -1)[::-1]
    n = np.stack(np.meshgrid(*[np.arange(s, dtype=np.float64) for s in geo.shape],
                             indexing="ij")).reshape(3, -1)
    return geo.osf * (n + d)


def _mut_scale_over_G(geo):
    return 1.0


def _mut_nyquist_positive(geo, axis):
    k = geo.kspace_freqs(axis).copy()
    k[k == -geo.shape[axis] // 2] = geo.shape[axis] // 2
    return np.mod(k, geo.grid[axis])


def _mut_no_kspace_deapod(geo, axis):
    return np.ones(geo.shape[axis])


def _mut_uncentred(geo, axis):
    return 1.0 / O.kb_kernel_ft(np.arange(geo.shape[axis]) / geo.grid[axis], geo.width, geo.beta)


def _mut_kspace_factor2(geo, omega):
    om = np.asarray(omega, dtype=np.float64).reshape(-1, 3)
    g = np.asarray(geo.grid, dtype=np.float64)[:, None]
    return om.T * g / np.pi


def _mut_no_conj(smaps, v):
    return np.sum(np.asarray(smaps, dtype=np.complex128) * v, axis=0)


def _mut_short_taps(q, g_size, width, beta):
    base = np.floor(q).astype(np.int64)
    off = np.arange(-(width // 2), width // 2, dtype=np.int64)
    g = base[:, None] + off[None, :]
    return np.mod(g, g_size), O.kb_kernel(q[:, None] - g, width, beta)


def _mut_kernel_no_edge(u, width, beta):
    from oracle.kernel import bessel_i0
    u = np.asarray(u, dtype=np.float64)
    x = 2.0 * u / width
    inside = np.abs(x) < 1.0
    return np.where(inside, bessel_i0(beta * np.sqrt(np.where(inside, 1 - x * x, 0.0))), 0.0)


MUTANTS = {
    "deapod at k/N instead of k/G": ("_deapod_table", _mut_deapod_uses_N),
    "push instead of pull displacement": ("warp_positions", _mut_push_warp),
    "displacement components on the wrong axes": ("warp_positions", _mut_axes_swapped),
    "inverse DFT scaled by 1/G instead of 1/N": ("_upsample_scale", _mut_scale_over_G),
    "Nyquist bin placed at +N/2": ("_pad_index", _mut_nyquist_positive),
    "k-space deapodization dropped": ("_centred_deapod", _mut_no_kspace_deapod),
    "k-space image index not centred": ("_centred_deapod", _mut_uncentred),
    "k-space positions off by a factor 2": ("kspace_positions", _mut_kspace_factor2),
    "coil adjoint without conjugate": ("coil_adjoint", _mut_no_conj),
    "one interpolation tap missing": ("_axis_taps", _mut_short_taps),
    "kernel without edge subtraction": ("kb_kernel", _mut_kernel_no_edge),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, monkeypatch):
    attr, fn = MUTANTS[name]
    monkeypatch.setattr(O, attr, fn)
    assert not _pins_hold(), f"no pin caught the planted mistake: {name}"
