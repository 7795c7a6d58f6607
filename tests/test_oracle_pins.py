"""Pins of the FP64 oracle against things other than itself (CPU only).

Each test ties an oracle function to a textbook value, a closed form, a
brute-force construction or a rigorous error bound, so that a dropped term, a
wrong sign or index, a transposed operand or a wrong scale fails at least one.
"""

import math
import os

import numpy as np
import pytest
import scipy.special

from oracle import kernel as K
from oracle import operators as O
from oracle import references as R
from oracle import solvers as S

HERE = os.path.dirname(os.path.abspath(__file__))


def _crandn(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _rel(a, b):
    return np.linalg.norm(np.ravel(a - b)) / max(np.linalg.norm(np.ravel(b)), 1e-300)


# ---------------------------------------------------------------- kernel ----

def test_i0_textbook_values():
    rows = [l.split() for l in open(os.path.join(HERE, "golden", "bessel_i0.txt"))
            if l.strip() and not l.startswith("#")]
    for z, v in rows:
        got = float(K.bessel_i0(float(z)))
        assert abs(got - float(v)) <= 2e-15 * float(v), (z, got, v)
        assert abs(got - float(scipy.special.i0(float(z)))) <= 2e-15 * float(v)


def test_i0_integral_identity():
    # int_{-1}^{1} I0(beta sqrt(1 - t^2)) dt = 2 sinh(beta) / beta
    t, w = np.polynomial.legendre.leggauss(200)
    for beta in (1.0, 8.996152293560439, 18.6):
        lhs = np.sum(w * K.bessel_i0(beta * np.sqrt(1 - t * t)))
        rhs = 2 * math.sinh(beta) / beta
        assert abs(lhs - rhs) <= 1e-13 * rhs


def test_kernel_edge_and_support():
    W, beta = 4, K.beatty_beta(4, 2)
    assert K.kb_kernel(2.0, W, beta) == 0.0 and K.kb_kernel(-2.0, W, beta) == 0.0
    assert K.kb_kernel(2.5, W, beta) == 0.0
    # continuous at the edge: c(W/2 - eps) -> 0 linearly
    eps = 1e-8
    assert 0 < K.kb_kernel(2.0 - eps, W, beta) < 1e-6
    assert abs(K.kb_kernel(0.0, W, beta) - (scipy.special.i0(beta) - 1)) < 1e-12 * scipy.special.i0(beta)


def test_kernel_ft_closed_form_vs_quadrature():
    # C(nu) = int c(u) exp(-2 pi i nu u) du by Gauss-Legendre on [-W/2, W/2]
    # (c is entire in u on the support, so the quadrature converges fast)
    for W, osf in ((4, 2), (6, 2), (8, 2), (6, 1.5)):
        beta = K.beatty_beta(W, osf)
        t, w = np.polynomial.legendre.leggauss(300)
        u = t * W / 2
        cu = K.kb_kernel(u, W, beta) * (W / 2)
        for nu in np.linspace(0.0, 3.0, 31):
            quad = np.sum(w * cu * np.cos(2 * np.pi * nu * u))
            closed = float(K.kb_kernel_ft(nu, W, beta))
            scale = float(K.kb_kernel_ft(0.0, W, beta))
            assert abs(quad - closed) <= 1e-12 * scale, (W, nu, quad, closed)


def test_fft_convention_matches_direct_dft(rng):
    # the oracle's forward transform is sum_n x[n] exp(-2 pi i k n / N)
    x = _crandn(rng, (4, 6, 8))
    X = O.sfft.fftn(x)
    D = [np.exp(-2j * np.pi * np.outer(np.arange(n), np.arange(n)) / n) for n in x.shape]
    direct = np.einsum("abc,ia,jb,kc->ijk", x, D[0], D[1], D[2])
    assert _rel(X, direct) < 1e-13


# ------------------------------------------------------- dense brute force --

SHAPE = (4, 6, 8)


def _small_disp(rng, shape, amp=1.3):
    return amp * rng.uniform(-1, 1, (3,) + shape)


def test_warp_matches_dense_factors(rng):
    geo = O.Geometry(SHAPE)
    d = _small_disp(rng, SHAPE)
    T = R.dense_warp(geo, d)
    x = _crandn(rng, SHAPE)
    w = _crandn(rng, SHAPE)
    assert _rel(O.warp_forward(geo, x, d).ravel(), T @ x.ravel()) < 1e-12
    assert _rel(O.warp_adjoint(geo, w, d).ravel(), T.conj().T @ w.ravel()) < 1e-12


def test_kspace_matches_dense_factors(rng):
    geo = O.Geometry(SHAPE)
    om = rng.uniform(-np.pi, np.pi, (150, 3))
    Gm = R.dense_kspace(geo, om)
    v = _crandn(rng, SHAPE)
    y = _crandn(rng, (150,))
    assert _rel(O.kspace_forward(geo, v, om), Gm @ v.ravel()) < 1e-12
    assert _rel(O.kspace_adjoint(geo, y, om).ravel(), Gm.conj().T @ y) < 1e-12


def test_sense_matches_dense_and_is_adjoint(rng):
    geo = O.Geometry(SHAPE)
    C, M = 3, 120
    d = _small_disp(rng, SHAPE)
    smaps = _crandn(rng, (C,) + SHAPE)
    om = rng.uniform(-np.pi, np.pi, (M, 3))
    A = R.dense_sense(geo, d, smaps, om)
    x = _crandn(rng, SHAPE)
    y = _crandn(rng, (M, C))
    assert _rel(O.sense_forward(geo, x, d, smaps, om).ravel(), A @ x.ravel()) < 1e-12
    assert _rel(O.sense_adjoint(geo, y, d, smaps, om).ravel(), A.conj().T @ y.ravel()) < 1e-12


def test_dot_test_stacked_model(rng):
    shape = (12, 10, 8)
    geo = O.Geometry(shape)
    P, C = 2, 3
    disps = [_small_disp(rng, shape, 2.5) for _ in range(P)]
    smaps = _crandn(rng, (C,) + shape)
    oms = [rng.uniform(-np.pi, np.pi, (300 + 50 * j, 3)) for j in range(P)]
    x = _crandn(rng, shape)
    ys = [_crandn(rng, (om.shape[0], C)) for om in oms]
    Ax = O.stacked_forward(geo, x, disps, smaps, oms)
    lhs = sum(np.vdot(y, a) for y, a in zip(ys, Ax))
    rhs = np.vdot(O.stacked_adjoint(geo, ys, disps, smaps, oms), x)
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)
    # image-space pair alone
    w = _crandn(rng, shape)
    l2 = np.vdot(w, O.warp_forward(geo, x, disps[0]))
    r2 = np.vdot(O.warp_adjoint(geo, w, disps[0]), x)
    assert abs(l2 - r2) <= 1e-13 * abs(l2)


# ----------------------------------------------------------- closed forms --

def test_zero_displacement_eigenvalues(rng):
    shape = (8, 12, 16)
    geo = O.Geometry(shape)
    x = _crandn(rng, shape)
    lam = R.warp_eigs_constant(geo, (0.0, 0.0, 0.0))
    ref = np.fft.ifftn(np.fft.fftn(x) * lam)
    assert _rel(O.warp_forward(geo, x, np.zeros((3,) + shape)), ref) < 1e-13
    # T(0) is close to, but not exactly, the identity
    err = _rel(O.warp_forward(geo, x, np.zeros((3,) + shape)), x)
    assert 1e-6 < err < 1e-2


@pytest.mark.parametrize("dvec", [(0.3, -1.7, 2.45), (-0.5, 0.25, 0.0), (3.9, -2.2, 1.0 / 3)])
def test_constant_displacement_phase_ramp(rng, dvec):
    shape = (8, 12, 16)
    geo = O.Geometry(shape)
    x = _crandn(rng, shape)
    d = np.broadcast_to(np.asarray(dvec)[:, None, None, None], (3,) + shape)
    lam = R.warp_eigs_constant(geo, dvec)
    ref = np.fft.ifftn(np.fft.fftn(x) * lam)
    assert _rel(O.warp_forward(geo, x, d), ref) < 1e-13
    # adjoint: multiplier conj(lambda)
    refh = np.fft.ifftn(np.fft.fftn(x) * np.conj(lam))
    assert _rel(O.warp_adjoint(geo, x, d), refh) < 1e-13


def test_integer_displacement_is_exact_shift(rng):
    shape = (8, 12, 16)
    geo = O.Geometry(shape)
    x = _crandn(rng, shape)
    t0 = O.warp_forward(geo, x, np.zeros((3,) + shape))
    for dv in ((1, 0, 0), (0, -3, 2), (5, 7, -9)):
        d = np.broadcast_to(np.asarray(dv, float)[:, None, None, None], (3,) + shape)
        shifted = np.roll(t0, shift=tuple(-v for v in dv), axis=(0, 1, 2))
        assert np.max(np.abs(O.warp_forward(geo, x, d) - shifted)) <= 1e-14 * np.max(np.abs(t0)) * 10


def test_alias_bound_decreases_with_width():
    eps = [R.alias_eps(O.Geometry((8, 8, 8), 2, W))[0] for W in (4, 6, 8)]
    assert eps[0] > eps[1] > eps[2]
    assert 5e-4 < eps[0] < 5e-3


def test_gridded_warp_within_bound_of_exact_warp(rng):
    import synth
    shape = (16, 12, 14)
    geo = O.Geometry(shape)
    x = synth.small_case(shape, 0, 1, 0, seed=3)["x"].astype(np.complex128)
    x = x + 0.1 * _crandn(rng, shape)
    d = synth.bump_displacement(shape, 9, 2.7, width_range=(2.0, 4.0)).astype(np.float64)
    eps1, eps3 = R.alias_eps(geo)
    got = O.warp_forward(geo, x, d)
    exact = R.warp_exact(geo, x, d)
    bound = eps3 * np.sum(np.abs(np.fft.fftn(x))) / np.prod(shape)
    err = np.max(np.abs(got - exact))
    assert err <= bound
    # the bound is not vacuous: the error is a visible fraction of it
    assert err > 1e-3 * bound
    # the same bound with the opposite displacement sign must fail: a sign
    # mistake in the pull convention would be caught
    wrong = R.warp_exact(geo, x, -d)
    assert np.max(np.abs(got - wrong)) > bound


def test_gridded_kspace_within_bound_of_nudft(rng):
    shape = (10, 12, 8)
    geo = O.Geometry(shape)
    v = _crandn(rng, shape)
    om = rng.uniform(-np.pi, np.pi, (400, 3))
    eps1, eps3 = R.alias_eps(geo)
    got = O.kspace_forward(geo, v, om)
    exact = R.nudft(geo, v, om)
    assert np.max(np.abs(got - exact)) <= eps3 * np.sum(np.abs(v))
    # conjugated exponent (sign mistake) lands far outside the bound
    wrong = R.nudft(geo, v, -om)
    assert np.max(np.abs(got - wrong)) > eps3 * np.sum(np.abs(v))


def test_zero_displacement_reduces_to_plain_sense(rng):
    shape = (8, 10, 12)
    geo = O.Geometry(shape)
    C = 2
    smaps = _crandn(rng, (C,) + shape)
    om = rng.uniform(-np.pi, np.pi, (200, 3))
    x = _crandn(rng, shape)
    plain = O.kspace_forward(geo, smaps * x[None], om)
    # identity warp flag: exactly G S
    assert np.array_equal(O.sense_forward(geo, x, None, smaps, om), plain)
    # gridded warp with d = 0: G S (T(0) - I), bounded by eps3
    eps1, eps3 = R.alias_eps(geo)
    A0 = O.sense_forward(geo, x, np.zeros((3,) + shape), smaps, om)
    t0 = O.warp_forward(geo, x, np.zeros((3,) + shape))
    assert np.max(np.abs(t0 - x)) <= eps3 * np.sum(np.abs(np.fft.fftn(x))) / np.prod(shape)
    assert _rel(A0, plain) < 3 * eps3


def test_cg_matches_dense_solve(rng):
    geo = O.Geometry((4, 6, 4))
    C, M = 2, 60
    d = _small_disp(rng, geo.shape, 0.8)
    smaps = _crandn(rng, (C,) + geo.shape)
    om = rng.uniform(-np.pi, np.pi, (M, 3))
    A = R.dense_sense(geo, d, smaps, om)
    lam = 1e-2 * np.linalg.norm(A, 2) ** 2
    y = _crandn(rng, (M, C))
    b = A.conj().T @ y.ravel()
    E = A.conj().T @ A + lam * np.eye(A.shape[1])
    ref = np.linalg.solve(E, b)
    x, it, hist = S.cg(lambda v: E @ v, b, tol=1e-13, maxit=500)
    assert _rel(x, ref) < 1e-10
    # the same through the matrix-free oracle normal operator
    x2, it2, _ = S.cg(lambda v: O.normal(geo, v.reshape(geo.shape), [d], smaps, [om], lam).ravel(),
                      b, tol=1e-13, maxit=500)
    assert _rel(x2, ref) < 1e-10


def test_appendix_iterative_inversion_beats_negated_field():
    # Appendix 1: recovering p from q = T p by a regularised least-squares
    # solve is more accurate than warping q with -d.
    import synth
    shape = (24, 24, 24)
    geo = O.Geometry(shape)
    p = synth.phantom(shape, 4).astype(np.complex128)
    d = synth.bump_displacement(shape, 5, 3.0, width_range=(3.0, 6.0)).astype(np.float64)
    q = O.warp_forward(geo, p, d)
    naive = O.warp_forward(geo, q, -d)
    b = O.warp_adjoint(geo, q, d)
    lam = 1e-6
    x, it, _ = S.cg(lambda v: O.warp_normal(geo, v.reshape(shape), [d], lam).ravel(),
                    b.ravel(), tol=1e-6, maxit=60)
    err_naive = _rel(naive, p)
    err_cg = _rel(x.reshape(shape), p)
    assert err_cg < 0.5 * err_naive


# --------------------------------------------------------------------------
# Smaller oversampling, sigma = 1.5 with W = 6 (G = 1.5 N need not be a
# multiple of N): the displaced positions 1.5 (n + d) no longer sit on a
# sub-lattice of the grid, so the circulant and shift closed forms above do
# not apply; the dense factor matrices and the rigorous aliasing bound do.
# --------------------------------------------------------------------------

def test_sigma_one_and_a_half_geometry():
    geo = O.Geometry((8, 10, 12), 1.5, 6)
    assert geo.grid == (12, 15, 18) and geo.osf == 1.5
    assert geo.beta == pytest.approx(K.beatty_beta(6, 1.5))
    with pytest.raises(ValueError):
        O.Geometry((6, 6, 6), 1.25, 6)  # 7.5 grid points


def test_sigma_one_and_a_half_matches_dense_factors(rng):
    shape = (8, 6, 8)
    geo = O.Geometry(shape, 1.5, 6)
    d = _small_disp(rng, shape)
    T = R.dense_warp(geo, d)
    x = _crandn(rng, shape)
    w = _crandn(rng, shape)
    assert _rel(O.warp_forward(geo, x, d).ravel(), T @ x.ravel()) < 1e-12
    assert _rel(O.warp_adjoint(geo, w, d).ravel(), T.conj().T @ w.ravel()) < 1e-12
    om = rng.uniform(-np.pi, np.pi, (150, 3))
    Gm = R.dense_kspace(geo, om)
    v = _crandn(rng, shape)
    y = _crandn(rng, (150,))
    assert _rel(O.kspace_forward(geo, v, om), Gm @ v.ravel()) < 1e-12
    assert _rel(O.kspace_adjoint(geo, y, om).ravel(), Gm.conj().T @ y) < 1e-12


def test_sigma_one_and_a_half_within_bound_of_exact(rng):
    import synth
    shape = (16, 12, 14)
    geo = O.Geometry(shape, 1.5, 6)
    eps1, eps3 = R.alias_eps(geo)
    # W = 6 at sigma 1.5 keeps the aliasing error near that of W = 4 at sigma 2
    eps_ref = R.alias_eps(O.Geometry(shape, 2, 4))[0]
    assert 0.1 * eps_ref < eps1 < 3 * eps_ref
    x = synth.small_case(shape, 0, 1, 0, seed=3)["x"].astype(np.complex128)
    x = x + 0.1 * _crandn(rng, shape)
    d = synth.bump_displacement(shape, 9, 2.7, width_range=(2.0, 4.0)).astype(np.float64)
    got = O.warp_forward(geo, x, d)
    bound = eps3 * np.sum(np.abs(np.fft.fftn(x))) / np.prod(shape)
    assert np.max(np.abs(got - R.warp_exact(geo, x, d))) <= bound
    assert np.max(np.abs(got - R.warp_exact(geo, x, -d))) > bound
    v = _crandn(rng, shape)
    om = rng.uniform(-np.pi, np.pi, (400, 3))
    gk = O.kspace_forward(geo, v, om)
    assert np.max(np.abs(gk - R.nudft(geo, v, om))) <= eps3 * np.sum(np.abs(v))
    assert np.max(np.abs(gk - R.nudft(geo, v, -om))) > eps3 * np.sum(np.abs(v))
