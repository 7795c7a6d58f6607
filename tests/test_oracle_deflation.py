"""Pins of the deflation oracle (oracle/deflation.py) against what the
mathematics fixes: the CG-Lanczos tridiagonal of a full-length run has the
spectrum of M E; Ritz values are Rayleigh quotients of their Ritz vectors
and lie inside the spectrum; deflating exact eigenvectors leaves only the
remaining distinct eigenvalues to the iteration; a basis of the whole space
solves the system at the start; every deflated residual is orthogonal to W.
"""

import numpy as np
import pytest

from oracle import deflation as D


def _hpd(n, eigs, seed):
    """Hermitian positive-definite n x n matrix with the given eigenvalues and
    a random unitary eigenbasis."""
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    U, _ = np.linalg.qr(X)
    return (U * np.asarray(eigs, dtype=np.float64)) @ U.conj().T, U


def _rhs(n, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(n) + 1j * rng.standard_normal(n)


def test_full_lanczos_recovers_the_spectrum_of_ME():
    n = 10
    eigs = np.geomspace(0.05, 3.0, n)
    A, _ = _hpd(n, eigs, 1)
    m = np.random.default_rng(2).uniform(0.5, 2.0, n)      # M = diag(m), HPD
    b = _rhs(n, 3)
    _, it, _, al, rho, Z = D.pcg_record(lambda v: A @ v, lambda r: m * r, b, tol=0.0,
                                        maxit=n, record=n)
    assert it == n and len(Z) == n
    T = D.lanczos_tridiagonal(al, rho, n)
    theta = np.linalg.eigvalsh(T)
    Ms = np.sqrt(m)
    ref = np.linalg.eigvalsh((Ms[:, None] * A) * Ms[None, :])  # spectrum of M^1/2 A M^1/2
    assert np.allclose(theta, ref, rtol=1e-8, atol=0)
    # the Lanczos vectors are orthonormal in the M^-1 inner product, and T is
    # the projection of E on them (signs of the off-diagonal included)
    V = np.stack(Z, 1)
    assert np.allclose(V.conj().T @ (V / m[:, None]), np.eye(n), atol=1e-8)
    assert np.allclose(V.conj().T @ A @ V, T, atol=1e-8 * np.abs(T).max())


def test_ritz_pairs_are_rayleigh_quotients_inside_the_spectrum():
    n, steps, k = 30, 6, 3
    eigs = np.geomspace(0.02, 5.0, n)
    A, _ = _hpd(n, eigs, 4)
    m = np.random.default_rng(5).uniform(0.5, 2.0, n)
    b = _rhs(n, 6)
    _, _, _, al, rho, Z = D.pcg_record(lambda v: A @ v, lambda r: m * r, b, tol=0.0,
                                       maxit=steps, record=steps)
    T = D.lanczos_tridiagonal(al, rho, steps)
    theta, W = D.ritz_space(T, Z, k)
    Ms = np.sqrt(m)
    lam = np.linalg.eigvalsh((Ms[:, None] * A) * Ms[None, :])
    assert np.all(theta >= lam[0] * (1 - 1e-12)) and np.all(theta <= lam[-1] * (1 + 1e-12))
    assert np.all(np.diff(theta) > 0)
    for t, u in zip(theta, W):
        rq = np.vdot(u, A @ u).real / np.vdot(u, u / m).real
        assert abs(rq - t) <= 1e-10 * t
    # plausible slips -- the tridiagonal without its beta / alpha diagonal
    # term, or with the off-diagonal sign of the other vector convention --
    # give Ritz vectors whose Rayleigh quotients are not their Ritz values
    for slip in ("diag", "sign"):
        T_bad = T.copy()
        for j in range(1, steps):
            if slip == "diag":
                T_bad[j, j] = 1.0 / al[j]
            else:
                T_bad[j - 1, j] = T_bad[j, j - 1] = -T[j, j - 1]
        theta_bad, W_bad = D.ritz_space(T_bad, Z, k)
        u = W_bad[0]
        rq = np.vdot(u, A @ u).real / np.vdot(u, u / m).real
        assert abs(rq - theta_bad[0]) > 1e-3 * theta_bad[0], slip


def test_deflating_exact_eigenvectors_leaves_the_other_distinct_eigenvalues():
    n, k = 24, 4
    small = [0.01, 0.02, 0.05, 0.1]
    rest = np.resize([1.0, 2.0, 3.0], n - k)
    A, U = _hpd(n, np.concatenate([small, rest]), 7)
    b = _rhs(n, 8)
    E = lambda v: A @ v  # noqa: E731
    I = lambda r: r      # noqa: E731
    x_ref = np.linalg.solve(A, b)
    _, it_plain, _, _, _, _ = D.pcg_record(E, I, b, tol=1e-10, maxit=100)
    x, it, hist, wr = D.deflated_pcg(E, I, b, [U[:, i] for i in range(k)], tol=1e-10, maxit=100)
    assert it <= 3 < it_plain                  # three distinct eigenvalues remain
    assert np.linalg.norm(x - x_ref) <= 1e-9 * np.linalg.norm(x_ref)
    assert wr <= 1e-12


def test_a_basis_of_the_whole_space_solves_at_the_start():
    n = 12
    A, _ = _hpd(n, np.geomspace(0.1, 4.0, n), 9)
    b = _rhs(n, 10)
    W = list(np.eye(n, dtype=np.complex128))
    x, it, hist, _ = D.deflated_pcg(lambda v: A @ v, lambda r: r, b, W, tol=1e-12, maxit=10)
    assert it == 0 and hist[0] <= 1e-12
    assert np.allclose(x, np.linalg.solve(A, b), rtol=0, atol=1e-12 * np.linalg.norm(b))


def test_deflated_residuals_stay_orthogonal_to_the_basis():
    n, k = 40, 5
    A, _ = _hpd(n, np.geomspace(0.01, 10.0, n), 11)
    m = np.random.default_rng(12).uniform(0.5, 2.0, n)
    b = _rhs(n, 13)
    rng = np.random.default_rng(14)
    W = [rng.standard_normal(n) + 1j * rng.standard_normal(n) for _ in range(k)]
    x, it, _, wr = D.deflated_pcg(lambda v: A @ v, lambda r: m * r, b, W, tol=1e-11,
                                  maxit=200, x_init=_rhs(n, 15))
    assert wr <= 1e-9
    assert np.linalg.norm(A @ x - b) <= 1e-10 * np.linalg.norm(b)


@pytest.mark.parametrize("k", [2, 6])
def test_recycled_ritz_space_on_a_sense_problem(k):
    """Circulant-preconditioned CG on a small nonrigid SENSE system: Ritz
    vectors from a solve with another right-hand side, used as the deflation
    basis, reach the same solution, residuals orthogonal to the basis, in no
    more iterations (on an 8 x 8 x 10 image the low end of the preconditioned
    spectrum is a continuum, so the count barely moves; at 128^3 it falls from
    19 to 12)."""
    import synth
    from oracle import operators as O
    from oracle import precond as PC
    shape = (8, 8, 10)
    case = synth.small_case(shape, 2, 2, [300, 260], seed=171, max_disp=1.5)
    geo = O.Geometry(shape)
    d64 = [d.astype(np.float64) for d in case["disp"]]
    E0 = lambda v: O.normal(geo, v, d64, case["smaps"], case["coords"], 0.0)  # noqa: E731
    lam = 1e-2 * 7.6e4
    E = lambda v: E0(v) + lam * v  # noqa: E731
    d = PC.circulant_diag(E0, shape, 10.0 * lam)
    M = lambda r: PC.apply_circulant(d, r)  # noqa: E731
    rng = np.random.default_rng(172)
    b_train = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    b = O.stacked_adjoint(geo, O.stacked_forward(geo, case["x"], d64, case["smaps"],
                                                 case["coords"]), d64, case["smaps"],
                          case["coords"])
    steps = 12
    _, _, _, al, rho, Z = D.pcg_record(E, M, b_train, tol=0.0, maxit=steps, record=steps)
    theta, W = D.ritz_space(D.lanczos_tridiagonal(al, rho, steps), Z, k)
    x_p, it_p, _, _, _, _ = D.pcg_record(E, M, b, tol=1e-8, maxit=300)
    x_d, it_d, _, wr = D.deflated_pcg(E, M, b, W, tol=1e-8, maxit=300)
    assert it_d <= it_p
    assert wr <= 1e-8
    assert np.linalg.norm(x_d - x_p) <= 1e-6 * np.linalg.norm(x_p)
