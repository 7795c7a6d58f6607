"""Pins of the wavelet-FISTA oracle (CPU only).

The Haar transform is checked against the Haar basis functions written out
in closed form (piecewise-constant scaling and wavelet functions of each
level), the soft threshold against a generic minimiser of its defining
problem, the FISTA iteration against the optimality conditions of the L1
problem (solved to convergence on a small dense operator), against Beck and
Teboulle's O(1/k^2) bound on the objective gap (their Theorem 4.4), against
the closed-form minimiser for a single wavelet atom under the identity
operator, and against the least-squares solution when lambda = 0.  The last
test plants plausible mistakes in the oracle and requires every one to fail
a pin.
"""

import itertools
import math

import numpy as np
import pytest
import scipy.optimize

from oracle import fista as F


def _crandn(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _haar_1d(n, level, p, wavelet):
    """Scaling (wavelet=False) or wavelet function of `level` at position p on
    n points: support [p 2^level, (p+1) 2^level), height 2^(-level/2), the
    wavelet positive on the first half of the support, negative on the second."""
    v = np.zeros(n)
    s = 1 << level
    h = 2.0 ** (-level / 2.0)
    if not wavelet:
        v[p * s:(p + 1) * s] = h
    else:
        v[p * s:p * s + s // 2] = h
        v[p * s + s // 2:(p + 1) * s] = -h
    return v


def haar_matrix(shape, levels):
    """Rows: the 3D Haar basis in the Mallat layout, built from the closed-form
    1D functions (no pairwise recursion)."""
    n = int(np.prod(shape))
    W = np.zeros((n, n))
    if levels == 0:
        return np.eye(n)

    def put(idx, rows):
        W[np.ravel_multi_index(idx, shape)] = np.einsum("i,j,k->ijk", *rows).ravel()

    for lev in range(1, levels + 1):
        m = [a >> lev for a in shape]
        for s in itertools.product((0, 1), repeat=3):
            if s == (0, 0, 0):
                continue
            for p in itertools.product(*(range(v) for v in m)):
                idx = tuple(s[a] * m[a] + p[a] for a in range(3))
                put(idx, [_haar_1d(shape[a], lev, p[a], s[a] == 1) for a in range(3)])
    m = [a >> levels for a in shape]
    for p in itertools.product(*(range(v) for v in m)):
        put(tuple(p), [_haar_1d(shape[a], levels, p[a], False) for a in range(3)])
    return W


# ------------------------------------------------------------- pins ----------

def pin_hadamard_one_level():
    """One level on 2x2x2 blocks is the normalised 3D Walsh-Hadamard transform:
    c[s * n/2 + p] = 8^(-1/2) sum_i (-1)^(s.i) x[2p + i]."""
    rng = np.random.Generator(np.random.PCG64(1))
    shape = (4, 6, 2)
    x = _crandn(rng, shape)
    c = F.haar_forward(x, 1)
    half = [a // 2 for a in shape]
    for p in itertools.product(*(range(h) for h in half)):
        for s in itertools.product((0, 1), repeat=3):
            want = sum((-1) ** (s[0] * i[0] + s[1] * i[1] + s[2] * i[2])
                       * x[2 * p[0] + i[0], 2 * p[1] + i[1], 2 * p[2] + i[2]]
                       for i in itertools.product((0, 1), repeat=3)) / math.sqrt(8.0)
            got = c[s[0] * half[0] + p[0], s[1] * half[1] + p[1], s[2] * half[2] + p[2]]
            assert abs(got - want) < 1e-12, (p, s)


def pin_haar_basis(shape=(8, 4, 12), levels=2):
    rng = np.random.Generator(np.random.PCG64(2))
    x = _crandn(rng, shape)
    W = haar_matrix(shape, levels)
    assert np.abs(F.haar_forward(x, levels).ravel() - W @ x.ravel()).max() < 1e-12
    c = _crandn(rng, shape)
    assert np.abs(F.haar_inverse(c, levels).ravel() - W.T @ c.ravel()).max() < 1e-12


def pin_constant_volume():
    """A constant volume has only approximation coefficients, each c 2^(3J/2)."""
    shape, J, c0 = (8, 8, 16), 3, 0.7 - 0.2j
    c = F.haar_forward(np.full(shape, c0), J)
    want = np.zeros(shape, complex)
    want[:1, :1, :2] = c0 * 2.0 ** (1.5 * J)
    assert np.abs(c - want).max() < 1e-12


def pin_soft_threshold_minimises():
    rng = np.random.Generator(np.random.PCG64(3))
    for c, tau in [(1.3 - 0.4j, 0.5), (0.2 + 0.1j, 0.5), (-2.0 + 0.0j, 0.25), (0.0j, 0.1)]:
        got = F.soft_threshold(np.array([c]), tau)[0]
        # closed form: modulus shrunk by tau, phase kept
        assert abs(abs(got) - max(abs(c) - tau, 0.0)) < 1e-14
        if abs(got) > 0:
            assert abs(got / abs(got) - c / abs(c)) < 1e-14
        obj = lambda u: 0.5 * ((u[0] - c.real) ** 2 + (u[1] - c.imag) ** 2) + tau * math.hypot(*u)
        best = min((scipy.optimize.minimize(obj, u0, method="Nelder-Mead",
                                            options=dict(xatol=1e-10, fatol=1e-14))
                    for u0 in ([c.real, c.imag], [0.0, 0.0], list(rng.standard_normal(2)))),
                   key=lambda r: r.fun)
        assert obj([got.real, got.imag]) <= best.fun + 1e-12


def pin_prox_minimises():
    """prox_{tau ||W.||_1}(v) has a lower value of 1/2||u - v||^2 + tau ||W u||_1
    than every small perturbation of it (W from the closed-form basis)."""
    rng = np.random.Generator(np.random.PCG64(4))
    shape, J, tau = (4, 4, 8), 2, 0.6
    W = haar_matrix(shape, J)
    v = _crandn(rng, shape)
    u = F.prox_wavelet_l1(v, tau, J).ravel()
    obj = lambda w: 0.5 * np.linalg.norm(w - v.ravel()) ** 2 + tau * np.abs(W @ w).sum()
    f0 = obj(u)
    for _ in range(200):
        assert f0 <= obj(u + 1e-4 * _crandn(rng, u.shape)) + 1e-12


def pin_single_atom_denoising():
    """A = I, y = a psi (one Haar atom): the minimiser of ||y - x||^2 +
    lambda ||W x||_1 is max(0, 1 - lambda / (2|a|)) a psi, and FISTA with
    L = 2 reaches it in one step."""
    shape, J = (8, 8, 4), 2
    psi = np.einsum("i,j,k->ijk", _haar_1d(8, 2, 1, True), _haar_1d(8, 2, 0, False),
                    _haar_1d(4, 2, 0, True))
    for a, lam in [(1.5 + 2.0j, 1.0), (0.3 - 0.1j, 1.0), (4.0 + 0.0j, 0.5)]:
        y = a * psi
        want = max(0.0, 1.0 - lam / (2.0 * abs(a))) * a * psi
        x, _ = F.fista(lambda v: v, y, lam, 2.0, J, 1)
        assert np.abs(x - want).max() < 1e-12, a


def _small_problem(seed=5, shape=(2, 2, 4), m=40):
    rng = np.random.Generator(np.random.PCG64(seed))
    n = int(np.prod(shape))
    A = _crandn(rng, (m, n)) / math.sqrt(m)
    y = _crandn(rng, m)
    E0 = A.conj().T @ A
    b = A.conj().T @ y
    L = 2.0 * float(np.linalg.eigvalsh(E0).max())
    apply_E0 = lambda v: (E0 @ v.ravel()).reshape(shape)
    return A, y, E0, b.reshape(shape), L, apply_E0, shape


def _objective(A, y, W, x, lam):
    return float(np.linalg.norm(y - A @ x.ravel()) ** 2 + lam * np.abs(W @ x.ravel()).sum())


def pin_fista_optimality():
    """After many iterations the iterate satisfies the L1 optimality conditions
    in the (closed-form) Haar coefficient domain: h = W grad f(x) equals
    -lambda c/|c| where c = W x is non-zero and |h| <= lambda where c = 0."""
    A, y, E0, b, L, apply_E0, shape = _small_problem()
    J, lam = 1, 0.9
    W = haar_matrix(shape, J)
    x, _ = F.fista(apply_E0, b, lam, L, J, 3000)
    c = W @ x.ravel()
    h = W @ (2.0 * (E0 @ x.ravel() - b.ravel()))
    nz = np.abs(c) > 1e-9
    assert 0 < nz.sum() < c.size  # lambda leaves some coefficients at zero
    assert np.abs(h[nz] + lam * c[nz] / np.abs(c[nz])).max() < 1e-8
    assert np.abs(h[~nz]).max() <= lam * (1 + 1e-8)
    return x


def pin_fista_rate():
    """Beck-Teboulle Theorem 4.4: F(x_k) - F* <= 2 L ||x_0 - x*||^2 / (k + 1)^2."""
    A, y, E0, b, L, apply_E0, shape = _small_problem()
    J, lam = 1, 0.9
    W = haar_matrix(shape, J)
    xs = pin_fista_optimality()
    Fs = _objective(A, y, W, xs, lam)
    gaps = []
    F.fista(apply_E0, b, lam, L, J, 150,
            callback=lambda k, x: gaps.append((k, _objective(A, y, W, x, lam) - Fs)))
    bound = 2.0 * L * np.linalg.norm(xs) ** 2
    for k, g in gaps:
        assert g <= bound / (k + 1) ** 2 + 1e-10, (k, g, bound / (k + 1) ** 2)
    assert gaps[-1][1] < 1e-3 * gaps[0][1]


def pin_fista_least_squares():
    """lambda = 0: FISTA converges to the least-squares solution E0^{-1} b."""
    A, y, E0, b, L, apply_E0, shape = _small_problem(seed=6)
    x, _ = F.fista(apply_E0, b, 0.0, L, 2 if min(shape) >= 4 else 1, 2000)
    want = np.linalg.solve(E0, b.ravel())
    assert np.linalg.norm(x.ravel() - want) < 1e-9 * np.linalg.norm(want)


def pin_momentum():
    """t_{k+1}^2 - t_{k+1} = t_k^2, t_k >= (k + 1) / 2 (Beck-Teboulle Lemma 4.3),
    t_2 = golden ratio, mu_1 = 0."""
    t, mu = F.momentum(50)
    assert t[0] == 1.0 and abs(t[1] - (1 + math.sqrt(5)) / 2) < 1e-15 and mu[0] == 0.0
    for k in range(50):
        assert abs(t[k + 1] ** 2 - t[k + 1] - t[k] ** 2) < 1e-10 * t[k + 1] ** 2
        assert t[k] >= (k + 2) / 2.0 - 1e-12  # t[k] holds t_{k+1}
        assert abs(mu[k] - (t[k] - 1) / t[k + 1]) < 1e-15


def pin_max_eig():
    rng = np.random.Generator(np.random.PCG64(8))
    Q, _ = np.linalg.qr(_crandn(rng, (24, 24)))
    ev = np.linspace(0.1, 1.0, 24)
    ev[-1] = 3.0
    M = (Q * ev) @ Q.conj().T
    rq, v = F.max_eig(lambda u: M @ u, _crandn(rng, 24), 60)
    assert abs(rq - 3.0) < 1e-10
    assert abs(abs(np.vdot(v, Q[:, -1])) - 1.0) < 1e-8


PINS = [pin_hadamard_one_level, pin_haar_basis, pin_constant_volume, pin_soft_threshold_minimises,
        pin_prox_minimises, pin_single_atom_denoising, pin_fista_optimality, pin_fista_rate,
        pin_fista_least_squares, pin_momentum, pin_max_eig]


@pytest.mark.parametrize("pin", PINS, ids=[p.__name__ for p in PINS])
def test_pin(pin):
    pin()


def test_levels_argument_checks():
    with pytest.raises(ValueError):
        F.haar_forward(np.zeros((4, 6, 8)), 2)
    with pytest.raises(ValueError):
        F.haar_forward(np.zeros((4, 4, 4)), -1)
    x = np.arange(64.0).reshape(4, 4, 4) + 0j
    assert np.array_equal(F.haar_forward(x, 0), x) and np.array_equal(F.haar_inverse(x, 0), x)


# ----------------------------------------------------------- mutants ---------

def _mutants():
    """(name, attribute, replacement): one plausible mistake each."""
    orig_soft, orig_fwd, orig_inv = F.soft_threshold, F.haar_forward, F.haar_inverse
    orig_mom = F.momentum

    def fista_grad_no_two(apply_E0, b, lam, L, levels, maxit, x0=None, callback=None):
        return orig_fista(lambda v: 0.5 * apply_E0(v) + 0.5 * 0, 0.5 * np.asarray(b), lam, L,
                          levels, maxit, x0, callback)

    def soft_double(c, tau):
        return orig_soft(c, 2.0 * tau)

    def soft_hard(c, tau):
        c = np.asarray(c, dtype=np.complex128)
        return np.where(np.abs(c) > tau, c, 0)

    def fwd_unnormalised(x, levels):
        return orig_fwd(x, levels) * (1.0 if levels == 0 else 2.0 ** (0.5 * levels))

    def fwd_swapped_bands(x, levels):
        c = orig_fwd(x, levels)
        if levels and c.shape[0] >= 2:
            h = c.shape[0] // 2
            c = np.concatenate((c[h:], c[:h]), axis=0)
        return c

    def inv_high_sign(c, levels):
        c2 = np.array(c, dtype=np.complex128)
        if levels:
            c2[c2.shape[0] // 2:] *= -1.0
        return orig_inv(c2, levels)

    def inv_flip_axis(c, levels):
        x = orig_inv(c, levels)
        return x[:, :, ::-1] if levels else x

    def momentum_ratio(maxit):
        t, _ = orig_mom(maxit)
        return t, t[:-1] / t[1:]

    def momentum_none(maxit):
        t, mu = orig_mom(maxit)
        return t, np.zeros_like(mu)

    orig_fista = F.fista
    return [
        ("gradient without the factor 2", "fista", fista_grad_no_two),
        ("threshold at 2 tau", "soft_threshold", soft_double),
        ("hard threshold", "soft_threshold", soft_hard),
        ("unnormalised Haar", "haar_forward", fwd_unnormalised),
        ("swapped sub-bands", "haar_forward", fwd_swapped_bands),
        ("inverse with the wrong high-band sign", "haar_inverse", inv_high_sign),
        ("inverse with a flipped axis", "haar_inverse", inv_flip_axis),
        ("momentum t_k / t_{k+1}", "momentum", momentum_ratio),
        ("no momentum (ISTA)", "momentum", momentum_none),
    ]


def _pins_hold():
    for pin in PINS:
        try:
            pin()
        except (AssertionError, ValueError, IndexError, np.linalg.LinAlgError):
            return False
    return True


def test_pins_catch_planted_mistakes(monkeypatch):
    assert _pins_hold()
    for name, attr, repl in _mutants():
        with monkeypatch.context() as m:
            m.setattr(F, attr, repl)
            assert not _pins_hold(), f"no pin catches: {name}"
