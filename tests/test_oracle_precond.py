"""Pins of the circulant preconditioner oracle (CPU only).

For an operator that is exactly circulant, E0 x = IDFT(q . DFT(x)), the
preconditioner is the closed-form inverse d = 1 / (q + lambda) and CG on
(E0 + lambda I) preconditioned by it converges in one step; the PSF of a
circular convolution is its kernel centred on the image centre; eigenvalues
below zero are clamped (d = 1 / lambda there).  The last test plants
mistakes and requires each to fail a pin.
"""

import numpy as np
import pytest

from oracle import precond as Pc
from oracle import solvers as S


def _circ(q):
    return lambda x: np.fft.ifftn(q * np.fft.fftn(x))


def pin_exact_inverse_of_circulant():
    rng = np.random.default_rng(1)
    shape, lam = (6, 8, 4), 0.3
    q = rng.uniform(0.5, 4.0, shape)
    d = Pc.circulant_diag(_circ(q), shape, lam)
    assert np.abs(d - 1.0 / (q + lam)).max() < 1e-12
    x = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    Ex = _circ(q)(x) + lam * x
    assert np.abs(Pc.apply_circulant(d, Ex) - x).max() < 1e-12 * np.abs(x).max()
    # preconditioned CG (CG on the similar system M^1/2 (E + lam) M^1/2) in one step
    sq = np.sqrt(d)
    b = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    Ms = lambda v: np.fft.ifftn(sq * np.fft.fftn(v))
    _, it, hist = S.cg(lambda v: Ms(_circ(q)(Ms(v)) + lam * Ms(v)), Ms(b), tol=1e-10, maxit=5)
    assert it == 1 and hist[-1] < 1e-10


def pin_psf_of_convolution():
    rng = np.random.default_rng(2)
    shape = (8, 6, 10)
    k = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)  # kernel, origin at 0
    conv = lambda x: np.fft.ifftn(np.fft.fftn(k) * np.fft.fftn(x))
    h = Pc.psf(conv, shape)
    want = np.roll(k, tuple(s // 2 for s in shape), axis=(0, 1, 2))
    assert np.abs(h - want).max() < 1e-12


def pin_negative_eigenvalues_clamped():
    rng = np.random.default_rng(3)
    shape, lam = (4, 4, 4), 0.25
    q = rng.uniform(-1.0, 2.0, shape)
    d = Pc.circulant_diag(_circ(q), shape, lam)
    want = np.where(q > 0, 1.0 / (q + lam), 1.0 / lam)
    assert np.abs(d - want).max() < 1e-11


PINS = [pin_exact_inverse_of_circulant, pin_psf_of_convolution, pin_negative_eigenvalues_clamped]


@pytest.mark.parametrize("pin", PINS, ids=[p.__name__ for p in PINS])
def test_pin(pin):
    pin()


def test_pins_catch_planted_mistakes(monkeypatch):
    orig_psf = Pc.psf

    def diag_no_roll(apply_E0, shape, lam):
        hhat = np.fft.fftn(orig_psf(apply_E0, shape))
        return 1.0 / (np.maximum(hhat.real, 0.0) + lam)

    def diag_abs(apply_E0, shape, lam):
        h = orig_psf(apply_E0, shape)
        hhat = np.fft.fftn(np.roll(h, tuple(-(s // 2) for s in shape), axis=(0, 1, 2)))
        return 1.0 / (np.abs(hhat) + lam)

    def psf_corner(apply_E0, shape):
        d = np.zeros(shape, dtype=np.complex128)
        d[0, 0, 0] = 1.0
        return apply_E0(d)

    for name, attr, repl in [("no centre shift", "circulant_diag", diag_no_roll),
                             ("modulus instead of real part", "circulant_diag", diag_abs),
                             ("impulse at the corner", "psf", psf_corner)]:
        with monkeypatch.context() as m:
            m.setattr(Pc, attr, repl)
            failed = False
            for pin in PINS:
                try:
                    pin()
                except AssertionError:
                    failed = True
            assert failed, f"no pin catches: {name}"
