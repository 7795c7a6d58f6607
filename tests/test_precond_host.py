"""Host-side logic of the preconditioner trainer (CPU only)."""

import numpy as np

from oracle import cnn as R
from paper_2501_16713_gb300 import precond
from paper_2501_16713_gb300.nrsense import Cnn


def _dc(v, a):
    p = np.pad(v, 1)
    hi = [slice(1, -1)] * 3
    lo = [slice(1, -1)] * 3
    hi[a], lo[a] = slice(2, None), slice(0, -2)
    return 0.5 * (p[tuple(hi)] - p[tuple(lo)])


def test_laplacian_params_give_i_minus_c_laplacian():
    rng = np.random.default_rng(0)
    shape = (5, 6, 4)
    r = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    c = 7.0
    params = [(w.astype(np.float64), b.astype(np.float64)) for w, b in precond.laplacian_params(c)]
    z, _ = R.forward_spd(params, r)
    u0 = r / R.input_scale(r)
    ref = u0 + c * sum(-_dc(_dc(u0, a), a) for a in range(3))
    assert np.allclose(z, ref, atol=1e-10)


def test_forward_stencil_gives_seven_point_laplacian():
    rng = np.random.default_rng(1)
    shape = (5, 4, 6)
    r = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    c = 3.0
    params = [(w.astype(np.float64), b.astype(np.float64))
              for w, b in precond.laplacian_params(c, "forward")]
    z, _ = R.forward_spd(params, r)
    u0 = r / R.input_scale(r)

    def df(v, a):  # forward difference with zero padding: v[i+1] - v[i]
        p = np.pad(v, [(0, 1) if k == a else (0, 0) for k in range(3)])
        hi = [slice(None)] * 3
        hi[a] = slice(1, None)
        return p[tuple(hi)] - v

    def dft(v, a):  # its transpose: v[i-1] - v[i]
        p = np.pad(v, [(1, 0) if k == a else (0, 0) for k in range(3)])
        lo = [slice(None)] * 3
        lo[a] = slice(0, -1)
        return p[tuple(lo)] - v

    ref = u0 + c * sum(dft(df(u0, a), a) for a in range(3))
    assert np.allclose(z, ref, atol=1e-10)


def test_param_flatten_roundtrip_and_count():
    params = R.init_params(3)
    flat = Cnn.flatten(params)
    assert flat.size == sum(w.size + b.size for w, b in params) == 22530
    back = Cnn.unflatten(flat)
    for (w, b), (w2, b2) in zip(params, back):
        assert np.array_equal(w.astype(np.float32), w2) and np.array_equal(b.astype(np.float32), b2)
