"""Pins of the FP64 preconditioner-network oracle (CPU only)."""

import numpy as np
import pytest
import scipy.ndimage

from oracle import cnn


def _rng(s=0):
    return np.random.Generator(np.random.PCG64(s))


def test_conv3d_matches_scipy_correlate():
    rng = _rng(1)
    x = rng.standard_normal((3, 5, 6, 7))
    w = rng.standard_normal((4, 3, 3, 3, 3))
    b = rng.standard_normal(4)
    got = cnn.conv3d(x, w, b)
    for o in range(4):
        ref = b[o] + sum(scipy.ndimage.correlate(x[c], w[o, c], mode="constant", cval=0.0)
                         for c in range(3))
        assert np.allclose(got[o], ref, rtol=1e-12, atol=1e-12)


def test_conv3d_delta_kernel_is_identity():
    rng = _rng(2)
    x = rng.standard_normal((4, 5, 5, 5))
    w = np.zeros((4, 4, 3, 3, 3))
    for c in range(4):
        w[c, c, 1, 1, 1] = 1.0
    assert np.array_equal(cnn.conv3d(x, w, np.zeros(4)), x)


def test_conv3d_backward_finite_differences():
    rng = _rng(3)
    x = rng.standard_normal((2, 4, 5, 3))
    w = rng.standard_normal((3, 2, 3, 3, 3))
    b = rng.standard_normal(3)
    dy = rng.standard_normal((3, 4, 5, 3))
    f = lambda xx, ww, bb: np.sum(dy * cnn.conv3d(xx, ww, bb))
    dx, dw, db = cnn.conv3d_backward(x, w, dy)
    h = 1e-6
    for _ in range(10):
        i = tuple(rng.integers(0, s) for s in x.shape)
        xp, xm = x.copy(), x.copy()
        xp[i] += h
        xm[i] -= h
        assert abs((f(xp, w, b) - f(xm, w, b)) / (2 * h) - dx[i]) < 1e-6 * (1 + abs(dx[i]))
        j = tuple(rng.integers(0, s) for s in w.shape)
        wp, wm = w.copy(), w.copy()
        wp[j] += h
        wm[j] -= h
        assert abs((f(x, wp, b) - f(x, wm, b)) / (2 * h) - dw[j]) < 1e-6 * (1 + abs(dw[j]))
    assert np.allclose(db, dy.sum(axis=(1, 2, 3)))


def test_network_gradients_finite_differences():
    rng = _rng(4)
    params = cnn.init_params(5)
    # non-zero biases so every path is exercised
    params = [(w, rng.standard_normal(b.shape) * 0.1) for w, b in params]
    shape = (4, 5, 4)
    r = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    e = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    L0, grads = cnn.loss_and_grads(params, r, e)
    assert 0.0 <= L0 <= 2.0
    h = 1e-6
    for l in range(len(params)):
        for _ in range(4):
            w, b = params[l]
            j = tuple(rng.integers(0, s) for s in w.shape)
            pp = [(ww.copy(), bb.copy()) for ww, bb in params]
            pm = [(ww.copy(), bb.copy()) for ww, bb in params]
            pp[l][0][j] += h
            pm[l][0][j] -= h
            fd = (cnn.loss_and_grads(pp, r, e)[0] - cnn.loss_and_grads(pm, r, e)[0]) / (2 * h)
            assert abs(fd - grads[l][0][j]) < 1e-6 * (1 + abs(fd)), (l, j)
        k = int(rng.integers(0, b.shape[0]))
        pp = [(ww.copy(), bb.copy()) for ww, bb in params]
        pm = [(ww.copy(), bb.copy()) for ww, bb in params]
        pp[l][1][k] += h
        pm[l][1][k] -= h
        fd = (cnn.loss_and_grads(pp, r, e)[0] - cnn.loss_and_grads(pm, r, e)[0]) / (2 * h)
        assert abs(fd - grads[l][1][k]) < 1e-6 * (1 + abs(fd))


def test_loss_is_scale_invariant_and_zero_at_target():
    rng = _rng(6)
    z = rng.standard_normal(50) + 1j * rng.standard_normal(50)
    assert cnn.loss(z, 3.7 * z) == pytest.approx(0.0, abs=1e-14)
    e = rng.standard_normal(50) + 1j * rng.standard_normal(50)
    assert cnn.loss(2.5 * z, e) == pytest.approx(cnn.loss(z, e), abs=1e-14)


def test_adam_first_step_textbook():
    # first Adam step moves each parameter by lr * sign(grad) (bias-corrected m/sqrt(v))
    params = [(np.array([[[[[1.0]]]]]), np.array([0.5]))]
    grads = [(np.array([[[[[0.3]]]]]), np.array([-2.0]))]
    new, state = cnn.adam_step(params, grads, cnn.adam_init(params), lr=0.01)
    assert new[0][0].item() == pytest.approx(1.0 - 0.01, abs=1e-9)
    assert new[0][1].item() == pytest.approx(0.5 + 0.01, abs=1e-9)


def test_adam_three_steps_textbook_values():
    # Kingma & Ba's Algorithm 1 worked by hand (decimal arithmetic) for one
    # scalar weight, lr 0.01, betas 0.9 / 0.999, eps 1e-8, gradients 0.3, -0.1, 0.2:
    #   t=1: m=0.03,   v=0.00009,     m^=0.3,        v^=0.09
    #   t=2: m=0.017,  v=0.00009991,  m^=0.017/0.19, v^=0.00009991/0.001999
    #   t=3: m=0.0353, v=0.00013981009, m^=0.0353/0.271, v^=0.00013981009/0.002997001
    # A bias correction that ignores t, or one applied to the wrong moment,
    # changes steps 2 and 3.
    expect = [(0.03, 0.00009, 0.9900000003333333222),
              (0.017, 0.00009991, 0.9859978147928080520),
              (0.0353, 0.00013981009, 0.9799669501576138839)]
    params = [(np.array([[[[[1.0]]]]]), np.array([0.0]))]
    state = cnn.adam_init(params)
    for g, (m, v, w) in zip((0.3, -0.1, 0.2), expect):
        grads = [(np.array([[[[[g]]]]]), np.array([0.0]))]
        params, state = cnn.adam_step(params, grads, state, lr=0.01)
        assert state[1][0][0].item() == pytest.approx(m, rel=1e-12)
        assert state[2][0][0].item() == pytest.approx(v, rel=1e-12)
        assert params[0][0].item() == pytest.approx(w, abs=1e-15)
    assert state[0] == 3


def test_adam_constant_gradient_moves_by_lr_every_step():
    # with a constant gradient g the bias-corrected moments are exactly g and
    # g^2 at every t, so each step moves by lr * sign(g) (up to eps)
    params = [(np.array([[[[[0.2, -0.4]]]]]), np.array([1.5]))]
    grads = [(np.array([[[[[2.5, -0.8]]]]]), np.array([-7.0]))]
    state = cnn.adam_init(params)
    for t in range(1, 6):
        params, state = cnn.adam_step(params, grads, state, lr=0.05)
        w, b = params[0]
        assert w.ravel() == pytest.approx([0.2 - 0.05 * t, -0.4 + 0.05 * t], abs=1e-8)
        assert b.item() == pytest.approx(1.5 + 0.05 * t, abs=1e-8)


def test_bf16_round_matches_torch():
    torch = pytest.importorskip("torch")
    rng = _rng(7)
    a = (rng.standard_normal(1000) * 10 ** rng.uniform(-5, 5, 1000)).astype(np.float32)
    ref = torch.from_numpy(a).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(cnn.bf16_round(a), ref)


def _spd(rng, n):
    a = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    return a.conj().T @ a + 0.5 * np.eye(n)


def test_energy_loss_zero_at_target_and_line_search_identity():
    # L(e) = 0; for any z, 1 - L(z) is the energy fraction removed by the
    # exact line search x + a z (computed here by brute minimisation over a)
    rng = _rng(8)
    n = 12
    E = _spd(rng, n)
    e = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    r = E @ e
    assert cnn.loss_energy(e, r, e, E @ e) == pytest.approx(0.0, abs=1e-12)
    z = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    err = lambda a: np.real(np.vdot(e - a * z, E @ (e - a * z)))
    coarse = np.linspace(-5, 5, 2001)
    a0 = coarse[np.argmin([err(t) for t in coarse])]
    fine = np.linspace(a0 - 0.01, a0 + 0.01, 4001)
    best = min(err(t) for t in fine)
    removed = 1.0 - best / err(0.0)
    c = np.real(np.vdot(z, r))
    L = cnn.loss_energy(z, r, e, E @ z)
    assert (1.0 - L) * np.sign(c) == pytest.approx(removed, abs=1e-6)
    assert cnn.loss_energy(-z, r, e, E @ -z) == pytest.approx(1.0 + removed, abs=1e-6)


def test_energy_loss_network_gradients_finite_differences():
    rng = _rng(9)
    params = cnn.init_params(10)
    params = [(w, rng.standard_normal(b.shape) * 0.1) for w, b in params]
    shape = (3, 4, 3)
    n = int(np.prod(shape))
    Em = _spd(rng, n)
    E = lambda v: (Em @ v.ravel()).reshape(shape)
    e = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    r = E(e)
    L0, grads = cnn.loss_and_grads_energy(params, r, e, E)
    h = 1e-6
    f = lambda pp: cnn.loss_and_grads_energy(pp, r, e, E)[0]
    for l in range(len(params)):
        for _ in range(3):
            w, b = params[l]
            j = tuple(rng.integers(0, s) for s in w.shape)
            pp = [(ww.copy(), bb.copy()) for ww, bb in params]
            pm = [(ww.copy(), bb.copy()) for ww, bb in params]
            pp[l][0][j] += h
            pm[l][0][j] -= h
            fd = (f(pp) - f(pm)) / (2 * h)
            assert abs(fd - grads[l][0][j]) < 1e-6 * (1 + abs(fd)), (l, j)


def test_conv3d_transpose_is_adjoint():
    rng = _rng(11)
    x = rng.standard_normal((3, 4, 5, 6))
    y = rng.standard_normal((2, 4, 5, 6))
    w = rng.standard_normal((2, 3, 3, 3, 3))
    lhs = np.sum(y * cnn.conv3d(x, w, np.zeros(2)))
    rhs = np.sum(x * cnn.conv3d_transpose(y, w))
    assert abs(lhs - rhs) < 1e-10 * abs(lhs)


def test_symmetric_form_is_spd_for_fixed_masks():
    # with the masks of one forward pass held fixed, u0 -> o is a linear map;
    # build its dense matrix column by column and check I + matrix is
    # symmetric with eigenvalues >= 1
    rng = _rng(12)
    params = cnn.init_params(13)
    shape = (4, 4, 4)
    r = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    _, (h, _, _) = cnn.forward_spd(params, r)
    L = len(params)
    zero = lambda w: np.zeros(w.shape[0])

    def o_of(u0):
        hh = u0
        for l in range(L - 1):
            hh = cnn.conv3d(hh, params[l][0], zero(params[l][0])) * (h[l + 1] > 0)
        w5 = params[L - 1][0]
        u = hh + cnn.conv3d_transpose(cnn.conv3d(hh, w5, zero(w5)), w5) * (h[L - 1] > 0)
        for l in range(L - 2, 0, -1):
            u = cnn.conv3d_transpose(u, params[l][0]) * (h[l] > 0)
        return cnn.conv3d_transpose(u, params[0][0])

    n = 2 * int(np.prod(shape))
    basis = np.eye(n).reshape(n, 2, *shape)
    M = np.stack([o_of(b).ravel() for b in basis], axis=1) + np.eye(n)
    assert np.allclose(M, M.T, atol=1e-10)
    assert np.linalg.eigvalsh(M).min() >= 1.0 - 1e-10
    # the forward pass is this map applied to u0 = r / s (masks consistent)
    z, _ = cnn.forward_spd(params, r)
    u0 = np.stack([r.real, r.imag]) / cnn.input_scale(r)
    zz = (M @ u0.ravel()).reshape(u0.shape)
    assert np.allclose(z, zz[0] + 1j * zz[1], atol=1e-10)


def test_symmetric_form_contains_the_laplacian():
    # first layer +-central differences, identity hidden layers, W_5 = 0:
    # z = u0 + c (-Laplacian_2h) u0 with the wide (2h) central stencil
    shape = (6, 5, 7)
    rng = _rng(16)
    params = []
    for cin, cout in zip(cnn.CHANNELS[:-1], cnn.CHANNELS[1:]):
        params.append((np.zeros((cout, cin, 3, 3, 3)), np.zeros(cout)))
    w1 = params[0][0]
    for a in range(3):
        for comp in range(2):
            ch = 4 * a + 2 * comp
            idx_p = [1, 1, 1]
            idx_m = [1, 1, 1]
            idx_p[a], idx_m[a] = 2, 0
            w1[ch, comp][tuple(idx_p)], w1[ch, comp][tuple(idx_m)] = 0.5, -0.5
            w1[ch + 1, comp][tuple(idx_p)], w1[ch + 1, comp][tuple(idx_m)] = -0.5, 0.5
    for l in (1, 2, 3):
        for ch in range(12):
            params[l][0][ch, ch, 1, 1, 1] = 1.0
    r = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    z, _ = cnn.forward_spd(params, r)
    u0 = r / cnn.input_scale(r)
    # -sum_a D_a^T D_a u0 with D_a the central difference (zero padding)
    def dc(v, a):
        p = np.pad(v, 1)
        sl_p = [slice(1, -1)] * 3
        sl_m = [slice(1, -1)] * 3
        sl_p[a], sl_m[a] = slice(2, None), slice(0, -2)
        return 0.5 * (p[tuple(sl_p)] - p[tuple(sl_m)])
    ref = u0 + sum(-dc(dc(u0, a), a) for a in range(3))
    assert np.allclose(z, ref, atol=1e-12)


def test_symmetric_form_gradients_finite_differences():
    rng = _rng(14)
    params = [(w, np.zeros_like(b)) for w, b in cnn.init_params(15)]
    params[-1] = (params[-1][0] * 10, params[-1][1])
    shape = (3, 4, 3)
    n = int(np.prod(shape))
    Em = _spd(rng, n)
    E = lambda v: (Em @ v.ravel()).reshape(shape)
    e = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    r = E(e)
    for EE in (None, E):
        L0, grads = cnn.loss_and_grads_spd(params, r, e, EE)
        h = 1e-6
        f = lambda pp: cnn.loss_and_grads_spd(pp, r, e, EE)[0]
        for l in range(len(params)):
            for _ in range(3):
                w, b = params[l]
                j = tuple(rng.integers(0, s) for s in w.shape)
                pp = [(ww.copy(), bb.copy()) for ww, bb in params]
                pm = [(ww.copy(), bb.copy()) for ww, bb in params]
                pp[l][0][j] += h
                pm[l][0][j] -= h
                fd = (f(pp) - f(pm)) / (2 * h)
                assert abs(fd - grads[l][0][j]) < 1e-6 * (1 + abs(fd)), (EE is None, l, j)
