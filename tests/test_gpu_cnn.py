"""GPU preconditioner network (forward, gradients, Adam) vs the FP64 oracle.

The GPU network stores weights, activations and back-propagated gradients in
BF16 and accumulates in FP32 on the tensor cores.  The oracle is run with the
same BF16 weights and, where stated, with its rounding hook set to BF16 round
to nearest even at the same points (network input, hidden activations,
dL/do, masked activation gradients).  What then differs is FP32 against FP64
accumulation (about 1e-7 relative) and the rare stored value that lands on
the other side of a BF16 rounding boundary because of it (one BF16 ulp,
2^-8 relative, in a small fraction of values); tolerances are set an order
of magnitude above the resulting 1e-4 level.  Without the rounding hook the
difference is the BF16 storage error itself, 2^-9 relative per stored value
over five layers, a few 1e-3.

The volume (9, 13, 37) spans several 4 x 8 x 16 output blocks per axis with a
ragged tail on every axis.
"""

import ctypes

import numpy as np
import pytest

from helpers import rel_l2, to_dev
from oracle import cnn as R

pytestmark = pytest.mark.gpu

SHAPE = (9, 13, 37)
TOL_EMULATED = 2e-3     # o = z - u0 with matching rounding points
TOL_EXACT = 3e-2        # o against the unrounded FP64 definition
TOL_GRAD = 1e-2         # parameter gradients, matching rounding points, per layer
# symmetric form: ten stored BF16 intermediates in series instead of five
TOL_EMULATED_SYM = 5e-3
TOL_EXACT_SYM = 8e-2


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()


def _params(seed):
    rng = np.random.default_rng(seed)
    params = R.init_params(seed)
    out = []
    for l, (w, b) in enumerate(params):
        # a larger last layer than the initialisation so o is not negligible
        w = w * (5.0 if l == len(params) - 1 else 1.0)
        out.append((w.astype(np.float32), (0.1 * rng.standard_normal(b.shape)).astype(np.float32)))
    return out


def _bf16_weights(params):
    return [(R.bf16_round(w), b.astype(np.float64)) for w, b in params]


def _field(seed, shape=SHAPE):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).astype(np.complex64)


def _net(params, shape=SHAPE, symmetric=False):  # plain form unless stated
    from paper_2501_16713_gb300 import Cnn
    net = Cnn(shape, symmetric=symmetric)
    net.set_params(params)
    return net


def _nobias(params):
    return [(w, np.zeros_like(b)) for w, b in params]


def test_param_roundtrip_and_invalid_arguments():
    from paper_2501_16713_gb300 import Cnn, NrsenseError
    p = _params(1)
    net = _net(p)
    q = net.get_params()
    for (w, b), (w2, b2) in zip(p, q):
        assert np.array_equal(w, w2) and np.array_equal(b, b2)
    flat = Cnn.flatten(p)
    with pytest.raises(ValueError):
        net.set_params(flat[:-1])
    bad = flat.copy()
    bad[7] = np.nan
    with pytest.raises(NrsenseError) as ei:
        net.set_params(bad)
    assert ei.value.code == -1
    with pytest.raises(NrsenseError):
        Cnn((0, 4, 4))
    assert net.lib.nrsense_cnn_create(None, 0, None, None) == -1
    n = (ctypes.c_int32 * 3)(4, 4, 4)
    h = ctypes.c_void_p()
    assert net.lib.nrsense_cnn_create(n, 0x80, None, ctypes.byref(h)) == -1  # unknown flag
    net.close()


def test_forward_matches_oracle():
    p = _params(2)
    net = _net(p)
    r = _field(3)
    z = net.apply(to_dev(r)).cpu().numpy()
    pb = _bf16_weights(p)
    r64 = r.astype(np.complex128)
    u0 = r64 / R.input_scale(r64)
    z_em, _ = R.forward(pb, r64, rnd=R.bf16_round)
    z_ex, _ = R.forward(pb, r64)
    o_gpu = z - u0
    e_em = rel_l2(o_gpu, z_em - u0)
    e_ex = rel_l2(o_gpu, z_ex - u0)
    print(f"o rel L2: emulated rounding {e_em:.2e}, exact {e_ex:.2e}; z rel L2 {rel_l2(z, z_em):.2e}")
    assert e_em < TOL_EMULATED
    assert e_ex < TOL_EXACT
    assert rel_l2(z, z_em) < TOL_EMULATED


def test_zero_residual_gives_zero_direction():
    import torch
    net = _net(_params(4))
    z = net.apply(torch.zeros(SHAPE, dtype=torch.complex64, device="cuda"))
    assert float(z.abs().max()) == 0.0


def test_gradients_match_oracle():
    p = _params(5)
    net = _net(p)
    r, e = _field(6), _field(7)
    L = net.gradients(to_dev(r), to_dev(e))
    g = net.get_grads()
    pb = _bf16_weights(p)
    L_ref, g_ref = R.loss_and_grads(pb, r.astype(np.complex128), e.astype(np.complex128),
                                    rnd=R.bf16_round)
    print(f"loss gpu {L:.8f} oracle {L_ref:.8f}")
    assert abs(L - L_ref) < 1e-4
    for l, ((gw, gb), (rw, rb)) in enumerate(zip(g, g_ref)):
        ew, eb = rel_l2(gw, rw), rel_l2(gb, rb)
        print(f"layer {l}: dW rel {ew:.2e}, db rel {eb:.2e}")
        assert ew < TOL_GRAD, l
        assert eb < TOL_GRAD, l


def test_energy_loss_gradients_match_oracle():
    # energy loss: E z from the GPU normal operator of a small plan; the
    # oracle applies its own FP64 normal operator to its own z
    import synth
    from helpers import make_plan
    from oracle import operators as O
    shape = (10, 14, 36)
    case = synth.small_case(shape, 2, 1, [3000], seed=18, max_disp=1.5, rigid=0.5)
    plan = make_plan(case, shape)
    geo = O.Geometry(shape)
    d64 = [d.astype(np.float64) for d in case["disp"]]
    lam = 5.0
    E = lambda v: O.normal(geo, v, d64, case["smaps"], case["coords"], lam)
    p = _params(19)
    net = _net(p, shape)
    # a valid pair: r = E e (so Re<e, r> = ||e||_E^2 > 0)
    e = _field(21, shape)
    r = E(e.astype(np.complex128)).astype(np.complex64)
    L = net.gradients(to_dev(r), to_dev(e), plan=plan, lam=lam)
    g = net.get_grads()
    L_ref, g_ref = R.loss_and_grads_energy(_bf16_weights(p), r.astype(np.complex128),
                                           e.astype(np.complex128), E, rnd=R.bf16_round)
    print(f"energy loss gpu {L:.8f} oracle {L_ref:.8f}")
    assert abs(L - L_ref) < 1e-4 * max(1.0, abs(L_ref))
    for l, ((gw, gb), (rw, rb)) in enumerate(zip(g, g_ref)):
        ew, eb = rel_l2(gw, rw), rel_l2(gb, rb)
        print(f"layer {l}: dW rel {ew:.2e}, db rel {eb:.2e}")
        assert ew < TOL_GRAD, l
        assert eb < TOL_GRAD, l
    plan.close()


def test_gradients_deterministic_and_accumulate():
    p = _params(8)
    net = _net(p)
    r1, e1, r2, e2 = (to_dev(_field(s)) for s in (9, 10, 11, 12))
    net.gradients(r1, e1)
    g1 = net.get_grads()
    net.gradients(r1, e1)
    g1b = net.get_grads()
    for (a, b), (c, d) in zip(g1, g1b):
        assert np.array_equal(a, c) and np.array_equal(b, d)
    net.gradients(r2, e2)
    g2 = net.get_grads()
    net.gradients(r1, e1)
    net.gradients(r2, e2, accumulate=True)
    g12 = net.get_grads()
    for (a, b), (c, d), (s, t) in zip(g1, g2, g12):
        assert np.array_equal(a + c, s) and np.array_equal(b + d, t)


def test_adam_first_step_moves_by_learning_rate():
    # from zero moments, Adam's first update is lr * g / (|g| + eps)
    p = _params(13)
    net = _net(p)
    net.gradients(to_dev(_field(14)), to_dev(_field(15)))
    g = net.get_grads()
    lr = 1e-3
    net.adam_step(lr)
    q = net.get_params()
    for (w0, b0), (gw, gb), (w1, b1) in zip(p, g, q):
        for a0, ga, a1 in ((w0, gw, w1), (b0, gb, b1)):
            big = np.abs(ga) > 1e-3
            step = a1.astype(np.float64) - a0.astype(np.float64)
            assert np.all(np.abs(step[big] + lr * np.sign(ga[big])) < 1e-6)
            assert np.all(step[ga == 0] == 0)


def test_adam_three_steps_match_oracle():
    # three updates with different gradients: the bias corrections 1 - beta^t
    # and the moment recursions for t = 2, 3 against the FP64 oracle's Adam
    # fed the same gradients (FP32 master weights: differences near 1e-7)
    p = _params(40)
    net = _net(p)
    ref = [(w.astype(np.float64), b.astype(np.float64)) for w, b in p]
    state = R.adam_init(ref)
    lr = 2e-3
    live = None
    for t, (sr, se) in enumerate(((41, 42), (43, 44), (45, 46))):
        net.gradients(to_dev(_field(sr)), to_dev(_field(se)))
        g = [(gw.astype(np.float64), gb.astype(np.float64)) for gw, gb in net.get_grads()]
        net.adam_step(lr)
        ref, state = R.adam_step(ref, g, state, lr)
        # entries whose gradient is tiny at some step make m / sqrt(v) ill-conditioned
        ok = [(np.abs(gw) > 1e-5, np.abs(gb) > 1e-5) for gw, gb in g]
        live = ok if live is None else [(a & c, b & d) for (a, b), (c, d) in zip(live, ok)]
        q = net.get_params()
        for (w1, b1), (wr, br), (lw, lb) in zip(q, ref, live):
            assert np.max(np.abs(w1[lw] - wr[lw])) < 1e-6, t
            assert np.max(np.abs(b1[lb] - br[lb])) < 1e-6, t
            assert lw.mean() > 0.5
    assert state[0] == 3


def test_training_steps_reduce_loss():
    from paper_2501_16713_gb300 import precond
    import torch
    p = _params(16)
    net = _net(p)
    r = to_dev(_field(17))
    # a smooth target: e = r blurred along every axis (a low-pass preconditioner)
    e = r.clone()
    for ax in range(3):
        e = 0.5 * e + 0.25 * (torch.roll(e, 1, ax) + torch.roll(e, -1, ax))
    L0 = precond.mean_loss(net, r[None], e[None])
    precond.train(net, r[None], e[None], steps=40, lr=3e-3, lr_final=1e-3, batch=1)
    L1 = precond.mean_loss(net, r[None], e[None])
    print(f"loss {L0:.4f} -> {L1:.4f}")
    assert L1 < 0.7 * L0


def test_symmetric_forward_matches_oracle():
    p = _nobias(_params(22))
    net = _net(p, symmetric=True)
    r = _field(23)
    z = net.apply(to_dev(r)).cpu().numpy()
    r64 = r.astype(np.complex128)
    u0 = r64 / R.input_scale(r64)
    z_em, _ = R.forward_spd(_bf16_weights(p), r64, rnd=R.bf16_round)
    z_ex, _ = R.forward_spd(_bf16_weights(p), r64)
    e_em, e_ex = rel_l2(z - u0, z_em - u0), rel_l2(z - u0, z_ex - u0)
    print(f"symmetric o rel L2: emulated {e_em:.2e}, exact {e_ex:.2e}")
    assert e_em < TOL_EMULATED_SYM and e_ex < TOL_EXACT_SYM


def test_symmetric_gradients_match_oracle():
    import synth
    from helpers import make_plan
    from oracle import operators as O
    shape = (10, 14, 36)
    case = synth.small_case(shape, 2, 1, [3000], seed=24, max_disp=1.5, rigid=0.5)
    plan = make_plan(case, shape)
    geo = O.Geometry(shape)
    d64 = [d.astype(np.float64) for d in case["disp"]]
    lam = 5.0
    E = lambda v: O.normal(geo, v, d64, case["smaps"], case["coords"], lam)
    p = _nobias(_params(25))
    net = _net(p, shape, symmetric=True)
    e = _field(26, shape)
    r = E(e.astype(np.complex128)).astype(np.complex64)
    pb = _bf16_weights(p)
    for energy in (False, True):
        L = net.gradients(to_dev(r), to_dev(e), plan=plan if energy else None, lam=lam)
        g = net.get_grads()
        L_ref, g_ref = R.loss_and_grads_spd(pb, r.astype(np.complex128), e.astype(np.complex128),
                                            E if energy else None, rnd=R.bf16_round)
        print(f"symmetric {'energy' if energy else 'cosine'} loss gpu {L:.8f} oracle {L_ref:.8f}")
        assert abs(L - L_ref) < 1e-4 * max(1.0, abs(L_ref))
        for l, ((gw, _), (rw, _)) in enumerate(zip(g, g_ref)):
            ew = rel_l2(gw, rw)
            print(f"  layer {l}: dW rel {ew:.2e}")
            assert ew < TOL_GRAD, (energy, l)
    plan.close()


@pytest.mark.parametrize("symmetric", [False, True])
def test_tcgen05_convolutions_match_mma_sync_and_oracle(symmetric):
    """The convolutions on the fifth-generation tensor cores (accumulators in
    tensor memory, one thread issuing the products) against the mma.sync
    kernels and the oracle: the same FP32 sums in another order, so the output
    agrees with the mma.sync path to about one BF16 ulp on a few stored values
    and meets the oracle tolerances; ragged blocks on every axis; bitwise
    reproducible; the device status word stays clear."""
    p = _nobias(_params(21)) if symmetric else _params(21)
    net = _net(p, symmetric=symmetric)
    r = _field(22)
    import torch
    z_mma = net.apply(to_dev(r)).cpu().numpy()
    net.set_conv(True)
    out = torch.full(SHAPE, float("nan"), dtype=torch.complex64, device="cuda")
    z_tc = net.apply(to_dev(r), out=out).cpu().numpy()  # every voxel written
    assert np.all(np.isfinite(z_tc))
    assert net.device_status() == 0
    assert np.array_equal(net.apply(to_dev(r)).cpu().numpy(), z_tc)
    r64 = r.astype(np.complex128)
    u0 = r64 / R.input_scale(r64)
    e = rel_l2(z_tc - u0, z_mma - u0)
    fwd = R.forward_spd if symmetric else R.forward
    z_em, _ = fwd(_bf16_weights(p), r64, rnd=R.bf16_round)
    e_em = rel_l2(z_tc - u0, z_em - u0)
    print(f"tcgen05 vs mma.sync: o rel L2 {e:.2e}; vs oracle (emulated rounding) {e_em:.2e}")
    assert e < (TOL_EMULATED_SYM if symmetric else TOL_EMULATED)
    assert e_em < (TOL_EMULATED_SYM if symmetric else TOL_EMULATED)
    net.set_conv(False)
    assert np.array_equal(net.apply(to_dev(r)).cpu().numpy(), z_mma)
    net.close()
