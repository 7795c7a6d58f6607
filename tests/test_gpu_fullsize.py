"""Full-size checks on the 128^3, 8-coil, 4-phase workload that bench.py times.

The same plan configuration as the benchmark (automatic phase chunking, the
autotuned kernel choices).  The FP64 oracle cannot run the whole operator at
this size in test time, so the checks are (a) sampled outputs the oracle
computes one by one from its own step-by-step intermediates (the warped image
at sampled voxels; k-space samples of one phase and two coils), (b) the
adjoint of data that are nonzero on 300 samples of one phase in two coils,
which the oracle computes exactly, and (c) properties that hold at any size:
adjointness of A, symmetry and positivity of the normal operator.
"""

import numpy as np
import pytest

import synth
from helpers import TOL_ADJ, TOL_FP32, make_plan, to_dev
from oracle import operators as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def full():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    w = synth.workload("sense128")
    plan = make_plan(w, w["spec"].shape)
    # the benchmark's launch configuration: the autotuned choices
    tuning = plan.autotune(reps=2)
    print("tuning", tuning)
    yield w, plan
    plan.close()


def _upsampled(geo, x):
    """The oracle's T_j intermediate u = F_G^H Z (1/C*) F_N x (steps 1-4)."""
    X = O.sfft.fftn(np.asarray(x, np.complex128))
    for a in range(3):
        shp = [1, 1, 1]
        shp[a] = -1
        X = X * O._deapod_table(geo, a, geo.kspace_freqs(a)).reshape(shp)
    U = np.zeros(geo.grid, np.complex128)
    U[np.ix_(*[O._pad_index(geo, a) for a in range(3)])] = X
    return O.sfft.ifftn(U) * O._upsample_scale(geo)


def test_full_warp_sampled_voxels(full):
    w, plan = full
    geo = O.Geometry(w["spec"].shape)
    m = plan.warp_forward(to_dev(w["x"])).cpu().numpy()
    u = _upsampled(geo, w["x"])
    rng = np.random.default_rng(0)
    nv = int(np.prod(geo.shape))
    for j in (0, 3):
        sel = rng.choice(nv, 400, replace=False)
        q = O.warp_positions(geo, w["disp"][j].astype(np.float64))[:, sel]
        ref = O.backprojection_core(u, q, geo.width, geo.beta)
        got = m[j].reshape(-1)[sel]
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < TOL_FP32


def test_full_forward_sampled_kspace(full):
    w, plan = full
    geo = O.Geometry(w["spec"].shape)
    y = plan.forward(to_dev(w["x"])).cpu().numpy()
    j = 1
    m = O.warp_forward(geo, w["x"], w["disp"][j].astype(np.float64))
    rng = np.random.default_rng(1)
    sel = rng.choice(w["coords"][j].shape[0], 300, replace=False)
    yj = plan.phase_slice(y, j)
    for c in (0, 5):
        ref = O.kspace_forward(geo, w["smaps"][c] * m, w["coords"][j][sel])
        got = yj[sel, c]
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < TOL_FP32, c


def test_full_adjointness_and_normal_operator(full):
    import torch
    w, plan = full
    shape = w["spec"].shape
    rng = np.random.default_rng(2)
    x = to_dev((rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).astype(np.complex64))
    z = to_dev((rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).astype(np.complex64))
    ysh = plan.forward_shape()
    y = to_dev((rng.standard_normal(ysh) + 1j * rng.standard_normal(ysh)).astype(np.complex64))
    d = lambda a: a.flatten().to(torch.complex128)
    Ax = plan.forward(x)
    Ahy = plan.adjoint(y)
    lhs, rhs = torch.vdot(d(y), d(Ax)), torch.vdot(d(Ahy), d(x))
    assert abs(complex(lhs - rhs)) / float(torch.linalg.norm(d(Ax)) * torch.linalg.norm(d(y))) < TOL_ADJ
    Ex, Ez = plan.normal(x, 0.0), plan.normal(z, 0.0)
    s1, s2 = torch.vdot(d(z), d(Ex)), torch.vdot(d(Ez), d(x))
    assert abs(complex(s1 - s2)) / float(torch.linalg.norm(d(Ex)) * torch.linalg.norm(d(z))) < TOL_ADJ
    xEx = torch.vdot(d(x), d(Ex))
    assert xEx.real.item() > 0 and abs(xEx.imag.item()) < 1e-5 * xEx.real.item()
    # E x equals A^H (A x) at full size
    AhAx = plan.adjoint(Ax)
    assert float(torch.linalg.norm(d(AhAx) - d(Ex)) / torch.linalg.norm(d(Ex))) < 1e-6


def test_full_adjoint_sparse_data(full):
    w, plan = full
    geo = O.Geometry(w["spec"].shape)
    rng = np.random.default_rng(3)
    j, coils = 1, (0, 5)
    M = [c.shape[0] for c in w["coords"]]
    sel = rng.choice(M[j], 300, replace=False)
    y = np.zeros((sum(M), 8), np.complex64)
    off = int(np.sum(M[:j]))
    vals = (rng.standard_normal((300, 2)) + 1j * rng.standard_normal((300, 2))).astype(np.complex64)
    for k, c in enumerate(coils):
        y[off + sel, c] = vals[:, k]
    got = plan.adjoint(to_dev(y)).cpu().numpy()
    # oracle: T_j^H sum_c conj(S_c) G_j^H y_c over the 300 samples
    v = np.zeros(geo.shape, np.complex128)
    for k, c in enumerate(coils):
        g = O.kspace_adjoint(geo, vals[:, k].astype(np.complex128), w["coords"][j][sel])
        v += np.conj(w["smaps"][c]) * g
    ref = O.warp_adjoint(geo, v, w["disp"][j].astype(np.float64))
    e = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    print(f"full-size adjoint of sparse data: rel L2 {e:.2e}")
    assert e < TOL_FP32


def test_full_phase_one_coil_every_value(full):
    # G_0 and G_0^H of the benchmark plan (its autotuned kernels) for one coil,
    # every output value against the oracle: all 1.5 M samples of the
    # forward, all 2.1 M voxels of the adjoint; the other coils' inputs are
    # zero and so must be their outputs
    from helpers import rel_l2
    w, plan = full
    shape = w["spec"].shape
    geo = O.Geometry(shape)
    C = w["spec"].n_coils
    om = w["coords"][0]
    v = np.zeros((C,) + shape, np.complex64)
    v[0] = (w["x"] * w["smaps"][0]).astype(np.complex64)
    y = plan.kspace_forward(0, to_dev(v)).cpu().numpy()
    yref = O.kspace_forward(geo, v[0].astype(np.complex128), om)
    e = rel_l2(y[:, 0], yref)
    print(f"G_0, coil 0, {yref.size} samples: rel L2 {e:.2e}")
    assert e < TOL_FP32
    assert not np.any(y[:, 1:])
    rng = np.random.default_rng(8)
    yin = np.zeros((om.shape[0], C), np.complex64)
    yin[:, 0] = (rng.standard_normal(om.shape[0]) + 1j * rng.standard_normal(om.shape[0]))
    xa = plan.kspace_adjoint(0, to_dev(yin)).cpu().numpy()
    xref = O.kspace_adjoint(geo, yin[:, 0].astype(np.complex128), om)
    ea = rel_l2(xa[0], xref)
    print(f"G_0^H, coil 0, {xref.size} voxels: rel L2 {ea:.2e}")
    assert ea < TOL_FP32
    assert not np.any(xa[1:])
