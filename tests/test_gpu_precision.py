"""Precision variants of the operator (GPU) against the FP64 oracle.

* NRSENSE_FP32: the 1e-5 relative L2 bar.
* NRSENSE_FP32_COMPENSATED: same bar; on a trajectory that piles hundreds of
  thousands of samples onto each central grid value, compensated spreading
  is at least as accurate as plain FP32 accumulation on the k-space adjoint,
  and both stay far below 1e-5: the split of heavy tiles into chunks of at
  most 1024 points already bounds every FP32 accumulation chain, so the
  remaining error is that of the FP32 kernel weights and FFTs.
* NRSENSE_BF16_STORE: the k-space coil grids are stored in BF16 (8-bit
  significand, unit roundoff 2^-9 ~ 2e-3 under round to nearest even) twice
  per direction (before and after the FFT) and transformed by cuFFT's BF16
  FFT; arithmetic is FP32 elsewhere.  A few 1e-3 relative L2 is the expected
  error, so the tolerance is 1e-2 for A, A^H and adjointness.
"""

import math

import numpy as np
import pytest

import synth
from helpers import TOL_ADJ, TOL_FP32, make_plan, rel_l2, to_dev
from oracle import operators as O

pytestmark = pytest.mark.gpu

TOL_BF16 = 1e-2


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()


def _case():
    shape = (16, 32, 32)  # oversampled grid 32 x 64 x 64: powers of two
    return shape, synth.small_case(shape, 4, 2, [3000, 2200], seed=31, max_disp=1.5, rigid=1.0)


def _oracle(shape, case, y_in):
    geo = O.Geometry(shape)
    d64 = [d.astype(np.float64) for d in case["disp"]]
    ys = O.stacked_forward(geo, case["x"], d64, case["smaps"], case["coords"])
    xa = O.stacked_adjoint(geo, y_in, d64, case["smaps"], case["coords"])
    return np.concatenate(ys), xa


@pytest.mark.parametrize("precision,tol", [(0, TOL_FP32), (2, TOL_FP32), (1, TOL_BF16)])
def test_variant_forward_adjoint_vs_oracle(precision, tol):
    import torch
    shape, case = _case()
    plan = make_plan(case, shape, precision=precision)
    rng = np.random.default_rng(5)
    M = plan.counts
    yl = [(rng.standard_normal((m, 4)) + 1j * rng.standard_normal((m, 4))) for m in M]
    y_ref, x_ref = _oracle(shape, case, yl)
    y = plan.forward(to_dev(case["x"])).cpu().numpy()
    x = plan.adjoint(to_dev(np.concatenate(yl).astype(np.complex64))).cpu().numpy()
    ef, ea = rel_l2(y, y_ref), rel_l2(x, x_ref)
    # adjointness of the GPU operator itself
    xd = to_dev(case["x"])
    yd = to_dev(np.concatenate(yl).astype(np.complex64))
    d = lambda a: a.flatten().to(torch.complex128)
    Ax, Ahy = plan.forward(xd), plan.adjoint(yd)
    adj = abs(complex(torch.vdot(d(yd), d(Ax)) - torch.vdot(d(Ahy), d(xd)))) / float(
        torch.linalg.norm(d(Ax)) * torch.linalg.norm(d(yd)))
    print(f"precision {precision}: A rel L2 {ef:.2e}, A^H rel L2 {ea:.2e}, adjointness {adj:.2e}")
    assert ef < tol and ea < tol
    assert adj < (TOL_ADJ if precision != 1 else TOL_BF16)
    plan.close()


def test_variant_argument_checks():
    from paper_2501_16713_gb300 import NrsenseError
    shape = (12, 16, 16)  # grid 24 x 32 x 32: 24 is not a power of two
    case = synth.small_case(shape, 2, 1, [500], seed=32)
    with pytest.raises(NrsenseError) as ei:
        make_plan(case, shape, precision=1)
    assert ei.value.code == -1
    with pytest.raises(NrsenseError):
        make_plan(case, shape, precision=2, width=6)
    with pytest.raises(NrsenseError):
        make_plan(case, shape, precision=7)


def test_dense_centre_accuracy_fp32_and_compensated():
    # 300k samples within |omega| < 0.25 rad: the central grid values receive
    # ~10^5 contributions each, with coherent values (1 + 10% noise) as near
    # the k-space centre.  Heavy tiles are split into chunks of at most 1024
    # points summed in slot order, so plain FP32 stays at the level of the
    # other FP32 steps (kernel weights, FFT); so does the compensated variant.
    shape = (16, 16, 16)
    rng = np.random.default_rng(33)
    m = 300_000
    u = rng.standard_normal((m, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    rad = 0.25 * rng.uniform(0, 1, m) ** (1 / 3)
    coords = (u * rad[:, None]).astype(np.float32)
    case = synth.small_case(shape, 2, 1, [10], seed=34)
    case["coords"] = [coords]
    yv = (1.0 + 0.1 * (rng.standard_normal((m, 2)) + 1j * rng.standard_normal((m, 2)))
          ).astype(np.complex64)
    geo = O.Geometry(shape)
    ref = O.kspace_adjoint(geo, yv.astype(np.complex128), coords)
    errs = {}
    for precision in (0, 2):
        plan = make_plan(case, shape, identity_warp=True, precision=precision)
        v = plan.kspace_adjoint(0, to_dev(yv)).cpu().numpy()
        errs[precision] = rel_l2(v, ref)
        plan.close()
    print(f"k-space adjoint, dense centre: FP32 {errs[0]:.2e}, compensated {errs[2]:.2e}")
    assert errs[0] < 1e-6 and errs[2] < 1e-6


def test_compensated_spread_recovers_swamped_contributions():
    # one sample of value 1e8 and 10^5 samples of value 1 at one k-space
    # position: every sample has the same kernel weights (their FP32 error is
    # a common relative factor ~1e-7), while an FP32 accumulator that holds
    # ~1e8 drops unit-size contributions (half an ulp of 1e8 is 4).  The exact
    # sum is (1e8 + 10^5) x the unit response; compensated summation keeps it.
    shape = (16, 16, 16)
    m = 100_001
    coords = np.tile(np.array([[0.3, -0.7, 1.1]], np.float32), (m, 1))
    case = synth.small_case(shape, 2, 1, [10], seed=35)
    case["coords"] = [coords]
    yv = np.ones((m, 2), np.complex64)
    yv[0, :] = 1e8
    geo = O.Geometry(shape)
    ref = O.kspace_adjoint(geo, yv.astype(np.complex128), coords)
    errs = {}
    for precision in (0, 2):
        plan = make_plan(case, shape, identity_warp=True, precision=precision)
        v = plan.kspace_adjoint(0, to_dev(yv)).cpu().numpy()
        errs[precision] = rel_l2(v, ref)
        plan.close()
    print(f"swamping: FP32 {errs[0]:.2e}, compensated {errs[2]:.2e}")
    assert errs[2] < 1e-6
    assert errs[2] < 0.1 * errs[0]


def test_bf16_storage_tensor_core_spread():
    """8 coils with BF16 coil grids: the register spread and the tensor-core
    spread (tile planes and 4^3 sub-blocks) accumulate in FP32 and round once
    to BF16 at the store, so each meets the BF16 bar against the oracle and
    they differ from one another only where FP32 summation order moves a
    value across a BF16 rounding boundary."""
    import ctypes
    from paper_2501_16713_gb300.nrsense import Tuning
    shape = (16, 32, 32)
    case = synth.small_case(shape, 8, 2, [3000, 2200], seed=32, max_disp=1.5, rigid=1.0)
    plan = make_plan(case, shape, precision=1)
    rng = np.random.default_rng(6)
    yl = [(rng.standard_normal((m, 8)) + 1j * rng.standard_normal((m, 8))) for m in plan.counts]
    geo = O.Geometry(shape)
    d64 = [d.astype(np.float64) for d in case["disp"]]
    x_ref = O.stacked_adjoint(geo, yl, d64, case["smaps"], case["coords"])
    yd = to_dev(np.concatenate(yl).astype(np.complex64))
    got = {}
    for name, (sv, wpc, cube) in {"register": (3, 1, 0), "planes": (4, 4, 0),
                                  "cube": (4, 4, 1)}.items():
        t = Tuning()
        t.spread_variant, t.interp_coils, t.interp_tma = sv, 8, 0
        t.spread_mma_wpc, t.spread_mma_cube = wpc, cube
        assert plan.lib.nrsense_plan_set_tuning(plan._h, ctypes.byref(t)) == 0
        got[name] = plan.adjoint(yd).cpu().numpy()
        e = rel_l2(got[name], x_ref)
        print(f"BF16 storage, {name} spread: A^H rel L2 {e:.2e}")
        assert e < TOL_BF16
    for name in ("planes", "cube"):
        d = rel_l2(got[name], got["register"])
        print(f"BF16 storage, {name} vs register spread: {d:.2e}")
        assert d < 3e-3
    assert plan.device_status() == 0
    plan.close()
