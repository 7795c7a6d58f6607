"""Own pruned coil-grid transforms (fan-out and coil combination fused) and
pruned image-space G^3 transforms of T / T^H (deapodization, zero-padding and
cropping fused) vs the FP64 oracle and vs the cuFFT paths.

Shape 16 x 32 x 64 gives grids of 32, 64 and 128 points: every supported
transform length but 256 in one plan (256 runs in the full-size tests and the
benchmark).  Both paths must match the oracle within the FP32 operator bar
and each other within 2e-6; switching between them must reproduce each
path's values bit for bit (the cuFFT path needs the zero padding the pruned
path overwrites); the per-coil stage call after a pruned application must
equal a fresh plan's; an unsupported geometry refuses the pruned choice.
"""

import ctypes

import numpy as np
import pytest

import synth
from helpers import TOL_FP32, make_plan, rel_l2, to_dev
from oracle import operators as O

pytestmark = pytest.mark.gpu

SHAPE = (16, 32, 64)


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()


def _set(plan, pruned, image=0):
    from paper_2501_16713_gb300.nrsense import Tuning
    t = Tuning()
    t.spread_variant, t.interp_coils, t.interp_tma = 3, 8, 1
    t.spread_image_warp, t.fft_pruned = 0, int(pruned)
    t.image_fft_pruned = int(image)
    return plan.lib.nrsense_plan_set_tuning(plan._h, ctypes.byref(t))


@pytest.fixture(scope="module")
def case():
    c = synth.small_case(SHAPE, 3, 2, [5000, 4200], seed=81, max_disp=1.5, rigid=0.5)
    plan = make_plan(c, SHAPE)
    yield c, plan
    plan.close()


def test_both_paths_match_oracle(case):
    c, plan = case
    geo = O.Geometry(SHAPE)
    d64 = [d.astype(np.float64) for d in c["disp"]]
    x = c["x"].astype(np.complex128)
    ys_ref = O.stacked_forward(geo, x, d64, c["smaps"], c["coords"])
    y_ref = np.concatenate(ys_ref)
    xa_ref = O.stacked_adjoint(geo, ys_ref, d64, c["smaps"], c["coords"])
    out = {}
    for pruned in (0, 1):
        assert _set(plan, pruned) == 0
        y = plan.forward(to_dev(c["x"]))
        xa = plan.adjoint(to_dev(y_ref.astype(np.complex64)))
        e_f, e_a = rel_l2(y.cpu().numpy(), y_ref), rel_l2(xa.cpu().numpy(), xa_ref)
        print(f"pruned={pruned}: forward rel L2 {e_f:.2e}, adjoint rel L2 {e_a:.2e}")
        assert e_f < TOL_FP32 and e_a < TOL_FP32
        out[pruned] = (y.cpu().numpy(), xa.cpu().numpy())
    assert rel_l2(out[1][0], out[0][0]) < 2e-6
    assert rel_l2(out[1][1], out[0][1]) < 2e-6
    assert plan.device_status() == 0


def test_switching_paths_is_reproducible(case):
    import torch
    c, plan = case
    x = to_dev(c["x"])
    res = {}
    for pruned in (1, 0, 1, 0):
        assert _set(plan, pruned) == 0
        e = plan.normal(x, 0.5)
        if pruned in res:
            assert torch.equal(e, res[pruned]), pruned
        else:
            res[pruned] = e
    assert rel_l2(res[1].cpu().numpy(), res[0].cpu().numpy()) < 2e-6


def test_stage_call_after_pruned_application(case):
    import torch
    c, plan = case
    rng = np.random.default_rng(82)
    v = to_dev((rng.standard_normal((3,) + SHAPE) + 1j * rng.standard_normal((3,) + SHAPE))
               .astype(np.complex64))
    assert _set(plan, 1) == 0
    plan.normal(to_dev(c["x"]), 0.0)           # leaves the intermediates in the pad buffers
    y1 = plan.kspace_forward(0, v)
    fresh = make_plan(c, SHAPE)
    y2 = fresh.kspace_forward(0, v)
    assert torch.equal(y1, y2)
    fresh.close()


def test_autotune_times_both_paths(case):
    _, plan = case
    res = plan.autotune(reps=2)
    print(res["fft_ms"], res["fft_pruned"], res["image_fft_ms"], res["image_fft_pruned"])
    assert res["fft_ms"][0] > 0 and res["fft_ms"][1] > 0 and res["fft_pruned"] in (0, 1)
    assert res["image_fft_ms"][0] > 0 and res["image_fft_ms"][1] > 0
    assert res["image_fft_pruned"] in (0, 1)


def _warp_refs(c):
    geo = O.Geometry(SHAPE)
    d64 = [d.astype(np.float64) for d in c["disp"]]
    m_ref = np.stack([O.warp_forward(geo, c["x"].astype(np.complex128), d) for d in d64])
    rng = np.random.default_rng(84)
    w = rng.standard_normal((len(d64),) + SHAPE) + 1j * rng.standard_normal((len(d64),) + SHAPE)
    xa_ref = sum(O.warp_adjoint(geo, w[j], d64[j]) for j in range(len(d64)))
    return m_ref, w, xa_ref


def test_image_transforms_both_paths_match_oracle(case):
    """T and T^H (all phases) with the image-space G^3 transforms by cuFFT and
    by the pruned passes: both within the FP32 bar of the oracle, within 2e-6
    of each other."""
    c, plan = case
    m_ref, w, xa_ref = _warp_refs(c)
    out = {}
    for image in (0, 1):
        assert _set(plan, 1, image) == 0
        m = plan.warp_forward(to_dev(c["x"])).cpu().numpy()
        xa = plan.warp_adjoint(to_dev(w.astype(np.complex64))).cpu().numpy()
        e_f, e_a = rel_l2(m, m_ref), rel_l2(xa, xa_ref)
        print(f"image pruned={image}: T rel L2 {e_f:.2e}, T^H rel L2 {e_a:.2e}")
        assert e_f < TOL_FP32 and e_a < TOL_FP32
        out[image] = (m, xa)
    assert rel_l2(out[1][0], out[0][0]) < 2e-6
    assert rel_l2(out[1][1], out[0][1]) < 2e-6
    assert plan.device_status() == 0


def test_image_transform_switching_is_reproducible(case):
    """The pruned passes keep their intermediates in the zero-padded spectrum
    buffer of the cuFFT path; switching back must restore its zeros (else the
    cuFFT path's T would change)."""
    import torch
    c, plan = case
    x = to_dev(c["x"])
    res = {}
    for image in (1, 0, 1, 0):
        assert _set(plan, 1, image) == 0
        e = plan.normal(x, 0.5)
        if image in res:
            assert torch.equal(e, res[image]), image
        else:
            res[image] = e
    assert rel_l2(res[1].cpu().numpy(), res[0].cpu().numpy()) < 2e-6


def test_image_transforms_without_coils():
    """A warp-only plan (no coils, no k space) takes the pruned image-space
    transforms by default and matches the oracle; with the same launch
    choices it computes bitwise the warp of a full plan on the same geometry
    and displacements."""
    import torch
    from paper_2501_16713_gb300 import Plan
    c = synth.small_case(SHAPE, 3, 2, [2000, 1500], seed=85, max_disp=1.5, rigid=0.5)
    disp = to_dev(np.stack(c["disp"]))
    warp_only = Plan(SHAPE, disp=disp, n_phases=2)
    x = to_dev(c["x"])
    geo = O.Geometry(SHAPE)
    d64 = [d.astype(np.float64) for d in c["disp"]]
    m_ref = np.stack([O.warp_forward(geo, c["x"].astype(np.complex128), d) for d in d64])
    m0 = warp_only.warp_forward(x)
    assert rel_l2(m0.cpu().numpy(), m_ref) < TOL_FP32
    xa_ref = sum(O.warp_adjoint(geo, m_ref[j], d64[j]) for j in range(2))
    assert rel_l2(warp_only.warp_adjoint(to_dev(m_ref.astype(np.complex64))).cpu().numpy(),
                  xa_ref) < TOL_FP32
    full = make_plan(c, SHAPE)
    assert _set(full, 1, 1) == 0
    assert _set(warp_only, 0, 1) == 0   # no coil grids: the coil-grid choice must be 0
    assert _set(warp_only, 1, 1) == -1
    m1 = warp_only.warp_forward(x)
    assert torch.equal(m1, full.warp_forward(x))
    assert torch.equal(warp_only.warp_adjoint(m1), full.warp_adjoint(m1))
    warp_only.close()
    full.close()


def test_unsupported_geometry_refuses_pruned():
    shape = (16, 16, 24)  # a 48-point grid
    c = synth.small_case(shape, 2, 1, [1500], seed=83)
    plan = make_plan(c, shape)
    assert _set(plan, 1) == -1
    assert _set(plan, 0, 1) == -1
    res = plan.autotune(reps=1)
    assert res["fft_pruned"] == 0 and res["fft_ms"] == [-1.0, -1.0]
    assert res["image_fft_pruned"] == 0 and res["image_fft_ms"] == [-1.0, -1.0]
    plan.close()


def test_pruned_skips_tiles_outside_the_union():
    """Samples confined to |omega| < 0.35 pi: most tiles of the 32 x 64 x 128
    grids are outside the union over phases, so the axis-0 passes skip them.
    The cuFFT path runs first and leaves values in every tile of the
    interpolation input; the pruned path then stores only union tiles, the
    interpolation reads only taps inside them, and the adjoint's axis-0 pass
    takes the other tiles as the zeros the spread target holds there."""
    c = synth.small_case(SHAPE, 3, 2, [3000, 2600], seed=82, max_disp=1.0, rigid=0.5)
    c["coords"] = [(0.35 * w).astype(np.float32) for w in c["coords"]]
    plan = make_plan(c, SHAPE)
    info = plan.info()
    fu, fc = info["union_fraction"], info["union_columns"]
    print(f"union: {fu:.3f} of the tiles, {fc:.3f} of the tile columns")
    assert 0.0 < fu <= fc < 0.5
    geo = O.Geometry(SHAPE)
    d64 = [d.astype(np.float64) for d in c["disp"]]
    x = c["x"].astype(np.complex128)
    ys_ref = O.stacked_forward(geo, x, d64, c["smaps"], c["coords"])
    xa_ref = O.stacked_adjoint(geo, ys_ref, d64, c["smaps"], c["coords"])
    e_ref = O.normal(geo, x, d64, c["smaps"], c["coords"], 0.5)
    assert _set(plan, False) == 0
    plan.forward(to_dev(c["x"]))
    y0 = to_dev(np.concatenate(ys_ref).astype(np.complex64))
    plan.adjoint(y0)
    assert _set(plan, True) == 0
    y = plan.forward(to_dev(c["x"])).cpu().numpy()
    xa = plan.adjoint(y0).cpu().numpy()
    e = plan.normal(to_dev(c["x"]), 0.5).cpu().numpy()
    errs = (rel_l2(y, np.concatenate(ys_ref)), rel_l2(xa, xa_ref), rel_l2(e, e_ref))
    print("pruned with skipped tiles: forward %.2e, adjoint %.2e, normal %.2e" % errs)
    assert max(errs) < TOL_FP32
    assert plan.device_status() == 0
    plan.close()
