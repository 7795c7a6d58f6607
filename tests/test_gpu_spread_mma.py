"""Tensor-core k-space spread (mma.sync TF32, operands split in three
products), a warp per tile plane or per 4^3 sub-block, vs the FP64 oracle and
vs the FMA register spread.

An 8-coil case whose cone-like trajectory concentrates 30000 samples of a
phase near the k-space centre, so that heavy tiles are split across work
items (the partial-tile scratch path) and light tiles are not.  The adjoint
and the normal operator must meet the FP32 operator bar against the oracle
and agree with the register kernel to 2e-6 (the split keeps each product to
about 2^-22 relative; the summation order differs).  Ragged tiles (grid sizes
4 mod 8: the high sub-blocks of an edge tile are empty), an odd coil count
(partial 8-coil chunk, per-value loads) and sample values at an 8-byte but
not 16-byte aligned address take the sub-block kernel's other paths.
"""

import ctypes

import numpy as np
import pytest

import synth
from helpers import TOL_FP32, make_plan, rel_l2, to_dev
from oracle import operators as O

pytestmark = pytest.mark.gpu

SHAPE = (16, 24, 32)


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()


def _set(plan, spread, pruned=0, wpc=1, cube=0):
    from paper_2501_16713_gb300.nrsense import Tuning
    t = Tuning()
    t.spread_variant, t.interp_coils, t.interp_tma = spread, 8, 0
    t.spread_image_warp, t.fft_pruned, t.spread_mma_wpc = 0, pruned, wpc
    t.spread_mma_cube = cube
    return plan.lib.nrsense_plan_set_tuning(plan._h, ctypes.byref(t))


@pytest.fixture(scope="module")
def case():
    c = synth.small_case(SHAPE, 8, 2, [30000, 9000], seed=91, max_disp=1.5, rigid=0.5)
    plan = make_plan(c, SHAPE)
    yield c, plan
    plan.close()


def test_split_tiles_present(case):
    _, plan = case
    info = plan.info()
    print(f"spread items {info['spread_items']}, split tiles {info['split_tiles']}")
    assert info["split_tiles"] > 0


def test_mma_spread_matches_oracle_and_register_kernel(case):
    c, plan = case
    geo = O.Geometry(SHAPE)
    d64 = [d.astype(np.float64) for d in c["disp"]]
    rng = np.random.default_rng(92)
    M = [x.shape[0] for x in c["coords"]]
    y = (rng.standard_normal((sum(M), 8)) + 1j * rng.standard_normal((sum(M), 8))).astype(np.complex64)
    ys = np.split(y.astype(np.complex128), np.cumsum(M)[:-1])
    xa_ref = O.stacked_adjoint(geo, ys, d64, c["smaps"], c["coords"])
    out = {}
    for sv in (3, 4):
        assert _set(plan, sv) == 0
        xa = plan.adjoint(to_dev(y)).cpu().numpy()
        e = rel_l2(xa, xa_ref)
        print(f"spread variant {sv}: adjoint rel L2 {e:.2e}")
        assert e < TOL_FP32
        out[sv] = xa
    d = rel_l2(out[4], out[3])
    print(f"tensor-core vs register spread: rel L2 {d:.2e}")
    assert d < 2e-6
    # 2 or 4 tile planes per CTA: the same per-plane work, bitwise the same
    for wpc in (2, 4):
        assert _set(plan, 4, wpc=wpc) == 0
        assert np.array_equal(plan.adjoint(to_dev(y)).cpu().numpy(), out[4]), wpc
    # a warp per 4^3 sub-block: its own summation order, the same bars;
    # 1, 2 or 4 sub-blocks per CTA bitwise the same
    assert _set(plan, 4, wpc=1, cube=1) == 0
    xc = plan.adjoint(to_dev(y)).cpu().numpy()
    e, d = rel_l2(xc, xa_ref), rel_l2(xc, out[3])
    print(f"sub-block tensor-core spread: adjoint rel L2 {e:.2e}, vs register {d:.2e}")
    assert e < TOL_FP32 and d < 2e-6
    for wpc in (2, 4):
        assert _set(plan, 4, wpc=wpc, cube=1) == 0
        assert np.array_equal(plan.adjoint(to_dev(y)).cpu().numpy(), xc), wpc
    assert _set(plan, 4, cube=2) != 0  # unknown geometry
    assert plan.device_status() == 0


def test_mma_spread_normal_operator(case):
    c, plan = case
    geo = O.Geometry(SHAPE)
    d64 = [d.astype(np.float64) for d in c["disp"]]
    x = c["x"].astype(np.complex128)
    e_ref = O.normal(geo, x, d64, c["smaps"], c["coords"], 0.25)
    for pruned in (0, 1):
        for cube in (0, 1):
            if _set(plan, 4, pruned, wpc=4, cube=cube) != 0:
                continue  # pruned transforms need power-of-two grids of 32..256
            e = plan.normal(to_dev(c["x"]), 0.25).cpu().numpy()
            err = rel_l2(e, e_ref)
            print(f"normal (tensor-core spread, pruned={pruned}, cube={cube}) rel L2 {err:.2e}")
            assert err < TOL_FP32


def test_autotune_reports_mma(case):
    _, plan = case
    res = plan.autotune(reps=2)
    print(res["spread_ms"], res["spread_mma_geo_ms"], res["spread_mma_wpc"],
          res["spread_mma_cube"], res["spread_variant"])
    assert res["spread_mma_ms"] > 0 and res["spread_variant"] in (1, 2, 3, 4)
    assert res["spread_mma_wpc"] in (1, 2, 4) and res["spread_mma_cube"] in (0, 1)
    assert min(res["spread_mma_geo_ms"]) > 0
    assert res["spread_mma_ms"] == min(res["spread_mma_geo_ms"])


@pytest.mark.parametrize("coils,aligned", [(5, True), (8, False)])
def test_cube_spread_ragged_tiles(coils, aligned):
    """Grid (36, 40, 28): edge tiles 4 wide along axes 0 and 2.  G_0^H per
    coil through every spread geometry vs the oracle's gridding adjoint."""
    import torch
    shape = (18, 20, 14)
    c = synth.small_case(shape, coils, 1, [7000], seed=93, max_disp=1.0, rigid=0.5)
    plan = make_plan(c, shape)
    geo = O.Geometry(shape)
    rng = np.random.default_rng(94)
    M = c["coords"][0].shape[0]
    y = (rng.standard_normal((M, coils)) + 1j * rng.standard_normal((M, coils))).astype(np.complex64)
    ref = np.stack([O.kspace_adjoint(geo, y[:, k].astype(np.complex128), c["coords"][0])
                    for k in range(coils)])
    if aligned:
        yd = to_dev(y)
    else:  # the values 8 bytes past a 16-byte boundary
        buf = torch.zeros(M * coils + 1, dtype=torch.complex64, device="cuda")
        yd = buf[1:].view(M, coils)
        yd.copy_(to_dev(y))
        assert yd.data_ptr() % 16 == 8
    got = {}
    for name, (sv, wpc, cube) in {"register": (3, 1, 0), "planes": (4, 4, 0),
                                  "cube1": (4, 1, 1), "cube4": (4, 4, 1)}.items():
        assert _set(plan, sv, wpc=wpc, cube=cube) == 0
        got[name] = plan.kspace_adjoint(0, yd).cpu().numpy()
        e = rel_l2(got[name], ref)
        print(f"{coils} coils, aligned={aligned}, {name}: rel L2 {e:.2e}")
        assert e < TOL_FP32
    assert rel_l2(got["cube4"], got["register"]) < 2e-6
    assert np.array_equal(got["cube1"], got["cube4"])
    assert plan.device_status() == 0
    plan.close()
