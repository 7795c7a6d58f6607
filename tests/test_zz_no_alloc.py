"""Allocation-free inner product, checked against the CG solver.

nrsense_dot_noalloc serves callers that may not allocate device memory (their
memory belongs to another allocator or a fixed pool, or an allocation could
block them) and so cannot create a plan: it keeps its block partial sums in a
fixed array inside the library.  Here it is called through the C ABI and
compared with the existing entry point that runs the same FP64 inner-product
kernel on plan-owned scratch: the true residual ||b - E x|| / ||b|| that
nrsense_solve_cg reports must equal sqrt(<r, r> / <b, b>) computed by two
calls in a row.  Lengths that span several 4096-element blocks and end in a
partial block exercise the shared array across blocks; a long call followed
by a short one would expose stale partial sums.  The inputs are exact in
FP64, so each result is compared with a complex128 reduction of the same
vectors to FP64 rounding (1e-12 of sum |x_i| |y_i|).  This file is collected
last so that a run stopping at the first failure has already run every
other test.
"""

import ctypes

import numpy as np
import pytest

import synth
from helpers import TOL_FP32, c64, make_plan, to_dev
from oracle import operators as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()


def _dot(lib, x, y, out):
    import torch
    return lib.nrsense_dot_noalloc(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                   ctypes.c_int64(x.numel()), ctypes.c_void_p(out.data_ptr()),
                                   ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def test_noalloc_dot_matches_cg_true_residual():
    import torch
    from paper_2501_16713_gb300 import nrsense
    shape = (16, 16, 16)
    case = synth.small_case(shape, 4, 2, [1500, 1200], seed=90)
    geo = O.Geometry(shape)
    d64 = [d.astype(np.float64) for d in case["disp"]]
    ys = O.stacked_forward(geo, case["x"], d64, case["smaps"], case["coords"])
    plan = make_plan(case, shape)
    y = to_dev(c64(np.concatenate(ys)))
    lam = 0.1
    x, it, hist, tres, code = plan.solve_cg(y, lam, tol=1e-12, maxit=4, check=False)
    assert it == 4 and tres > 0
    b = plan.adjoint(y)
    r = b - plan.normal(x, lam)
    lib = nrsense.load()
    out_r = torch.empty(2, dtype=torch.float64, device="cuda")
    out_b = torch.empty(2, dtype=torch.float64, device="cuda")
    assert _dot(lib, r, r, out_r) == 0
    assert _dot(lib, b, b, out_b) == 0      # second call in a row reuses the scratch
    torch.cuda.synchronize()
    rr, bb = out_r.cpu().numpy(), out_b.cpu().numpy()
    assert abs(np.sqrt(rr[0] / bb[0]) - tres) <= TOL_FP32 * tres
    # each call against a plain FP64 reduction of the same vectors
    for v, o in ((r, rr), (b, bb)):
        _check_fp64(o, v.flatten(), v.flatten())
    # two more calls in a row, on a complex-valued product, leave no stale state
    for a, c in ((x, b), (b, x)):
        assert _dot(lib, a, c, out_r) == 0
        _check_fp64(out_r.cpu().numpy(), a.flatten(), c.flatten())
    plan.close()


def test_noalloc_dot_limits():
    import torch
    from paper_2501_16713_gb300 import nrsense
    lib = nrsense.load()
    v = torch.ones(8, dtype=torch.complex64, device="cuda")
    out = torch.full((2,), 7.0, dtype=torch.float64, device="cuda")
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    # beyond the fixed scratch: rejected before anything is launched
    too_many = ctypes.c_int64(nrsense.DOT_NOALLOC_MAX_N + 1)
    assert lib.nrsense_dot_noalloc(ctypes.c_void_p(v.data_ptr()), ctypes.c_void_p(v.data_ptr()),
                                   too_many, ctypes.c_void_p(out.data_ptr()), s) == -1
    # empty input: zero
    assert lib.nrsense_dot_noalloc(ctypes.c_void_p(v.data_ptr()), ctypes.c_void_p(v.data_ptr()),
                                   ctypes.c_int64(0), ctypes.c_void_p(out.data_ptr()), s) == 0
    torch.cuda.synchronize()
    assert out.cpu().tolist() == [0.0, 0.0]


def _rand(n, seed):
    import torch
    gen = torch.Generator(device="cuda").manual_seed(seed)
    return torch.randn(n, dtype=torch.complex64, device="cuda", generator=gen)


def _check_fp64(got, a, c):
    import torch
    a64, c64_ = a.to(torch.complex128), c.to(torch.complex128)
    ref = complex(torch.vdot(a64, c64_).item())
    scale = float((a64.abs() * c64_.abs()).sum().item())
    assert abs(complex(got[0], got[1]) - ref) <= 1e-12 * scale, (got, ref, scale)


def test_noalloc_dot_many_blocks_and_partial_tail():
    import torch
    from paper_2501_16713_gb300 import nrsense
    lib = nrsense.load()
    out = torch.empty(2, dtype=torch.float64, device="cuda")
    # long before short: the short call's final sum must not see the long
    # call's partial sums left in the array
    for n, seed in ((2 ** 20 + 5, 1), (3 * 4096 + 17, 2), (4096 + 1, 3), (4095, 4), (1, 5),
                    (2 ** 20 + 5, 6), (4 * 4096, 7)):
        a, c = _rand(n, seed), _rand(n, seed + 100)
        assert _dot(lib, a, c, out) == 0
        _check_fp64(out.cpu().numpy(), a, c)


def test_noalloc_dot_python_wrapper_matches_abi():
    import torch
    from paper_2501_16713_gb300 import nrsense
    lib = nrsense.load()
    a, c = _rand(3 * 4096 + 17, 11), _rand(3 * 4096 + 17, 12)
    raw = torch.empty(2, dtype=torch.float64, device="cuda")
    assert _dot(lib, a, c, raw) == 0
    got = nrsense.dot_noalloc(a, c)
    torch.cuda.synchronize()
    assert torch.equal(got, raw)
    with pytest.raises(ValueError):
        nrsense.dot_noalloc(a, c[:-1])
