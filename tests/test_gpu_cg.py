"""GPU conjugate gradients on the Tikhonov normal equations vs the FP64 oracle.

The GPU solver keeps vectors in FP32 and every inner product, step size and
residual norm in FP64 on the device.  Its solution is compared with the FP64
oracle CG solution of the same system (same seeded data); the difference is
bounded by the FP32 operator error amplified by the system's conditioning, so
the tolerance is stated per test.
"""

import numpy as np
import pytest

import synth
from helpers import c64, make_plan, rel_l2, to_dev
from oracle import operators as O
from oracle import solvers as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()


def _problem(seed=70):
    shape = (16, 16, 16)
    case = synth.small_case(shape, 4, 2, [1500, 1200], seed=seed, max_disp=2.0, rigid=1.0)
    geo = O.Geometry(shape)
    d64 = [d.astype(np.float64) for d in case["disp"]]
    ys = O.stacked_forward(geo, case["x"], d64, case["smaps"], case["coords"])
    rng = np.random.default_rng(seed)
    ys = [y + 0.01 * np.abs(y).max() * (rng.standard_normal(y.shape) + 1j * rng.standard_normal(y.shape))
          for y in ys]
    return shape, case, geo, d64, ys


def _lambda_max(geo, d64, case, iters=15):
    rng = np.random.default_rng(1)
    v = rng.standard_normal(geo.shape) + 1j * rng.standard_normal(geo.shape)
    lam = 0.0
    for _ in range(iters):
        w = O.normal(geo, v, d64, case["smaps"], case["coords"])
        lam = np.linalg.norm(w) / np.linalg.norm(v)
        v = w / np.linalg.norm(w)
    return lam


def test_cg_matches_oracle_solution():
    shape, case, geo, d64, ys = _problem()
    lam = 1e-2 * _lambda_max(geo, d64, case)
    yin = c64(np.concatenate(ys))
    yl = [y.astype(np.complex64).astype(np.complex128) for y in ys]
    b = O.stacked_adjoint(geo, yl, d64, case["smaps"], case["coords"])
    xo, it_o, hist_o = S.cg(lambda v: O.normal(geo, v.reshape(shape), d64, case["smaps"],
                                               case["coords"], lam).ravel(),
                            b.ravel(), tol=1e-6, maxit=200)
    plan = make_plan(case, shape)
    x, it, hist, tres, code = plan.solve_cg(to_dev(yin), lam, tol=1e-6, maxit=200)
    xg = x.cpu().numpy()
    assert code == 0
    assert abs(it - it_o) <= max(3, it_o // 5)
    assert hist[0] == pytest.approx(1.0)
    assert hist[-1] <= 1e-6
    # recursive and true residual agree to FP32 operator accuracy
    assert tres < 1e-4
    assert rel_l2(xg, xo.reshape(shape)) < 1e-4
    plan.close()


def test_cg_graph_replay_is_bitwise_identical():
    import torch
    shape, case, geo, d64, ys = _problem(71)
    lam = 1e-2 * _lambda_max(geo, d64, case)
    plan = make_plan(case, shape)
    y = to_dev(c64(np.concatenate(ys)))
    x1, it1, h1, _, c1 = plan.solve_cg(y, lam, tol=1e-5, maxit=60, graph=False)
    assert c1 == 0
    x1 = x1.clone()
    buf = torch.empty_like(x1)
    x2, it2, h2, _, _ = plan.solve_cg(y, lam, tol=1e-5, maxit=60, graph=True, out=buf)
    x2 = x2.clone()
    x3, it3, h3, _, _ = plan.solve_cg(y, lam, tol=1e-5, maxit=60, graph=True, out=buf)  # replay
    assert it1 == it2 == it3
    assert h1 == h2 == h3
    assert torch.equal(x1, x2) and torch.equal(x2, x3)
    plan.close()


def test_cg_initial_guess_and_not_converged():
    shape, case, geo, d64, ys = _problem(72)
    lam = 1e-2 * _lambda_max(geo, d64, case)
    plan = make_plan(case, shape)
    y = to_dev(c64(np.concatenate(ys)))
    x, it, hist, tres, code = plan.solve_cg(y, lam, tol=1e-12, maxit=3, check=False)
    assert code == -6 and it == 3          # maxit reached above tol
    x_ref, it_ref, h_ref, _, code_ref = plan.solve_cg(y, lam, tol=1e-5, maxit=100)
    assert code_ref == 0
    # restart from the 3-iteration iterate: converges, and to the same solution
    x2, it2, h2, tres2, code2 = plan.solve_cg(y, lam, tol=1e-5, maxit=100, x0=x.clone())
    assert code2 == 0 and h2[0] < 1.0
    assert rel_l2(x2.cpu().numpy(), x_ref.cpu().numpy()) < 1e-4
    plan.close()
