"""Deflated flexible CG with a recycled subspace (nrsense_set_deflation,
nrsense_deflation_from_solve, NRSENSE_CG_DEFLATE) against the FP64 oracle
(oracle/deflation.py) on a small nonrigid SENSE problem.

* With the same explicit basis W and the circulant preconditioner, the
  library's residual history follows the oracle's A-DEF2 iteration and the
  solution matches the oracle's.
* The Ritz values the library extracts from its recorded circulant-CG run
  match the oracle's from the same run (same data, lambda and step count), and
  the space they span gives a solve that converges to the same solution.
* A graph-captured deflated solve is bitwise the eager one; argument and
  state errors are reported.
"""

import ctypes

import numpy as np
import pytest

import synth
from helpers import make_plan, rel_l2, to_dev
from oracle import deflation as D
from oracle import operators as O
from oracle import precond as PC

pytestmark = pytest.mark.gpu

SHAPE = (16, 16, 24)
COILS = 4


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()


@pytest.fixture(scope="module")
def prob():
    import torch
    case = synth.small_case(SHAPE, COILS, 2, [2600, 2100], seed=191, max_disp=1.5, rigid=0.5)
    plan = make_plan(case, SHAPE)
    geo = O.Geometry(SHAPE)
    d64 = [d.astype(np.float64) for d in case["disp"]]

    def E0(v):
        return O.normal(geo, v, d64, case["smaps"], case["coords"], 0.0)

    rng = np.random.default_rng(192)
    v = rng.standard_normal(SHAPE) + 0j
    for _ in range(25):
        wv = E0(v)
        lmax = np.linalg.norm(wv) / np.linalg.norm(v)
        v = wv / np.linalg.norm(wv)
    lam = 1e-2 * lmax
    plan.set_circulant(10.0 * lam)
    y = np.concatenate(O.stacked_forward(geo, case["x"].astype(np.complex128), d64,
                                         case["smaps"], case["coords"]))
    y_train = rng.standard_normal(y.shape) + 1j * rng.standard_normal(y.shape)
    counts = [c.shape[0] for c in case["coords"]]

    def adjoint(yy):
        parts = np.split(yy, np.cumsum(counts)[:-1])
        return O.stacked_adjoint(geo, parts, d64, case["smaps"], case["coords"])

    d = PC.circulant_diag(E0, SHAPE, 10.0 * lam)
    ops = dict(E=lambda u: E0(u) + lam * u, M=lambda r: PC.apply_circulant(d, r))
    yield dict(plan=plan, lam=lam, y=y, y_train=y_train, adjoint=adjoint, **ops)
    plan.set_deflation(None)
    plan.close()
    torch.cuda.synchronize()


def test_explicit_basis_follows_the_oracle(prob):
    plan, lam = prob["plan"], prob["lam"]
    rng = np.random.default_rng(193)
    k = 4
    W = (rng.standard_normal((k,) + SHAPE) + 1j * rng.standard_normal((k,) + SHAPE)).astype(
        np.complex64)
    assert plan.set_deflation(to_dev(W)) == k
    x, it, hist, tres, code, fb = plan.solve_fcg(to_dev(prob["y"].astype(np.complex64)), lam,
                                                 None, tol=1e-6, maxit=300, circulant=True,
                                                 deflate=True)
    b = prob["adjoint"](prob["y"])
    x_o, it_o, hist_o, wr = D.deflated_pcg(prob["E"], prob["M"], b, list(W.astype(np.complex128)),
                                           tol=1e-6, maxit=300)
    print(f"deflated: library {it} iterations, oracle {it_o}; W^H r <= {wr:.1e}")
    assert code == 0 and fb == 0 and tres < 2e-6
    assert abs(it - it_o) <= 1
    h, ho = np.asarray(hist[:8]), np.asarray(hist_o[:8])
    assert np.all(np.abs(h - ho) <= 1e-3 * ho)
    assert rel_l2(x.cpu().numpy(), x_o) < 1e-4


def test_ritz_space_from_a_solve_matches_the_oracle(prob):
    plan, lam = prob["plan"], prob["lam"]
    steps, k = 12, 4
    theta, kept = plan.deflation_from_solve(to_dev(prob["y_train"].astype(np.complex64)), lam,
                                            steps=steps, k=k, circulant=True)
    assert kept == k
    b_train = prob["adjoint"](prob["y_train"].astype(np.complex64).astype(np.complex128))
    _, _, _, al, rho, Z = D.pcg_record(prob["E"], prob["M"], b_train, tol=0.0, maxit=steps,
                                       record=steps)
    theta_o, _ = D.ritz_space(D.lanczos_tridiagonal(al, rho, steps), Z, k)
    print("Ritz values: library", theta, "oracle", theta_o)
    assert np.all(np.abs(theta - theta_o) <= 1e-3 * theta_o)
    # the recycled space: same solution, no more iterations than without it
    y = to_dev(prob["y"].astype(np.complex64))
    x_c, it_c, _, _, _, _ = plan.solve_fcg(y, lam, None, tol=1e-6, maxit=300, circulant=True)
    x_d, it_d, _, tres, code, _ = plan.solve_fcg(y, lam, None, tol=1e-6, maxit=300,
                                                 circulant=True, deflate=True)
    print(f"circulant {it_c} iterations, with the recycled space {it_d}")
    assert code == 0 and tres < 2e-6 and it_d <= it_c
    assert rel_l2(x_d.cpu().numpy(), x_c.cpu().numpy()) < 1e-4


def test_repeated_and_dependent_vectors_are_dropped(prob):
    """A basis holding a vector twice (and a scaled copy) spans what the
    distinct vectors span: three vectors are kept, and the deflated solve
    agrees with the one on the distinct vectors alone up to FP32 rounding."""
    plan, lam = prob["plan"], prob["lam"]
    rng = np.random.default_rng(194)
    V = (rng.standard_normal((3,) + SHAPE) + 1j * rng.standard_normal((3,) + SHAPE)).astype(
        np.complex64)
    Wrep = np.stack([V[0], V[1], V[0], (2.0 - 0.5j) * V[1], V[2]]).astype(np.complex64)
    y = to_dev(prob["y"].astype(np.complex64))
    assert plan.set_deflation(to_dev(Wrep)) == 3
    x_r, it_r, _, _, code_r, _ = plan.solve_fcg(y, lam, None, tol=1e-6, maxit=300,
                                                circulant=True, deflate=True)
    assert plan.set_deflation(to_dev(V)) == 3
    x_v, it_v, _, _, code_v, _ = plan.solve_fcg(y, lam, None, tol=1e-6, maxit=300,
                                                circulant=True, deflate=True)
    assert code_r == 0 and code_v == 0 and abs(it_r - it_v) <= 1
    assert rel_l2(x_r.cpu().numpy(), x_v.cpu().numpy()) < 1e-5


def test_graph_replay_matches_eager(prob):
    import torch
    plan, lam = prob["plan"], prob["lam"]
    y = to_dev(prob["y"].astype(np.complex64))
    out = torch.empty(SHAPE, dtype=torch.complex64, device="cuda")
    x_e, it_e, h_e, _, _, _ = plan.solve_fcg(y, lam, None, tol=1e-5, maxit=100, circulant=True,
                                             deflate=True, out=out.clone())
    x_g, it_g, h_g, _, _, _ = plan.solve_fcg(y, lam, None, tol=1e-5, maxit=100, circulant=True,
                                             deflate=True, graph=True, out=out)
    assert it_e == it_g and h_e == h_g
    assert torch.equal(x_e, x_g)


def test_graph_recaptured_after_changes(prob):
    """A captured solve graph bakes in buffer addresses and launch choices: a
    rebuilt deflation space of another size (buffers freed and reallocated,
    possibly at the same addresses), a longer maxit (history buffer
    reallocated) and autotuning (launch choices, re-tiled k-space buffers)
    must each re-capture it, so the replay equals the eager solve."""
    import torch
    plan, lam = prob["plan"], prob["lam"]
    y = to_dev(prob["y"].astype(np.complex64))
    rng = np.random.default_rng(195)
    out = torch.empty(SHAPE, dtype=torch.complex64, device="cuda")

    def both(maxit):
        x_e, it_e, _, _, _, _ = plan.solve_fcg(y, lam, None, tol=1e-6, maxit=maxit,
                                               circulant=True, deflate=True, out=out.clone())
        x_g, it_g, _, _, _, _ = plan.solve_fcg(y, lam, None, tol=1e-6, maxit=maxit,
                                               circulant=True, deflate=True, graph=True, out=out)
        assert it_e == it_g
        assert torch.equal(x_e, x_g)

    for k, maxit in ((6, 8), (2, 8), (5, 40)):
        W = (rng.standard_normal((k,) + SHAPE) + 1j * rng.standard_normal((k,) + SHAPE))
        assert plan.set_deflation(to_dev(W.astype(np.complex64))) == k
        both(maxit)
    plan.autotune(reps=1)
    both(40)


def test_errors(prob):
    import torch
    from paper_2501_16713_gb300.nrsense import CG_DEFLATE, _stream
    plan, lam = prob["plan"], prob["lam"]
    lib, h, st = plan.lib, plan._h, _stream(None)
    kept = ctypes.c_int32()
    assert lib.nrsense_set_deflation(h, None, 3, ctypes.byref(kept), st) == -1   # no basis
    assert lib.nrsense_set_deflation(h, None, 65, None, st) == -1               # k above 64
    z = torch.zeros((2,) + SHAPE, dtype=torch.complex64, device="cuda")
    assert lib.nrsense_set_deflation(h, ctypes.c_void_p(z.data_ptr()), 2, None, st) == -5
    y = to_dev(prob["y"].astype(np.complex64))
    yp = ctypes.c_void_p(y.data_ptr())
    ritz = (ctypes.c_double * 4)()
    assert lib.nrsense_deflation_from_solve(h, yp, lam, 0, 4, 0, ritz, None, st) == -1
    assert lib.nrsense_deflation_from_solve(h, yp, lam, 3, 4, 0, ritz, None, st) == -1  # k > steps
    assert lib.nrsense_deflation_from_solve(h, yp, lam, 8, 4, CG_DEFLATE, ritz, None, st) == -1
    x = torch.zeros(SHAPE, dtype=torch.complex64, device="cuda")
    it = ctypes.c_int32()
    assert lib.nrsense_solve_cg(h, yp, lam, 1e-4, 10, CG_DEFLATE, ctypes.c_void_p(x.data_ptr()),
                                ctypes.byref(it), None, None, st) == -1
    plan.set_deflation(None)
    _, _, _, _, code, _ = plan.solve_fcg(y, lam, None, tol=1e-4, maxit=10, circulant=True,
                                         deflate=True, check=False)
    assert code == -9                                               # no space: ERR_STATE
