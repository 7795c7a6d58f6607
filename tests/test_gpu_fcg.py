"""Flexible CG with the learned preconditioner against plain CG (GPU).

A 32^3, 4-coil, 2-phase problem with cone-like trajectories (sample density
falling as 1/|k|^2) and Tikhonov lambda = 1e-3 lambda_max (lambda_max from a
power iteration on the GPU normal operator).  Checks: flexible CG without a
network reproduces plain CG; a network with zero weights (z = r / s) does
too; recorded CG pairs satisfy E e_k = r_k; a network trained on recorded
pairs reaches the same 1e-4 relative residual in fewer iterations; graph
replay of flexible CG is bitwise identical to eager execution.
"""

import numpy as np
import pytest

import synth
from helpers import make_plan, to_dev

pytestmark = pytest.mark.gpu

SHAPE = (32, 32, 32)
TOL = 1e-4


@pytest.fixture(scope="module")
def prob():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    case = synth.small_case(SHAPE, 4, 2, [14000, 11000], seed=90, max_disp=2.0, rigid=1.0)
    plan = make_plan(case, SHAPE)
    # lambda = 1e-3 lambda_max (power iteration on the GPU normal operator)
    gen = torch.Generator(device="cuda").manual_seed(0)
    v = torch.randn(SHAPE, dtype=torch.complex64, device="cuda", generator=gen)
    lam_max = 0.0
    for _ in range(20):
        w = plan.normal(v, 0.0)
        lam_max = float(torch.linalg.norm(w) / torch.linalg.norm(v))
        v = w / torch.linalg.norm(w)
    lam = 1e-3 * lam_max
    x = to_dev(case["x"])
    y0 = plan.forward(x)
    noise = torch.randn(y0.shape, dtype=torch.complex64, device="cuda", generator=gen)
    y = y0 + 0.03 * float(y0.abs().max()) * noise
    yield plan, lam, y, gen
    plan.close()


def _rhs(plan, gen, k):
    """k random right-hand sides: y = A x_rand + noise, x_rand white noise
    smoothed 0..3 times."""
    import torch
    ys = []
    for i in range(k):
        xr = torch.randn(SHAPE, dtype=torch.complex64, device="cuda", generator=gen)
        for _ in range(i % 4):
            for ax in range(3):
                xr = 0.5 * xr + 0.25 * (torch.roll(xr, 1, ax) + torch.roll(xr, -1, ax))
        y = plan.forward(xr)
        y = y + 0.03 * float(y.abs().max()) * torch.randn(
            y.shape, dtype=torch.complex64, device="cuda", generator=gen)
        ys.append(y)
    return ys


def test_fcg_without_network_matches_cg(prob):
    plan, lam, y, _ = prob
    x_cg, it_cg, _, tr_cg, code_cg = plan.solve_cg(y, lam, tol=TOL, maxit=400)
    x_f, it_f, _, tr_f, code_f, fb = plan.solve_fcg(y, lam, None, tol=TOL, maxit=400)
    print(f"CG {it_cg} it (true res {tr_cg:.2e}), FCG(no net) {it_f} it (true res {tr_f:.2e})")
    assert code_cg == 0 and code_f == 0 and fb == 0
    assert abs(it_cg - it_f) <= max(2, 0.1 * it_cg)
    assert tr_f < 2 * TOL
    d = float((x_cg - x_f).norm() / x_cg.norm())
    assert d < 1e-2


def test_fcg_with_zero_network_is_plain_cg(prob):
    from paper_2501_16713_gb300 import Cnn
    plan, lam, y, _ = prob
    net = Cnn(SHAPE)  # all parameters zero: z = r / s
    _, it_cg, _, _, _ = plan.solve_cg(y, lam, tol=TOL, maxit=400)
    _, it_f, _, tr_f, code, fb = plan.solve_fcg(y, lam, net, tol=TOL, maxit=400)
    # z = fl(r / s) perturbs the directions at FP32 rounding level; CG at
    # condition number ~1e3 in FP32 shifts its count by a few iterations
    print(f"CG {it_cg} it, FCG(zero net) {it_f} it")
    assert code == 0 and fb == 0
    assert abs(it_cg - it_f) <= max(2, 0.1 * it_cg) and tr_f < 2 * TOL
    net.close()


def test_recorded_pairs_satisfy_normal_equations(prob):
    plan, lam, y, _ = prob
    x, it, hist, tres, code, r, e = plan.solve_cg_record(y, lam, 10, tol=1e-5, maxit=400)
    assert code == 0 and r.shape[0] == 10 and e.shape[0] == 10
    bnorm = None
    for k in range(10):
        Ee = plan.normal(e[k].contiguous(), lam)
        err = float((Ee - r[k]).norm())
        if bnorm is None:
            bnorm = float(r[0].norm())  # x0 = 0: r_0 = b
        # E (x* - x_k) = r_k - r*, |r*| <= 1e-5 |b|; FP32 recursion drift on top
        assert err < 1e-4 * bnorm, (k, err / bnorm)


def test_trained_network_reduces_iterations(prob):
    # symmetric form, cosine loss on pairs from plain-CG runs
    from paper_2501_16713_gb300 import Cnn, precond
    plan, lam, y, gen = prob
    r, e, iters = precond.generate_pairs(plan, _rhs(plan, gen, 12), lam, tol=1e-5, maxit=400)
    net = Cnn(SHAPE, seed=1)
    # the same network before training: what the training gains
    _, it_u, _, _, code_u, _ = plan.solve_fcg(y, lam, net, tol=TOL, maxit=400, check=False)
    losses = precond.train(net, r, e, steps=1000, lr=1e-3, lr_final=3e-5, batch=4, seed=0,
                           log_every=100)
    _, it_cg, _, tr_cg, _ = plan.solve_cg(y, lam, tol=TOL, maxit=400)
    x_f, it_f, _, tr_f, code, fb = plan.solve_fcg(y, lam, net, tol=TOL, maxit=400)
    print(f"pairs {r.shape[0]} from runs {iters}; loss {[round(l, 4) for l in losses if l == l]}")
    print(f"plain CG {it_cg} it, true res {tr_cg:.2e}; FCG+net {it_f} it, true res {tr_f:.2e}, "
          f"fallbacks {fb}; untrained network {it_u} it")
    assert code == 0
    assert tr_f < 2 * TOL
    assert it_f < it_cg
    assert it_f < it_u
    net.close()


def test_fcg_graph_replay_matches_eager(prob):
    import torch
    from paper_2501_16713_gb300 import Cnn
    plan, lam, y, _ = prob
    net = Cnn(SHAPE, seed=3)
    out = torch.empty(SHAPE, dtype=torch.complex64, device="cuda")
    x_e, it_e, h_e, _, _, _ = plan.solve_fcg(y, lam, net, tol=TOL, maxit=60, out=out.clone())
    x_g, it_g, h_g, _, _, _ = plan.solve_fcg(y, lam, net, tol=TOL, maxit=60, graph=True, out=out)
    x_g2, it_g2, _, _, _, _ = plan.solve_fcg(y, lam, net, tol=TOL, maxit=60, graph=True, out=out)
    assert it_e == it_g == it_g2
    assert np.array_equal(h_e, h_g)
    assert torch.equal(x_e, x_g) and torch.equal(x_g, x_g2)
    net.close()
