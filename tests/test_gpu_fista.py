"""Wavelet-FISTA on the GPU against the FP64 oracle.

The Haar transform, its inverse and the proximal map are compared value by
value with the oracle on shapes that span several shared-memory boxes per
axis with a partial box at the end (and every level count 0..4).  The FISTA
iterates, the per-iteration change history and the power-iteration estimate
are compared with the oracle run on the oracle's own FP64 normal operator,
with the step bound L taken from the oracle's power iteration.  Graph replay
must reproduce eager execution bit for bit.  The warp-only problem of the
paper's Appendix 1 (recover p from q = T p, 400 iterations, lambda = 1e-6)
is solved on a 3D piecewise-constant phantom and must beat the naive
inversion that warps q by -d, as the appendix reports.

Tolerances: the GPU path is FP32 (the transform adds at most 3 J + 1
roundings per value); the transform comparisons use 2e-6 of the largest
value.  FISTA iterates carry the FP32 normal operator's error (about 1e-6
relative) through a non-expansive proximal step and a momentum factor below
one, so after 12 iterations 2e-5 relative L2 holds with a wide margin.
"""

import numpy as np
import pytest

import synth
from helpers import make_plan, rel_l2, to_dev
from oracle import fista as F
from oracle import operators as O

pytestmark = pytest.mark.gpu

TOL_WAVELET = 2e-6
TOL_FISTA = 2e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()


def _field(seed, shape):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).astype(np.complex64)


def _maxrel(a, b):
    return float(np.abs(np.asarray(a) - b).max() / max(np.abs(b).max(), 1e-300))


WAVELET_CASES = [((24, 40, 56), 3), ((48, 16, 80), 4), ((6, 10, 34), 1), ((12, 20, 36), 2),
                 ((5, 7, 33), 0), ((16, 16, 32), 4), ((8, 8, 8), 3)]


@pytest.mark.parametrize("shape,levels", WAVELET_CASES)
def test_wavelet_transform_matches_oracle(shape, levels):
    from paper_2501_16713_gb300 import wavelet_forward, wavelet_inverse, wavelet_shrink
    x = _field(1, shape)
    c_ref = F.haar_forward(x.astype(np.complex128), levels)
    c = wavelet_forward(to_dev(x), levels).cpu().numpy()
    assert _maxrel(c, c_ref) < TOL_WAVELET
    cc = _field(2, shape)
    x_ref = F.haar_inverse(cc.astype(np.complex128), levels)
    xi = wavelet_inverse(to_dev(cc), levels).cpu().numpy()
    assert _maxrel(xi, x_ref) < TOL_WAVELET
    # threshold at the median modulus: about half the coefficients vanish
    tau = float(np.median(np.abs(c_ref)))
    u_ref = F.prox_wavelet_l1(x.astype(np.complex128), tau, levels)
    u = wavelet_shrink(to_dev(x), tau, levels).cpu().numpy()
    assert _maxrel(u, u_ref) < TOL_WAVELET
    # in place
    xd = to_dev(x)
    wavelet_shrink(xd, tau, levels, out=xd)
    assert np.array_equal(xd.cpu().numpy(), u)


def test_wavelet_invalid_arguments():
    import torch
    from paper_2501_16713_gb300 import NrsenseError, wavelet_forward, wavelet_shrink
    x = torch.zeros((8, 8, 12), dtype=torch.complex64, device="cuda")
    for lev in (-1, 3, 5):  # 12 is not divisible by 8; 5 > 4 levels
        with pytest.raises(NrsenseError) as ei:
            wavelet_forward(x, lev)
        assert ei.value.code == -1
    with pytest.raises(NrsenseError):
        wavelet_forward(x, 1, out=x)  # aliasing
    with pytest.raises(NrsenseError):
        wavelet_shrink(x, -1.0, 1)


@pytest.fixture(scope="module")
def sense_prob():
    shape = (16, 16, 24)
    case = synth.small_case(shape, 4, 2, [3000, 2500], seed=31, max_disp=1.5, rigid=0.5)
    plan = make_plan(case, shape)
    geo = O.Geometry(shape)
    d64 = [d.astype(np.float64) for d in case["disp"]]
    E0 = lambda v: O.normal(geo, v, d64, case["smaps"], case["coords"], 0.0)
    ys = O.stacked_forward(geo, case["x"].astype(np.complex128), d64, case["smaps"],
                           case["coords"])
    rng = np.random.default_rng(32)
    ys = [y + 0.02 * np.abs(y).max() * (rng.standard_normal(y.shape)
                                        + 1j * rng.standard_normal(y.shape)) for y in ys]
    y = np.concatenate(ys).astype(np.complex64)
    b = O.stacked_adjoint(geo, [yy.astype(np.complex128) for yy in np.split(
        y, np.cumsum([c.shape[0] for c in case["coords"]])[:-1])], d64, case["smaps"],
        case["coords"])
    v0 = _field(33, shape)
    lam_max, _ = F.max_eig(E0, v0.astype(np.complex128), 20)
    yield dict(shape=shape, plan=plan, E0=E0, y=y, b=b, v0=v0, lam_max=lam_max)
    plan.close()


def test_power_iteration_matches_oracle(sense_prob):
    p = sense_prob
    v = to_dev(p["v0"])
    est, _ = p["plan"].max_eig(v, 20)
    print(f"lambda_max GPU {est:.8e} oracle {p['lam_max']:.8e}")
    assert abs(est - p["lam_max"]) < 1e-5 * p["lam_max"]


def test_lipschitz_bound_matches_oracle(sense_prob):
    # the library forms the step bound L = 2 margin lambda_max itself
    import ctypes
    from paper_2501_16713_gb300 import nrsense
    p = sense_prob
    v = to_dev(p["v0"])
    lib = nrsense.load()
    L = ctypes.c_double()
    st = lib.nrsense_fista_lipschitz(p["plan"]._h, ctypes.c_void_p(v.data_ptr()), 20,
                                     ctypes.c_double(1.05), ctypes.byref(L), None)
    assert st == 0
    assert abs(L.value - 2.0 * 1.05 * p["lam_max"]) < 1e-5 * L.value
    # a margin below 1 would give a bound under 2 lambda_max: rejected
    assert lib.nrsense_fista_lipschitz(p["plan"]._h, ctypes.c_void_p(v.data_ptr()), 20,
                                       ctypes.c_double(0.9), ctypes.byref(L), None) == -1


@pytest.mark.parametrize("levels", [2, 3])
def test_fista_matches_oracle(sense_prob, levels):
    p = sense_prob
    L = 2.0 * 1.02 * p["lam_max"]
    # threshold tau = lambda / L at the 60th percentile of the coefficient
    # moduli of the first step's input, so that many coefficients vanish
    lam = L * float(np.quantile(np.abs(F.haar_forward(2.0 * p["b"] / L, levels)), 0.6))
    K = 12
    x_ref, h_ref = F.fista(p["E0"], p["b"], lam, L, levels, K)
    x, h, _ = p["plan"].solve_fista(to_dev(p["y"]), lam, levels=levels, L=L, maxit=K, graph=False)
    x = x.cpu().numpy()
    zero_frac = float(np.mean(np.abs(F.haar_forward(x_ref, levels)) < 1e-12))
    e = rel_l2(x, x_ref)
    print(f"levels {levels}: rel L2 {e:.2e}, zero coefficients {zero_frac:.2f}, "
          f"change {h[-1]:.3e} vs {h_ref[-1]:.3e}")
    assert 0.1 < zero_frac < 0.95
    assert e < TOL_FISTA
    assert np.allclose(h, h_ref, rtol=1e-3, atol=1e-7)


def test_fista_initial_guess_and_zero_iterations(sense_prob):
    p = sense_prob
    L = 2.0 * 1.02 * p["lam_max"]
    lam, levels = 1e-3 * L, 2
    x0 = _field(34, p["shape"])
    x_ref, _ = F.fista(p["E0"], p["b"], lam, L, levels, 4, x0=x0.astype(np.complex128))
    x, _, _ = p["plan"].solve_fista(to_dev(p["y"]), lam, levels=levels, L=L, maxit=4,
                                    x0=to_dev(x0), graph=False)
    assert rel_l2(x.cpu().numpy(), x_ref) < TOL_FISTA
    x, h, _ = p["plan"].solve_fista(to_dev(p["y"]), lam, levels=levels, L=L, maxit=0,
                                    x0=to_dev(x0))
    assert np.array_equal(x.cpu().numpy(), x0) and h == []
    x, _, _ = p["plan"].solve_fista(to_dev(p["y"]), lam, levels=levels, L=L, maxit=0)
    assert float(x.abs().max()) == 0.0


def test_fista_graph_replay_matches_eager(sense_prob):
    import torch
    p = sense_prob
    L = 2.0 * 1.02 * p["lam_max"]
    lam = 0.05 * L
    out = torch.empty(p["shape"], dtype=torch.complex64, device="cuda")
    y = to_dev(p["y"])
    # 70 = two captured 32-iteration chunks and 6 eager iterations
    x_e, h_e, _ = p["plan"].solve_fista(y, lam, levels=3, L=L, maxit=70, graph=False,
                                        out=out.clone())
    x_g, h_g, _ = p["plan"].solve_fista(y, lam, levels=3, L=L, maxit=70, graph=True, out=out)
    x_g2, h_g2, _ = p["plan"].solve_fista(y, lam, levels=3, L=L, maxit=70, graph=True, out=out)
    assert torch.equal(x_e, x_g) and torch.equal(x_g, x_g2)
    assert h_e == h_g == h_g2
    assert p["plan"].device_status() == 0


def test_fista_invalid_arguments(sense_prob):
    from paper_2501_16713_gb300 import NrsenseError
    p = sense_prob
    y = to_dev(p["y"])
    for kw in (dict(levels=4), dict(levels=-1), dict(L=0.0), dict(L=float("nan"))):
        args = dict(levels=2, L=1.0, maxit=2)
        args.update(kw)
        with pytest.raises(NrsenseError) as ei:  # 24 is not divisible by 16
            p["plan"].solve_fista(y, 0.1, **args)
        assert ei.value.code == -1
    with pytest.raises(NrsenseError):
        p["plan"].solve_fista(y, -1.0, levels=2, L=1.0, maxit=2)


def test_appendix_warp_inversion():
    """Appendix 1 in 3D: q = T p for a piecewise-constant phantom and a smooth
    nonrigid field; 400 FISTA iterations at lambda = 1e-6 recover p far better
    than warping q by -d.  The first iterations match the oracle."""
    shape = (32, 32, 32)
    p_img = synth.phantom(shape, 41, n_ellipsoids=8, smooth_vox=0.0)
    d = synth.bump_displacement(shape, 42, 3.0, width_range=(4.0, 8.0))
    plan = make_plan({"disp": [d]}, shape)
    neg = make_plan({"disp": [(-d).astype(np.float32)]}, shape)
    q = plan.warp_forward(to_dev(p_img))
    naive = neg.warp_forward(q[0])[0].cpu().numpy()
    L = plan.lipschitz(iters=40)
    x, hist, _ = plan.solve_fista(q.reshape(plan.forward_shape()), 1e-6, levels=3, L=L,
                                  maxit=400)
    x = x.cpu().numpy()
    e_fista, e_naive = rel_l2(x, p_img), rel_l2(naive, p_img)
    print(f"relative error: FISTA {e_fista:.3e}, naive -d warp {e_naive:.3e}; "
          f"last change {hist[-1]:.2e}")
    assert e_fista < 0.25 * e_naive
    # oracle parity on the first iterations: q and L from the oracle, the
    # same q given to the GPU solve
    geo = O.Geometry(shape)
    d64 = [d.astype(np.float64)]
    qn = O.warp_forward(geo, p_img.astype(np.complex128), d64[0])
    b = O.warp_adjoint(geo, qn, d64[0])
    E0 = lambda v: O.warp_normal(geo, v, d64, 0.0)
    lam_max, _ = F.max_eig(E0, _field(43, shape).astype(np.complex128), 6)
    L_ref = 2.04 * lam_max
    x_ref, _ = F.fista(E0, b, 1e-6, L_ref, 3, 6)
    qd = to_dev(qn.astype(np.complex64)[None])
    x6, _, _ = plan.solve_fista(qd, 1e-6, levels=3, L=L_ref, maxit=6)
    e6 = rel_l2(x6.cpu().numpy(), x_ref)
    print(f"6 iterations vs oracle: rel L2 {e6:.2e}")
    assert e6 < TOL_FISTA
    plan.close()
    neg.close()
