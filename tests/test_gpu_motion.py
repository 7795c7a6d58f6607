"""Motion capture on the GPU against the FP64 oracle, and end to end.

Parity: Pipe-Menon weights (10 iterations, 2 phases of a cone-like case),
the density-weighted adjoint, the magnitude cross-correlation translation
(integer peak equal, refined value within 1e-3 voxel), the phase ramp and
k-means (labels bit-exact, centres to 1e-12 on well-separated clusters,
where no distance tie can arise).

End to end (ground truth, no oracle): 32 heartbeats of a 32^3, 4-coil iNAV
acquisition whose images are the phantom translated by respiratory
positions of four phases along axis 0 plus jitter; the library computes the
density compensation, the gridding reconstruction of every heartbeat, the
translations against heartbeat 0, the k-means phases and the phase-ramp
correction.  The translations must match the truth within 0.3 voxel, the
phases must match up to relabelling, and the corrected reconstructions must
be much closer to the reference than the uncorrected ones (measured spread
2.33 before, 0.54 after).

Tolerances: the DCF divides by an FP32 convolution sum each iteration (1e-6
relative each), so 10 iterations stay within 1e-4; the adjoint is the FP32
operator (1e-5, the operator bar); the phase ramp rounds the reduced phase to
FP32 before sincosf (about 1e-6).
"""

import numpy as np
import pytest

import synth
from helpers import TOL_FP32, make_plan, rel_l2, to_dev
from oracle import motion as Mo
from oracle import operators as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()


def _crandn(rng, shape):
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).astype(np.complex64)


@pytest.fixture(scope="module")
def case():
    shape = (16, 16, 24)
    c = synth.small_case(shape, 2, 2, [3000, 2500], seed=61, max_disp=1.5, rigid=0.5)
    plan = make_plan(c, shape)
    yield shape, c, plan
    plan.close()


def test_dcf_matches_oracle(case):
    shape, c, plan = case
    geo = O.Geometry(shape)
    for j in range(2):
        w = plan.dcf(j, iters=10).cpu().numpy()
        w_ref, bpw = Mo.dcf_pipe_menon(geo, c["coords"][j].astype(np.float64), 10)
        e = float(np.abs(w / w_ref - 1).max())
        print(f"phase {j}: DCF max rel {e:.2e}; oracle max |BPw - 1| {np.abs(bpw - 1).max():.2e}")
        assert e < 1e-4
    assert plan.device_status() == 0


def test_weighted_adjoint_matches_oracle(case):
    shape, c, plan = case
    geo = O.Geometry(shape)
    rng = np.random.default_rng(62)
    M = [x.shape[0] for x in c["coords"]]
    y = _crandn(rng, (sum(M), 2))
    w = rng.uniform(0.2, 2.0, sum(M)).astype(np.float32)
    x = plan.adjoint_weighted(to_dev(y), to_dev(w)).cpu().numpy()
    yw = (y.astype(np.complex128) * w.astype(np.float64)[:, None])
    ys = np.split(yw, np.cumsum(M)[:-1])
    d64 = [d.astype(np.float64) for d in c["disp"]]
    x_ref = O.stacked_adjoint(geo, ys, d64, c["smaps"], c["coords"])
    e = rel_l2(x, x_ref)
    print(f"weighted adjoint rel L2 {e:.2e}")
    assert e < TOL_FP32


def test_translation_xcorr_matches_oracle():
    from paper_2501_16713_gb300 import translation_xcorr
    rng = np.random.default_rng(63)
    shape = (24, 20, 32)
    ref = _crandn(rng, shape)
    # no shift of exactly n/2: its wrap would hang on the sign of a tiny refinement
    shifts = [(3, -2, 5), (0, 0, 0), (-7, 9, -12), (11, 9, 15), (1, 1, -1)]
    imgs = np.stack([np.roll(ref, t, axis=(0, 1, 2)) for t in shifts])
    # smooth blobs with sub-voxel shifts as a second batch
    r = np.stack(np.meshgrid(*[np.arange(n) for n in shape], indexing="ij"))
    blob = lambda c0: np.exp(-((r - np.asarray(c0)[:, None, None, None]) ** 2).sum(0) / 8.0)
    bref = blob([12.0, 10.0, 16.0]).astype(np.complex64)
    bimgs = np.stack([blob([12.0 + a, 10.0 + b, 16.0 + cc]) for a, b, cc in
                      [(0.3, -0.4, 1.25), (-2.6, 0.0, 0.5), (4.1, 3.3, -5.7)]]).astype(np.complex64)
    for rf, im in ((ref, imgs), (bref, bimgs)):
        got = translation_xcorr(to_dev(rf), to_dev(im))
        want = np.stack([Mo.translation(rf.astype(np.complex128), x.astype(np.complex128))
                         for x in im])
        print(np.round(got, 4), np.round(want, 4))
        assert np.array_equal(np.rint(got), np.rint(want))
        assert np.abs(got - want).max() < 1e-3


def test_phase_ramp_matches_oracle():
    from paper_2501_16713_gb300 import phase_ramp
    rng = np.random.default_rng(64)
    rows, C = 5000, 3
    om = rng.uniform(-np.pi, np.pi, (rows, 3)).astype(np.float32)
    y = _crandn(rng, (rows, C))
    off = [100, 1200, 1201, 4800]  # rows 0..99 and 4800.. untouched; one empty-ish segment
    sh = np.array([[1.5, -2.25, 7.0], [0.0, 0.0, 0.0], [-11.3, 4.4, 0.6]])
    yd = to_dev(y)
    phase_ramp(to_dev(om), yd, off, sh)
    got = yd.cpu().numpy()
    want = y.astype(np.complex128).copy()
    for s in range(3):
        a, b = off[s], off[s + 1]
        want[a:b] = Mo.phase_ramp(want[a:b], om[a:b].astype(np.float64), sh[s])
    e = float(np.abs(got - want).max() / np.abs(want).max())
    print(f"phase ramp max rel {e:.2e}")
    assert e < 2e-6
    assert np.array_equal(got[:100], y[:100]) and np.array_equal(got[4800:], y[4800:])


def test_kmeans_matches_oracle():
    from paper_2501_16713_gb300 import NrsenseError, kmeans
    rng = np.random.default_rng(65)
    centres = np.array([[0.0, 0, 0], [3.0, 0.5, 0], [6.0, -0.5, 0.2], [9.0, 0, -0.3]])
    p = np.concatenate([c + 0.4 * rng.standard_normal((50, 3)) for c in centres])
    p = p[rng.permutation(len(p))]
    for k in (2, 3, 4, 6):
        labels, cen, inertia, iters, ref = kmeans(p, k)
        l_o, c_o, i_o, it_o = Mo.kmeans(p, k)
        assert np.array_equal(labels, l_o), k
        assert np.abs(cen - c_o).max() < 1e-12 and abs(inertia - i_o) < 1e-9 * i_o
        assert iters == it_o and ref == Mo.reference_cluster(p, l_o, c_o)
    with pytest.raises(NrsenseError):
        kmeans(p[:3], 4)


def test_motion_capture_end_to_end():
    import torch
    from paper_2501_16713_gb300 import Plan, kmeans, phase_ramp, translation_xcorr
    rng = np.random.default_rng(66)
    shape, C, H = (32, 32, 32), 4, 32
    x = synth.phantom(shape, 67, n_ellipsoids=10, smooth_vox=1.0)
    smaps = synth.coil_maps(shape, C, 68)
    om = synth.cones_trajectory(12, 400, 69).astype(np.float32)
    M = om.shape[0]
    plan = Plan(shape, coords=[to_dev(om)], smaps=to_dev(smaps), n_phases=1, identity_warp=True)
    phase_of = np.arange(H) % 4
    pos = np.array([0.0, 1.2, 2.4, 3.6])
    t = np.zeros((H, 3))
    t[:, 0] = pos[phase_of] + 0.1 * rng.standard_normal(H)
    t[:, 1:] = 0.1 * rng.standard_normal((H, 2))
    y_ref = plan.forward(to_dev(x))                           # (M, C)
    omd = to_dev(om)
    ys = y_ref.repeat(H, 1).contiguous()                     # heartbeat h: rows h M .. (h+1) M
    big = torch.cat([omd] * H).contiguous()
    off = np.arange(H + 1) * M
    phase_ramp(big, ys, off, -t)                             # image of heartbeat h moved by +t_h
    scale = 0.01 * float(y_ref.abs().max())
    ys += scale * torch.randn(ys.shape, dtype=torch.complex64, device="cuda",
                              generator=torch.Generator(device="cuda").manual_seed(70))
    w = plan.dcf(0, iters=10)
    recon = torch.stack([plan.adjoint_weighted(ys[h * M:(h + 1) * M], w) for h in range(H)])
    est = translation_xcorr(recon[0].contiguous(), recon)
    err = np.abs(est - (t - t[0])).max()
    print(f"translation error max {err:.3f} voxel")
    assert err < 0.3
    labels, _, _, _, ref = kmeans(est, 4)
    # the same partition as the true phases, up to relabelling
    for j in range(4):
        assert len(set(labels[phase_of == j])) == 1
    assert len(set(labels)) == 4 and 0 <= ref < 4
    # correction: move every heartbeat back by its estimate
    yc = ys.clone()
    phase_ramp(big, yc, off, est)
    rc = torch.stack([plan.adjoint_weighted(yc[h * M:(h + 1) * M], w) for h in range(H)])
    d_before = float(torch.linalg.norm(recon - recon[0]) / torch.linalg.norm(recon[0]))
    d_after = float(torch.linalg.norm(rc - rc[0]) / torch.linalg.norm(rc[0]))
    print(f"spread of the heartbeat reconstructions: before {d_before:.3f}, after {d_after:.3f}")
    # what remains is each heartbeat's own noise (1 % of the peak sample,
    # through the density-weighted gridding), not misregistration
    assert d_after < 0.3 * d_before
    plan.close()
