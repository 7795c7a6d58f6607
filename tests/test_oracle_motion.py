"""Pins of the motion-capture oracle (CPU only).

Density compensation: for samples on every point of the oversampled grid
the Pipe-Menon weights are the closed-form constant 1 / S^2, S the sum of the
3D kernel over the integer taps, reached in one step and a fixed point;
duplicating every sample halves the weights; the convolution B P equals the
dense matrix sum_g c(q_s - g) c(q_s' - g) built from the kernel function.
Correlation: the FFT form equals the direct circular sum; an integer circular
shift of a random image is recovered (the peak exactly, the refined value
within 0.05), a sub-voxel shift of a smooth
blob within 0.1 voxel; the parabolic refinement finds the vertex of an exact
parabola.  Phase ramp: against the brute-force NUDFT of a shifted image with
compact support.  k-means: Lloyd's result on well-separated clusters equals
the optimum found by enumerating every assignment; the inertia never
increases; labels do not depend on the input order, a translation or a
scaling of the points; the least-variance cluster is found.  The last test
plants mistakes in the oracle and requires each to fail a pin.
"""

import itertools
import math

import numpy as np
import pytest

from oracle import kernel as K
from oracle import motion as Mo
from oracle import operators as O
from oracle import references as R


def _crandn(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


# ---------------------------------------------------------------- DCF ------

def _grid_omegas(geo):
    """Samples on every point of the oversampled grid: q = omega G / 2 pi integer."""
    axes = [np.arange(-g // 2, g // 2) * (2 * np.pi / g) for g in geo.grid]
    w = np.stack(np.meshgrid(*axes, indexing="ij"), axis=-1).reshape(-1, 3)
    return w


def pin_dcf_uniform_grid():
    geo = O.Geometry((4, 4, 6))
    om = _grid_omegas(geo)
    s1 = sum(K.kb_kernel(float(t), geo.width, geo.beta) for t in range(-(geo.width // 2) + 1,
                                                                      geo.width // 2))
    want = 1.0 / s1 ** 6  # (S_1^3)^2
    for iters in (1, 3):
        w, bpw = Mo.dcf_pipe_menon(geo, om, iters)
        assert np.abs(w / want - 1).max() < 1e-12
        assert np.abs(bpw - 1).max() < 1e-12


def pin_dcf_duplicates_halve():
    rng = np.random.default_rng(1)
    geo = O.Geometry((6, 6, 6))
    om = rng.uniform(-np.pi, np.pi, (60, 3))
    w, _ = Mo.dcf_pipe_menon(geo, om, 4)
    w2, _ = Mo.dcf_pipe_menon(geo, np.concatenate([om, om]), 4)
    assert np.abs(w2[:60] / (0.5 * w) - 1).max() < 1e-12
    assert np.abs(w2[60:] / (0.5 * w) - 1).max() < 1e-12


def pin_dcf_dense_convolution():
    """One and two iterations against the dense matrix K[s, s'] built from the
    kernel function over every grid point (periodic taps)."""
    rng = np.random.default_rng(2)
    geo = O.Geometry((4, 4, 4))
    om = rng.uniform(-np.pi, np.pi, (30, 3))
    q = O.kspace_positions(geo, om)
    G = geo.grid
    half = geo.width / 2.0
    A = np.zeros((q.shape[1], int(np.prod(G))))
    for s in range(q.shape[1]):
        for g in itertools.product(*(range(n) for n in G)):
            w = 1.0
            for a in range(3):
                # nearest periodic image of grid point g to q
                d = (q[a, s] - g[a] + G[a] / 2.0) % G[a] - G[a] / 2.0
                w *= K.kb_kernel(d, geo.width, geo.beta) if abs(d) < half else 0.0
            A[s, np.ravel_multi_index(g, G)] = w
    Km = A @ A.T
    w1 = 1.0 / (Km @ np.ones(q.shape[1]))
    w2 = w1 / (Km @ w1)
    for it, want in ((1, w1), (2, w2)):
        w, _ = Mo.dcf_pipe_menon(geo, om, it)
        assert np.abs(w / want - 1).max() < 1e-11, it


# -------------------------------------------------------- correlation ------

def pin_xcorr_direct_sum():
    rng = np.random.default_rng(3)
    shape = (4, 5, 6)
    a, b = _crandn(rng, shape), _crandn(rng, shape)
    c = Mo.xcorr(a, b)
    for t in itertools.product(*(range(n) for n in shape)):
        want = sum(abs(a[n]) * abs(b[tuple((n[i] + t[i]) % shape[i] for i in range(3))])
                   for n in itertools.product(*(range(m) for m in shape)))
        assert abs(c[t] - want) < 1e-10 * max(1.0, want)


def pin_integer_shift_recovered():
    rng = np.random.default_rng(4)
    shape = (12, 10, 16)
    ref = _crandn(rng, shape)
    for t in [(3, -2, 5), (0, 0, 0), (-5, 4, -7), (6, 5, 8)]:
        img = np.roll(ref, t, axis=(0, 1, 2))  # img[n] = ref[n - t]
        est = Mo.translation(ref, img)
        want = [((t[a] + shape[a] // 2 - 1) % shape[a]) - shape[a] // 2 + 1 for a in range(3)]
        # the peak is exact; the parabolic refinement moves it by a small
        # fraction (the neighbours of a white-noise correlation peak differ)
        assert np.array_equal(np.rint(est), np.asarray(want, dtype=float)), (t, est)
        assert np.abs(est - want).max() < 0.05, (t, est)


def pin_subvoxel_shift():
    shape = (24, 24, 24)
    r = np.stack(np.meshgrid(*[np.arange(n) for n in shape], indexing="ij"))
    c0 = np.array([12.0, 11.0, 12.5])
    blob = lambda c: np.exp(-((r - c[:, None, None, None]) ** 2).sum(0) / (2 * 2.0 ** 2))
    for t in ([0.3, -0.4, 1.25], [-2.6, 0.0, 0.5]):
        est = Mo.translation(blob(c0), blob(c0 + np.asarray(t)))
        assert np.abs(est - np.asarray(t)).max() < 0.1, (t, est)


def pin_parabola_vertex():
    shape = (9, 8, 10)
    r = np.stack(np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")).astype(float)
    v = np.array([4.3, 3.8, 5.1])
    c = 100.0 - ((r - v[:, None, None, None]) ** 2).sum(0)
    est = Mo.peak_shift(c)
    want = np.where(v > np.asarray(shape) / 2, v - np.asarray(shape), v)
    assert np.abs(est - want).max() < 1e-12


def pin_phase_ramp_undoes_shift():
    """y of an image shifted by integer t (support kept inside the volume)
    times exp(+i omega . t) is y of the unshifted image (brute-force NUDFT)."""
    rng = np.random.default_rng(5)
    geo = O.Geometry((8, 8, 10))
    x = np.zeros(geo.shape, complex)
    x[2:5, 3:6, 3:6] = _crandn(rng, (3, 3, 3))
    t = np.array([2, -1, 3])
    xs = np.roll(x, tuple(t), axis=(0, 1, 2))
    om = rng.uniform(-np.pi, np.pi, (40, 3))
    y = R.nudft(geo, x, om)
    ys = R.nudft(geo, xs, om)
    yc = Mo.phase_ramp(ys[:, None], om, t)[:, 0]
    assert np.abs(yc - y).max() < 1e-10 * np.abs(y).max()


# ------------------------------------------------------------- k-means ----

def _clusters(seed, n_per, centres, spread=0.3):
    rng = np.random.default_rng(seed)
    pts = np.concatenate([c + spread * rng.standard_normal((n_per, 3)) for c in centres])
    return pts[rng.permutation(len(pts))]


def _inertia(p, labels, k):
    tot = 0.0
    for j in range(k):
        sel = labels == j
        if sel.any():
            tot += ((p[sel] - p[sel].mean(0)) ** 2).sum()
    return tot


def pin_kmeans_optimal_small():
    for seed, k in ((6, 2), (7, 3)):
        centres = [np.array([0, 0, 0.]), np.array([5, 1, 0.]), np.array([1, 6, 2.])][:k]
        p = _clusters(seed, 3, centres)
        labels, _, inertia, _ = Mo.kmeans(p, k)
        best = min(_inertia(p, np.asarray(a), k)
                   for a in itertools.product(range(k), repeat=len(p)))
        assert abs(inertia - best) < 1e-9 * best


def pin_kmeans_monotone():
    p = _clusters(8, 40, [np.zeros(3), np.array([2., 0, 0]), np.array([0, 2., 1]),
                          np.array([2., 2, 0])], spread=0.8)
    prev = np.inf
    for it in range(1, 12):
        labels, centres, inertia, _ = Mo.kmeans(p, 4, max_iter=it)
        cur = _inertia(p, labels, 4)
        assert cur <= prev + 1e-9
        prev = cur


def pin_kmeans_invariances():
    p = _clusters(9, 25, [np.zeros(3), np.array([4., 0, 0]), np.array([0, 4., 0]),
                          np.array([4., 4, 3])])
    labels, _, _, _ = Mo.kmeans(p, 4)
    perm = np.random.default_rng(10).permutation(len(p))
    l2, _, _, _ = Mo.kmeans(p[perm], 4)
    assert np.array_equal(l2, labels[perm])
    l3, _, _, _ = Mo.kmeans(3.0 * p + np.array([1.0, -2.0, 7.0]), 4)
    assert np.array_equal(l3, labels)


def pin_reference_cluster():
    rng = np.random.default_rng(11)
    tight = 0.05 * rng.standard_normal((20, 3))
    loose = np.array([6.0, 0, 0]) + 1.0 * rng.standard_normal((20, 3))
    p = np.concatenate([loose, tight])
    labels, centres, _, _ = Mo.kmeans(p, 2)
    j = Mo.reference_cluster(p, labels, centres)
    assert np.all(labels[20:] == j) and np.all(labels[:20] != j)


PINS = [pin_dcf_uniform_grid, pin_dcf_duplicates_halve, pin_dcf_dense_convolution,
        pin_xcorr_direct_sum, pin_integer_shift_recovered, pin_subvoxel_shift,
        pin_parabola_vertex, pin_phase_ramp_undoes_shift, pin_kmeans_optimal_small,
        pin_kmeans_monotone, pin_kmeans_invariances, pin_reference_cluster]


@pytest.mark.parametrize("pin", PINS, ids=[p.__name__ for p in PINS])
def test_pin(pin):
    pin()


# ------------------------------------------------------------ mutants -----

def _mutants():
    orig_xcorr, orig_peak, orig_ramp = Mo.xcorr, Mo.peak_shift, Mo.phase_ramp
    orig_dcf, orig_init = Mo.dcf_pipe_menon, Mo.kmeans_init

    def xcorr_conv(ref, img):  # convolution instead of correlation
        a, b = np.abs(ref), np.abs(img)
        return np.real(np.fft.ifftn(np.fft.fftn(a) * np.fft.fftn(b)))

    def peak_sign(c):
        c = np.asarray(c, dtype=np.float64)
        t = np.unravel_index(int(np.argmax(c)), c.shape)
        out = []
        for a in range(3):
            n = c.shape[a]
            ip, im = list(t), list(t)
            ip[a] = (t[a] + 1) % n
            im[a] = (t[a] - 1) % n
            cm, c0, cp = c[tuple(im)], c[t], c[tuple(ip)]
            den = cm - 2.0 * c0 + cp
            d = 0.5 * (cp - cm) / den if den < 0 else 0.0
            v = t[a] + d
            out.append(v - n if v > n / 2 else v)
        return np.asarray(out)

    def ramp_sign(y, omega, t):
        return orig_ramp(y, omega, -np.asarray(t, dtype=float))

    def dcf_multiply(geo, omega, iters):
        q = O.kspace_positions(geo, np.asarray(omega))
        w = np.ones(q.shape[1])
        for _ in range(iters):
            g = O.projection_core(w.astype(complex), q, geo.grid, geo.width, geo.beta)
            w = w * O.backprojection_core(g, q, geo.width, geo.beta).real
        g = O.projection_core(w.astype(complex), q, geo.grid, geo.width, geo.beta)
        return w, O.backprojection_core(g, q, geo.width, geo.beta).real

    def dcf_one_kernel(geo, omega, iters):  # spread only, no interpolation back
        q = O.kspace_positions(geo, np.asarray(omega))
        w = np.ones(q.shape[1])
        for _ in range(iters):
            idx = np.floor(q).astype(int) % np.asarray(geo.grid)[:, None]
            g = O.projection_core(w.astype(complex), q, geo.grid, geo.width, geo.beta)
            w = w / np.abs(g[idx[0], idx[1], idx[2]]).real
        return w, np.ones_like(w)

    def init_first(points, k):
        return np.asarray(points, dtype=float)[:k].copy()

    def kmeans_no_update(points, k, max_iter=100):
        p = np.asarray(points, dtype=float)
        centres = orig_init(p, k)
        d2 = ((p[:, None, :] - centres[None]) ** 2).sum(2)
        labels = np.argmin(d2, axis=1)
        return labels, centres, float(((p - centres[labels]) ** 2).sum()), 1

    return [
        ("convolution instead of correlation", "xcorr", xcorr_conv),
        ("parabola vertex with the wrong sign", "peak_shift", peak_sign),
        ("phase ramp with the wrong sign", "phase_ramp", ramp_sign),
        ("DCF multiplies", "dcf_pipe_menon", dcf_multiply),
        ("DCF without interpolation", "dcf_pipe_menon", dcf_one_kernel),
        ("k-means started from the first k points", "kmeans_init", init_first),
        ("k-means without centre updates", "kmeans", kmeans_no_update),
    ]


def _pins_hold():
    for pin in PINS:
        try:
            pin()
        except (AssertionError, ValueError, IndexError, FloatingPointError, ZeroDivisionError):
            return False
    return True


def test_pins_catch_planted_mistakes(monkeypatch):
    for name, attr, repl in _mutants():
        with monkeypatch.context() as m:
            m.setattr(Mo, attr, repl)
            assert not _pins_hold(), f"no pin catches: {name}"
