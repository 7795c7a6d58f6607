"""Motion capture for segmented acquisitions (oracle; test infrastructure:
only the tests, the smoke check and the benchmark's CPU baseline use this
module).

Section "Motion Capturing for Segmented Data Acquisitions": every heartbeat
acquires a full low-resolution trajectory; its direct (gridding)
reconstruction, from "sampled, density corrected" data (notation table), is
the heartbeat's 3D iNAV.  Bulk translation per heartbeat comes from
correlations between a reference iNAV and the others and is corrected by
linear phase shifts of the k-space data; k-means on the translation
estimates gives the respiratory phases ("Nonrigid Respiratory Motion
Correction": four phases, the end-expiration cluster, the one with the
least variance, is the reference).  Readings taken here (the paper names the
steps, not their formulas):

  * Density compensation: Pipe and Menon's fixed-point iteration
    w <- w / (B P w) from w = 1, with P the k-space spread onto the
    oversampled grid and B the interpolation back to the samples, both with
    the gridding kernel c (so B P w[s] = sum_s' sum_g c(q_s - g) c(q_s' - g) w_s').
  * Correlation: circular cross-correlation of the magnitude images,
    c[t] = sum_n |ref[n]| |img[n + t]|; the estimate is the integer argmax
    (first in C order on ties) refined per axis by the vertex of the parabola
    through c at t - 1, t, t + 1 (no refinement when that parabola is not
    concave), wrapped to (-n/2, n/2].  img[n] = ref[n - t] gives t.
  * Phase-ramp correction: the data of an image shifted by +t carry the
    factor exp(-i omega . t) (forward transform exp(-i omega . n)), so the
    correction multiplies by exp(+i omega . t).
  * k-means: Lloyd's iteration (nearest centre, ties to the lower index;
    centres = cluster means, an empty cluster keeps its centre) until the
    assignment stops changing, started from the points at the quantile
    positions (i + 1/2) n / k of the order along the first principal axis
    (sign fixed so that its largest-magnitude entry is positive; ties in the
    projection keep input order).
"""

from __future__ import annotations

import numpy as np

from . import operators as O


# ---------------------------------------------------------------- DCF ------

def dcf_pipe_menon(geo: O.Geometry, omega, iters: int):
    """Pipe-Menon density compensation weights of the samples omega (M x 3
    radians) on geo's oversampled grid; returns (w, B P w of the last w)."""
    q = O.kspace_positions(geo, np.asarray(omega))
    w = np.ones(q.shape[1])
    for _ in range(iters):
        grid = O.projection_core(w.astype(np.complex128), q, geo.grid, geo.width, geo.beta)
        s = O.backprojection_core(grid, q, geo.width, geo.beta).real
        w = w / s
    grid = O.projection_core(w.astype(np.complex128), q, geo.grid, geo.width, geo.beta)
    return w, O.backprojection_core(grid, q, geo.width, geo.beta).real


# ------------------------------------------------------- correlation ------

def xcorr(ref, img):
    """c[t] = sum_n |ref[n]| |img[n + t]| (circular), via the FFT."""
    a = np.abs(np.asarray(ref, dtype=np.complex128))
    b = np.abs(np.asarray(img, dtype=np.complex128))
    return np.real(np.fft.ifftn(np.conj(np.fft.fftn(a)) * np.fft.fftn(b)))


def peak_shift(c):
    """Integer argmax of c refined per axis by a three-point parabola, wrapped
    to (-n/2, n/2] per axis."""
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
        d = 0.5 * (cm - cp) / den if den < 0 else 0.0
        v = t[a] + d
        if v > n / 2:
            v -= n
        out.append(v)
    return np.asarray(out)


def translation(ref, img):
    return peak_shift(xcorr(ref, img))


def phase_ramp(y, omega, t):
    """y (M x C) times exp(+i omega . t) per sample (undoes a shift by +t)."""
    ph = np.asarray(omega, dtype=np.float64) @ np.asarray(t, dtype=np.float64)
    return np.asarray(y) * np.exp(1j * ph)[:, None]


# ----------------------------------------------------------- k-means ------

def kmeans_init(points, k):
    p = np.asarray(points, dtype=np.float64)
    c = p - p.mean(axis=0)
    _, _, vt = np.linalg.svd(c, full_matrices=False)
    v = vt[0]
    if v[np.argmax(np.abs(v))] < 0:
        v = -v
    order = np.argsort(c @ v, kind="stable")
    n = p.shape[0]
    return p[order[[int((i + 0.5) * n / k) for i in range(k)]]].copy()


def kmeans(points, k, max_iter=100):
    """Returns (labels, centres, inertia, iterations)."""
    p = np.asarray(points, dtype=np.float64)
    centres = kmeans_init(p, k)
    labels = None
    it = 0
    while it < max_iter:
        d2 = ((p[:, None, :] - centres[None, :, :]) ** 2).sum(axis=2)
        new = np.argmin(d2, axis=1)
        it += 1
        if labels is not None and np.array_equal(new, labels):
            break
        labels = new
        for j in range(k):
            sel = labels == j
            if sel.any():
                centres[j] = p[sel].mean(axis=0)
    inertia = float(((p - centres[labels]) ** 2).sum())
    return labels, centres, inertia, it


def reference_cluster(points, labels, centres):
    """Index of the cluster with the least variance (mean squared distance of
    its members to its centre); empty clusters are skipped."""
    p = np.asarray(points, dtype=np.float64)
    best, bv = -1, np.inf
    for j in range(centres.shape[0]):
        sel = labels == j
        if not sel.any():
            continue
        v = float(((p[sel] - centres[j]) ** 2).sum(axis=1).mean())
        if v < bv:
            best, bv = j, v
    return best
