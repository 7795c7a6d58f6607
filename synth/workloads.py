"""Seeded synthetic workloads (inputs only; no operator arithmetic here).

Array conventions shared by every consumer:

* image            : (N0, N1, N2) complex64, C order (axis 2 fastest)
* displacement d_j : (3, N0, N1, N2) float32; component a moves along array
                     axis a, in voxel units of the N grid (pull convention of
                     the displacement-field equation: m_j[r] = m(r + d[r]))
* coil maps        : (C, N0, N1, N2) complex64, sum over coils of |S_c|^2 = 1
* trajectory       : per phase (M_j, 3) float32 radians in (-pi, pi); column a
                     is the angular frequency along image axis a

The workload recipes restate the five benchmark configurations of the method's
hot path: a 32^3 image-space-only warp, the 128^3 8-coil 4-phase operator,
the 192^3 16-coil 6-phase CG problem with uneven phase sizes, the learned
preconditioner problem on the 128^3 geometry, and the 256^3 32-coil 8-phase
precision sweep.
"""

from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np
from scipy import ndimage

# Interleaves acquired per heartbeat (R-R interval) in the paper's in-vivo
# protocol ("Nonrigid Respiratory Motion Correction": 18 conic interleaves of
# a 3D cones phyllotaxis trajectory per R-R).
INTERLEAVES_PER_HEARTBEAT = 18
GOLDEN_ANGLE = math.pi * (3.0 - math.sqrt(5.0))


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _grid(shape):
    """Voxel coordinates (3, N0, N1, N2) as float64."""
    return np.stack(np.meshgrid(*[np.arange(s, dtype=np.float64) for s in shape],
                                indexing="ij"))


def phantom(shape, seed: int, n_ellipsoids: int = 20, smooth_vox: float = 1.5,
            support: float = 0.4) -> np.ndarray:
    """Random smooth complex phantom: ellipsoids inside radius support*N,
    Gaussian-smoothed, times a smooth (linear plus constant) phase."""
    rng = _rng(seed)
    shape = tuple(int(s) for s in shape)
    n = np.asarray(shape, dtype=np.float64)
    r = _grid(shape) - (n / 2.0)[:, None, None, None]
    img = np.zeros(shape, dtype=np.float64)
    for _ in range(n_ellipsoids):
        # centre inside a ball so the ellipsoid stays inside radius support*N
        while True:
            c = rng.uniform(-0.25, 0.25, 3)
            if np.linalg.norm(c) <= 0.25:
                break
        c = c * n
        axes = rng.uniform(0.04, 0.15, 3) * n
        q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
        rr = np.tensordot(q.T, r - c[:, None, None, None], axes=1)
        inside = np.sum((rr / axes[:, None, None, None]) ** 2, axis=0) <= 1.0
        img += rng.uniform(0.2, 1.0) * inside
    radius = np.sqrt(np.sum((r / n[:, None, None, None]) ** 2, axis=0))
    img *= radius <= support
    img = ndimage.gaussian_filter(img, smooth_vox, mode="wrap")
    slope = rng.uniform(-1.0, 1.0, 3)
    phase = rng.uniform(-math.pi, math.pi) + np.tensordot(
        slope, r / n[:, None, None, None], axes=1)
    out = img * np.exp(1j * phase)
    out /= max(np.abs(out).max(), 1e-30)
    return out.astype(np.complex64)


def bump_displacement(shape, seed: int, max_disp: float, n_bumps: int = 6,
                      width_range=(3.0, 8.0)) -> np.ndarray:
    """Smooth displacement field: a sum of Gaussian bumps with random vector
    amplitudes, centres uniform in [0.2N, 0.8N]^3, scaled so that the largest
    per-voxel Euclidean displacement equals max_disp voxels."""
    rng = _rng(seed)
    shape = tuple(int(s) for s in shape)
    n = np.asarray(shape, dtype=np.float64)
    r = _grid(shape)
    d = np.zeros((3,) + shape, dtype=np.float64)
    for _ in range(n_bumps):
        c = rng.uniform(0.2, 0.8, 3) * n
        w = rng.uniform(*width_range)
        amp = rng.standard_normal(3)
        g = np.exp(-np.sum((r - c[:, None, None, None]) ** 2, axis=0) / (2 * w * w))
        d += amp[:, None, None, None] * g[None]
    mag = np.sqrt(np.sum(d * d, axis=0)).max()
    if max_disp == 0.0 or mag == 0.0:
        return np.zeros((3,) + shape, dtype=np.float32)
    d *= max_disp / mag
    return d.astype(np.float32)


def rigid_translation(seed: int, radius: float) -> np.ndarray:
    """A translation vector drawn uniformly from the ball of the given radius."""
    rng = _rng(seed)
    while True:
        t = rng.uniform(-1.0, 1.0, 3)
        if np.linalg.norm(t) <= 1.0:
            return (t * radius).astype(np.float64)


def coil_maps(shape, n_coils: int, seed: int, width: float = 0.4,
              ring: float = 0.6) -> np.ndarray:
    """Gaussian-profile complex coil sensitivities on a ring around the FOV,
    with smooth phase, normalised so that sum_c |S_c|^2 = 1 at every voxel."""
    rng = _rng(seed)
    shape = tuple(int(s) for s in shape)
    n = np.asarray(shape, dtype=np.float64)
    r = _grid(shape) - (n / 2.0)[:, None, None, None]
    s = width * float(n.max())
    maps = np.zeros((n_coils,) + shape, dtype=np.complex128)
    for c in range(n_coils):
        ang = 2 * math.pi * c / max(n_coils, 1) + rng.uniform(-0.1, 0.1)
        ring_idx = c % 2 if n_coils > 8 else 0
        h = (0.15 if ring_idx else -0.15) * n[0] if n_coils > 8 else 0.0
        centre = np.array([h, ring * n[1] * math.cos(ang), ring * n[2] * math.sin(ang)])
        dist2 = np.sum((r - centre[:, None, None, None]) ** 2, axis=0)
        mag = np.exp(-dist2 / (2 * s * s))
        slope = rng.uniform(-1.5, 1.5, 3)
        phase = rng.uniform(-math.pi, math.pi) + np.tensordot(
            slope, r / n[:, None, None, None], axes=1)
        maps[c] = mag * np.exp(1j * phase)
    rss = np.sqrt(np.sum(np.abs(maps) ** 2, axis=0))
    maps /= rss[None]
    return maps.astype(np.complex64)


def cones_trajectory(n_interleaves: int, readout: int, seed: int,
                     interleave_ids=None, n_total: int | None = None,
                     turns: float = 4.0, kmax: float = math.pi * 0.999) -> np.ndarray:
    """Cone-like 3D interleaves on a phyllotaxis set of cone angles.

    Interleave i (global id) has cone half-angle theta_i with cos(theta_i)
    uniform on [-1, 1] and start azimuth i * golden angle; along the readout the
    radius grows linearly in time (so the sample density falls as 1/|k|^2) while
    the azimuth winds `turns` times around the cone.  Returns (M, 3) float32
    with |omega| < pi.
    """
    rng = _rng(seed)
    if interleave_ids is None:
        interleave_ids = np.arange(n_interleaves)
    ids = np.asarray(interleave_ids, dtype=np.float64)
    if n_total is None:
        n_total = int(ids.max()) + 1 if ids.size else 1
    cos_t = 1.0 - 2.0 * (ids + 0.5) / n_total
    sin_t = np.sqrt(np.maximum(0.0, 1.0 - cos_t * cos_t))
    phi0 = ids * GOLDEN_ANGLE + rng.uniform(0, 2 * math.pi)
    t = (np.arange(readout, dtype=np.float64) + 0.5) / readout
    rad = kmax * t
    psi = 2 * math.pi * turns * t
    ang = phi0[:, None] + psi[None, :]
    k = np.empty((ids.size, readout, 3), dtype=np.float64)
    k[..., 0] = rad[None, :] * cos_t[:, None]
    k[..., 1] = rad[None, :] * sin_t[:, None] * np.cos(ang)
    k[..., 2] = rad[None, :] * sin_t[:, None] * np.sin(ang)
    return k.reshape(-1, 3).astype(np.float32)


def phase_sample_counts(targets, readout: int, seed: int, poisson: bool,
                        lo: float | None = None, hi: float | None = None):
    """Heartbeats per phase (and hence samples per phase).

    With poisson=True, the heartbeat count of phase j is Poisson with mean
    target_j / (18 * readout), then clamped so that the sample count stays in
    [lo, hi].  Returns the list of heartbeat counts."""
    rng = _rng(seed)
    per_hb = INTERLEAVES_PER_HEARTBEAT * readout
    beats = []
    for tgt in targets:
        mu = tgt / per_hb
        h = int(rng.poisson(mu)) if poisson else int(round(mu))
        if lo is not None:
            h = max(h, int(math.ceil(lo / per_hb)))
        if hi is not None:
            h = min(h, int(math.floor(hi / per_hb)))
        beats.append(max(h, 0))
    return beats


@dataclass
class Spec:
    name: str
    shape: tuple
    n_coils: int
    n_phases: int
    max_disp: float
    rigid: float
    seed: int
    readout: int = 1042
    sample_targets: list = field(default_factory=list)
    poisson: bool = False
    sample_lo: float | None = None
    sample_hi: float | None = None
    description: str = ""


WORKLOADS = {
    # image-space gridding warp only (no coils, no k-space)
    "warp32": Spec("warp32", (32, 32, 32), 0, 1, 3.0, 0.0, 1,
                   description="32^3 image-space warp T/T^H, 6 Gaussian bumps, "
                               "max |d| 3 voxels, sigma 2, W 4"),
    # full nonrigid SENSE operator
    "sense128": Spec("sense128", (128, 128, 128), 8, 4, 8.0, 4.0, 2,
                     sample_targets=[1.5e6] * 4,
                     description="128^3, 8 coils, 4 phases, ~1.5M cone samples "
                                 "per phase, max |d| 8 + rigid <= 4"),
    # batched CG problem with uneven phases
    "cg192": Spec("cg192", (192, 192, 192), 16, 6, 8.0, 4.0, 3,
                  sample_targets=[0.6e6, 0.9e6, 1.2e6, 1.5e6, 1.9e6, 2.4e6],
                  poisson=True, sample_lo=0.6e6, sample_hi=2.4e6,
                  description="192^3, 16 coils, 6 phases, Poisson-drawn "
                              "0.6M-2.4M samples per phase"),
    # large precision sweep
    "sweep256": Spec("sweep256", (256, 256, 256), 32, 8, 12.0, 4.0, 5,
                     sample_targets=[4.0e6] * 8,
                     description="256^3, 32 coils, 8 phases, ~4M samples per "
                                 "phase, max |d| 12"),
}


def make(spec: Spec, phases=None, coils=None):
    """Materialise a workload spec (optionally only some phases)."""
    shape = spec.shape
    x = phantom(shape, spec.seed)
    P = spec.n_phases
    phases = list(range(P)) if phases is None else list(phases)
    disp = []
    for j in phases:
        d = bump_displacement(shape, spec.seed * 1000 + 17 * j + 1, spec.max_disp)
        if spec.rigid > 0:
            t = rigid_translation(spec.seed * 1000 + 17 * j + 2, spec.rigid)
            d = (d.astype(np.float64) + t[:, None, None, None]).astype(np.float32)
        disp.append(d)
    out = {"spec": spec, "x": x, "disp": disp, "phases": phases}
    if spec.n_coils > 0:
        smaps = coil_maps(shape, spec.n_coils, spec.seed * 1000 + 500)
        if coils is not None:
            smaps = smaps[:coils]
        out["smaps"] = smaps
        beats = phase_sample_counts(spec.sample_targets, spec.readout,
                                    spec.seed * 1000 + 600, spec.poisson,
                                    spec.sample_lo, spec.sample_hi)
        total_il = INTERLEAVES_PER_HEARTBEAT * sum(beats)
        hb_total = sum(beats)
        traj = []
        start = 0
        for j in range(P):
            hbs = np.arange(start, start + beats[j])
            start += beats[j]
            # heartbeat h acquires interleaves h, h + H, h + 2H, ... of the
            # phyllotaxis ordering, so each heartbeat spans the whole sphere
            ids = (hbs[:, None] + hb_total * np.arange(INTERLEAVES_PER_HEARTBEAT)[None, :]).ravel()
            if j in phases:
                traj.append(cones_trajectory(ids.size, spec.readout,
                                             spec.seed * 1000 + 700 + j,
                                             interleave_ids=ids, n_total=total_il))
        out["coords"] = traj
    return out


def workload(name: str, phases=None, coils=None):
    return make(WORKLOADS[name], phases=phases, coils=coils)


def small_case(shape, n_coils, n_phases, samples_per_phase, seed, max_disp=2.0,
               rigid=1.0, uniform_coords=False):
    """A small seeded case for parity tests: arbitrary (even) image shape,
    any coil/phase count, and either cone-like or uniformly random samples."""
    rng = _rng(seed)
    shape = tuple(int(s) for s in shape)
    x = phantom(shape, seed, n_ellipsoids=6, smooth_vox=1.0)
    # add a little white noise so every frequency is exercised
    x = (x + 0.05 * (rng.standard_normal(shape) + 1j * rng.standard_normal(shape))
         ).astype(np.complex64)
    disp = []
    for j in range(n_phases):
        d = bump_displacement(shape, seed * 100 + j, max_disp,
                              width_range=(1.0, max(1.5, min(shape) / 4)))
        if rigid > 0:
            t = rigid_translation(seed * 100 + 50 + j, rigid)
            d = (d.astype(np.float64) + t[:, None, None, None]).astype(np.float32)
        disp.append(d)
    out = {"x": x, "disp": disp}
    if n_coils > 0:
        out["smaps"] = coil_maps(shape, n_coils, seed * 100 + 77)
        coords = []
        for j in range(n_phases):
            m = int(samples_per_phase[j] if np.ndim(samples_per_phase) else samples_per_phase)
            if uniform_coords:
                c = rng.uniform(-math.pi, math.pi, (m, 3)).astype(np.float32)
                c = np.where(c >= np.float32(math.pi), np.float32(-math.pi), c)
            else:
                readout = max(8, min(128, m))
                nil = -(-m // readout)
                c = cones_trajectory(nil, readout, seed * 100 + 90 + j)[:m]
            coords.append(np.ascontiguousarray(c, dtype=np.float32))
        out["coords"] = coords
    return out
