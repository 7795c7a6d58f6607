"""Shared helpers for the GPU parity tests (seeded inputs -> torch, errors)."""

import numpy as np

# FP32 operator vs FP64 oracle: relative L2 tolerance of the FP32 path.
TOL_FP32 = 1e-5
# FP32 adjointness |<Ax,y> - <x,A^H y>| / (|Ax| |y|)
TOL_ADJ = 1e-6


def rel_l2(a, b):
    a = np.asarray(a).ravel()
    b = np.asarray(b).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def to_dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def c64(a):
    return np.ascontiguousarray(np.asarray(a).astype(np.complex64))


def crandn(rng, shape):
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).astype(np.complex64)


def make_plan(case, shape, identity_warp=False, **kw):
    from paper_2501_16713_gb300 import Plan
    disp = None if identity_warp else to_dev(np.stack(case["disp"]).astype(np.float32))
    coords = [to_dev(c) for c in case["coords"]] if "coords" in case else None
    smaps = to_dev(case["smaps"]) if "smaps" in case else None
    n_phases = len(case["disp"]) if "disp" in case else len(case["coords"])
    return Plan(shape, disp=disp, coords=coords, smaps=smaps, n_phases=n_phases,
                identity_warp=identity_warp, **kw)
