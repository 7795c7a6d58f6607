"""Write the FP64 oracle references of the 256^3 precision sweep.

Calls only the seeded generators (synth) and the FP64 oracle (oracle/): for
phase 0 and coils 0..3 of the 256^3, 32-coil, 8-phase workload it computes
  * the warp T_0 x on the central 64^3 crop,
  * A_0 x for coils 0..3 at a seeded 1% subset of phase 0's samples,
  * A^H y on the central 64^3 crop for y nonzero only at that subset and
    those coils (values drawn here, stored as complex64 and used by the
    oracle in FP64 exactly as stored),
and writes them, rounded to complex64, to sweep256_oracle.npz beside this
script.  Run:  python tests/golden/make_sweep256_oracle.py  (about 15 minutes
and 20 GB of host memory).
"""

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import synth  # noqa: E402
from oracle import operators as O  # noqa: E402

N_COILS = 4


def main():
    t0 = time.time()
    w = synth.workload("sweep256")
    shape = w["spec"].shape
    geo = O.Geometry(shape)
    rng = np.random.default_rng(256)
    d0 = w["disp"][0].astype(np.float64)
    crop = tuple(slice(s // 2 - 32, s // 2 + 32) for s in shape)
    M0 = w["coords"][0].shape[0]
    sub = np.sort(rng.choice(M0, M0 // 100, replace=False)).astype(np.int64)
    om = w["coords"][0][sub]
    y_sub = (rng.standard_normal((sub.size, N_COILS))
             + 1j * rng.standard_normal((sub.size, N_COILS))).astype(np.complex64)
    print(f"generated in {time.time() - t0:.0f}s", flush=True)
    m0 = O.warp_forward(geo, w["x"], d0)
    print(f"warp in {time.time() - t0:.0f}s", flush=True)
    y_ref = np.stack([O.kspace_forward(geo, w["smaps"][c] * m0, om) for c in range(N_COILS)],
                     axis=1)
    print(f"k-space forward in {time.time() - t0:.0f}s", flush=True)
    warp_crop = m0[crop].copy()
    del m0
    v = sum(np.conj(w["smaps"][c].astype(np.complex128))
            * O.kspace_adjoint(geo, y_sub[:, c].astype(np.complex128), om)
            for c in range(N_COILS))
    xa = O.warp_adjoint(geo, v, d0)
    print(f"adjoint in {time.time() - t0:.0f}s", flush=True)
    np.savez(os.path.join(HERE, "sweep256_oracle.npz"),
             sub=sub, y_sub=y_sub, n_coils=np.int64(N_COILS),
             warp_crop=warp_crop.astype(np.complex64),
             y_ref=y_ref.astype(np.complex64),
             adj_crop=xa[crop].astype(np.complex64))
    print(f"written in {time.time() - t0:.0f}s", flush=True)


if __name__ == "__main__":
    main()
