"""Benchmark of the nonrigid SENSE normal operator E = sum_j A_j^H A_j.

Workload (default): 128^3 complex64 image, 8 coils, 4 respiratory phases,
~1.5M cone-like k-space samples per phase (synthetic, seeded), sigma 2, W 4.
One step = one application of E (all phases, all coils): the operator a CG
iteration applies.  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle (the only reference this method
has) on a bounded sample of the same workload and reports the same metric.
Under torchrun each rank runs an independent replica (weak scaling).
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "nonrigid-SENSE A^H.A applies/s"
UNIT = "applies/s"

# stage -> CUDA source file of its kernels (the key of the committed ncu traffic records)
STAGE_KERNEL_SOURCE = {
    "interp_kspace": "kernels_kspace.cu", "spread_kspace": "kernels_spread.cu",
    "interp_image": "kernels_image.cu", "spread_image": "spread_home.cu",
    "coil_fanout_pad": "kernels_kspace.cu", "crop_coilsum": "kernels_kspace.cu",
    "deapod_pad": "kernels_image.cu", "crop_deapod": "kernels_image.cu",
    "vector": "kernels_image.cu", "fista": "fista.cu", "fft_pruned": "fft_pruned.cu",
}
FFT_STAGES = ("fft_n", "fft_g", "fft_gc")
# kernels behind each stage name reported as the dominant kernel
DOM_KERNELS = {
    "spread_kspace": "spread_coils_cube_kernel (tensor-core sub-block spread) + split-tile "
                     "reduce_kernel",
    "interp_kspace": "interp_tma_kernel (or interp_tile_kernel)",
    "spread_image": "spread_home_kernel + home_rim_kernel (or spread_single_kernel)",
    "interp_image": "interp_image_kernel",
    "fft_pruned": "fwd_x/y/z_kernel or inv_z/y/x_kernel (one of three passes)",
}


def stage_bytes(info, shape, C, P, M):
    """Compulsory HBM bytes per E apply, per stage.

    Grids count occupied tiles only (rho = fraction of (phase, tile) pairs with
    samples); coordinates count 12 B per point (3 x f32); complex values 8 B."""
    N3 = float(shape[0] * shape[1] * shape[2])
    G3 = float(info["grid"][0] * info["grid"][1] * info["grid"][2])
    rho = info["occupied_fraction"]
    Ms = float(sum(M))
    k = 8.0 * C * rho * G3 * P + (12.0 + 8.0 * C) * Ms
    img = 8.0 * G3 + (12.0 + 8.0) * P * N3
    # own pruned coil-grid transforms (sigma 2), per coil grid and E: forward
    # reads S_c (and the phase image once per C grids), writes and re-reads
    # T1 (N0 N1 G2) and T2 (N0 G1 G2), writes the grid; the adjoint mirrors it.
    # The axis-0 passes touch only the tiles of the union over phases (fu of
    # the grid; the rest is never read forward and is zero in the adjoint) and
    # the forward one reads T2 only for tile columns holding such tiles (fc)
    G2 = float(info["grid"][2])
    G1 = float(info["grid"][1])
    fu = info.get("union_fraction", 1.0)
    fc = info.get("union_columns", 1.0)
    t1 = 8.0 * shape[0] * shape[1] * G2
    t2 = 8.0 * shape[0] * G1 * G2
    per_grid = (2.0 * (8.0 * N3 + 8.0 * N3 / max(C, 1)) + 4.0 * t1 + (3.0 + fc) * t2 +
                2.0 * 8.0 * fu * G3)
    # the method's floor for the coil-grid transforms: every one of the 2 C P
    # transforms of an E reads and writes its G^3 grid once, plus the coil
    # fan-out and combination reads and writes of the N^3 images
    floor_grid = 2.0 * 2.0 * 8.0 * G3 + 2.0 * (8.0 * N3 + 8.0 * N3 / max(C, 1))
    return {
        "fft_pruned": P * C * floor_grid,
        "fft_pruned_passes": P * C * per_grid,
        "fft_n": 2.0 * 2.0 * 8.0 * N3, "fft_g": 2.0 * 2.0 * 8.0 * G3,
        "interp_kspace": k, "spread_kspace": k,
        "interp_image": img, "spread_image": img,
        "deapod_pad": 16.0 * N3, "crop_deapod": 16.0 * N3,
        "coil_fanout_pad": P * 8.0 * (1 + 2 * C) * N3,
        "crop_coilsum": P * 8.0 * (1 + 2 * C) * N3,
    }


def source_hash(name):
    path = os.path.join(ROOT, "paper_2501_16713_gb300", "csrc", name)
    with open(path, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def ncu_traffic(stage, workload):
    """DRAM bytes per launch of `stage` from the committed ncu summary, if it
    was taken on the current source of that kernel."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
    except OSError:
        return None
    r = rec.get(workload, {}).get(stage)
    if not r or r.get("source_sha") != source_hash(STAGE_KERNEL_SOURCE[stage]):
        return None
    return r.get("dram_bytes_per_launch")


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------
# CPU oracle leg (bounded sample)
# --------------------------------------------------------------------------

class OracleSample:
    """The FP64 oracle's E apply, measured as complete oracle calls.

    E = sum_j (T_j^H T_j-side calls) + sum_j sum_c (S_c, G_j, G_j^H, S_c^H): the
    oracle runs, per phase, one warp_forward and one warp_adjoint (FFTs of N^3
    and G^3, deapodization, padding, gridding cores over the N^3 displaced
    voxels) and, per phase and coil, one coil product, one kspace_forward, one
    kspace_adjoint (FFT of G^3, deapodization, padding, gridding cores over the
    M_j samples) and one conjugate coil product.  Each piece below is one of
    those calls at full size on the workload's own data (phase 0, coil 0),
    except that the gridding cores inside the four gridding calls are timed
    apart: the call itself with its core replaced by a zero result, and the
    core on a contiguous `frac` of its points, scaled by the exact point
    count.  E is the sum of the pieces times their multiplicities (P phases,
    C coils, M_j / M_0 for the k-space cores).  Single thread (FFT workers 1)."""

    def __init__(self, w, frac=1.0 / 8, seed=0):
        import numpy as np
        from oracle import operators as O
        self.O = O
        spec = w["spec"]
        self.shape = spec.shape
        self.geo = O.Geometry(self.shape)
        self.P, self.C = len(w["disp"]), spec.n_coils
        self.M = [c.shape[0] for c in w["coords"]]
        self.frac = frac
        rng = np.random.default_rng(seed)
        cplx = lambda shp: rng.standard_normal(shp) + 1j * rng.standard_normal(shp)  # noqa: E731
        geo, N3 = self.geo, int(np.prod(self.shape))
        self.x = cplx(self.shape)
        self.d0 = w["disp"][0].astype(np.float64)
        self.om0 = w["coords"][0]
        self.s0 = w["smaps"][:1]
        self.v1 = cplx((1,) + self.shape)
        self.y1 = cplx((self.M[0], 1))
        self.ug = cplx(geo.grid)
        nv = max(1, int(N3 * frac))
        st = int(rng.integers(0, N3 - nv + 1))
        self.qi = O.warp_positions(geo, self.d0)[:, st:st + nv]
        self.wi = cplx(nv)
        self.scale_i = N3 / nv
        nk = max(1, int(self.M[0] * frac))
        stk = int(rng.integers(0, self.M[0] - nk + 1))
        self.qk = O.kspace_positions(geo, self.om0[stk:stk + nk])
        self.yk = cplx(nk)
        self.scale_k = self.M[0] / nk
        self.pieces = ["warp_forward", "interp_image_core", "warp_adjoint", "spread_image_core",
                       "kspace_forward", "interp_kspace_core", "kspace_adjoint",
                       "spread_kspace_core", "coil_products"]
        self.times = {k: [] for k in self.pieces}

    def _stubbed(self, fn):
        """Time fn() with the oracle's gridding cores returning zeros."""
        import numpy as np
        O = self.O
        bp, pc = O.backprojection_core, O.projection_core
        O.backprojection_core = lambda grid, q, width, beta: np.zeros(
            (q.shape[1],) + grid.shape[3:], dtype=np.complex128)
        O.projection_core = lambda vals, q, gs, width, beta: np.zeros(
            tuple(gs) + np.shape(vals)[1:], dtype=np.complex128)
        try:
            t = time.perf_counter()
            fn()
            return time.perf_counter() - t
        finally:
            O.backprojection_core, O.projection_core = bp, pc

    def _timed(self, fn):
        t = time.perf_counter()
        fn()
        return time.perf_counter() - t

    def run(self, i):
        """Run piece i (mod the piece count); returns its wall time (s)."""
        O, geo = self.O, self.geo
        name = self.pieces[i % len(self.pieces)]
        W, b = geo.width, geo.beta
        if name == "warp_forward":
            t = self._stubbed(lambda: O.warp_forward(geo, self.x, self.d0))
        elif name == "warp_adjoint":
            t = self._stubbed(lambda: O.warp_adjoint(geo, self.x, self.d0))
        elif name == "kspace_forward":
            t = self._stubbed(lambda: O.kspace_forward(geo, self.v1, self.om0))
        elif name == "kspace_adjoint":
            t = self._stubbed(lambda: O.kspace_adjoint(geo, self.y1, self.om0))
        elif name == "interp_image_core":
            t = self._timed(lambda: O.backprojection_core(self.ug, self.qi, W, b))
        elif name == "spread_image_core":
            t = self._timed(lambda: O.projection_core(self.wi, self.qi, geo.grid, W, b))
        elif name == "interp_kspace_core":
            t = self._timed(lambda: O.backprojection_core(self.ug, self.qk, W, b))
        elif name == "spread_kspace_core":
            t = self._timed(lambda: O.projection_core(self.yk, self.qk, geo.grid, W, b))
        else:  # one coil: S_c m and conj(S_c) v
            t = self._timed(lambda: (O.coil_forward(self.s0, self.x),
                                     O.coil_adjoint(self.s0, self.v1)))
        self.times[name].append(t)
        return t

    def estimate(self):
        """Seconds of one E apply from the mean time of every piece (pieces not
        yet measured are run here first)."""
        for k, name in enumerate(self.pieces):
            if not self.times[name]:
                self.run(k)
        m = {k: statistics.mean(v) for k, v in self.times.items()}
        t_phase = (m["warp_forward"] + m["interp_image_core"] * self.scale_i +
                   m["warp_adjoint"] + m["spread_image_core"] * self.scale_i)
        e = self.P * t_phase
        for Mj in self.M:
            r = Mj / self.M[0]
            e += self.C * (m["kspace_forward"] + m["kspace_adjoint"] + m["coil_products"] +
                           r * self.scale_k * (m["interp_kspace_core"] + m["spread_kspace_core"]))
        return e

    def describe(self):
        n = sum(len(v) for v in self.times.values())
        work = sum(sum(v) for v in self.times.values())
        return (f"FP64 numpy oracle, single thread: one E apply assembled from complete oracle "
                f"calls on the workload's phase 0 / coil 0 data at full size (warp_forward, "
                f"warp_adjoint, kspace_forward, kspace_adjoint, coil products), each timed with "
                f"its gridding core apart; the cores timed on a contiguous {self.frac:.4g} of "
                f"their points and scaled by the point counts; E = P x (T-side calls) + "
                f"sum_j C x (coil products + G-side calls, cores x M_j/M_0); {n} piece runs, "
                f"{work:.1f} s of CPU work")


def oracle_cost(w, frac=1.0 / 8, seed=0):
    """Seconds of one oracle E apply (OracleSample, every piece run once) and
    the description of the sample."""
    smp = OracleSample(w, frac=frac, seed=seed)
    for k in range(len(smp.pieces)):
        smp.run(k)
    return smp.estimate(), smp.describe()


# --------------------------------------------------------------------------
# GPU leg
# --------------------------------------------------------------------------

def max_over_ranks(value, device, world):
    """The largest `value` over all ranks (the job's time is its slowest
    rank's); the identity on a single rank."""
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(ms_max, world):
    """Whole-job applies/s of `world` replicas, each one apply per step, timed
    by the slowest rank (weak scaling)."""
    return world * 1000.0 / ms_max


def _lambda_max(plan, shape, dev, iters=20, seed=4):
    import torch
    gen = torch.Generator(device=dev).manual_seed(seed)
    v = torch.randn(shape, dtype=torch.complex64, device=dev, generator=gen)
    lam = 0.0
    for _ in range(iters):
        w = plan.normal(v, 0.0)
        lam = float(torch.linalg.norm(w) / torch.linalg.norm(v))
        v = w / torch.linalg.norm(w)
    return lam


def _noisy(plan, x, gen, snr_scale=0.03):
    import torch
    y = plan.forward(x)
    return y + snr_scale * float(y.abs().max()) * torch.randn(
        y.shape, dtype=torch.complex64, device=y.device, generator=gen)


def _timed_solve(fn):
    """Solve once to warm (graph capture), then time one solve with CUDA events."""
    import torch
    fn()
    torch.cuda.synchronize()
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    res = fn()
    e1.record(s)
    torch.cuda.synchronize()
    return res, e0.elapsed_time(e1)


CIRC_LAMBDA_FACTOR = 5.0
# recycled deflation space: Ritz vectors of the k largest Ritz values of a
# DEFL_STEPS-iteration circulant-CG run on another right-hand side (the low
# end of the circulant-preconditioned spectrum is a large cluster near
# lambda / (CIRC_LAMBDA_FACTOR lambda); the outliers sit at the top)
DEFL_STEPS = 30
DEFL_KS = (16, 24)


def cg_compare(plan, x, shape, dev, net, tol=1e-4, maxit=500, rel_lambda=1e-3, seed=5,
               train_runs=0):
    """Plain CG and flexible CG with `net` to tol on y = A x + noise,
    lambda = rel_lambda * lambda_max (power iteration); both captured as CUDA
    graphs (10 iterations per graph launch)."""
    import torch
    lam_max = _lambda_max(plan, shape, dev)
    lam = rel_lambda * lam_max
    gen = torch.Generator(device=dev).manual_seed(seed)
    y = _noisy(plan, x, gen)
    out = torch.empty(shape, dtype=torch.complex64, device=dev)
    (cg, ms_cg) = _timed_solve(lambda: plan.solve_cg(y, lam, tol=tol, maxit=maxit, graph=True,
                                                     out=out))
    x_cg = out.clone()
    (fcg, ms_f) = _timed_solve(lambda: plan.solve_fcg(y, lam, net, tol=tol, maxit=maxit,
                                                      graph=True, out=out))
    diff = float((out - x_cg).norm() / x_cg.norm())
    # circulant preconditioner (set up once per lambda: one E application,
    # timed apart), alone and followed by the network; built for
    # CIRC_LAMBDA_FACTOR x lambda (the sweep of `--workload cgsweep128`:
    # 1x 28, 2x 23, 3x 21, 5x 18, 10x 19 iterations)
    t0 = time.perf_counter()
    plan.set_circulant(CIRC_LAMBDA_FACTOR * lam)
    ms_setup = (time.perf_counter() - t0) * 1000.0
    (pc, ms_pc) = _timed_solve(lambda: plan.solve_fcg(y, lam, None, tol=tol, maxit=maxit,
                                                      graph=True, out=out, circulant=True))
    diff_pc = float((out - x_cg).norm() / x_cg.norm())
    (pcn, ms_pcn) = _timed_solve(lambda: plan.solve_fcg(y, lam, net, tol=tol, maxit=maxit,
                                                        graph=True, out=out, circulant=True))
    diff_pcn = float((out - x_cg).norm() / x_cg.norm())
    # circulant plus a deflation space recycled from an earlier solve with
    # another right-hand side (built once per operator, timed apart)
    deflated = {}
    dgen = torch.Generator(device=dev).manual_seed(seed + 200)
    y_tr = _noisy(plan, torch.randn(shape, dtype=torch.complex64, device=dev, generator=dgen), dgen)
    for k in DEFL_KS:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ritz, kept = plan.deflation_from_solve(y_tr, lam, steps=DEFL_STEPS, k=k, circulant=True,
                                               largest=True)
        torch.cuda.synchronize()
        ms_ds = (time.perf_counter() - t0) * 1000.0
        (pd, ms_pd) = _timed_solve(lambda: plan.solve_fcg(y, lam, None, tol=tol, maxit=maxit,
                                                          graph=True, out=out, circulant=True,
                                                          deflate=True))
        deflated[k] = {"iters": pd[1], "ms": round(ms_pd, 2), "true_res": pd[3],
                       "solution_rel_diff": float((out - x_cg).norm() / x_cg.norm()),
                       "setup_ms": round(ms_ds, 1), "ritz_largest": float(ritz[0]),
                       "ritz_kth": float(ritz[-1]), "kept": kept, "steps": DEFL_STEPS,
                       "speedup_vs_plain": round(ms_cg / ms_pd, 3)}
    plan.set_deflation(None)
    ms_defl = min(v["ms"] for v in deflated.values())
    # a network trained here from its random start (symmetric form, cosine
    # loss on pairs of plain-CG runs, blocks kept by the flexible-CG iterations
    # of a held-out problem), against the same network untrained
    trained = None
    if train_runs > 0:
        from paper_2501_16713_gb300 import Cnn, precond
        t0 = time.perf_counter()
        tgen = torch.Generator(device=dev).manual_seed(seed + 100)
        rhs = [_noisy(plan, torch.randn(shape, dtype=torch.complex64, device=dev,
                                        generator=tgen), tgen) for _ in range(train_runs + 1)]
        r, e, runs = precond.generate_pairs(plan, rhs[:-1], lam, tol=1e-5, maxit=maxit,
                                            per_run=40)
        tnet = Cnn(shape, seed=1)
        (fu, ms_fu) = _timed_solve(lambda: plan.solve_fcg(y, lam, tnet, tol=tol, maxit=maxit,
                                                          graph=True, out=out))
        score = lambda n_: precond.fcg_iterations(plan, rhs[-1], lam, n_)  # noqa: E731
        hist = precond.train_select(tnet, r, e, [(300, 1e-3, 3e-4), (300, 3e-4, 1e-4)], score)
        t_train = time.perf_counter() - t0
        (ft, ms_ft) = _timed_solve(lambda: plan.solve_fcg(y, lam, tnet, tol=tol, maxit=maxit,
                                                          graph=True, out=out))
        trained = {"iters": ft[1], "ms": round(ms_ft, 2), "true_res": ft[3], "fallbacks": ft[5],
                   "untrained_iters": fu[1], "untrained_ms": round(ms_fu, 2),
                   "speedup_vs_plain": round(ms_cg / ms_ft, 3),
                   "pairs": int(r.shape[0]), "pair_runs": len(runs), "train_s": round(t_train, 1),
                   "selection": [(b, sc) for b, _, sc in hist]}
        tnet.close()
        del r, e
    best = min(ms_f, ms_pc, ms_pcn, ms_defl)
    return {"tol": tol, "lambda": lam, "lambda_rel": rel_lambda, "lambda_max": lam_max,
            "plain": {"iters": cg[1], "ms": round(ms_cg, 2), "true_res": cg[3]},
            "fcg": {"iters": fcg[1], "ms": round(ms_f, 2), "true_res": fcg[3],
                    "fallbacks": fcg[5], "solution_rel_diff": diff},
            "circulant": {"iters": pc[1], "ms": round(ms_pc, 2), "true_res": pc[3],
                          "solution_rel_diff": diff_pc, "setup_ms": round(ms_setup, 2),
                          "lambda_factor": CIRC_LAMBDA_FACTOR},
            "circulant_net": {"iters": pcn[1], "ms": round(ms_pcn, 2), "true_res": pcn[3],
                              "fallbacks": pcn[5], "solution_rel_diff": diff_pcn},
            "circulant_deflated": {str(k): v for k, v in deflated.items()},
            "fcg_trained": trained, "target_speedup": 3.0,
            "speedup": round(ms_cg / best, 3), "speedup_fcg_net": round(ms_cg / ms_f, 3)}


def run_cgsweep128(args):
    """The CG preconditioning knobs on the 128^3 8-coil 4-phase problem at
    lambda = 1e-3 lambda_max, to 1e-4: the circulant preconditioner's lambda
    factor, alone and with recycled deflation spaces (Ritz vectors of the
    largest or smallest Ritz values of a circulant-CG run of `steps` iterations
    on another right-hand side, k asked / kept).  Solves as CUDA graphs, wall
    time by CUDA events, each space's setup timed apart."""
    import numpy as np
    import torch

    import synth
    from paper_2501_16713_gb300 import Plan, build

    build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    w = synth.workload("sense128")
    shape = w["spec"].shape
    plan = Plan(shape, disp=torch.from_numpy(np.stack(w["disp"])).to(dev),
                coords=[torch.from_numpy(c).to(dev) for c in w["coords"]],
                smaps=torch.from_numpy(w["smaps"]).to(dev))
    plan.autotune(reps=2)
    x = torch.from_numpy(w["x"]).to(dev)
    lam = 1e-3 * _lambda_max(plan, shape, dev)
    gen = torch.Generator(device=dev).manual_seed(5)
    y = _noisy(plan, x, gen)
    out = torch.empty(shape, dtype=torch.complex64, device=dev)
    tol, maxit = 1e-4, 500
    (cg, ms_cg) = _timed_solve(lambda: plan.solve_cg(y, lam, tol=tol, maxit=maxit, graph=True,
                                                     out=out))
    dgen = torch.Generator(device=dev).manual_seed(205)
    y_tr = _noisy(plan, torch.randn(shape, dtype=torch.complex64, device=dev, generator=dgen), dgen)
    rows = []
    for fac in (1.0, 2.0, 3.0, 5.0, 10.0):
        plan.set_circulant(fac * lam)
        (pc, ms_pc) = _timed_solve(lambda: plan.solve_fcg(y, lam, None, tol=tol, maxit=maxit,
                                                          graph=True, out=out, circulant=True))
        row = {"factor": fac, "circulant": {"iters": pc[1], "ms": round(ms_pc, 2)}, "deflated": []}
        for steps, k, largest in ((30, 16, True), (40, 24, True), (40, 32, True), (30, 8, False)):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ritz, kept = plan.deflation_from_solve(y_tr, lam, steps=steps, k=k, circulant=True,
                                                   largest=largest)
            torch.cuda.synchronize()
            setup = (time.perf_counter() - t0) * 1000.0
            (pd, ms) = _timed_solve(lambda: plan.solve_fcg(y, lam, None, tol=tol, maxit=maxit,
                                                           graph=True, out=out, circulant=True,
                                                           deflate=True))
            row["deflated"].append({"steps": steps, "k": k, "end": "largest" if largest else
                                    "smallest", "kept": kept, "iters": pd[1], "ms": round(ms, 2),
                                    "true_res": pd[3], "setup_ms": round(setup, 1),
                                    "ritz_first": float(ritz[0]), "ritz_last": float(ritz[-1]),
                                    "speedup_vs_plain": round(ms_cg / ms, 3)})
        plan.set_deflation(None)
        rows.append(row)
    plan.close()
    return {"metric": "CG wall time to 1e-4 relative residual", "value": min(
        d["ms"] for r in rows for d in r["deflated"]), "unit": "ms", "higher_is_better": False,
        "data": "synthetic", "config": {"workload": "cgsweep128", "image": list(shape),
                                        "lambda_rel": 1e-3, "tol": tol},
        "plain": {"iters": cg[1], "ms": round(ms_cg, 2)}, "sweep": rows}


def run_precond(args):
    """Learned preconditioner end to end on the 128^3 8-coil 4-phase geometry:
    training pairs from plain-CG runs on random right-hand sides, training on
    the GPU (symmetric form, cosine loss; one network from a random start, one
    from the Laplacian construction; blocks kept by flexible-CG iterations on
    a held-out problem), then plain CG vs flexible CG on the phantom data."""
    import numpy as np
    import torch

    import synth
    from paper_2501_16713_gb300 import Cnn, Plan, build, precond

    build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    w = synth.workload("sense128")
    shape = w["spec"].shape
    plan = Plan(shape, disp=torch.from_numpy(np.stack(w["disp"])).to(dev),
                coords=[torch.from_numpy(c).to(dev) for c in w["coords"]],
                smaps=torch.from_numpy(w["smaps"]).to(dev))
    x = torch.from_numpy(w["x"]).to(dev)
    lam = 1e-3 * _lambda_max(plan, shape, dev)
    gen = torch.Generator(device=dev).manual_seed(40)

    def rhs(i):
        xr = torch.randn(shape, dtype=torch.complex64, device=dev, generator=gen)
        for _ in range(i % 4):
            for ax in range(3):
                xr = 0.5 * xr + 0.25 * (torch.roll(xr, 1, ax) + torch.roll(xr, -1, ax))
        return _noisy(plan, xr, gen)

    t0 = time.perf_counter()
    rs, es, iters = [], [], []
    for i in range(args.pair_runs):
        r, e, it = precond.generate_pairs(plan, [rhs(i)], lam, tol=1e-5, maxit=500, per_run=60)
        rs.append(r[::2].clone())
        es.append(e[::2].clone())
        iters += it
        del r, e
    r = torch.cat(rs)
    e = torch.cat(es)
    del rs, es
    torch.cuda.synchronize()
    t_pairs = time.perf_counter() - t0
    y_val = rhs(1)
    score = lambda net: precond.fcg_iterations(plan, y_val, lam, net)
    blocks = [(300, 1e-3, 3e-4), (300, 3e-4, 1e-4), (300, 1e-4, 3e-5)]
    t1 = time.perf_counter()
    nets = {}
    for name in ("random_init", "laplacian_init"):
        net = Cnn(shape, seed=1)
        if name == "laplacian_init":
            net.set_params(precond.laplacian_params(args.lap_c))
        hist = precond.train_select(net, r, e, blocks, score)
        nets[name] = (net, hist)
    t_train = time.perf_counter() - t1
    res = {}
    for name, (net, hist) in nets.items():
        res[name] = {"selection": [{"block": b, "loss": (None if l != l else round(l, 4)),
                                    "val_iters": sc} for b, l, sc in hist],
                     **cg_compare(plan, x, shape, dev, net)}
    best = min(res, key=lambda k: res[k]["fcg"]["ms"])
    cmp = res[best]
    line = {"metric": "CG time to 1e-4 relative residual (flexible CG + learned preconditioner)",
            "value": cmp["fcg"]["ms"], "unit": "ms", "higher_is_better": False,
            "n_gpus": 1, "steps": 1, "warmup": 1, "ms_per_step": cmp["fcg"]["ms"],
            "scaling": "weak", "vs_baseline": None, "dtype": "c64/f32 operator, bf16 network",
            "data": "synthetic (seeded phantom, random right-hand sides for training)",
            "config": {"workload": "precond128", "image": list(shape), "coils": w["spec"].n_coils,
                       "phases": len(w["coords"]), "lambda_rel": 1e-3,
                       "pairs": int(r.shape[0]), "pair_runs": args.pair_runs,
                       "pair_run_iters": iters, "pairs_s": round(t_pairs, 1),
                       "train_s": round(t_train, 1), "blocks": blocks,
                       "network": "symmetric form z = u0 + N4^T (I + W5^T W5) N4 u0, "
                                  "5 conv 3x3x3, 2-16-16-16-16-2, BF16",
                       "laplacian_c": args.lap_c, "selected": best},
            "plain_ms": cmp["plain"]["ms"], "speedup_vs_plain": cmp["speedup"],
            "results": res}
    plan.close()
    return line


def run_cg192(args):
    """Batched CG workload: 192^3, 16 coils, 6 phases with uneven (Poisson-drawn)
    sample counts, Tikhonov lambda = 1e-3 lambda_max, 30 CG iterations captured
    in one CUDA graph; FP32 operator, FP64 inner products."""
    import numpy as np
    import torch

    import synth
    from paper_2501_16713_gb300 import Plan, build

    build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    w = synth.workload("cg192")
    shape = w["spec"].shape
    t0 = time.perf_counter()
    plan = Plan(shape, disp=torch.from_numpy(np.stack(w["disp"])).to(dev),
                coords=[torch.from_numpy(c).to(dev) for c in w["coords"]],
                smaps=torch.from_numpy(w["smaps"]).to(dev))
    t_plan = time.perf_counter() - t0
    tuning = plan.autotune(reps=3)
    info = plan.info()
    x = torch.from_numpy(w["x"]).to(dev)
    lam_max = _lambda_max(plan, shape, dev)
    lam = 1e-3 * lam_max
    gen = torch.Generator(device=dev).manual_seed(6)
    y = _noisy(plan, x, gen)
    out = torch.empty(shape, dtype=torch.complex64, device=dev)
    iters = 30
    for _ in range(max(1, args.warmup - 2)):
        plan.solve_cg(y, lam, tol=0.0, maxit=iters, graph=True, out=out)
    torch.cuda.synchronize()
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    clocks = ClockSampler(vis.split(",")[0] if vis else "0")
    clocks.start()
    time.sleep(0.3)
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = max(1, min(args.steps, 3))
    e0.record(s)
    for _ in range(reps):
        res = plan.solve_cg(y, lam, tol=0.0, maxit=iters, graph=True, out=out)
    e1.record(s)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / reps
    # one E apply alone, for applies/s
    for _ in range(2):
        plan.normal(x, lam, out)
    torch.cuda.synchronize()
    e0.record(s)
    for _ in range(5):
        plan.normal(x, lam, out)
    e1.record(s)
    torch.cuda.synchronize()
    ms_e = e0.elapsed_time(e1) / 5
    hist = res[2]
    line = {"metric": "CG: 30 iterations in one CUDA graph", "value": ms, "unit": "ms",
            "higher_is_better": False, "n_gpus": 1, "steps": reps, "warmup": args.warmup,
            "ms_per_step": ms, "scaling": "weak", "vs_baseline": None,
            "dtype": "c64/f32 operator, f64 CG scalars", "data": "synthetic",
            "config": {"workload": "cg192", "image": list(shape), "coils": w["spec"].n_coils,
                       "phases": len(plan.counts), "samples_per_phase": plan.counts,
                       "lambda": lam, "lambda_rel": 1e-3, "iterations": iters,
                       "phase_chunk": info["phase_chunk"], "plan_s": round(t_plan, 1),
                       "tuning": tuning,
                       "device_bytes": info["device_bytes"]},
            "ms_per_iteration": ms / iters, "normal_applies_per_s": 1000.0 / ms_e,
            "rel_residual_after_30": hist[-1] if hist else None,
            "residual_history": [float(f"{h:.3e}") for h in hist[::5]],
            "clocks": clk}
    plan.close()
    return line


FISTA_LEVELS = 4
FISTA_ITERS = 400     # the iteration count of the paper's wavelet-FISTA (Appendix 1)
FISTA_TAU = 1e-3      # lambda / L: threshold at 1e-3 of the unit peak image intensity
FISTA_STEP_BYTES = 48  # per voxel: read z, E0 z, b, x_{k-1}; write x_k, z_{k+1} (complex64)


def run_cnn128(args):
    """The learned preconditioner's network at 128^3 (the image of the default
    workload): one application z = N(r) of the symmetric form (10 convolutions)
    and of the plain form (5 convolutions), each with the mma.sync and the
    tcgen05 convolution kernels, timed with CUDA events around `steps`
    applications after the warm-up; the two kernels must give bitwise the same
    z.  The roofline is the tensor-core one: algorithmic FLOPs of the real
    channel counts (2 -> 16 -> 16 -> 16 -> 16 -> 2) over the measured time."""
    import torch

    from paper_2501_16713_gb300 import Cnn, build

    build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    shape = (128, 128, 128)
    nvox = shape[0] * shape[1] * shape[2]
    gen = torch.Generator(device=dev).manual_seed(8)
    r = torch.randn(shape, dtype=torch.complex64, device=dev, generator=gen)
    # MACs per voxel of one plain pass: 27 taps x (2x16 + 3 x 16x16 + 16x2)
    macs_plain = 27 * (2 * 16 + 3 * 16 * 16 + 16 * 2)
    s = torch.cuda.current_stream()
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    clocks = ClockSampler(vis.split(",")[0] if vis else "0")
    clocks.start()
    time.sleep(0.3)
    res, launches = {}, 0
    for symmetric in (True, False):
        net = Cnn(shape, seed=1, symmetric=symmetric)
        outs = {}
        for tc in (False, True):
            net.set_conv(tc)
            z = torch.empty_like(r)
            for _ in range(args.warmup):
                net.apply(r, z)
            torch.cuda.synchronize()
            l0 = net.launches()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            for _ in range(args.steps):
                net.apply(r, z)
            e1.record(s)
            torch.cuda.synchronize()
            launches += net.launches() - l0
            ms = e0.elapsed_time(e1) / args.steps
            flops = 2.0 * macs_plain * nvox * (2 if symmetric else 1)
            res[("symmetric" if symmetric else "plain", "tcgen05" if tc else "mma_sync")] = (
                ms, flops / (ms * 1e-3) / 1e12)
            outs[tc] = z.clone()
        if not torch.equal(outs[False], outs[True]):
            raise RuntimeError("tcgen05 and mma.sync convolutions differ")
        if net.device_status() != 0:
            raise RuntimeError("network kernels reported a device error")
        net.close()
    clk = clocks.stop()
    peaks, peak_kind = measured_peaks()
    peak = float(peaks["bf16_tflops"])
    best = min(res, key=lambda k: res[k][0] if k[0] == "symmetric" else 1e30)
    ms, tf = res[best]
    return {"metric": "network applications/s (symmetric form, 128^3)", "value": 1000.0 / ms,
            "unit": "applications/s", "higher_is_better": True, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16 (fp32 accumulation)", "data": "synthetic",
            "config": {"workload": "cnn128", "image": list(shape),
                       "channels": "2-16-16-16-16-2", "kernel": "3x3x3",
                       "l2": "activations 64 MB per layer at 128^3 (16 BF16 channels); no flush"},
            "ms": {f"{f}/{k}": round(v[0], 4) for (f, k), v in res.items()},
            "tflops": {f"{f}/{k}": round(v[1], 1) for (f, k), v in res.items()},
            "roofline": {"kernel": "conv3d (" + best[1] + ")", "bound": "tensor",
                         "achieved": round(tf, 1), "peak": peak, "unit": "TFLOP/s",
                         "frac": round(tf / peak, 4),
                         "peak_source": f"{peak_kind} MEASURED_PEAKS.json bf16_tflops",
                         "traffic": None},
            "gpu_launches": int(launches), "clocks": clk}


def run_fista128(args):
    """Wavelet-FISTA on the 128^3, 8-coil, 4-phase workload (the default E
    workload): 400 iterations of the fused FISTA step (gradient step, 4-level
    Haar shrinkage, momentum) around the normal operator, replayed as CUDA
    graphs of 32 iterations; lambda = 1e-3 L, L = 2.04 lambda_max (power
    iteration).  Reports iterations/s, the per-iteration split between the
    normal operator and the step kernel (from an eager 32-iteration profile)
    and the step kernel's roofline."""
    import numpy as np
    import torch

    import synth
    from paper_2501_16713_gb300 import Plan, build

    build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    w = synth.workload("sense128")
    spec = w["spec"]
    shape = spec.shape
    plan = Plan(shape, disp=torch.from_numpy(np.stack(w["disp"])).to(dev),
                coords=[torch.from_numpy(c).to(dev) for c in w["coords"]],
                smaps=torch.from_numpy(w["smaps"]).to(dev))
    tuning = plan.autotune(reps=3)
    x_true = torch.from_numpy(w["x"]).to(dev)
    gen = torch.Generator(device=dev).manual_seed(6)
    y = _noisy(plan, x_true, gen)
    L = plan.lipschitz(iters=20, seed=4)
    lam = FISTA_TAU * L
    out = torch.empty(shape, dtype=torch.complex64, device=dev)
    # warm-up: graph capture and caches
    for _ in range(max(1, args.warmup - 2)):
        plan.solve_fista(y, lam, levels=FISTA_LEVELS, L=L, maxit=64, graph=True, out=out)
    torch.cuda.synchronize()
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    clocks = ClockSampler(vis.split(",")[0] if vis else "0")
    clocks.start()
    time.sleep(0.3)
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = max(1, min(args.steps, 2))
    e0.record(s)
    for _ in range(reps):
        x, hist, _ = plan.solve_fista(y, lam, levels=FISTA_LEVELS, L=L, maxit=FISTA_ITERS,
                                      graph=True, out=out)
    e1.record(s)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / reps
    err = float(torch.linalg.norm(x - x_true) / torch.linalg.norm(x_true))
    # eager 32-iteration profile: normal operator vs the fused step kernel
    out2 = torch.empty_like(out)
    plan.profile_start(max_launches=32 * 64 + 64)
    plan.solve_fista(y, lam, levels=FISTA_LEVELS, L=L, maxit=32, graph=False, out=out2)
    stages, own = plan.profile_stop()
    f_ms, f_n = stages["fista"]
    step_ms = f_ms / max(f_n, 1)
    normal_ms = (sum(v[0] for k, v in stages.items() if k != "fista")) / 32
    nvox = int(np.prod(shape))
    step_bytes = FISTA_STEP_BYTES * nvox
    achieved = step_bytes / (step_ms * 1e-3) / 1e9
    peaks, peak_kind = measured_peaks()
    peak = float(peaks["hbm_gbs"])
    # end to end through the public API: data from pinned host memory, the
    # image back to pinned host memory
    yh = y.cpu().pin_memory()
    xh = torch.empty(shape, dtype=torch.complex64).pin_memory()
    yd = torch.empty_like(y)
    te = time.perf_counter()
    yd.copy_(yh, non_blocking=True)
    plan.solve_fista(yd, lam, levels=FISTA_LEVELS, L=L, maxit=FISTA_ITERS, graph=True, out=out)
    xh.copy_(out, non_blocking=True)
    torch.cuda.synchronize()
    e2e_ms = (time.perf_counter() - te) * 1000.0
    line = {"metric": "wavelet-FISTA iterations/s", "value": FISTA_ITERS * 1000.0 / ms,
            "unit": "iterations/s", "higher_is_better": True, "n_gpus": 1, "steps": reps,
            "warmup": args.warmup, "ms_per_step": ms, "scaling": "weak", "vs_baseline": None,
            "dtype": "c64/f32 operator and step, f64 reductions", "data": "synthetic",
            "config": {"workload": "fista128", "image": list(shape), "coils": spec.n_coils,
                       "phases": len(plan.counts), "samples_per_phase": plan.counts,
                       "iterations": FISTA_ITERS, "levels": FISTA_LEVELS,
                       "lambda_over_L": FISTA_TAU, "L": L, "graph_chunk": 32,
                       "tuning": tuning,
                       "l2": "one step = one E apply (~12 GB touched) + the step kernel; no flush"},
            "ms_per_iteration": ms / FISTA_ITERS,
            "split_ms_per_iteration": {"normal": round(normal_ms, 4), "fista_step": round(step_ms, 4)},
            "roofline": {"kernel": "fista_step", "bound": "hbm", "achieved": round(achieved, 1),
                         "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 4),
                         "peak_source": f"{peak_kind} MEASURED_PEAKS.json hbm_gbs",
                         "alg_bytes_per_launch": step_bytes, "ms_per_launch": step_ms,
                         "traffic": ncu_traffic("fista", "fista128")},
            "e2e": {"value": FISTA_ITERS * 1000.0 / e2e_ms, "unit": "iterations/s",
                    "h2d_bytes_per_step": int(yh.numel() * 8) // FISTA_ITERS,
                    "d2h_bytes_per_step": int(xh.numel() * 8) // FISTA_ITERS},
            "gpu_launches": int(own),
            "rel_error_vs_phantom": err, "last_rel_change": hist[-1],
            "clocks": clk}
    plan.close()
    return line


def run_fista_warp192(args):
    """Appendix 1 in 3D at 192^3: recover a piecewise-constant phantom p from
    q = T p (one nonrigid warp, image-space gridding, no coils) with 400
    wavelet-FISTA iterations at lambda = 1e-6; the naive inversion warps q by
    -d.  Reports iterations/s, both recovery errors and the step kernel's
    roofline (192^3: the step moves 340 MB, more than L2)."""
    import numpy as np
    import torch

    import synth
    from paper_2501_16713_gb300 import Plan, build

    build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    shape = (192, 192, 192)
    p_img = torch.from_numpy(synth.phantom(shape, 41, n_ellipsoids=20, smooth_vox=0.0)).to(dev)
    d = synth.bump_displacement(shape, 42, 6.0, width_range=(12.0, 30.0))
    plan = Plan(shape, disp=torch.from_numpy(d[None]).to(dev))
    q = plan.warp_forward(p_img)
    neg = Plan(shape, disp=torch.from_numpy((-d)[None]).to(dev))
    naive = neg.warp_forward(q[0])[0]
    neg.close()
    L = plan.lipschitz(iters=20, seed=4)
    lam = 1e-6
    out = torch.empty(shape, dtype=torch.complex64, device=dev)
    for _ in range(max(1, args.warmup - 2)):
        plan.solve_fista(q, lam, levels=FISTA_LEVELS, L=L, maxit=64, graph=True, out=out)
    torch.cuda.synchronize()
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    clocks = ClockSampler(vis.split(",")[0] if vis else "0")
    clocks.start()
    time.sleep(0.3)
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    x, hist, _ = plan.solve_fista(q, lam, levels=FISTA_LEVELS, L=L, maxit=FISTA_ITERS,
                                  graph=True, out=out)
    e1.record(s)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    nrm = float(torch.linalg.norm(p_img))
    err = float(torch.linalg.norm(x - p_img)) / nrm
    err_naive = float(torch.linalg.norm(naive - p_img)) / nrm
    out2 = torch.empty_like(out)
    plan.profile_start(max_launches=32 * 64 + 64)
    plan.solve_fista(q, lam, levels=FISTA_LEVELS, L=L, maxit=32, graph=False, out=out2)
    stages, own = plan.profile_stop()
    f_ms, f_n = stages["fista"]
    step_ms = f_ms / max(f_n, 1)
    normal_ms = (sum(v[0] for k, v in stages.items() if k != "fista")) / 32
    step_bytes = FISTA_STEP_BYTES * int(np.prod(shape))
    achieved = step_bytes / (step_ms * 1e-3) / 1e9
    peaks, peak_kind = measured_peaks()
    peak = float(peaks["hbm_gbs"])
    line = {"metric": "wavelet-FISTA iterations/s", "value": FISTA_ITERS * 1000.0 / ms,
            "unit": "iterations/s", "higher_is_better": True, "n_gpus": 1, "steps": 1,
            "warmup": args.warmup, "ms_per_step": ms, "scaling": "weak", "vs_baseline": None,
            "dtype": "c64/f32 operator and step, f64 reductions", "data": "synthetic",
            "config": {"workload": "fista_warp192", "image": list(shape), "coils": 0,
                       "phases": 1, "max_disp_vox": 6.0, "iterations": FISTA_ITERS,
                       "levels": FISTA_LEVELS, "lambda": lam, "L": L, "graph_chunk": 32,
                       "l2": "step kernel moves 340 MB per launch (> L2); no flush"},
            "ms_per_iteration": ms / FISTA_ITERS,
            "split_ms_per_iteration": {"normal": round(normal_ms, 4), "fista_step": round(step_ms, 4)},
            "roofline": {"kernel": "fista_step", "bound": "hbm", "achieved": round(achieved, 1),
                         "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 4),
                         "peak_source": f"{peak_kind} MEASURED_PEAKS.json hbm_gbs",
                         "alg_bytes_per_launch": step_bytes, "ms_per_launch": step_ms,
                         "traffic": ncu_traffic("fista", "fista_warp192")},
            "gpu_launches": int(own),
            "rel_error": {"fista": err, "naive_minus_d": err_naive},
            "last_rel_change": hist[-1], "clocks": clk}
    plan.close()
    return line


MOTION_SHAPE = (64, 64, 64)   # low-resolution iNAV
MOTION_COILS = 8
MOTION_BEATS = 256
MOTION_INTERLEAVES, MOTION_READOUT = 16, 1024


def run_motion64(args):
    """Motion capture on 256 heartbeats of a 64^3, 8-coil iNAV acquisition
    (the full low-resolution cone trajectory, 16 x 1024 samples, every
    heartbeat; images translated by four respiratory positions plus jitter):
    Pipe-Menon density compensation (10 iterations), the density-weighted
    gridding reconstruction of every heartbeat, the cross-correlation
    translations against heartbeat 0, k-means into 4 phases and the
    phase-ramp correction of all data.  One step = the whole pipeline;
    value = heartbeats/s."""
    import numpy as np
    import torch

    import synth
    from paper_2501_16713_gb300 import Plan, build, kmeans, phase_ramp, translation_xcorr

    build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    shape, C, H = MOTION_SHAPE, MOTION_COILS, MOTION_BEATS
    rng = np.random.default_rng(71)
    x = torch.from_numpy(synth.phantom(shape, 72, n_ellipsoids=20)).to(dev)
    smaps = torch.from_numpy(synth.coil_maps(shape, C, 73)).to(dev)
    om = torch.from_numpy(synth.cones_trajectory(MOTION_INTERLEAVES, MOTION_READOUT, 74)).to(dev)
    M = int(om.shape[0])
    plan = Plan(shape, coords=[om], smaps=smaps, n_phases=1, identity_warp=True)
    tuning = plan.autotune(reps=3)
    info = plan.info()
    phase_of = np.arange(H) % 4
    t = np.zeros((H, 3))
    t[:, 0] = np.array([0.0, 1.5, 3.0, 4.5])[phase_of] + 0.2 * rng.standard_normal(H)
    t[:, 1:] = 0.2 * rng.standard_normal((H, 2))
    y_ref = plan.forward(x)
    big = torch.cat([om] * H).contiguous()
    off = np.arange(H + 1) * M
    y0 = y_ref.repeat(H, 1).contiguous()
    phase_ramp(big, y0, off, -t)
    y0 += 0.01 * float(y_ref.abs().max()) * torch.randn(
        y0.shape, dtype=torch.complex64, device=dev, generator=torch.Generator(device=dev).manual_seed(75))
    recon = torch.empty((H,) + shape, dtype=torch.complex64, device=dev)

    def pipeline(y):
        w = plan.dcf(0, iters=10)
        for h in range(H):
            plan.adjoint_weighted(y[h * M:(h + 1) * M], w, out=recon[h])
        est = translation_xcorr(recon[0], recon)          # synchronises
        labels, _, _, _, ref = kmeans(est, 4)
        phase_ramp(big, y, off, est)                      # synchronises
        return est, labels, ref

    for _ in range(max(1, args.warmup - 2)):
        pipeline(y0.clone())
    torch.cuda.synchronize()
    ys = [y0.clone() for _ in range(2)]
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    clocks = ClockSampler(vis.split(",")[0] if vis else "0")
    clocks.start()
    time.sleep(0.3)
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    plan.profile_start(max_launches=2 * H * 64 + 4096)
    e0.record(s)
    for y in ys:
        est, labels, ref = pipeline(y)
    e1.record(s)
    torch.cuda.synchronize()
    stages, own = plan.profile_stop()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / len(ys)
    err = float(np.abs(est - (t - t[0])).max())
    phases_ok = all(len(set(labels[phase_of == j])) == 1 for j in range(4)) and len(set(labels)) == 4
    sb = stage_bytes(info, shape, C, 1, [M])
    own_stages = {k: v for k, v in stages.items() if k not in FFT_STAGES and v[1] > 0}
    dom = max(own_stages, key=lambda k: own_stages[k][0])
    dom_ms, dom_n = own_stages[dom]
    # the adjoint-side stages run once per reconstruction; the DCF adds one
    # single-channel spread and interpolation per iteration (not counted in sb)
    achieved = (sb.get(dom, 0.0) * H * len(ys)) / (dom_ms * 1e-3) / 1e9 if dom in sb else None
    peaks, peak_kind = measured_peaks()
    peak = float(peaks["hbm_gbs"])
    line = {"metric": "motion-capture heartbeats/s", "value": H * 1000.0 / ms,
            "unit": "heartbeats/s", "higher_is_better": True, "n_gpus": 1, "steps": len(ys),
            "warmup": args.warmup, "ms_per_step": ms, "scaling": "weak", "vs_baseline": None,
            "dtype": "c64/f32 gridding and FFTs, f64 shifts and k-means", "data": "synthetic",
            "config": {"workload": "motion64", "image": list(shape), "coils": C,
                       "heartbeats": H, "samples_per_heartbeat": M, "dcf_iterations": 10,
                       "phases": 4, "tuning": tuning},
            "ms_per_heartbeat": ms / H,
            "breakdown": {k: {"ms_per_step": round(v[0] / len(ys), 3),
                              "launches_per_step": v[1] / len(ys)}
                          for k, v in stages.items() if v[1] > 0},
            "roofline": {"kernel": dom, "bound": "hbm",
                         "achieved": round(achieved, 1) if achieved else None, "peak": peak,
                         "unit": "GB/s", "frac": round(achieved / peak, 4) if achieved else None,
                         "peak_source": f"{peak_kind} MEASURED_PEAKS.json hbm_gbs",
                         "traffic": None},
            "gpu_launches": int(own),
            "translation_error_max_vox": err, "phases_recovered": phases_ok,
            "clocks": clk}
    plan.close()
    return line


def run_sweep256(args):
    """Precision sweep on the 256^3, 32-coil, 8-phase workload (4 M samples per
    phase): for FP32, BF16 storage and compensated FP32 spreading, E applies/s
    and the error against the FP64 oracle.  The oracle references (phase 0,
    coils 0..3: the warp T_0 x on the central 64^3 crop, A_0 x at a seeded 1%
    subset of phase 0's samples, A^H y on the crop for y nonzero only on that
    subset) were written by tests/golden/make_sweep256_oracle.py; the full
    32-coil 8-phase FP64 operator does not fit a bench run.  Adjointness is
    measured on the full GPU operator with random x, y."""
    import numpy as np
    import torch

    import synth
    from paper_2501_16713_gb300 import Plan, build

    build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    t0 = time.perf_counter()
    w = synth.workload("sweep256")
    spec = w["spec"]
    shape = spec.shape
    t_gen = time.perf_counter() - t0
    ref = np.load(os.path.join(ROOT, "tests", "golden", "sweep256_oracle.npz"))
    sub, y_sub, n_ref_coils = ref["sub"], ref["y_sub"], int(ref["n_coils"])
    m0c, y_ref, xa_refc = ref["warp_crop"], ref["y_ref"], ref["adj_crop"]
    crop = tuple(slice(s_ // 2 - 32, s_ // 2 + 32) for s_ in shape)
    M0 = w["coords"][0].shape[0]

    x = torch.from_numpy(w["x"]).to(dev)
    variants = {}
    names = {0: "fp32", 1: "bf16_store", 2: "fp32_compensated"}
    for precision in (0, 1, 2):
        t1 = time.perf_counter()
        try:
            plan = Plan(shape, disp=torch.from_numpy(np.stack(w["disp"])).to(dev),
                        coords=[torch.from_numpy(c).to(dev) for c in w["coords"]],
                        smaps=torch.from_numpy(w["smaps"]).to(dev), precision=precision)
        except Exception as ex:  # record and go on with the other variants
            variants[names[precision]] = {"error": str(ex)}
            torch.cuda.empty_cache()
            continue
        t_plan = time.perf_counter() - t1
        info = plan.info()
        out = torch.empty_like(x)
        for _ in range(2):
            plan.normal(x, 0.0, out)
        torch.cuda.synchronize()
        s = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 3
        e0.record(s)
        for _ in range(reps):
            plan.normal(x, 0.0, out)
        e1.record(s)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        m = plan.warp_forward(x)[0][crop].cpu().numpy()
        e_warp = float(np.linalg.norm(m - m0c) / np.linalg.norm(m0c))
        y = plan.forward(x)
        y0 = plan.phase_slice(y, 0)[torch.from_numpy(sub).to(dev), :n_ref_coils].cpu().numpy()
        e_fwd = float(np.linalg.norm(y0 - y_ref) / np.linalg.norm(y_ref))
        yin = torch.zeros_like(y)
        rows = torch.from_numpy(sub).to(dev) + int(plan.offsets[0])
        yin[rows, :n_ref_coils] = torch.from_numpy(y_sub).to(dev)
        xa = plan.adjoint(yin)[crop].cpu().numpy()
        e_adj = float(np.linalg.norm(xa - xa_refc) / np.linalg.norm(xa_refc))
        gen = torch.Generator(device=dev).manual_seed(7)
        xr = torch.randn(shape, dtype=torch.complex64, device=dev, generator=gen)
        yr = torch.randn(y.shape, dtype=torch.complex64, device=dev, generator=gen)
        d = lambda a: a.flatten().to(torch.complex128)
        Ax, Ahy = plan.forward(xr), plan.adjoint(yr)
        adj = abs(complex(torch.vdot(d(yr), d(Ax)) - torch.vdot(d(Ahy), d(xr)))) / float(
            torch.linalg.norm(d(Ax)) * torch.linalg.norm(d(yr)))
        variants[names[precision]] = {
            "normal_ms": round(ms, 2), "normal_applies_per_s": 1000.0 / ms,
            "err_warp_crop64": e_warp, "err_forward_subset": e_fwd, "err_adjoint_crop64": e_adj,
            "adjointness": adj, "plan_s": round(t_plan, 1), "phase_chunk": info["phase_chunk"],
            "device_bytes": info["device_bytes"]}
        del y, yin, Ax, Ahy, yr, out
        plan.close()
        torch.cuda.empty_cache()
    base = variants["fp32"].get("normal_ms")
    for v_ in variants.values():
        if base and "normal_ms" in v_:
            v_["speedup_vs_fp32"] = round(base / v_["normal_ms"], 3)
    line = {"metric": "precision sweep: E applies/s and error vs FP64 oracle per variant",
            "value": variants["fp32"].get("normal_applies_per_s"), "unit": "applies/s",
            "higher_is_better": True, "n_gpus": 1, "steps": 3, "warmup": 2,
            "ms_per_step": base, "scaling": "weak", "vs_baseline": None,
            "dtype": "c64/f32 (bf16 grid storage in one variant)", "data": "synthetic",
            "config": {"workload": "sweep256", "image": list(shape), "coils": spec.n_coils,
                       "phases": len(w["coords"]), "samples_per_phase": M0,
                       "oracle": f"phase 0, coils 0..{n_ref_coils - 1}; 64^3 centre crop; "
                                 f"{sub.size} samples (1%); stored complex64 "
                                 "(tests/golden/sweep256_oracle.npz)",
                       "generate_s": round(t_gen, 1)},
            "variants": variants}
    return line


def run_gpu(args, rank, world, local_rank):
    import numpy as np
    import torch
    import torch.distributed as dist

    import synth
    from paper_2501_16713_gb300 import Plan, build

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if rank == 0:
        build()
    if world > 1:
        dist.barrier()
    build()
    w = synth.workload(args.workload,
                       phases=None if args.phases is None else list(range(args.phases)))
    spec = w["spec"]
    shape = spec.shape
    disp = torch.from_numpy(np.stack(w["disp"])).to(dev)
    smaps = torch.from_numpy(w["smaps"]).to(dev)
    coords = [torch.from_numpy(c).to(dev) for c in w["coords"]]
    plan = Plan(shape, disp=disp, coords=coords, smaps=smaps, osf=args.osf, width=args.width)
    del disp, smaps, coords
    tuning = plan.autotune(reps=3)  # launch choices, timed on this plan (untimed region)
    info = plan.info()
    x = torch.from_numpy(w["x"]).to(dev)
    out = torch.empty_like(x)
    stream = torch.cuda.current_stream()

    for _ in range(args.warmup):
        plan.normal(x, args.lam, out)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()

    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    clocks = ClockSampler(vis.split(",")[local_rank] if vis else str(local_rank))
    clocks.start()
    time.sleep(0.3)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    plan.profile_start(max_launches=args.steps * 64 + 64)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    e0.record(stream)
    for _ in range(args.steps):
        plan.normal(x, args.lam, out)
    e1.record(stream)
    torch.cuda.synchronize()
    stages, own = plan.profile_stop()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    ms_max = max_over_ranks(ms, dev, world)

    # forward / adjoint split (untimed region; context only)
    y = plan.forward(x)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(3):
        plan.forward(x, y)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_fwd = e0.elapsed_time(e1) / 3
    e0.record(stream)
    for _ in range(3):
        plan.adjoint(y, out)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_adj = e0.elapsed_time(e1) / 3
    del y

    # CG to 1e-4 relative residual: plain vs flexible CG (Laplacian-initialised
    # symmetric network, untrained); outside the timed region
    cg = None
    if world == 1 and not args.no_cg:
        from paper_2501_16713_gb300 import Cnn, precond
        net = Cnn(shape)
        net.set_params(precond.laplacian_params(args.lap_c))
        cg = cg_compare(plan, x, shape, dev, net, train_runs=8)
        cg["network"] = (f"fcg: symmetric form, Laplacian construction c={args.lap_c}, untrained; "
                         "fcg_trained: the same form trained from random weights on the pairs of "
                         "8 plain-CG runs (bench.py --workload precond128 trains on 70)")
        net.close()

    # end to end through the public API with host buffers
    xh = torch.from_numpy(w["x"]).pin_memory()
    oh = torch.empty(shape, dtype=torch.complex64).pin_memory()
    xd = torch.empty_like(x)
    for _ in range(2):
        xd.copy_(xh, non_blocking=True)
        plan.normal(xd, args.lam, out)
        oh.copy_(out, non_blocking=True)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ke = max(3, args.steps // 2)
    # every step copies its input from pinned host memory and its result back
    # to pinned host memory (one host buffer per step), as a streaming caller
    # would: the copies run on a copy stream, overlapped with the previous or
    # next step's E on the compute stream, device buffers double-buffered and
    # ordered by events; the host clock spans all steps and one final wait
    ohs = [torch.empty(shape, dtype=torch.complex64).pin_memory() for _ in range(ke)]
    cs = torch.cuda.Stream()
    comp = torch.cuda.current_stream()
    xds = [torch.empty_like(x) for _ in range(2)]
    outs = [torch.empty_like(x) for _ in range(2)]
    ev_in = [torch.cuda.Event() for _ in range(2)]    # input b landed
    ev_done = [torch.cuda.Event() for _ in range(2)]  # E of buffer b finished
    ev_out = [torch.cuda.Event() for _ in range(2)]   # result b copied out
    torch.cuda.synchronize()
    te = time.perf_counter()
    with torch.cuda.stream(cs):
        xds[0].copy_(xh, non_blocking=True)
        ev_in[0].record(cs)
    for k in range(ke):
        b = k % 2
        comp.wait_event(ev_in[b])
        if k >= 2:
            comp.wait_event(ev_out[b])  # outs[b] was copied out
        plan.normal(xds[b], args.lam, outs[b])
        ev_done[b].record(comp)
        with torch.cuda.stream(cs):
            if k + 1 < ke:
                if k >= 1:
                    cs.wait_event(ev_done[1 - b])  # xds[1 - b] is free again
                xds[1 - b].copy_(xh, non_blocking=True)
                ev_in[1 - b].record(cs)
            cs.wait_event(ev_done[b])
            ohs[k].copy_(outs[b], non_blocking=True)
            ev_out[b].record(cs)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks((time.perf_counter() - te) * 1000.0 / ke, dev, world)
    # the streamed results are the operator's: the last one, read on the host,
    # equals a direct application to the same image bit for bit
    ref = plan.normal(x, args.lam)
    torch.cuda.synchronize()
    if not torch.equal(ohs[-1], ref.cpu()):
        raise RuntimeError("end-to-end result differs from the direct application")

    M = plan.counts
    sb = stage_bytes(info, shape, spec.n_coils, len(M), M)
    # the dominant kernel: the stage with the largest time per kernel (the
    # pruned transforms run three passes per stage launch, the home-tile image
    # spread a spread and a rim kernel; the split-tile reductions of the
    # halo-list spreads are a small second kernel and stay in their stage's time)
    img_kernels = 2 if tuning.get("spread_image_warp") == 2 else 1
    kernels_per = {"fft_pruned": 3, "spread_image": img_kernels}
    own_stages = {k: v for k, v in stages.items() if k not in FFT_STAGES and v[1] > 0}
    dom = max(own_stages, key=lambda k: own_stages[k][0] / kernels_per.get(k, 1))
    dom_ms, dom_n = own_stages[dom]
    per_step_launches = dom_n / args.steps
    bytes_per_launch = sb.get(dom, 0.0) / per_step_launches
    achieved = bytes_per_launch / (dom_ms / dom_n * 1e-3) / 1e9
    peaks, peak_kind = measured_peaks()
    peak = float(peaks["hbm_gbs"])
    traffic = ncu_traffic(dom, args.workload)
    # the whole E: algorithmic bytes of every stage that ran (cuFFT's image-space
    # transforms at their read + write floor) over the device time of an E
    e_bytes = sum(sb[k] for k, v in stages.items() if v[1] > 0 and k in sb)
    e_achieved = e_bytes / (ms_max * 1e-3) / 1e9
    fft_ms = sum(stages[k][0] for k in FFT_STAGES) / args.steps
    breakdown = {k: {"ms_per_step": round(v[0] / args.steps, 4),
                     "launches_per_step": v[1] / args.steps,
                     "gbs": (round(sb[k] / (v[0] / args.steps * 1e-3) / 1e9, 1)
                             if k in sb and v[0] > 0 else None)}
                 for k, v in stages.items() if v[1] > 0}
    result = {
        "metric": METRIC, "value": job_throughput(ms_max, world), "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "c64/f32 (FP32 arithmetic)",
        "data": "synthetic (seeded phantom, Gaussian-bump displacements, Gaussian coil "
                "maps, cone-like trajectory); no trained weights",
        "config": {"workload": args.workload, "image": list(shape), "coils": spec.n_coils,
                   "phases": len(M), "samples_per_phase": M, "osf": args.osf,
                   "kb_width": args.width, "grid": info["grid"],
                   "lambda": args.lam, "parallelism": f"replicas x{world}",
                   "tuning": tuning,
                   "l2": "inputs larger than L2: per-phase coil grids 1.07 GB, "
                         "E touches ~12 GB per step; no flush"},
        "roofline": {"kernel": dom, "bound": "hbm", "achieved": round(achieved, 1),
                     "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 4),
                     "peak_source": f"{peak_kind} MEASURED_PEAKS.json hbm_gbs"
                     if peak_kind == "measured" else "fallback 6.8 TB/s",
                     "alg_bytes_per_launch": bytes_per_launch,
                     "ms_per_launch": dom_ms / dom_n,
                     "kernels": DOM_KERNELS.get(dom, dom),
                     "traffic": traffic},
        "e_roofline": {"bound": "hbm", "alg_bytes_per_apply": e_bytes,
                       "achieved": round(e_achieved, 1), "peak": peak, "unit": "GB/s",
                       "frac": round(e_achieved / peak, 4),
                       "note": "every stage of one E apply (gridding per the method's data "
                               "flow, coil-grid and image-space transforms at their read + "
                               "write floor) over the device time of the apply"},
        "e2e": {"value": job_throughput(e2e_ms, world), "unit": UNIT,
                "h2d_bytes_per_step": int(xh.numel() * 8),
                "d2h_bytes_per_step": int(oh.numel() * 8),
                "note": "per step: the image copied from pinned host memory, E through "
                        "nrsense_apply_normal, the result copied to pinned host memory; the "
                        "copies on a second stream overlapped with the neighbouring steps' E "
                        "(double-buffered, event-ordered); host clock around all steps and "
                        "one wait"},
        "gpu_launches": int(own),
        "fft_ms_per_step": round(fft_ms, 3),
        "forward_ms": round(ms_fwd, 3), "adjoint_ms": round(ms_adj, 3),
        "breakdown": breakdown,
        "clocks": clk,
        "cg": cg,
    }
    plan.close()
    return result, w


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="sense128")
    ap.add_argument("--lam", type=float, default=0.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--phases", type=int, default=None,
                    help="use only the first K phases (a smaller case for profiling)")
    ap.add_argument("--no-cg", action="store_true", help="skip the CG comparison")
    ap.add_argument("--osf", type=float, default=2.0,
                    help="oversampling sigma (rational: G = sigma N per axis must be whole)")
    ap.add_argument("--width", type=int, default=4, help="kernel width W (4 or 6)")
    ap.add_argument("--lap-c", type=float, default=30.0)
    ap.add_argument("--pair-runs", type=int, default=70)
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    special = {"precond128": run_precond, "cgsweep128": run_cgsweep128, "cg192": run_cg192,
               "sweep256": run_sweep256,
               "fista128": run_fista128, "fista_warp192": run_fista_warp192,
               "motion64": run_motion64, "cnn128": run_cnn128}
    if args.workload in special and args.impl == "ours":
        if int(os.environ.get("RANK", "0")) == 0:
            print(json.dumps(special[args.workload](args)), flush=True)
        return

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        # the oracle on the host cores; rank 0 only
        if rank != 0:
            return
        if args.workload in ("precond128", "cgsweep128", "fista_warp192", "motion64", "cnn128"):
            print(json.dumps({"impl": "reference", "unavailable":
                              f"the {args.workload} workload has no CPU reference arm"}))
            return
        import synth
        metric, unit = METRIC, UNIT
        w = synth.workload("sense128" if args.workload == "fista128" else args.workload)
        smp = OracleSample(w)
        extra = None
        if args.workload == "fista128":
            # one FISTA iteration: an E apply plus the FP64 Haar proximal step
            metric, unit = "wavelet-FISTA iterations/s", "iterations/s"
            from oracle import fista as OF
            import numpy as np
            rng = np.random.default_rng(3)
            v = rng.standard_normal(w["spec"].shape) + 1j * rng.standard_normal(w["spec"].shape)
            extra = lambda: OF.prox_wavelet_l1(v, 0.1, FISTA_LEVELS)  # noqa: E731
            smp.pieces.append("fista_prox")
            smp.times["fista_prox"] = []
        n_pieces = len(smp.pieces)

        def step(k):
            if smp.pieces[k % n_pieces] == "fista_prox":
                t = time.perf_counter()
                extra()
                dt = time.perf_counter() - t
                smp.times["fista_prox"].append(dt)
                return dt
            return smp.run(k)

        for k in range(args.warmup):  # untimed; each step runs the next piece
            step(k)
        for name in smp.pieces:
            smp.times[name] = []
        t0 = time.perf_counter()
        for k in range(args.steps):
            step(k)
        wall = time.perf_counter() - t0
        for k, name in enumerate(smp.pieces):  # pieces the timed steps did not reach
            if not smp.times[name]:
                step(k)
        e_s = smp.estimate() + (statistics.mean(smp.times["fista_prox"]) if extra else 0.0)
        v = 1.0 / e_s
        desc = (smp.describe() + f"; each bench step ran one piece in turn ({n_pieces} pieces"
                + (", the last the Haar proximal step" if extra else "") + ")")
        line = {"impl": "reference", "metric": metric, "value": v, "unit": unit,
                "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": wall * 1000.0 / max(args.steps, 1), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": args.workload},
                "seconds_per_apply": e_s,
                "cpu_baseline": {"value": v, "unit": unit, "cores": 1, "kind": "oracle",
                                 "sample": desc},
                "e2e": {"value": v, "unit": unit, "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return

    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    result, w = run_gpu(args, rank, world, local_rank)
    if rank == 0:
        if world == 1 and not args.no_cpu_baseline:
            e, desc = oracle_cost(w)
            result["cpu_baseline"] = {"value": 1.0 / e, "unit": UNIT, "cores": 1,
                                      "kind": "oracle", "sample": desc}
        else:
            result["cpu_baseline"] = None
        print(json.dumps(result), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
