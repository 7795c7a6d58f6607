// Operator application: the process diagrams of the paper as sequences of
// cuFFT calls and the library's kernels, all on the caller's stream.
//
//  T_j   (image-space gridding, forward):  F_N -> K1 (1/C*, Z) -> F_G^H -> K2 (B_j^(i))
//        The first three steps do not depend on j and run once for all phases.
//  T^H   (adjoint, summed over phases):    K3 (P_j^(i), all phases into one
//        grid) -> F_G -> K4 (Z^H, 1/C) -> F_N^H
//  G_j S (per phase):                       K5 (S, 1/c*, Z) -> F_G (C coils
//        batched) -> K6 (B^(k))
//  S^H G_j^H (per phase):                   K7 (P^(k), into a buffer whose
//        empty tiles stay zero) -> F_G^H (batched, out of place) ->
//        K8 (Z^H, 1/c, S^H)
#include <cufftXt.h>

#include <algorithm>
#include <cstring>

#include "plan_internal.h"

using namespace nrs;

namespace {

#define NRS_TRY(expr)                  \
  do {                                 \
    nrsense_status _st = (expr);       \
    if (_st != NRSENSE_OK) return _st; \
  } while (0)

nrsense_status fft(nrsense_plan_s* p, int stage, cufftHandle h, cudaStream_t s, void* in,
                   void* out, int dir, int nph = 0) {
  StageMark mark(p, stage, s);
  if (cufftSetStream(h, s) != CUFFT_SUCCESS) return NRSENSE_ERR_CUFFT;
  if (stage == NRSENSE_STAGE_FFT_GC && p->grid_bf16) {
    // BF16 coil grids: cufftXt plans of fewer than 2^31 elements, run as
    // consecutive full sub-batches over the nph * C grids
    const long long total = (long long)nph * p->C;
    const long long sub = bf16_sub_batch(total, p->geo.ngrid);  // as at plan time
    if (sub < 1) return NRSENSE_ERR_CUFFT;
    const size_t step = size_t(sub) * size_t(p->geo.ngrid) * 4;  // bytes of sub grids
    for (long long k = 0; k < total; k += sub) {
      char* i = static_cast<char*>(in) + size_t(k / sub) * step;
      char* o = static_cast<char*>(out) + size_t(k / sub) * step;
      if (cufftXtExec(h, i, o, dir) != CUFFT_SUCCESS) return NRSENSE_ERR_CUFFT;
    }
    return NRSENSE_OK;
  }
  const cufftResult r =
      cufftExecC2C(h, static_cast<cufftComplex*>(in), static_cast<cufftComplex*>(out), dir);
  return r == CUFFT_SUCCESS ? NRSENSE_OK : NRSENSE_ERR_CUFFT;
}

nrsense_status launched() {
  return cudaGetLastError() == cudaSuccess ? NRSENSE_OK : NRSENSE_ERR_CUDA;
}

// Launch one stage of the library's kernels: event marks when profiling, and
// the launch count.
#define STAGE(stage, call)                          \
  do {                                              \
    StageMark _mark(p, NRSENSE_STAGE_##stage, s);   \
    p->launches += (call);                          \
  } while (0)

cufftHandle gc_plan(nrsense_plan_s* p, int nph) {
  for (auto& fp : p->fft_gc_plans)
    if (fp.first == nph) return fp.second;
  return 0;
}

// Phase table of phases [j0, j1) of the k-space point sets; value/output rows
// of phase j start at off_j - row_base.
PhaseTable kspace_table(const nrsense_plan_s* p, int j0, int j1, bool spread, long long row_base) {
  PhaseTable t;
  std::memset(&t, 0, sizeof(t));
  t.nphase = j1 - j0;
  int ai = 0, ar = 0, as = 0;
  for (int jj = 0; jj < t.nphase; ++jj) {
    const PointSet& ps = p->kpts[j0 + jj];
    t.qs[jj] = ps.qs;
    t.perm[jj] = ps.perm;
    t.list[jj] = ps.list;
    t.bins[jj] = ps.bins;
    t.items[jj] = spread ? ps.items : ps.iitems;
    t.reduces[jj] = ps.reduces;
    t.row0[jj] = p->off[j0 + jj] - row_base;
    t.item0[jj] = ai;
    ai += spread ? ps.n_items : ps.n_iitems;
    t.red0[jj] = ar;
    ar += spread ? ps.n_reduces : 0;
    t.slot0[jj] = as;
    as += ps.n_slots;
  }
  t.item0[t.nphase] = ai;
  t.red0[t.nphase] = ar;
  return t;
}

PhaseTable image_table(const nrsense_plan_s* p) {
  PhaseTable t;
  std::memset(&t, 0, sizeof(t));
  const PointSet& ps = p->ipts;
  t.nphase = 1;
  t.qs[0] = ps.qs;
  t.perm[0] = ps.perm;
  t.list[0] = ps.list;
  t.bins[0] = ps.bins;
  t.items[0] = ps.items;
  t.reduces[0] = ps.reduces;
  t.item0[1] = ps.n_items;
  t.red0[1] = ps.n_reduces;
  return t;
}

// m (P x nvox) = T_j x for all phases
nrsense_status warp_forward(nrsense_plan_s* p, const nrsense_c64* x, nrsense_c64* m,
                            cudaStream_t s) {
  const Geo& g = p->geo;
  if (p->identity_warp) {
    STAGE(VECTOR, launch_copy_phases(g, p->P, x, m, s));
    return launched();
  }
  NRS_TRY(fft(p, NRSENSE_STAGE_FFT_N, p->fft_n, s, const_cast<nrsense_c64*>(x), p->b_xhat, CUFFT_FORWARD));
  STAGE(DEAPOD_PAD, launch_deapod_pad(g, p->deapod, p->b_xhat, p->b_upad, s));
  NRS_TRY(launched());
  NRS_TRY(fft(p, NRSENSE_STAGE_FFT_G, p->fft_g, s, p->b_upad, p->b_ugrid, CUFFT_INVERSE));
  STAGE(INTERP_IMAGE, launch_interp_image(g, p->W, p->kc, p->P, p->disp, p->b_ugrid, m, s));
  return launched();
}

// x = sum_j T_j^H m_j
nrsense_status warp_adjoint(nrsense_plan_s* p, const nrsense_c64* m, nrsense_c64* x,
                            cudaStream_t s) {
  const Geo& g = p->geo;
  if (p->identity_warp) {
    STAGE(VECTOR, launch_sum_phases(g, p->P, m, x, s));
    return launched();
  }
  const PhaseTable t = image_table(p);
  STAGE(SPREAD_IMAGE, launch_spread(g, p->W, p->kc, 1, p->itiles, t, m, p->b_ugrid, false,
                                    p->comp_spread, p->spread_variant, p->b_scratch, p->d_status, s));
  NRS_TRY(launched());
  NRS_TRY(fft(p, NRSENSE_STAGE_FFT_G, p->fft_g, s, p->b_ugrid, p->b_ugrid, CUFFT_FORWARD));
  STAGE(CROP_DEAPOD, launch_crop_deapod(g, p->deapod, p->b_ugrid, x, s));
  NRS_TRY(launched());
  return fft(p, NRSENSE_STAGE_FFT_N, p->fft_n, s, x, x, CUFFT_INVERSE);
}

// y rows of phases [j0, j1) (row off_j - row_base of y) = G_j S m_j, where m
// holds the chunk's warped images consecutively.
nrsense_status sense_chunk_forward(nrsense_plan_s* p, int j0, int j1, const nrsense_c64* m,
                                   nrsense_c64* y, long long row_base, cudaStream_t s) {
  const Geo& g = p->geo;
  const int nph = j1 - j0;
  STAGE(COIL_FANOUT, launch_coil_fanout_pad(g, p->C, nph, p->deapod, p->smaps, m, p->b_xpad,
                                            p->grid_bf16, s));
  NRS_TRY(launched());
  NRS_TRY(fft(p, NRSENSE_STAGE_FFT_GC, gc_plan(p, nph), s, p->b_xpad, p->b_xwork, CUFFT_FORWARD,
              nph));
  const PhaseTable t = kspace_table(p, j0, j1, /*spread=*/false, row_base);
  STAGE(INTERP_KSPACE, launch_interp_kspace(g, p->W, p->kc, p->C, p->ktiles, t, p->b_xwork,
                                            p->grid_bf16, y, p->interp_coils, s));
  return launched();
}

// w (nph x nvox) = S^H G_j^H y_j for phases [j0, j1)
nrsense_status sense_chunk_adjoint(nrsense_plan_s* p, int j0, int j1, const nrsense_c64* y,
                                   long long row_base, nrsense_c64* w, cudaStream_t s) {
  const Geo& g = p->geo;
  const int nph = j1 - j0;
  const PhaseTable t = kspace_table(p, j0, j1, /*spread=*/true, row_base);
  STAGE(SPREAD_KSPACE, launch_spread(g, p->W, p->kc, p->C, p->ktiles, t, y, p->b_xspread,
                                     p->grid_bf16, p->comp_spread, p->spread_variant, p->b_scratch, p->d_status, s));
  NRS_TRY(launched());
  NRS_TRY(fft(p, NRSENSE_STAGE_FFT_GC, gc_plan(p, nph), s, p->b_xspread, p->b_xwork, CUFFT_INVERSE,
              nph));
  STAGE(CROP_COILSUM, launch_crop_coilsum(g, p->C, nph, p->deapod, p->smaps, p->b_xwork,
                                          p->grid_bf16, w, s));
  return launched();
}

}  // namespace

extern "C" {

nrsense_status nrsense_warp_forward(nrsense_plan_t p, const nrsense_c64* x, nrsense_c64* m,
                                    void* stream) {
  if (p == nullptr || x == nullptr || m == nullptr) return NRSENSE_ERR_ARG;
  return warp_forward(p, x, m, static_cast<cudaStream_t>(stream));
}

nrsense_status nrsense_warp_adjoint(nrsense_plan_t p, const nrsense_c64* m, nrsense_c64* x,
                                    void* stream) {
  if (p == nullptr || x == nullptr || m == nullptr) return NRSENSE_ERR_ARG;
  return warp_adjoint(p, m, x, static_cast<cudaStream_t>(stream));
}

nrsense_status nrsense_kspace_forward(nrsense_plan_t p, int32_t phase, const nrsense_c64* v,
                                      nrsense_c64* y, void* stream) {
  if (p == nullptr || v == nullptr || y == nullptr) return NRSENSE_ERR_ARG;
  if (p->C == 0) return NRSENSE_ERR_STATE;
  if (phase < 0 || phase >= p->P) return NRSENSE_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  STAGE(COIL_FANOUT, launch_image_to_padded(p->geo, p->C, p->deapod, v, p->b_xpad, p->grid_bf16, s));
  NRS_TRY(launched());
  NRS_TRY(fft(p, NRSENSE_STAGE_FFT_GC, gc_plan(p, 1), s, p->b_xpad, p->b_xwork, CUFFT_FORWARD, 1));
  const PhaseTable t = kspace_table(p, phase, phase + 1, false, p->off[phase]);
  STAGE(INTERP_KSPACE, launch_interp_kspace(p->geo, p->W, p->kc, p->C, p->ktiles, t, p->b_xwork,
                                            p->grid_bf16, y, p->interp_coils, s));
  return launched();
}

nrsense_status nrsense_kspace_adjoint(nrsense_plan_t p, int32_t phase, const nrsense_c64* y,
                                      nrsense_c64* v, void* stream) {
  if (p == nullptr || v == nullptr || y == nullptr) return NRSENSE_ERR_ARG;
  if (p->C == 0) return NRSENSE_ERR_STATE;
  if (phase < 0 || phase >= p->P) return NRSENSE_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const PhaseTable t = kspace_table(p, phase, phase + 1, true, p->off[phase]);
  STAGE(SPREAD_KSPACE, launch_spread(p->geo, p->W, p->kc, p->C, p->ktiles, t, y, p->b_xspread,
                                     p->grid_bf16, p->comp_spread, p->spread_variant, p->b_scratch, p->d_status, s));
  NRS_TRY(launched());
  NRS_TRY(fft(p, NRSENSE_STAGE_FFT_GC, gc_plan(p, 1), s, p->b_xspread, p->b_xwork, CUFFT_INVERSE, 1));
  STAGE(CROP_COILSUM, launch_crop_to_coils(p->geo, p->C, p->deapod, p->b_xwork, p->grid_bf16, v, s));
  return launched();
}

nrsense_status nrsense_apply_forward(nrsense_plan_t p, const nrsense_c64* x, nrsense_c64* y,
                                     void* stream) {
  if (p == nullptr || x == nullptr || y == nullptr) return NRSENSE_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (p->C == 0) return warp_forward(p, x, y, s);
  NRS_TRY(warp_forward(p, x, p->b_m, s));
  for (int j0 = 0; j0 < p->P; j0 += p->phase_chunk) {
    const int j1 = std::min(p->P, j0 + p->phase_chunk);
    NRS_TRY(sense_chunk_forward(p, j0, j1, p->b_m + (long long)j0 * p->geo.nvox, y, 0, s));
  }
  return NRSENSE_OK;
}

nrsense_status nrsense_apply_adjoint(nrsense_plan_t p, const nrsense_c64* y, nrsense_c64* x,
                                     void* stream) {
  if (p == nullptr || x == nullptr || y == nullptr) return NRSENSE_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (p->C == 0) return warp_adjoint(p, y, x, s);
  for (int j0 = 0; j0 < p->P; j0 += p->phase_chunk) {
    const int j1 = std::min(p->P, j0 + p->phase_chunk);
    NRS_TRY(sense_chunk_adjoint(p, j0, j1, y, 0, p->b_m + (long long)j0 * p->geo.nvox, s));
  }
  return warp_adjoint(p, p->b_m, x, s);
}

nrsense_status nrsense_apply_normal(nrsense_plan_t p, const nrsense_c64* x, double lambda,
                                    nrsense_c64* out, void* stream) {
  if (p == nullptr || x == nullptr || out == nullptr || x == out) return NRSENSE_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  NRS_TRY(warp_forward(p, x, p->b_m, s));
  if (p->C > 0) {
    for (int j0 = 0; j0 < p->P; j0 += p->phase_chunk) {
      const int j1 = std::min(p->P, j0 + p->phase_chunk);
      nrsense_c64* mj = p->b_m + (long long)j0 * p->geo.nvox;
      NRS_TRY(sense_chunk_forward(p, j0, j1, mj, p->b_y, 0, s));
      NRS_TRY(sense_chunk_adjoint(p, j0, j1, p->b_y, 0, mj, s));
    }
  }
  NRS_TRY(warp_adjoint(p, p->b_m, out, s));
  if (lambda != 0.0) {
    STAGE(VECTOR, launch_axpby(p->geo.nvox, x, float(lambda), out, 1.0f, s));
    NRS_TRY(launched());
  }
  return NRSENSE_OK;
}

nrsense_status nrsense_plan_set_tuning(nrsense_plan_t p, const nrsense_tuning* t) {
  if (p == nullptr || t == nullptr) return NRSENSE_ERR_ARG;
  if (t->spread_variant != NRSENSE_TUNE_SPREAD_REGISTER &&
      t->spread_variant != NRSENSE_TUNE_SPREAD_SHARED)
    return NRSENSE_ERR_ARG;
  if (t->interp_coils != 4 && t->interp_coils != 8) return NRSENSE_ERR_ARG;
  p->spread_variant = t->spread_variant == NRSENSE_TUNE_SPREAD_REGISTER ? kSpreadRegister
                                                                         : kSpreadShared;
  p->interp_coils = t->interp_coils;
  return NRSENSE_OK;
}

nrsense_status nrsense_plan_autotune(nrsense_plan_t p, int32_t reps, nrsense_tuning* out,
                                     void* stream) {
  if (p == nullptr || out == nullptr || reps < 1 || reps > 100) return NRSENSE_ERR_ARG;
  std::memset(out, 0, sizeof(*out));
  out->spread_variant = p->spread_variant == kSpreadRegister ? NRSENSE_TUNE_SPREAD_REGISTER
                                                             : NRSENSE_TUNE_SPREAD_SHARED;
  out->interp_coils = p->interp_coils;
  if (p->C == 0) return NRSENSE_OK;  // nothing to choose without k space
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const Geo& g = p->geo;
  const int j1 = std::min(p->P, p->phase_chunk);
  const PhaseTable ts = kspace_table(p, 0, j1, true, 0);
  const PhaseTable ti = kspace_table(p, 0, j1, false, 0);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return NRSENSE_ERR_CUDA;
  // times the candidates on the plan's own point sets and internal buffers
  // (their contents are overwritten by every application)
  auto time_ms = [&](auto&& launch) -> double {
    launch();
    cudaEventRecord(e0, s);
    for (int r = 0; r < reps; ++r) launch();
    cudaEventRecord(e1, s);
    float ms = -1.f;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
      return -1.0;
    return double(ms) / reps;
  };
  const int variants[2] = {kSpreadRegister, kSpreadShared};
  for (int k = 0; k < 2; ++k)
    out->spread_ms[k] = time_ms([&] {
      p->launches += launch_spread(g, p->W, p->kc, p->C, p->ktiles, ts, p->b_y, p->b_xspread,
                                   p->grid_bf16, p->comp_spread, variants[k], p->b_scratch,
                                   p->d_status, s);
    });
  const int chunks[2] = {8, 4};
  for (int k = 0; k < 2; ++k)
    out->interp_ms[k] = time_ms([&] {
      p->launches += launch_interp_kspace(g, p->W, p->kc, p->C, p->ktiles, ti, p->b_xwork,
                                          p->grid_bf16, p->b_y, chunks[k], s);
    });
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (cudaGetLastError() != cudaSuccess) return NRSENSE_ERR_CUDA;
  for (int k = 0; k < 2; ++k)
    if (!(out->spread_ms[k] >= 0.0) || !(out->interp_ms[k] >= 0.0)) return NRSENSE_ERR_CUDA;
  // the compensated variant has only the shared-memory kernel: keep the default there
  if (!p->comp_spread)
    p->spread_variant = out->spread_ms[1] < out->spread_ms[0] ? kSpreadShared : kSpreadRegister;
  p->interp_coils = out->interp_ms[1] < out->interp_ms[0] ? 4 : 8;
  out->spread_variant = p->spread_variant == kSpreadRegister ? NRSENSE_TUNE_SPREAD_REGISTER
                                                             : NRSENSE_TUNE_SPREAD_SHARED;
  out->interp_coils = p->interp_coils;
  return NRSENSE_OK;
}

}  // extern "C"
