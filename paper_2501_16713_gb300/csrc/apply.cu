// Operator application: the process diagrams of the paper as sequences of
// cuFFT calls and the library's kernels, all on the caller's stream.
//
//  T_j   (image-space gridding, forward):  F_N -> K1 (1/C*, Z) -> F_G^H -> K2 (B_j^(i))
//        The first three steps do not depend on j and run once for all phases.
//  T^H   (adjoint, summed over phases):    K3 (P_j^(i), all phases into one
//        grid) -> F_G -> K4 (Z^H, 1/C) -> F_N^H
//  G_j S (per phase):                       K5 (S, 1/c*, Z) -> F_G (C coils,
//        pruned to the zero padding) -> K6 (B^(k))
//  S^H G_j^H (per phase):                   K7 (P^(k), into a buffer whose
//        empty tiles stay zero) -> F_G^H (pruned to the cropped planes, out
//        of place) -> K8 (Z^H, 1/c, S^H)
#include <cufftXt.h>

#include <algorithm>
#include <cstring>

#include "plan_internal.h"

using namespace nrs;

namespace {

// image-space spread variant <-> nrsense_tuning.spread_image_warp (0 CTA per
// tile, 1 CTA per plane pair, 2 home tiles)
int image_variant_of(int tuning) {
  return tuning == 2 ? kSpreadHome : tuning == 1 ? kSpreadRegisterWarp : kSpreadShared;
}
int image_tuning_of(int variant) {
  return variant == kSpreadHome ? 2 : variant == kSpreadRegisterWarp ? 1 : 0;
}

// The phase sum of this plan's motion states is complete only with the other
// ranks' states: hand the image to the caller's reduction (an all-reduce)
nrsense_status reduce_phases(nrsense_plan_s* p, nrsense_c64* img, cudaStream_t s) {
  if (p->reduce_fn == nullptr) return NRSENSE_OK;
  const nrsense_status st = p->reduce_fn(p->reduce_user, img, p->geo.nvox, s);
  return st == NRSENSE_OK ? NRSENSE_OK : NRSENSE_ERR_CUDA;
}

#define NRS_TRY(expr)                  \
  do {                                 \
    nrsense_status _st = (expr);       \
    if (_st != NRSENSE_OK) return _st; \
  } while (0)

nrsense_status fft(nrsense_plan_s* p, int stage, cufftHandle h, cudaStream_t s, void* in,
                   void* out, int dir) {
  StageMark mark(p, stage, s);
  if (cufftSetStream(h, s) != CUFFT_SUCCESS) return NRSENSE_ERR_CUFFT;
  const cufftResult r =
      cufftExecC2C(h, static_cast<cufftComplex*>(in), static_cast<cufftComplex*>(out), dir);
  return r == CUFFT_SUCCESS ? NRSENSE_OK : NRSENSE_ERR_CUFFT;
}

// F_G (dir forward) or F_G^H (dir inverse) of nph * C consecutive coil grids,
// pruned to the zero padding.  In every grid only the centred n0 z planes,
// [0, n0/2) and [G0 - n0/2, G0), can hold data on the way in (forward) or are
// read on the way out (inverse, before the crop); across consecutive grids
// these planes form blocks of n0 contiguous planes.  Forward: 2D transforms
// of those blocks from `in` into b_xmid (whose other planes stay zero), then
// the strided 1D transform along z of every grid into `out`.  Inverse: the 1D
// transforms along z from `in` into `out`, then the 2D transforms of the
// blocks in place.  Each output equals the full 3D transform on the planes
// that are used.
nrsense_status fft_gc(nrsense_plan_s* p, int nph, void* in, void* out, int dir, cudaStream_t s) {
  StageMark mark(p, NRSENSE_STAGE_FFT_GC, s);
  const Geo& g = p->geo;
  const size_t esz = p->grid_bf16 ? 4 : 8;
  const size_t plane = size_t(g.g1) * g.g2 * esz;
  const size_t grid = size_t(g.g0) * plane;
  const long long n = (long long)nph * p->C;
  const int half = g.n0 / 2;
  for (cufftHandle h : {p->fft_p2, p->fft_p2h, p->fft_z})
    if (cufftSetStream(h, s) != CUFFT_SUCCESS) return NRSENSE_ERR_CUFFT;
  auto exec = [&](cufftHandle h, char* a, char* b) {
    const cufftResult r = p->grid_bf16 ? cufftXtExec(h, a, b, dir)
                                       : cufftExecC2C(h, reinterpret_cast<cufftComplex*>(a),
                                                      reinterpret_cast<cufftComplex*>(b), dir);
    return r == CUFFT_SUCCESS;
  };
  auto blocks = [&](char* a, char* b) {
    if (!exec(p->fft_p2h, a, b)) return false;  // grid 0, planes [0, n0/2)
    for (long long k = 1; k < n; ++k) {         // top of grid k-1 and bottom of grid k
      const size_t off = size_t(k) * grid - size_t(half) * plane;
      if (!exec(p->fft_p2, a + off, b + off)) return false;
    }
    const size_t last = size_t(n) * grid - size_t(half) * plane;  // top of the last grid
    return exec(p->fft_p2h, a + last, b + last);
  };
  char* ci = static_cast<char*>(in);
  char* co = static_cast<char*>(out);
  char* mid = static_cast<char*>(p->b_xmid);
  if (dir == CUFFT_FORWARD) {
    if (!blocks(ci, mid)) return NRSENSE_ERR_CUFFT;
    for (long long k = 0; k < n; ++k)
      if (!exec(p->fft_z, mid + size_t(k) * grid, co + size_t(k) * grid)) return NRSENSE_ERR_CUFFT;
  } else {
    for (long long k = 0; k < n; ++k)
      if (!exec(p->fft_z, ci + size_t(k) * grid, co + size_t(k) * grid)) return NRSENSE_ERR_CUFFT;
    if (!blocks(co, co)) return NRSENSE_ERR_CUFFT;
  }
  return NRSENSE_OK;
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

// tensor map for the TMA-staged interpolation, or null for the per-value staging
const CUtensorMap* interp_tmap(const nrsense_plan_s* p) {
  if (!p->interp_tma || !p->tma_ok || p->W != 4) return nullptr;
  if (p->interp_coils == 2) return &p->tmap_xwork2;
  return (p->interp_coils == 8 && p->C > 4) ? &p->tmap_xwork8 : &p->tmap_xwork4;
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
    t.clist[jj] = ps.clist;
    t.cbins[jj] = ps.cbins;
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

// The G^3 half of T: u = F_G^-1 of the deapodized, zero-padded spectrum in
// b_xhat, into b_ugrid.
nrsense_status image_grid_forward(nrsense_plan_s* p, cudaStream_t s) {
  const Geo& g = p->geo;
  if (p->image_fft_pruned) {
    nrsense_c64* t1 = p->b_upad;
    nrsense_c64* t2 = p->b_upad + (long long)g.n0 * g.n1 * g.g2;
    STAGE(FFT_G, launch_pruned_image_forward(g, p->deapod, p->b_xhat, t1, t2, p->b_ugrid, s));
    p->upad_dirty = true;
    return launched();
  }
  if (p->upad_dirty) {
    if (cudaMemsetAsync(p->b_upad, 0, size_t(g.ngrid) * sizeof(nrsense_c64), s) != cudaSuccess)
      return NRSENSE_ERR_CUDA;
    p->upad_dirty = false;
  }
  STAGE(DEAPOD_PAD, launch_deapod_pad(g, p->deapod, p->b_xhat, p->b_upad, s));
  NRS_TRY(launched());
  return fft(p, NRSENSE_STAGE_FFT_G, p->fft_g, s, p->b_upad, p->b_ugrid, CUFFT_INVERSE);
}

// The G^3 half of T^H: xhat = deapodized crop of F_G of the spread grid in
// b_ugrid (which the cuFFT path overwrites).
nrsense_status image_grid_adjoint(nrsense_plan_s* p, nrsense_c64* xhat, cudaStream_t s) {
  const Geo& g = p->geo;
  if (p->image_fft_pruned) {
    nrsense_c64* t1 = p->b_upad;
    nrsense_c64* t2 = p->b_upad + (long long)g.n0 * g.n1 * g.g2;
    STAGE(FFT_G, launch_pruned_image_adjoint(g, p->deapod, p->b_ugrid, t2, t1, xhat, s));
    p->upad_dirty = true;
    return launched();
  }
  NRS_TRY(fft(p, NRSENSE_STAGE_FFT_G, p->fft_g, s, p->b_ugrid, p->b_ugrid, CUFFT_FORWARD));
  STAGE(CROP_DEAPOD, launch_crop_deapod(g, p->deapod, p->b_ugrid, xhat, s));
  return launched();
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
  NRS_TRY(image_grid_forward(p, s));
  if (p->interp_home && p->home_ok) {
    STAGE(INTERP_IMAGE, launch_interp_home(g, p->kc, p->ihome, p->b_ugrid, m, s));
  } else {
    STAGE(INTERP_IMAGE, launch_interp_image(g, p->W, p->kc, p->P, p->disp, p->b_ugrid, m, s));
  }
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
  if (p->spread_image_variant == kSpreadHome && p->home_ok) {
    STAGE(SPREAD_IMAGE, launch_spread_home(g, p->kc, p->ihome, m, p->b_ugrid, p->home_scratch, s));
  } else {
    const PhaseTable t = image_table(p);
    STAGE(SPREAD_IMAGE, launch_spread(g, p->W, p->kc, 1, p->itiles, t, m, p->b_ugrid, false,
                                      p->comp_spread, p->spread_image_variant, p->b_scratch,
                                      p->d_status, s));
  }
  NRS_TRY(launched());
  NRS_TRY(image_grid_adjoint(p, x, s));
  return fft(p, NRSENSE_STAGE_FFT_N, p->fft_n, s, x, x, CUFFT_INVERSE);
}

// The cuFFT forward path reads the zero padding of b_xpad and b_xmid; the
// pruned transforms keep their intermediates there, so re-zero after them.
nrsense_status clean_pads(nrsense_plan_s* p, cudaStream_t s) {
  if (!p->pad_dirty) return NRSENSE_OK;
  const size_t cgb = size_t(p->geo.ngrid) * p->C * p->phase_chunk * (p->grid_bf16 ? 4 : 8);
  if (cudaMemsetAsync(p->b_xpad, 0, cgb, s) != cudaSuccess ||
      cudaMemsetAsync(p->b_xmid, 0, cgb, s) != cudaSuccess)
    return NRSENSE_ERR_CUDA;
  p->pad_dirty = false;
  return NRSENSE_OK;
}

// y rows of phases [j0, j1) (row off_j - row_base of y) = G_j S m_j, where m
// holds the chunk's warped images consecutively.
nrsense_status sense_chunk_forward(nrsense_plan_s* p, int j0, int j1, const nrsense_c64* m,
                                   nrsense_c64* y, long long row_base, cudaStream_t s) {
  const Geo& g = p->geo;
  const int nph = j1 - j0;
  if (p->fft_pruned) {
    STAGE(FFT_PRUNED, launch_pruned_forward(g, p->C, nph, p->kcolmask, p->deapod, p->smaps, m, p->b_xpad,
                                            p->b_xmid, p->b_xwork, s));
    p->pad_dirty = true;
    NRS_TRY(launched());
  } else {
    NRS_TRY(clean_pads(p, s));
    STAGE(COIL_FANOUT, launch_coil_fanout_pad(g, p->C, nph, p->deapod, p->smaps, m, p->b_xpad,
                                              p->grid_bf16, s));
    NRS_TRY(launched());
    NRS_TRY(fft_gc(p, nph, p->b_xpad, p->b_xwork, CUFFT_FORWARD, s));
  }
  const PhaseTable t = kspace_table(p, j0, j1, /*spread=*/false, row_base);
  STAGE(INTERP_KSPACE, launch_interp_kspace(g, p->W, p->kc, p->C, p->ktiles, t, p->b_xwork,
                                            p->grid_bf16, y, p->interp_coils, interp_tmap(p), p->d_status, s,
                                            p->tma_poll_limit));
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
  if (p->fft_pruned) {
    STAGE(FFT_PRUNED, launch_pruned_inverse(g, p->C, nph, p->kcolmask, p->deapod, p->smaps, p->b_xspread,
                                            p->b_xmid, p->b_xpad, w, s));
    p->pad_dirty = true;
    return launched();
  }
  NRS_TRY(fft_gc(p, nph, p->b_xspread, p->b_xwork, CUFFT_INVERSE, s));
  STAGE(CROP_COILSUM, launch_crop_coilsum(g, p->C, nph, p->deapod, p->smaps, p->b_xwork,
                                          p->grid_bf16, w, s));
  return launched();
}

}  // namespace

namespace nrs {
PhaseTable kspace_phase_table(const nrsense_plan_s* p, int phase, bool spread) {
  return kspace_table(p, phase, phase + 1, spread, p->off[phase]);
}
}  // namespace nrs

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
  NRS_TRY(clean_pads(p, s));
  STAGE(COIL_FANOUT, launch_image_to_padded(p->geo, p->C, p->deapod, v, p->b_xpad, p->grid_bf16, s));
  NRS_TRY(launched());
  NRS_TRY(fft_gc(p, 1, p->b_xpad, p->b_xwork, CUFFT_FORWARD, s));
  const PhaseTable t = kspace_table(p, phase, phase + 1, false, p->off[phase]);
  STAGE(INTERP_KSPACE, launch_interp_kspace(p->geo, p->W, p->kc, p->C, p->ktiles, t, p->b_xwork,
                                            p->grid_bf16, y, p->interp_coils, interp_tmap(p), p->d_status, s,
                                            p->tma_poll_limit));
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
  NRS_TRY(fft_gc(p, 1, p->b_xspread, p->b_xwork, CUFFT_INVERSE, s));
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
  if (p->C == 0) {
    NRS_TRY(warp_adjoint(p, y, x, s));
    return reduce_phases(p, x, s);
  }
  for (int j0 = 0; j0 < p->P; j0 += p->phase_chunk) {
    const int j1 = std::min(p->P, j0 + p->phase_chunk);
    NRS_TRY(sense_chunk_adjoint(p, j0, j1, y, 0, p->b_m + (long long)j0 * p->geo.nvox, s));
  }
  NRS_TRY(warp_adjoint(p, p->b_m, x, s));
  return reduce_phases(p, x, s);
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
  NRS_TRY(reduce_phases(p, out, s));
  if (lambda != 0.0) {
    STAGE(VECTOR, launch_axpby(p->geo.nvox, x, float(lambda), out, 1.0f, s));
    NRS_TRY(launched());
  }
  return NRSENSE_OK;
}

nrsense_status nrsense_plan_set_tuning(nrsense_plan_t p, const nrsense_tuning* t) {
  if (p == nullptr || t == nullptr) return NRSENSE_ERR_ARG;
  // every field is checked before any is applied: a rejected call leaves the
  // plan's choices as they were
  if (t->spread_variant != NRSENSE_TUNE_SPREAD_REGISTER &&
      t->spread_variant != NRSENSE_TUNE_SPREAD_SHARED &&
      t->spread_variant != NRSENSE_TUNE_SPREAD_REGISTER_WARP &&
      t->spread_variant != NRSENSE_TUNE_SPREAD_MMA)
    return NRSENSE_ERR_ARG;
  if (t->interp_coils != 2 && t->interp_coils != 4 && t->interp_coils != 8) return NRSENSE_ERR_ARG;
  if (t->interp_tma != 0 && t->interp_tma != 1) return NRSENSE_ERR_ARG;
  if (t->spread_mma_cube != 0 && t->spread_mma_cube != 1) return NRSENSE_ERR_ARG;
  if (t->spread_image_warp < 0 || t->spread_image_warp > 2) return NRSENSE_ERR_ARG;
  if (t->spread_image_warp == 2 && !p->home_ok) return NRSENSE_ERR_ARG;
  if (t->interp_image_home != 0 && t->interp_image_home != 1) return NRSENSE_ERR_ARG;
  if (t->interp_image_home == 1 && !p->home_ok) return NRSENSE_ERR_ARG;
  if (t->fft_pruned != 0 && t->fft_pruned != 1) return NRSENSE_ERR_ARG;
  if (t->fft_pruned == 1 && !p->fft_pruned_ok) return NRSENSE_ERR_ARG;
  const int m = t->spread_max_item;
  if (m != 0 && m != 512 && m != 1024 && m != 2048) return NRSENSE_ERR_ARG;
  if (t->image_fft_pruned != 0 && t->image_fft_pruned != 1) return NRSENSE_ERR_ARG;
  if (t->image_fft_pruned == 1 && !p->image_fft_ok) return NRSENSE_ERR_ARG;
  // the one step that can fail for want of memory comes first
  if (m != 0) NRS_TRY(retile_kspace(p, m, nullptr));
  p->spread_variant = t->spread_variant == NRSENSE_TUNE_SPREAD_REGISTER   ? kSpreadRegister
                      : t->spread_variant == NRSENSE_TUNE_SPREAD_SHARED ? kSpreadShared
                      : t->spread_variant == NRSENSE_TUNE_SPREAD_MMA
                          ? spread_mma_variant(t->spread_mma_wpc == 2 || t->spread_mma_wpc == 4
                                                   ? t->spread_mma_wpc
                                                   : 1,
                                               t->spread_mma_cube == 1)
                          : kSpreadRegisterWarp;
  p->interp_coils = t->interp_coils;
  p->interp_tma = t->interp_tma == 1 && p->tma_ok;
  p->interp_home = t->interp_image_home == 1;
  p->spread_image_variant = image_variant_of(t->spread_image_warp);
  p->fft_pruned = t->fft_pruned == 1;
  p->image_fft_pruned = t->image_fft_pruned == 1;
  p->epoch += 1;
  return NRSENSE_OK;
}

nrsense_status nrsense_plan_autotune(nrsense_plan_t p, int32_t reps, nrsense_tuning* out,
                                     void* stream) {
  if (p) p->epoch += 1;  // choices and (re-tiled) buffers change below
  if (p == nullptr || out == nullptr || reps < 1 || reps > 100) return NRSENSE_ERR_ARG;
  std::memset(out, 0, sizeof(*out));
  out->spread_variant = p->spread_variant == kSpreadRegister ? NRSENSE_TUNE_SPREAD_REGISTER
                        : p->spread_variant == kSpreadShared ? NRSENSE_TUNE_SPREAD_SHARED
                        : spread_base(p->spread_variant) == kSpreadMMA ? NRSENSE_TUNE_SPREAD_MMA
                                                             : NRSENSE_TUNE_SPREAD_REGISTER_WARP;
  out->interp_coils = p->interp_coils;
  out->interp_tma = p->interp_tma ? 1 : 0;
  out->spread_image_warp = image_tuning_of(p->spread_image_variant);
  out->spread_image_ms[2] = -1.0;
  out->interp_image_home = p->interp_home ? 1 : 0;
  out->interp_image_ms[0] = out->interp_image_ms[1] = -1.0;
  out->spread_max_item = p->spread_max_item;
  for (int k = 0; k < 3; ++k) out->spread_item_ms[k] = -1.0;
  out->fft_pruned = p->fft_pruned ? 1 : 0;
  out->fft_ms[0] = out->fft_ms[1] = -1.0;
  out->image_fft_pruned = p->image_fft_pruned ? 1 : 0;
  out->image_fft_ms[0] = out->image_fft_ms[1] = -1.0;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const Geo& g = p->geo;
  if (!p->identity_warp && p->ipts.tp.t0 == 16) {
    // image-space spread: CTA per tile or per plane pair, timed on the plan's
    // displaced voxels (values: the internal warped-image buffer)
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess)
      return NRSENSE_ERR_CUDA;
    const PhaseTable tim = image_table(p);
    const int iv[3] = {kSpreadShared, kSpreadRegisterWarp, kSpreadHome};
    for (int k = 0; k < 3; ++k) {
      if (iv[k] == kSpreadHome && !p->home_ok) break;
      auto run = [&] {
        if (iv[k] == kSpreadHome)
          p->launches += launch_spread_home(g, p->kc, p->ihome, p->b_m, p->b_ugrid,
                                            p->home_scratch, s);
        else
          p->launches += launch_spread(g, p->W, p->kc, 1, p->itiles, tim, p->b_m, p->b_ugrid,
                                       false, p->comp_spread, iv[k], p->b_scratch, p->d_status, s);
      };
      run();
      cudaEventRecord(a, s);
      for (int r = 0; r < reps; ++r) run();
      cudaEventRecord(b, s);
      float ms = -1.f;
      if (cudaEventSynchronize(b) != cudaSuccess || cudaEventElapsedTime(&ms, a, b) != cudaSuccess) {
        cudaEventDestroy(a);
        cudaEventDestroy(b);
        return NRSENSE_ERR_CUDA;
      }
      out->spread_image_ms[k] = double(ms) / reps;
    }
    // image-space interpolation: thread per voxel, or super-tiles staged in
    // shared memory (input: the plan's upsampled-image buffer)
    for (int k = 0; k < 2 && (k == 0 || p->home_ok); ++k) {
      auto run = [&] {
        if (k == 1)
          p->launches += launch_interp_home(g, p->kc, p->ihome, p->b_ugrid, p->b_m, s);
        else
          p->launches += launch_interp_image(g, p->W, p->kc, p->P, p->disp, p->b_ugrid, p->b_m, s);
      };
      run();
      cudaEventRecord(a, s);
      for (int r = 0; r < reps; ++r) run();
      cudaEventRecord(b, s);
      float ms = -1.f;
      if (cudaEventSynchronize(b) != cudaSuccess || cudaEventElapsedTime(&ms, a, b) != cudaSuccess) {
        cudaEventDestroy(a);
        cudaEventDestroy(b);
        return NRSENSE_ERR_CUDA;
      }
      out->interp_image_ms[k] = double(ms) / reps;
    }
    p->interp_home = out->interp_image_ms[1] >= 0.0 &&
                     out->interp_image_ms[1] < out->interp_image_ms[0];
    out->interp_image_home = p->interp_home ? 1 : 0;
    // image-space G^3 transforms with their deapodization, forward and
    // adjoint: cuFFT path vs the pruned passes (inputs: the plan's buffers)
    for (int k = 0; k < 2 && p->image_fft_ok; ++k) {
      p->image_fft_pruned = k == 1;
      nrsense_status st = NRSENSE_OK;
      auto run = [&] {
        if (st == NRSENSE_OK) st = image_grid_forward(p, s);
        if (st == NRSENSE_OK) st = image_grid_adjoint(p, p->b_tmp, s);
      };
      run();
      cudaEventRecord(a, s);
      for (int r = 0; r < reps; ++r) run();
      cudaEventRecord(b, s);
      float ms = -1.f;
      if (st != NRSENSE_OK || cudaEventSynchronize(b) != cudaSuccess ||
          cudaEventElapsedTime(&ms, a, b) != cudaSuccess) {
        cudaEventDestroy(a);
        cudaEventDestroy(b);
        return st != NRSENSE_OK ? st : NRSENSE_ERR_CUDA;
      }
      out->image_fft_ms[k] = double(ms) / reps;
    }
    p->image_fft_pruned = p->image_fft_ok && out->image_fft_ms[1] >= 0.0 &&
                          out->image_fft_ms[1] < out->image_fft_ms[0];
    out->image_fft_pruned = p->image_fft_pruned ? 1 : 0;
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    int bi = out->spread_image_ms[1] < out->spread_image_ms[0] ? 1 : 0;
    if (out->spread_image_ms[2] >= 0.0 && out->spread_image_ms[2] < out->spread_image_ms[bi]) bi = 2;
    p->spread_image_variant = iv[bi];
    out->spread_image_warp = image_tuning_of(p->spread_image_variant);
  }
  if (p->C == 0) return NRSENSE_OK;  // nothing more to choose without k space
  const int j1 = std::min(p->P, p->phase_chunk);
  const PhaseTable ts = kspace_table(p, 0, j1, true, 0);
  const PhaseTable ti = kspace_table(p, 0, j1, false, 0);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  struct EventPair {
    cudaEvent_t &a, &b;
    ~EventPair() {
      if (a) cudaEventDestroy(a);
      if (b) cudaEventDestroy(b);
    }
  } event_guard{e0, e1};
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
  const int variants[3] = {kSpreadRegister, kSpreadShared, kSpreadRegisterWarp};
  for (int k = 0; k < 3; ++k)
    out->spread_ms[k] = time_ms([&] {
      p->launches += launch_spread(g, p->W, p->kc, p->C, p->ktiles, ts, p->b_y, p->b_xspread,
                                   p->grid_bf16, p->comp_spread, variants[k], p->b_scratch,
                                   p->d_status, s);
    });
  const bool mma_ok = p->W == 4 && p->C > 4 && !p->comp_spread;
  out->spread_mma_ms = -1.0;
  out->spread_mma_wpc = 0;
  out->spread_mma_cube = 0;
  out->spread_mma_geo_ms[0] = out->spread_mma_geo_ms[1] = -1.0;
  if (mma_ok) {
    const int wpcs[3] = {1, 2, 4};
    for (int cube = 0; cube < 2; ++cube) {
      if (cube == 1 && ts.clist[0] == nullptr) break;
      for (int k = 0; k < 3; ++k) {
        const double ms = time_ms([&] {
          p->launches += launch_spread(g, p->W, p->kc, p->C, p->ktiles, ts, p->b_y,
                                       p->b_xspread, p->grid_bf16, false,
                                       spread_mma_variant(wpcs[k], cube == 1), p->b_scratch,
                                       p->d_status, s);
        });
        if (ms < 0.0) continue;
        double& geo_ms = out->spread_mma_geo_ms[cube];
        if (geo_ms < 0.0 || ms < geo_ms) geo_ms = ms;
        if (out->spread_mma_ms < 0.0 || ms < out->spread_mma_ms) {
          out->spread_mma_ms = ms;
          out->spread_mma_wpc = wpcs[k];
          out->spread_mma_cube = cube;
        }
      }
    }
  }
  const int chunks[2] = {8, 4};
  const bool saved_tma = p->interp_tma;
  for (int t = 0; t < 2; ++t) {
    if (t == 1 && !(p->tma_ok && p->W == 4)) {
      out->interp_tma_ms[0] = out->interp_tma_ms[1] = -1.0;
      break;
    }
    for (int k = 0; k < 2; ++k) {
      p->interp_tma = t == 1;
      p->interp_coils = chunks[k];
      const CUtensorMap* tm = interp_tmap(p);
      const double ms = time_ms([&] {
        p->launches += launch_interp_kspace(g, p->W, p->kc, p->C, p->ktiles, ti, p->b_xwork,
                                            p->grid_bf16, p->b_y, chunks[k], tm, p->d_status, s);
      });
      (t == 0 ? out->interp_ms : out->interp_tma_ms)[k] = ms;
    }
  }
  // TMA staging with 2 coils per CTA (halo of 23 KB: more CTAs per SM)
  out->interp_tma2_ms = -1.0;
  if (p->tma_ok && p->W == 4) {
    p->interp_tma = true;
    p->interp_coils = 2;
    const CUtensorMap* tm = interp_tmap(p);
    out->interp_tma2_ms = time_ms([&] {
      p->launches += launch_interp_kspace(g, p->W, p->kc, p->C, p->ktiles, ti, p->b_xwork,
                                          p->grid_bf16, p->b_y, 2, tm, p->d_status, s);
    });
  }
  p->interp_tma = saved_tma;
  if (p->fft_pruned_ok) {
    // coil-grid transforms: cuFFT with the K5 / K8 kernels vs the own pruned
    // passes, timed as the first chunk's forward and adjoint (zero inputs: the
    // same work, no growth over the repetitions)
    const bool saved = p->fft_pruned;
    if (cudaMemsetAsync(p->b_m, 0, size_t(j1) * g.nvox * sizeof(nrsense_c64), s) != cudaSuccess)
      return NRSENSE_ERR_CUDA;
    for (int k = 0; k < 2; ++k) {
      p->fft_pruned = k == 1;
      nrsense_status st = NRSENSE_OK;
      out->fft_ms[k] = time_ms([&] {
        if (st == NRSENSE_OK) st = sense_chunk_forward(p, 0, j1, p->b_m, p->b_y, 0, s);
        if (st == NRSENSE_OK) st = sense_chunk_adjoint(p, 0, j1, p->b_y, 0, p->b_m, s);
      });
      if (st != NRSENSE_OK) {
        p->fft_pruned = saved;
        return st;
      }
    }
    p->fft_pruned = out->fft_ms[1] >= 0.0 && out->fft_ms[1] < out->fft_ms[0];
    out->fft_pruned = p->fft_pruned ? 1 : 0;
  }
  if (cudaGetLastError() != cudaSuccess) return NRSENSE_ERR_CUDA;
  for (int k = 0; k < 3; ++k)
    if (!(out->spread_ms[k] >= 0.0)) return NRSENSE_ERR_CUDA;
  for (int k = 0; k < 2; ++k)
    if (!(out->interp_ms[k] >= 0.0)) return NRSENSE_ERR_CUDA;
  // the compensated variant has only the shared-memory kernel: keep the default there
  if (!p->comp_spread) {
    int bk = 0;
    for (int k = 1; k < 3; ++k)
      if (out->spread_ms[k] < out->spread_ms[bk]) bk = k;
    p->spread_variant = variants[bk];
    if (mma_ok && out->spread_mma_ms >= 0.0 && out->spread_mma_ms < out->spread_ms[bk])
      p->spread_variant = spread_mma_variant(out->spread_mma_wpc, out->spread_mma_cube == 1);
  }
  // fastest interpolation: staging (per value / TMA) x coils per CTA (8 / 4; TMA also 2)
  double best = out->interp_ms[0];
  p->interp_tma = false;
  p->interp_coils = 8;
  for (int t = 0; t < 2; ++t)
    for (int k = 0; k < 2; ++k) {
      const double ms = (t == 0 ? out->interp_ms : out->interp_tma_ms)[k];
      if (ms >= 0.0 && ms < best) {
        best = ms;
        p->interp_tma = t == 1;
        p->interp_coils = chunks[k];
      }
    }
  if (out->interp_tma2_ms >= 0.0 && out->interp_tma2_ms < best) {
    p->interp_tma = true;
    p->interp_coils = 2;
  }
  out->spread_variant = p->spread_variant == kSpreadRegister ? NRSENSE_TUNE_SPREAD_REGISTER
                        : p->spread_variant == kSpreadShared ? NRSENSE_TUNE_SPREAD_SHARED
                        : spread_base(p->spread_variant) == kSpreadMMA ? NRSENSE_TUNE_SPREAD_MMA
                                                             : NRSENSE_TUNE_SPREAD_REGISTER_WARP;
  out->interp_coils = p->interp_coils;
  out->interp_tma = p->interp_tma ? 1 : 0;
  // work-item split of the k-space spread, timed with the chosen kernel: each
  // size re-tiles the plan (host work, outside the timed launches)
  {
    const int sizes[3] = {512, 1024, 2048};
    int best_m = p->spread_max_item;
    double best_ms = -1.0;
    for (int k = 0; k < 3; ++k) {
      NRS_TRY(retile_kspace(p, sizes[k], s));
      const PhaseTable tk = kspace_table(p, 0, j1, true, 0);
      const double ms = time_ms([&] {
        p->launches += launch_spread(g, p->W, p->kc, p->C, p->ktiles, tk, p->b_y, p->b_xspread,
                                     p->grid_bf16, p->comp_spread, p->spread_variant,
                                     p->b_scratch, p->d_status, s);
      });
      out->spread_item_ms[k] = ms;
      if (ms >= 0.0 && (best_ms < 0.0 || ms < best_ms)) {
        best_ms = ms;
        best_m = sizes[k];
      }
    }
    NRS_TRY(retile_kspace(p, best_m, s));
    out->spread_max_item = p->spread_max_item;
  }
  return NRSENSE_OK;
}

nrsense_status nrsense_plan_set_reduce(nrsense_plan_t p, nrsense_reduce_fn fn, void* user) {
  if (p == nullptr) return NRSENSE_ERR_ARG;
  p->reduce_fn = fn;
  p->reduce_user = user;
  p->epoch += 1;
  return NRSENSE_OK;
}

nrsense_status nrsense_copy_c64(nrsense_c64* dst_dev, const nrsense_c64* src_dev, int64_t n,
                                void* stream) {
  if (n < 0 || (n > 0 && (dst_dev == nullptr || src_dev == nullptr))) return NRSENSE_ERR_ARG;
  if (n == 0) return NRSENSE_OK;
  return cudaMemcpyAsync(dst_dev, src_dev, size_t(n) * sizeof(nrsense_c64),
                         cudaMemcpyDeviceToDevice, static_cast<cudaStream_t>(stream)) == cudaSuccess
             ? NRSENSE_OK
             : NRSENSE_ERR_CUDA;
}

}  // extern "C"
