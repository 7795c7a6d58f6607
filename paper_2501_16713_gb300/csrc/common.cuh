// Shared device-side definitions of the nonrigid SENSE library (sm_103a).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/nrsense.h"

namespace nrs {

// Coefficients of the per-tap kernel polynomials (see kb_host.cu):
// weight of tap t for fractional offset f in [0, 1) is
//   c(f + W/2 - 1 - t) ~= sum_k coef[t][k] * s^k,  s = 2f - 1.
constexpr int kNumCoef = 10;
constexpr int kMaxWidth = 6;

struct KernelCoefs {
  float c[kMaxWidth][kNumCoef];
};

// Per-axis geometry passed by value to every kernel.
struct Geo {
  int n0, n1, n2;     // image size
  int g0, g1, g2;     // oversampled grid size
  int osf;
  long long nvox;     // n0*n1*n2
  long long ngrid;    // g0*g1*g2
};

// A point (k-space sample or displaced voxel) after plan-time preprocessing:
// fractional offsets of the first tap per axis and the first tap's grid index
// packed 10 bits per axis (axis 0 in the high bits).
__host__ __device__ inline uint32_t pack_base(int b0, int b1, int b2) {
  return (uint32_t(b0) << 20) | (uint32_t(b1) << 10) | uint32_t(b2);
}
__host__ __device__ inline void unpack_base(uint32_t p, int& b0, int& b1, int& b2) {
  b0 = int(p >> 20);
  b1 = int((p >> 10) & 1023u);
  b2 = int(p & 1023u);
}

// One block of output-stationary spreading work: the points listed in
// list[begin, end) are spread into grid tile `tile`; slot < 0 writes the tile
// to the grid directly, slot >= 0 writes a partial tile to scratch slot
// `slot` (heavy tiles are split into several items and reduced afterwards).
// The same record describes interpolation work (sorted point range of a tile).
struct SpreadItem {
  int32_t tile;
  int32_t begin;
  int32_t end;
  int32_t slot;
};

// Offsets (relative to the item's begin) of the list entries of each
// first-tap plane offset r0 in (-W, T), stored per spreading item:
// bins[b] = first entry with r0 + W - 1 >= b, b = 0 .. W + T - 1.
constexpr int kMaxBins = kMaxWidth + 16;

// Up to kMaxChunkPhases motion states are processed by one launch.  The
// per-phase point data stay in their own arrays; a launch receives this table
// by value and finds the phase of a CTA from the item prefix sums.
constexpr int kMaxChunkPhases = 16;
// Footprint classes of a point in an 8^3 tile (3 per axis: low half only, both
// halves, high half only) and the per-item offsets that delimit them.
constexpr int kCubeBins = 27 + 1;
struct SpreadItem;
struct ReduceItem;
struct PhaseTable {
  const float4* qs[kMaxChunkPhases];
  const int32_t* perm[kMaxChunkPhases];
  const int2* list[kMaxChunkPhases];
  const int32_t* bins[kMaxChunkPhases];
  const int2* clist[kMaxChunkPhases];     // class-ordered lists (8^3 tiles, W = 4), or null
  const int32_t* cbins[kMaxChunkPhases];  // kCubeBins class starts per item
  const SpreadItem* items[kMaxChunkPhases];
  const ReduceItem* reduces[kMaxChunkPhases];
  long long row0[kMaxChunkPhases];    // first value/output row of the phase
  int item0[kMaxChunkPhases + 1];     // prefix sums of the launch's items per phase
  int red0[kMaxChunkPhases + 1];      // prefix sums of reduce items per phase
  int slot0[kMaxChunkPhases];         // first scratch slot of the phase
  int nphase;
};

// Image-space points (the displaced voxels of all phases) sorted by the 8^3
// home tile of their first tap, then by cell; home tiles are grouped 2 x 2 x 2
// into 16^3 super-tiles (spread_home.cu).
struct HomeSet {
  const float4* qs;       // sorted: (f0, f1, f2, packed first tap)
  const int32_t* perm;    // sorted index -> value row
  const int32_t* tstart;  // per home tile: first sorted index (nt0 nt1 nt2 + 1 entries)
  int nt0, nt1, nt2;      // home tiles per axis (ceil(G / 8))
  int ns0, ns1, ns2;      // super-tiles per axis (ceil(G / 16))
  // per grid coordinate of each axis: (count, covers...) with every cover
  // packed as super-tile * 32 + position in its 19-point padded extent
  const int4* cover0;
  const int4* cover1;
  const int4* cover2;
};

// Phase slot of work item `i` of a launch (linear search; nphase is small).
__device__ __forceinline__ int phase_of(const int* prefix, int nphase, int i) {
  int jj = 0;
  while (jj + 1 < nphase && i >= prefix[jj + 1]) ++jj;
  return jj;
}

// A split tile: partial tiles in scratch slots [first, first + count).
struct ReduceItem {
  int32_t tile;
  int32_t first;
  int32_t count;
  int32_t pad;
};

// Evaluate the W kernel weights of one axis for fractional offset f.
template <int W>
__device__ __forceinline__ void kernel_weights(float f, const KernelCoefs& kc, float (&w)[W]) {
  const float s = fmaf(2.0f, f, -1.0f);
#pragma unroll
  for (int t = 0; t < W; ++t) {
    float acc = kc.c[t][kNumCoef - 1];
#pragma unroll
    for (int k = kNumCoef - 2; k >= 0; --k) acc = fmaf(acc, s, kc.c[t][k]);
    w[t] = acc;
  }
}

// Select w[t] for a runtime t in [0, W) without dynamic register indexing.
template <int W>
__device__ __forceinline__ float select_tap(const float (&w)[W], int t) {
  float r = 0.f;
#pragma unroll
  for (int k = 0; k < W; ++k) r = (t == k) ? w[k] : r;
  return r;
}

// cp.async helpers (sm_80+): 8-byte global -> shared copy, zero-filled when
// `valid` is false.
__device__ __forceinline__ void cp_async_8(void* smem, const void* gmem, bool valid) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  const int src_size = valid ? 8 : 0;
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(s), "l"(gmem),
               "r"(src_size));
}
__device__ __forceinline__ void cp_async_4(void* smem, const void* gmem, bool valid) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  const int src_size = valid ? 4 : 0;
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(s), "l"(gmem),
               "r"(src_size));
}
// asynchronous copy of one stored grid value (complex FP32: 8 bytes; complex BF16: 4)
template <typename GT>
__device__ __forceinline__ void cp_async_grid(GT* smem, const GT* gmem, bool valid) {
  if constexpr (sizeof(GT) == 8)
    cp_async_8(smem, gmem, valid);
  else
    cp_async_4(smem, gmem, valid);
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// Storage of the k-space coil grids: complex FP32 (float2) or complex BF16
// (__nv_bfloat162, round to nearest even); arithmetic is FP32 either way.
using bf162 = __nv_bfloat162;
__device__ __forceinline__ float2 grid_ld(const float2* p) { return __ldg(p); }
__device__ __forceinline__ float2 grid_ld(const bf162* p) {
  const unsigned u = __ldg(reinterpret_cast<const unsigned*>(p));
  return __bfloat1622float2(*reinterpret_cast<const bf162*>(&u));
}
__device__ __forceinline__ void grid_st(float2* p, float2 v) { *p = v; }
__device__ __forceinline__ void grid_st(bf162* p, float2 v) { *p = __float22bfloat162_rn(v); }
__device__ __forceinline__ float2 grid_ld_shared(const float2* p) { return *p; }
__device__ __forceinline__ float2 grid_ld_shared(const bf162* p) { return __bfloat1622float2(*p); }
// two consecutive stored values (coils 2q, 2q+1) from shared memory as float4
__device__ __forceinline__ float4 grid_ld2_shared(const float2* p) {
  return *reinterpret_cast<const float4*>(p);
}
__device__ __forceinline__ float4 grid_ld2_shared(const bf162* p) {
  const uint2 u = *reinterpret_cast<const uint2*>(p);
  const float2 a = __bfloat1622float2(*reinterpret_cast<const bf162*>(&u.x));
  const float2 b = __bfloat1622float2(*reinterpret_cast<const bf162*>(&u.y));
  return make_float4(a.x, a.y, b.x, b.y);
}

__device__ __forceinline__ int wrap_once(int i, int g) {
  // i in [0, 2g): one conditional subtract
  return i >= g ? i - g : i;
}

__device__ __forceinline__ int wrap_any(int i, int g) {
  int r = i % g;
  return r < 0 ? r + g : r;
}

}  // namespace nrs
