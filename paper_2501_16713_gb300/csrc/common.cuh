// Shared device-side definitions of the nonrigid SENSE library (sm_103a).
#pragma once

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
struct SpreadItem {
  int32_t tile;
  int32_t begin;
  int32_t end;
  int32_t slot;
};

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

__device__ __forceinline__ int wrap_once(int i, int g) {
  // i in [0, 2g): one conditional subtract
  return i >= g ? i - g : i;
}

__device__ __forceinline__ int wrap_any(int i, int g) {
  int r = i % g;
  return r < 0 ? r + g : r;
}

}  // namespace nrs
