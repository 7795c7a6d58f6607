// Learned preconditioner network: inference and training kernels.
//
// The network maps a CG residual r to a search direction z for flexible CG:
//   s = sqrt(mean |r|^2), u0 = [Re r, Im r] / s,
//   h_l = relu(conv_l(h_{l-1})) (l = 1..4, 16 channels), o = conv_5(h_4),
//   z = (u0 + o) read as a complex image,
// conv = 3x3x3 cross-correlation with zero padding and a bias.  The training
// loss is scale invariant (flexible CG does not depend on the scale of z):
// for the target e = E^{-1} r either the cosine distance
// L = 1 - Re<z, e> / (||z|| ||e||) or the energy loss
// L = 1 - c|c| / (<z, E z> <e, r>), c = Re<z, r>, the error energy left after
// a line search along z (one normal-operator application per pair).  The paper has no learned
// component: this network is the learned preconditioner of the Tikhonov CG
// solve of the reconstruction problem.
//
// Arithmetic: BF16 weights and activations, FP32 accumulation on the tensor
// cores (mma.sync m16n8k16 fed by ldmatrix), FP64 reductions for the input
// scale and the loss, FP32 master weights, gradients and Adam moments.
// Every layer runs as a 16 -> 16 channel convolution with zero weights in the
// padding (the 2-channel input and output layers included); activations are
// channels-last [voxel][16] BF16 (32 bytes per voxel).  Weight gradients are
// per-warp partial sums in a fixed grid order, reduced in FP64: training is
// bitwise reproducible.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include <atomic>

#include "plan_internal.h"

namespace nrs {
namespace cnnk {

using bf16 = __nv_bfloat16;

constexpr int kCh = 16;                       // channels of every (padded) layer
constexpr int kLayers = 5;
constexpr int kTaps = 27;
constexpr int BZ = 4, BY = 8, BX = 16;        // output block: 512 voxels
constexpr int HZ = BZ + 2, HY = BY + 2, HX = BX + 2;
constexpr int kHalo = HZ * HY * HX;           // 1080 input voxels
constexpr int kBlockVox = BZ * BY * BX;
constexpr int kVS = 24;                       // smem voxel stride (48 B): ldmatrix conflict-free
constexpr int kConvThreads = 256;             // 8 warps: one z plane, 4 rows each
constexpr int kWgThreads = 384;               // 12 warps: (tap plane tz) x (z plane)
constexpr int kWgParts = 4;                   // partial sums per wgrad CTA (one per z plane)
constexpr int kLayerW = kTaps * kCh * kCh;    // padded weights of one layer [tap][o][c]
constexpr int kLayerP = kLayerW + kCh;        // + biases
constexpr int kPack = kTaps * kCh * kVS;      // packed BF16 weights of one layer
constexpr int kRedThreads = 256;
constexpr int kRedBlocks = 1184;              // fixed grid: deterministic summation order
constexpr int kCin[kLayers] = {2, 16, 16, 16, 16};
constexpr int kCout[kLayers] = {16, 16, 16, 16, 2};
constexpr size_t kConvSmem = size_t(kHalo + kTaps * kCh) * kVS * sizeof(bf16);
constexpr size_t kWgSmem = size_t(kHalo + kBlockVox) * kVS * sizeof(bf16);

struct Vol {
  int d, h, w;
  long long n;
  int bz, by, bx;
  int nblocks;
};

struct Scalars {
  double sumsq;    // sum |r|^2
  double inv_s;    // 1 / sqrt(mean |r|^2), 0 when r == 0
  float inv_s_f;
  int ok;          // r != 0
  double zz, ee, ze, loss;
  double k1, k2;   // dL/dz = k2 z - k1 e
};

// kReluBf16: relu(acc + b); kMaskBf16: acc where mask > 0, else 0;
// kResidualC64: z = u0 + acc (channels 0, 1); kLinearBf16: acc + b;
// kAddMaskBf16: addend + (acc where mask > 0, else 0)
enum Epilogue { kReluBf16 = 0, kMaskBf16 = 1, kResidualC64 = 2, kLinearBf16 = 3, kAddMaskBf16 = 4 };

struct ConvArgs {
  Vol v;
  const bf16* in;       // [n][16]
  const bf16* wpk;      // [27][16][kVS] packed weights
  const float* bias;    // [16] or null
  int epi;
  const bf16* mask;     // kMaskBf16 / kAddMaskBf16: ReLU mask source [n][16]
  const bf16* addend;   // kAddMaskBf16: [n][16]
  bf16* out;            // kReluBf16 / kMaskBf16 output [n][16]
  const float2* r;      // kResidualC64: network input residual
  const Scalars* sc;
  float2* z;            // kResidualC64 output
};

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void ldsm_x4(unsigned addr, unsigned& r0, unsigned& r1, unsigned& r2,
                                        unsigned& r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(addr)
               : "memory");
}

__device__ __forceinline__ void ldsm_x4_t(unsigned addr, unsigned& r0, unsigned& r1, unsigned& r2,
                                          unsigned& r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(addr)
               : "memory");
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], unsigned a0, unsigned a1, unsigned a2,
                                         unsigned a3, unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// 16-byte asynchronous copy; zero-fills the destination when !valid.
__device__ __forceinline__ void cp_async_16(void* smem, const void* gmem, bool valid) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32(smem)),
               "l"(gmem), "r"(valid ? 16 : 0));
}

__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

__device__ __forceinline__ void block_origin(const Vol& v, int b, int& z0, int& y0, int& x0) {
  x0 = (b % v.bx) * BX;
  y0 = ((b / v.bx) % v.by) * BY;
  z0 = (b / (v.bx * v.by)) * BZ;
}

// Input halo of output block (z0, y0, x0): (BZ+2)(BY+2)(BX+2) voxels x 16
// channels, zero outside the volume (the convolution's zero padding).
__device__ __forceinline__ void stage_halo(const Vol& v, const bf16* __restrict__ in, bf16* sx,
                                           int z0, int y0, int x0) {
  for (int i = threadIdx.x; i < kHalo * 2; i += blockDim.x) {
    const int vox = i >> 1, half = i & 1;
    const int hz = vox / (HY * HX), hy = (vox / HX) % HY, hx = vox % HX;
    const int gz = z0 + hz - 1, gy = y0 + hy - 1, gx = x0 + hx - 1;
    const bool valid = (unsigned)gz < (unsigned)v.d && (unsigned)gy < (unsigned)v.h &&
                       (unsigned)gx < (unsigned)v.w;
    const long long gv = valid ? ((long long)gz * v.h + gy) * v.w + gx : 0;
    cp_async_16(sx + vox * kVS + half * 8, in + gv * kCh + half * 8, valid);
  }
}

// out[v][o] = epi(bias[o] + sum_{tap, c} W[tap][o][c] in[v + tap - 1][c]).
// A = activations (M = 16 voxels of one row, K = 16 channels), B = weights
// (K = channels, N = 8 output channels): per tap one K step.  Warp w owns
// z plane w/2, rows 4(w%2) .. 4(w%2)+3 of the block: 4 m-tiles x 2 n-tiles.
__global__ void __launch_bounds__(kConvThreads) conv3d_kernel(ConvArgs a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  bf16* sx = reinterpret_cast<bf16*>(smem_raw);  // [kHalo][kVS]
  bf16* sw = sx + kHalo * kVS;                    // [27 * 16][kVS]
  const Vol& v = a.v;
  int z0, y0, x0;
  block_origin(v, blockIdx.x, z0, y0, x0);
  stage_halo(v, a.in, sx, z0, y0, x0);
  for (int i = threadIdx.x; i < kTaps * kCh * 2; i += blockDim.x)
    cp_async_16(sw + (i >> 1) * kVS + (i & 1) * 8, a.wpk + (i >> 1) * kVS + (i & 1) * 8, true);
  cp_async_wait_all();
  __syncthreads();

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wz = warp >> 1, wy0 = (warp & 1) * 4;
  // ldmatrix row addresses: A (voxel rows, channel halves), B (o rows, c halves)
  const int arow = (lane & 7) + ((lane >> 3) & 1) * 8, acol = (lane >> 4) * 8;
  const int brow = (lane & 7) + (lane >> 4) * 8, bcol = ((lane >> 3) & 1) * 8;
  const unsigned sx_a = smem_u32(sx + arow * kVS + acol);
  const unsigned sw_b = smem_u32(sw + brow * kVS + bcol);

  float acc[4][2][4];
#pragma unroll
  for (int m = 0; m < 4; ++m)
#pragma unroll
    for (int n = 0; n < 2; ++n)
#pragma unroll
      for (int k = 0; k < 4; ++k) acc[m][n][k] = 0.f;

#pragma unroll 1
  for (int tz = 0; tz < 3; ++tz) {
#pragma unroll
    for (int t9 = 0; t9 < 9; ++t9) {
      const int ty = t9 / 3, tx = t9 % 3;
      const int tap = tz * 9 + t9;
      unsigned b00, b10, b01, b11;
      ldsm_x4(sw_b + tap * kCh * kVS * 2, b00, b10, b01, b11);
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        const int hrow = ((wz + tz) * HY + (wy0 + m + ty)) * HX + tx;
        unsigned a0, a1, a2, a3;
        ldsm_x4(sx_a + hrow * kVS * 2, a0, a1, a2, a3);
        mma_bf16(acc[m][0], a0, a1, a2, a3, b00, b10);
        mma_bf16(acc[m][1], a0, a1, a2, a3, b01, b11);
      }
    }
  }

  // epilogue: D[row g (+8)][col 2t, 2t+1] of each tile = voxel x, channel n*8 + 2t
  const int g = lane >> 2, t = lane & 3;
  float bias[2][2];
#pragma unroll
  for (int n = 0; n < 2; ++n) {
    bias[n][0] = a.bias ? a.bias[n * 8 + 2 * t] : 0.f;
    bias[n][1] = a.bias ? a.bias[n * 8 + 2 * t + 1] : 0.f;
  }
  const int z = z0 + wz;
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    const int y = y0 + wy0 + m;
#pragma unroll
    for (int hr = 0; hr < 2; ++hr) {
      const int x = x0 + g + 8 * hr;
      if (z >= v.d || y >= v.h || x >= v.w) continue;
      const long long vox = ((long long)z * v.h + y) * v.w + x;
      if (a.epi == kResidualC64) {
        if (t == 0) {
          // output channels 0, 1 = Re, Im of o; z = u0 + o (0 when r == 0)
          const float f0 = acc[m][0][2 * hr] + bias[0][0];
          const float f1 = acc[m][0][2 * hr + 1] + bias[0][1];
          const float2 rv = a.r[vox];
          float2 zv = make_float2(0.f, 0.f);
          if (a.sc->ok) zv = make_float2(fmaf(rv.x, a.sc->inv_s_f, f0), fmaf(rv.y, a.sc->inv_s_f, f1));
          a.z[vox] = zv;
        }
        continue;
      }
#pragma unroll
      for (int n = 0; n < 2; ++n) {
        const int o = n * 8 + 2 * t;
        float f0 = acc[m][n][2 * hr] + bias[n][0];
        float f1 = acc[m][n][2 * hr + 1] + bias[n][1];
        if (a.epi == kReluBf16) {
          f0 = fmaxf(f0, 0.f);
          f1 = fmaxf(f1, 0.f);
        } else if (a.epi == kMaskBf16 || a.epi == kAddMaskBf16) {
          const __nv_bfloat162 mk = *reinterpret_cast<const __nv_bfloat162*>(a.mask + vox * kCh + o);
          f0 = __bfloat162float(mk.x) > 0.f ? f0 : 0.f;
          f1 = __bfloat162float(mk.y) > 0.f ? f1 : 0.f;
          if (a.epi == kAddMaskBf16) {
            const __nv_bfloat162 ad =
                *reinterpret_cast<const __nv_bfloat162*>(a.addend + vox * kCh + o);
            f0 += __bfloat162float(ad.x);
            f1 += __bfloat162float(ad.y);
          }
        }
        *reinterpret_cast<__nv_bfloat162*>(a.out + vox * kCh + o) = __floats2bfloat162_rn(f0, f1);
      }
    }
  }
}

// Weight and bias gradients of one layer:
//   dW[tap][o][c] = sum_v g[v][o] in[v + tap - 1][c],  db[o] = sum_v g[v][o].
// A = g^T (M = 16 output channels, K = 16 voxels), B = shifted input
// (K = voxels, N = 8 input channels); both need voxel-consecutive pairs,
// which ldmatrix.trans delivers from the channels-last tiles.  Persistent
// grid; warp w accumulates the 9 taps of plane tz = w/4 over z plane w%4 of
// every block its CTA visits and writes one partial [27][16][16] slice.
__global__ void __launch_bounds__(kWgThreads, 1) wgrad_kernel(Vol v, const bf16* __restrict__ in,
                                                               const bf16* __restrict__ gr,
                                                               float* __restrict__ part_w,
                                                               float* __restrict__ part_b) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  bf16* sx = reinterpret_cast<bf16*>(smem_raw);  // [kHalo][kVS]
  bf16* sg = sx + kHalo * kVS;                    // [kBlockVox][kVS]
  __shared__ float sb[kWgThreads / kCh][kCh];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tz = warp >> 2, wz = warp & 3;
  const int grow = (lane & 7) + (lane >> 4) * 8, gcol = ((lane >> 3) & 1) * 8;
  const int xrow = (lane & 7) + ((lane >> 3) & 1) * 8, xcol = (lane >> 4) * 8;
  const unsigned sg_a = smem_u32(sg + (wz * BY * BX + grow) * kVS + gcol);
  const unsigned sx_b = smem_u32(sx + xrow * kVS + xcol);
  const int bch = threadIdx.x & (kCh - 1), bpart = threadIdx.x / kCh;

  float acc[9][2][4];
#pragma unroll
  for (int k = 0; k < 9; ++k)
#pragma unroll
    for (int n = 0; n < 2; ++n)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[k][n][e] = 0.f;
  float bacc = 0.f;

  for (int b = blockIdx.x; b < v.nblocks; b += gridDim.x) {
    int z0, y0, x0;
    block_origin(v, b, z0, y0, x0);
    __syncthreads();  // previous block's readers are done
    stage_halo(v, in, sx, z0, y0, x0);
    for (int i = threadIdx.x; i < kBlockVox * 2; i += blockDim.x) {
      const int vox = i >> 1, half = i & 1;
      const int lz = vox / (BY * BX), ly = (vox / BX) % BY, lx = vox % BX;
      const int gz = z0 + lz, gy = y0 + ly, gx = x0 + lx;
      const bool valid = gz < v.d && gy < v.h && gx < v.w;
      const long long gv = valid ? ((long long)gz * v.h + gy) * v.w + gx : 0;
      cp_async_16(sg + vox * kVS + half * 8, gr + gv * kCh + half * 8, valid);
    }
    cp_async_wait_all();
    __syncthreads();
    for (int vox = bpart; vox < kBlockVox; vox += kWgThreads / kCh)
      bacc += __bfloat162float(sg[vox * kVS + bch]);
#pragma unroll 1
    for (int y = 0; y < BY; ++y) {
      unsigned a0, a1, a2, a3;
      ldsm_x4_t(sg_a + y * BX * kVS * 2, a0, a1, a2, a3);
#pragma unroll
      for (int t9 = 0; t9 < 9; ++t9) {
        const int ty = t9 / 3, tx = t9 % 3;
        const int hrow = ((wz + tz) * HY + (y + ty)) * HX + tx;
        unsigned b00, b10, b01, b11;
        ldsm_x4_t(sx_b + hrow * kVS * 2, b00, b10, b01, b11);
        mma_bf16(acc[t9][0], a0, a1, a2, a3, b00, b10);
        mma_bf16(acc[t9][1], a0, a1, a2, a3, b01, b11);
      }
    }
  }

  // D[m = o][n = c]: c0 = (g, 2t), c1 = (g, 2t+1), c2 = (g+8, 2t), c3 = (g+8, 2t+1)
  const int g = lane >> 2, t = lane & 3;
  float* pw = part_w + (size_t(blockIdx.x) * kWgParts + wz) * kLayerW;
#pragma unroll
  for (int t9 = 0; t9 < 9; ++t9) {
    const int tap = tz * 9 + t9;
#pragma unroll
    for (int n = 0; n < 2; ++n)
#pragma unroll
      for (int hr = 0; hr < 2; ++hr) {
        const int o = g + 8 * hr, c = n * 8 + 2 * t;
        *reinterpret_cast<float2*>(pw + (tap * kCh + o) * kCh + c) =
            make_float2(acc[t9][n][2 * hr], acc[t9][n][2 * hr + 1]);
      }
  }
  sb[bpart][bch] = bacc;
  __syncthreads();
  if (threadIdx.x < kCh) {
    float s = 0.f;
    for (int p = 0; p < kWgThreads / kCh; ++p) s += sb[p][threadIdx.x];
    part_b[size_t(blockIdx.x) * kCh + threadIdx.x] = s;
  }
}

// grad[i] (+)= sum over partials, in fixed order, FP64.
__global__ void wgrad_reduce_kernel(const float* __restrict__ part_w, int n_wparts,
                                    const float* __restrict__ part_b, int n_bparts,
                                    float* __restrict__ grad, int accumulate) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kLayerP) return;
  double s = 0.0;
  if (i < kLayerW) {
    for (int p = 0; p < n_wparts; ++p) s += part_w[size_t(p) * kLayerW + i];
  } else {
    for (int p = 0; p < n_bparts; ++p) s += part_b[size_t(p) * kCh + (i - kLayerW)];
  }
  grad[i] = accumulate ? grad[i] + (float)s : (float)s;
}

__device__ __forceinline__ double warp_sum(double x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

template <int K>
__device__ void block_sum_k(double (&x)[K]) {
  __shared__ double s[K][kRedThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    x[k] = warp_sum(x[k]);
    if (lane == 0) s[k][warp] = x[k];
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      double tt = lane < kRedThreads / 32 ? s[k][lane] : 0.0;
      x[k] = warp_sum(tt);
    }
  }
  __syncthreads();
}

// FP64 block partials of sum |r|^2.
__global__ void __launch_bounds__(kRedThreads) sumsq_partial_kernel(const float2* __restrict__ r,
                                                                    long long n,
                                                                    double* __restrict__ partial) {
  double acc[1] = {0.0};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float2 a = r[i];
    acc[0] = fma((double)a.x, (double)a.x, fma((double)a.y, (double)a.y, acc[0]));
  }
  block_sum_k<1>(acc);
  if (threadIdx.x == 0) partial[blockIdx.x] = acc[0];
}

// Input scale from partials (or from an FP64 sum already on the device).
__global__ void scale_final_kernel(const double* __restrict__ partial, int nb,
                                   const double* __restrict__ ext_sumsq, long long n, Scalars* sc) {
  double acc[1] = {0.0};
  if (!ext_sumsq)
    for (int i = threadIdx.x; i < nb; i += blockDim.x) acc[0] += partial[i];
  block_sum_k<1>(acc);
  if (threadIdx.x == 0) {
    const double ss = ext_sumsq ? *ext_sumsq : acc[0];
    const bool ok = ss > 0.0 && isfinite(ss);
    sc->sumsq = ss;
    sc->ok = ok ? 1 : 0;
    sc->inv_s = ok ? 1.0 / sqrt(ss / (double)n) : 0.0;
    sc->inv_s_f = (float)sc->inv_s;
  }
}

// a0[v] = bf16([Re r, Im r] / s, 0, ..., 0)
__global__ void input_kernel(const float2* __restrict__ r, long long n, const Scalars* __restrict__ sc,
                             bf16* __restrict__ a0) {
  const float is = sc->inv_s_f;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float2 v = r[i];
    const __nv_bfloat162 h = __floats2bfloat162_rn(v.x * is, v.y * is);
    uint4 q0 = make_uint4(*reinterpret_cast<const unsigned*>(&h), 0u, 0u, 0u);
    uint4* dst = reinterpret_cast<uint4*>(a0 + i * kCh);
    dst[0] = q0;
    dst[1] = make_uint4(0u, 0u, 0u, 0u);
  }
}

// FP64 block partials of three real inner products Re<a_k, b_k>.
struct Dot3 {
  const float2* a[3];
  const float2* b[3];
};

__global__ void __launch_bounds__(kRedThreads) dot3_partial_kernel(Dot3 d, long long n,
                                                                   double* __restrict__ partial) {
  double acc[3] = {0.0, 0.0, 0.0};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float2 x = d.a[k][i], y = d.b[k][i];
      acc[k] = fma((double)x.x, (double)y.x, fma((double)x.y, (double)y.y, acc[k]));
    }
  }
  block_sum_k<3>(acc);
  if (threadIdx.x == 0) {
    partial[blockIdx.x] = acc[0];
    partial[gridDim.x + blockIdx.x] = acc[1];
    partial[2 * gridDim.x + blockIdx.x] = acc[2];
  }
}

// Loss and its gradient coefficients, dL/dz = k2 U - k1 V:
//   cosine (energy == 0): sums <z,z>, <e,e>, Re<z,e>; U = z, V = e;
//   energy (energy != 0): sums Re<z,Ez>, Re<e,r>, c = Re<z,r>; U = E z, V = r.
__global__ void loss_final_kernel(const double* __restrict__ partial, int nb, int energy,
                                  Scalars* sc) {
  double acc[3] = {0.0, 0.0, 0.0};
  for (int i = threadIdx.x; i < nb; i += blockDim.x) {
    acc[0] += partial[i];
    acc[1] += partial[nb + i];
    acc[2] += partial[2 * nb + i];
  }
  block_sum_k<3>(acc);
  if (threadIdx.x == 0) {
    sc->zz = acc[0];
    sc->ee = acc[1];
    sc->ze = acc[2];
    sc->loss = 1.0;
    sc->k1 = 0.0;
    sc->k2 = 0.0;
    if (!energy) {
      const double nz = sqrt(acc[0]), ne = sqrt(acc[1]);
      if (nz > 0.0 && ne > 0.0 && isfinite(nz) && isfinite(ne) && isfinite(acc[2])) {
        sc->loss = 1.0 - acc[2] / (nz * ne);
        sc->k1 = 1.0 / (nz * ne);
        sc->k2 = acc[2] / (nz * nz * nz * ne);
      }
    } else {
      const double zez = acc[0], er = acc[1], c = acc[2];
      if (zez > 0.0 && er > 0.0 && isfinite(zez) && isfinite(er) && isfinite(c)) {
        sc->loss = 1.0 - c * fabs(c) / (zez * er);
        sc->k1 = 2.0 * fabs(c) / (zez * er);
        sc->k2 = 2.0 * c * fabs(c) / (zez * zez * er);
      }
    }
  }
}

// g[v] = bf16(dL/do) = bf16(k2 U - k1 V) in channels 0, 1.
__global__ void loss_grad_kernel(const float2* __restrict__ U, const float2* __restrict__ V,
                                 long long n, const Scalars* __restrict__ sc, bf16* __restrict__ g) {
  const double k1 = sc->k1, k2 = sc->k2;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float gx = (float)(k2 * U[i].x - k1 * V[i].x);
    const float gy = (float)(k2 * U[i].y - k1 * V[i].y);
    const __nv_bfloat162 h = __floats2bfloat162_rn(gx, gy);
    uint4* dst = reinterpret_cast<uint4*>(g + i * kCh);
    dst[0] = make_uint4(*reinterpret_cast<const unsigned*>(&h), 0u, 0u, 0u);
    dst[1] = make_uint4(0u, 0u, 0u, 0u);
  }
}

__host__ __device__ constexpr int cin_of(int l) { return l == 0 ? 2 : kCh; }
__host__ __device__ constexpr int cout_of(int l) { return l == kLayers - 1 ? 2 : kCh; }

__device__ __forceinline__ bool param_valid(int i, int l) {
  const int k = i - l * kLayerP;
  if (k >= kLayerW) return (k - kLayerW) < cout_of(l);
  const int o = (k / kCh) % kCh, c = k % kCh;
  return o < cout_of(l) && c < cin_of(l);
}

// Adam (Kingma & Ba) on the FP32 master weights; padding stays zero.
__global__ void adam_kernel(float* __restrict__ w, float* __restrict__ m, float* __restrict__ vv,
                            const float* __restrict__ grad, float gscale, float lr, float b1,
                            float b2, float eps, float bc1, float bc2, int freeze_bias) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kLayers * kLayerP) return;
  const int l = i / kLayerP;
  if (!param_valid(i, l)) {
    w[i] = 0.f;
    return;
  }
  if (freeze_bias && i - l * kLayerP >= kLayerW) return;
  const float gi = grad[i] * gscale;
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * vv[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  vv[i] = vi;
  w[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
}

// BF16 packed weights: forward [tap][o][c] and input-gradient weights
// [tap'][c][o] = W[26 - tap'][o][c] (flipped taps, swapped channels).
__global__ void pack_kernel(const float* __restrict__ w, bf16* __restrict__ fwd,
                            bf16* __restrict__ bwd) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kLayers * kLayerW) return;
  const int l = i / kLayerW, k = i % kLayerW;
  const int tap = k / (kCh * kCh), o = (k / kCh) % kCh, c = k % kCh;
  const bf16 h = __float2bfloat16_rn(w[size_t(l) * kLayerP + k]);
  fwd[size_t(l) * kPack + (tap * kCh + o) * kVS + c] = h;
  bwd[size_t(l) * kPack + ((kTaps - 1 - tap) * kCh + c) * kVS + o] = h;
}

}  // namespace cnnk
}  // namespace nrs

using namespace nrs::cnnk;

struct nrsense_cnn_s {
  Vol vol;
  uint64_t serial = 0;  // creation number: solver graphs key on it, not on the address
  int device = 0;
  int wg_grid = 0;
  bf16* act[kLayers] = {};  // a0 .. a4 (inference uses a0, a1 as ping-pong)
  bf16* gb[3] = {};         // gradient ping-pong (+ one more in the symmetric form)
  bool spd = false;         // symmetric form z = u0 + N4^T (I + W5^T W5) N4 u0
  bf16* h5 = nullptr;       // symmetric form: t5 = W5 h4 (2 channels, padded)
  bf16* ut[4] = {};         // symmetric form: transposed chain u_1 .. u_4
  float2* zbuf = nullptr;   // training forward output
  float2* ezbuf = nullptr;  // E z for the energy loss (allocated on first use)
  float* master = nullptr;  // [5][kLayerP] FP32
  float* grad = nullptr;
  float* am = nullptr;
  float* av = nullptr;
  bf16* wfwd = nullptr;     // [5][kPack]
  bf16* wbwd = nullptr;
  float* part_w = nullptr;  // [wg_grid * kWgParts][kLayerW]
  float* part_b = nullptr;  // [wg_grid][16]
  double* red = nullptr;    // 3 * kRedBlocks
  Scalars* sc = nullptr;
  int adam_t = 0;
  long long launches = 0;
  std::vector<void*> allocations;
};

namespace {

int ew_grid(long long n) {
  return (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, 152LL * 16));
}

nrsense_status cuda_ok() {
  return cudaGetLastError() == cudaSuccess ? NRSENSE_OK : NRSENSE_ERR_CUDA;
}

void conv(nrsense_cnn_s* net, int layer, bool backward, const bf16* in, int epi, const bf16* mask,
          bf16* out, const float2* r, float2* z, cudaStream_t s, const bf16* addend = nullptr) {
  ConvArgs a;
  a.addend = addend;
  a.v = net->vol;
  a.in = in;
  a.wpk = (backward ? net->wbwd : net->wfwd) + size_t(layer) * kPack;
  a.bias = (backward || net->spd) ? nullptr : net->master + size_t(layer) * kLayerP + kLayerW;
  a.epi = epi;
  a.mask = mask;
  a.out = out;
  a.r = r;
  a.sc = net->sc;
  a.z = z;
  conv3d_kernel<<<net->vol.nblocks, kConvThreads, kConvSmem, s>>>(a);
  net->launches += 1;
}

// forward pass; keep = true stores every activation (training).  The
// symmetric form always keeps them: its transposed chain reuses the masks.
void forward(nrsense_cnn_s* net, const float2* r, const double* sumsq_dev, float2* z, bool keep,
             cudaStream_t s) {
  const long long n = net->vol.n;
  if (!sumsq_dev) {
    sumsq_partial_kernel<<<kRedBlocks, kRedThreads, 0, s>>>(r, n, net->red);
    net->launches += 1;
  }
  scale_final_kernel<<<1, kRedThreads, 0, s>>>(net->red, kRedBlocks, sumsq_dev, n, net->sc);
  input_kernel<<<ew_grid(n), 256, 0, s>>>(r, n, net->sc, net->act[0]);
  net->launches += 2;
  if (net->spd) {
    // h_l = D_l W_l h_{l-1} (l = 1..4), t5 = W5 h4
    for (int l = 0; l < kLayers - 1; ++l)
      conv(net, l, false, net->act[l], kReluBf16, nullptr, net->act[l + 1], nullptr, nullptr, s);
    conv(net, kLayers - 1, false, net->act[kLayers - 1], kLinearBf16, nullptr, net->h5, nullptr,
         nullptr, s);
    // u_4 = h4 + D_4 W5^T t5 (= D_4 m), u_l = D_l W_{l+1}^T u_{l+1}, z = u0 + W_1^T u_1
    conv(net, kLayers - 1, true, net->h5, kAddMaskBf16, net->act[kLayers - 1], net->ut[kLayers - 2],
         nullptr, nullptr, s, net->act[kLayers - 1]);
    for (int l = kLayers - 2; l >= 1; --l)
      conv(net, l, true, net->ut[l], kMaskBf16, net->act[l], net->ut[l - 1], nullptr, nullptr, s);
    conv(net, 0, true, net->ut[0], kResidualC64, nullptr, nullptr, r, z, s);
    return;
  }
  for (int l = 0; l < kLayers - 1; ++l) {
    const bf16* in = keep ? net->act[l] : net->act[l & 1];
    bf16* out = keep ? net->act[l + 1] : net->act[(l + 1) & 1];
    conv(net, l, false, in, kReluBf16, nullptr, out, nullptr, nullptr, s);
  }
  conv(net, kLayers - 1, false, keep ? net->act[kLayers - 1] : net->act[(kLayers - 1) & 1],
       kResidualC64, nullptr, nullptr, r, z, s);
}

// dW_l (+)= sum_v g[v][o] in[v + tap - 1][c] and db_l (+)= sum_v g[v][o]
void wgrad(nrsense_cnn_s* net, int l, const bf16* in, const bf16* g, bool accumulate,
           cudaStream_t s) {
  wgrad_kernel<<<net->wg_grid, kWgThreads, kWgSmem, s>>>(net->vol, in, g, net->part_w, net->part_b);
  wgrad_reduce_kernel<<<(kLayerP + 255) / 256, 256, 0, s>>>(
      net->part_w, net->wg_grid * kWgParts, net->part_b, net->wg_grid,
      net->grad + size_t(l) * kLayerP, accumulate ? 1 : 0);
  net->launches += 2;
}

void* dalloc(nrsense_cnn_s* net, size_t bytes) {
  void* p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  net->allocations.push_back(p);
  return p;
}

void release(nrsense_cnn_s* net) {
  for (void* p : net->allocations) cudaFree(p);
  delete net;
}

// splitmix64 and Box-Muller: a seeded normal generator for initialisation
struct Normal {
  uint64_t state;
  uint64_t next() {
    uint64_t z = (state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  }
  double uniform() { return (double(next() >> 11) + 0.5) * (1.0 / 9007199254740992.0); }
  double operator()() {
    const double u1 = uniform(), u2 = uniform();
    return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
  }
};

// natural layout: per layer W (cout, cin, 3, 3, 3) then b (cout)
int64_t natural_count() {
  int64_t c = 0;
  for (int l = 0; l < kLayers; ++l) c += int64_t(kCout[l]) * kCin[l] * kTaps + kCout[l];
  return c;
}

void natural_to_padded(const float* nat, std::vector<float>& pad) {
  pad.assign(size_t(kLayers) * kLayerP, 0.f);
  size_t k = 0;
  for (int l = 0; l < kLayers; ++l) {
    float* P = pad.data() + size_t(l) * kLayerP;
    for (int o = 0; o < kCout[l]; ++o)
      for (int c = 0; c < kCin[l]; ++c)
        for (int tap = 0; tap < kTaps; ++tap) P[(tap * kCh + o) * kCh + c] = nat[k++];
    for (int o = 0; o < kCout[l]; ++o) P[kLayerW + o] = nat[k++];
  }
}

void padded_to_natural(const std::vector<float>& pad, float* nat) {
  size_t k = 0;
  for (int l = 0; l < kLayers; ++l) {
    const float* P = pad.data() + size_t(l) * kLayerP;
    for (int o = 0; o < kCout[l]; ++o)
      for (int c = 0; c < kCin[l]; ++c)
        for (int tap = 0; tap < kTaps; ++tap) nat[k++] = P[(tap * kCh + o) * kCh + c];
    for (int o = 0; o < kCout[l]; ++o) nat[k++] = P[kLayerW + o];
  }
}

nrsense_status upload_params(nrsense_cnn_s* net, const std::vector<float>& pad, cudaStream_t s) {
  const size_t bytes = pad.size() * sizeof(float);
  if (cudaMemcpyAsync(net->master, pad.data(), bytes, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemsetAsync(net->am, 0, bytes, s) != cudaSuccess ||
      cudaMemsetAsync(net->av, 0, bytes, s) != cudaSuccess ||
      cudaMemsetAsync(net->grad, 0, bytes, s) != cudaSuccess)
    return NRSENSE_ERR_CUDA;
  pack_kernel<<<(kLayers * kLayerW + 255) / 256, 256, 0, s>>>(net->master, net->wfwd, net->wbwd);
  net->launches += 1;
  net->adam_t = 0;
  if (cudaStreamSynchronize(s) != cudaSuccess) return NRSENSE_ERR_CUDA;
  return cuda_ok();
}

}  // namespace

namespace nrs {

long long cnn_nvox(const nrsense_cnn_s* net) { return net->vol.n; }

uint64_t cnn_serial(const nrsense_cnn_s* net) { return net ? net->serial : 0; }

bool cnn_shape_matches(const nrsense_cnn_s* net, int n0, int n1, int n2) {
  return net->vol.d == n0 && net->vol.h == n1 && net->vol.w == n2;
}

long long cnn_apply_async(nrsense_cnn_s* net, const float2* r, const double* sumsq_dev, float2* z,
                          cudaStream_t s) {
  const long long l0 = net->launches;
  forward(net, r, sumsq_dev, z, false, s);
  return net->launches - l0;
}

}  // namespace nrs

extern "C" {

nrsense_status nrsense_cnn_create(const int32_t* n_host, uint32_t flags, void* stream,
                                  nrsense_cnn_t* out) {
  if (!n_host || !out || (flags & ~NRSENSE_CNN_SYMMETRIC)) return NRSENSE_ERR_ARG;
  *out = nullptr;
  for (int a = 0; a < 3; ++a)
    if (n_host[a] < 1 || n_host[a] > 4096) return NRSENSE_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  nrsense_cnn_s* net = new (std::nothrow) nrsense_cnn_s();
  if (!net) return NRSENSE_ERR_OOM;
  static std::atomic<uint64_t> next_serial{1};
  net->serial = next_serial.fetch_add(1);
  net->spd = (flags & NRSENSE_CNN_SYMMETRIC) != 0;
  Vol& v = net->vol;
  v.d = n_host[0];
  v.h = n_host[1];
  v.w = n_host[2];
  v.n = (long long)v.d * v.h * v.w;
  v.bz = (v.d + BZ - 1) / BZ;
  v.by = (v.h + BY - 1) / BY;
  v.bx = (v.w + BX - 1) / BX;
  const long long nb = (long long)v.bz * v.by * v.bx;
  if (nb > (1LL << 30)) {
    delete net;
    return NRSENSE_ERR_ARG;
  }
  v.nblocks = (int)nb;
  int sms = 0;
  if (cudaGetDevice(&net->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, net->device) != cudaSuccess ||
      cudaFuncSetAttribute(conv3d_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)kConvSmem) != cudaSuccess ||
      cudaFuncSetAttribute(wgrad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)kWgSmem) != cudaSuccess) {
    cudaGetLastError();
    delete net;
    return NRSENSE_ERR_CUDA;
  }
  net->wg_grid = std::max(1, std::min(v.nblocks, sms));
  const size_t ab = size_t(v.n) * kCh * sizeof(bf16);
  const size_t pb = size_t(kLayers) * kLayerP * sizeof(float);
  bool ok = true;
  for (int l = 0; l < kLayers && ok; ++l) ok = (net->act[l] = (bf16*)dalloc(net, ab)) != nullptr;
  for (int k = 0; k < 2 && ok; ++k) ok = (net->gb[k] = (bf16*)dalloc(net, ab)) != nullptr;
  if (net->spd) {
    ok = ok && (net->gb[2] = (bf16*)dalloc(net, ab)) != nullptr;
    ok = ok && (net->h5 = (bf16*)dalloc(net, ab)) != nullptr;
    for (int k = 0; k < 4 && ok; ++k) ok = (net->ut[k] = (bf16*)dalloc(net, ab)) != nullptr;
  }
  ok = ok && (net->zbuf = (float2*)dalloc(net, size_t(v.n) * sizeof(float2))) != nullptr;
  ok = ok && (net->master = (float*)dalloc(net, pb)) != nullptr;
  ok = ok && (net->grad = (float*)dalloc(net, pb)) != nullptr;
  ok = ok && (net->am = (float*)dalloc(net, pb)) != nullptr;
  ok = ok && (net->av = (float*)dalloc(net, pb)) != nullptr;
  ok = ok && (net->wfwd = (bf16*)dalloc(net, size_t(kLayers) * kPack * sizeof(bf16))) != nullptr;
  ok = ok && (net->wbwd = (bf16*)dalloc(net, size_t(kLayers) * kPack * sizeof(bf16))) != nullptr;
  ok = ok && (net->part_w = (float*)dalloc(
                  net, size_t(net->wg_grid) * kWgParts * kLayerW * sizeof(float))) != nullptr;
  ok = ok && (net->part_b = (float*)dalloc(net, size_t(net->wg_grid) * kCh * sizeof(float))) != nullptr;
  ok = ok && (net->red = (double*)dalloc(net, 3 * kRedBlocks * sizeof(double))) != nullptr;
  ok = ok && (net->sc = (Scalars*)dalloc(net, sizeof(Scalars))) != nullptr;
  if (!ok) {
    release(net);
    return NRSENSE_ERR_OOM;
  }
  if (cudaMemsetAsync(net->wfwd, 0, size_t(kLayers) * kPack * sizeof(bf16), s) != cudaSuccess ||
      cudaMemsetAsync(net->wbwd, 0, size_t(kLayers) * kPack * sizeof(bf16), s) != cudaSuccess ||
      cudaMemsetAsync(net->sc, 0, sizeof(Scalars), s) != cudaSuccess) {
    release(net);
    return NRSENSE_ERR_CUDA;
  }
  std::vector<float> pad(size_t(kLayers) * kLayerP, 0.f);
  const nrsense_status st = upload_params(net, pad, s);
  if (st != NRSENSE_OK) {
    release(net);
    return st;
  }
  *out = net;
  return NRSENSE_OK;
}

nrsense_status nrsense_cnn_destroy(nrsense_cnn_t net) {
  if (!net) return NRSENSE_OK;
  cudaDeviceSynchronize();
  release(net);
  return NRSENSE_OK;
}

int64_t nrsense_cnn_num_params(void) { return natural_count(); }

nrsense_status nrsense_cnn_init_params(nrsense_cnn_t net, uint64_t seed, void* stream) {
  if (!net) return NRSENSE_ERR_ARG;
  Normal rng{seed};
  std::vector<float> nat(static_cast<size_t>(natural_count()));
  size_t k = 0;
  for (int l = 0; l < kLayers; ++l) {
    // He initialisation; the last layer starts small so that z ~ r / s
    const double sd = std::sqrt(2.0 / (kTaps * kCin[l])) * (l == kLayers - 1 ? 0.1 : 1.0);
    for (int i = 0; i < kCout[l] * kCin[l] * kTaps; ++i) nat[k++] = (float)(sd * rng());
    for (int o = 0; o < kCout[l]; ++o) nat[k++] = 0.f;
  }
  std::vector<float> pad;
  natural_to_padded(nat.data(), pad);
  return upload_params(net, pad, static_cast<cudaStream_t>(stream));
}

nrsense_status nrsense_cnn_set_params(nrsense_cnn_t net, const float* params_host, int64_t count,
                                      void* stream) {
  if (!net || !params_host || count != natural_count()) return NRSENSE_ERR_ARG;
  for (int64_t i = 0; i < count; ++i)
    if (!std::isfinite(params_host[i])) return NRSENSE_ERR_ARG;
  std::vector<float> pad;
  natural_to_padded(params_host, pad);
  return upload_params(net, pad, static_cast<cudaStream_t>(stream));
}

static nrsense_status download(nrsense_cnn_t net, const float* src, float* dst, int64_t count,
                               void* stream) {
  if (!net || !dst || count != natural_count()) return NRSENSE_ERR_ARG;
  std::vector<float> pad(size_t(kLayers) * kLayerP);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cudaMemcpyAsync(pad.data(), src, pad.size() * sizeof(float), cudaMemcpyDeviceToHost, s) !=
          cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return NRSENSE_ERR_CUDA;
  padded_to_natural(pad, dst);
  return NRSENSE_OK;
}

nrsense_status nrsense_cnn_get_params(nrsense_cnn_t net, float* params_host, int64_t count,
                                      void* stream) {
  return download(net, net ? net->master : nullptr, params_host, count, stream);
}

nrsense_status nrsense_cnn_get_grads(nrsense_cnn_t net, float* grads_host, int64_t count,
                                     void* stream) {
  return download(net, net ? net->grad : nullptr, grads_host, count, stream);
}

nrsense_status nrsense_cnn_apply(nrsense_cnn_t net, const nrsense_c64* r_dev, nrsense_c64* z_dev,
                                 void* stream) {
  if (!net || !r_dev || !z_dev) return NRSENSE_ERR_ARG;
  forward(net, reinterpret_cast<const float2*>(r_dev), nullptr, reinterpret_cast<float2*>(z_dev),
          false, static_cast<cudaStream_t>(stream));
  return cuda_ok();
}

nrsense_status nrsense_cnn_gradients(nrsense_cnn_t net, nrsense_plan_t plan, double lambda,
                                     const nrsense_c64* r_dev, const nrsense_c64* e_dev,
                                     int32_t accumulate, double* loss_host, void* stream) {
  if (!net || !r_dev || !e_dev) return NRSENSE_ERR_ARG;
  if (plan && (!nrs::cnn_shape_matches(net, plan->geo.n0, plan->geo.n1, plan->geo.n2) ||
               !(lambda >= 0.0) || !std::isfinite(lambda)))
    return NRSENSE_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const long long n = net->vol.n;
  const float2* r = reinterpret_cast<const float2*>(r_dev);
  const float2* e = reinterpret_cast<const float2*>(e_dev);
  if (plan && !net->ezbuf && !(net->ezbuf = (float2*)dalloc(net, size_t(n) * sizeof(float2))))
    return NRSENSE_ERR_OOM;
  forward(net, r, nullptr, net->zbuf, true, s);
  Dot3 d;
  const float2 *U, *V;
  if (plan) {
    nrsense_status st = nrsense_apply_normal(plan, reinterpret_cast<const nrsense_c64*>(net->zbuf),
                                             lambda, reinterpret_cast<nrsense_c64*>(net->ezbuf),
                                             stream);
    if (st != NRSENSE_OK) return st;
    d = Dot3{{net->zbuf, e, net->zbuf}, {net->ezbuf, r, r}};
    U = net->ezbuf;
    V = r;
  } else {
    d = Dot3{{net->zbuf, e, net->zbuf}, {net->zbuf, e, e}};
    U = net->zbuf;
    V = e;
  }
  dot3_partial_kernel<<<kRedBlocks, kRedThreads, 0, s>>>(d, n, net->red);
  loss_final_kernel<<<1, kRedThreads, 0, s>>>(net->red, kRedBlocks, plan ? 1 : 0, net->sc);
  loss_grad_kernel<<<ew_grid(n), 256, 0, s>>>(U, V, n, net->sc, net->gb[0]);
  net->launches += 3;
  int cur = 0;
  if (net->spd) {
    // adjoint of the transposed chain o = W_1^T u_1, u_l = D_l W_{l+1}^T u_{l+1}:
    // dW_{l+1} (+)= wgrad(g, u_{l+1}); the gradient passes on as D_{l+1} W_{l+1} g
    for (int l = 0; l < kLayers - 1; ++l) {
      wgrad(net, l, net->gb[cur], net->ut[l], accumulate != 0, s);
      conv(net, l, false, net->gb[cur], kMaskBf16, net->act[l + 1], net->gb[cur ^ 1], nullptr,
           nullptr, s);
      cur ^= 1;
    }
    // gb[cur] = dL/dm (masked); middle m = h4 + W5^T W5 h4 with q = W5 dL/dm:
    // dW5 = wgrad(h4, q) + wgrad(dL/dm, t5), D_4 dL/dh4 = dL/dm + D_4 W5^T q
    const int L5 = kLayers - 1;
    bf16* q = net->gb[2];
    conv(net, L5, false, net->gb[cur], kLinearBf16, nullptr, q, nullptr, nullptr, s);
    wgrad(net, L5, net->act[L5], q, accumulate != 0, s);
    wgrad(net, L5, net->gb[cur], net->h5, true, s);
    conv(net, L5, true, q, kAddMaskBf16, net->act[L5], net->gb[cur ^ 1], nullptr, nullptr, s,
         net->gb[cur]);
    cur ^= 1;
    // back through the forward chain h_l = D_l W_l h_{l-1}, l = 4 .. 1
    for (int l = L5 - 1; l >= 0; --l) {
      wgrad(net, l, net->act[l], net->gb[cur], true, s);
      if (l > 0) {
        conv(net, l, true, net->gb[cur], kMaskBf16, net->act[l], net->gb[cur ^ 1], nullptr, nullptr,
             s);
        cur ^= 1;
      }
    }
  } else {
    // backward through the forward chain: g holds dL/d(output of layer l)
    for (int l = kLayers - 1; l >= 0; --l) {
      wgrad(net, l, net->act[l], net->gb[cur], accumulate != 0, s);
      if (l > 0) {
        conv(net, l, true, net->gb[cur], kMaskBf16, net->act[l], net->gb[cur ^ 1], nullptr, nullptr,
             s);
        cur ^= 1;
      }
    }
  }
  nrsense_status st = cuda_ok();
  if (st != NRSENSE_OK) return st;
  if (loss_host) {
    Scalars h;
    if (cudaMemcpyAsync(&h, net->sc, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return NRSENSE_ERR_CUDA;
    *loss_host = h.loss;
  }
  return NRSENSE_OK;
}

nrsense_status nrsense_cnn_adam_step(nrsense_cnn_t net, float lr, float grad_scale, float beta1,
                                     float beta2, float eps, uint32_t flags, void* stream) {
  if (!net || !(lr >= 0.f) || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) ||
      !(eps > 0.f) || !std::isfinite(grad_scale))
    return NRSENSE_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  net->adam_t += 1;
  const float bc1 = (float)(1.0 - std::pow((double)beta1, net->adam_t));
  const float bc2 = (float)(1.0 - std::pow((double)beta2, net->adam_t));
  adam_kernel<<<(kLayers * kLayerP + 255) / 256, 256, 0, s>>>(net->master, net->am, net->av,
                                                              net->grad, grad_scale, lr, beta1,
                                                              beta2, eps, bc1, bc2,
                                                              ((flags & NRSENSE_CNN_FREEZE_BIAS) || net->spd) ? 1 : 0);
  pack_kernel<<<(kLayers * kLayerW + 255) / 256, 256, 0, s>>>(net->master, net->wfwd, net->wbwd);
  net->launches += 2;
  return cuda_ok();
}

nrsense_status nrsense_cnn_launches(nrsense_cnn_t net, int64_t* out_host) {
  if (!net || !out_host) return NRSENSE_ERR_ARG;
  *out_host = net->launches;
  return NRSENSE_OK;
}

}  // extern "C"
