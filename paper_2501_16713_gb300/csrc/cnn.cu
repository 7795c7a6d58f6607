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
#include <cudaTypedefs.h>

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
__global__ void __launch_bounds__(kConvThreads, 3) conv3d_kernel(ConvArgs a) {
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

// ---------------------------------------------------------------------------
// The same convolution on the fifth-generation tensor cores (tcgen05): an
// implicit GEMM D[voxel][o] = sum_{tap, c} A_tap[voxel][c] B_tap[o][c] with the
// accumulators in tensor memory.  An output block of 4 x 16 x 8 voxels is four
// M = 128, N = 16 tiles (output plane z: 16 rows y x 8 voxels x); each of the
// 27 taps adds one K = 16 (BF16) product to each tile, issued by a single
// thread: 108 MMAs per block.
//
// Operands sit in shared memory in the canonical K-major layout without
// swizzling: core matrices of 8 rows x 16 bytes (8 channels), rows 16 bytes
// apart, the two channel halves (K) a fixed stride (LBO) apart and the 8-row
// groups a fixed stride (SBO) apart.  A tile's 8-row groups are its 16 y rows
// of 8 consecutive voxels, so a tap's A operand is a view of the one staged
// halo ([half][hz][hy][hx] x 16 bytes, 6 x 18 x 10 voxels, loaded by two bulk
// tensor copies, one per channel half, zero outside the volume): start at the
// shifted first voxel, SBO = one halo row (160 bytes), LBO = one channel
// half.  Weights: [half][tap][o] x 16 bytes (per-thread asynchronous copies).
// 48 KB of shared memory: four CTAs per SM, one block each.  Tensor memory:
// 64 columns (4 tiles x 16 channels) over the 128 lanes; warp w reads lanes
// 32 (w mod 4) .. + 31 of tiles 2 (w / 4) and 2 (w / 4) + 1.  Both waits on
// mbarriers (halo landed, products done) are bounded; on expiry the CTA
// records NRSENSE_ERR_TIMEOUT, stores nothing, waits (bounded) for what it has
// in flight, frees its tensor memory and returns.  (Measured alternatives: the
// halo by per-thread copies, 3 % faster; persistent CTAs with a two-stage
// copy / product / epilogue pipeline, 20 % slower: with two CTAs per SM
// nothing hides the epilogue.)

constexpr int TBZ = 4, TBY = 16, TBX = 8;               // output block of the tcgen05 kernel
constexpr int THZ = TBZ + 2, THY = TBY + 2, THX = TBX + 2;
constexpr int kTcHaloVox = THZ * THY * THX;             // 1080
constexpr int kTcThreads = 256;
constexpr int kTcHalfBytes = kTcHaloVox * 16;           // one channel half of the halo: 17280
constexpr int kTcStageBytes = 2 * kTcHalfBytes;         // the halo, both halves: 34560
constexpr int kTcWHalfBytes = kTaps * kCh * 16;         // 6912
constexpr size_t kTcSmem = size_t(kTcStageBytes) + size_t(2) * kTcWHalfBytes + 128;  // 48 KB
constexpr uint32_t kTcCols = 64;                        // tensor-memory columns (4 tiles)
constexpr long long kTcMaxPoll = 1LL << 24;

__host__ __device__ inline int tc_blocks(const Vol& v) {
  return ((v.d + TBZ - 1) / TBZ) * ((v.h + TBY - 1) / TBY) * ((v.w + TBX - 1) / TBX);
}

// Shared-memory matrix descriptor (no swizzling): start address, leading
// (K-direction) and stride (M/N-direction) byte offsets in 16-byte units,
// descriptor version 1 at bits 46-47.
__device__ __forceinline__ uint64_t tc_desc(unsigned saddr, unsigned lbo, unsigned sbo) {
  return uint64_t((saddr >> 4) & 0x3FFFu) | (uint64_t((lbo >> 4) & 0x3FFFu) << 16) |
         (uint64_t((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: F32 accumulators (bits 4-5 = 1), BF16 A
// and B (bits 7-9, 10-12 = 1), both K-major, N / 8 at bits 17-22, M / 16 at
// bits 24-28 (M = 128, N = 16).
constexpr uint32_t kTcIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((16u >> 3) << 17) |
                              ((128u >> 4) << 24);

__device__ __forceinline__ bool tc_mbar_try_wait(unsigned mbar, unsigned parity) {
  unsigned done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(mbar), "r"(parity)
      : "memory");
  return done != 0;
}

// One thread: D(tmem) (+)= A B^T over K = 16
__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                       uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(kTcIdesc), "r"(accumulate)
      : "memory");
}

// 16 consecutive accumulator columns of this thread's lane
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

// The epilogue of one output voxel from its 16 channel sums (bias not yet
// added): the same operations as conv3d_kernel's.
__device__ __forceinline__ void conv_store_voxel(const ConvArgs& a, long long vox,
                                                 const float (&acc)[16]) {
  if (a.epi == kResidualC64) {
    const float f0 = acc[0] + (a.bias ? a.bias[0] : 0.f);
    const float f1 = acc[1] + (a.bias ? a.bias[1] : 0.f);
    const float2 rv = a.r[vox];
    float2 zv = make_float2(0.f, 0.f);
    if (a.sc->ok) zv = make_float2(fmaf(rv.x, a.sc->inv_s_f, f0), fmaf(rv.y, a.sc->inv_s_f, f1));
    a.z[vox] = zv;
    return;
  }
#pragma unroll
  for (int o = 0; o < kCh; o += 2) {
    float f0 = acc[o] + (a.bias ? a.bias[o] : 0.f);
    float f1 = acc[o + 1] + (a.bias ? a.bias[o + 1] : 0.f);
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

// block b's origin (z0, y0, x0)
__device__ __forceinline__ void tc_origin(const Vol& v, int b, int& z0, int& y0, int& x0) {
  const int nbx = (v.w + TBX - 1) / TBX, nby = (v.h + TBY - 1) / TBY;
  x0 = (b % nbx) * TBX;
  y0 = ((b / nbx) % nby) * TBY;
  z0 = (b / (nbx * nby)) * TBZ;
}

__global__ void __launch_bounds__(kTcThreads, 4) conv3d_tc_kernel(
    ConvArgs a, const __grid_constant__ CUtensorMap tm_lo, const __grid_constant__ CUtensorMap tm_hi,
    int* status, long long poll_limit) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  // bulk tensor copies need 128-byte aligned destinations: round up (the
  // launch reserves 128 extra bytes)
  const unsigned raw = smem_u32(smem_raw);
  unsigned char* xs = smem_raw + ((128u - (raw & 127u)) & 127u);  // [2][THZ][THY][THX] x 16 B
  unsigned char* ws = xs + size_t(kTcStageBytes);                  // [2][27][16] x 16 B
  __shared__ __align__(8) unsigned long long bars[2];             // halo landed, products done
  __shared__ uint32_t tmem_sh;
  const Vol& v = a.v;
  int z0, y0, x0;
  tc_origin(v, blockIdx.x, z0, y0, x0);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     smem_u32(&tmem_sh)),
                 "r"(kTcCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  const unsigned bar_x = smem_u32(&bars[0]), bar_p = smem_u32(&bars[1]);
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar_x) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar_p) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  // the halo: two bulk tensor copies (channel halves, zero outside the
  // volume), box origin (channel 0, x0 - 1, y0 - 1, z0 - 1)
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar_x),
                 "r"(unsigned(kTcStageBytes))
                 : "memory");
    const CUtensorMap* maps[2] = {&tm_lo, &tm_hi};
#pragma unroll
    for (int h = 0; h < 2; ++h)
      asm volatile(
          "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
          " [%0], [%1, {%2, %3, %4, %5}], [%6];\n" ::"r"(smem_u32(xs + h * kTcHalfBytes)),
          "l"(reinterpret_cast<unsigned long long>(maps[h])), "r"(0), "r"(x0 - 1), "r"(y0 - 1),
          "r"(z0 - 1), "r"(bar_x)
          : "memory");
  }
  // weights [tap][o][c] -> [half][tap][o] x 8 channels
  for (int i = threadIdx.x; i < kTaps * kCh * 2; i += blockDim.x) {
    const int half = i & 1, to = i >> 1;
    cp_async_16(ws + size_t(half * kTaps * kCh + to) * 16, a.wpk + to * kVS + half * 8, true);
  }
  cp_async_wait_all();
  bool ok = false;
  for (long long k = 0; k < poll_limit && !ok; ++k) ok = tc_mbar_try_wait(bar_x, 0);
  // the staged weights become visible to the tensor core (async proxy); the
  // tensor-memory address to every thread; one decision for the CTA
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  ok = __syncthreads_and(ok);
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = tmem_sh;
  bool issued = false;
  if (ok) {
    issued = true;
    if (threadIdx.x == 0) {
      // descriptors of tap 0 / tile 0; the start-address field (address / 16,
      // 14 bits, no carry for shared-memory addresses) takes each tap's and
      // tile's offset by a plain add of compile-time constants
      const uint64_t a0 = tc_desc(smem_u32(xs), kTcHalfBytes, THX * 16);
      const uint64_t b0 = tc_desc(smem_u32(ws), kTcWHalfBytes, 128);
#pragma unroll 1
      for (int tl = 0; tl < TBZ; ++tl) {
        const uint64_t a_tl = a0 + uint64_t(tl * THY * THX);  // (16-byte units)
        const uint32_t d = tmem + uint32_t(tl * 16);
#pragma unroll
        for (int tap = 0; tap < kTaps; ++tap) {
          const int tz = tap / 9, ty = (tap / 3) % 3, tx = tap % 3;
          tc_mma(d, a_tl + uint64_t((tz * THY + ty) * THX + tx), b0 + uint64_t(tap * kCh),
                 tap > 0 ? 1u : 0u);
        }
      }
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
              bar_p)
          : "memory");
    }
    bool done = false;
    for (long long k = 0; k < poll_limit && !done; ++k) done = tc_mbar_try_wait(bar_p, 0);
    ok = __syncthreads_and(done);
  }
  if (ok) {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const int row = 32 * (warp & 3) + lane;  // = y * 8 + x of a tile
    const int y = row >> 3, x = row & 7;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int tl = 2 * (warp >> 2) + j;
      float acc[16];
      tc_ld16(tmem + (uint32_t(32 * (warp & 3)) << 16) + uint32_t(tl * 16), acc);
      const int zz = z0 + tl, yy = y0 + y, xx = x0 + x;
      if (zz < v.d && yy < v.h && xx < v.w)
        conv_store_voxel(a, ((long long)zz * v.h + yy) * v.w + xx, acc);
    }
  } else {
    // a wait expired: record it, store nothing, give what is in flight (the
    // halo copy, the products) a last bounded chance before freeing
    if (threadIdx.x == 0 && status) atomicCAS(status, 0, NRSENSE_ERR_TIMEOUT);
    bool d = false;
    for (long long k = 0; k < kTcMaxPoll && !d; ++k) d = tc_mbar_try_wait(bar_x, 0);
    d = !issued;
    for (long long k = 0; k < kTcMaxPoll && !d; ++k) d = tc_mbar_try_wait(bar_p, 0);
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
                 "r"(kTcCols)
                 : "memory");
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
  bool tc = false;            // convolutions on tcgen05 (conv3d_tc_kernel), else mma.sync
  bool tc_ok = false;         // tensor maps of every activation buffer built
  int sms = 0;                // SMs of the device (persistent tcgen05 grid: two CTAs each)
  int* tc_status = nullptr;   // device status word of the tcgen05 convolutions' waits
  // per activation buffer that a convolution reads: its two channel-half
  // tensor maps (the halo's bulk tensor copies)
  struct ActMaps {
    const void* base;
    CUtensorMap half[2];
  };
  std::vector<ActMaps> act_maps;
  std::vector<void*> allocations;
};

namespace {

// creation (and configuration) numbers of networks: solver graphs key on them
uint64_t next_cnn_serial() {
  static std::atomic<uint64_t> next{1};
  return next.fetch_add(1);
}

int ew_grid(long long n) {
  return (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, 152LL * 16));
}

nrsense_status cuda_ok() {
  return cudaGetLastError() == cudaSuccess ? NRSENSE_OK : NRSENSE_ERR_CUDA;
}

// Two tensor maps per activation buffer [n][16 channels] (BF16): dimensions
// (8 channels, x, y, z) with strides (32 B, 32 W B, 32 H W B), the second map's
// base 16 bytes on (channels 8..15); box 8 x THX x THY x THZ, zero fill outside.
bool make_act_maps(nrsense_cnn_s* net, const void* base, nrsense_cnn_s::ActMaps* out) {
  const auto encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(nrs::tensor_map_encoder());
  if (encode == nullptr) return false;
  const Vol& v = net->vol;
  const cuuint64_t dims[4] = {8, cuuint64_t(v.w), cuuint64_t(v.h), cuuint64_t(v.d)};
  const cuuint64_t strides[3] = {cuuint64_t(kCh) * 2, cuuint64_t(v.w) * kCh * 2,
                                 cuuint64_t(v.h) * v.w * kCh * 2};
  const cuuint32_t box[4] = {8, cuuint32_t(THX), cuuint32_t(THY), cuuint32_t(THZ)};
  const cuuint32_t elem[4] = {1, 1, 1, 1};
  out->base = base;
  for (int h = 0; h < 2; ++h) {
    void* b = const_cast<char*>(static_cast<const char*>(base) + h * 16);
    if (encode(&out->half[h], CU_TENSOR_MAP_DATA_TYPE_UINT16, 4, b, dims, strides, box, elem,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return false;
  }
  return true;
}

// the maps of every buffer a convolution reads; tc_ok on success
void build_act_maps(nrsense_cnn_s* net) {
  std::vector<const void*> bufs;
  for (int l = 0; l < kLayers; ++l) bufs.push_back(net->act[l]);
  for (int k = 0; k < 3; ++k)
    if (net->gb[k]) bufs.push_back(net->gb[k]);
  if (net->h5) bufs.push_back(net->h5);
  for (int k = 0; k < 4; ++k)
    if (net->ut[k]) bufs.push_back(net->ut[k]);
  net->act_maps.clear();
  for (const void* b : bufs) {
    nrsense_cnn_s::ActMaps m;
    if (!make_act_maps(net, b, &m)) {
      net->act_maps.clear();
      net->tc_ok = false;
      return;
    }
    net->act_maps.push_back(m);
  }
  net->tc_ok = true;
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
  const nrsense_cnn_s::ActMaps* maps = nullptr;
  if (net->tc)
    for (const auto& m : net->act_maps)
      if (m.base == in) maps = &m;
  if (maps)
    conv3d_tc_kernel<<<tc_blocks(net->vol), kTcThreads, kTcSmem, s>>>(
        a, maps->half[0], maps->half[1], net->tc_status, kTcMaxPoll);
  else
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
  net->serial = next_cnn_serial();
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
      // three CTAs of 72.6 KB per SM need the largest shared-memory carveout
      cudaFuncSetAttribute(conv3d_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                           int(cudaSharedmemCarveoutMaxShared)) != cudaSuccess ||
      cudaFuncSetAttribute(conv3d_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)kTcSmem) != cudaSuccess ||
      cudaFuncSetAttribute(wgrad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)kWgSmem) != cudaSuccess) {
    cudaGetLastError();
    delete net;
    return NRSENSE_ERR_CUDA;
  }
  net->wg_grid = std::max(1, std::min(v.nblocks, sms));
  net->sms = sms;
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
  ok = ok && (net->tc_status = (int*)dalloc(net, sizeof(int))) != nullptr;
  if (!ok) {
    release(net);
    return NRSENSE_ERR_OOM;
  }
  build_act_maps(net);
  if (cudaMemsetAsync(net->wfwd, 0, size_t(kLayers) * kPack * sizeof(bf16), s) != cudaSuccess ||
      cudaMemsetAsync(net->wbwd, 0, size_t(kLayers) * kPack * sizeof(bf16), s) != cudaSuccess ||
      cudaMemsetAsync(net->sc, 0, sizeof(Scalars), s) != cudaSuccess ||
      cudaMemsetAsync(net->tc_status, 0, sizeof(int), s) != cudaSuccess) {
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

nrsense_status nrsense_cnn_set_conv(nrsense_cnn_t net, int32_t kind) {
  if (!net || (kind != NRSENSE_CNN_CONV_MMA && kind != NRSENSE_CNN_CONV_TCGEN05))
    return NRSENSE_ERR_ARG;
  const bool tc = kind == NRSENSE_CNN_CONV_TCGEN05;
  if (tc && !net->tc_ok) return NRSENSE_ERR_STATE;
  if (tc != net->tc) {
    net->tc = tc;
    net->serial = next_cnn_serial();  // graphs captured with the other kernel are re-captured
  }
  return NRSENSE_OK;
}

nrsense_status nrsense_cnn_device_status(nrsense_cnn_t net, int32_t clear, int32_t* out_host,
                                         void* stream) {
  if (!net || !out_host) return NRSENSE_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int v = 0;
  if (cudaMemcpyAsync(&v, net->tc_status, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return NRSENSE_ERR_CUDA;
  if (clear && v != 0 &&
      (cudaMemsetAsync(net->tc_status, 0, sizeof(int), s) != cudaSuccess ||
       cudaStreamSynchronize(s) != cudaSuccess))
    return NRSENSE_ERR_CUDA;
  *out_host = v;
  return NRSENSE_OK;
}

}  // extern "C"
