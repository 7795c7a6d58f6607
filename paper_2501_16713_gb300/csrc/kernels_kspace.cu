// k-space half of the nonrigid SENSE operator: coil sensitivities S and
// inverse k-space gridding G_j (section "k-space Gridding", inverse gridding
// diagram 1/c* -> Z -> F -> B^(k)) and the elementwise ends of k-space
// gridding G_j^H (F^H -> Z^H -> 1/c, then S^H).  Coil grids are coil-major
// ([C][G^3]) so that cuFFT transforms contiguous batches; coil maps keep the
// caller's (C, N^3) layout.
#include <cudaTypedefs.h>

#include <algorithm>

#include "plan_internal.h"

namespace nrs {

namespace {

// centred index n' = i - N/2 placed on the periodic G grid
__device__ __forceinline__ int centred_pos(int i, int N, int G) {
  const int c = i - (N >> 1);
  return c < 0 ? c + G : c;
}

struct VoxelPos {
  long long grid;  // linear index of the centred voxel on the G grid
  float deapod;    // 1/C3(n'/G)
};

__device__ __forceinline__ VoxelPos voxel_pos(const Geo& g, const float* __restrict__ dtab,
                                              long long idx) {
  const int i2 = int(idx % g.n2);
  const long long r = idx / g.n2;
  const int i1 = int(r % g.n1);
  const int i0 = int(r / g.n1);
  VoxelPos v;
  v.deapod = __ldg(dtab + i0) * __ldg(dtab + g.n0 + i1) * __ldg(dtab + g.n0 + g.n1 + i2);
  v.grid = ((long long)centred_pos(i0, g.n0, g.g0) * g.g1 + centred_pos(i1, g.n1, g.g1)) * g.g2 +
           centred_pos(i2, g.n2, g.g2);
  return v;
}

// K5: v_{j,c}[n'] = S_c[n] m_j[n] / C3(n'/G) written into the centred N^3 block
// of the zero-padded coil grids (steps S, 1/c* and Z), for the nph phases of
// a chunk at once.  Thread = (phase, coil, voxel); grid slot of (phase jj,
// coil c) is jj * C + c.
template <typename GT>
__global__ void coil_fanout_pad_kernel(Geo g, int C, int nph, const float* __restrict__ dtab,
                                       const float2* __restrict__ smaps,  // [C][nvox]
                                       const float2* __restrict__ m,      // [nph][nvox]
                                       GT* __restrict__ xpad) {           // [nph*C][G^3]
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= g.nvox * C * nph) return;
  const long long sc = t / g.nvox;  // jj * C + c
  const int c = int(sc % C);
  const long long jj = sc / C;
  const long long idx = t - sc * g.nvox;
  const VoxelPos vp = voxel_pos(g, dtab, idx);
  const float2 mv = __ldg(m + jj * g.nvox + idx);
  const float2 sv = __ldg(smaps + (long long)c * g.nvox + idx);
  const float w = vp.deapod;
  grid_st(xpad + sc * g.ngrid + vp.grid,
          make_float2((sv.x * mv.x - sv.y * mv.y) * w, (sv.x * mv.y + sv.y * mv.x) * w));
}

// Stage variant of K5 without S: coil images v (C, N^3) -> padded grids.
template <typename GT>
__global__ void image_to_padded_kernel(Geo g, int C, const float* __restrict__ dtab,
                                       const float2* __restrict__ v, GT* __restrict__ xpad) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= g.nvox * C) return;
  const int c = int(t / g.nvox);
  const long long idx = t - (long long)c * g.nvox;
  const VoxelPos vp = voxel_pos(g, dtab, idx);
  const float2 vv = __ldg(v + t);
  grid_st(xpad + (long long)c * g.ngrid + vp.grid, make_float2(vv.x * vp.deapod, vv.y * vp.deapod));
}

// K6: y_{j,s,c} = sum_taps c3(q_s - g) X_{j,c}[g] (Backprojection Core B^(k)).
// CTA = one 8^3 tile and the sorted samples whose first tap lies in it: the
// tile plus its (W-1)-point upper halo of CC coil grids is staged once into
// shared memory with asynchronous copies, coil-interleaved ([z][y][x][c]).
// A group of W*CC/2 lanes serves one sample: lane = (tap x, coil pair), so a
// quarter-warp reads 128 contiguous bytes of one tap row (no bank
// conflicts); each lane evaluates only its own tap's weights (coefficients
// in shared memory), gets the other axes' by shuffles, and the tap-x partial
// sums are reduced by shuffles at the end.
template <int W, int CC, typename GT>
__global__ void __launch_bounds__(256) interp_tile_kernel(
    Geo g, KernelCoefs kc, int C, TilePlan tp, PhaseTable pt, const GT* __restrict__ grids,
    float2* __restrict__ y) {
  constexpr int T = 8, H = T + W - 1, H3 = H * H * H;
  constexpr int NQ = CC / 2, LPS = W * NQ, SPW = 32 / LPS;  // lanes/sample, samples/warp
  extern __shared__ float4 smem_raw[];
  GT* halo = reinterpret_cast<GT*>(smem_raw);  // [H][H][H][CC] stored values
  __shared__ float s_coef[W][kNumCoef];
  const int jj = phase_of(pt.item0, pt.nphase, blockIdx.x);
  const SpreadItem it = pt.items[jj][blockIdx.x - pt.item0[jj]];
  const float4* __restrict__ qs = pt.qs[jj];
  const int32_t* __restrict__ perm = pt.perm[jj];
  const GT* __restrict__ grid = grids + (long long)jj * C * g.ngrid;
  const long long row0 = pt.row0[jj];
  const int coil0 = blockIdx.y * CC;
  const int tz = it.tile / (tp.nt1 * tp.nt2);
  const int rem = it.tile - tz * (tp.nt1 * tp.nt2);
  const int ty = rem / tp.nt2;
  const int tx = rem - ty * tp.nt2;
  const int o0 = tz * T, o1 = ty * T, o2 = tx * T;
  if (threadIdx.x < W * kNumCoef) s_coef[threadIdx.x / kNumCoef][threadIdx.x % kNumCoef] =
      kc.c[threadIdx.x / kNumCoef][threadIdx.x % kNumCoef];
  // stage: lanes walk (coil, x) with the coil fastest, so shared writes are
  // contiguous and each global sector (4 consecutive x of one coil) is fully used
  for (int i = threadIdx.x; i < CC * H3; i += blockDim.x) {
    const int c = i % CC;
    const int r = i / CC;
    const int z = r / (H * H), yy = (r / H) % H, x = r % H;
    const int gz = wrap_once(o0 + z, g.g0), gy = wrap_once(o1 + yy, g.g1),
              gx = wrap_once(o2 + x, g.g2);
    const bool valid = coil0 + c < C;
    const GT* src =
        grid + (valid ? (long long)(coil0 + c) * g.ngrid + ((long long)gz * g.g1 + gy) * g.g2 + gx
                      : 0);
    cp_async_grid(halo + r * CC + c, src, valid);
  }
  cp_async_wait_all();
  __syncthreads();

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int grp = lane / LPS;                 // sample slot in the warp
  const int gl = lane - grp * LPS;            // lane in the group
  const int q = gl % NQ, txl = gl / NQ;       // coil pair, tap x
  const int gbase = grp * LPS;
  const bool active_lane = grp < SPW;
  const int nwarps = blockDim.x >> 5;
  // polynomial coefficients of this lane's tap (fixed per lane)
  float cf[kNumCoef];
#pragma unroll
  for (int k = 0; k < kNumCoef; ++k) cf[k] = s_coef[txl][k];
  for (int s0 = it.begin + warp * SPW; s0 < it.end; s0 += nwarps * SPW) {
    const int s = s0 + grp;
    const bool live = active_lane && s < it.end;
    float4 qv = make_float4(0.f, 0.f, 0.f, 0.f);
    int l0 = 0, l1 = 0, l2 = 0;
    if (live) {
      qv = __ldg(qs + s);
      int b0, b1, b2;
      unpack_base(__float_as_uint(qv.w), b0, b1, b2);
      l0 = min(max(b0 - o0, 0), T - 1);  // in range for a well-formed plan
      l1 = min(max(b1 - o1, 0), T - 1);
      l2 = min(max(b2 - o2, 0), T - 1);
    }
    // this lane's tap txl on each axis
    float w0t = 0.f, w1t = 0.f, w2t = 0.f;
    {
      const float s0f = fmaf(2.f, qv.x, -1.f), s1f = fmaf(2.f, qv.y, -1.f),
                  s2f = fmaf(2.f, qv.z, -1.f);
      float a0 = cf[kNumCoef - 1], a1 = a0, a2 = a0;
#pragma unroll
      for (int k = kNumCoef - 2; k >= 0; --k) {
        const float ck = cf[k];
        a0 = fmaf(a0, s0f, ck);
        a1 = fmaf(a1, s1f, ck);
        a2 = fmaf(a2, s2f, ck);
      }
      w0t = a0;
      w1t = a1;
      w2t = a2;
    }
    float w0[W], w1[W];
#pragma unroll
    for (int t = 0; t < W; ++t) {
      w0[t] = __shfl_sync(0xffffffffu, w0t, gbase + t * NQ);
      w1[t] = __shfl_sync(0xffffffffu, w1t, gbase + t * NQ);
    }
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    if (live) {
      const GT* base = halo + ((l0 * H + l1) * H + l2 + txl) * CC + 2 * q;
#pragma unroll
      for (int t0 = 0; t0 < W; ++t0) {
        const float w02 = w0[t0] * w2t;
#pragma unroll
        for (int t1 = 0; t1 < W; ++t1) {
          const float w = w02 * w1[t1];
          const float4 v = grid_ld2_shared(base + ((t0 * H + t1) * H) * CC);
          acc.x = fmaf(w, v.x, acc.x);
          acc.y = fmaf(w, v.y, acc.y);
          acc.z = fmaf(w, v.z, acc.z);
          acc.w = fmaf(w, v.w, acc.w);
        }
      }
    }
    // reduce over tap x (lanes NQ apart within the group)
#pragma unroll
    for (int off = NQ; off < LPS; off <<= 1) {
      if ((W & (W - 1)) == 0) {
        acc.x += __shfl_xor_sync(0xffffffffu, acc.x, off);
        acc.y += __shfl_xor_sync(0xffffffffu, acc.y, off);
        acc.z += __shfl_xor_sync(0xffffffffu, acc.z, off);
        acc.w += __shfl_xor_sync(0xffffffffu, acc.w, off);
      }
    }
    if constexpr ((W & (W - 1)) != 0) {
      // W not a power of two: gather the tap-x partials explicitly
      float4 sum = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int t = 0; t < W; ++t) {
        sum.x += __shfl_sync(0xffffffffu, acc.x, gbase + t * NQ + q);
        sum.y += __shfl_sync(0xffffffffu, acc.y, gbase + t * NQ + q);
        sum.z += __shfl_sync(0xffffffffu, acc.z, gbase + t * NQ + q);
        sum.w += __shfl_sync(0xffffffffu, acc.w, gbase + t * NQ + q);
      }
      acc = sum;
    }
    if (live && txl == 0) {
      const int c0 = coil0 + 2 * q;
      float2* out = y + (row0 + __ldg(perm + s)) * C + c0;
      if ((C & 1) == 0 && c0 + 1 < C) {
        reinterpret_cast<float4*>(out)[0] = acc;
      } else {
        if (c0 < C) out[0] = make_float2(acc.x, acc.y);
        if (c0 + 1 < C) out[1] = make_float2(acc.z, acc.w);
      }
    }
  }
}

// K6 with the tile halo loaded by the tensor memory accelerator (W = 4).
// One cp.async.bulk.tensor copy per CTA moves the (8+3)^3 halo of CC coil
// grids (box x extent 12 for 16-byte rows) into shared memory as
// [c][z][y][x]; an mbarrier tracks the transaction bytes and every thread
// waits on it with a bounded poll (on expiry the CTA records
// NRSENSE_ERR_TIMEOUT, waits again, bounded, for its copy in flight to land
// in shared memory, and returns without computing).  The first limit is the
// caller's (at most kTmaMaxPoll polls; a test sets 0 to make it expire).  Tiles whose halo wraps
// the periodic grid edge are staged by per-value asynchronous copies into the
// same layout.  A group of W * CC lanes serves one sample: lane = (tap x,
// coil), so the CC coils of one tap read distinct banks; tap-x partial sums
// are reduced by shuffles.
constexpr int kTmaXP = 12;                 // box x extent (12 values = 96 / 48 bytes)
constexpr long long kTmaMaxPoll = 1LL << 24;

__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ bool mbar_try_wait(unsigned mbar, unsigned parity) {
  unsigned done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(mbar), "r"(parity)
      : "memory");
  return done != 0;
}

template <int CC, typename GT>
__global__ void __launch_bounds__(256, CC == 2 ? 6 : CC == 4 ? 4 : 1) interp_tma_kernel(
    const __grid_constant__ CUtensorMap tmap, Geo g, KernelCoefs kc, int C, TilePlan tp,
    PhaseTable pt, const GT* __restrict__ grids, float2* __restrict__ y,
    int32_t* __restrict__ status, long long poll_limit) {
  constexpr int W = 4, T = 8, H = T + W - 1, XP = kTmaXP;
  constexpr int LPS = W * CC, SPW = 32 / LPS;  // lanes per sample, samples per warp
  static_assert(LPS <= 32, "coil chunk");
  constexpr unsigned kBytes = unsigned(CC * H * H * XP * sizeof(GT));
  extern __shared__ float4 smem_raw[];
  // the bulk tensor copy needs a 128-byte aligned destination: round up
  // (the launch reserves 128 extra bytes)
  const unsigned raw = smem_addr(smem_raw);
  GT* halo = reinterpret_cast<GT*>(reinterpret_cast<unsigned char*>(smem_raw) +
                                   ((128u - (raw & 127u)) & 127u));  // [CC][H][H][XP]
  __shared__ float s_coef[W][kNumCoef];
  // per warp and sample slot: the sample's tap weights of axes 0, 1, 2 (CC >= 4)
  __shared__ __align__(16) float4 s_wrec[8][CC >= 4 ? SPW : 1][3];
  __shared__ __align__(8) unsigned long long mbar;
  const int jj = phase_of(pt.item0, pt.nphase, blockIdx.x);
  const SpreadItem it = pt.items[jj][blockIdx.x - pt.item0[jj]];
  const float4* __restrict__ qs = pt.qs[jj];
  const int32_t* __restrict__ perm = pt.perm[jj];
  const GT* __restrict__ grid = grids + (long long)jj * C * g.ngrid;
  const long long row0 = pt.row0[jj];
  const int coil0 = blockIdx.y * CC;
  const int tz = it.tile / (tp.nt1 * tp.nt2);
  const int rem = it.tile - tz * (tp.nt1 * tp.nt2);
  const int ty = rem / tp.nt2;
  const int tx = rem - ty * tp.nt2;
  const int o0 = tz * T, o1 = ty * T, o2 = tx * T;
  if (threadIdx.x < W * kNumCoef) s_coef[threadIdx.x / kNumCoef][threadIdx.x % kNumCoef] =
      kc.c[threadIdx.x / kNumCoef][threadIdx.x % kNumCoef];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int grp = lane / LPS;          // sample slot in the warp
  const int gl = lane - grp * LPS;     // lane in the group
  const int c = gl % CC, txl = gl / CC;
  const int gbase = grp * LPS;
  const bool active_lane = grp < SPW;
  const int nwarps = blockDim.x >> 5;
  const int stride = nwarps * SPW;
  // the first sample's position record and output row, loaded while the
  // halo is in flight; each iteration then loads the next one's
  float4 q_next = make_float4(0.f, 0.f, 0.f, 0.f);
  int row_next = 0;
  {
    const int s = it.begin + warp * SPW + grp;
    if (active_lane && s < it.end) {
      q_next = __ldg(qs + s);
      row_next = __ldg(perm + s);
    }
  }
  const bool use_tma = o0 + H <= g.g0 && o1 + H <= g.g1 && o2 + XP <= g.g2;
  if (use_tma) {
    const unsigned mb = smem_addr(&mbar);
    if (threadIdx.x == 0) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mb) : "memory");
      asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(mb),
                   "r"(kBytes)
                   : "memory");
      // box origin (x, y, z, grid slot); x * sizeof(GT) is a multiple of 16
      asm volatile(
          "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
          " [%0], [%1, {%2, %3, %4, %5}], [%6];\n" ::"r"(smem_addr(halo)),
          "l"(reinterpret_cast<unsigned long long>(&tmap)), "r"(o2), "r"(o1), "r"(o0),
          "r"(jj * C + coil0), "r"(mb)
          : "memory");
    }
    bool ok = false;
    for (long long k = 0; k < poll_limit && !ok; ++k) ok = mbar_try_wait(mb, 0);
    // one decision for the whole CTA: the warps below use full-warp shuffles
    if (!__syncthreads_and(ok)) {
      if (threadIdx.x == 0 && status) atomicCAS(status, 0, NRSENSE_ERR_TIMEOUT);
      // give the copy in flight a last bounded chance to land before leaving
      for (long long k = 0; k < kTmaMaxPoll && !ok; ++k) ok = mbar_try_wait(mb, 0);
      return;
    }
  } else {
    // wrapped halo: per-value copies into the same [c][z][y][x] layout
    for (int i = threadIdx.x; i < CC * H * H * H; i += blockDim.x) {
      const int x = i % H;
      const int r = i / H;
      const int yy = r % H, z = (r / H) % H, c = r / (H * H);
      const int gz = wrap_once(o0 + z, g.g0), gy = wrap_once(o1 + yy, g.g1),
                gx = wrap_once(o2 + x, g.g2);
      const bool valid = coil0 + c < C;
      const GT* src =
          grid + (valid ? (long long)(coil0 + c) * g.ngrid + ((long long)gz * g.g1 + gy) * g.g2 + gx
                        : 0);
      cp_async_grid(halo + ((c * H + z) * H + yy) * XP + x, src, valid);
    }
    cp_async_wait_all();
    __syncthreads();
  }

  // polynomial coefficients of this lane's tap (fixed per lane)
  float cf[kNumCoef];
#pragma unroll
  for (int k = 0; k < kNumCoef; ++k) cf[k] = s_coef[txl][k];
  for (int s0 = it.begin + warp * SPW; s0 < it.end; s0 += stride) {
    const int s = s0 + grp;
    const bool live = active_lane && s < it.end;
    const float4 qv = q_next;
    const int row = row_next;
    if (active_lane && s + stride < it.end) {
      q_next = __ldg(qs + s + stride);
      row_next = __ldg(perm + s + stride);
    }
    // first tap relative to the tile: a sample belongs to the tile of its first
    // tap and tiles are 8-aligned, so this is b mod 8 (and stays inside the
    // halo for any record; dead lanes compute on in-range garbage and do not
    // store)
    const uint32_t pk = __float_as_uint(qv.w);
    const int l0 = int(pk >> 20) & (T - 1), l1 = int(pk >> 10) & (T - 1), l2 = int(pk) & (T - 1);
    // kernel weights of the sample: axis a at tap t
    float w0[W], w1[W], w2t;
    if constexpr (CC >= 4) {
      // lane (txl, c) evaluates axis min(c, 2) at tap txl; lanes c <= 2 put
      // their value in the sample's weight record in shared memory and every
      // lane reads the taps it needs (three broadcast loads: shuffles would
      // take nine passes of the shared-memory data path the tap reads use;
      // the same values as evaluating all three here)
      const float f = c == 0 ? qv.x : (c == 1 ? qv.y : qv.z);
      const float sf = fmaf(2.f, f, -1.f);
      float a = cf[kNumCoef - 1];
#pragma unroll
      for (int k = kNumCoef - 2; k >= 0; --k) a = fmaf(a, sf, cf[k]);
      float4* sw = s_wrec[warp][active_lane ? grp : 0];
      __syncwarp();  // the previous sample's record has been read
      if (active_lane && c <= 2) reinterpret_cast<float*>(&sw[c])[txl] = a;
      __syncwarp();
      const float4 v0 = sw[0], v1 = sw[1];
      w0[0] = v0.x;
      w0[1] = v0.y;
      w0[2] = v0.z;
      w0[3] = v0.w;
      w1[0] = v1.x;
      w1[1] = v1.y;
      w1[2] = v1.z;
      w1[3] = v1.w;
      w2t = reinterpret_cast<const float*>(&sw[2])[txl];
    } else {
      // this lane's tap txl on each axis
      const float s0f = fmaf(2.f, qv.x, -1.f), s1f = fmaf(2.f, qv.y, -1.f),
                  s2f = fmaf(2.f, qv.z, -1.f);
      float a0 = cf[kNumCoef - 1], a1 = a0, a2 = a0;
#pragma unroll
      for (int k = kNumCoef - 2; k >= 0; --k) {
        const float ck = cf[k];
        a0 = fmaf(a0, s0f, ck);
        a1 = fmaf(a1, s1f, ck);
        a2 = fmaf(a2, s2f, ck);
      }
      w2t = a2;
#pragma unroll
      for (int t = 0; t < W; ++t) {
        w0[t] = __shfl_sync(0xffffffffu, a0, gbase + t * CC);
        w1[t] = __shfl_sync(0xffffffffu, a1, gbase + t * CC);
      }
    }
    float2 acc = make_float2(0.f, 0.f);
    {
      const GT* base = halo + ((c * H + l0) * H + l1) * XP + l2 + txl;
#pragma unroll
      for (int t0 = 0; t0 < W; ++t0) {
        const float w02 = w0[t0] * w2t;
#pragma unroll
        for (int t1 = 0; t1 < W; ++t1) {
          const float w = w02 * w1[t1];
          const float2 v = grid_ld_shared(base + (t0 * H + t1) * XP);
          // real and imaginary part in one paired FMA (each part rounded as fmaf)
          acc = __ffma2_rn(make_float2(w, w), v, acc);
        }
      }
    }
    // reduce over tap x (lanes CC apart within the group)
#pragma unroll
    for (int off = CC; off < LPS; off <<= 1)
      acc = __fadd2_rn(acc, make_float2(__shfl_xor_sync(0xffffffffu, acc.x, off),
                                        __shfl_xor_sync(0xffffffffu, acc.y, off)));
    if (live && txl == 0 && coil0 + c < C) y[(row0 + row) * C + coil0 + c] = acc;
  }
}

template <int CC, typename GT>
constexpr size_t interp_tma_smem() {  // halo + alignment slack
  return size_t(CC) * (8 + 3) * (8 + 3) * kTmaXP * sizeof(GT) + 128;
}

template <int W, int CC, typename GT>
constexpr size_t interp_smem() {
  return size_t(8 + W - 1) * (8 + W - 1) * (8 + W - 1) * CC * sizeof(GT);
}

// K8: w_j[n] = sum_c conj(S_c[n]) Xt_c[n' mod G] / C3(n'/G) (steps Z^H, 1/c of
// k-space gridding, then S^H), for the nph phases of a chunk.  Thread = (phase, voxel).
template <typename GT>
__global__ void crop_coilsum_kernel(Geo g, int C, int nph, const float* __restrict__ dtab,
                                    const float2* __restrict__ smaps,  // [C][nvox]
                                    const GT* __restrict__ xg,         // [nph*C][G^3]
                                    float2* __restrict__ w) {          // [nph][nvox]
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= g.nvox * nph) return;
  const long long jj = t / g.nvox;
  const long long idx = t - jj * g.nvox;
  const VoxelPos vp = voxel_pos(g, dtab, idx);
  const GT* xs = xg + jj * C * g.ngrid + vp.grid;
  float ar = 0.f, ai = 0.f;
  for (int c = 0; c < C; ++c) {
    const float2 s = __ldg(smaps + (long long)c * g.nvox + idx);
    const float2 v = grid_ld(xs + (long long)c * g.ngrid);
    ar = fmaf(s.x, v.x, fmaf(s.y, v.y, ar));
    ai = fmaf(s.x, v.y, fmaf(-s.y, v.x, ai));
  }
  w[t] = make_float2(ar * vp.deapod, ai * vp.deapod);
}

// Stage variant of K8 without S^H: padded grids -> coil images (C, N^3).
template <typename GT>
__global__ void crop_to_coils_kernel(Geo g, int C, const float* __restrict__ dtab,
                                     const GT* __restrict__ xg, float2* __restrict__ v) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= g.nvox * C) return;
  const int c = int(t / g.nvox);
  const long long idx = t - (long long)c * g.nvox;
  const VoxelPos vp = voxel_pos(g, dtab, idx);
  const float2 x = grid_ld(xg + (long long)c * g.ngrid + vp.grid);
  v[t] = make_float2(x.x * vp.deapod, x.y * vp.deapod);
}

inline unsigned blocks_for(long long n, int threads) {
  return unsigned((n + threads - 1) / threads);
}

}  // namespace

int launch_coil_fanout_pad(const Geo& g, int C, int nph, const float* deapod,
                           const nrsense_c64* smaps, const nrsense_c64* m, void* xpad, bool bf16,
                           cudaStream_t s) {
  const auto* sm = reinterpret_cast<const float2*>(smaps);
  const auto* mm = reinterpret_cast<const float2*>(m);
  const unsigned nb = blocks_for(g.nvox * C * nph, 256);
  if (bf16)
    coil_fanout_pad_kernel<<<nb, 256, 0, s>>>(g, C, nph, deapod, sm, mm, static_cast<bf162*>(xpad));
  else
    coil_fanout_pad_kernel<<<nb, 256, 0, s>>>(g, C, nph, deapod, sm, mm, static_cast<float2*>(xpad));
  return 1;
}

int launch_image_to_padded(const Geo& g, int C, const float* deapod, const nrsense_c64* v,
                           void* xpad, bool bf16, cudaStream_t s) {
  const auto* vv = reinterpret_cast<const float2*>(v);
  const unsigned nb = blocks_for(g.nvox * C, 256);
  if (bf16)
    image_to_padded_kernel<<<nb, 256, 0, s>>>(g, C, deapod, vv, static_cast<bf162*>(xpad));
  else
    image_to_padded_kernel<<<nb, 256, 0, s>>>(g, C, deapod, vv, static_cast<float2*>(xpad));
  return 1;
}

namespace {
template <int CC, typename GT>
cudaError_t set_tma_smem() {
  return cudaFuncSetAttribute(interp_tma_kernel<CC, GT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              int(interp_tma_smem<CC, GT>()));
}

template <int W, int CC, typename GT>
cudaError_t set_interp_smem() {
  return cudaFuncSetAttribute(interp_tile_kernel<W, CC, GT>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                              int(interp_smem<W, CC, GT>()));
}

template <typename GT>
void interp_dispatch(const Geo& g, int W, const KernelCoefs& kc, int C, const TilePlan& tp,
                     const PhaseTable& pt, const GT* gp, float2* yp, int nitems, int coil_chunk,
                     cudaStream_t s) {
  if (W == 4 && C > 4 && coil_chunk == 8) {  // per-value staging: 8 or 4 coils
    const dim3 gd(nitems, (C + 7) / 8);
    interp_tile_kernel<4, 8, GT><<<gd, 256, interp_smem<4, 8, GT>(), s>>>(g, kc, C, tp, pt, gp, yp);
  } else if (W == 4) {
    interp_tile_kernel<4, 4, GT><<<dim3(nitems, (C + 3) / 4), 256, interp_smem<4, 4, GT>(), s>>>(
        g, kc, C, tp, pt, gp, yp);
  } else {
    const dim3 gd(nitems, (C + 3) / 4);
    interp_tile_kernel<6, 4, GT><<<gd, 256, interp_smem<6, 4, GT>(), s>>>(g, kc, C, tp, pt, gp, yp);
  }
}
}  // namespace

cudaError_t configure_kernels() {
  cudaError_t e = configure_spread_kernels();
  if (e == cudaSuccess) e = set_interp_smem<4, 8, float2>();
  if (e == cudaSuccess) e = set_interp_smem<4, 4, float2>();
  if (e == cudaSuccess) e = set_interp_smem<6, 4, float2>();
  if (e == cudaSuccess) e = set_interp_smem<4, 8, bf162>();
  if (e == cudaSuccess) e = set_interp_smem<4, 4, bf162>();
  if (e == cudaSuccess) e = set_interp_smem<6, 4, bf162>();
  if (e == cudaSuccess) e = set_tma_smem<4, float2>();
  if (e == cudaSuccess) e = set_tma_smem<8, float2>();
  if (e == cudaSuccess) e = set_tma_smem<4, bf162>();
  if (e == cudaSuccess) e = set_tma_smem<8, bf162>();
  if (e == cudaSuccess) e = set_tma_smem<2, float2>();
  if (e == cudaSuccess) e = set_tma_smem<2, bf162>();
  return e;
}

void* tensor_map_encoder() {
  static void* fn = nullptr;
  if (fn == nullptr) {
    cudaDriverEntryPointQueryResult q;
    void* f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || f == nullptr) {
      cudaGetLastError();
      return nullptr;
    }
    fn = f;
  }
  return fn;
}

bool make_grid_tensor_map(CUtensorMap* m, const void* base, const Geo& g, long long slots,
                          bool bf16, int coil_chunk) {
  const auto encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(tensor_map_encoder());
  if (encode == nullptr) return false;
  const cuuint64_t esz = bf16 ? 4 : 8;
  // x innermost; strides in bytes for dimensions 1..3 (multiples of 16)
  const cuuint64_t dims[4] = {cuuint64_t(g.g2), cuuint64_t(g.g1), cuuint64_t(g.g0),
                              cuuint64_t(slots)};
  const cuuint64_t strides[3] = {cuuint64_t(g.g2) * esz, cuuint64_t(g.g1) * g.g2 * esz,
                                 cuuint64_t(g.ngrid) * esz};
  for (int k = 0; k < 3; ++k)
    if (strides[k] % 16) return false;
  const cuuint32_t box[4] = {cuuint32_t(kTmaXP), 11u, 11u, cuuint32_t(coil_chunk)};
  const cuuint32_t elem[4] = {1, 1, 1, 1};
  const CUresult r = encode(m, bf16 ? CU_TENSOR_MAP_DATA_TYPE_UINT32 : CU_TENSOR_MAP_DATA_TYPE_UINT64,
                            4, const_cast<void*>(base), dims, strides, box, elem,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

int launch_interp_kspace(const Geo& g, int W, const KernelCoefs& kc, int C, const TilePlan& tp,
                         const PhaseTable& pt, const void* grids, bool bf16, nrsense_c64* y,
                         int coil_chunk, const CUtensorMap* tmap, int32_t* status,
                         cudaStream_t s, long long poll_limit) {
  const int nitems = pt.item0[pt.nphase];
  if (nitems == 0) return 0;
  auto* yp = reinterpret_cast<float2*>(y);
  const long long lim = poll_limit < 0 ? kTmaMaxPoll : std::min(poll_limit, kTmaMaxPoll);
  if (tmap != nullptr && W == 4) {
    // the tensor map's coil box must match: 8 (C > 4), 2, else 4
    const int cc = (coil_chunk == 8 && C > 4) ? 8 : coil_chunk == 2 ? 2 : 4;
    const dim3 gd(nitems, (C + cc - 1) / cc);
    if (bf16) {
      const auto* gp = static_cast<const bf162*>(grids);
      if (cc == 8)
        interp_tma_kernel<8, bf162><<<gd, 256, interp_tma_smem<8, bf162>(), s>>>(
            *tmap, g, kc, C, tp, pt, gp, yp, status, lim);
      else if (cc == 2)
        interp_tma_kernel<2, bf162><<<gd, 256, interp_tma_smem<2, bf162>(), s>>>(
            *tmap, g, kc, C, tp, pt, gp, yp, status, lim);
      else
        interp_tma_kernel<4, bf162><<<gd, 256, interp_tma_smem<4, bf162>(), s>>>(
            *tmap, g, kc, C, tp, pt, gp, yp, status, lim);
    } else {
      const auto* gp = static_cast<const float2*>(grids);
      if (cc == 8)
        interp_tma_kernel<8, float2><<<gd, 256, interp_tma_smem<8, float2>(), s>>>(
            *tmap, g, kc, C, tp, pt, gp, yp, status, lim);
      else if (cc == 2)
        interp_tma_kernel<2, float2><<<gd, 256, interp_tma_smem<2, float2>(), s>>>(
            *tmap, g, kc, C, tp, pt, gp, yp, status, lim);
      else
        interp_tma_kernel<4, float2><<<gd, 256, interp_tma_smem<4, float2>(), s>>>(
            *tmap, g, kc, C, tp, pt, gp, yp, status, lim);
    }
    return 1;
  }
  if (bf16)
    interp_dispatch(g, W, kc, C, tp, pt, static_cast<const bf162*>(grids), yp, nitems, coil_chunk,
                    s);
  else
    interp_dispatch(g, W, kc, C, tp, pt, static_cast<const float2*>(grids), yp, nitems,
                    coil_chunk, s);
  return 1;
}

int launch_crop_coilsum(const Geo& g, int C, int nph, const float* deapod,
                        const nrsense_c64* smaps, const void* xg, bool bf16, nrsense_c64* w,
                        cudaStream_t s) {
  const auto* sm = reinterpret_cast<const float2*>(smaps);
  auto* wp = reinterpret_cast<float2*>(w);
  const unsigned nb = blocks_for(g.nvox * nph, 256);
  if (bf16)
    crop_coilsum_kernel<<<nb, 256, 0, s>>>(g, C, nph, deapod, sm, static_cast<const bf162*>(xg), wp);
  else
    crop_coilsum_kernel<<<nb, 256, 0, s>>>(g, C, nph, deapod, sm, static_cast<const float2*>(xg), wp);
  return 1;
}

int launch_crop_to_coils(const Geo& g, int C, const float* deapod, const void* xg, bool bf16,
                         nrsense_c64* v, cudaStream_t s) {
  auto* vp = reinterpret_cast<float2*>(v);
  const unsigned nb = blocks_for(g.nvox * C, 256);
  if (bf16)
    crop_to_coils_kernel<<<nb, 256, 0, s>>>(g, C, deapod, static_cast<const bf162*>(xg), vp);
  else
    crop_to_coils_kernel<<<nb, 256, 0, s>>>(g, C, deapod, static_cast<const float2*>(xg), vp);
  return 1;
}

}  // namespace nrs
