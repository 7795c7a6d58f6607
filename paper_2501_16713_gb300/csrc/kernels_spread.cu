// Projection Cores P^(k) (k-space gridding) and P_j^(i) (adjoint image-space
// gridding): spread point values onto the oversampled grid,
//     grid[c][g] = sum_p c3(q_p - g) vals[p, c]
// (section "k-space Gridding", Projection Core; section "Image-space
// Gridding", adjoint diagram).
//
// Output-stationary and atomic-free: each CTA owns one grid tile (and a chunk
// of coils), reads the plan-time list of points whose W^3 footprint touches
// the tile, and accumulates in shared memory.  Every tile plane (axis 0) is
// owned by one warp (or half-warp).  The plan sorts each tile's list by the
// plane offset of the point's first tap, so the owner of a plane visits the
// points that touch it as one contiguous range; every shared-memory address
// is updated by one warp only, in list order, so the result is bitwise
// deterministic.  A heavy tile is split over several CTAs that write partial
// tiles to scratch; a second kernel adds the partials in a fixed order.
//
// Storage and accumulation variants: the k-space coil grids are stored as
// complex FP32 or complex BF16 (accumulation is FP32 in shared memory either
// way); the W = 4 kernels optionally accumulate with an error-free
// transformation (compensated summation: the rounding error of every product
// (FMA residual) and of every addition (TwoSum) is summed in a companion
// array and added at write-out), which removes the growth of the
// accumulation error with the number of points per grid value.
#include "plan_internal.h"

namespace nrs {

namespace {

constexpr int kThreads = 256;

struct TileOrigin {
  int o0, o1, o2, e0, e1, e2;
};

__device__ __forceinline__ TileOrigin tile_origin(const Geo& g, const TilePlan& tp, int tile) {
  const int tz = tile / (tp.nt1 * tp.nt2);
  const int rem = tile - tz * (tp.nt1 * tp.nt2);
  const int ty = rem / tp.nt2;
  const int tx = rem - ty * tp.nt2;
  TileOrigin t;
  t.o0 = tz * tp.t0;
  t.o1 = ty * tp.t1;
  t.o2 = tx * tp.t2;
  t.e0 = min(tp.t0, g.g0 - t.o0);
  t.e1 = min(tp.t1, g.g1 - t.o1);
  t.e2 = min(tp.t2, g.g2 - t.o2);
  return t;
}

// Stage `cnt` list entries: per-axis weights, first-tap offsets from the tile
// origin (in (-W, T)), and CC values.
template <int W, int T, int CC, int R>
__device__ __forceinline__ void stage_round(const Geo& g, const KernelCoefs& kc, int C, int coil0,
                                            const TileOrigin& to, const int2* __restrict__ lst,
                                            int cnt, const float4* __restrict__ qs,
                                            const float2* __restrict__ vals, long long row0,
                                            float (*s_w)[3][W], int (*s_r)[3], float2 (*s_val)[CC],
                                            int tid) {
  for (int i = tid; i < cnt * 3; i += kThreads) {
    const int p = i / 3, a = i - 3 * p;
    const int si = __ldg(&lst[p].x);
    const float4 q = __ldg(qs + si);
    int b0, b1, b2;
    unpack_base(__float_as_uint(q.w), b0, b1, b2);
    float w[W];
    kernel_weights<W>(a == 0 ? q.x : (a == 1 ? q.y : q.z), kc, w);
#pragma unroll
    for (int t = 0; t < W; ++t) s_w[p][a][t] = w[t];
    const int Ga = a == 0 ? g.g0 : (a == 1 ? g.g1 : g.g2);
    int r = a == 0 ? b0 - to.o0 : (a == 1 ? b1 - to.o1 : b2 - to.o2);
    if (r < 0) r += Ga;
    if (r >= T) r -= Ga;
    s_r[p][a] = r;
  }
  for (int i = tid; i < cnt * CC; i += kThreads) {
    const int p = i / CC, c = i - p * CC;
    const long long row = row0 + __ldg(&lst[p].y);
    s_val[p][c] = (coil0 + c < C) ? __ldg(vals + row * C + coil0 + c) : make_float2(0.f, 0.f);
  }
}

// s_bin[b] = first staged entry with r0 + W - 1 >= b (entries sorted by r0);
// offsets are clamped so a malformed list cannot index out of range.
template <int W, int T>
__device__ __forceinline__ void bin_round(int (*s_r)[3], int* s_bin, int cnt, int tid) {
  if (tid < cnt) {
    const int r = min(max(s_r[tid][0], 1 - W), T - 1) + W - 1;
    const int rp = tid == 0 ? -1 : min(max(s_r[tid - 1][0], 1 - W), T - 1) + W - 1;
    for (int bb = rp + 1; bb <= r; ++bb) s_bin[bb] = tid;
    if (tid == cnt - 1)
      for (int bb = r + 1; bb < W + T; ++bb) s_bin[bb] = cnt;
  }
}

template <int T, int CC, typename GT>
__device__ __forceinline__ void write_tile(const Geo& g, int C, int coil0, const TileOrigin& to,
                                          int slot, const float2* acc, const float2* comp,
                                          GT* __restrict__ grid, float2* __restrict__ scratch,
                                          int tid) {
  constexpr int kPts = T * T * T;
  auto value = [&](int i) {
    float2 v = acc[i];
    if (comp) {
      v.x += comp[i].x;
      v.y += comp[i].y;
    }
    return v;
  };
  if (slot < 0) {
    // coil fastest across lanes: contiguous shared reads, full global sectors
    for (int i = tid; i < kPts * CC; i += kThreads) {
      const int c = i % CC;
      const int pt = i / CC;
      const int lx = pt % T, ly = (pt / T) % T, lz = pt / (T * T);
      if (lz < to.e0 && ly < to.e1 && lx < to.e2 && coil0 + c < C) {
        const long long gi = ((long long)(to.o0 + lz) * g.g1 + (to.o1 + ly)) * g.g2 + (to.o2 + lx);
        grid_st(grid + (long long)(coil0 + c) * g.ngrid + gi, value(i));
      }
    }
  } else {
    float2* dst = scratch + ((long long)slot * gridDim.y + blockIdx.y) * (kPts * CC);
    for (int i = tid; i < kPts * CC; i += kThreads) dst[i] = value(i);
  }
}

// acc += w * v with the rounding errors of the product and the sum added to
// comp (FMA residual + TwoSum; Ogita, Rump & Oishi's compensated dot product)
__device__ __forceinline__ void comp_fma(float w, float v, float& acc, float& comp) {
  const float p = w * v;
  const float ep = fmaf(w, v, -p);
  const float s = acc + p;
  const float bb = s - acc;
  const float es = (acc - (s - bb)) + (p - bb);
  acc = s;
  comp += es + ep;
}

// Resolve a launch's work item through the phase table.
struct ItemRef {
  SpreadItem it;
  int jj, local;
};
__device__ __forceinline__ ItemRef item_ref(const PhaseTable& pt, int index) {
  ItemRef r;
  r.jj = phase_of(pt.item0, pt.nphase, index);
  r.local = index - pt.item0[r.jj];
  r.it = pt.items[r.jj][r.local];
  return r;
}
__device__ __forceinline__ ItemRef item_ref(const PhaseTable& pt) {
  return item_ref(pt, blockIdx.x);
}
__device__ __forceinline__ int scratch_slot(const PhaseTable& pt, const ItemRef& r) {
  return r.it.slot < 0 ? -1 : pt.slot0[r.jj] + r.it.slot;
}

// ---------------------------------------------------------------------------
// W = 4, CC in {2, 4, 8} coils, 8^3 tiles.  Warp w owns plane w and streams
// its own range of the item's list (no CTA-wide barriers): in batches of 32,
// lane p stages point p (the plane's z weight times the y weights, the x
// weights, offsets and CC values) into the warp's shared buffer, then the
// warp applies the batch with lane = (coil pair, tap x, row), each lane
// updating two coils of one grid point with a 128-bit read-modify-write.
template <int CC>
struct CoilStage {
  float wzy[4];
  float wx[4];
  int r1, r2, pad0, pad1;
  float2 val[CC];
};

template <int CC, typename GT, bool COMP>
__global__ void __launch_bounds__(kThreads) spread_coils_kernel(
    Geo g, KernelCoefs kc, int C, TilePlan tp, PhaseTable pt, const float2* __restrict__ vals,
    GT* __restrict__ grids, float2* __restrict__ scratch) {
  constexpr int W = 4, T = 8, B = 32, NB = W + T + 1;
  static_assert(CC == 2 || CC == 4 || CC == 8, "coil chunk");
  extern __shared__ float4 smem_raw[];
  float2* acc = reinterpret_cast<float2*>(smem_raw);  // [T][T][T][CC]
  float2* comp = COMP ? acc + T * T * T * CC : nullptr;  // compensation terms
  __shared__ __align__(16) CoilStage<CC> stg[kThreads / 32][B];

  const ItemRef ir = item_ref(pt);
  const SpreadItem it = ir.it;
  const int2* __restrict__ list = pt.list[ir.jj];
  const float4* __restrict__ qs = pt.qs[ir.jj];
  const long long row0 = pt.row0[ir.jj];
  GT* __restrict__ grid = grids + (long long)ir.jj * C * g.ngrid;
  const int coil0 = blockIdx.y * CC;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const TileOrigin to = tile_origin(g, tp, it.tile);
  for (int i = tid; i < T * T * T * CC * (COMP ? 2 : 1); i += kThreads)
    acc[i] = make_float2(0.f, 0.f);
  __syncthreads();

  const int lz = warp;
  if (lz < to.e0) {
    const int32_t* ib = pt.bins[ir.jj] + (long long)ir.local * NB;
    const int beg = it.begin + __ldg(ib + min(lz, NB - 1));
    const int end = it.begin + __ldg(ib + min(lz + W, NB - 1));
    // lane = (coil pair q, tap x, row half): a quarter-warp covers 128
    // contiguous bytes of one row (conflict-free 128-bit accesses)
    constexpr int NQ = CC / 2;               // coil pairs per point
    constexpr int LPR = NQ * W;               // lanes per tap row
    constexpr int RPI = 32 / LPR;             // rows per iteration
    const int q = lane % NQ, tx = (lane / NQ) % W, tyh = lane / LPR;
    CoilStage<CC>* st = stg[warp];
    for (int base = beg; base < end; base += B) {
      const int n = min(B, end - base);
      if (lane < n) {
        const int2 e = __ldg(list + base + lane);
        const float4 qq = __ldg(qs + e.x);
        int b0, b1, b2;
        unpack_base(__float_as_uint(qq.w), b0, b1, b2);
        int r0 = b0 - to.o0, r1 = b1 - to.o1, r2 = b2 - to.o2;
        if (r0 < 0) r0 += g.g0;
        if (r0 >= T) r0 -= g.g0;
        if (r1 < 0) r1 += g.g1;
        if (r1 >= T) r1 -= g.g1;
        if (r2 < 0) r2 += g.g2;
        if (r2 >= T) r2 -= g.g2;
        float wz[W], wy[W], wx[W];
        kernel_weights<W>(qq.x, kc, wz);
        kernel_weights<W>(qq.y, kc, wy);
        kernel_weights<W>(qq.z, kc, wx);
        const int t0 = lz - r0;
        const float wzt = ((unsigned)t0 < (unsigned)W) ? select_tap<W>(wz, t0) : 0.f;
        CoilStage<CC>& d = st[lane];
#pragma unroll
        for (int t = 0; t < W; ++t) {
          d.wzy[t] = wzt * wy[t];
          d.wx[t] = wx[t];
        }
        d.r1 = r1;
        d.r2 = r2;
        const float2* src = vals + (row0 + e.y) * C + coil0;
#pragma unroll
        for (int c = 0; c < CC; ++c)
          d.val[c] = (coil0 + c < C) ? __ldg(src + c) : make_float2(0.f, 0.f);
      }
      __syncwarp();
      for (int p = 0; p < n; ++p) {
        const CoilStage<CC>& d = st[p];
        const int lx = d.r2 + tx;
        const float4 v = reinterpret_cast<const float4*>(d.val)[q];
        const float wxt = d.wx[tx];
#pragma unroll
        for (int k = 0; k < (W + RPI - 1) / RPI; ++k) {
          const int ty = tyh + RPI * k;
          const int ly = d.r1 + ty;
          if (ty < W && (unsigned)ly < (unsigned)to.e1 && (unsigned)lx < (unsigned)to.e2) {
            const float w = d.wzy[ty & (W - 1)] * wxt;
            const int off = ((lz * T + ly) * T + lx) * CC;
            float4* a = reinterpret_cast<float4*>(acc + off) + q;
            float4 cur = *a;
            if constexpr (COMP) {
              float4* ca = reinterpret_cast<float4*>(comp + off) + q;
              float4 cc = *ca;
              comp_fma(w, v.x, cur.x, cc.x);
              comp_fma(w, v.y, cur.y, cc.y);
              comp_fma(w, v.z, cur.z, cc.z);
              comp_fma(w, v.w, cur.w, cc.w);
              *ca = cc;
            } else {
              cur.x = fmaf(w, v.x, cur.x);
              cur.y = fmaf(w, v.y, cur.y);
              cur.z = fmaf(w, v.z, cur.z);
              cur.w = fmaf(w, v.w, cur.w);
            }
            *a = cur;
          }
        }
      }
      __syncwarp();
    }
  }
  __syncthreads();
  write_tile<T, CC, GT>(g, C, coil0, to, scratch_slot(pt, ir), acc, comp, grid, scratch, tid);
}

// ---------------------------------------------------------------------------
// W = 4, CC coils, 8^3 tiles, register accumulation.  Warp w owns plane w of
// the tile; lane (x = lane % 8, yh = lane / 8) owns the two grid points
// (w, yh, x) and (w, yh + 4, x) for all CC coils in registers.  The warp
// streams its plane's range of the list with the same per-warp staging as
// spread_coils_kernel; every lane then adds each staged point's contribution
// to its own two points (zero weight outside the point's 4 x 4 footprint in
// the plane), one half-plane at a time so that points whose footprint misses
// the half are skipped, and nothing is read back from or written to shared
// memory per update.  The result (and the order of every sum) is the same per grid value
// as for the shared-memory kernel: list order within the item.
// WPC = 8: a CTA is a work item's tile, warp w its plane w.  WPC = 1: a CTA
// is one warp, block b serves plane b % 8 of item b / 8, so a plane's warp
// frees its resources as soon as it is done (the planes of a tile carry
// different amounts of work).  Same summation order, same result.
template <int CC, typename GT, int WPC>
__global__ void __launch_bounds__(32 * WPC, WPC == 1 ? 24 : 3) spread_coils_reg_kernel(
    Geo g, KernelCoefs kc, int C, TilePlan tp, PhaseTable pt, const float2* __restrict__ vals,
    GT* __restrict__ grids, float2* __restrict__ scratch) {
  constexpr int W = 4, T = 8, B = 32, NB = W + T + 1;
  static_assert(CC == 2 || CC == 4 || CC == 8, "coil chunk");
  static_assert(WPC == 1 || WPC == 8, "warps per CTA");
  __shared__ __align__(16) CoilStage<CC> stg[WPC][B];

  const ItemRef ir = item_ref(pt, WPC == 8 ? int(blockIdx.x) : int(blockIdx.x >> 3));
  const SpreadItem it = ir.it;
  const int2* __restrict__ list = pt.list[ir.jj];
  const float4* __restrict__ qs = pt.qs[ir.jj];
  const long long row0 = pt.row0[ir.jj];
  GT* __restrict__ grid = grids + (long long)ir.jj * C * g.ngrid;
  const int coil0 = blockIdx.y * CC;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const TileOrigin to = tile_origin(g, tp, it.tile);
  const int lz = WPC == 8 ? warp : int(blockIdx.x & 7), x = lane & 7, yh = lane >> 3;

  float2 acc[2][CC];
#pragma unroll
  for (int h = 0; h < 2; ++h)
#pragma unroll
    for (int c = 0; c < CC; ++c) acc[h][c] = make_float2(0.f, 0.f);

  if (lz < to.e0) {
    const int32_t* ib = pt.bins[ir.jj] + (long long)ir.local * NB;
    const int beg = it.begin + __ldg(ib + min(lz, NB - 1));
    const int end = it.begin + __ldg(ib + min(lz + W, NB - 1));
    CoilStage<CC>* st = stg[warp];
    for (int base = beg; base < end; base += B) {
      const int n = min(B, end - base);
      if (lane < n) {
        const int2 e = __ldg(list + base + lane);
        const float4 qq = __ldg(qs + e.x);
        int b0, b1, b2;
        unpack_base(__float_as_uint(qq.w), b0, b1, b2);
        int r0 = b0 - to.o0, r1 = b1 - to.o1, r2 = b2 - to.o2;
        if (r0 < 0) r0 += g.g0;
        if (r0 >= T) r0 -= g.g0;
        if (r1 < 0) r1 += g.g1;
        if (r1 >= T) r1 -= g.g1;
        if (r2 < 0) r2 += g.g2;
        if (r2 >= T) r2 -= g.g2;
        float wz[W], wy[W], wx[W];
        kernel_weights<W>(qq.x, kc, wz);
        kernel_weights<W>(qq.y, kc, wy);
        kernel_weights<W>(qq.z, kc, wx);
        const int t0 = lz - r0;
        const float wzt = ((unsigned)t0 < (unsigned)W) ? select_tap<W>(wz, t0) : 0.f;
        CoilStage<CC>& d = st[lane];
#pragma unroll
        for (int t = 0; t < W; ++t) {
          d.wzy[t] = wzt * wy[t];
          d.wx[t] = wx[t];
        }
        d.r1 = r1;
        d.r2 = r2;
        const float2* src = vals + (row0 + e.y) * C + coil0;
#pragma unroll
        for (int c = 0; c < CC; ++c)
          d.val[c] = (coil0 + c < C) ? __ldg(src + c) : make_float2(0.f, 0.f);
      }
      __syncwarp();
      // one pass per half-plane (rows 0-3: acc[0], rows 4-7: acc[1]); a point
      // whose 4-row footprint (rows r1 .. r1 + 3) misses the half is skipped
      // (a warp-uniform branch) -- it would only add zero-weight terms
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        for (int p = 0; p < n; ++p) {
          const CoilStage<CC>& d = st[p];
          if (h == 0 ? d.r1 > 3 : d.r1 < 1) continue;
          const int tx = x - d.r2, ty = yh + 4 * h - d.r1;
          const float wxv = (unsigned)tx < (unsigned)W ? d.wx[tx & (W - 1)] : 0.f;
          const float w = (unsigned)ty < (unsigned)W ? d.wzy[ty & (W - 1)] * wxv : 0.f;
#pragma unroll
          for (int c2 = 0; c2 < CC / 2; ++c2) {
            const float4 v = reinterpret_cast<const float4*>(d.val)[c2];
            acc[h][2 * c2].x = fmaf(w, v.x, acc[h][2 * c2].x);
            acc[h][2 * c2].y = fmaf(w, v.y, acc[h][2 * c2].y);
            acc[h][2 * c2 + 1].x = fmaf(w, v.z, acc[h][2 * c2 + 1].x);
            acc[h][2 * c2 + 1].y = fmaf(w, v.w, acc[h][2 * c2 + 1].y);
          }
        }
      }
      __syncwarp();
    }
  }
  // write out: rows yh and yh + 4 of plane lz (outside the grid: not written)
  const int slot = scratch_slot(pt, ir);
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int ly = yh + 4 * h;
    if (slot < 0) {
      if (lz < to.e0 && ly < to.e1 && x < to.e2) {
        const long long gi = ((long long)(to.o0 + lz) * g.g1 + (to.o1 + ly)) * g.g2 + (to.o2 + x);
#pragma unroll
        for (int c = 0; c < CC; ++c)
          if (coil0 + c < C) grid_st(grid + (long long)(coil0 + c) * g.ngrid + gi, acc[h][c]);
      }
    } else {
      float2* dst = scratch + ((long long)slot * gridDim.y + blockIdx.y) * (T * T * T * CC) +
                    ((lz * T + ly) * T + x) * CC;
#pragma unroll
      for (int c2 = 0; c2 < CC / 2; ++c2)
        reinterpret_cast<float4*>(dst)[c2] =
            make_float4(acc[h][2 * c2].x, acc[h][2 * c2].y, acc[h][2 * c2 + 1].x,
                        acc[h][2 * c2 + 1].y);
    }
  }
}

// ---------------------------------------------------------------------------
// W = 4, 8 coils, 8^3 tiles, tensor cores.  One warp (CTA) per tile plane with
// the same per-warp staging of 32 points as spread_coils_reg_kernel<8, GT, 1>;
// a staged batch updates the plane by the contraction
//   C[m][n] += sum_k A[m][k] V[k][n],   m = ly * 8 + lx (grid point of the
//   plane), k = point of the batch, n = 2 coil + (0: re, 1: im),
//   A[m][k] = wz_k wy_k(ly - r1_k) wx_k(lx - r2_k)  (0 outside the footprint),
// run as mma.sync m16n8k8 TF32 products with FP32 accumulation (4 row tiles
// x 2 column tiles x 4 k steps per batch).  Each operand is split x = hi + lo
// (hi = x rounded to TF32, lo = the rest rounded to TF32) and the products
// hi.hi + hi.lo + lo.hi are accumulated, which keeps the error near FP32
// rounding (the dropped lo.lo term is below 2^-22 relative).  The summation
// order differs from the FMA kernels, so the result is not bitwise theirs.
// Fragment layouts (PTX, m16n8k8 .tf32): g = lane / 4, q = lane % 4;
// A: a0 (g, q), a1 (g + 8, q), a2 (g, q + 4), a3 (g + 8, q + 4);
// B: b0 (k = q, n = g), b1 (k = q + 4, n = g);
// C: c0, c1 (g, 2q, 2q + 1), c2, c3 (g + 8, 2q, 2q + 1).
__device__ __forceinline__ uint32_t tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// x = hi + lo: hi = x rounded to TF32; the remainder x - hi is exact in FP32
// and goes to the tensor core as it is (no second rounding: one instruction
// less per operand element), which uses its TF32 part, within 2^-10 of it,
// i.e. within 2^-21 of x.
__device__ __forceinline__ void split_tf32(float x, uint32_t& hi, uint32_t& lo) {
  hi = tf32_rna(x);
  lo = __float_as_uint(x - __uint_as_float(hi));
}

__device__ __forceinline__ void mma_tf32(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2,
                                         uint32_t a3, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0, %1, %2, %3}, "
      "{%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// WPC warps per CTA, warp w serving plane (blockIdx.x * WPC + w) % 8 of item
// (blockIdx.x * WPC + w) / 8 (WPC divides 8).
template <typename GT, int WPC>
__global__ void __launch_bounds__(32 * WPC, WPC == 4 ? 5 : 16 / WPC) spread_coils_mma_kernel(
    Geo g, KernelCoefs kc, int C, TilePlan tp, PhaseTable pt, const float2* __restrict__ vals,
    GT* __restrict__ grids, float2* __restrict__ scratch) {
  constexpr int CC = 8, W = 4, T = 8, B = 32, NB = W + T + 1;
  static_assert(WPC == 1 || WPC == 2 || WPC == 4, "warps per CTA");
  __shared__ __align__(16) CoilStage<CC> stg_all[WPC][B];
  const int warp = int(threadIdx.x >> 5);
  CoilStage<CC>* stg = stg_all[warp];
  const int plane_id = int(blockIdx.x) * WPC + warp;

  const ItemRef ir = item_ref(pt, plane_id >> 3);
  const SpreadItem it = ir.it;
  const int2* __restrict__ list = pt.list[ir.jj];
  const float4* __restrict__ qs = pt.qs[ir.jj];
  const long long row0 = pt.row0[ir.jj];
  GT* __restrict__ grid = grids + (long long)ir.jj * C * g.ngrid;
  const int coil0 = blockIdx.y * CC;
  const int lane = threadIdx.x & 31, gq = lane >> 2, q = lane & 3;
  const TileOrigin to = tile_origin(g, tp, it.tile);
  const int lz = plane_id & 7;

  float acc[4][2][4];
#pragma unroll
  for (int mt = 0; mt < 4; ++mt)
#pragma unroll
    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
      for (int i = 0; i < 4; ++i) acc[mt][nt][i] = 0.f;

  if (lz < to.e0) {
    const int32_t* ib = pt.bins[ir.jj] + (long long)ir.local * NB;
    const int beg = it.begin + __ldg(ib + min(lz, NB - 1));
    const int end = it.begin + __ldg(ib + min(lz + W, NB - 1));
    for (int base = beg; base < end; base += B) {
      const int n = min(B, end - base);
      if (lane < n) {
        const int2 e = __ldg(list + base + lane);
        const float4 qq = __ldg(qs + e.x);
        int b0, b1, b2;
        unpack_base(__float_as_uint(qq.w), b0, b1, b2);
        int r0 = b0 - to.o0, r1 = b1 - to.o1, r2 = b2 - to.o2;
        if (r0 < 0) r0 += g.g0;
        if (r0 >= T) r0 -= g.g0;
        if (r1 < 0) r1 += g.g1;
        if (r1 >= T) r1 -= g.g1;
        if (r2 < 0) r2 += g.g2;
        if (r2 >= T) r2 -= g.g2;
        float wz[W], wy[W], wx[W];
        kernel_weights<W>(qq.x, kc, wz);
        kernel_weights<W>(qq.y, kc, wy);
        kernel_weights<W>(qq.z, kc, wx);
        const int t0 = lz - r0;
        const float wzt = ((unsigned)t0 < (unsigned)W) ? select_tap<W>(wz, t0) : 0.f;
        CoilStage<CC>& d = stg[lane];
#pragma unroll
        for (int t = 0; t < W; ++t) {
          d.wzy[t] = wzt * wy[t];
          d.wx[t] = wx[t];
        }
        d.r1 = r1;
        d.r2 = r2;
        const float2* src = vals + (row0 + e.y) * C + coil0;
#pragma unroll
        for (int c = 0; c < CC; ++c)
          d.val[c] = (coil0 + c < C) ? __ldg(src + c) : make_float2(0.f, 0.f);
      }
      __syncwarp();
#pragma unroll 1
      for (int ks = 0; ks < 4; ++ks) {
        if (8 * ks >= n) break;  // warp-uniform
        // this lane's A columns: points k0 (a0, a1) and k0 + 4 (a2, a3), at
        // grid column lx = gq, every row ly
        float wa[2][T];
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          const int k = 8 * ks + q + 4 * j;
          const bool live = k < n;
          const CoilStage<CC>& d = stg[live ? k : 0];
          const int tx = gq - d.r2;
          const float wxv = (live && (unsigned)tx < (unsigned)W) ? d.wx[tx & (W - 1)] : 0.f;
#pragma unroll
          for (int ly = 0; ly < T; ++ly) {
            const int ty = ly - d.r1;
            wa[j][ly] = (unsigned)ty < (unsigned)W ? d.wzy[ty & (W - 1)] * wxv : 0.f;
          }
        }
        // B: values of points k0 (b0) and k0 + 4 (b1), column n = 8 nt + gq:
        // coil 4 nt + gq / 2, real part for even gq
        uint32_t bh[2][2], bl[2][2];
#pragma unroll
        for (int nt = 0; nt < 2; ++nt)
#pragma unroll
          for (int j = 0; j < 2; ++j) {
            const int k = 8 * ks + q + 4 * j;
            const float2 v = k < n ? stg[k].val[4 * nt + (gq >> 1)] : make_float2(0.f, 0.f);
            split_tf32((gq & 1) ? v.y : v.x, bh[nt][j], bl[nt][j]);
          }
#pragma unroll
        for (int mt = 0; mt < 4; ++mt) {
          uint32_t ah[4], al[4];
          split_tf32(wa[0][2 * mt], ah[0], al[0]);
          split_tf32(wa[0][2 * mt + 1], ah[1], al[1]);
          split_tf32(wa[1][2 * mt], ah[2], al[2]);
          split_tf32(wa[1][2 * mt + 1], ah[3], al[3]);
#pragma unroll
          for (int nt = 0; nt < 2; ++nt) {
            mma_tf32(acc[mt][nt], ah[0], ah[1], ah[2], ah[3], bh[nt][0], bh[nt][1]);
            mma_tf32(acc[mt][nt], ah[0], ah[1], ah[2], ah[3], bl[nt][0], bl[nt][1]);
            mma_tf32(acc[mt][nt], al[0], al[1], al[2], al[3], bh[nt][0], bh[nt][1]);
          }
        }
      }
      __syncwarp();
    }
  }
  // write out: grid column lx = gq, rows 2 mt (c0, c1) and 2 mt + 1 (c2, c3),
  // coils 4 nt + q
  const int slot = scratch_slot(pt, ir);
  const int lx = gq;
#pragma unroll
  for (int mt = 0; mt < 4; ++mt)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int ly = 2 * mt + h;
#pragma unroll
      for (int nt = 0; nt < 2; ++nt) {
        const int c = 4 * nt + q;
        const float2 v = make_float2(acc[mt][nt][2 * h], acc[mt][nt][2 * h + 1]);
        if (slot < 0) {
          if (lz < to.e0 && ly < to.e1 && lx < to.e2 && coil0 + c < C) {
            const long long gi =
                ((long long)(to.o0 + lz) * g.g1 + (to.o1 + ly)) * g.g2 + (to.o2 + lx);
            grid_st(grid + (long long)(coil0 + c) * g.ngrid + gi, v);
          }
        } else {
          scratch[((long long)slot * gridDim.y + blockIdx.y) * (T * T * T * CC) +
                  ((lz * T + ly) * T + lx) * CC + c] = v;
        }
      }
    }
}

// ---------------------------------------------------------------------------
// The same contraction over 4^3 sub-blocks of an 8^3 tile instead of tile
// planes.  Warp w serves sub-block sb = (blockIdx.x * WPC + w) % 8 (bits z, y,
// x from high to low) of item (blockIdx.x * WPC + w) / 8 and streams the
// points whose footprint meets it: in the item's class-ordered list, per axis
// the classes "low half only" and "both halves" for a low sub-block, "both"
// and "high half only" for a high one, i.e. four runs of two adjacent
// classes.  A point meets (7/4)^3 = 5.4 sub-blocks on average against
// 4 x (11/8)^2 = 7.6 tile planes, so staging, operand building and products
// fall by 29 %.  Rows m = 16 z + 4 y + x of the sub-block (z, y, x in 0..3):
// lane (g, q) holds x = g % 4 with y = g / 4 (row g) and y + 2 (row g + 8) for
// every m-tile z.  Columns and the TF32 split are those of the plane kernel.
// A k-step skips the m-tiles none of its eight points reaches (the runs are in
// first-tap z order, so neighbouring points mostly share their z planes).  The
// launch bound of 28 warps per SM holds the kernel at 72 registers; with one
// warp per CTA (the usual choice) a CTA's slot frees as soon as its sub-block
// is done, whatever the other sub-blocks' point counts.
struct CubeStage {
  float wz[4], wy[4], wx[4];
  int r0, r1, r2, pad0;  // first tap relative to the sub-block origin, in [-3, 3]
  float2 val[8];
  float pad1[4];  // 144-byte records: the four points a k-step reads sit on disjoint banks
};
static_assert(sizeof(CubeStage) == 144, "staging record");

template <typename GT, int WPC>
__global__ void __launch_bounds__(32 * WPC, 28 / WPC) spread_coils_cube_kernel(
    Geo g, KernelCoefs kc, int C, TilePlan tp, PhaseTable pt, const float2* __restrict__ vals,
    GT* __restrict__ grids, float2* __restrict__ scratch) {
  constexpr int CC = 8, W = 4, T = 8, B = 32;
  static_assert(WPC == 1 || WPC == 2 || WPC == 4, "warps per CTA");
  __shared__ __align__(16) CubeStage stg_all[WPC][B];
  // per warp: starts of runs 1-3 in the sub-block's sequence, and for each
  // run the list index minus the sequence position (kept in shared memory,
  // not registers: they are read once per batch)
  __shared__ int run_all[WPC][8];
  const int warp = int(threadIdx.x >> 5);
  CubeStage* stg = stg_all[warp];
  int* run = run_all[warp];
  const int block_id = int(blockIdx.x) * WPC + warp;

  const ItemRef ir = item_ref(pt, block_id >> 3);
  const SpreadItem it = ir.it;
  const int2* __restrict__ list = pt.clist[ir.jj];
  const float4* __restrict__ qs = pt.qs[ir.jj];
  const long long row0 = pt.row0[ir.jj];
  GT* __restrict__ grid = grids + (long long)ir.jj * C * g.ngrid;
  const int coil0 = blockIdx.y * CC;
  const int lane = threadIdx.x & 31, gq = lane >> 2, q = lane & 3;
  const TileOrigin to = tile_origin(g, tp, it.tile);
  const int sb = block_id & 7, bz = sb >> 2, by = (sb >> 1) & 1, bx = sb & 1;
  const int sz = 4 * bz, sy = 4 * by, sx = 4 * bx;  // sub-block origin in the tile

  float acc[4][2][4];
#pragma unroll
  for (int mt = 0; mt < 4; ++mt)
#pragma unroll
    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
      for (int i = 0; i < 4; ++i) acc[mt][nt][i] = 0.f;

  if (sz < to.e0 && sy < to.e1 && sx < to.e2) {
    // the four runs (classes 9 cz + 3 cy + {bx, bx + 1}, cz in {bz, bz + 1},
    // cy in {by, by + 1}) and their prefix sums
    const int32_t* cb = pt.cbins[ir.jj] + (long long)ir.local * kCubeBins;
    int total = 0;
    if (lane < 4) {
      const int c = 9 * (bz + (lane >> 1)) + 3 * (by + (lane & 1)) + bx;
      const int rs = __ldg(cb + c), len = __ldg(cb + c + 2) - rs;
      // inclusive prefix of the four run lengths over lanes 0-3
      int incl = len;
#pragma unroll
      for (int d = 1; d < 4; d <<= 1) {
        const int t = __shfl_up_sync(0xfu, incl, d, 4);
        if (lane >= d) incl += t;
      }
      const int start = incl - len;
      if (lane > 0) run[lane - 1] = start;
      run[4 + lane] = it.begin + rs - start;
      total = incl;
    }
    total = __shfl_sync(0xffffffffu, total, 3);
    __syncwarp();
    // 16-byte value loads when every staged row segment is 16-byte aligned
    const bool vec_vals = (C & 1) == 0 && coil0 + CC <= C &&
                          (reinterpret_cast<uintptr_t>(vals) & 15) == 0;
    for (int base = 0; base < total; base += B) {
      const int n = min(B, total - base);
      if (lane < n) {
        const int i = base + lane;
        const int r = (i >= run[0]) + (i >= run[1]) + (i >= run[2]);
        const int2 e = __ldg(list + i + run[4 + r]);
        const float4 qq = __ldg(qs + e.x);
        int b0, b1, b2;
        unpack_base(__float_as_uint(qq.w), b0, b1, b2);
        int r0 = b0 - to.o0, r1 = b1 - to.o1, r2 = b2 - to.o2;
        if (r0 < 0) r0 += g.g0;
        if (r0 >= T) r0 -= g.g0;
        if (r1 < 0) r1 += g.g1;
        if (r1 >= T) r1 -= g.g1;
        if (r2 < 0) r2 += g.g2;
        if (r2 >= T) r2 -= g.g2;
        float wz[W], wy[W], wx[W];
        kernel_weights<W>(qq.x, kc, wz);
        kernel_weights<W>(qq.y, kc, wy);
        kernel_weights<W>(qq.z, kc, wx);
        CubeStage& d = stg[lane];
        reinterpret_cast<float4*>(d.wz)[0] = make_float4(wz[0], wz[1], wz[2], wz[3]);
        reinterpret_cast<float4*>(d.wy)[0] = make_float4(wy[0], wy[1], wy[2], wy[3]);
        reinterpret_cast<float4*>(d.wx)[0] = make_float4(wx[0], wx[1], wx[2], wx[3]);
        reinterpret_cast<int4*>(&d.r0)[0] = make_int4(r0 - sz, r1 - sy, r2 - sx, 0);
        const float2* src = vals + (row0 + e.y) * C + coil0;
        if (vec_vals) {
#pragma unroll
          for (int c2 = 0; c2 < CC / 2; ++c2)
            reinterpret_cast<float4*>(d.val)[c2] = __ldg(reinterpret_cast<const float4*>(src) + c2);
        } else {
#pragma unroll
          for (int c = 0; c < CC; ++c)
            d.val[c] = (coil0 + c < C) ? __ldg(src + c) : make_float2(0.f, 0.f);
        }
      }
      __syncwarp();
#pragma unroll 1
      for (int ks = 0; ks < 4; ++ks) {
        if (8 * ks >= n) break;  // warp-uniform
        // this lane's A entries: points k0 (a0, a1) and k0 + 4 (a2, a3) at
        // column x = g % 4, rows y = g / 4 and y + 2, factor wy wx here, wz
        // per m-tile below
        float pyx[2][2];
        int rz[2];
        const CubeStage* dj[2];
        unsigned planes = 0;  // m-tiles (z planes) the lane's two points reach
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          const int k = 8 * ks + q + 4 * j;
          const bool live = k < n;
          const CubeStage& d = stg[live ? k : 0];
          dj[j] = &d;
          const int4 rr = *reinterpret_cast<const int4*>(&d.r0);
          rz[j] = rr.x;
          // z taps rz .. rz + 3 meet planes max(rz, 0) .. min(rz + 3, 3)
          if (live) planes |= rr.x >= 0 ? (0xFu << min(rr.x, 4)) & 0xFu : 0xFu >> min(-rr.x, 4);
          const int tx = (gq & 3) - rr.z;
          const float wxv = (live && (unsigned)tx < (unsigned)W) ? d.wx[tx & (W - 1)] : 0.f;
          const int ty0 = (gq >> 2) - rr.y, ty1 = ty0 + 2;
          pyx[j][0] = (unsigned)ty0 < (unsigned)W ? d.wy[ty0 & (W - 1)] * wxv : 0.f;
          pyx[j][1] = (unsigned)ty1 < (unsigned)W ? d.wy[ty1 & (W - 1)] * wxv : 0.f;
        }
        uint32_t bh[2][2], bl[2][2];
#pragma unroll
        for (int nt = 0; nt < 2; ++nt)
#pragma unroll
          for (int j = 0; j < 2; ++j) {
            const int k = 8 * ks + q + 4 * j;
            const float2 v = k < n ? stg[k].val[4 * nt + (gq >> 1)] : make_float2(0.f, 0.f);
            split_tf32((gq & 1) ? v.y : v.x, bh[nt][j], bl[nt][j]);
          }
        // an m-tile none of the k-step's eight points reaches has all-zero A
        // entries and would add exact zeros: skipped (warp-uniform).  The
        // plan keeps every footprint-class run in first-tap z order, so the
        // points of a k-step mostly share their planes.
        planes = __reduce_or_sync(0xffffffffu, planes);
#pragma unroll
        for (int mt = 0; mt < 4; ++mt) {
          if (!(planes & (1u << mt))) continue;
          float a[2][2];
#pragma unroll
          for (int j = 0; j < 2; ++j) {
            const int tz = mt - rz[j];
            const float wzv = (unsigned)tz < (unsigned)W ? dj[j]->wz[tz & (W - 1)] : 0.f;
            a[j][0] = wzv * pyx[j][0];
            a[j][1] = wzv * pyx[j][1];
          }
          uint32_t ah[4], al[4];
          split_tf32(a[0][0], ah[0], al[0]);
          split_tf32(a[0][1], ah[1], al[1]);
          split_tf32(a[1][0], ah[2], al[2]);
          split_tf32(a[1][1], ah[3], al[3]);
#pragma unroll
          for (int nt = 0; nt < 2; ++nt) {
            mma_tf32(acc[mt][nt], ah[0], ah[1], ah[2], ah[3], bh[nt][0], bh[nt][1]);
            mma_tf32(acc[mt][nt], ah[0], ah[1], ah[2], ah[3], bl[nt][0], bl[nt][1]);
            mma_tf32(acc[mt][nt], al[0], al[1], al[2], al[3], bh[nt][0], bh[nt][1]);
          }
        }
      }
      __syncwarp();
    }
  }
  // write out: m-tile mt is tile plane sz + mt; rows y = g / 4 (c0, c1) and
  // y + 2 (c2, c3), column x = g % 4; coils 4 nt + q
  const int slot = scratch_slot(pt, ir);
  const int lx = sx + (gq & 3);
  if (slot < 0 && sz + 4 <= to.e0 && sy + 4 <= to.e1 && sx + 4 <= to.e2 && coil0 + CC <= C) {
    // the whole sub-block and coil chunk lie in the grid: one base address,
    // constant strides (plane, two rows, four coils)
    const long long plane = (long long)g.g1 * g.g2;
    GT* base = grid + (long long)(coil0 + q) * g.ngrid +
               ((long long)(to.o0 + sz) * g.g1 + (to.o1 + sy + (gq >> 2))) * g.g2 + (to.o2 + lx);
#pragma unroll
    for (int mt = 0; mt < 4; ++mt)
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int nt = 0; nt < 2; ++nt)
          grid_st(base + mt * plane + 2 * h * g.g2 + 4LL * nt * g.ngrid,
                  make_float2(acc[mt][nt][2 * h], acc[mt][nt][2 * h + 1]));
    return;
  }
#pragma unroll
  for (int mt = 0; mt < 4; ++mt)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int lz = sz + mt, ly = sy + (gq >> 2) + 2 * h;
#pragma unroll
      for (int nt = 0; nt < 2; ++nt) {
        const int c = 4 * nt + q;
        const float2 v = make_float2(acc[mt][nt][2 * h], acc[mt][nt][2 * h + 1]);
        if (slot < 0) {
          if (lz < to.e0 && ly < to.e1 && lx < to.e2 && coil0 + c < C) {
            const long long gi =
                ((long long)(to.o0 + lz) * g.g1 + (to.o1 + ly)) * g.g2 + (to.o2 + lx);
            grid_st(grid + (long long)(coil0 + c) * g.ngrid + gi, v);
          }
        } else {
          scratch[((long long)slot * gridDim.y + blockIdx.y) * (T * T * T * CC) +
                  ((lz * T + ly) * T + lx) * CC + c] = v;
        }
      }
    }
}

// ---------------------------------------------------------------------------
// W = 4, one channel (image space), 16^3 tiles.  Warp w owns planes 2w and
// 2w+1 (one per half-warp) and streams the union of their list ranges, with
// the same per-warp staging as above; lane = (tap x, tap y, plane).
struct SingleStage {
  float wzy[2][4];
  float wx[4];
  int r1, r2;
  float2 val;
  float pad[4];  // 80-byte records: a quarter-warp's 16-byte stores hit disjoint banks
};
static_assert(sizeof(SingleStage) == 80, "staging record");

// WPC = 8: a CTA is a work item's tile (8 warps, 2 planes each, accumulator
// of the whole tile); WPC = 1: a CTA is one warp with planes 2w, 2w+1 of item
// b / 8, w = b % 8, and an accumulator of those two planes only, so each
// plane pair frees its resources when done.  Same summation order.
template <bool COMP, int WPC>
__global__ void __launch_bounds__(32 * WPC) spread_single_kernel(
    Geo g, KernelCoefs kc, TilePlan tp, PhaseTable pt, const float2* __restrict__ vals,
    float2* __restrict__ grids, float2* __restrict__ scratch) {
  constexpr int W = 4, T = 16, B = 32, NB = W + T + 1;
  constexpr int RS = T + 4;  // padded row stride: 4 tap rows hit disjoint banks
  constexpr int NP = WPC == 8 ? T : 2;  // planes held in shared memory
  static_assert(WPC == 1 || WPC == 8, "warps per CTA");
  extern __shared__ float4 smem_raw[];
  float2* acc = reinterpret_cast<float2*>(smem_raw);  // [NP][T][RS]
  float2* comp = COMP ? acc + NP * T * RS : nullptr;
  __shared__ __align__(16) SingleStage stg[WPC][B];

  const ItemRef ir = item_ref(pt, WPC == 8 ? int(blockIdx.x) : int(blockIdx.x >> 3));
  const SpreadItem it = ir.it;
  const int2* __restrict__ list = pt.list[ir.jj];
  const float4* __restrict__ qs = pt.qs[ir.jj];
  const long long row0 = pt.row0[ir.jj];
  float2* __restrict__ grid = grids + (long long)ir.jj * g.ngrid;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const TileOrigin to = tile_origin(g, tp, it.tile);
  const int pw = WPC == 8 ? warp : int(blockIdx.x & 7);  // plane pair of this warp
  const int pbase = WPC == 8 ? 0 : 2 * pw;               // first plane held
  for (int i = tid; i < NP * T * RS * (COMP ? 2 : 1); i += 32 * WPC)
    acc[i] = make_float2(0.f, 0.f);
  __syncthreads();

  const int z0 = 2 * pw;
  if (z0 < to.e0) {
    const int32_t* ib = pt.bins[ir.jj] + (long long)ir.local * NB;
    const int beg = it.begin + __ldg(ib + min(z0, NB - 1));
    const int end = it.begin + __ldg(ib + min(z0 + W + 1, NB - 1));
    const int tx = lane & 3, ty = (lane >> 2) & 3, hz = lane >> 4;
    const int lz = z0 + hz;
    SingleStage* st = stg[warp];
    // each batch loads the next batch's list entries
    int2 e_next = make_int2(0, 0);
    if (beg + lane < end) e_next = __ldg(list + beg + lane);
    for (int base = beg; base < end; base += B) {
      const int n = min(B, end - base);
      const int2 e = e_next;
      if (base + B + lane < end) e_next = __ldg(list + base + B + lane);
      if (lane < n) {
        const float4 q = __ldg(qs + e.x);
        int b0, b1, b2;
        unpack_base(__float_as_uint(q.w), b0, b1, b2);
        int r0 = b0 - to.o0, r1 = b1 - to.o1, r2 = b2 - to.o2;
        if (r0 < 0) r0 += g.g0;
        if (r0 >= T) r0 -= g.g0;
        if (r1 < 0) r1 += g.g1;
        if (r1 >= T) r1 -= g.g1;
        if (r2 < 0) r2 += g.g2;
        if (r2 >= T) r2 -= g.g2;
        float wz[W], wy[W], wx[W];
        kernel_weights<W>(q.x, kc, wz);
        kernel_weights<W>(q.y, kc, wy);
        kernel_weights<W>(q.z, kc, wx);
        const int ta = z0 - r0, tb = z0 + 1 - r0;
        const float wa = ((unsigned)ta < (unsigned)W) ? select_tap<W>(wz, ta) : 0.f;
        const float wb = ((unsigned)tb < (unsigned)W && z0 + 1 < to.e0) ? select_tap<W>(wz, tb) : 0.f;
        SingleStage& d = st[lane];
        const float2 v = __ldg(vals + row0 + e.y);
        float4* d4 = reinterpret_cast<float4*>(&d);
        d4[0] = make_float4(wa * wy[0], wa * wy[1], wa * wy[2], wa * wy[3]);
        d4[1] = make_float4(wb * wy[0], wb * wy[1], wb * wy[2], wb * wy[3]);
        d4[2] = make_float4(wx[0], wx[1], wx[2], wx[3]);
        d4[3] = make_float4(__int_as_float(r1), __int_as_float(r2), v.x, v.y);
      }
      __syncwarp();
      for (int p = 0; p < n; ++p) {
        const SingleStage& d = st[p];
        const float4 rv = reinterpret_cast<const float4*>(&d)[3];  // r1, r2, value
        const int ly = __float_as_int(rv.x) + ty, lx = __float_as_int(rv.y) + tx;
        if ((unsigned)ly < (unsigned)to.e1 && (unsigned)lx < (unsigned)to.e2 && lz < to.e0) {
          const float w = d.wzy[hz][ty] * d.wx[tx];
          const int off = ((lz - pbase) * T + ly) * RS + lx;
          float2 cur = acc[off];
          if constexpr (COMP) {
            float2 cc = comp[off];
            comp_fma(w, rv.z, cur.x, cc.x);
            comp_fma(w, rv.w, cur.y, cc.y);
            comp[off] = cc;
          } else {
            cur.x = fmaf(w, rv.z, cur.x);
            cur.y = fmaf(w, rv.w, cur.y);
          }
          acc[off] = cur;
        }
      }
      __syncwarp();
    }
  }
  __syncthreads();
  // write the held planes of the tile (or partial tile), dropping the row padding
  constexpr int kPts = T * T * T;
  const int slot = scratch_slot(pt, ir);
  auto value = [&](int lz, int ly, int lx) {
    const int off = ((lz - pbase) * T + ly) * RS + lx;
    float2 v = acc[off];
    if constexpr (COMP) {
      v.x += comp[off].x;
      v.y += comp[off].y;
    }
    return v;
  };
  if (slot < 0) {
    for (int i = tid; i < NP * T * T; i += 32 * WPC) {
      const int lx = i % T, ly = (i / T) % T, lz = pbase + i / (T * T);
      if (lz < to.e0 && ly < to.e1 && lx < to.e2) {
        const long long gi = ((long long)(to.o0 + lz) * g.g1 + (to.o1 + ly)) * g.g2 + (to.o2 + lx);
        grid[gi] = value(lz, ly, lx);
      }
    }
  } else {
    float2* dst = scratch + (long long)slot * kPts + pbase * T * T;
    for (int i = tid; i < NP * T * T; i += 32 * WPC) {
      const int lx = i % T, ly = (i / T) % T, lz = pbase + i / (T * T);
      dst[i] = value(lz, ly, lx);
    }
  }
}

// ---------------------------------------------------------------------------
// Generic kernel (any W <= kMaxWidth, any CC), 8^3 tiles, warp per plane,
// lanes over (coil, tap x, tap y) combinations.
template <int W, int CC, typename GT>
__global__ void __launch_bounds__(kThreads) spread_generic_kernel(
    Geo g, KernelCoefs kc, int C, TilePlan tp, PhaseTable pt, const float2* __restrict__ vals,
    GT* __restrict__ grids, float2* __restrict__ scratch) {
  constexpr int T = 8, R = 64;
  extern __shared__ float4 smem_raw[];
  float2* acc = reinterpret_cast<float2*>(smem_raw);  // [T][T][T][CC]
  __shared__ float s_w[R][3][W];
  __shared__ int s_r[R][3];
  __shared__ float2 s_val[R][CC];
  __shared__ int s_bin[W + T];

  const ItemRef ir = item_ref(pt);
  const SpreadItem it = ir.it;
  const int2* __restrict__ list = pt.list[ir.jj];
  const float4* __restrict__ qs = pt.qs[ir.jj];
  GT* __restrict__ grid = grids + (long long)ir.jj * C * g.ngrid;
  const int coil0 = blockIdx.y * CC;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const TileOrigin to = tile_origin(g, tp, it.tile);
  for (int i = tid; i < T * T * T * CC; i += kThreads) acc[i] = make_float2(0.f, 0.f);

  const int n = it.end - it.begin;
  for (int base = 0; base < n; base += R) {
    const int cnt = min(R, n - base);
    __syncthreads();
    stage_round<W, T, CC, R>(g, kc, C, coil0, to, list + it.begin + base, cnt, qs, vals,
                             pt.row0[ir.jj], s_w, s_r, s_val, tid);
    __syncthreads();
    bin_round<W, T>(s_r, s_bin, cnt, tid);
    __syncthreads();
    const int lz = warp;
    if (lz < to.e0) {
      const int pend = s_bin[lz + W];
      for (int p = s_bin[lz]; p < pend; ++p) {
        const int t0 = lz - s_r[p][0];
        if ((unsigned)t0 >= (unsigned)W) continue;
        const float wz = s_w[p][0][t0];
        const int r1 = s_r[p][1], r2 = s_r[p][2];
#pragma unroll
        for (int k0 = 0; k0 < (CC * W * W + 31) / 32; ++k0) {
          const int k = lane + 32 * k0;
          if (k < CC * W * W) {
            const int c = k % CC;
            const int tx2 = (k / CC) % W;
            const int ty1 = k / (CC * W);
            const int ly = r1 + ty1, lx = r2 + tx2;
            if ((unsigned)ly < (unsigned)to.e1 && (unsigned)lx < (unsigned)to.e2) {
              const float w = wz * s_w[p][1][ty1] * s_w[p][2][tx2];
              const float2 v = s_val[p][c];
              float2* a = acc + ((lz * T + ly) * T + lx) * CC + c;
              float2 cur = *a;
              cur.x = fmaf(w, v.x, cur.x);
              cur.y = fmaf(w, v.y, cur.y);
              *a = cur;
            }
          }
        }
      }
    }
  }
  __syncthreads();
  write_tile<T, CC, GT>(g, C, coil0, to, scratch_slot(pt, ir), acc, nullptr, grid, scratch, tid);
}

// Sum the partial tiles of split tiles in slot order (deterministic); COMP:
// Neumaier's compensated summation of the partials.
template <int T, int CC, typename GT, bool COMP>
__global__ void reduce_kernel(Geo g, int C, TilePlan tp, PhaseTable pt,
                              const float2* __restrict__ scratch, GT* __restrict__ grids) {
  const int jj = phase_of(pt.red0, pt.nphase, blockIdx.x);
  ReduceItem r = pt.reduces[jj][blockIdx.x - pt.red0[jj]];
  r.first += pt.slot0[jj];
  GT* __restrict__ grid = grids + (long long)jj * C * g.ngrid;
  const int coil0 = blockIdx.y * CC;
  const TileOrigin to = tile_origin(g, tp, r.tile);
  constexpr int kPts = T * T * T;
  const long long tile_elems = kPts * CC;
  for (int i = threadIdx.x; i < tile_elems; i += blockDim.x) {
    const int c = i % CC;
    const int pt = i / CC;
    const int lx = pt % T, ly = (pt / T) % T, lz = pt / (T * T);
    float2 s = make_float2(0.f, 0.f), e = make_float2(0.f, 0.f);
    for (int k = 0; k < r.count; ++k) {
      const float2 v =
          scratch[((long long)(r.first + k) * gridDim.y + blockIdx.y) * tile_elems + i];
      if constexpr (COMP) {
        const float tx = s.x + v.x, ty = s.y + v.y;
        e.x += fabsf(s.x) >= fabsf(v.x) ? (s.x - tx) + v.x : (v.x - tx) + s.x;
        e.y += fabsf(s.y) >= fabsf(v.y) ? (s.y - ty) + v.y : (v.y - ty) + s.y;
        s.x = tx;
        s.y = ty;
      } else {
        s.x += v.x;
        s.y += v.y;
      }
    }
    if constexpr (COMP) {
      s.x += e.x;
      s.y += e.y;
    }
    if (lz < to.e0 && ly < to.e1 && lx < to.e2 && coil0 + c < C) {
      const long long gi = ((long long)(to.o0 + lz) * g.g1 + (to.o1 + ly)) * g.g2 + (to.o2 + lx);
      grid_st(grid + (long long)(coil0 + c) * g.ngrid + gi, s);
    }
  }
}

template <int T, int CC, typename GT, bool COMP = false>
int launch_reduce(const Geo& g, int C, const TilePlan& tp, const PhaseTable& pt, int chunks,
                  GT* grids, const float2* scratch, cudaStream_t s) {
  const int nred = pt.red0[pt.nphase];
  if (nred == 0) return 0;
  reduce_kernel<T, CC, GT, COMP><<<dim3(nred, chunks), 256, 0, s>>>(g, C, tp, pt, scratch, grids);
  return 1;
}

template <int CC, typename GT, bool COMP>
int dispatch_coils(const Geo& g, const KernelCoefs& kc, int C, const TilePlan& tp,
                   const PhaseTable& pt, const float2* vals, GT* grids, float2* scratch,
                   int variant, cudaStream_t s) {
  const int chunks = (C + CC - 1) / CC;
  const dim3 grid(pt.item0[pt.nphase], chunks);
  const int mma_wpc = spread_mma_wpc(variant);
  const bool mma_cube = spread_mma_cube(variant);
  variant = spread_base(variant);
  if (COMP || variant == kSpreadShared) {
    const size_t smem = size_t(8 * 8 * 8) * CC * sizeof(float2) * (COMP ? 2 : 1);
    spread_coils_kernel<CC, GT, COMP><<<grid, kThreads, smem, s>>>(g, kc, C, tp, pt, vals, grids,
                                                                   scratch);
  } else if (variant == kSpreadMMA && CC == 8 && mma_cube && pt.clist[0] != nullptr) {
    const unsigned blocks = 8u * pt.item0[pt.nphase];
    if (mma_wpc == 4)
      spread_coils_cube_kernel<GT, 4><<<dim3(blocks / 4, chunks), 128, 0, s>>>(
          g, kc, C, tp, pt, vals, grids, scratch);
    else if (mma_wpc == 2)
      spread_coils_cube_kernel<GT, 2><<<dim3(blocks / 2, chunks), 64, 0, s>>>(
          g, kc, C, tp, pt, vals, grids, scratch);
    else
      spread_coils_cube_kernel<GT, 1><<<dim3(blocks, chunks), 32, 0, s>>>(
          g, kc, C, tp, pt, vals, grids, scratch);
  } else if (variant == kSpreadMMA && CC == 8) {
    const unsigned planes = 8u * pt.item0[pt.nphase];
    if (mma_wpc == 4)
      spread_coils_mma_kernel<GT, 4><<<dim3(planes / 4, chunks), 128, 0, s>>>(
          g, kc, C, tp, pt, vals, grids, scratch);
    else if (mma_wpc == 2)
      spread_coils_mma_kernel<GT, 2><<<dim3(planes / 2, chunks), 64, 0, s>>>(
          g, kc, C, tp, pt, vals, grids, scratch);
    else
      spread_coils_mma_kernel<GT, 1><<<dim3(planes, chunks), 32, 0, s>>>(
          g, kc, C, tp, pt, vals, grids, scratch);
  } else if (variant == kSpreadRegisterWarp || variant == kSpreadMMA) {
    const dim3 wgrid(8u * pt.item0[pt.nphase], chunks);
    spread_coils_reg_kernel<CC, GT, 1><<<wgrid, 32, 0, s>>>(g, kc, C, tp, pt, vals, grids,
                                                            scratch);
  } else {
    spread_coils_reg_kernel<CC, GT, 8><<<grid, kThreads, 0, s>>>(g, kc, C, tp, pt, vals, grids,
                                                                 scratch);
  }
  return 1 + launch_reduce<8, CC, GT, COMP>(g, C, tp, pt, chunks, grids, scratch, s);
}

template <int W, int CC, typename GT>
int dispatch_generic(const Geo& g, const KernelCoefs& kc, int C, const TilePlan& tp,
                     const PhaseTable& pt, const float2* vals, GT* grids, float2* scratch,
                     cudaStream_t s) {
  const int chunks = (C + CC - 1) / CC;
  const size_t smem = size_t(8 * 8 * 8) * CC * sizeof(float2);
  spread_generic_kernel<W, CC, GT><<<dim3(pt.item0[pt.nphase], chunks), kThreads, smem, s>>>(
      g, kc, C, tp, pt, vals, grids, scratch);
  return 1 + launch_reduce<8, CC, GT>(g, C, tp, pt, chunks, grids, scratch, s);
}

template <typename GT, bool COMP>
int spread_multi(const Geo& g, int W, const KernelCoefs& kc, int C, const TilePlan& tp,
                 const PhaseTable& pt, const float2* v, GT* gr, float2* sc, int variant,
                 cudaStream_t s) {
  if (W == 4) {
    if (C == 1) return dispatch_generic<4, 1, GT>(g, kc, C, tp, pt, v, gr, sc, s);
    if (C <= 2) return dispatch_coils<2, GT, COMP>(g, kc, C, tp, pt, v, gr, sc, variant, s);
    if (C <= 4) return dispatch_coils<4, GT, COMP>(g, kc, C, tp, pt, v, gr, sc, variant, s);
    return dispatch_coils<8, GT, COMP>(g, kc, C, tp, pt, v, gr, sc, variant, s);
  }
  if (C == 1) return dispatch_generic<6, 1, GT>(g, kc, C, tp, pt, v, gr, sc, s);
  if (C <= 2) return dispatch_generic<6, 2, GT>(g, kc, C, tp, pt, v, gr, sc, s);
  if (C <= 4) return dispatch_generic<6, 4, GT>(g, kc, C, tp, pt, v, gr, sc, s);
  return dispatch_generic<6, 8, GT>(g, kc, C, tp, pt, v, gr, sc, s);
}

template <typename GT, bool COMP>
cudaError_t set_coils_smem() {
  const int big = 96 * 1024;
  cudaError_t e = cudaFuncSetAttribute(spread_coils_kernel<8, GT, COMP>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(spread_coils_kernel<4, GT, COMP>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(spread_coils_kernel<2, GT, COMP>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  return e;
}

}  // namespace

cudaError_t configure_spread_kernels() {
  const int big = 96 * 1024;
  cudaError_t e = set_coils_smem<float2, false>();
  if (e == cudaSuccess) e = set_coils_smem<float2, true>();
  if (e == cudaSuccess) e = set_coils_smem<bf162, false>();
  if (e == cudaSuccess) e = set_coils_smem<bf162, true>();
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(spread_single_kernel<false, 8>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(spread_single_kernel<true, 8>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  return e;
}

int spread_tile_edge(int W, int C, int gmin) {
  return (W == 4 && C == 1 && gmin >= 16 + W - 1) ? 16 : 8;
}

int spread_coil_chunk(int C) { return C == 1 ? 1 : (C <= 2 ? 2 : (C <= 4 ? 4 : 8)); }

int launch_spread(const Geo& g, int W, const KernelCoefs& kc, int C, const TilePlan& tp,
                  const PhaseTable& pt, const nrsense_c64* vals, void* grids, bool bf16,
                  bool comp, int variant, nrsense_c64* scratch, int32_t* status, cudaStream_t s) {
  (void)status;
  if (pt.item0[pt.nphase] == 0) return 0;
  const auto* v = reinterpret_cast<const float2*>(vals);
  auto* sc = reinterpret_cast<float2*>(scratch);
  if (W == 4 && C == 1 && tp.t0 == 16 && !bf16) {
    // single channel (image space), FP32 grid; variant == kSpreadRegisterWarp
    // selects a CTA per plane pair
    auto* gr = static_cast<float2*>(grids);
    const bool per_warp = variant == kSpreadRegisterWarp;
    const int np = per_warp ? 2 : 16;
    const size_t smem = size_t(np * 16 * 20) * sizeof(float2) * (comp ? 2 : 1);
    const unsigned items = pt.item0[pt.nphase];
    const dim3 grid(per_warp ? 8u * items : items, 1);
    const int threads = per_warp ? 32 : kThreads;
    if (comp) {
      if (per_warp)
        spread_single_kernel<true, 1><<<grid, threads, smem, s>>>(g, kc, tp, pt, v, gr, sc);
      else
        spread_single_kernel<true, 8><<<grid, threads, smem, s>>>(g, kc, tp, pt, v, gr, sc);
      return 1 + launch_reduce<16, 1, float2, true>(g, 1, tp, pt, 1, gr, sc, s);
    }
    if (per_warp)
      spread_single_kernel<false, 1><<<grid, threads, smem, s>>>(g, kc, tp, pt, v, gr, sc);
    else
      spread_single_kernel<false, 8><<<grid, threads, smem, s>>>(g, kc, tp, pt, v, gr, sc);
    return 1 + launch_reduce<16, 1, float2>(g, 1, tp, pt, 1, gr, sc, s);
  }
  if (bf16) {
    auto* gb = static_cast<bf162*>(grids);
    return comp ? spread_multi<bf162, true>(g, W, kc, C, tp, pt, v, gb, sc, variant, s)
                : spread_multi<bf162, false>(g, W, kc, C, tp, pt, v, gb, sc, variant, s);
  }
  auto* gf = static_cast<float2*>(grids);
  return comp ? spread_multi<float2, true>(g, W, kc, C, tp, pt, v, gf, sc, variant, s)
              : spread_multi<float2, false>(g, W, kc, C, tp, pt, v, gf, sc, variant, s);
}

}  // namespace nrs
