// Projection Core P_j^(i) of the adjoint image-space gridding (section
// "Image-space Gridding", adjoint diagram), all phases into one grid,
//     u[g] = sum_j sum_n c3(sigma (n + d_j[n]) - g) w_j[n],
// by home tiles instead of halo lists.
//
// Every displaced voxel is spread exactly once, by the warp that owns the
// 8^3 home tile holding its first tap.  The warp keeps an 11^3 accumulator in
// shared memory (the tile plus the W - 1 = 3 points its footprints reach past
// the tile's high side), so all 64 taps of a point land inside it: no halo
// lists, no bounds tests, one read-modify-write per tap.  Lane (x, y, z-pair)
// updates taps (z, y, x) and (z + 2, y, x) of each point in list order, so the
// sum at every accumulator position is bitwise reproducible.
//
// A CTA is a 16^3 super-tile of 2 x 2 x 2 home tiles (one warp each).  After
// its warps are done it adds the eight accumulators, in warp order, into the
// super-tile's 19^3 padded region.  The core of the region, the positions at
// least 3 past the super-tile's low faces, receives nothing from any other
// super-tile: it goes straight to the grid.  The rest (the low 3-wide rim, the
// high 3-wide rim and any position that wraps around the periodic grid) goes
// to a scratch slot of the super-tile, and a second kernel sums, for every grid
// point outside the cores, the scratch values of the (at most 2 per axis)
// super-tiles whose padded regions cover it, in a fixed order.
//
// Covers along one axis (plan time): super-tile c (origin 16 c, extent
// e_c = min(16, G - 16 c)) covers grid coordinate x at position x - 16 c if
// 16 c <= x < 16 c + e_c + 3, and at x + G - 16 c if the same holds for x + G
// (its rim wraps around the periodic grid).
#include "plan_internal.h"

namespace nrs {

namespace {

constexpr int kHT = 8;                  // home tile edge (one warp)
constexpr int kHS = 2 * kHT;            // super-tile edge (one CTA)
constexpr int kHA = kHT + 3;            // accumulator extent along z and y
constexpr int kHAX = 12;                // accumulator row stride along x (11 used)
constexpr int kHAcc = kHA * kHA * kHAX;  // float2 per warp accumulator
constexpr int kHP = kHS + 3;            // padded super-tile extent (scratch layout)
constexpr int kHWarps = 8;
constexpr int kHB = 32;                 // points staged per batch

static_assert(kHAX >= kHA, "accumulator rows");

// one staged point: weights (z in the order 0, 2, 1, 3 so that a lane's two
// z taps are one 8-byte load), accumulator offset of the first tap, value;
// 80-byte records: the 16-byte stores of a quarter-warp hit disjoint banks
struct HomeStage {
  float wz[4];
  float wy[4];
  float wx[4];
  int off;
  float vx, vy;
  int pad;
  float pad2[4];
};
static_assert(sizeof(HomeStage) == 80, "staging record");

__device__ __forceinline__ int home_extent(int G, int o) { return min(kHS, G - o); }

}  // namespace

__global__ void __launch_bounds__(32 * kHWarps, 2)
    spread_home_kernel(Geo g, KernelCoefs kc, HomeSet hs, const float2* __restrict__ vals,
                       float2* __restrict__ grid, float2* __restrict__ scratch) {
  extern __shared__ float4 smem_home[];
  float2* acc_all = reinterpret_cast<float2*>(smem_home);  // [warp][kHAcc]
  // a separate array: its loads may move ahead of the accumulator stores
  __shared__ __align__(16) HomeStage stg_all[kHWarps * kHB];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // super-tile and its extents
  const int s = blockIdx.x;
  const int s2 = s % hs.ns2, s1 = (s / hs.ns2) % hs.ns1, s0 = s / (hs.ns2 * hs.ns1);
  const int o0 = kHS * s0, o1 = kHS * s1, o2 = kHS * s2;
  const int e0 = home_extent(g.g0, o0), e1 = home_extent(g.g1, o1), e2 = home_extent(g.g2, o2);
  // this warp's home tile
  const int w0 = (warp >> 2) & 1, w1 = (warp >> 1) & 1, w2 = warp & 1;
  const bool live = kHT * w0 < e0 && kHT * w1 < e1 && kHT * w2 < e2;
  float2* acc = acc_all + warp * kHAcc;
  HomeStage* stg = stg_all + warp * kHB;
  static_assert(kHAcc % 2 == 0, "16-byte zeroing");
  for (int i = lane; i < kHAcc / 2; i += 32)
    reinterpret_cast<float4*>(acc)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  __syncwarp();
  if (live) {
    const int t = ((2 * s0 + w0) * hs.nt1 + (2 * s1 + w1)) * hs.nt2 + (2 * s2 + w2);
    const int beg = __ldg(hs.tstart + t), end = __ldg(hs.tstart + t + 1);
    const int h0 = o0 + kHT * w0, h1 = o1 + kHT * w1, h2 = o2 + kHT * w2;  // home tile origin
    const int tx = lane & 3, ty = (lane >> 2) & 3, tz = lane >> 4;
    const int lane_off = (tz * kHA + ty) * kHAX + tx;
    // the next batch's point records are loaded while this batch is applied,
    // and their values after it (the value row comes with the record)
    float4 qn = make_float4(0.f, 0.f, 0.f, 0.f);
    float2 vn = make_float2(0.f, 0.f);
    int rown = 0;
    if (beg + lane < end) {
      qn = __ldg(hs.qs + beg + lane);
      rown = __ldg(hs.perm + beg + lane);
      vn = __ldg(vals + rown);
    }
    for (int base = beg; base < end; base += kHB) {
      const int n = min(kHB, end - base);
      const float4 q = qn;
      const float2 v = vn;
      const bool more = base + kHB + lane < end;
      if (more) {
        qn = __ldg(hs.qs + base + kHB + lane);
        rown = __ldg(hs.perm + base + kHB + lane);
      }
      if (lane < n) {
        int b0, b1, b2;
        unpack_base(__float_as_uint(q.w), b0, b1, b2);
        // the first tap lies in the home tile: offsets in [0, 8)
        const int r0 = b0 - h0, r1 = b1 - h1, r2 = b2 - h2;
        float wz[4], wy[4], wx[4];
        kernel_weights<4>(q.x, kc, wz);
        kernel_weights<4>(q.y, kc, wy);
        kernel_weights<4>(q.z, kc, wx);
        float4* d = reinterpret_cast<float4*>(stg + lane);
        d[0] = make_float4(wz[0], wz[2], wz[1], wz[3]);
        d[1] = make_float4(wy[0], wy[1], wy[2], wy[3]);
        d[2] = make_float4(wx[0], wx[1], wx[2], wx[3]);
        d[3] = make_float4(__int_as_float((r0 * kHA + r1) * kHAX + r2), v.x, v.y, 0.f);
      }
      __syncwarp();
#pragma unroll 4
      for (int p = 0; p < n; ++p) {
        const HomeStage& d = stg[p];
        const float4 meta = *reinterpret_cast<const float4*>(&d.off);
        const float2 wzp = *reinterpret_cast<const float2*>(&d.wz[2 * tz]);
        const float wyx = d.wy[ty] * d.wx[tx];
        const float2 wab = __fmul2_rn(wzp, make_float2(wyx, wyx));
        const float2 vv = make_float2(meta.y, meta.z);
        float2* a = acc + __float_as_int(meta.x) + lane_off;
        float2 ca = a[0], cb = a[2 * kHA * kHAX];
        // paired FMAs: each part rounded as fmaf
        ca = __ffma2_rn(make_float2(wab.x, wab.x), vv, ca);
        cb = __ffma2_rn(make_float2(wab.y, wab.y), vv, cb);
        a[0] = ca;
        a[2 * kHA * kHAX] = cb;
      }
      if (more) vn = __ldg(vals + rown);
      __syncwarp();
    }
  }
  __syncthreads();
  // add the home tiles' accumulators into the padded super-tile region, in warp
  // order; a thread takes one (P1, P2) column of the region and keeps its 19
  // sums in registers.  The core goes to the grid, the rest to this
  // super-tile's scratch slot.
  const int p0n = e0 + 3, p1n = e1 + 3, p2n = e2 + 3;
  float2* slot = scratch + (long long)s * (kHP * kHP * kHP);
  for (int c = tid; c < p1n * p2n; c += 32 * kHWarps) {
    const int P1 = c / p2n, P2 = c - P1 * p2n;
    float2 col[kHP];
#pragma unroll
    for (int k = 0; k < kHP; ++k) col[k] = make_float2(0.f, 0.f);
#pragma unroll
    for (int w0 = 0; w0 < 2; ++w0) {
      if (kHT * w0 >= e0) break;
#pragma unroll
      for (int w1 = 0; w1 < 2; ++w1) {
        const int a1 = P1 - kHT * w1;
        if (kHT * w1 >= e1 || (unsigned)a1 >= (unsigned)kHA) continue;
#pragma unroll
        for (int w2 = 0; w2 < 2; ++w2) {
          const int a2 = P2 - kHT * w2;
          if (kHT * w2 >= e2 || (unsigned)a2 >= (unsigned)kHA) continue;
          const float2* src = acc_all + ((w0 << 2) | (w1 << 1) | w2) * kHAcc + a1 * kHAX + a2;
#pragma unroll
          for (int a0 = 0; a0 < kHA; ++a0) {
            const float2 v = src[a0 * (kHA * kHAX)];
            col[kHT * w0 + a0].x += v.x;
            col[kHT * w0 + a0].y += v.y;
          }
        }
      }
    }
    const bool core12 = P1 >= 3 && P1 < e1 && P2 >= 3 && P2 < e2;
    float2* gcol = grid + ((long long)o0 * g.g1 + (o1 + P1)) * g.g2 + (o2 + P2);
    float2* scol = slot + P1 * kHP + P2;
    const long long plane = (long long)g.g1 * g.g2;
#pragma unroll
    for (int P0 = 0; P0 < kHP; ++P0) {
      if (P0 >= p0n) break;
      if (core12 && P0 >= 3 && P0 < e0)
        gcol[P0 * plane] = col[P0];
      else
        scol[P0 * (kHP * kHP)] = col[P0];
    }
  }
}

// Grid points of a super-tile outside its core (some position < 3): the sum
// of the scratch values of every super-tile whose padded region covers them.
// The covers of every coordinate along each axis (at most 3, increasing
// super-tile order, each packed as super-tile * 32 + position) come from
// plan-time tables, so every grid point sums in a fixed order.
__global__ void __launch_bounds__(256) home_rim_kernel(Geo g, HomeSet hs,
                                                       const float2* __restrict__ scratch,
                                                       float2* __restrict__ grid) {
  const int s = blockIdx.x;
  const int s2 = s % hs.ns2, s1 = (s / hs.ns2) % hs.ns1, s0 = s / (hs.ns2 * hs.ns1);
  const int o0 = kHS * s0, o1 = kHS * s1, o2 = kHS * s2;
  const int e0 = home_extent(g.g0, o0), e1 = home_extent(g.g1, o1), e2 = home_extent(g.g2, o2);
  const int r0 = min(3, e0), r1 = min(3, e1), r2 = min(3, e2);
  // the rim as three slabs: P0 < 3; P0 >= 3 and P1 < 3; P0, P1 >= 3 and P2 < 3
  const int na = r0 * e1 * e2, nb = (e0 - r0) * r1 * e2, nc = (e0 - r0) * (e1 - r1) * r2;
  const bool full = e0 == kHS && e1 == kHS && e2 == kHS;
  int t = blockIdx.y * blockDim.x + threadIdx.x;
  int P0, P1, P2;
  if (full && t < na + nb + nc) {
    // 16^3 super-tile: slabs of 768, 624 and 507 points, rows of 16 or 3
    if (t < 768) {
      P2 = t & 15;
      P1 = (t >> 4) & 15;
      P0 = t >> 8;
    } else if ((t -= 768) < 624) {
      P2 = t & 15;
      const int r = t >> 4;  // (P0 - 3) * 3 + P1
      P0 = 3 + r / 3;
      P1 = r - (P0 - 3) * 3;
    } else {
      t -= 624;
      const int r = t / 3;  // (P0 - 3) * 13 + (P1 - 3)
      P2 = t - 3 * r;
      P0 = 3 + r / 13;
      P1 = 3 + (r - (P0 - 3) * 13);
    }
  } else if (full) {
    return;
  } else if (t < na) {
    P2 = t % e2;
    P1 = (t / e2) % e1;
    P0 = t / (e2 * e1);
  } else if ((t -= na) < nb) {
    P2 = t % e2;
    P1 = (t / e2) % r1;
    P0 = r0 + t / (e2 * r1);
  } else if ((t -= nb) < nc) {
    P2 = t % r2;
    P1 = r1 + (t / r2) % (e1 - r1);
    P0 = r0 + t / (r2 * (e1 - r1));
  } else {
    return;
  }
  const int x0 = o0 + P0, x1 = o1 + P1, x2 = o2 + P2;
  const int4 c0 = __ldg(hs.cover0 + x0), c1 = __ldg(hs.cover1 + x1), c2 = __ldg(hs.cover2 + x2);
  const int a0[3] = {c0.y, c0.z, c0.w}, a1[3] = {c1.y, c1.z, c1.w}, a2[3] = {c2.y, c2.z, c2.w};
  float2 sum = make_float2(0.f, 0.f);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (a >= c0.x) break;
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      if (b >= c1.x) break;
      const long long row = ((long long)(a0[a] >> 5) * hs.ns1 + (a1[b] >> 5)) * hs.ns2;
      const int prow = ((a0[a] & 31) * kHP + (a1[b] & 31)) * kHP;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        if (c >= c2.x) break;
        const float2 v =
            __ldg(scratch + (row + (a2[c] >> 5)) * (kHP * kHP * kHP) + prow + (a2[c] & 31));
        sum.x += v.x;
        sum.y += v.y;
      }
    }
  }
  grid[((long long)x0 * g.g1 + x1) * g.g2 + x2] = sum;
}

// Backprojection Core B_j^(i) (section "Image-space Gridding", forward
// diagram) on the same super-tiles: m_j[n] = sum_taps c3(q - g) u[g mod G],
// q = sigma (n + d_j[n]).  A CTA copies the 19^3 padded region of its
// super-tile (16^3 plus the 3 points footprints reach past it, wrapped around
// the periodic grid) from u into shared memory with per-value asynchronous
// copies, then every thread takes displaced voxels of the super-tile's eight
// home tiles (all phases) and sums its 64 taps from shared memory: the gathers
// never leave the SM.  Taps are summed as the per-voxel kernel does (x taps
// weighted first, then the (z, y) weight), the result goes to the voxel's row.
constexpr int kHR = kHP;  // staged region extent per axis (19)

__global__ void __launch_bounds__(256) interp_home_kernel(Geo g, KernelCoefs kc, HomeSet hs,
                                                          const float2* __restrict__ u,
                                                          float2* __restrict__ m) {
  extern __shared__ float4 smem_ih[];
  float2* reg = reinterpret_cast<float2*>(smem_ih);  // [kHR][kHR][kHR]
  __shared__ int s_beg[kHWarps + 1], s_start[kHWarps];
  const int s = blockIdx.x;
  const int s2 = s % hs.ns2, s1 = (s / hs.ns2) % hs.ns1, s0 = s / (hs.ns2 * hs.ns1);
  const int o0 = kHS * s0, o1 = kHS * s1, o2 = kHS * s2;
  const int e0 = home_extent(g.g0, o0), e1 = home_extent(g.g1, o1), e2 = home_extent(g.g2, o2);
  const int p0n = e0 + 3, p1n = e1 + 3, p2n = e2 + 3;
  {
    // a warp copies (z, y) rows, lane = x (at most 19 of the 32 lanes)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int gx = wrap_once(o2 + lane, g.g2);
    for (int z = 0; z < p0n; ++z) {
      const long long zoff = (long long)wrap_once(o0 + z, g.g0) * g.g1;
      for (int y = warp; y < p1n; y += nw)
        if (lane < p2n)
          cp_async_8(reg + (z * kHR + y) * kHR + lane,
                     u + (zoff + wrap_once(o1 + y, g.g1)) * g.g2 + gx, true);
    }
  }
  if (threadIdx.x == 0) {
    // the points of the eight home tiles, as one flat range
    int acc = 0;
    for (int w = 0; w < kHWarps; ++w) {
      const int w0 = (w >> 2) & 1, w1 = (w >> 1) & 1, w2 = w & 1;
      int b = 0, n = 0;
      if (kHT * w0 < e0 && kHT * w1 < e1 && kHT * w2 < e2) {
        const int t = ((2 * s0 + w0) * hs.nt1 + (2 * s1 + w1)) * hs.nt2 + (2 * s2 + w2);
        b = __ldg(hs.tstart + t);
        n = __ldg(hs.tstart + t + 1) - b;
      }
      s_beg[w] = acc;
      s_start[w] = b;
      acc += n;
    }
    s_beg[kHWarps] = acc;
  }
  cp_async_wait_all();
  __syncthreads();
  const int total = s_beg[kHWarps];
  for (int f = threadIdx.x; f < total; f += blockDim.x) {
    int w = 0;
#pragma unroll
    for (int k = 1; k < kHWarps; ++k) w += f >= s_beg[k] ? 1 : 0;
    const int i = s_start[w] + (f - s_beg[w]);
    const float4 q = __ldg(hs.qs + i);
    const int row = __ldg(hs.perm + i);
    int b0, b1, b2;
    unpack_base(__float_as_uint(q.w), b0, b1, b2);
    float w0[4], w1[4], w2[4];
    kernel_weights<4>(q.x, kc, w0);
    kernel_weights<4>(q.y, kc, w1);
    kernel_weights<4>(q.z, kc, w2);
    const float2* base = reg + ((b0 - o0) * kHR + (b1 - o1)) * kHR + (b2 - o2);
    float2 aw = make_float2(0.f, 0.f);
#pragma unroll
    for (int t0 = 0; t0 < 4; ++t0)
#pragma unroll
      for (int t1 = 0; t1 < 4; ++t1) {
        const float w01 = w0[t0] * w1[t1];
        const float2* rowp = base + (t0 * kHR + t1) * kHR;
        float2 rw = make_float2(0.f, 0.f);
#pragma unroll
        for (int t2 = 0; t2 < 4; ++t2) {
          const float2 v = rowp[t2];
          rw = __ffma2_rn(make_float2(w2[t2], w2[t2]), v, rw);  // each part as fmaf
        }
        aw = __ffma2_rn(make_float2(w01, w01), rw, aw);
      }
    m[row] = aw;
  }
}

size_t interp_home_smem_bytes() { return size_t(kHR) * kHR * kHR * sizeof(float2); }

int launch_interp_home(const Geo& g, const KernelCoefs& kc, const HomeSet& hs,
                       const nrsense_c64* u, nrsense_c64* m, cudaStream_t s) {
  const unsigned nsuper = unsigned(hs.ns0 * hs.ns1 * hs.ns2);
  interp_home_kernel<<<nsuper, 256, interp_home_smem_bytes(), s>>>(
      g, kc, hs, reinterpret_cast<const float2*>(u), reinterpret_cast<float2*>(m));
  return 1;
}

size_t home_smem_bytes() { return size_t(kHWarps) * kHAcc * sizeof(float2); }

long long home_scratch_elems(const HomeSet& hs) {
  return (long long)hs.ns0 * hs.ns1 * hs.ns2 * (kHP * kHP * kHP);
}

cudaError_t configure_home_kernels() {
  const cudaError_t e = cudaFuncSetAttribute(
      spread_home_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(home_smem_bytes()));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(interp_home_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              int(interp_home_smem_bytes()));
}

int launch_spread_home(const Geo& g, const KernelCoefs& kc, const HomeSet& hs,
                       const nrsense_c64* vals, nrsense_c64* grid, nrsense_c64* scratch,
                       cudaStream_t s) {
  const unsigned nsuper = unsigned(hs.ns0 * hs.ns1 * hs.ns2);
  spread_home_kernel<<<nsuper, 32 * kHWarps, home_smem_bytes(), s>>>(
      g, kc, hs, reinterpret_cast<const float2*>(vals), reinterpret_cast<float2*>(grid),
      reinterpret_cast<float2*>(scratch));
  // rim points of a full super-tile: 16^3 - 13^3 = 1899
  constexpr int kRim = kHS * kHS * kHS - (kHS - 3) * (kHS - 3) * (kHS - 3);
  home_rim_kernel<<<dim3(nsuper, (kRim + 255) / 256), 256, 0, s>>>(
      g, hs, reinterpret_cast<const float2*>(scratch), reinterpret_cast<float2*>(grid));
  return 2;
}

}  // namespace nrs
