// Projection Cores P^(k) (k-space gridding) and P_j^(i) (adjoint image-space
// gridding): spread point values onto the oversampled grid,
//     grid[g, c] = sum_p c3(q_p - g) vals[p, c]
// (section "k-space Gridding", Projection Core; section "Image-space
// Gridding", adjoint diagram).
//
// Output-stationary and atomic-free: each CTA owns one 8x8x8 grid tile (and a
// chunk of coils), reads the plan-time list of points whose W^3 footprint
// touches the tile, and accumulates in shared memory.  Warp w owns tile plane
// w (axis 0), so every shared-memory address is updated by one warp only, in
// list order: the result is bitwise deterministic.  A heavy tile is split over
// several CTAs that write partial tiles to scratch; a second kernel adds the
// partials in a fixed order.
#include "plan_internal.h"

namespace nrs {

namespace {

constexpr int kTile = kSpreadTile;  // tile edge (grid points); 8 warps own 8 planes
constexpr int kStage = 32;        // points staged per round
constexpr int kThreads = 256;

template <int W, int CC>
__global__ void __launch_bounds__(kThreads) spread_kernel(
    Geo g, KernelCoefs kc, int C, TilePlan tp, const SpreadItem* __restrict__ items,
    const int32_t* __restrict__ list, const float4* __restrict__ qs,
    const int32_t* __restrict__ perm, const float2* __restrict__ vals,
    float2* __restrict__ grid, float2* __restrict__ scratch) {
  extern __shared__ float4 smem_raw[];
  float2* acc = reinterpret_cast<float2*>(smem_raw);  // [8][8][8][CC]
  __shared__ float s_w[kStage][3][W];
  __shared__ int s_rel[kStage][3];
  __shared__ float2 s_val[kStage][CC];

  const SpreadItem it = items[blockIdx.x];
  const int coil0 = blockIdx.y * CC;
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;

  const int tz = it.tile / (tp.nt1 * tp.nt2);
  const int rem = it.tile - tz * (tp.nt1 * tp.nt2);
  const int ty = rem / tp.nt2;
  const int tx = rem - ty * tp.nt2;
  const int o0 = tz * kTile, o1 = ty * kTile, o2 = tx * kTile;
  const int e0 = min(kTile, g.g0 - o0), e1 = min(kTile, g.g1 - o1), e2 = min(kTile, g.g2 - o2);

  for (int i = tid; i < kTile * kTile * kTile * CC; i += kThreads) acc[i] = make_float2(0.f, 0.f);

  const int n = it.end - it.begin;
  for (int base = 0; base < n; base += kStage) {
    const int cnt = min(kStage, n - base);
    __syncthreads();  // previous round fully consumed (and acc zeroed)
    if (tid < cnt * 3) {
      const int p = tid / 3, a = tid - 3 * (tid / 3);
      const int si = list[it.begin + base + p];
      const float4 q = __ldg(qs + si);
      int b[3];
      unpack_base(__float_as_uint(q.w), b[0], b[1], b[2]);
      const float f = a == 0 ? q.x : (a == 1 ? q.y : q.z);
      float w[W];
      kernel_weights<W>(f, kc, w);
#pragma unroll
      for (int t = 0; t < W; ++t) s_w[p][a][t] = w[t];
      const int o = a == 0 ? o0 : (a == 1 ? o1 : o2);
      const int G = a == 0 ? g.g0 : (a == 1 ? g.g1 : g.g2);
      int r = b[a] - o;
      if (r < 0) r += G;
      s_rel[p][a] = r;  // first tap's offset from the tile origin, mod G
    }
    for (int i = tid; i < cnt * CC; i += kThreads) {
      const int p = i / CC, c = i - p * CC;
      const int si = list[it.begin + base + p];
      s_val[p][c] = (coil0 + c < C) ? __ldg(vals + (long long)__ldg(perm + si) * C + coil0 + c)
                                    : make_float2(0.f, 0.f);
    }
    __syncthreads();
    // warp `warp` owns plane lz = warp
    const int lz = warp;
    if (lz < e0) {
      for (int p = 0; p < cnt; ++p) {
        int t0 = lz - s_rel[p][0];
        if (t0 < 0) t0 += g.g0;
        if (t0 >= W) continue;  // warp-uniform
        const float wz = s_w[p][0][t0];
        const int r1 = s_rel[p][1], r2 = s_rel[p][2];
        // combos (c fastest, then tap x, then tap y)
        for (int k = lane; k < CC * W * W; k += 32) {
          const int c = k % CC;
          const int tx2 = (k / CC) % W;
          const int ty1 = k / (CC * W);
          int ly = r1 + ty1;
          if (ly >= g.g1) ly -= g.g1;
          int lx = r2 + tx2;
          if (lx >= g.g2) lx -= g.g2;
          if (ly < e1 && lx < e2) {
            const float w = wz * s_w[p][1][ty1] * s_w[p][2][tx2];
            const float2 v = s_val[p][c];
            float2* a = acc + ((lz * kTile + ly) * kTile + lx) * CC + c;
            float2 cur = *a;
            cur.x = fmaf(w, v.x, cur.x);
            cur.y = fmaf(w, v.y, cur.y);
            *a = cur;
          }
        }
      }
    }
  }
  __syncthreads();
  // write the tile (or the partial tile)
  if (it.slot < 0) {
    for (int i = tid; i < kTile * kTile * kTile * CC; i += kThreads) {
      const int c = i % CC;
      const int pt = i / CC;
      const int lx = pt % kTile, ly = (pt / kTile) % kTile, lz = pt / (kTile * kTile);
      if (lz < e0 && ly < e1 && lx < e2 && coil0 + c < C) {
        const long long gi = ((long long)(o0 + lz) * g.g1 + (o1 + ly)) * g.g2 + (o2 + lx);
        grid[gi * C + coil0 + c] = acc[i];
      }
    }
  } else {
    float2* dst = scratch + ((long long)it.slot * gridDim.y + blockIdx.y) * (kTile * kTile * kTile * CC);
    for (int i = tid; i < kTile * kTile * kTile * CC; i += kThreads) dst[i] = acc[i];
  }
}

// Sum the partial tiles of split tiles in slot order (deterministic).
template <int CC>
__global__ void reduce_kernel(Geo g, int C, TilePlan tp, const ReduceItem* __restrict__ red,
                              const float2* __restrict__ scratch, float2* __restrict__ grid) {
  const ReduceItem r = red[blockIdx.x];
  const int coil0 = blockIdx.y * CC;
  const int tz = r.tile / (tp.nt1 * tp.nt2);
  const int rem = r.tile - tz * (tp.nt1 * tp.nt2);
  const int ty = rem / tp.nt2;
  const int tx = rem - ty * tp.nt2;
  const int o0 = tz * kTile, o1 = ty * kTile, o2 = tx * kTile;
  const int e0 = min(kTile, g.g0 - o0), e1 = min(kTile, g.g1 - o1), e2 = min(kTile, g.g2 - o2);
  const long long tile_elems = kTile * kTile * kTile * CC;
  for (int i = threadIdx.x; i < tile_elems; i += blockDim.x) {
    const int c = i % CC;
    const int pt = i / CC;
    const int lx = pt % kTile, ly = (pt / kTile) % kTile, lz = pt / (kTile * kTile);
    float2 s = make_float2(0.f, 0.f);
    for (int k = 0; k < r.count; ++k) {
      const float2 v = scratch[((long long)(r.first + k) * gridDim.y + blockIdx.y) * tile_elems + i];
      s.x += v.x;
      s.y += v.y;
    }
    if (lz < e0 && ly < e1 && lx < e2 && coil0 + c < C) {
      const long long gi = ((long long)(o0 + lz) * g.g1 + (o1 + ly)) * g.g2 + (o2 + lx);
      grid[gi * C + coil0 + c] = s;
    }
  }
}

template <int W, int CC>
int spread_dispatch(const Geo& g, const KernelCoefs& kc, int C, const TilePlan& tp,
                     const PointSet& ps, const float2* vals, float2* grid, float2* scratch,
                     cudaStream_t s) {
  const int coil_chunks = (C + CC - 1) / CC;
  const size_t smem = size_t(kTile) * kTile * kTile * CC * sizeof(float2);  // <= 32 KB
  dim3 grid_dim(ps.n_items, coil_chunks);
  spread_kernel<W, CC><<<grid_dim, kThreads, smem, s>>>(g, kc, C, tp, ps.items, ps.list, ps.qs,
                                                        ps.perm, vals, grid, scratch);
  if (ps.n_reduces > 0) {
    dim3 rd(ps.n_reduces, coil_chunks);
    reduce_kernel<CC><<<rd, 256, 0, s>>>(g, C, tp, ps.reduces, scratch, grid);
    return 2;
  }
  return 1;
}

}  // namespace

int launch_spread(const Geo& g, int W, const KernelCoefs& kc, int C, const TilePlan& tp,
                   const PointSet& ps, const nrsense_c64* vals, nrsense_c64* grid,
                   nrsense_c64* scratch, int32_t* status, cudaStream_t s) {
  (void)status;
  if (ps.n_items == 0) return 0;
  const auto* v = reinterpret_cast<const float2*>(vals);
  auto* gr = reinterpret_cast<float2*>(grid);
  auto* sc = reinterpret_cast<float2*>(scratch);
  if (W == 4) {
    if (C == 1) return spread_dispatch<4, 1>(g, kc, C, tp, ps, v, gr, sc, s);
    else if (C <= 2) return spread_dispatch<4, 2>(g, kc, C, tp, ps, v, gr, sc, s);
    else if (C <= 4) return spread_dispatch<4, 4>(g, kc, C, tp, ps, v, gr, sc, s);
    else return spread_dispatch<4, 8>(g, kc, C, tp, ps, v, gr, sc, s);
  } else {
    if (C == 1) return spread_dispatch<6, 1>(g, kc, C, tp, ps, v, gr, sc, s);
    else if (C <= 2) return spread_dispatch<6, 2>(g, kc, C, tp, ps, v, gr, sc, s);
    else if (C <= 4) return spread_dispatch<6, 4>(g, kc, C, tp, ps, v, gr, sc, s);
    else return spread_dispatch<6, 8>(g, kc, C, tp, ps, v, gr, sc, s);
  }
}

int spread_coil_chunk(int C) { return C == 1 ? 1 : (C <= 2 ? 2 : (C <= 4 ? 4 : 8)); }

}  // namespace nrs
