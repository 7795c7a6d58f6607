// Pruned coil-grid transforms (steps 5-6 and 9 of the operator) with the
// coil fan-out and the coil combination fused in.
//
// With sigma = 2 the data of a coil image occupy, along every axis, the
// grid positions [0, G/4) and [3G/4, G) (centred index n' = n - N/2 placed
// on the periodic grid); the rest of the zero-padded grid is zero.  So the
// forward 3D DFT of a padded coil grid runs as three passes of 1D DFTs of
// length G that load only the data half of their inputs: along x for the
// N0 x N1 data rows (computing S_c m_j / C3 on the fly from the phase image
// and the coil map: the coil fan-out), along y for the N0 data planes, along
// z for every (y, x) column.  The adjoint runs the passes in the other order
// and stores only the data half of their outputs; its last pass (along x)
// multiplies by conj(S_c) / C3 and sums the coils of a phase in coil order
// (the coil combination).  Intermediates are compact: T1[slot][i0][i1][x]
// (data planes and rows, full x) and T2[slot][i0][y][x] (data planes), with
// the plane and row index the image index.
//
// One CTA computes 16 transforms of length L = R1 R2 (Cooley-Tukey with
// n = R2 n1 + n2, k = k1 + R1 k2): threads n2 < R2 load x[R2 n1 + n2] for the
// data n1, run a radix-2 DFT of length R1 in registers and multiply by
// W_L^(n2 k1); after an exchange through shared memory threads k1 < R1 run
// the length-R2 DFTs and write X[k1 + R1 k2].  Loads and stores of a fixed n1
// (k2) are contiguous over the 16 transforms (columns) or over n2 (k1)
// (rows).  No scaling (as cuFFT): forward exp(-2 pi i n k / L), inverse
// exp(+2 pi i n k / L).
#include <cmath>

#include "plan_internal.h"

namespace nrs {

namespace {

constexpr int kCols = 16;  // transforms per CTA

__constant__ float2 c_w16[16];  // exp(-2 pi i j / 16)

__host__ __device__ constexpr int bitrev(int i, int r) {
  int o = 0;
  for (int b = 1; b < r; b <<= 1) {
    o = (o << 1) | (i & 1);
    i >>= 1;
  }
  return o;
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// In-register radix-2 DFT of length R (R <= 16): a[k] = sum_n a[n] W_R^(+-nk).
template <int R, bool INV>
__device__ __forceinline__ void dft(float2 (&a)[R]) {
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const int j = bitrev(i, R);
    if (j > i) {
      const float2 t = a[i];
      a[i] = a[j];
      a[j] = t;
    }
  }
#pragma unroll
  for (int len = 2; len <= R; len <<= 1) {
    const int half = len >> 1;
#pragma unroll
    for (int i = 0; i < R; i += len) {
#pragma unroll
      for (int k = 0; k < half; ++k) {
        float2 w = c_w16[(16 / len) * k];
        if (INV) w.y = -w.y;
        const float2 u = a[i + k];
        const float2 v = cmul(a[i + k + half], w);
        a[i + k] = make_float2(u.x + v.x, u.y + v.y);
        a[i + k + half] = make_float2(u.x - v.x, u.y - v.y);
      }
    }
  }
}

// image index of data grid position n (centred placement, G = 2N)
__device__ __forceinline__ int img_of(int n, int N, int G) {
  return n < (N >> 1) ? n + (N >> 1) : n - G + (N >> 1);
}
template <int R1, int R2>
struct Shape {
  static constexpr int L = R1 * R2;
  static constexpr int T = R1 > R2 ? R1 : R2;
  static constexpr int threads = kCols * T;
  static constexpr int ypitch = R2 + 1;  // row-pass shared pitch (float2), breaks bank stride
  static constexpr int smem = kCols * R1 * ypitch > kCols * R1 * R2 ? kCols * R1 * ypitch
                                                                     : kCols * R1 * R2;
};

// exp(-2 pi i j / L), j < L, into shared memory (every thread of the CTA
// calls it; a barrier follows before use)
template <int L>
__device__ __forceinline__ void fill_twiddles(float2* tw) {
  for (int j = threadIdx.x; j < L; j += blockDim.x) {
    float sn, cs;
    sincospif(-2.0f * float(j) / float(L), &sn, &cs);
    tw[j] = make_float2(cs, sn);
  }
  __syncthreads();
}

// The two-step transform of 16 columns.  ROWS: transform elements are
// contiguous (threads: n2 fastest); else columns are (threads: column
// fastest).  PIN: load only the data half of the input; POUT: store only the
// data half of the output.  ld(col, n) -> float2, st(col, k, k2, value) with
// k = k1 + R1 k2 (k2 a compile-time index after unrolling).
// Shared exchange layout: row passes keep n2 fastest (a warp spans n2 and
// k1 of a few rows), column passes keep the column fastest (a warp spans the
// 16 columns), so neither direction of the exchange has bank conflicts.
template <int R1, int R2, bool ROWS>
__device__ __forceinline__ int yidx(int col, int k1, int n2) {
  return ROWS ? (col * R1 + k1) * Shape<R1, R2>::ypitch + n2 : (k1 * R2 + n2) * kCols + col;
}

template <int R1, int R2, bool INV, bool ROWS, bool PIN, bool POUT, class Ld, class St>
__device__ __forceinline__ void fft16(float2* sy, const float2* tw, const Ld& ld, const St& st) {
  using S = Shape<R1, R2>;
  const int tid = threadIdx.x;
  const int col = ROWS ? tid / S::T : tid % kCols;
  const int t = ROWS ? tid % S::T : tid / kCols;
  if (t < R2) {
    float2 a[R1];
#pragma unroll
    for (int n1 = 0; n1 < R1; ++n1) {
      const bool data = !PIN || n1 < R1 / 4 || n1 >= 3 * R1 / 4;
      a[n1] = data ? ld(col, R2 * n1 + t) : make_float2(0.f, 0.f);
    }
    dft<R1, INV>(a);
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) {
      float2 w = tw[(t * k1) % S::L];
      if (INV) w.y = -w.y;
      sy[yidx<R1, R2, ROWS>(col, k1, t)] = cmul(a[k1], w);
    }
  }
  __syncthreads();
  if (t < R1) {
    float2 b[R2];
#pragma unroll
    for (int n2 = 0; n2 < R2; ++n2) b[n2] = sy[yidx<R1, R2, ROWS>(col, t, n2)];
    dft<R2, INV>(b);
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) {
      const bool data = !POUT || k2 < R2 / 4 || k2 >= 3 * R2 / 4;
      if (data) st(col, t + R1 * k2, k2, b[k2]);
    }
  }
  __syncthreads();
}

struct PassGeo {
  int n0, n1, n2, g0, g1, g2;
  int C, nph;
};

// F1: T1[slot][i0][i1][:] = DFT_x of S_c m_j / C3 on the data row (i0, i1),
// for every coil c of phase jj.  CTA: (jj, i0, block of 16 rows i1).
template <int R1, int R2>
__global__ void __launch_bounds__(Shape<R1, R2>::threads, 4) fwd_x_kernel(
    PassGeo g, const float* __restrict__ dtab, const float2* __restrict__ smaps,
    const float2* __restrict__ m, float2* __restrict__ t1) {
  __shared__ float2 sy[Shape<R1, R2>::smem];
  __shared__ float2 tw[R1 * R2];
  fill_twiddles<R1 * R2>(tw);
  const int rb = blockIdx.x, i0 = blockIdx.y, jj = blockIdx.z;
  const long long nvox = (long long)g.n0 * g.n1 * g.n2;
  const float d0 = __ldg(dtab + i0);
  for (int c = 0; c < g.C; ++c) {
    const long long slot = (long long)jj * g.C + c;
    auto ld = [&](int col, int n) -> float2 {
      const int i1 = rb * kCols + col;
      if (i1 >= g.n1) return make_float2(0.f, 0.f);
      const int i2 = img_of(n, g.n2, g.g2);
      const long long v = ((long long)i0 * g.n1 + i1) * g.n2 + i2;
      const float2 mv = __ldg(m + jj * nvox + v);
      const float2 sv = __ldg(smaps + c * nvox + v);
      const float w = d0 * __ldg(dtab + g.n0 + i1) * __ldg(dtab + g.n0 + g.n1 + i2);
      return make_float2((sv.x * mv.x - sv.y * mv.y) * w, (sv.x * mv.y + sv.y * mv.x) * w);
    };
    auto st = [&](int col, int k, int, float2 v) {
      const int i1 = rb * kCols + col;
      if (i1 < g.n1) t1[((slot * g.n0 + i0) * g.n1 + i1) * g.g2 + k] = v;
    };
    fft16<R1, R2, false, true, true, false>(sy, tw, ld, st);
  }
}

// F2: T2[slot][i0][:][x] = DFT_y of T1[slot][i0][data rows][x].
// CTA: (block of 16 x, i0, slot).
template <int R1, int R2>
__global__ void __launch_bounds__(Shape<R1, R2>::threads) fwd_y_kernel(
    PassGeo g, const float2* __restrict__ t1, float2* __restrict__ t2) {
  __shared__ float2 sy[Shape<R1, R2>::smem];
  __shared__ float2 tw[R1 * R2];
  fill_twiddles<R1 * R2>(tw);
  const int xb = blockIdx.x, i0 = blockIdx.y;
  const long long slot = blockIdx.z;
  const float2* src = t1 + (slot * g.n0 + i0) * g.n1 * (long long)g.g2;
  float2* dst = t2 + (slot * g.n0 + i0) * g.g1 * (long long)g.g2;
  auto ld = [&](int col, int n) -> float2 {
    return src[(long long)img_of(n, g.n1, g.g1) * g.g2 + xb * kCols + col];
  };
  auto st = [&](int col, int k, int, float2 v) {
    dst[(long long)k * g.g2 + xb * kCols + col] = v;
  };
  fft16<R1, R2, false, false, true, false>(sy, tw, ld, st);
}

// F3: grid[slot][:][y][x] = DFT_z of T2[slot][data planes][y][x].
// CTA: (block of 16 x, y, slot).
template <int R1, int R2>
__global__ void __launch_bounds__(Shape<R1, R2>::threads) fwd_z_kernel(
    PassGeo g, const float2* __restrict__ t2, float2* __restrict__ grid) {
  __shared__ float2 sy[Shape<R1, R2>::smem];
  __shared__ float2 tw[R1 * R2];
  fill_twiddles<R1 * R2>(tw);
  const int xb = blockIdx.x, y = blockIdx.y;
  const long long slot = blockIdx.z;
  const long long plane = (long long)g.g1 * g.g2;
  const float2* src = t2 + slot * g.n0 * plane + (long long)y * g.g2 + xb * kCols;
  float2* dst = grid + slot * g.g0 * plane + (long long)y * g.g2 + xb * kCols;
  auto ld = [&](int col, int n) -> float2 { return src[img_of(n, g.n0, g.g0) * plane + col]; };
  auto st = [&](int col, int k, int, float2 v) { dst[k * plane + col] = v; };
  fft16<R1, R2, false, false, true, false>(sy, tw, ld, st);
}

// I3: T2[slot][i0][y][x] = (inverse DFT_z of grid[slot][:][y][x]) at the data planes.
template <int R1, int R2>
__global__ void __launch_bounds__(Shape<R1, R2>::threads) inv_z_kernel(
    PassGeo g, const float2* __restrict__ grid, float2* __restrict__ t2) {
  __shared__ float2 sy[Shape<R1, R2>::smem];
  __shared__ float2 tw[R1 * R2];
  fill_twiddles<R1 * R2>(tw);
  const int xb = blockIdx.x, y = blockIdx.y;
  const long long slot = blockIdx.z;
  const long long plane = (long long)g.g1 * g.g2;
  const float2* src = grid + slot * g.g0 * plane + (long long)y * g.g2 + xb * kCols;
  float2* dst = t2 + slot * g.n0 * plane + (long long)y * g.g2 + xb * kCols;
  auto ld = [&](int col, int n) -> float2 { return src[n * plane + col]; };
  auto st = [&](int col, int k, int, float2 v) {
    dst[img_of(k, g.n0, g.g0) * plane + col] = v;
  };
  fft16<R1, R2, true, false, false, true>(sy, tw, ld, st);
}

// I2: T1[slot][i0][i1][x] = (inverse DFT_y of T2[slot][i0][:][x]) at the data rows.
template <int R1, int R2>
__global__ void __launch_bounds__(Shape<R1, R2>::threads) inv_y_kernel(
    PassGeo g, const float2* __restrict__ t2, float2* __restrict__ t1) {
  __shared__ float2 sy[Shape<R1, R2>::smem];
  __shared__ float2 tw[R1 * R2];
  fill_twiddles<R1 * R2>(tw);
  const int xb = blockIdx.x, i0 = blockIdx.y;
  const long long slot = blockIdx.z;
  const float2* src = t2 + (slot * g.n0 + i0) * g.g1 * (long long)g.g2;
  float2* dst = t1 + (slot * g.n0 + i0) * g.n1 * (long long)g.g2;
  auto ld = [&](int col, int n) -> float2 { return src[(long long)n * g.g2 + xb * kCols + col]; };
  auto st = [&](int col, int k, int, float2 v) {
    dst[(long long)img_of(k, g.n1, g.g1) * g.g2 + xb * kCols + col] = v;
  };
  fft16<R1, R2, true, false, false, true>(sy, tw, ld, st);
}

// I1: w[jj][i0][i1][i2] = C3^-1 sum_c conj(S_c) (inverse DFT_x of T1[slot][i0][i1][:])
// at the data positions, coils summed in order.  CTA: (block of 16 rows i1, i0, jj).
template <int R1, int R2>
__global__ void __launch_bounds__(Shape<R1, R2>::threads, 3) inv_x_kernel(
    PassGeo g, const float* __restrict__ dtab, const float2* __restrict__ smaps,
    const float2* __restrict__ t1, float2* __restrict__ w) {
  using S = Shape<R1, R2>;
  __shared__ float2 sy[S::smem];
  __shared__ float2 tw[R1 * R2];
  fill_twiddles<R1 * R2>(tw);
  const int rb = blockIdx.x, i0 = blockIdx.y, jj = blockIdx.z;
  const long long nvox = (long long)g.n0 * g.n1 * g.n2;
  // this thread's outputs: k = t + R1 k2 for the data k2 (step 2 threads t < R1)
  constexpr int NK = R2 / 2;
  float acc_r[NK], acc_i[NK];
#pragma unroll
  for (int q = 0; q < NK; ++q) acc_r[q] = acc_i[q] = 0.f;
  const int tid = threadIdx.x;
  const int mycol = tid / S::T, myt = tid % S::T;
  const int myi1 = rb * kCols + mycol;
  for (int c = 0; c < g.C; ++c) {
    const long long slot = (long long)jj * g.C + c;
    const float2* src = t1 + (slot * g.n0 + i0) * g.n1 * (long long)g.g2;
    auto ld = [&](int col, int n) -> float2 {
      const int i1 = rb * kCols + col;
      return i1 < g.n1 ? src[(long long)i1 * g.g2 + n] : make_float2(0.f, 0.f);
    };
    auto st = [&](int col, int k, int k2, float2 v) {
      const int i1 = rb * kCols + col;
      if (i1 >= g.n1) return;
      const int i2 = img_of(k, g.n2, g.g2);
      const float2 s = __ldg(smaps + c * nvox + ((long long)i0 * g.n1 + i1) * g.n2 + i2);
      const int q = k2 < R2 / 4 ? k2 : k2 - R2 / 2;  // index among the data k2
      acc_r[q] = fmaf(s.x, v.x, fmaf(s.y, v.y, acc_r[q]));
      acc_i[q] = fmaf(s.x, v.y, fmaf(-s.y, v.x, acc_i[q]));
    };
    fft16<R1, R2, true, true, false, true>(sy, tw, ld, st);
  }
  if (myt < R1 && myi1 < g.n1) {
    const float d01 = __ldg(dtab + i0) * __ldg(dtab + g.n0 + myi1);
#pragma unroll
    for (int q = 0; q < NK; ++q) {
      const int k2 = q < R2 / 4 ? q : q + R2 / 2;
      const int i2 = img_of(myt + R1 * k2, g.n2, g.g2);
      const float dep = d01 * __ldg(dtab + g.n0 + g.n1 + i2);
      w[jj * nvox + ((long long)i0 * g.n1 + myi1) * g.n2 + i2] =
          make_float2(acc_r[q] * dep, acc_i[q] * dep);
    }
  }
}

bool radix_of(int L, int* r1, int* r2) {
  switch (L) {
    case 32: *r1 = 8; *r2 = 4; return true;
    case 64: *r1 = 8; *r2 = 8; return true;
    case 128: *r1 = 16; *r2 = 8; return true;
    case 256: *r1 = 16; *r2 = 16; return true;
    default: return false;
  }
}

#define NRS_LAUNCH_L(KER, L, GRID, S, ...)                                          \
  do {                                                                             \
    switch (L) {                                                                   \
      case 32: KER<8, 4><<<GRID, Shape<8, 4>::threads, 0, S>>>(__VA_ARGS__); break;   \
      case 64: KER<8, 8><<<GRID, Shape<8, 8>::threads, 0, S>>>(__VA_ARGS__); break;   \
      case 128: KER<16, 8><<<GRID, Shape<16, 8>::threads, 0, S>>>(__VA_ARGS__); break; \
      default: KER<16, 16><<<GRID, Shape<16, 16>::threads, 0, S>>>(__VA_ARGS__); break; \
    }                                                                              \
  } while (0)

PassGeo pass_geo(const Geo& g, int C, int nph) {
  return PassGeo{g.n0, g.n1, g.n2, g.g0, g.g1, g.g2, C, nph};
}

}  // namespace

bool pruned_fft_supported(const Geo& g, int C, bool bf16) {
  if (bf16 || C < 1 || g.osf != 2) return false;
  int r1, r2;
  return radix_of(g.g0, &r1, &r2) && radix_of(g.g1, &r1, &r2) && radix_of(g.g2, &r1, &r2);
}

cudaError_t init_pruned_fft() {
  static cudaError_t done = [] {
    float2 w[16];
    for (int j = 0; j < 16; ++j)
      w[j] = make_float2(float(std::cos(2.0 * M_PI * j / 16.0)),
                         float(-std::sin(2.0 * M_PI * j / 16.0)));
    return cudaMemcpyToSymbol(c_w16, w, sizeof(w));
  }();
  return done;
}

int launch_pruned_forward(const Geo& g, int C, int nph, const float* deapod,
                          const nrsense_c64* smaps, const nrsense_c64* m, void* t1, void* t2,
                          void* grid, cudaStream_t s) {
  const PassGeo pg = pass_geo(g, C, nph);
  auto* T1 = static_cast<float2*>(t1);
  auto* T2 = static_cast<float2*>(t2);
  auto* Gd = static_cast<float2*>(grid);
  const unsigned slots = unsigned(C * nph);
  NRS_LAUNCH_L(fwd_x_kernel, g.g2, dim3((g.n1 + kCols - 1) / kCols, g.n0, nph), s, pg, deapod,
               reinterpret_cast<const float2*>(smaps), reinterpret_cast<const float2*>(m), T1);
  NRS_LAUNCH_L(fwd_y_kernel, g.g1, dim3(g.g2 / kCols, g.n0, slots), s, pg, T1, T2);
  NRS_LAUNCH_L(fwd_z_kernel, g.g0, dim3(g.g2 / kCols, g.g1, slots), s, pg, T2, Gd);
  return 3;
}

int launch_pruned_inverse(const Geo& g, int C, int nph, const float* deapod,
                          const nrsense_c64* smaps, const void* grid, void* t2, void* t1,
                          nrsense_c64* w, cudaStream_t s) {
  const PassGeo pg = pass_geo(g, C, nph);
  auto* T1 = static_cast<float2*>(t1);
  auto* T2 = static_cast<float2*>(t2);
  const auto* Gd = static_cast<const float2*>(grid);
  const unsigned slots = unsigned(C * nph);
  NRS_LAUNCH_L(inv_z_kernel, g.g0, dim3(g.g2 / kCols, g.g1, slots), s, pg, Gd, T2);
  NRS_LAUNCH_L(inv_y_kernel, g.g1, dim3(g.g2 / kCols, g.n0, slots), s, pg, T2, T1);
  NRS_LAUNCH_L(inv_x_kernel, g.g2, dim3((g.n1 + kCols - 1) / kCols, g.n0, nph), s, pg, deapod,
               reinterpret_cast<const float2*>(smaps), T1, reinterpret_cast<float2*>(w));
  return 3;
}

}  // namespace nrs
