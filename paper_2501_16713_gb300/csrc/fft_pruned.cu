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
#include <type_traits>

#include "plan_internal.h"

namespace nrs {

namespace {

constexpr int kCols = 16;  // transforms per CTA

// cos and sin of 2 pi j / 16 for j < 8: W_16^j = exp(-2 pi i j / 16) = c16(j) - i s16(j)
__host__ __device__ constexpr float c16(int j) {
  return j == 0 ? 1.0f
       : j == 1 ? 0.923879532511286756f
       : j == 2 ? 0.707106781186547524f
       : j == 3 ? 0.382683432365089772f
       : j == 4 ? 0.0f
       : j == 5 ? -0.382683432365089772f
       : j == 6 ? -0.707106781186547524f
                : -0.923879532511286756f;
}
__host__ __device__ constexpr float s16(int j) {  // sin(2 pi j / 16) = cos(2 pi |4 - j| / 16)
  return c16(j < 4 ? 4 - j : j - 4);
}

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

// Compile-time loop: f(std::integral_constant<int, I>) for I = B .. E-1, so
// every register-array index below is a constant (no local-memory arrays).
template <int B, int E, class F>
__device__ __forceinline__ void static_for(F&& f) {
  if constexpr (B < E) {
    f(std::integral_constant<int, B>{});
    static_for<B + 1, E>(f);
  }
}

// a * W_16^J (forward) or a * conj(W_16^J) (inverse), J < 8: the factors 1
// and -+i are a move and a swap, not multiplies.
template <bool INV, int J>
__device__ __forceinline__ float2 twiddle16(float2 a) {
  if constexpr (J == 0) {
    return a;
  } else if constexpr (J == 4) {
    return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
  } else {
    constexpr float c = c16(J), sn = INV ? s16(J) : -s16(J);
    return make_float2(a.x * c - a.y * sn, a.x * sn + a.y * c);
  }
}

// In-register radix-2 DFT of length R (R <= 16): a[k] = sum_n a[n] W_R^(+-nk)
// (bit-reversed input order, then log2 R butterfly stages).  ZMID: the inputs
// n in [R/4, 3R/4) are zero, so the first stage, which pairs n and n + R/2,
// is a copy (u, u) or a copy and a negation (v, -v).
template <int R, bool INV, bool ZMID = false>
__device__ __forceinline__ void dft(float2 (&a)[R]) {
  static_for<0, R>([&](auto ic) {
    constexpr int i = decltype(ic)::value, j = bitrev(i, R);
    if constexpr (j > i) {
      const float2 t = a[i];
      a[i] = a[j];
      a[j] = t;
    }
  });
  static_for<1, 5>([&](auto sc) {
    constexpr int len = 1 << decltype(sc)::value, half = len >> 1;
    if constexpr (len <= R) {
      static_for<0, R / len>([&](auto gc) {
        constexpr int i = decltype(gc)::value * len;
        static_for<0, half>([&](auto kc) {
          constexpr int k = decltype(kc)::value;
          if constexpr (ZMID && len == 2) {
            // original indices bitrev(i) < R/2 and bitrev(i) + R/2
            constexpr int n = bitrev(i, R);
            if constexpr (n < R / 4) {
              a[i + 1] = a[i];
            } else {
              a[i] = a[i + 1];
              a[i + 1] = make_float2(-a[i].x, -a[i].y);
            }
          } else {
            const float2 u = a[i + k];
            const float2 v = twiddle16<INV, (16 / len) * k>(a[i + k + half]);
            a[i + k] = make_float2(u.x + v.x, u.y + v.y);
            a[i + k + half] = make_float2(u.x - v.x, u.y - v.y);
          }
        });
      });
    }
  });
}

// Image index of data grid position n = R2 n1 + t of a length-L axis
// (centred placement, G = L = 2N: data at [0, L/4) and [3L/4, L)); the half
// is decided by n1 alone, known after unrolling.
template <int R1, int R2>
__device__ __forceinline__ int img_in(int n1, int t) {
  constexpr int L = R1 * R2;
  return n1 < R1 / 4 ? R2 * n1 + t + L / 4 : R2 * n1 + t - 3 * L / 4;
}
// Image index of data output position k = k1 + R1 k2 (decided by k2).
template <int R1, int R2>
__device__ __forceinline__ int img_out(int k1, int k2) {
  constexpr int L = R1 * R2;
  return k2 < R2 / 4 ? k1 + R1 * k2 + L / 4 : k1 + R1 * k2 - 3 * L / 4;
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
// data half of the output.  ld(col, n1, n2) -> float2 for n = R2 n1 + n2,
// st(col, k1, k2, value) for k = k1 + R1 k2 (n1 and k2 known after unrolling).
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
    static_for<0, R1>([&](auto nc) {
      constexpr int n1 = decltype(nc)::value;
      if constexpr (!PIN || n1 < R1 / 4 || n1 >= 3 * R1 / 4)
        a[n1] = ld(col, n1, t);
      else
        a[n1] = make_float2(0.f, 0.f);
    });
    dft<R1, INV, PIN>(a);
    static_for<0, R1>([&](auto kc) {
      constexpr int k1 = decltype(kc)::value;
      float2 v = a[k1];
      if constexpr (k1 > 0) {
        float2 w = tw[(t * k1) % S::L];
        if (INV) w.y = -w.y;
        v = cmul(v, w);
      }
      sy[yidx<R1, R2, ROWS>(col, k1, t)] = v;
    });
  }
  __syncthreads();
  if (t < R1) {
    float2 b[R2];
    static_for<0, R2>([&](auto nc) {
      constexpr int n2 = decltype(nc)::value;
      b[n2] = sy[yidx<R1, R2, ROWS>(col, t, n2)];
    });
    dft<R2, INV>(b);
    static_for<0, R2>([&](auto kc) {
      constexpr int k2 = decltype(kc)::value;
      if constexpr (!POUT || k2 < R2 / 4 || k2 >= 3 * R2 / 4) st(col, t, kc, b[k2]);
    });
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
#pragma unroll 1
  for (int c = 0; c < g.C; ++c) {
    const long long slot = (long long)jj * g.C + c;
    auto ld = [&](int col, int n1, int t) -> float2 {
      const int i1 = rb * kCols + col;
      if (i1 >= g.n1) return make_float2(0.f, 0.f);
      const int i2 = img_in<R1, R2>(n1, t);
      const long long v = ((long long)i0 * g.n1 + i1) * g.n2 + i2;
      const float2 mv = __ldg(m + jj * nvox + v);
      const float2 sv = __ldg(smaps + c * nvox + v);
      const float w = d0 * __ldg(dtab + g.n0 + i1) * __ldg(dtab + g.n0 + g.n1 + i2);
      return make_float2((sv.x * mv.x - sv.y * mv.y) * w, (sv.x * mv.y + sv.y * mv.x) * w);
    };
    auto st = [&](int col, int k1, auto k2c, float2 v) {
      constexpr int k2 = decltype(k2c)::value;
      const int i1 = rb * kCols + col;
      if (i1 < g.n1) t1[((slot * g.n0 + i0) * g.n1 + i1) * g.g2 + k1 + R1 * k2] = v;
    };
    fft16<R1, R2, false, true, true, false>(sy, tw, ld, st);
  }
}

// F2: T2[slot][i0][:][x] = DFT_y of T1[slot][i0][data rows][x] (exponent sign
// + for INV).
// CTA: (block of 16 x, i0, slot).
template <int R1, int R2, bool INV>
__global__ void __launch_bounds__(Shape<R1, R2>::threads, 5) fwd_y_kernel(
    PassGeo g, const float2* __restrict__ t1, float2* __restrict__ t2) {
  __shared__ float2 sy[Shape<R1, R2>::smem];
  __shared__ float2 tw[R1 * R2];
  fill_twiddles<R1 * R2>(tw);
  const int xb = blockIdx.x, i0 = blockIdx.y;
  const long long slot = blockIdx.z;
  const float2* src = t1 + (slot * g.n0 + i0) * g.n1 * (long long)g.g2;
  float2* dst = t2 + (slot * g.n0 + i0) * g.g1 * (long long)g.g2;
  auto ld = [&](int col, int n1, int t) -> float2 {
    return src[img_in<R1, R2>(n1, t) * g.g2 + xb * kCols + col];
  };
  auto st = [&](int col, int k1, auto k2c, float2 v) {
    constexpr int k2 = decltype(k2c)::value;
    dst[(k1 + R1 * k2) * g.g2 + xb * kCols + col] = v;
  };
  fft16<R1, R2, INV, false, true, false>(sy, tw, ld, st);
}

// F3: grid[slot][:][y][x] = DFT_z of T2[slot][data planes][y][x] (sign + for INV).
// CTA: (block of 16 x, y, slot).  colmask (or null): per (y, x) 8^3-tile
// column a bit per z tile that is ever read; other tiles are not stored, and
// a CTA whose two tile columns have none returns at once.
template <int R1, int R2, bool INV>
__global__ void __launch_bounds__(Shape<R1, R2>::threads, 5) fwd_z_kernel(
    PassGeo g, const uint32_t* __restrict__ colmask, const float2* __restrict__ t2,
    float2* __restrict__ grid) {
  __shared__ float2 sy[Shape<R1, R2>::smem];
  __shared__ float2 tw[R1 * R2];
  const int xb = blockIdx.x, y = blockIdx.y;
  uint32_t m0 = ~0u, m1 = ~0u;  // tile columns of x in [16 xb, 16 xb + 8) and [.. + 8, .. + 16)
  if (colmask != nullptr) {
    const uint32_t* cm = colmask + (y >> 3) * (g.g2 >> 3) + 2 * xb;
    m0 = __ldg(cm);
    m1 = __ldg(cm + 1);
    if ((m0 | m1) == 0u) return;  // CTA-uniform
  }
  fill_twiddles<R1 * R2>(tw);
  const long long slot = blockIdx.z;
  const long long plane = (long long)g.g1 * g.g2;
  const float2* src = t2 + slot * g.n0 * plane + (long long)y * g.g2 + xb * kCols;
  float2* dst = grid + slot * g.g0 * plane + (long long)y * g.g2 + xb * kCols;
  auto ld = [&](int col, int n1, int t) -> float2 {
    return src[img_in<R1, R2>(n1, t) * plane + col];
  };
  auto st = [&](int col, int k1, auto k2c, float2 v) {
    constexpr int k2 = decltype(k2c)::value;
    const int z = k1 + R1 * k2;
    if (((col < 8 ? m0 : m1) >> (z >> 3)) & 1u) dst[z * plane + col] = v;
  };
  fft16<R1, R2, INV, false, true, false>(sy, tw, ld, st);
}

// I3: T2[slot][i0][y][x] = (DFT_z of grid[slot][:][y][x], sign + for INV) at the
// data planes.
// colmask (or null): z tiles outside it are zero in the grid and not loaded.
template <int R1, int R2, bool INV>
__global__ void __launch_bounds__(Shape<R1, R2>::threads, 5) inv_z_kernel(
    PassGeo g, const uint32_t* __restrict__ colmask, const float2* __restrict__ grid,
    float2* __restrict__ t2) {
  __shared__ float2 sy[Shape<R1, R2>::smem];
  __shared__ float2 tw[R1 * R2];
  fill_twiddles<R1 * R2>(tw);
  const int xb = blockIdx.x, y = blockIdx.y;
  uint32_t m0 = ~0u, m1 = ~0u;
  if (colmask != nullptr) {
    const uint32_t* cm = colmask + (y >> 3) * (g.g2 >> 3) + 2 * xb;
    m0 = __ldg(cm);
    m1 = __ldg(cm + 1);
  }
  const long long slot = blockIdx.z;
  const long long plane = (long long)g.g1 * g.g2;
  const float2* src = grid + slot * g.g0 * plane + (long long)y * g.g2 + xb * kCols;
  float2* dst = t2 + slot * g.n0 * plane + (long long)y * g.g2 + xb * kCols;
  auto ld = [&](int col, int n1, int t) -> float2 {
    const int z = R2 * n1 + t;
    return (((col < 8 ? m0 : m1) >> (z >> 3)) & 1u) ? src[z * plane + col]
                                                    : make_float2(0.f, 0.f);
  };
  auto st = [&](int col, int k1, auto k2c, float2 v) {
    constexpr int k2 = decltype(k2c)::value;
    dst[img_out<R1, R2>(k1, k2) * plane + col] = v;
  };
  fft16<R1, R2, INV, false, false, true>(sy, tw, ld, st);
}

// I2: T1[slot][i0][i1][x] = (DFT_y of T2[slot][i0][:][x], sign + for INV) at the
// data rows.
template <int R1, int R2, bool INV>
__global__ void __launch_bounds__(Shape<R1, R2>::threads, 5) inv_y_kernel(
    PassGeo g, const float2* __restrict__ t2, float2* __restrict__ t1) {
  __shared__ float2 sy[Shape<R1, R2>::smem];
  __shared__ float2 tw[R1 * R2];
  fill_twiddles<R1 * R2>(tw);
  const int xb = blockIdx.x, i0 = blockIdx.y;
  const long long slot = blockIdx.z;
  const float2* src = t2 + (slot * g.n0 + i0) * g.g1 * (long long)g.g2;
  float2* dst = t1 + (slot * g.n0 + i0) * g.n1 * (long long)g.g2;
  auto ld = [&](int col, int n1, int t) -> float2 {
    return src[(R2 * n1 + t) * g.g2 + xb * kCols + col];
  };
  auto st = [&](int col, int k1, auto k2c, float2 v) {
    constexpr int k2 = decltype(k2c)::value;
    dst[img_out<R1, R2>(k1, k2) * g.g2 + xb * kCols + col] = v;
  };
  fft16<R1, R2, INV, false, false, true>(sy, tw, ld, st);
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
  static_for<0, NK>([&](auto qc) { acc_r[decltype(qc)::value] = acc_i[decltype(qc)::value] = 0.f; });
  const int tid = threadIdx.x;
  const int mycol = tid / S::T, myt = tid % S::T;
  const int myi1 = rb * kCols + mycol;
#pragma unroll 1
  for (int c = 0; c < g.C; ++c) {
    const long long slot = (long long)jj * g.C + c;
    const float2* src = t1 + (slot * g.n0 + i0) * g.n1 * (long long)g.g2;
    auto ld = [&](int col, int n1, int t) -> float2 {
      const int i1 = rb * kCols + col;
      return i1 < g.n1 ? src[(long long)i1 * g.g2 + R2 * n1 + t] : make_float2(0.f, 0.f);
    };
    auto st = [&](int col, int k1, auto k2c, float2 v) {
      constexpr int k2 = decltype(k2c)::value;
      const int i1 = rb * kCols + col;
      if (i1 >= g.n1) return;
      const int i2 = img_out<R1, R2>(k1, k2);
      const float2 s = __ldg(smaps + c * nvox + ((long long)i0 * g.n1 + i1) * g.n2 + i2);
      constexpr int q = k2 < R2 / 4 ? k2 : k2 - R2 / 2;  // index among the data k2
      acc_r[q] = fmaf(s.x, v.x, fmaf(s.y, v.y, acc_r[q]));
      acc_i[q] = fmaf(s.x, v.y, fmaf(-s.y, v.x, acc_i[q]));
    };
    fft16<R1, R2, true, true, false, true>(sy, tw, ld, st);
  }
  if (myt < R1 && myi1 < g.n1) {
    const float d01 = __ldg(dtab + i0) * __ldg(dtab + g.n0 + myi1);
    static_for<0, NK>([&](auto qc) {
      constexpr int q = decltype(qc)::value;
      constexpr int k2 = q < R2 / 4 ? q : q + R2 / 2;
      const int i2 = img_out<R1, R2>(myt, k2);
      const float dep = d01 * __ldg(dtab + g.n0 + g.n1 + i2);
      w[jj * nvox + ((long long)i0 * g.n1 + myi1) * g.n2 + i2] =
          make_float2(acc_r[q] * dep, acc_i[q] * dep);
    });
  }
}

// The image-space transforms of T_j (forward diagram F -> 1/C* -> Z -> F^H)
// and T_j^H (F -> Z^H -> 1/C -> F^H) over the one G^3 grid.  Frequency k of
// an axis sits at grid position k mod G: with the centred index i = k + N/2
// that is the same placement as the coil images' (data at [0, G/4) and
// [3G/4, G)), so the y and z passes above serve unchanged; only the x passes
// differ: they read (write) the N^3 spectrum in FFT order, index
// f = (i + N/2) mod N, and apply 1/(N^3 C3(k/G)) on the way.

__device__ __forceinline__ int fft_index(int i, int n) { return i < (n >> 1) ? i + (n >> 1) : i - (n >> 1); }

// T forward, x pass: T1[i0][i1][:] = inverse DFT_x of U on the data row
// (i0, i1), U[k] = Xhat[k] / (N^3 C3(k/G)) (steps 1/C* and Z fused into the
// loads).  CTA: (block of 16 rows i1, i0).
template <int R1, int R2>
__global__ void __launch_bounds__(Shape<R1, R2>::threads, 4) timg_fwd_x_kernel(
    PassGeo g, const float* __restrict__ dtab, float scale, const float2* __restrict__ xhat,
    float2* __restrict__ t1) {
  __shared__ float2 sy[Shape<R1, R2>::smem];
  __shared__ float2 tw[R1 * R2];
  fill_twiddles<R1 * R2>(tw);
  const int rb = blockIdx.x, i0 = blockIdx.y;
  const int f0 = fft_index(i0, g.n0);
  const float d0 = __ldg(dtab + i0);
  auto ld = [&](int col, int n1, int t) -> float2 {
    const int i1 = rb * kCols + col;
    if (i1 >= g.n1) return make_float2(0.f, 0.f);
    const int i2 = img_in<R1, R2>(n1, t);
    const float2 v = __ldg(xhat + ((long long)f0 * g.n1 + fft_index(i1, g.n1)) * g.n2 +
                           fft_index(i2, g.n2));
    const float w = d0 * __ldg(dtab + g.n0 + i1) * __ldg(dtab + g.n0 + g.n1 + i2) * scale;
    return make_float2(v.x * w, v.y * w);
  };
  auto st = [&](int col, int k1, auto k2c, float2 v) {
    constexpr int k2 = decltype(k2c)::value;
    const int i1 = rb * kCols + col;
    if (i1 < g.n1) t1[((long long)i0 * g.n1 + i1) * g.g2 + k1 + R1 * k2] = v;
  };
  fft16<R1, R2, true, true, true, false>(sy, tw, ld, st);
}

// T adjoint, x pass: Xhat[k] = (DFT_x of T1[i0][i1][:]) at the data
// positions / (N^3 C3(k/G)) (steps Z^H and 1/C fused into the stores).
template <int R1, int R2>
__global__ void __launch_bounds__(Shape<R1, R2>::threads, 4) timg_inv_x_kernel(
    PassGeo g, const float* __restrict__ dtab, float scale, const float2* __restrict__ t1,
    float2* __restrict__ xhat) {
  __shared__ float2 sy[Shape<R1, R2>::smem];
  __shared__ float2 tw[R1 * R2];
  fill_twiddles<R1 * R2>(tw);
  const int rb = blockIdx.x, i0 = blockIdx.y;
  const int f0 = fft_index(i0, g.n0);
  const float d0 = __ldg(dtab + i0);
  const float2* src = t1 + (long long)i0 * g.n1 * g.g2;
  auto ld = [&](int col, int n1, int t) -> float2 {
    const int i1 = rb * kCols + col;
    return i1 < g.n1 ? src[(long long)i1 * g.g2 + R2 * n1 + t] : make_float2(0.f, 0.f);
  };
  auto st = [&](int col, int k1, auto k2c, float2 v) {
    constexpr int k2 = decltype(k2c)::value;
    const int i1 = rb * kCols + col;
    if (i1 >= g.n1) return;
    const int i2 = img_out<R1, R2>(k1, k2);
    const float w = d0 * __ldg(dtab + g.n0 + i1) * __ldg(dtab + g.n0 + g.n1 + i2) * scale;
    xhat[((long long)f0 * g.n1 + fft_index(i1, g.n1)) * g.n2 + fft_index(i2, g.n2)] =
        make_float2(v.x * w, v.y * w);
  };
  fft16<R1, R2, false, true, false, true>(sy, tw, ld, st);
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

#define NRS_LAUNCH_LS(KER, INV, L, GRID, S, ...)                                               \
  do {                                                                                          \
    switch (L) {                                                                                \
      case 32: KER<8, 4, INV><<<GRID, Shape<8, 4>::threads, 0, S>>>(__VA_ARGS__); break;         \
      case 64: KER<8, 8, INV><<<GRID, Shape<8, 8>::threads, 0, S>>>(__VA_ARGS__); break;         \
      case 128: KER<16, 8, INV><<<GRID, Shape<16, 8>::threads, 0, S>>>(__VA_ARGS__); break;      \
      default: KER<16, 16, INV><<<GRID, Shape<16, 16>::threads, 0, S>>>(__VA_ARGS__); break;     \
    }                                                                                           \
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

bool pruned_image_fft_supported(const Geo& g) {
  int r1, r2;
  return g.osf == 2 && radix_of(g.g0, &r1, &r2) && radix_of(g.g1, &r1, &r2) &&
         radix_of(g.g2, &r1, &r2);
}

cudaError_t init_pruned_fft() { return cudaSuccess; }  // no tables to upload

int launch_pruned_forward(const Geo& g, int C, int nph, const uint32_t* colmask,
                          const float* deapod,
                          const nrsense_c64* smaps, const nrsense_c64* m, void* t1, void* t2,
                          void* grid, cudaStream_t s) {
  const PassGeo pg = pass_geo(g, C, nph);
  auto* T1 = static_cast<float2*>(t1);
  auto* T2 = static_cast<float2*>(t2);
  auto* Gd = static_cast<float2*>(grid);
  const unsigned slots = unsigned(C * nph);
  NRS_LAUNCH_L(fwd_x_kernel, g.g2, dim3((g.n1 + kCols - 1) / kCols, g.n0, nph), s, pg, deapod,
               reinterpret_cast<const float2*>(smaps), reinterpret_cast<const float2*>(m), T1);
  NRS_LAUNCH_LS(fwd_y_kernel, false, g.g1, dim3(g.g2 / kCols, g.n0, slots), s, pg, T1, T2);
  NRS_LAUNCH_LS(fwd_z_kernel, false, g.g0, dim3(g.g2 / kCols, g.g1, slots), s, pg, colmask, T2,
                Gd);
  return 3;
}

int launch_pruned_inverse(const Geo& g, int C, int nph, const uint32_t* colmask,
                          const float* deapod,
                          const nrsense_c64* smaps, const void* grid, void* t2, void* t1,
                          nrsense_c64* w, cudaStream_t s) {
  const PassGeo pg = pass_geo(g, C, nph);
  auto* T1 = static_cast<float2*>(t1);
  auto* T2 = static_cast<float2*>(t2);
  const auto* Gd = static_cast<const float2*>(grid);
  const unsigned slots = unsigned(C * nph);
  NRS_LAUNCH_LS(inv_z_kernel, true, g.g0, dim3(g.g2 / kCols, g.g1, slots), s, pg, colmask, Gd,
                T2);
  NRS_LAUNCH_LS(inv_y_kernel, true, g.g1, dim3(g.g2 / kCols, g.n0, slots), s, pg, T2, T1);
  NRS_LAUNCH_L(inv_x_kernel, g.g2, dim3((g.n1 + kCols - 1) / kCols, g.n0, nph), s, pg, deapod,
               reinterpret_cast<const float2*>(smaps), T1, reinterpret_cast<float2*>(w));
  return 3;
}

// u = F_G^-1 of the deapodized, zero-padded spectrum of xhat (scratch: T1,
// N0 N1 G2 values; T2, N0 G1 G2 values)
int launch_pruned_image_forward(const Geo& g, const float* deapod, const nrsense_c64* xhat,
                                void* t1, void* t2, nrsense_c64* ugrid, cudaStream_t s) {
  const PassGeo pg = pass_geo(g, 1, 1);
  auto* T1 = static_cast<float2*>(t1);
  auto* T2 = static_cast<float2*>(t2);
  const float scale = float(1.0 / double(g.nvox));
  NRS_LAUNCH_L(timg_fwd_x_kernel, g.g2, dim3((g.n1 + kCols - 1) / kCols, g.n0, 1), s, pg, deapod,
               scale, reinterpret_cast<const float2*>(xhat), T1);
  NRS_LAUNCH_LS(fwd_y_kernel, true, g.g1, dim3(g.g2 / kCols, g.n0, 1), s, pg, T1, T2);
  NRS_LAUNCH_LS(fwd_z_kernel, true, g.g0, dim3(g.g2 / kCols, g.g1, 1), s, pg, nullptr, T2,
                reinterpret_cast<float2*>(ugrid));
  return 3;
}

// xhat = deapodized crop of F_G of the spread grid u
int launch_pruned_image_adjoint(const Geo& g, const float* deapod, const nrsense_c64* ugrid,
                                void* t2, void* t1, nrsense_c64* xhat, cudaStream_t s) {
  const PassGeo pg = pass_geo(g, 1, 1);
  auto* T1 = static_cast<float2*>(t1);
  auto* T2 = static_cast<float2*>(t2);
  const float scale = float(1.0 / double(g.nvox));
  NRS_LAUNCH_LS(inv_z_kernel, false, g.g0, dim3(g.g2 / kCols, g.g1, 1), s, pg, nullptr,
                reinterpret_cast<const float2*>(ugrid), T2);
  NRS_LAUNCH_LS(inv_y_kernel, false, g.g1, dim3(g.g2 / kCols, g.n0, 1), s, pg, T2, T1);
  NRS_LAUNCH_L(timg_inv_x_kernel, g.g2, dim3((g.n1 + kCols - 1) / kCols, g.n0, 1), s, pg, deapod,
               scale, T1, reinterpret_cast<float2*>(xhat));
  return 3;
}

}  // namespace nrs
