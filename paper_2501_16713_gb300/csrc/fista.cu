// Wavelet-FISTA for the L1-regularised reconstruction problem.
//
// The reconstruction problem (reconstruction optimisation equation) is
//   minimise ||y - A x||^2 + lambda ||W x||_1,   A = [A_0; ...; A_{P-1}],
// solved in the paper by wavelet-FISTA (Beck and Teboulle), also for the
// warp-only inversion of Appendix 1 (400 iterations, lambda = 1e-6).  W is
// read as the orthonormal separable 3D Haar transform with J <= 4 levels and
// ||.||_1 as the sum of complex moduli over every coefficient, so that
//   x_k     = W^H soft(W v_k, lambda / L),  v_k = z_k - (2 / L)(E0 z_k - b),
//   z_{k+1} = x_k + mu_k (x_k - x_{k-1}),   mu_k = (t_k - 1) / t_{k+1},
// with E0 = sum_j A_j^H A_j, b = sum_j A_j^H y_j and L >= 2 lambda_max(E0).
//
// GPU design.  Haar filters have disjoint two-point supports, so a J-level
// 3D Haar pyramid acts on each aligned 2^J cube independently and the
// proximal step needs no global transform.  One CTA takes a box of whole
// cubes (8 x 8 x 32 voxels for J <= 3, 16 x 16 x 16 for J = 4) and each
// thread one 2 x 2 x 2 voxel group of it, read and written as four 16-byte
// row pairs.  Level 1 of the pyramid acts inside a group, so it runs in
// registers, and its seven detail coefficients are thresholded there; only
// the group's approximation goes to shared memory, where levels 2..J run as
// in-place lifting passes over the (1/8-size) array of approximations: level
// l combines the entries i and i + 2^(l-2) (i a multiple of 2^(l-1)) into the
// low-pass value at i and the high-pass value at i + 2^(l-2), one axis after
// the other, so every pass updates disjoint pairs.  The threshold touches
// each coefficient exactly once whatever the layout, so the proximal map is
// that of the Mallat layout; the stand-alone transform entry points scatter
// to (gather from) the Mallat layout.  The gradient step, the threshold, the
// inverse and the momentum update are one kernel: it reads z, E0 z, b and
// x_{k-1} and writes x_k and z_{k+1} (48 bytes per voxel); every load of a
// thread is issued before the transform (x_{k-1} as cp.async copies into
// shared memory, which hold no registers) so that they overlap it.  The
// momentum sequence depends only on k, so it is a device table indexed by a
// device iteration counter and the iteration has no host round trip: 32
// iterations (normal operator, step kernel, a one-block finish kernel) are
// captured once as a CUDA graph and replayed.  ||x_k - x_{k-1}|| / ||x_k|| is
// reduced with a fixed summation order (FP32 over a thread's eight voxels,
// FP64 above) and kept per iteration.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "plan_internal.h"

using namespace nrs;

namespace {

constexpr int kMaxLevels = 4;
constexpr int kThreads = 256;     // reduction kernels
constexpr int kRedBlocks = 1184;  // power iteration reductions: fixed grid, fixed order
constexpr int kChunk = 32;        // FISTA iterations per captured graph
constexpr float kSqrtHalf = 0.70710678118654752440f;

// Box of whole 2^J cubes staged by one CTA; one thread per 2 x 2 x 2 group.
template <int J>
struct Box {
  static constexpr int b0 = J == 4 ? 16 : 8;
  static constexpr int b1 = b0;
  static constexpr int b2 = J == 4 ? 16 : 32;
  static constexpr int g0 = b0 / 2, g1 = b1 / 2, g2 = b2 / 2;  // groups per axis
  static constexpr int nt = g0 * g1 * g2;                     // threads: 256 or 512
};

void box_dims(int J, int* b0, int* b1, int* b2) {
  *b0 = *b1 = J == 4 ? 16 : 8;
  *b2 = J == 4 ? 16 : 32;
}

struct Vol {
  int n0, n1, n2;
  int nb1, nb2;  // boxes along axes 1 and 2
  int vec;       // 16-byte row-pair accesses allowed (n2 even, pointers aligned)
};

// The thread's group: global coordinates of its first voxel, whether any or
// all of its eight voxels lie inside the volume.
struct Group {
  int x0, x1, x2;
  bool any, full;
};

template <int J>
__device__ __forceinline__ Group group_of(const Vol& g) {
  using D = Box<J>;
  const int t = threadIdx.x;
  const int q2 = t % D::g2, q1 = (t / D::g2) % D::g1, q0 = t / (D::g2 * D::g1);
  const long long box = blockIdx.x;
  const long long bz = box / ((long long)g.nb1 * g.nb2);
  const int rem = int(box - bz * (long long)g.nb1 * g.nb2);
  Group r;
  r.x0 = int(bz) * D::b0 + 2 * q0;
  r.x1 = (rem / g.nb2) * D::b1 + 2 * q1;
  r.x2 = (rem % g.nb2) * D::b2 + 2 * q2;
  r.any = r.x0 < g.n0 && r.x1 < g.n1 && r.x2 < g.n2;
  r.full = r.x0 + 1 < g.n0 && r.x1 + 1 < g.n1 && r.x2 + 1 < g.n2;
  return r;
}

__device__ __forceinline__ long long lin(const Vol& g, int x0, int x1, int x2) {
  return ((long long)x0 * g.n1 + x1) * g.n2 + x2;
}

// v[4 d0 + 2 d1 + d2] = p[x + d] (zero outside the volume).
__device__ __forceinline__ void load8(const float2* __restrict__ p, const Vol& g, const Group& gr,
                                      float2 v[8]) {
  if (g.vec && gr.full) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const float4 f =
          *reinterpret_cast<const float4*>(p + lin(g, gr.x0 + (r >> 1), gr.x1 + (r & 1), gr.x2));
      v[2 * r] = make_float2(f.x, f.y);
      v[2 * r + 1] = make_float2(f.z, f.w);
    }
  } else {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int x0 = gr.x0 + (k >> 2), x1 = gr.x1 + ((k >> 1) & 1), x2 = gr.x2 + (k & 1);
      v[k] = (x0 < g.n0 && x1 < g.n1 && x2 < g.n2) ? p[lin(g, x0, x1, x2)]
                                                   : make_float2(0.0f, 0.0f);
    }
  }
}

__device__ __forceinline__ void store8(float2* __restrict__ p, const Vol& g, const Group& gr,
                                       const float2 v[8]) {
  if (g.vec && gr.full) {
#pragma unroll
    for (int r = 0; r < 4; ++r)
      *reinterpret_cast<float4*>(p + lin(g, gr.x0 + (r >> 1), gr.x1 + (r & 1), gr.x2)) =
          make_float4(v[2 * r].x, v[2 * r].y, v[2 * r + 1].x, v[2 * r + 1].y);
  } else {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int x0 = gr.x0 + (k >> 2), x1 = gr.x1 + ((k >> 1) & 1), x2 = gr.x2 + (k & 1);
      if (x0 < g.n0 && x1 < g.n1 && x2 < g.n2) p[lin(g, x0, x1, x2)] = v[k];
    }
  }
}

// Prefetch the group's eight values of p into shared memory without staging
// them in registers: sx[r * nt + t] holds row pair r (v[2r], v[2r+1]) of
// thread t.  16-byte cp.async copies (cache-global) for whole aligned groups,
// plain loads otherwise; the caller waits with cp_async_wait_all.
template <int NT>
__device__ __forceinline__ void prefetch8(const float2* __restrict__ p, const Vol& g,
                                          const Group& gr, float4* sx) {
  const int t = threadIdx.x;
  if (g.vec && gr.full) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const uint32_t sa = static_cast<uint32_t>(__cvta_generic_to_shared(sx + r * NT + t));
      const float2* ga = p + lin(g, gr.x0 + (r >> 1), gr.x1 + (r & 1), gr.x2);
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(ga) : "memory");
    }
  } else {
    float2 v[8];
    load8(p, g, gr, v);
#pragma unroll
    for (int r = 0; r < 4; ++r)
      sx[r * NT + t] = make_float4(v[2 * r].x, v[2 * r].y, v[2 * r + 1].x, v[2 * r + 1].y);
  }
}

__device__ __forceinline__ void haar2(float2& a, float2& c) {
  const float2 s = make_float2((a.x + c.x) * kSqrtHalf, (a.y + c.y) * kSqrtHalf);
  c = make_float2((a.x - c.x) * kSqrtHalf, (a.y - c.y) * kSqrtHalf);
  a = s;
}

// Level 1 inside a group: (a, c) -> ((a + c) / sqrt2, (a - c) / sqrt2) along
// axes 0, 1, 2; afterwards v[4 s0 + 2 s1 + s2] holds sub-band (s0, s1, s2).
// The 2 x 2 map is its own inverse, so the inverse runs the axes in reverse.
__device__ __forceinline__ void haar8_forward(float2 v[8]) {
#pragma unroll
  for (int k = 0; k < 4; ++k) haar2(v[k], v[k + 4]);
#pragma unroll
  for (int k = 0; k < 8; k += 4) {
    haar2(v[k], v[k + 2]);
    haar2(v[k + 1], v[k + 3]);
  }
#pragma unroll
  for (int k = 0; k < 8; k += 2) haar2(v[k], v[k + 1]);
}

__device__ __forceinline__ void haar8_inverse(float2 v[8]) {
#pragma unroll
  for (int k = 0; k < 8; k += 2) haar2(v[k], v[k + 1]);
#pragma unroll
  for (int k = 0; k < 8; k += 4) {
    haar2(v[k], v[k + 2]);
    haar2(v[k + 1], v[k + 3]);
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) haar2(v[k], v[k + 4]);
}

// Complex soft threshold: c max(0, 1 - tau / |c|), the modulus through the
// reciprocal square root of |c|^2 (rsqrtf, within 2 ulp).  |c|^2 <= tau^2
// (c = 0 included) gives 0; tau = 0 gives c.
__device__ __forceinline__ float2 soft(float2 c, float tau) {
  const float r2 = c.x * c.x + c.y * c.y;
  const float k = r2 > tau * tau ? 1.0f - tau * rsqrtf(r2) : 0.0f;
  return make_float2(c.x * k, c.y * k);
}

// One lifting pass over the shared array of level-1 approximations (dims
// g0 x g1 x g2): pairs at distance ST along AXIS.
template <int J, int ST, int AXIS>
__device__ __forceinline__ void haar_pass(float2* s) {
  using D = Box<J>;
  constexpr int d0 = AXIS == 0 ? D::g0 / (2 * ST) : D::g0 / ST;
  constexpr int d1 = AXIS == 1 ? D::g1 / (2 * ST) : D::g1 / ST;
  constexpr int d2 = AXIS == 2 ? D::g2 / (2 * ST) : D::g2 / ST;
  constexpr int s0 = AXIS == 0 ? 2 * ST : ST;
  constexpr int s1 = AXIS == 1 ? 2 * ST : ST;
  constexpr int s2 = AXIS == 2 ? 2 * ST : ST;
  constexpr int off = AXIS == 0 ? ST * D::g1 * D::g2 : AXIS == 1 ? ST * D::g2 : ST;
  constexpr int npairs = d0 * d1 * d2;
  for (int q = threadIdx.x; q < npairs; q += D::nt) {
    const int j2 = q % d2;
    const int r = q / d2;
    const int j1 = r % d1;
    const int j0 = r / d1;
    const int ia = ((j0 * s0) * D::g1 + j1 * s1) * D::g2 + j2 * s2;
    haar2(s[ia], s[ia + off]);
  }
  __syncthreads();
}

template <int J, int L>
__device__ __forceinline__ void haar_level(float2* s, bool inverse) {
  constexpr int st = 1 << (L - 2);  // level L >= 2 on the level-1 approximations
  if (!inverse) {
    haar_pass<J, st, 0>(s);
    haar_pass<J, st, 1>(s);
    haar_pass<J, st, 2>(s);
  } else {
    haar_pass<J, st, 2>(s);
    haar_pass<J, st, 1>(s);
    haar_pass<J, st, 0>(s);
  }
}

// Levels 2..J forward (inverse) on the shared approximations; callers
// synchronise before the first pass.
template <int J>
__device__ void upper_forward(float2* s) {
  if constexpr (J >= 2) haar_level<J, 2>(s, false);
  if constexpr (J >= 3) haar_level<J, 3>(s, false);
  if constexpr (J >= 4) haar_level<J, 4>(s, false);
}

template <int J>
__device__ void upper_inverse(float2* s) {
  if constexpr (J >= 4) haar_level<J, 4>(s, true);
  if constexpr (J >= 3) haar_level<J, 3>(s, true);
  if constexpr (J >= 2) haar_level<J, 2>(s, true);
}

// In place: v <- W^H soft(W v, tau) for the group's eight values, levels
// 2..J shared through s (every thread of the CTA must call it).
template <int J>
__device__ __forceinline__ void prox_group(float2 v[8], float2* s, float tau) {
  if constexpr (J == 0) {
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = soft(v[k], tau);
  } else {
    haar8_forward(v);
#pragma unroll
    for (int k = 1; k < 8; ++k) v[k] = soft(v[k], tau);
    if constexpr (J == 1) {
      v[0] = soft(v[0], tau);
    } else {
      s[threadIdx.x] = v[0];
      __syncthreads();
      upper_forward<J>(s);
      s[threadIdx.x] = soft(s[threadIdx.x], tau);
      __syncthreads();
      upper_inverse<J>(s);
      v[0] = s[threadIdx.x];
    }
    haar8_inverse(v);
  }
}

// Mallat-layout index of the coefficient that the lifting layout holds at
// global position (x0, x1, x2): within its cube, the smallest count of
// trailing zero bits over the three local coordinates gives the level
// (l = 1 + min) and the axes attaining it the high-pass sub-band; all-zero
// local coordinates hold the approximation.
template <int J>
__device__ __forceinline__ long long mallat_index(const Vol& g, int x0, int x1, int x2) {
  constexpr int b = 1 << J;
  const int c[3] = {x0 >> J, x1 >> J, x2 >> J};
  const int l[3] = {x0 & (b - 1), x1 & (b - 1), x2 & (b - 1)};
  const int n[3] = {g.n0, g.n1, g.n2};
  int t[3];
  int mn = J;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    t[a] = l[a] ? min(__ffs(l[a]) - 1, J) : J;
    mn = min(mn, t[a]);
  }
  int G[3];
  if (mn >= J) {
#pragma unroll
    for (int a = 0; a < 3; ++a) G[a] = c[a];
  } else {
    const int lev = mn + 1;
#pragma unroll
    for (int a = 0; a < 3; ++a)
      G[a] = (t[a] == mn ? (n[a] >> lev) : 0) + (c[a] << (J - lev)) + (l[a] >> lev);
  }
  return lin(g, G[0], G[1], G[2]);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block sum over NT threads; result valid in thread 0.
template <int NT>
__device__ double block_sum(double v) {
  __shared__ double red[NT / 32];
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) t = warp_sum(threadIdx.x < NT / 32 ? red[threadIdx.x] : 0.0);
  __syncthreads();
  return t;
}

// ---- FISTA step -------------------------------------------------------------
// v = z - step (g - b); x_new = W^H soft(W v, tau); z = x_new + mu (x_new - x);
// x = x_new.  partial[box] = |x_new - x|^2, partial[nbox + box] = |x_new|^2
// over the box.
template <int J>
__global__ void __launch_bounds__(Box<J>::nt, Box<J>::nt == 512 ? 2 : 3) fista_step_kernel(
    const float2* __restrict__ gz, const float2* __restrict__ bv, float2* __restrict__ x,
    float2* __restrict__ z, Vol g, float step, float tau, const double* __restrict__ mu_tab,
    const int* __restrict__ iter, double* __restrict__ partial) {
  constexpr int NT = Box<J>::nt;
  __shared__ float2 s[NT];
  __shared__ float4 sx[4 * NT];  // x_{k-1}, prefetched during the transform
  const Group gr = group_of<J>(g);
  float2 v[8], xo[8];
  if (gr.any) {
    prefetch8<NT>(x, g, gr, sx);
    float2 zz[8], gg[8], bb[8];
    load8(z, g, gr, zz);
    load8(gz, g, gr, gg);
    load8(bv, g, gr, bb);
#pragma unroll
    for (int k = 0; k < 8; ++k)
      v[k] = make_float2(fmaf(-step, gg[k].x - bb[k].x, zz[k].x),
                         fmaf(-step, gg[k].y - bb[k].y, zz[k].y));
  } else {
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = make_float2(0.0f, 0.0f);
  }
  prox_group<J>(v, s, tau);
  cp_async_wait_all();
  if (gr.any) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const float4 f = sx[r * NT + threadIdx.x];
      xo[2 * r] = make_float2(f.x, f.y);
      xo[2 * r + 1] = make_float2(f.z, f.w);
    }
  } else {
#pragma unroll
    for (int k = 0; k < 8; ++k) xo[k] = make_float2(0.0f, 0.0f);
  }
  const float mu = (float)mu_tab[*iter];
  // the group's eight terms in FP32 (FP64 arithmetic is a slow pipe on this
  // part), block and grid sums in FP64; outside the volume v = xo = 0
  float ddf = 0.0f, xxf = 0.0f;
  float2 zn[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const float dx = v[k].x - xo[k].x, dy = v[k].y - xo[k].y;
    zn[k] = make_float2(fmaf(mu, dx, v[k].x), fmaf(mu, dy, v[k].y));
    ddf = fmaf(dx, dx, fmaf(dy, dy, ddf));
    xxf = fmaf(v[k].x, v[k].x, fmaf(v[k].y, v[k].y, xxf));
  }
  double dd = ddf, xx = xxf;
  if (gr.any) {
    store8(x, g, gr, v);
    store8(z, g, gr, zn);
  }
  dd = block_sum<Box<J>::nt>(dd);
  xx = block_sum<Box<J>::nt>(xx);
  if (threadIdx.x == 0) {
    partial[blockIdx.x] = dd;
    partial[gridDim.x + blockIdx.x] = xx;
  }
}

// hist[k] = sqrt(sum dd / sum xx) (0 when x_k = 0); k += 1.
__global__ void __launch_bounds__(kThreads) fista_finish_kernel(const double* __restrict__ partial,
                                                                int nbox, int* iter,
                                                                double* __restrict__ hist) {
  double dd = 0.0, xx = 0.0;
  for (int i = threadIdx.x; i < nbox; i += kThreads) {
    dd += partial[i];
    xx += partial[nbox + i];
  }
  dd = block_sum<kThreads>(dd);
  xx = block_sum<kThreads>(xx);
  if (threadIdx.x == 0) {
    const int k = *iter;
    hist[k] = xx > 0.0 ? sqrt(dd / xx) : 0.0;
    *iter = k + 1;
  }
}

// ---- stand-alone transform ----------------------------------------------
// mode 0: c = W x (Mallat layout); 1: x = W^H c; 2: u = W^H soft(W v, tau).
template <int J, int MODE>
__global__ void __launch_bounds__(Box<J>::nt) wavelet_kernel(const float2* __restrict__ in,
                                                             float2* __restrict__ out, Vol g,
                                                             float tau) {
  __shared__ float2 s[Box<J>::nt];
  const Group gr = group_of<J>(g);
  float2 v[8];
  if (MODE == 2) {
    if (gr.any) load8(in, g, gr, v);
    else
#pragma unroll
      for (int k = 0; k < 8; ++k) v[k] = make_float2(0.0f, 0.0f);
    prox_group<J>(v, s, tau);
    if (gr.any) store8(out, g, gr, v);
    return;
  }
  if (MODE == 0) {
    if (gr.any) load8(in, g, gr, v);
    else
#pragma unroll
      for (int k = 0; k < 8; ++k) v[k] = make_float2(0.0f, 0.0f);
    if constexpr (J >= 1) haar8_forward(v);
    if constexpr (J >= 2) {
      s[threadIdx.x] = v[0];
      __syncthreads();
      upper_forward<J>(s);
      v[0] = s[threadIdx.x];
    }
    if (!gr.any) return;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int x0 = gr.x0 + (k >> 2), x1 = gr.x1 + ((k >> 1) & 1), x2 = gr.x2 + (k & 1);
      if (x0 < g.n0 && x1 < g.n1 && x2 < g.n2) out[mallat_index<J>(g, x0, x1, x2)] = v[k];
    }
    return;
  }
  // MODE 1: gather from the Mallat layout, inverse
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int x0 = gr.x0 + (k >> 2), x1 = gr.x1 + ((k >> 1) & 1), x2 = gr.x2 + (k & 1);
    v[k] = (x0 < g.n0 && x1 < g.n1 && x2 < g.n2) ? in[mallat_index<J>(g, x0, x1, x2)]
                                                 : make_float2(0.0f, 0.0f);
  }
  if constexpr (J >= 2) {
    s[threadIdx.x] = v[0];
    __syncthreads();
    upper_inverse<J>(s);
    v[0] = s[threadIdx.x];
  }
  if constexpr (J >= 1) haar8_inverse(v);
  if (gr.any) store8(out, g, gr, v);
}

// ---- power iteration ------------------------------------------------------
// partial[blk] = Re<v, w>, partial[nb + blk] = <w, w>.
__global__ void __launch_bounds__(kThreads) dot2_kernel(const float2* __restrict__ v,
                                                        const float2* __restrict__ w, long long n,
                                                        double* __restrict__ partial) {
  double a = 0.0, b = 0.0;
  for (long long i = blockIdx.x * (long long)kThreads + threadIdx.x; i < n;
       i += (long long)gridDim.x * kThreads) {
    const float2 vi = v[i], wi = w[i];
    a = fma((double)vi.x, (double)wi.x, fma((double)vi.y, (double)wi.y, a));
    b = fma((double)wi.x, (double)wi.x, fma((double)wi.y, (double)wi.y, b));
  }
  a = block_sum<kThreads>(a);
  b = block_sum<kThreads>(b);
  if (threadIdx.x == 0) {
    partial[blockIdx.x] = a;
    partial[gridDim.x + blockIdx.x] = b;
  }
}

// scal[0] = Re<v, w> (the Rayleigh quotient when |v| = 1), scal[1] = 1 / |w|
// (0 when w = 0).
__global__ void __launch_bounds__(kThreads) eig_scalar_kernel(const double* __restrict__ partial,
                                                              int nb, double* scal) {
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < nb; i += kThreads) {
    a += partial[i];
    b += partial[nb + i];
  }
  a = block_sum<kThreads>(a);
  b = block_sum<kThreads>(b);
  if (threadIdx.x == 0) {
    scal[0] = a;
    scal[1] = b > 0.0 ? 1.0 / sqrt(b) : 0.0;
  }
}

// v = scal[1] w
__global__ void scale_kernel(const float2* __restrict__ w, float2* __restrict__ v, long long n,
                             const double* __restrict__ scal) {
  const float k = (float)scal[1];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float2 a = w[i];
    v[i] = make_float2(a.x * k, a.y * k);
  }
}

bool levels_ok(int J, int n0, int n1, int n2) {
  if (J < 0 || J > kMaxLevels || n0 < 1 || n1 < 1 || n2 < 1) return false;
  const int m = (1 << J) - 1;
  return !(n0 & m) && !(n1 & m) && !(n2 & m);
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

// Box grid of a volume for J levels; vec: every pointer the kernel touches is
// 16-byte aligned (row pairs are then aligned when n2 is even).
Vol make_vol(int J, int n0, int n1, int n2, bool vec, long long* nbox) {
  int b0, b1, b2;
  box_dims(J, &b0, &b1, &b2);
  Vol g{n0, n1, n2, (n1 + b1 - 1) / b1, (n2 + b2 - 1) / b2, (vec && n2 % 2 == 0) ? 1 : 0};
  *nbox = (long long)((n0 + b0 - 1) / b0) * g.nb1 * g.nb2;
  return g;
}

template <int J>
void launch_step_J(long long nbox, const Vol& g, const float2* gz, const float2* bv, float2* x,
                   float2* z, float step, float tau, const double* mu, const int* iter,
                   double* partial, cudaStream_t s) {
  fista_step_kernel<J><<<unsigned(nbox), Box<J>::nt, 0, s>>>(gz, bv, x, z, g, step, tau, mu, iter,
                                                            partial);
}

void launch_step(int J, long long nbox, const Vol& g, const float2* gz, const float2* bv,
                 float2* x, float2* z, float step, float tau, const double* mu, const int* iter,
                 double* partial, cudaStream_t s) {
  switch (J) {
    case 0: launch_step_J<0>(nbox, g, gz, bv, x, z, step, tau, mu, iter, partial, s); break;
    case 1: launch_step_J<1>(nbox, g, gz, bv, x, z, step, tau, mu, iter, partial, s); break;
    case 2: launch_step_J<2>(nbox, g, gz, bv, x, z, step, tau, mu, iter, partial, s); break;
    case 3: launch_step_J<3>(nbox, g, gz, bv, x, z, step, tau, mu, iter, partial, s); break;
    default: launch_step_J<4>(nbox, g, gz, bv, x, z, step, tau, mu, iter, partial, s); break;
  }
}

template <int J>
void launch_wavelet_J(int mode, long long nbox, const Vol& g, const float2* in, float2* out,
                      float tau, cudaStream_t s) {
  const unsigned nb = unsigned(nbox);
  constexpr int nt = Box<J>::nt;
  if (mode == 0) wavelet_kernel<J, 0><<<nb, nt, 0, s>>>(in, out, g, tau);
  else if (mode == 1) wavelet_kernel<J, 1><<<nb, nt, 0, s>>>(in, out, g, tau);
  else wavelet_kernel<J, 2><<<nb, nt, 0, s>>>(in, out, g, tau);
}

nrsense_status wavelet_call(int mode, const nrsense_c64* in, nrsense_c64* out, const int32_t* n,
                            int32_t J, double tau, void* stream) {
  if (in == nullptr || out == nullptr || n == nullptr) return NRSENSE_ERR_ARG;
  if (!levels_ok(J, n[0], n[1], n[2])) return NRSENSE_ERR_ARG;
  if (mode != 2 && (const void*)in == (const void*)out) return NRSENSE_ERR_ARG;
  if (mode == 2 && !(tau >= 0.0 && std::isfinite(tau))) return NRSENSE_ERR_ARG;
  long long nbox = 0;
  const Vol g = make_vol(J, n[0], n[1], n[2], aligned16(in) && aligned16(out), &nbox);
  if (nbox > 0x7fffffffLL) return NRSENSE_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const float2* a = reinterpret_cast<const float2*>(in);
  float2* o = reinterpret_cast<float2*>(out);
  switch (J) {
    case 0: launch_wavelet_J<0>(mode, nbox, g, a, o, float(tau), s); break;
    case 1: launch_wavelet_J<1>(mode, nbox, g, a, o, float(tau), s); break;
    case 2: launch_wavelet_J<2>(mode, nbox, g, a, o, float(tau), s); break;
    case 3: launch_wavelet_J<3>(mode, nbox, g, a, o, float(tau), s); break;
    default: launch_wavelet_J<4>(mode, nbox, g, a, o, float(tau), s); break;
  }
  return cudaGetLastError() == cudaSuccess ? NRSENSE_OK : NRSENSE_ERR_CUDA;
}

#define NRS_TRY(expr)                  \
  do {                                 \
    nrsense_status _st = (expr);       \
    if (_st != NRSENSE_OK) return _st; \
  } while (0)

}  // namespace

// ---------------------------------------------------------------------------

struct nrsense_fista_ws {
  nrsense_c64 *z = nullptr, *g = nullptr, *b = nullptr;
  double* partial = nullptr;  // 2 * max(boxes, kRedBlocks)
  long long partial_cap = 0;
  double* mu = nullptr;       // momentum table
  double* hist = nullptr;     // relative change per iteration
  int cap = 0;                // entries of mu and hist
  int* iter = nullptr;        // device iteration counter
  double* scal = nullptr;     // power iteration scalars
  cudaStream_t cs = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  cudaGraphExec_t gexec = nullptr;
  // what the captured graph baked in
  const void* g_x = nullptr;
  int g_J = -1;
  float g_step = 0.0f, g_tau = 0.0f;
  const void* g_mu = nullptr;
  const void* g_partial = nullptr;
  uint64_t g_epoch = ~0ull;  // plan epoch (buffers and choices of the operator)
};

namespace nrs {

void fista_release(nrsense_plan_s* p) {
  nrsense_fista_ws* w = p->fista;
  if (!w) return;
  if (w->gexec) cudaGraphExecDestroy(w->gexec);
  if (w->cs) cudaStreamDestroy(w->cs);
  if (w->ev0) cudaEventDestroy(w->ev0);
  if (w->ev1) cudaEventDestroy(w->ev1);
  cudaFree(w->z);
  cudaFree(w->g);
  cudaFree(w->b);
  cudaFree(w->partial);
  cudaFree(w->mu);
  cudaFree(w->hist);
  cudaFree(w->iter);
  cudaFree(w->scal);
  delete w;
  p->fista = nullptr;
}

}  // namespace nrs

namespace {

nrsense_status fista_workspace(nrsense_plan_s* p, int maxit, long long nbox) {
  const size_t vb = size_t(p->geo.nvox) * sizeof(nrsense_c64);
  if (!p->fista) {
    p->fista = new (std::nothrow) nrsense_fista_ws();
    if (!p->fista) return NRSENSE_ERR_OOM;
    nrsense_fista_ws* w = p->fista;
    if (cudaMalloc(&w->z, vb) != cudaSuccess || cudaMalloc(&w->g, vb) != cudaSuccess ||
        cudaMalloc(&w->b, vb) != cudaSuccess || cudaMalloc(&w->iter, sizeof(int)) != cudaSuccess ||
        cudaMalloc(&w->scal, 2 * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      return NRSENSE_ERR_OOM;
    }
    if (cudaStreamCreateWithFlags(&w->cs, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&w->ev0, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&w->ev1, cudaEventDisableTiming) != cudaSuccess)
      return NRSENSE_ERR_CUDA;
  }
  nrsense_fista_ws* w = p->fista;
  const long long need = 2 * std::max<long long>(nbox, kRedBlocks);
  if (w->partial_cap < need) {
    cudaFree(w->partial);
    w->partial = nullptr;
    w->partial_cap = 0;
    if (cudaMalloc(&w->partial, size_t(need) * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      return NRSENSE_ERR_OOM;
    }
    w->partial_cap = need;
  }
  if (w->cap < std::max(maxit, 1)) {
    cudaFree(w->mu);
    cudaFree(w->hist);
    w->mu = w->hist = nullptr;
    w->cap = 0;
    const int c = std::max(maxit, 1);
    if (cudaMalloc(&w->mu, size_t(c) * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&w->hist, size_t(c) * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      return NRSENSE_ERR_OOM;
    }
    w->cap = c;
  }
  return NRSENSE_OK;
}

nrsense_status launched() {
  return cudaGetLastError() == cudaSuccess ? NRSENSE_OK : NRSENSE_ERR_CUDA;
}

// One FISTA iteration on stream s: g = E0 z, the fused step, the finish kernel.
nrsense_status fista_iteration(nrsense_plan_s* p, int J, long long nbox, const Vol& vol,
                               nrsense_c64* x, float step, float tau, cudaStream_t s) {
  nrsense_fista_ws* w = p->fista;
  NRS_TRY(nrsense_apply_normal(p, w->z, 0.0, w->g, s));
  StageMark m(p, NRSENSE_STAGE_FISTA, s);
  launch_step(J, nbox, vol, reinterpret_cast<const float2*>(w->g),
              reinterpret_cast<const float2*>(w->b), reinterpret_cast<float2*>(x),
              reinterpret_cast<float2*>(w->z), step, tau, w->mu, w->iter, w->partial, s);
  fista_finish_kernel<<<1, kThreads, 0, s>>>(w->partial, int(nbox), w->iter, w->hist);
  p->launches += 2;
  return launched();
}

}  // namespace

extern "C" {

nrsense_status nrsense_wavelet_forward(const nrsense_c64* x, nrsense_c64* c, const int32_t* n,
                                       int32_t levels, void* stream) {
  return wavelet_call(0, x, c, n, levels, 0.0, stream);
}

nrsense_status nrsense_wavelet_inverse(const nrsense_c64* c, nrsense_c64* x, const int32_t* n,
                                       int32_t levels, void* stream) {
  return wavelet_call(1, c, x, n, levels, 0.0, stream);
}

nrsense_status nrsense_wavelet_shrink(const nrsense_c64* v, nrsense_c64* u, const int32_t* n,
                                      int32_t levels, double tau, void* stream) {
  return wavelet_call(2, v, u, n, levels, tau, stream);
}

nrsense_status nrsense_normal_max_eig(nrsense_plan_t p, nrsense_c64* v, int32_t iters,
                                      double* eig, void* stream) {
  if (p == nullptr || v == nullptr || eig == nullptr || iters < 1 || iters > 100000)
    return NRSENSE_ERR_ARG;
  NRS_TRY(fista_workspace(p, 1, 0));
  nrsense_fista_ws* w = p->fista;
  const long long n = p->geo.nvox;
  cudaStream_t us = static_cast<cudaStream_t>(stream), s = w->cs;
  if (cudaEventRecord(w->ev0, us) != cudaSuccess || cudaStreamWaitEvent(s, w->ev0, 0) != cudaSuccess)
    return NRSENSE_ERR_CUDA;
  float2* vf = reinterpret_cast<float2*>(v);
  {
    StageMark m(p, NRSENSE_STAGE_FISTA, s);
    dot2_kernel<<<kRedBlocks, kThreads, 0, s>>>(vf, vf, n, w->partial);
    eig_scalar_kernel<<<1, kThreads, 0, s>>>(w->partial, kRedBlocks, w->scal);
    scale_kernel<<<kRedBlocks, kThreads, 0, s>>>(vf, vf, n, w->scal);
    p->launches += 3;
  }
  for (int k = 0; k < iters; ++k) {
    NRS_TRY(nrsense_apply_normal(p, v, 0.0, w->g, s));
    StageMark m(p, NRSENSE_STAGE_FISTA, s);
    const float2* gf = reinterpret_cast<const float2*>(w->g);
    dot2_kernel<<<kRedBlocks, kThreads, 0, s>>>(vf, gf, n, w->partial);
    eig_scalar_kernel<<<1, kThreads, 0, s>>>(w->partial, kRedBlocks, w->scal);
    scale_kernel<<<kRedBlocks, kThreads, 0, s>>>(gf, vf, n, w->scal);
    p->launches += 3;
  }
  NRS_TRY(launched());
  double h[2];
  if (cudaMemcpyAsync(h, w->scal, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return NRSENSE_ERR_CUDA;
  *eig = h[0];
  if (cudaEventRecord(w->ev1, s) != cudaSuccess || cudaStreamWaitEvent(us, w->ev1, 0) != cudaSuccess)
    return NRSENSE_ERR_CUDA;
  return NRSENSE_OK;
}

nrsense_status nrsense_fista_lipschitz(nrsense_plan_t p, nrsense_c64* v, int32_t iters,
                                      double margin, double* lipschitz, void* stream) {
  if (lipschitz == nullptr || !(margin >= 1.0) || !std::isfinite(margin)) return NRSENSE_ERR_ARG;
  double q = 0.0;
  NRS_TRY(nrsense_normal_max_eig(p, v, iters, &q, stream));
  // the gradient of ||y - A x||^2 is 2 (E0 x - b): its Lipschitz constant is
  // 2 lambda_max(E0); q approaches lambda_max from below, hence the margin
  *lipschitz = 2.0 * margin * q;
  return NRSENSE_OK;
}

nrsense_status nrsense_solve_fista(nrsense_plan_t p, const nrsense_c64* y, double lambda,
                                   int32_t levels, double lipschitz, int32_t maxit, uint32_t flags,
                                   nrsense_c64* x, double* hist_host, void* stream) {
  if (p == nullptr || y == nullptr || x == nullptr || maxit < 0 || maxit > (1 << 20) ||
      !(lambda >= 0.0) || !std::isfinite(lambda) || !(lipschitz > 0.0) ||
      !std::isfinite(lipschitz) || (flags & ~uint32_t(NRSENSE_CG_X0 | NRSENSE_CG_GRAPH)))
    return NRSENSE_ERR_ARG;
  const Geo& geo = p->geo;
  if (!levels_ok(levels, geo.n0, geo.n1, geo.n2)) return NRSENSE_ERR_ARG;
  long long nbox = 0;
  // workspace vectors come from cudaMalloc (256-byte aligned); x is the caller's
  const Vol vol = make_vol(levels, geo.n0, geo.n1, geo.n2, aligned16(x), &nbox);
  NRS_TRY(fista_workspace(p, maxit, nbox));
  nrsense_fista_ws* w = p->fista;
  const size_t vb = size_t(geo.nvox) * sizeof(nrsense_c64);
  cudaStream_t us = static_cast<cudaStream_t>(stream), s = w->cs;
  if (cudaEventRecord(w->ev0, us) != cudaSuccess || cudaStreamWaitEvent(s, w->ev0, 0) != cudaSuccess)
    return NRSENSE_ERR_CUDA;

  // momentum table: t_1 = 1, t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2, mu_k = (t_k - 1) / t_{k+1}
  std::vector<double> mu(size_t(std::max(maxit, 1)), 0.0);
  double t = 1.0;
  for (int k = 0; k < maxit; ++k) {
    const double tn = 0.5 * (1.0 + std::sqrt(1.0 + 4.0 * t * t));
    mu[size_t(k)] = (t - 1.0) / tn;
    t = tn;
  }
  if (cudaMemcpyAsync(w->mu, mu.data(), mu.size() * sizeof(double), cudaMemcpyHostToDevice, s) !=
          cudaSuccess ||
      cudaMemsetAsync(w->iter, 0, sizeof(int), s) != cudaSuccess)
    return NRSENSE_ERR_CUDA;

  // b = sum_j A_j^H y_j;  z_1 = x_0
  NRS_TRY(nrsense_apply_adjoint(p, y, w->b, s));
  if (!(flags & NRSENSE_CG_X0) && cudaMemsetAsync(x, 0, vb, s) != cudaSuccess)
    return NRSENSE_ERR_CUDA;
  if (cudaMemcpyAsync(w->z, x, vb, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return NRSENSE_ERR_CUDA;

  const float step = float(2.0 / lipschitz);
  const float tau = float(lambda / lipschitz);
  const bool graph = (flags & NRSENSE_CG_GRAPH) != 0;
  int done = 0;
  if (graph && maxit >= kChunk) {
    if (w->gexec == nullptr || w->g_x != x || w->g_J != levels || w->g_step != step ||
        w->g_tau != tau || w->g_mu != w->mu || w->g_partial != w->partial ||
        w->g_epoch != p->epoch) {
      if (w->gexec) {
        cudaGraphExecDestroy(w->gexec);
        w->gexec = nullptr;
      }
      cudaGraph_t gph = nullptr;
      if (cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed) != cudaSuccess)
        return NRSENSE_ERR_CUDA;
      nrsense_status cst = NRSENSE_OK;
      for (int k = 0; k < kChunk && cst == NRSENSE_OK; ++k)
        cst = fista_iteration(p, levels, nbox, vol, x, step, tau, s);
      const cudaError_t e = cudaStreamEndCapture(s, &gph);
      if (cst != NRSENSE_OK) {
        if (gph) cudaGraphDestroy(gph);
        return cst;
      }
      if (e != cudaSuccess || cudaGraphInstantiate(&w->gexec, gph, 0) != cudaSuccess) {
        if (gph) cudaGraphDestroy(gph);
        cudaGetLastError();
        w->gexec = nullptr;
        return NRSENSE_ERR_CUDA;
      }
      cudaGraphDestroy(gph);
      w->g_x = x;
      w->g_J = levels;
      w->g_step = step;
      w->g_tau = tau;
      w->g_mu = w->mu;
      w->g_partial = w->partial;
      w->g_epoch = p->epoch;
    }
    for (; done + kChunk <= maxit; done += kChunk) {
      if (cudaGraphLaunch(w->gexec, s) != cudaSuccess) return NRSENSE_ERR_CUDA;
      p->launches += 2LL * kChunk;  // the captured operator's kernels are not recounted
    }
  }
  for (; done < maxit; ++done) NRS_TRY(fista_iteration(p, levels, nbox, vol, x, step, tau, s));

  if (hist_host && maxit > 0 &&
      cudaMemcpyAsync(hist_host, w->hist, size_t(maxit) * sizeof(double), cudaMemcpyDeviceToHost,
                      s) != cudaSuccess)
    return NRSENSE_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return NRSENSE_ERR_CUDA;
  if (cudaEventRecord(w->ev1, s) != cudaSuccess || cudaStreamWaitEvent(us, w->ev1, 0) != cudaSuccess)
    return NRSENSE_ERR_CUDA;
  return NRSENSE_OK;
}

}  // extern "C"
