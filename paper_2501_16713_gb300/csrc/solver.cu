// Conjugate gradients on the normal equations of the reconstruction problem.
//
// The paper poses the motion-corrected reconstruction as a regularised least
// squares problem over the stacked nonrigid SENSE operators (reconstruction
// optimisation equation).  With a Tikhonov term lambda ||x||^2 the minimiser
// solves E x = b, E = sum_j A_j^H A_j + lambda I, b = sum_j A_j^H y_j; E is
// Hermitian positive definite for lambda > 0 and CG (Hestenes-Stiefel) applies.
//
// GPU layout: vectors x, r, p, E p are FP32 complex; every inner product,
// step size (alpha, beta) and residual norm is FP64 and stays on the device.
// Inner products are block partial sums in a fixed grid order followed by a
// one-block sum, so results are bitwise reproducible.  The host only starts
// the solve, launches the iteration chunks (optionally as a captured CUDA
// graph) and reads the iteration count and residual history at the end (and
// the converged flag between chunks).
//
// Flexible CG (Notay's FCG(1), Polak-Ribiere form) takes z_k = M(r_k) from
// the learned preconditioner network, a nonlinear map, so the search
// directions are re-conjugated only against the previous one:
//   alpha = Re<r, z> / Re<p, E p>,  beta = Re<z_new, r_new - r> / Re<z, r>
//         = -alpha Re<z_new, E p> / Re<z, r>,  p = z_new + beta p.
// Real parts of the complex inner products are the inner product of the
// equivalent real system, on which E is symmetric positive definite.  When the
// network returns a direction with Re<r, z> <= 0 (not a descent direction)
// the iteration falls back to z = r and restarts (beta = 0): a plain CG step.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>

#include "plan_internal.h"

using namespace nrs;

namespace {

constexpr int kRedThreads = 256;
constexpr int kRedBlocks = 1184;  // fixed grid: deterministic summation order (8 x 148)
constexpr int kGraphMax = 64;     // iterations captured in one graph (fixed-count solves)

struct CgState {
  double rr;      // <r, r>
  double bb;      // <b, b>
  double alpha;
  double beta;
  double tol2;    // tol^2 <b, b>
  int iter;       // completed iterations
  int done;       // converged, broken down or maxit reached
  int status;     // NRSENSE_OK or NRSENSE_ERR_BREAKDOWN
  int maxit;
  double rz;      // flexible CG: Re<r, z>
  int fb;         // flexible CG: this step falls back to z = r
  int n_fb;       // flexible CG: fallbacks taken
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum of v over the block (result valid in thread 0).
__device__ double block_sum(double v) {
  __shared__ double s[kRedThreads / 32];
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) s[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (warp == 0) {
    t = lane < (int)(blockDim.x >> 5) ? s[lane] : 0.0;
    t = warp_sum(t);
  }
  __syncthreads();
  return t;
}

// partial[block] = sum Re(conj(x_i) y_i) in FP64 over a fixed grid-stride range.
__global__ void __launch_bounds__(kRedThreads) dot_partial_kernel(const float2* __restrict__ x,
                                                                  const float2* __restrict__ y,
                                                                  long long n,
                                                                  double* __restrict__ partial) {
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float2 a = x[i], b = y[i];
    acc = fma((double)a.x, (double)b.x, fma((double)a.y, (double)b.y, acc));
  }
  acc = block_sum(acc);
  if (threadIdx.x == 0) partial[blockIdx.x] = acc;
}

__device__ double sum_partials(const double* __restrict__ partial, int nb) {
  double acc = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) acc += partial[i];
  return block_sum(acc);
}

// Start: <b,b> from partials (and <r,r> from partials2 when an initial guess
// was given, else r = b).
__global__ void cg_init_kernel(const double* __restrict__ partial, const double* __restrict__ partial2,
                               int nb, double tol, int maxit, CgState* st, double* hist) {
  const double bb = sum_partials(partial, nb);
  const double rr = partial2 ? sum_partials(partial2, nb) : bb;
  if (threadIdx.x == 0) {
    st->bb = bb;
    st->rr = rr;
    st->tol2 = tol * tol * bb;
    st->iter = 0;
    st->alpha = 0.0;
    st->beta = 0.0;
    st->maxit = maxit;
    st->status = NRSENSE_OK;
    st->rz = rr;
    st->fb = 0;
    st->n_fb = 0;
    const double rel = bb > 0.0 ? sqrt(rr / bb) : 0.0;
    hist[0] = rel;
    st->done = (bb == 0.0 || rr <= st->tol2 || maxit <= 0) ? 1 : 0;
  }
}

// alpha = <r,r> / <p, E p>; breakdown on non-positive or non-finite curvature.
// (flexible CG: alpha = Re<r, z> / <p, E p>)
__global__ void cg_alpha_kernel(const double* __restrict__ partial, int nb, CgState* st,
                                int flexible) {
  const double pAp = sum_partials(partial, nb);
  if (threadIdx.x == 0) {
    const double num = flexible ? st->rz : st->rr;
    if (st->done) {
      st->alpha = 0.0;
    } else if (!(pAp > 0.0) || !isfinite(pAp) || !isfinite(num)) {
      st->alpha = 0.0;
      st->status = NRSENSE_ERR_BREAKDOWN;
      st->done = 1;
    } else {
      st->alpha = num / pAp;
    }
  }
}

// x += alpha p; r -= alpha E p; partial = |r|^2 (FP64).
__global__ void __launch_bounds__(kRedThreads) cg_update_xr_kernel(
    float2* __restrict__ x, float2* __restrict__ r, const float2* __restrict__ p,
    const float2* __restrict__ Ep, long long n, const CgState* __restrict__ st,
    double* __restrict__ partial) {
  const float a = (float)st->alpha;
  const bool skip = st->done && a == 0.0f;
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    float2 ri = r[i];
    if (!skip) {
      const float2 pi = p[i], ei = Ep[i];
      float2 xi = x[i];
      xi.x = fmaf(a, pi.x, xi.x);
      xi.y = fmaf(a, pi.y, xi.y);
      x[i] = xi;
      ri.x = fmaf(-a, ei.x, ri.x);
      ri.y = fmaf(-a, ei.y, ri.y);
      r[i] = ri;
    }
    acc = fma((double)ri.x, (double)ri.x, fma((double)ri.y, (double)ri.y, acc));
  }
  acc = block_sum(acc);
  if (threadIdx.x == 0) partial[blockIdx.x] = acc;
}

// beta = <r,r>_new / <r,r>; record the residual; test convergence.
__global__ void cg_beta_kernel(const double* __restrict__ partial, int nb, CgState* st,
                               double* hist) {
  const double rr_new = sum_partials(partial, nb);
  if (threadIdx.x == 0) {
    if (st->done) {
      st->beta = 0.0;
    } else {
      st->beta = rr_new / st->rr;
      st->rr = rr_new;
      st->iter += 1;
      hist[st->iter] = sqrt(rr_new / st->bb);
      if (rr_new <= st->tol2 || st->iter >= st->maxit) st->done = 1;
      if (!isfinite(rr_new)) {
        st->status = NRSENSE_ERR_BREAKDOWN;
        st->done = 1;
      }
    }
  }
}

// p = r + beta p (skipped once done).
__global__ void cg_update_p_kernel(const float2* __restrict__ r, float2* __restrict__ p, long long n,
                                   const CgState* __restrict__ st) {
  if (st->done) return;
  const float b = (float)st->beta;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float2 ri = r[i];
    float2 pi = p[i];
    pi.x = fmaf(b, pi.x, ri.x);
    pi.y = fmaf(b, pi.y, ri.y);
    p[i] = pi;
  }
}

// Flexible CG: record |r|^2 after the update and test convergence.
__global__ void fcg_check_kernel(const double* __restrict__ partial, int nb, CgState* st,
                                 double* hist) {
  const double rr_new = sum_partials(partial, nb);
  if (threadIdx.x == 0 && !st->done) {
    st->rr = rr_new;
    st->iter += 1;
    hist[st->iter] = sqrt(rr_new / st->bb);
    if (rr_new <= st->tol2 || st->iter >= st->maxit) st->done = 1;
    if (!isfinite(rr_new)) {
      st->status = NRSENSE_ERR_BREAKDOWN;
      st->done = 1;
    }
  }
}

// partial = Re<z, r>, partial[nb..] = Re<z, q> (q may be null: not needed).
__global__ void __launch_bounds__(kRedThreads) dot2_partial_kernel(
    const float2* __restrict__ z, const float2* __restrict__ r, const float2* __restrict__ q,
    long long n, double* __restrict__ partial) {
  double a = 0.0, b = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float2 zi = z[i], ri = r[i];
    a = fma((double)zi.x, (double)ri.x, fma((double)zi.y, (double)ri.y, a));
    if (q) {
      const float2 qi = q[i];
      b = fma((double)zi.x, (double)qi.x, fma((double)zi.y, (double)qi.y, b));
    }
  }
  a = block_sum(a);
  b = block_sum(b);
  if (threadIdx.x == 0) {
    partial[blockIdx.x] = a;
    partial[gridDim.x + blockIdx.x] = b;
  }
}

// Flexible CG direction coefficient.  start != 0: first direction (beta = 0).
// Non-descent network output (Re<r, z> <= 0 or non-finite): z = r, beta = 0.
__global__ void fcg_beta_kernel(const double* __restrict__ partial, int nb, CgState* st, int start) {
  const double rz_new = sum_partials(partial, nb);
  const double zq = sum_partials(partial + nb, nb);
  if (threadIdx.x == 0) {
    if (st->done && !start) {
      st->beta = 0.0;
      return;
    }
    if (!(rz_new > 0.0) || !isfinite(rz_new) || !isfinite(zq)) {
      st->fb = 1;
      st->n_fb += 1;
      st->beta = 0.0;
      st->rz = st->rr;
    } else {
      st->fb = 0;
      st->beta = start ? 0.0 : -st->alpha * zq / st->rz;
      st->rz = rz_new;
    }
  }
}

// p = (fb ? r : z) + beta p; p = (fb ? r : z) when beta == 0.
__global__ void fcg_update_p_kernel(const float2* __restrict__ z, const float2* __restrict__ r,
                                    float2* __restrict__ p, long long n,
                                    const CgState* __restrict__ st, int start) {
  if (st->done && !start) return;
  const float b = (float)st->beta;
  const float2* __restrict__ src = st->fb ? r : z;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float2 si = src[i];
    float2 pi = si;
    if (b != 0.0f) {
      pi = p[i];
      pi.x = fmaf(b, pi.x, si.x);
      pi.y = fmaf(b, pi.y, si.y);
    }
    p[i] = pi;
  }
}

// e_k = x - e_k (recorded iterates become errors against the final iterate)
__global__ void rsub_kernel(const float2* __restrict__ x, float2* __restrict__ e, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float2 a = x[i];
    float2 v = e[i];
    v.x = a.x - v.x;
    v.y = a.y - v.y;
    e[i] = v;
  }
}

// ---------------------------------------------------------------------------
// Deflation (A-DEF2 of Tang, Nabben and Vuik) with a basis W of k vectors.

constexpr int kDeflBlocks = 296;  // fixed grid of the k-vector dot products
constexpr int kDeflMax = 64;

// partial[(2 i + c) nb + block] = Re (c = 0) / Im (c = 1) of sum conj(V_i) z
// over the block's fixed grid-stride range, V_i = V + i n (FP64).
__global__ void __launch_bounds__(kRedThreads) defl_dots_kernel(const float2* __restrict__ V,
                                                                const float2* __restrict__ z,
                                                                long long n,
                                                                double* __restrict__ partial) {
  const int i = blockIdx.y;
  const float2* __restrict__ vi = V + (long long)i * n;
  double re = 0.0, im = 0.0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    const float2 a = vi[t], b = z[t];
    re = fma((double)a.x, (double)b.x, fma((double)a.y, (double)b.y, re));
    im = fma((double)a.x, (double)b.y, fma(-(double)a.y, (double)b.x, im));
  }
  re = block_sum(re);
  im = block_sum(im);
  if (threadIdx.x == 0) {
    partial[(2 * i) * gridDim.x + blockIdx.x] = re;
    partial[(2 * i + 1) * gridDim.x + blockIdx.x] = im;
  }
}

// d = the summed partials (W^H v, k complex, each summed in block order);
// coef = E_c^-1 d (complex FP64, E_c^-1 row-major).
__global__ void defl_coef_kernel(const double* __restrict__ partial, int nb, int k,
                                 const double* __restrict__ ecinv, double* __restrict__ coef) {
  __shared__ double d[2 * kDeflMax];
  for (int c = threadIdx.x; c < 2 * k; c += blockDim.x) {
    double acc = 0.0;
    for (int b = 0; b < nb; ++b) acc += partial[c * nb + b];
    d[c] = acc;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    double re = 0.0, im = 0.0;
    for (int j = 0; j < k; ++j) {
      const double ar = ecinv[2 * (i * k + j)], ai = ecinv[2 * (i * k + j) + 1];
      re += ar * d[2 * j] - ai * d[2 * j + 1];
      im += ar * d[2 * j + 1] + ai * d[2 * j];
    }
    coef[2 * i] = re;
    coef[2 * i + 1] = im;
  }
}

// out = in - sum_i c_i U_i (in may equal out); with x2: x2 += sum_i c_i U2_i.
// Terms in increasing i.
__global__ void __launch_bounds__(kRedThreads) defl_update_kernel(
    float2* out, const float2* in, const float2* __restrict__ U, const double* __restrict__ coef,
    int k, long long n, float2* x2, const float2* __restrict__ U2) {
  __shared__ float2 c[kDeflMax];
  if (threadIdx.x < k) c[threadIdx.x] = make_float2(float(coef[2 * threadIdx.x]),
                                                    float(coef[2 * threadIdx.x + 1]));
  __syncthreads();
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    float2 a = in[t];
    float2 xa = x2 ? x2[t] : make_float2(0.f, 0.f);
    for (int i = 0; i < k; ++i) {
      const float2 ci = c[i];
      const float2 u = U[(long long)i * n + t];
      a.x = fmaf(-ci.x, u.x, fmaf(ci.y, u.y, a.x));
      a.y = fmaf(-ci.x, u.y, fmaf(-ci.y, u.x, a.y));
      if (x2) {
        const float2 u2 = U2[(long long)i * n + t];
        xa.x = fmaf(ci.x, u2.x, fmaf(-ci.y, u2.y, xa.x));
        xa.y = fmaf(ci.x, u2.y, fmaf(ci.y, u2.x, xa.y));
      }
    }
    out[t] = a;
    if (x2) x2[t] = xa;
  }
}

// ew = e0w + lambda w over k n values
__global__ void defl_form_ew_kernel(float2* __restrict__ ew, const float2* __restrict__ e0w,
                                    const float2* __restrict__ w, float lambda, long long total) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const float2 a = e0w[t], b = w[t];
    ew[t] = make_float2(fmaf(lambda, b.x, a.x), fmaf(lambda, b.y, a.y));
  }
}

// dst = scale src (dst may equal src)
__global__ void defl_scale_kernel(float2* dst, const float2* src, float scale, long long n) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    const float2 a = src[t];
    dst[t] = make_float2(a.x * scale, a.y * scale);
  }
}

// out = sum_j coef[j] Z_j (real coefficients, j < m, in increasing j)
__global__ void defl_combine_kernel(float2* __restrict__ out, const float2* __restrict__ Z,
                                    const float* __restrict__ coef, int m, long long n) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    float2 a = make_float2(0.f, 0.f);
    for (int j = 0; j < m; ++j) {
      const float2 z = Z[(long long)j * n + t];
      a.x = fmaf(coef[j], z.x, a.x);
      a.y = fmaf(coef[j], z.y, a.y);
    }
    out[t] = a;
  }
}

// r = b - E x (r holds b on entry, Ex holds E x)
__global__ void sub_kernel(float2* __restrict__ r, const float2* __restrict__ ex, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    float2 v = r[i];
    const float2 e = ex[i];
    v.x -= e.x;
    v.y -= e.y;
    r[i] = v;
  }
}

// unit impulse at linear index idx (the vector is zeroed before)
__global__ void impulse_kernel(float2* x, long long idx) { x[idx] = make_float2(1.f, 0.f); }

// d[k] = 1 / (max(Re hhat_c[k], 0) + lam), hhat_c the DFT of the PSF with the
// image centre moved to the origin: for even N, DFT(roll(h, -N/2))[k] =
// (-1)^(k0 + k1 + k2) DFT(h)[k].
__global__ void circ_diag_kernel(const float2* __restrict__ hhat, float* __restrict__ d, int n0,
                                 int n1, int n2, float lam) {
  const long long n = (long long)n0 * n1 * n2;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int k2 = int(i % n2), k1 = int((i / n2) % n1), k0 = int(i / ((long long)n1 * n2));
    const float re = ((k0 + k1 + k2) & 1) ? -hhat[i].x : hhat[i].x;
    d[i] = 1.0f / (fmaxf(re, 0.0f) + lam);
  }
}

// t *= d / N (the inverse DFT's 1/N)
__global__ void circ_scale_kernel(float2* __restrict__ t, const float* __restrict__ d, long long n,
                                  float inv_n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float k = d[i] * inv_n;
    const float2 v = t[i];
    t[i] = make_float2(v.x * k, v.y * k);
  }
}

#define NRS_TRY(expr)                  \
  do {                                 \
    nrsense_status _st = (expr);       \
    if (_st != NRSENSE_OK) return _st; \
  } while (0)

nrsense_status launched() {
  return cudaGetLastError() == cudaSuccess ? NRSENSE_OK : NRSENSE_ERR_CUDA;
}

}  // namespace

// ---------------------------------------------------------------------------

struct nrsense_cg_ws {
  nrsense_c64 *r = nullptr, *p = nullptr, *Ep = nullptr, *b = nullptr;
  nrsense_c64* z = nullptr;    // flexible CG only (allocated on first use)
  nrsense_c64* zc = nullptr;   // circulant-preconditioned residual (allocated on first use)
  double* partial = nullptr;   // 2 * kRedBlocks
  CgState* st = nullptr;
  double* hist = nullptr;
  int hist_cap = 0;
  cudaStream_t cs = nullptr;   // capture / launch stream
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  cudaGraphExec_t gexec = nullptr;
  // what the captured graph baked in
  const void* g_x = nullptr;
  uint64_t g_net = 0;      // network serial
  uint64_t g_epoch = ~0ull;  // plan epoch
  int g_mode = -1;
  double g_lambda = 0.0;
  int g_chunk = 0;
};

namespace nrs {

void defl_release(nrsense_plan_s* p) {
  void* bufs[] = {p->defl_w, p->defl_e0w, p->defl_ew, p->defl_ecinv, p->defl_coef,
                  p->defl_partial};
  for (void* b : bufs) cudaFree(b);
  p->defl_w = p->defl_e0w = p->defl_ew = nullptr;
  p->defl_ecinv = p->defl_coef = p->defl_partial = nullptr;
  p->defl_k = 0;
  p->defl_lambda = -1.0;
  p->defl_g0.clear();
  p->defl_gw.clear();
  p->epoch += 1;
}

void cg_release(nrsense_plan_s* p) {
  defl_release(p);
  if (p->have_fft_circ) cufftDestroy(p->fft_circ);
  p->have_fft_circ = false;
  cudaFree(p->circ_d);
  cudaFree(p->circ_tmp);
  p->circ_d = nullptr;
  p->circ_tmp = nullptr;
  p->circ_on = false;
  nrsense_cg_ws* w = p->cg;
  if (!w) return;
  if (w->gexec) cudaGraphExecDestroy(w->gexec);
  if (w->cs) cudaStreamDestroy(w->cs);
  if (w->ev0) cudaEventDestroy(w->ev0);
  if (w->ev1) cudaEventDestroy(w->ev1);
  cudaFree(w->r);
  cudaFree(w->p);
  cudaFree(w->Ep);
  cudaFree(w->b);
  cudaFree(w->z);
  cudaFree(w->zc);
  cudaFree(w->partial);
  cudaFree(w->st);
  cudaFree(w->hist);
  delete w;
  p->cg = nullptr;
}

}  // namespace nrs

namespace {

nrsense_status cg_workspace(nrsense_plan_s* p, int maxit, bool flexible, bool circ = false) {
  const size_t vb = size_t(p->geo.nvox) * sizeof(nrsense_c64);
  if (!p->cg) {
    p->cg = new (std::nothrow) nrsense_cg_ws();
    if (!p->cg) return NRSENSE_ERR_OOM;
    nrsense_cg_ws* w = p->cg;
    if (cudaMalloc(&w->r, vb) != cudaSuccess || cudaMalloc(&w->p, vb) != cudaSuccess ||
        cudaMalloc(&w->Ep, vb) != cudaSuccess || cudaMalloc(&w->b, vb) != cudaSuccess ||
        cudaMalloc(&w->partial, 2 * kRedBlocks * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&w->st, sizeof(CgState)) != cudaSuccess) {
      cudaGetLastError();
      return NRSENSE_ERR_OOM;
    }
    if (cudaStreamCreateWithFlags(&w->cs, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&w->ev0, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&w->ev1, cudaEventDisableTiming) != cudaSuccess)
      return NRSENSE_ERR_CUDA;
  }
  nrsense_cg_ws* w = p->cg;
  if ((flexible && !w->z) || (circ && !w->zc) || w->hist_cap < maxit + 1) p->epoch += 1;
  if (flexible && !w->z && cudaMalloc(&w->z, vb) != cudaSuccess) {
    cudaGetLastError();
    w->z = nullptr;
    return NRSENSE_ERR_OOM;
  }
  if (circ && !w->zc && cudaMalloc(&w->zc, vb) != cudaSuccess) {
    cudaGetLastError();
    w->zc = nullptr;
    return NRSENSE_ERR_OOM;
  }
  if (w->hist_cap < maxit + 1) {
    cudaFree(w->hist);
    w->hist = nullptr;
    if (cudaMalloc(&w->hist, size_t(maxit + 1) * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      w->hist_cap = 0;
      return NRSENSE_ERR_OOM;
    }
    w->hist_cap = maxit + 1;
  }
  return NRSENSE_OK;
}

// z = M_c r = IDFT(d . DFT(r)) (circulant preconditioner; z may equal r)
nrsense_status circ_apply(nrsense_plan_s* p, const nrsense_c64* r, nrsense_c64* z, cudaStream_t s) {
  StageMark m(p, NRSENSE_STAGE_SOLVER, s);
  const long long n = p->geo.nvox;
  if (cufftSetStream(p->fft_circ, s) != CUFFT_SUCCESS ||
      cufftExecC2C(p->fft_circ, reinterpret_cast<cufftComplex*>(const_cast<nrsense_c64*>(r)),
                   reinterpret_cast<cufftComplex*>(p->circ_tmp), CUFFT_FORWARD) != CUFFT_SUCCESS)
    return NRSENSE_ERR_CUFFT;
  circ_scale_kernel<<<kRedBlocks, kRedThreads, 0, s>>>(reinterpret_cast<float2*>(p->circ_tmp),
                                                       p->circ_d, n, 1.0f / float(n));
  p->launches += 1;
  if (cufftExecC2C(p->fft_circ, reinterpret_cast<cufftComplex*>(p->circ_tmp),
                   reinterpret_cast<cufftComplex*>(z), CUFFT_INVERSE) != CUFFT_SUCCESS)
    return NRSENSE_ERR_CUFFT;
  return launched();
}

// Eigen-decomposition of a real symmetric m x m matrix (row-major) by cyclic
// Jacobi rotations (each rotation in the (p, q) plane zeroes A[p][q]; sweeps
// until the off-diagonal mass is below 1e-30 of the total): on return the
// diagonal of A holds the eigenvalues and column i of V the eigenvector of
// A[i][i].
void jacobi_eigen(int m, std::vector<double>& A, std::vector<double>& V) {
  V.assign(size_t(m) * m, 0.0);
  for (int i = 0; i < m; ++i) V[size_t(i) * m + i] = 1.0;
  for (int sweep = 0; sweep < 64; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int r = 0; r < m; ++r)
      for (int c = 0; c < m; ++c) {
        const double v = A[size_t(r) * m + c] * A[size_t(r) * m + c];
        tot += v;
        if (r != c) off += v;
      }
    if (off == 0.0 || off <= 1e-30 * tot) break;
    for (int pp = 0; pp < m - 1; ++pp)
      for (int q = pp + 1; q < m; ++q) {
        const double apq = A[size_t(pp) * m + q];
        if (apq == 0.0) continue;
        const double tau = (A[size_t(q) * m + q] - A[size_t(pp) * m + pp]) / (2.0 * apq);
        const double t = (tau >= 0.0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1.0 + tau * tau));
        const double c = 1.0 / std::sqrt(1.0 + t * t), sn = t * c;
        for (int r = 0; r < m; ++r) {  // A J
          const double arp = A[size_t(r) * m + pp], arq = A[size_t(r) * m + q];
          A[size_t(r) * m + pp] = c * arp - sn * arq;
          A[size_t(r) * m + q] = sn * arp + c * arq;
        }
        for (int r = 0; r < m; ++r) {  // J^T (A J)
          const double apr = A[size_t(pp) * m + r], aqr = A[size_t(q) * m + r];
          A[size_t(pp) * m + r] = c * apr - sn * aqr;
          A[size_t(q) * m + r] = sn * apr + c * aqr;
        }
        for (int r = 0; r < m; ++r) {  // V J
          const double vrp = V[size_t(r) * m + pp], vrq = V[size_t(r) * m + q];
          V[size_t(r) * m + pp] = c * vrp - sn * vrq;
          V[size_t(r) * m + q] = sn * vrp + c * vrq;
        }
      }
  }
}

// Eigenvalues ascending, eigenvectors as the columns of vecs (row-major).
void symmetric_eigen_sorted(int m, const double* a, double* vals, double* vecs) {
  std::vector<double> A(a, a + size_t(m) * m), V;
  jacobi_eigen(m, A, V);
  std::vector<int> order(m);
  for (int i = 0; i < m; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
    return A[size_t(x) * m + x] < A[size_t(y) * m + y];
  });
  for (int i = 0; i < m; ++i) {
    vals[i] = A[size_t(order[i]) * m + order[i]];
    for (int r = 0; r < m; ++r) vecs[size_t(r) * m + i] = V[size_t(r) * m + order[i]];
  }
}

// Pseudo-inverse of a Hermitian positive-semidefinite k x k complex matrix
// (row-major (re, im) pairs, FP64), in place: through the real symmetric
// embedding H = [[Re, -Im], [Im, Re]] (each eigenvalue twice), H^+ = sum over
// eigenvalues above 1e-10 of the largest of v v^T / theta, whose blocks are
// Re and Im of the pseudo-inverse.  Directions of nearly dependent basis
// vectors (repeated Ritz vectors of a long run) are dropped instead of
// amplified.  Returns the number of kept eigenvalue pairs (0: nothing left).
int pinv_hermitian(std::vector<double>& a, int k) {
  const int m = 2 * k;
  std::vector<double> H(size_t(m) * m), vals(m), vecs(size_t(m) * m);
  for (int r = 0; r < k; ++r)
    for (int c = 0; c < k; ++c) {
      const double re = 0.5 * (a[2 * (r * k + c)] + a[2 * (c * k + r)]);       // Hermitian part
      const double im = 0.5 * (a[2 * (r * k + c) + 1] - a[2 * (c * k + r) + 1]);
      H[size_t(r) * m + c] = re;
      H[size_t(r + k) * m + c + k] = re;
      H[size_t(r) * m + c + k] = -im;
      H[size_t(r + k) * m + c] = im;
    }
  symmetric_eigen_sorted(m, H.data(), vals.data(), vecs.data());
  const double top = vals[m - 1];
  if (!(top > 0.0) || !std::isfinite(top)) return 0;
  std::vector<double> P(size_t(m) * m, 0.0);
  int kept = 0;
  for (int e = 0; e < m; ++e) {
    if (!(vals[e] > 1e-10 * top)) continue;
    ++kept;
    const double inv = 1.0 / vals[e];
    for (int r = 0; r < m; ++r) {
      const double vr = vecs[size_t(r) * m + e] * inv;
      for (int c = 0; c < m; ++c) P[size_t(r) * m + c] += vr * vecs[size_t(c) * m + e];
    }
  }
  for (int r = 0; r < k; ++r)
    for (int c = 0; c < k; ++c) {
      a[2 * (r * k + c)] = P[size_t(r) * m + c];
      a[2 * (r * k + c) + 1] = P[size_t(r + k) * m + c];
    }
  return kept / 2;
}

// V^H z partial sums into p->defl_partial (V: `count` consecutive vectors)
void defl_dots(nrsense_plan_s* p, const nrsense_c64* V, int count, const nrsense_c64* z,
               cudaStream_t s) {
  defl_dots_kernel<<<dim3(kDeflBlocks, count), kRedThreads, 0, s>>>(
      reinterpret_cast<const float2*>(V), reinterpret_cast<const float2*>(z), p->geo.nvox,
      p->defl_partial);
  p->launches += 1;
}

// V^H z on the host (2 count values, each summed in block order)
nrsense_status defl_dots_host(nrsense_plan_s* p, const nrsense_c64* V, int count,
                              const nrsense_c64* z, cudaStream_t s, double* out) {
  const int k = count;
  defl_dots(p, V, count, z, s);
  std::vector<double> h(size_t(2) * k * kDeflBlocks);
  if (cudaMemcpyAsync(h.data(), p->defl_partial, h.size() * sizeof(double),
                      cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return NRSENSE_ERR_CUDA;
  for (int c = 0; c < 2 * k; ++c) {
    double acc = 0.0;
    for (int b = 0; b < kDeflBlocks; ++b) acc += h[size_t(c) * kDeflBlocks + b];
    out[c] = acc;
  }
  return NRSENSE_OK;
}

// Buffers for a space of k vectors (W itself is filled by the caller).
nrsense_status defl_alloc(nrsense_plan_s* p, int k) {
  defl_release(p);
  const size_t vb = size_t(p->geo.nvox) * sizeof(nrsense_c64);
  if (cudaMalloc(&p->defl_w, k * vb) != cudaSuccess ||
      cudaMalloc(&p->defl_e0w, k * vb) != cudaSuccess ||
      cudaMalloc(&p->defl_ew, k * vb) != cudaSuccess ||
      cudaMalloc(&p->defl_ecinv, size_t(2) * k * k * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&p->defl_coef, size_t(2) * k * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&p->defl_partial, size_t(2) * k * kDeflBlocks * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    defl_release(p);
    return NRSENSE_ERR_OOM;
  }
  p->defl_k = k;
  return NRSENSE_OK;
}

// W orthonormalised in place by modified Gram-Schmidt (twice per vector,
// FP64 inner products, FP32 vectors); a vector with less than 1 % of its norm
// outside the span of the kept ones (a repeated Ritz vector of a long run) is
// dropped.  The kept vectors move to the front; p->defl_k becomes their count.
nrsense_status defl_orthonormalize(nrsense_plan_s* p, cudaStream_t s) {
  const int k = p->defl_k;
  const long long n = p->geo.nvox;
  int kept = 0;
  std::vector<double> c(size_t(2) * k);
  double nn[2];
  for (int i = 0; i < k; ++i) {
    nrsense_c64* wi = p->defl_w + i * n;
    NRS_TRY(defl_dots_host(p, wi, 1, wi, s, nn));
    const double n0 = std::sqrt(std::max(nn[0], 0.0));
    if (!(n0 > 0.0) || !std::isfinite(n0)) continue;
    for (int pass = 0; pass < 2 && kept > 0; ++pass) {
      NRS_TRY(defl_dots_host(p, p->defl_w, kept, wi, s, c.data()));
      if (cudaMemcpyAsync(p->defl_coef, c.data(), size_t(2) * kept * sizeof(double),
                          cudaMemcpyHostToDevice, s) != cudaSuccess)
        return NRSENSE_ERR_CUDA;
      defl_update_kernel<<<kRedBlocks, kRedThreads, 0, s>>>(
          reinterpret_cast<float2*>(wi), reinterpret_cast<const float2*>(wi),
          reinterpret_cast<const float2*>(p->defl_w), p->defl_coef, kept, n, nullptr, nullptr);
      p->launches += 1;
    }
    NRS_TRY(defl_dots_host(p, wi, 1, wi, s, nn));
    const double n1 = std::sqrt(std::max(nn[0], 0.0));
    if (!(n1 >= 1e-2 * n0)) continue;
    defl_scale_kernel<<<kRedBlocks, kRedThreads, 0, s>>>(
        reinterpret_cast<float2*>(p->defl_w + kept * n), reinterpret_cast<const float2*>(wi),
        float(1.0 / n1), n);
    p->launches += 1;
    NRS_TRY(launched());
    ++kept;
  }
  if (cudaStreamSynchronize(s) != cudaSuccess) return NRSENSE_ERR_CUDA;
  p->defl_k = kept;
  p->epoch += 1;  // the count of basis vectors is a launch parameter
  return NRSENSE_OK;
}

// With W in place: W orthonormalised, E0 W (one normal-operator application
// per kept vector, lambda = 0) and the Gram matrices W^H E0 W, W^H W (host,
// FP64).  ERR_BREAKDOWN when no vector is kept.
nrsense_status defl_install(nrsense_plan_s* p, cudaStream_t s) {
  NRS_TRY(defl_orthonormalize(p, s));
  if (p->defl_k == 0) return NRSENSE_ERR_BREAKDOWN;
  const int k = p->defl_k;
  const long long n = p->geo.nvox;
  for (int i = 0; i < k; ++i)
    NRS_TRY(nrsense_apply_normal(p, p->defl_w + i * n, 0.0, p->defl_e0w + i * n, s));
  p->defl_g0.assign(size_t(2) * k * k, 0.0);
  p->defl_gw.assign(size_t(2) * k * k, 0.0);
  std::vector<double> col(size_t(2) * k);
  for (int j = 0; j < k; ++j) {
    NRS_TRY(defl_dots_host(p, p->defl_w, k, p->defl_e0w + j * n, s, col.data()));
    for (int i = 0; i < k; ++i) {
      p->defl_g0[2 * (i * k + j)] = col[2 * i];
      p->defl_g0[2 * (i * k + j) + 1] = col[2 * i + 1];
    }
    NRS_TRY(defl_dots_host(p, p->defl_w, k, p->defl_w + j * n, s, col.data()));
    for (int i = 0; i < k; ++i) {
      p->defl_gw[2 * (i * k + j)] = col[2 * i];
      p->defl_gw[2 * (i * k + j) + 1] = col[2 * i + 1];
    }
  }
  p->defl_lambda = -1.0;
  return NRSENSE_OK;
}

// E W = E0 W + lambda W and E_c^-1 = (W^H E0 W + lambda W^H W)^-1 for this
// lambda (kept until lambda changes).  Synchronises s.
nrsense_status defl_prepare(nrsense_plan_s* p, double lambda, cudaStream_t s) {
  if (p->defl_lambda == lambda) return NRSENSE_OK;
  const int k = p->defl_k;
  const long long total = (long long)k * p->geo.nvox;
  defl_form_ew_kernel<<<kRedBlocks, kRedThreads, 0, s>>>(
      reinterpret_cast<float2*>(p->defl_ew), reinterpret_cast<const float2*>(p->defl_e0w),
      reinterpret_cast<const float2*>(p->defl_w), float(lambda), total);
  p->launches += 1;
  NRS_TRY(launched());
  std::vector<double> ec(p->defl_g0);
  for (size_t i = 0; i < ec.size(); ++i) ec[i] += lambda * p->defl_gw[i];
  if (pinv_hermitian(ec, k) == 0) return NRSENSE_ERR_BREAKDOWN;
  if (cudaMemcpyAsync(p->defl_ecinv, ec.data(), ec.size() * sizeof(double),
                      cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return NRSENSE_ERR_CUDA;
  p->defl_lambda = lambda;
  return NRSENSE_OK;
}

// out = P^T in = in - W E_c^-1 (E W)^H in (out may equal in)
nrsense_status defl_project(nrsense_plan_s* p, const nrsense_c64* in, nrsense_c64* out,
                            cudaStream_t s) {
  StageMark m(p, NRSENSE_STAGE_SOLVER, s);
  defl_dots(p, p->defl_ew, p->defl_k, in, s);
  defl_coef_kernel<<<1, kRedThreads, 0, s>>>(p->defl_partial, kDeflBlocks, p->defl_k,
                                             p->defl_ecinv, p->defl_coef);
  defl_update_kernel<<<kRedBlocks, kRedThreads, 0, s>>>(
      reinterpret_cast<float2*>(out), reinterpret_cast<const float2*>(in),
      reinterpret_cast<const float2*>(p->defl_w), p->defl_coef, p->defl_k, p->geo.nvox, nullptr,
      nullptr);
  p->launches += 2;
  return launched();
}

// start: c = E_c^-1 W^H r, x += W c, r -= (E W) c
nrsense_status defl_start(nrsense_plan_s* p, nrsense_c64* x, nrsense_c64* r, cudaStream_t s) {
  StageMark m(p, NRSENSE_STAGE_SOLVER, s);
  defl_dots(p, p->defl_w, p->defl_k, r, s);
  defl_coef_kernel<<<1, kRedThreads, 0, s>>>(p->defl_partial, kDeflBlocks, p->defl_k,
                                             p->defl_ecinv, p->defl_coef);
  defl_update_kernel<<<kRedBlocks, kRedThreads, 0, s>>>(
      reinterpret_cast<float2*>(r), reinterpret_cast<const float2*>(r),
      reinterpret_cast<const float2*>(p->defl_ew), p->defl_coef, p->defl_k, p->geo.nvox,
      reinterpret_cast<float2*>(x), reinterpret_cast<const float2*>(p->defl_w));
  p->launches += 2;
  return launched();
}

// z = M(r) (the network), z = M_c r (circulant), z = M(M_c r) (both) or
// z = r (neither), projected by P^T when deflating, then the flexible CG
// coefficient and direction.  start: first direction.
nrsense_status fcg_direction(nrsense_plan_s* p, nrsense_cnn_s* net, bool circ, bool defl,
                             bool start, cudaStream_t s) {
  nrsense_cg_ws* w = p->cg;
  const long long n = p->geo.nvox;
  const float2* r = reinterpret_cast<const float2*>(w->r);
  const float2* z = r;
  const double* sumsq = &w->st->rr;  // |r|^2 of the network input, when it is r
  if (circ) {
    NRS_TRY(circ_apply(p, w->r, w->zc, s));
    z = reinterpret_cast<const float2*>(w->zc);
    sumsq = nullptr;
  }
  if (net) {
    StageMark m(p, NRSENSE_STAGE_CNN, s);
    p->launches += cnn_apply_async(net, z, sumsq, reinterpret_cast<float2*>(w->z), s);
    z = reinterpret_cast<const float2*>(w->z);
  }
  if (defl) {
    // project in place, or into the network buffer when z is the residual
    nrsense_c64* dst = z == r ? w->z : reinterpret_cast<nrsense_c64*>(const_cast<float2*>(z));
    NRS_TRY(defl_project(p, reinterpret_cast<const nrsense_c64*>(z), dst, s));
    z = reinterpret_cast<const float2*>(dst);
  }
  StageMark m(p, NRSENSE_STAGE_SOLVER, s);
  dot2_partial_kernel<<<kRedBlocks, kRedThreads, 0, s>>>(
      z, r, start ? nullptr : reinterpret_cast<const float2*>(w->Ep), n, w->partial);
  fcg_beta_kernel<<<1, kRedThreads, 0, s>>>(w->partial, kRedBlocks, w->st, start ? 1 : 0);
  fcg_update_p_kernel<<<kRedBlocks, kRedThreads, 0, s>>>(z, r, reinterpret_cast<float2*>(w->p), n,
                                                         w->st, start ? 1 : 0);
  p->launches += 3;
  return launched();
}

// One CG (net == nullptr, flexible == false) or flexible CG iteration on
// stream s, without host synchronisation.
nrsense_status cg_iteration(nrsense_plan_s* p, nrsense_c64* x, double lambda, bool flexible,
                            nrsense_cnn_s* net, bool circ, bool defl, cudaStream_t s) {
  nrsense_cg_ws* w = p->cg;
  const long long n = p->geo.nvox;
  NRS_TRY(nrsense_apply_normal(p, w->p, lambda, w->Ep, s));
  {
    StageMark m(p, NRSENSE_STAGE_SOLVER, s);
    dot_partial_kernel<<<kRedBlocks, kRedThreads, 0, s>>>(
        reinterpret_cast<const float2*>(w->p), reinterpret_cast<const float2*>(w->Ep), n,
        w->partial);
    cg_alpha_kernel<<<1, kRedThreads, 0, s>>>(w->partial, kRedBlocks, w->st, flexible ? 1 : 0);
    cg_update_xr_kernel<<<kRedBlocks, kRedThreads, 0, s>>>(
        reinterpret_cast<float2*>(x), reinterpret_cast<float2*>(w->r),
        reinterpret_cast<const float2*>(w->p), reinterpret_cast<const float2*>(w->Ep), n, w->st,
        w->partial);
    if (!flexible) {
      cg_beta_kernel<<<1, kRedThreads, 0, s>>>(w->partial, kRedBlocks, w->st, w->hist);
      cg_update_p_kernel<<<kRedBlocks, kRedThreads, 0, s>>>(reinterpret_cast<const float2*>(w->r),
                                                            reinterpret_cast<float2*>(w->p), n,
                                                            w->st);
    } else {
      fcg_check_kernel<<<1, kRedThreads, 0, s>>>(w->partial, kRedBlocks, w->st, w->hist);
    }
    p->launches += 5;
  }
  if (flexible) NRS_TRY(fcg_direction(p, net, circ, defl, false, s));
  return launched();
}

nrsense_status read_state(nrsense_plan_s* p, cudaStream_t s, CgState* h) {
  if (cudaMemcpyAsync(h, p->cg->st, sizeof(*h), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return NRSENSE_ERR_CUDA;
  return NRSENSE_OK;
}

struct Record {
  nrsense_c64* r;   // capacity x N^3
  nrsense_c64* e;   // capacity x N^3
  int capacity;
  int count;
};

struct SolveOut {
  int32_t* iters;
  double* res_hist;
  double* true_res;
  int32_t* fallbacks;
};

nrsense_status solve_impl(nrsense_plan_s* p, bool flexible, nrsense_cnn_s* net,
                          const nrsense_c64* y, double lambda, double tol, int32_t maxit,
                          uint32_t flags, nrsense_c64* x, const SolveOut& out, Record* rec,
                          cudaStream_t us) {
  const bool circ = flexible && (flags & NRSENSE_CG_CIRCULANT) != 0;
  const bool defl = flexible && (flags & NRSENSE_CG_DEFLATE) != 0;
  if (circ && !p->circ_on) return NRSENSE_ERR_STATE;
  if (defl && p->defl_k == 0) return NRSENSE_ERR_STATE;
  NRS_TRY(cg_workspace(p, maxit, flexible, circ));
  nrsense_cg_ws* w = p->cg;
  const long long n = p->geo.nvox;
  const size_t vb = size_t(n) * sizeof(nrsense_c64);
  // run everything on the plan's own stream, ordered after the caller's work
  cudaStream_t s = w->cs;
  if (cudaEventRecord(w->ev0, us) != cudaSuccess || cudaStreamWaitEvent(s, w->ev0, 0) != cudaSuccess)
    return NRSENSE_ERR_CUDA;
  if (defl) NRS_TRY(defl_prepare(p, lambda, s));

  // b = sum_j A_j^H y_j;  r = b - E x0 (or b);  p = r (or z = M(r))
  NRS_TRY(nrsense_apply_adjoint(p, y, w->b, s));
  const bool use_x0 = (flags & NRSENSE_CG_X0) != 0;
  {
    StageMark m(p, NRSENSE_STAGE_SOLVER, s);
    dot_partial_kernel<<<kRedBlocks, kRedThreads, 0, s>>>(reinterpret_cast<const float2*>(w->b),
                                                          reinterpret_cast<const float2*>(w->b), n,
                                                          w->partial);
    p->launches += 1;
  }
  if (cudaMemcpyAsync(w->r, w->b, vb, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return NRSENSE_ERR_CUDA;
  if (use_x0) {
    NRS_TRY(nrsense_apply_normal(p, x, lambda, w->Ep, s));
    StageMark m(p, NRSENSE_STAGE_SOLVER, s);
    sub_kernel<<<kRedBlocks, kRedThreads, 0, s>>>(reinterpret_cast<float2*>(w->r),
                                                  reinterpret_cast<const float2*>(w->Ep), n);
    dot_partial_kernel<<<kRedBlocks, kRedThreads, 0, s>>>(
        reinterpret_cast<const float2*>(w->r), reinterpret_cast<const float2*>(w->r), n,
        w->partial + kRedBlocks);
    p->launches += 2;
  } else {
    if (cudaMemsetAsync(x, 0, vb, s) != cudaSuccess) return NRSENSE_ERR_CUDA;
  }
  if (defl) {
    // x += W E_c^-1 W^H r, r -= E W E_c^-1 W^H r; then |r|^2 of the result
    NRS_TRY(defl_start(p, x, w->r, s));
    StageMark m(p, NRSENSE_STAGE_SOLVER, s);
    dot_partial_kernel<<<kRedBlocks, kRedThreads, 0, s>>>(
        reinterpret_cast<const float2*>(w->r), reinterpret_cast<const float2*>(w->r), n,
        w->partial + kRedBlocks);
    p->launches += 1;
  }
  cg_init_kernel<<<1, kRedThreads, 0, s>>>(
      w->partial, (use_x0 || defl) ? w->partial + kRedBlocks : nullptr, kRedBlocks, tol, maxit,
      w->st, w->hist);
  p->launches += 1;
  NRS_TRY(launched());
  if (flexible) {
    NRS_TRY(fcg_direction(p, net, circ, defl, true, s));
  } else if (cudaMemcpyAsync(w->p, w->r, vb, cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
    return NRSENSE_ERR_CUDA;
  }

  // iterations, in chunks; the converged flag is read between chunks
  const bool graph = (flags & NRSENSE_CG_GRAPH) != 0;
  // graph chunks: a fixed-count solve (tol == 0) is one graph of up to kGraphMax
  // iterations; a tolerance-driven solve replays 2-iteration graphs and reads
  // the converged flag between them (an iteration after convergence changes
  // nothing but still applies the operator, so short chunks waste at most one)
  const int chunk = rec ? 1
                  : graph ? std::max(1, std::min<int>(maxit, tol == 0.0 ? kGraphMax : 2))
                          : 5;
  const int mode = (flexible ? (circ ? 2 : 1) : 0) + (defl ? 4 : 0);
  const uint64_t gnet = cnn_serial(net);
  if (graph && (w->gexec == nullptr || w->g_x != x || w->g_lambda != lambda ||
                w->g_chunk != chunk || w->g_mode != mode || w->g_net != gnet ||
                w->g_epoch != p->epoch)) {
    if (w->gexec) {
      cudaGraphExecDestroy(w->gexec);
      w->gexec = nullptr;
    }
    cudaGraph_t gph = nullptr;
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed) != cudaSuccess)
      return NRSENSE_ERR_CUDA;
    nrsense_status cst = NRSENSE_OK;
    for (int k = 0; k < chunk && cst == NRSENSE_OK; ++k)
      cst = cg_iteration(p, x, lambda, flexible, net, circ, defl, s);
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
    w->g_lambda = lambda;
    w->g_chunk = chunk;
    w->g_mode = mode;
    w->g_net = gnet;
    w->g_epoch = p->epoch;
  }
  CgState h;
  for (int it = 0; it < maxit; it += chunk) {
    NRS_TRY(read_state(p, s, &h));
    if (h.done) break;
    if (rec && rec->count < rec->capacity) {
      // iterate k = it before the update: (r_k, x_k); x_k becomes x* - x_k at exit
      const size_t off = size_t(rec->count) * size_t(n);
      if (cudaMemcpyAsync(rec->r + off, w->r, vb, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
          cudaMemcpyAsync(rec->e + off, x, vb, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return NRSENSE_ERR_CUDA;
      rec->count += 1;
    }
    if (graph) {
      if (cudaGraphLaunch(w->gexec, s) != cudaSuccess) return NRSENSE_ERR_CUDA;
      p->launches += 5LL * chunk;  // approximate: kernels of the captured operator not recounted
    } else {
      for (int k = 0; k < chunk && it + k < maxit; ++k)
        NRS_TRY(cg_iteration(p, x, lambda, flexible, net, circ, defl, s));
    }
  }
  if (rec) {
    for (int k = 0; k < rec->count; ++k)
      rsub_kernel<<<kRedBlocks, kRedThreads, 0, s>>>(
          reinterpret_cast<const float2*>(x),
          reinterpret_cast<float2*>(rec->e + size_t(k) * size_t(n)), n);
    p->launches += rec->count;
    NRS_TRY(launched());
  }

  NRS_TRY(read_state(p, s, &h));
  if (out.iters) *out.iters = h.iter;
  if (out.fallbacks) *out.fallbacks = h.n_fb;
  if (out.res_hist && h.iter + 1 > 0 &&
      cudaMemcpy(out.res_hist, w->hist, size_t(h.iter + 1) * sizeof(double),
                 cudaMemcpyDeviceToHost) != cudaSuccess)
    return NRSENSE_ERR_CUDA;
  if (out.true_res) {
    // true residual ||b - E x|| / ||b||, recomputed once
    NRS_TRY(nrsense_apply_normal(p, x, lambda, w->Ep, s));
    sub_kernel<<<kRedBlocks, kRedThreads, 0, s>>>(reinterpret_cast<float2*>(w->b),
                                                  reinterpret_cast<const float2*>(w->Ep), n);
    dot_partial_kernel<<<kRedBlocks, kRedThreads, 0, s>>>(
        reinterpret_cast<const float2*>(w->b), reinterpret_cast<const float2*>(w->b), n,
        w->partial);
    p->launches += 2;
    double* hp = new double[kRedBlocks];
    const bool ok = cudaMemcpyAsync(hp, w->partial, kRedBlocks * sizeof(double),
                                    cudaMemcpyDeviceToHost, s) == cudaSuccess &&
                    cudaStreamSynchronize(s) == cudaSuccess;
    double acc = 0.0;
    for (int i = 0; i < kRedBlocks; ++i) acc += hp[i];
    delete[] hp;
    if (!ok) return NRSENSE_ERR_CUDA;
    *out.true_res = h.bb > 0.0 ? std::sqrt(acc / h.bb) : 0.0;
  }
  // order the caller's stream after the solve
  if (cudaEventRecord(w->ev1, s) != cudaSuccess || cudaStreamWaitEvent(us, w->ev1, 0) != cudaSuccess)
    return NRSENSE_ERR_CUDA;
  if (h.status != NRSENSE_OK) return h.status;
  if (h.rr > h.tol2 && h.bb > 0.0) return NRSENSE_ERR_NOT_CONVERGED;
  return NRSENSE_OK;
}

bool solve_args_ok(nrsense_plan_t p, const nrsense_c64* y, nrsense_c64* x, double lambda,
                   double tol, int32_t maxit) {
  return p != nullptr && y != nullptr && x != nullptr && maxit >= 0 && maxit <= (1 << 20) &&
         tol >= 0.0 && lambda >= 0.0 && std::isfinite(tol) && std::isfinite(lambda);
}

}  // namespace

extern "C" {

nrsense_status nrsense_solve_cg(nrsense_plan_t p, const nrsense_c64* y, double lambda, double tol,
                                int32_t maxit, uint32_t flags, nrsense_c64* x, int32_t* iters,
                                double* res_hist, double* true_res, void* stream) {
  if (!solve_args_ok(p, y, x, lambda, tol, maxit)) return NRSENSE_ERR_ARG;
  if (flags & (NRSENSE_CG_CIRCULANT | NRSENSE_CG_DEFLATE)) return NRSENSE_ERR_ARG;
  const SolveOut out{iters, res_hist, true_res, nullptr};
  return solve_impl(p, false, nullptr, y, lambda, tol, maxit, flags, x, out, nullptr,
                    static_cast<cudaStream_t>(stream));
}

nrsense_status nrsense_solve_cg_record(nrsense_plan_t p, const nrsense_c64* y, double lambda,
                                       double tol, int32_t maxit, uint32_t flags, nrsense_c64* x,
                                       int32_t* iters, double* res_hist, double* true_res,
                                       nrsense_c64* rec_r, nrsense_c64* rec_e, int32_t capacity,
                                       int32_t* rec_count, void* stream) {
  if (!solve_args_ok(p, y, x, lambda, tol, maxit) ||
      (flags & (NRSENSE_CG_GRAPH | NRSENSE_CG_CIRCULANT | NRSENSE_CG_DEFLATE)) || capacity < 0 ||
      (capacity > 0 && (rec_r == nullptr || rec_e == nullptr)) || rec_count == nullptr)
    return NRSENSE_ERR_ARG;
  Record rec{rec_r, rec_e, capacity, 0};
  const SolveOut out{iters, res_hist, true_res, nullptr};
  const nrsense_status st = solve_impl(p, false, nullptr, y, lambda, tol, maxit, flags, x, out,
                                       &rec, static_cast<cudaStream_t>(stream));
  *rec_count = rec.count;
  return st;
}

nrsense_status nrsense_solve_fcg(nrsense_plan_t p, nrsense_cnn_t net, const nrsense_c64* y,
                                 double lambda, double tol, int32_t maxit, uint32_t flags,
                                 nrsense_c64* x, int32_t* iters, double* res_hist,
                                 double* true_res, int32_t* fallbacks, void* stream) {
  if (!solve_args_ok(p, y, x, lambda, tol, maxit)) return NRSENSE_ERR_ARG;
  if (net && !cnn_shape_matches(net, p->geo.n0, p->geo.n1, p->geo.n2)) return NRSENSE_ERR_ARG;
  const SolveOut out{iters, res_hist, true_res, fallbacks};
  return solve_impl(p, true, net, y, lambda, tol, maxit, flags, x, out, nullptr,
                    static_cast<cudaStream_t>(stream));
}

nrsense_status nrsense_set_circulant(nrsense_plan_t p, double lambda, int32_t enable,
                                     void* stream) {
  if (p == nullptr || !(lambda >= 0.0) || !std::isfinite(lambda)) return NRSENSE_ERR_ARG;
  if (!enable) {
    p->circ_on = false;
    return NRSENSE_OK;
  }
  const Geo& g = p->geo;
  const long long n = g.nvox;
  const size_t vb = size_t(n) * sizeof(nrsense_c64);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (!p->circ_d) {
    if (cudaMalloc(&p->circ_d, size_t(n) * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&p->circ_tmp, vb) != cudaSuccess) {
      cudaGetLastError();
      cudaFree(p->circ_d);
      cudaFree(p->circ_tmp);
      p->circ_d = nullptr;
      p->circ_tmp = nullptr;
      return NRSENSE_ERR_OOM;
    }
  }
  if (!p->have_fft_circ) {
    if (cufftPlan3d(&p->fft_circ, g.n0, g.n1, g.n2, CUFFT_C2C) != CUFFT_SUCCESS)
      return NRSENSE_ERR_CUFFT;
    p->have_fft_circ = true;
  }
  // h = E0 delta at the image centre, hhat = DFT(h), d from hhat
  nrsense_c64* h = nullptr;
  if (cudaMalloc(&h, vb) != cudaSuccess) {
    cudaGetLastError();
    return NRSENSE_ERR_OOM;
  }
  nrsense_status st = NRSENSE_OK;
  const long long centre = ((long long)(g.n0 / 2) * g.n1 + g.n1 / 2) * g.n2 + g.n2 / 2;
  if (cudaMemsetAsync(p->circ_tmp, 0, vb, s) != cudaSuccess) st = NRSENSE_ERR_CUDA;
  if (st == NRSENSE_OK) {
    impulse_kernel<<<1, 1, 0, s>>>(reinterpret_cast<float2*>(p->circ_tmp), centre);
    p->launches += 1;
    st = launched();
  }
  if (st == NRSENSE_OK) st = nrsense_apply_normal(p, p->circ_tmp, 0.0, h, s);
  if (st == NRSENSE_OK &&
      (cufftSetStream(p->fft_circ, s) != CUFFT_SUCCESS ||
       cufftExecC2C(p->fft_circ, reinterpret_cast<cufftComplex*>(h),
                    reinterpret_cast<cufftComplex*>(p->circ_tmp), CUFFT_FORWARD) != CUFFT_SUCCESS))
    st = NRSENSE_ERR_CUFFT;
  if (st == NRSENSE_OK) {
    circ_diag_kernel<<<kRedBlocks, kRedThreads, 0, s>>>(reinterpret_cast<const float2*>(p->circ_tmp),
                                                        p->circ_d, g.n0, g.n1, g.n2,
                                                        float(lambda));
    p->launches += 1;
    st = launched();
  }
  if (cudaStreamSynchronize(s) != cudaSuccess && st == NRSENSE_OK) st = NRSENSE_ERR_CUDA;
  cudaFree(h);
  p->circ_on = st == NRSENSE_OK;
  return st;
}

nrsense_status nrsense_apply_circulant(nrsense_plan_t p, const nrsense_c64* r, nrsense_c64* z,
                                       void* stream) {
  if (p == nullptr || r == nullptr || z == nullptr) return NRSENSE_ERR_ARG;
  if (!p->circ_on) return NRSENSE_ERR_STATE;
  return circ_apply(p, r, z, static_cast<cudaStream_t>(stream));
}

nrsense_status nrsense_set_deflation(nrsense_plan_t p, const nrsense_c64* w, int32_t k,
                                     int32_t* kept, void* stream) {
  if (kept) *kept = 0;
  if (p == nullptr || k < 0 || k > kDeflMax || (k > 0 && w == nullptr)) return NRSENSE_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (k == 0) {
    if (cudaStreamSynchronize(s) != cudaSuccess) return NRSENSE_ERR_CUDA;
    defl_release(p);
    return NRSENSE_OK;
  }
  NRS_TRY(defl_alloc(p, k));
  const size_t vb = size_t(p->geo.nvox) * sizeof(nrsense_c64);
  if (cudaMemcpyAsync(p->defl_w, w, k * vb, cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
    defl_release(p);
    return NRSENSE_ERR_CUDA;
  }
  const nrsense_status st = defl_install(p, s);
  if (st != NRSENSE_OK) {
    defl_release(p);
    return st;
  }
  if (kept) *kept = p->defl_k;
  return NRSENSE_OK;
}

nrsense_status nrsense_deflation_from_solve(nrsense_plan_t p, const nrsense_c64* y, double lambda,
                                            int32_t steps, int32_t k, uint32_t flags,
                                            double* ritz, int32_t* kept, void* stream) {
  if (kept) *kept = 0;
  if (p == nullptr || y == nullptr || !(lambda >= 0.0) || !std::isfinite(lambda) || steps < 1 ||
      steps > 256 || k < 1 || k > std::min<int>(steps, kDeflMax) ||
      (flags & ~(NRSENSE_CG_CIRCULANT | NRSENSE_DEFLATE_LARGEST)) != 0)
    return NRSENSE_ERR_ARG;
  const bool largest = (flags & NRSENSE_DEFLATE_LARGEST) != 0;
  const bool circ = (flags & NRSENSE_CG_CIRCULANT) != 0;
  if (circ && !p->circ_on) return NRSENSE_ERR_STATE;
  NRS_TRY(cg_workspace(p, steps + 1, true, circ));
  nrsense_cg_ws* w = p->cg;
  const long long n = p->geo.nvox;
  const size_t vb = size_t(n) * sizeof(nrsense_c64);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // scratch: the iterate, the recorded preconditioned residuals, coefficients
  struct Scratch {
    nrsense_c64* x = nullptr;
    nrsense_c64* Z = nullptr;
    float* coef = nullptr;
    ~Scratch() {
      cudaFree(x);
      cudaFree(Z);
      cudaFree(coef);
    }
  } sc;
  if (cudaMalloc(&sc.x, vb) != cudaSuccess || cudaMalloc(&sc.Z, size_t(steps) * vb) != cudaSuccess ||
      cudaMalloc(&sc.coef, size_t(steps) * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    return NRSENSE_ERR_OOM;
  }
  // b = sum_j A_j^H y_j, r = b, x = 0; run past `steps` so that rho_steps is formed
  NRS_TRY(nrsense_apply_adjoint(p, y, w->b, s));
  dot_partial_kernel<<<kRedBlocks, kRedThreads, 0, s>>>(reinterpret_cast<const float2*>(w->b),
                                                        reinterpret_cast<const float2*>(w->b), n,
                                                        w->partial);
  p->launches += 1;
  if (cudaMemcpyAsync(w->r, w->b, vb, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
      cudaMemsetAsync(sc.x, 0, vb, s) != cudaSuccess)
    return NRSENSE_ERR_CUDA;
  cg_init_kernel<<<1, kRedThreads, 0, s>>>(w->partial, nullptr, kRedBlocks, 0.0, steps + 1, w->st,
                                           w->hist);
  p->launches += 1;
  NRS_TRY(launched());
  NRS_TRY(fcg_direction(p, nullptr, circ, false, true, s));
  CgState h;
  NRS_TRY(read_state(p, s, &h));
  std::vector<double> alpha, rho{h.rz};
  int m = 0;
  const nrsense_c64* zsrc = circ ? w->zc : w->r;
  for (int j = 0; j < steps && !h.done; ++j) {
    if (cudaMemcpyAsync(sc.Z + size_t(j) * n, zsrc, vb, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
      return NRSENSE_ERR_CUDA;
    NRS_TRY(cg_iteration(p, sc.x, lambda, true, nullptr, circ, false, s));
    NRS_TRY(read_state(p, s, &h));
    if (h.status != NRSENSE_OK || h.n_fb != 0) return NRSENSE_ERR_BREAKDOWN;
    alpha.push_back(h.alpha);
    if (h.done) break;  // exact convergence: rho_{j+1} is not formed
    rho.push_back(h.rz);
    m = j + 1;
  }
  if (m < 1) return NRSENSE_ERR_BREAKDOWN;
  for (int j = 0; j <= m; ++j)
    if (!(rho[j] > 0.0) || !std::isfinite(rho[j])) return NRSENSE_ERR_BREAKDOWN;
  // the CG-Lanczos tridiagonal for v_j = z_j / sqrt(rho_j), its eigenpairs
  std::vector<double> T(size_t(m) * m, 0.0), vals(m), vecs(size_t(m) * m);
  for (int j = 0; j < m; ++j) {
    T[size_t(j) * m + j] = 1.0 / alpha[j] + (j > 0 ? (rho[j] / rho[j - 1]) / alpha[j - 1] : 0.0);
    if (j + 1 < m)
      T[size_t(j) * m + j + 1] = T[size_t(j + 1) * m + j] =
          -std::sqrt(rho[j + 1] / rho[j]) / alpha[j];
  }
  symmetric_eigen_sorted(m, T.data(), vals.data(), vecs.data());
  const int kk = std::min<int>(k, m);
  NRS_TRY(defl_alloc(p, kk));
  std::vector<float> c(m);
  // the Ritz pair taken i-th: ascending from the smallest, or descending
  // from the largest
  auto pick = [&](int i) { return largest ? m - 1 - i : i; };
  for (int i = 0; i < kk; ++i) {
    const int e = pick(i);
    for (int j = 0; j < m; ++j) c[j] = float(vecs[size_t(j) * m + e] / std::sqrt(rho[j]));
    if (cudaMemcpyAsync(sc.coef, c.data(), m * sizeof(float), cudaMemcpyHostToDevice, s) !=
        cudaSuccess) {
      defl_release(p);
      return NRSENSE_ERR_CUDA;
    }
    defl_combine_kernel<<<kRedBlocks, kRedThreads, 0, s>>>(
        reinterpret_cast<float2*>(p->defl_w + size_t(i) * n),
        reinterpret_cast<const float2*>(sc.Z), sc.coef, m, n);
    p->launches += 1;
    // c is rewritten for the next vector: wait for this copy to be consumed
    if (cudaStreamSynchronize(s) != cudaSuccess) {
      defl_release(p);
      return NRSENSE_ERR_CUDA;
    }
  }
  const nrsense_status st = defl_install(p, s);
  if (st != NRSENSE_OK) {
    defl_release(p);
    return st;
  }
  if (ritz)
    for (int i = 0; i < k; ++i) ritz[i] = i < kk ? vals[pick(i)] : std::nan("");
  if (kept) *kept = p->defl_k;
  return NRSENSE_OK;
}

nrsense_status nrsense_symmetric_eigen(int32_t m, const double* a, double* vals, double* vecs) {
  if (m < 1 || m > 256 || a == nullptr || vals == nullptr || vecs == nullptr)
    return NRSENSE_ERR_ARG;
  symmetric_eigen_sorted(m, a, vals, vecs);
  return NRSENSE_OK;
}

}  // extern "C"
