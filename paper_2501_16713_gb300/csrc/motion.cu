// Motion capture for segmented acquisitions (section "Motion Capturing for
// Segmented Data Acquisitions"; phase binning in "Nonrigid Respiratory
// Motion Correction").
//
// Every heartbeat acquires a full low-resolution trajectory whose direct
// gridding reconstruction from density-corrected data is that heartbeat's
// 3D iNAV; bulk translation comes from correlations between a reference iNAV
// and the others and is removed by linear phase shifts of the k-space data;
// k-means on the translations gives the respiratory phases, the cluster with
// the least variance being the reference.  This file holds:
//   * Pipe-Menon density compensation w <- w / (B P w) on the plan's own
//     k-space point sets (P: spread onto the oversampled grid with the
//     gridding kernel, B: interpolation back), one channel, FP32 grids;
//   * the density-weighted adjoint (gridding reconstruction) A^H (w . y);
//   * translation by circular cross-correlation of magnitude images (cuFFT
//     real transforms, batched over heartbeats), integer argmax (first index
//     on ties) refined per axis by a three-point parabola;
//   * the phase-ramp correction y <- y exp(+i omega . t) per row segment;
//   * k-means (Lloyd) on the host, started from the points at quantile
//     positions along the first principal axis.
#include <cufft.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include "plan_internal.h"

using namespace nrs;

namespace {

constexpr int kThreads = 256;
constexpr int kBlocks = 1184;

#define NRS_TRY(expr)                  \
  do {                                 \
    nrsense_status _st = (expr);       \
    if (_st != NRSENSE_OK) return _st; \
  } while (0)

nrsense_status launched() {
  return cudaGetLastError() == cudaSuccess ? NRSENSE_OK : NRSENSE_ERR_CUDA;
}

// v = (w, 0)
__global__ void to_complex_kernel(const float* __restrict__ w, float2* __restrict__ v, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    v[i] = make_float2(w[i], 0.0f);
}

__global__ void fill_kernel(float* __restrict__ w, float v, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    w[i] = v;
}

// w = w / Re(s)
__global__ void dcf_update_kernel(float* __restrict__ w, const float2* __restrict__ s, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    w[i] = w[i] / s[i].x;
}

// out[r][c] = w[r] y[r][c]
__global__ void scale_rows_kernel(const float2* __restrict__ y, const float* __restrict__ w,
                                  float2* __restrict__ out, long long rows, int C) {
  const long long n = rows * C;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float a = w[i / C];
    const float2 v = y[i];
    out[i] = make_float2(a * v.x, a * v.y);
  }
}

__global__ void magnitude_kernel(const float2* __restrict__ z, float* __restrict__ m, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float2 v = z[i];
    m[i] = sqrtf(v.x * v.x + v.y * v.y);
  }
}

// spec[1 + b][i] *= conj(spec[0][i]) for b < count
__global__ void cross_spectrum_kernel(cufftComplex* __restrict__ spec, long long per, int count) {
  const long long n = per * count;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const cufftComplex r = spec[i % per];
    const cufftComplex a = spec[per + i];
    spec[per + i] = make_float2(a.x * r.x + a.y * r.y, a.y * r.x - a.x * r.y);
  }
}

// One CTA per image: argmax of corr (first index on ties), then the
// three-point parabola per axis and the wrap to (-n/2, n/2].
__global__ void __launch_bounds__(kThreads) peak_kernel(const float* __restrict__ corr, int n0,
                                                        int n1, int n2, double* __restrict__ shifts) {
  __shared__ float sv[kThreads];
  __shared__ long long si[kThreads];
  const long long N = (long long)n0 * n1 * n2;
  const float* c = corr + N * blockIdx.x;
  float best = -INFINITY;
  long long bi = N;
  for (long long i = threadIdx.x; i < N; i += kThreads) {
    const float v = c[i];
    if (v > best) {  // ascending i per thread: the first maximum is kept
      best = v;
      bi = i;
    }
  }
  sv[threadIdx.x] = best;
  si[threadIdx.x] = bi;
  __syncthreads();
  for (int o = kThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      const float v = sv[threadIdx.x + o];
      const long long j = si[threadIdx.x + o];
      if (v > sv[threadIdx.x] || (v == sv[threadIdx.x] && j < si[threadIdx.x])) {
        sv[threadIdx.x] = v;
        si[threadIdx.x] = j;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const long long t = si[0] < N ? si[0] : 0;
    const int n[3] = {n0, n1, n2};
    int p[3] = {int(t / ((long long)n1 * n2)), int((t / n2) % n1), int(t % n2)};
    const double c0 = c[t];
    for (int a = 0; a < 3; ++a) {
      int q[3] = {p[0], p[1], p[2]};
      q[a] = (p[a] + 1) % n[a];
      const double cp = c[((long long)q[0] * n1 + q[1]) * n2 + q[2]];
      q[a] = (p[a] - 1 + n[a]) % n[a];
      const double cm = c[((long long)q[0] * n1 + q[1]) * n2 + q[2]];
      const double den = cm - 2.0 * c0 + cp;
      const double d = den < 0.0 ? 0.5 * (cm - cp) / den : 0.0;
      double v = p[a] + d;
      if (v > 0.5 * n[a]) v -= n[a];
      shifts[3 * blockIdx.x + a] = v;
    }
  }
}

// y[r][c] *= exp(+i omega_r . t_s) for rows r of segment s.
__global__ void phase_ramp_kernel(const float* __restrict__ coords, float2* __restrict__ y,
                                  int C, const long long* __restrict__ seg_off, int nseg,
                                  const double* __restrict__ shifts) {
  const long long r0 = seg_off[0], r1 = seg_off[nseg];
  for (long long r = r0 + blockIdx.x * (long long)blockDim.x + threadIdx.x; r < r1;
       r += (long long)gridDim.x * blockDim.x) {
    int lo = 0, hi = nseg - 1;  // largest s with seg_off[s] <= r
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (seg_off[mid] <= r) lo = mid;
      else hi = mid - 1;
    }
    const double* t = shifts + 3 * lo;
    double ph = (double)coords[3 * r] * t[0] + (double)coords[3 * r + 1] * t[1] +
                (double)coords[3 * r + 2] * t[2];
    ph -= 6.283185307179586 * rint(ph * 0.15915494309189535);
    float sn, cs;
    sincosf((float)ph, &sn, &cs);
    float2* row = y + r * C;
    for (int c = 0; c < C; ++c) {
      const float2 v = row[c];
      row[c] = make_float2(v.x * cs - v.y * sn, v.x * sn + v.y * cs);
    }
  }
}

// ---- k-means (host) ---------------------------------------------------------

// Eigenvector of the largest eigenvalue of a symmetric 3 x 3 matrix (cyclic
// Jacobi rotations).
void top_eigenvector(double A[3][3], double v[3]) {
  double V[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
  for (int sweep = 0; sweep < 64; ++sweep) {
    const double off = A[0][1] * A[0][1] + A[0][2] * A[0][2] + A[1][2] * A[1][2];
    const double diag = A[0][0] * A[0][0] + A[1][1] * A[1][1] + A[2][2] * A[2][2];
    if (off <= 1e-32 * diag || off == 0.0) break;
    for (int p = 0; p < 2; ++p)
      for (int q = p + 1; q < 3; ++q) {
        if (A[p][q] == 0.0) continue;
        const double theta = (A[q][q] - A[p][p]) / (2.0 * A[p][q]);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < 3; ++k) {  // A <- A J (columns p, q)
          const double akp = A[k][p], akq = A[k][q];
          A[k][p] = c * akp - s * akq;
          A[k][q] = s * akp + c * akq;
        }
        for (int k = 0; k < 3; ++k) {  // A <- J^T A (rows p, q)
          const double apk = A[p][k], aqk = A[q][k];
          A[p][k] = c * apk - s * aqk;
          A[q][k] = s * apk + c * aqk;
        }
        for (int k = 0; k < 3; ++k) {
          const double vkp = V[k][p], vkq = V[k][q];
          V[k][p] = c * vkp - s * vkq;
          V[k][q] = s * vkp + c * vkq;
        }
      }
  }
  int best = 0;
  for (int i = 1; i < 3; ++i)
    if (A[i][i] > A[best][best]) best = i;
  for (int k = 0; k < 3; ++k) v[k] = V[k][best];
  int big = 0;  // largest-magnitude entry positive (first on ties)
  for (int k = 1; k < 3; ++k)
    if (std::fabs(v[k]) > std::fabs(v[big])) big = k;
  if (v[big] < 0)
    for (int k = 0; k < 3; ++k) v[k] = -v[k];
}

}  // namespace

// ---------------------------------------------------------------------------

struct nrsense_motion_ws {
  nrsense_c64* vals = nullptr;  // DCF: (w, 0) per sample; weighted adjoint: w . y
  nrsense_c64* out = nullptr;   // DCF: B P w per sample
  long long vals_cap = 0, out_cap = 0;
};

namespace nrs {

void motion_release(nrsense_plan_s* p) {
  nrsense_motion_ws* w = p->motion;
  if (!w) return;
  cudaFree(w->vals);
  cudaFree(w->out);
  delete w;
  p->motion = nullptr;
}

}  // namespace nrs

namespace {

nrsense_status motion_workspace(nrsense_plan_s* p, long long vals, long long out) {
  if (!p->motion) {
    p->motion = new (std::nothrow) nrsense_motion_ws();
    if (!p->motion) return NRSENSE_ERR_OOM;
  }
  nrsense_motion_ws* w = p->motion;
  if (w->vals_cap < vals) {
    cudaFree(w->vals);
    w->vals = nullptr;
    w->vals_cap = 0;
    if (cudaMalloc(&w->vals, size_t(vals) * sizeof(nrsense_c64)) != cudaSuccess) {
      cudaGetLastError();
      return NRSENSE_ERR_OOM;
    }
    w->vals_cap = vals;
  }
  if (w->out_cap < out) {
    cudaFree(w->out);
    w->out = nullptr;
    w->out_cap = 0;
    if (cudaMalloc(&w->out, size_t(out) * sizeof(nrsense_c64)) != cudaSuccess) {
      cudaGetLastError();
      return NRSENSE_ERR_OOM;
    }
    w->out_cap = out;
  }
  return NRSENSE_OK;
}

unsigned grid_for(long long n) {
  return unsigned(std::max<long long>(1, std::min<long long>(kBlocks, (n + kThreads - 1) / kThreads)));
}

}  // namespace

extern "C" {

nrsense_status nrsense_dcf(nrsense_plan_t p, int32_t phase, int32_t iters, float* w_dev,
                           void* stream) {
  if (p == nullptr || w_dev == nullptr || iters < 0 || iters > 10000) return NRSENSE_ERR_ARG;
  if (p->C == 0 || p->grid_bf16) return NRSENSE_ERR_STATE;
  if (phase < 0 || phase >= p->P) return NRSENSE_ERR_ARG;
  const long long m = p->M[phase];
  if (m == 0) return NRSENSE_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  NRS_TRY(motion_workspace(p, m, m));
  nrsense_motion_ws* w = p->motion;
  const PhaseTable ts = kspace_phase_table(p, phase, true);
  const PhaseTable ti = kspace_phase_table(p, phase, false);
  const unsigned nb = grid_for(m);
  {
    StageMark mk(p, NRSENSE_STAGE_VECTOR, s);
    fill_kernel<<<nb, kThreads, 0, s>>>(w_dev, 1.0f, m);
    p->launches += 1;
  }
  NRS_TRY(launched());
  for (int it = 0; it < iters; ++it) {
    {
      StageMark mk(p, NRSENSE_STAGE_VECTOR, s);
      to_complex_kernel<<<nb, kThreads, 0, s>>>(w_dev, reinterpret_cast<float2*>(w->vals), m);
      p->launches += 1;
    }
    {
      // P: one channel into the first coil grid (FP32, no compensation)
      StageMark mk(p, NRSENSE_STAGE_SPREAD_KSPACE, s);
      p->launches += launch_spread(p->geo, p->W, p->kc, 1, p->ktiles, ts, w->vals, p->b_xspread,
                                   false, false, kSpreadShared, p->b_scratch, p->d_status, s);
    }
    NRS_TRY(launched());
    {
      // B: interpolation from the same grid (per-value staging)
      StageMark mk(p, NRSENSE_STAGE_INTERP_KSPACE, s);
      p->launches += launch_interp_kspace(p->geo, p->W, p->kc, 1, p->ktiles, ti, p->b_xspread,
                                          false, w->out, 4, nullptr, p->d_status, s);
    }
    NRS_TRY(launched());
    {
      StageMark mk(p, NRSENSE_STAGE_VECTOR, s);
      dcf_update_kernel<<<nb, kThreads, 0, s>>>(w_dev, reinterpret_cast<const float2*>(w->out), m);
      p->launches += 1;
    }
    NRS_TRY(launched());
  }
  return NRSENSE_OK;
}

nrsense_status nrsense_apply_adjoint_weighted(nrsense_plan_t p, const nrsense_c64* y_dev,
                                              const float* w_dev, nrsense_c64* x_dev,
                                              void* stream) {
  if (p == nullptr || y_dev == nullptr || w_dev == nullptr || x_dev == nullptr)
    return NRSENSE_ERR_ARG;
  if (p->C == 0) return NRSENSE_ERR_STATE;
  long long rows = 0;
  for (int j = 0; j < p->P; ++j) rows += p->M[j];
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  NRS_TRY(motion_workspace(p, std::max(rows * p->C, 1LL), 0));
  nrsense_motion_ws* w = p->motion;
  if (rows > 0) {
    StageMark mk(p, NRSENSE_STAGE_VECTOR, s);
    scale_rows_kernel<<<grid_for(rows * p->C), kThreads, 0, s>>>(
        reinterpret_cast<const float2*>(y_dev), w_dev, reinterpret_cast<float2*>(w->vals), rows,
        p->C);
    p->launches += 1;
  }
  NRS_TRY(launched());
  return nrsense_apply_adjoint(p, w->vals, x_dev, stream);
}

nrsense_status nrsense_translation_xcorr(const nrsense_c64* ref_dev, const nrsense_c64* imgs_dev,
                                         const int32_t* n_host, int32_t count, double* shifts_host,
                                         void* stream) {
  if (ref_dev == nullptr || imgs_dev == nullptr || n_host == nullptr || shifts_host == nullptr ||
      count < 1)
    return NRSENSE_ERR_ARG;
  const int n0 = n_host[0], n1 = n_host[1], n2 = n_host[2];
  if (n0 < 2 || n1 < 2 || n2 < 2 || (long long)n0 * n1 * n2 > (1LL << 28)) return NRSENSE_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const long long N = (long long)n0 * n1 * n2;
  const long long per = (long long)n0 * n1 * (n2 / 2 + 1);
  float* mag = nullptr;
  cufftComplex* spec = nullptr;
  double* d_shifts = nullptr;
  cufftHandle fwd = 0, inv = 0;
  bool have_fwd = false, have_inv = false;
  nrsense_status st = NRSENSE_OK;
  int dims[3] = {n0, n1, n2};
  if (cudaMalloc(&mag, size_t(N) * (count + 1) * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&spec, size_t(per) * (count + 1) * sizeof(cufftComplex)) != cudaSuccess ||
      cudaMalloc(&d_shifts, size_t(count) * 3 * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    st = NRSENSE_ERR_OOM;
  }
  if (st == NRSENSE_OK) {
    have_fwd = cufftPlanMany(&fwd, 3, dims, nullptr, 1, 0, nullptr, 1, 0, CUFFT_R2C, count + 1) ==
               CUFFT_SUCCESS;
    have_inv = have_fwd && cufftPlanMany(&inv, 3, dims, nullptr, 1, 0, nullptr, 1, 0, CUFFT_C2R,
                                         count) == CUFFT_SUCCESS;
    if (!have_fwd || !have_inv || cufftSetStream(fwd, s) != CUFFT_SUCCESS ||
        cufftSetStream(inv, s) != CUFFT_SUCCESS)
      st = NRSENSE_ERR_CUFFT;
  }
  if (st == NRSENSE_OK) {
    magnitude_kernel<<<grid_for(N), kThreads, 0, s>>>(reinterpret_cast<const float2*>(ref_dev),
                                                      mag, N);
    magnitude_kernel<<<grid_for(N * count), kThreads, 0, s>>>(
        reinterpret_cast<const float2*>(imgs_dev), mag + N, N * count);
    if (cudaGetLastError() != cudaSuccess) st = NRSENSE_ERR_CUDA;
  }
  if (st == NRSENSE_OK && cufftExecR2C(fwd, mag, spec) != CUFFT_SUCCESS) st = NRSENSE_ERR_CUFFT;
  if (st == NRSENSE_OK) {
    cross_spectrum_kernel<<<grid_for(per * count), kThreads, 0, s>>>(spec, per, count);
    if (cudaGetLastError() != cudaSuccess) st = NRSENSE_ERR_CUDA;
  }
  // correlations overwrite the image magnitudes (no longer needed)
  if (st == NRSENSE_OK && cufftExecC2R(inv, spec + per, mag + N) != CUFFT_SUCCESS)
    st = NRSENSE_ERR_CUFFT;
  if (st == NRSENSE_OK) {
    peak_kernel<<<count, kThreads, 0, s>>>(mag + N, n0, n1, n2, d_shifts);
    if (cudaGetLastError() != cudaSuccess) st = NRSENSE_ERR_CUDA;
  }
  if (st == NRSENSE_OK &&
      (cudaMemcpyAsync(shifts_host, d_shifts, size_t(count) * 3 * sizeof(double),
                       cudaMemcpyDeviceToHost, s) != cudaSuccess ||
       cudaStreamSynchronize(s) != cudaSuccess))
    st = NRSENSE_ERR_CUDA;
  if (have_fwd) cufftDestroy(fwd);
  if (have_inv) cufftDestroy(inv);
  cudaStreamSynchronize(s);
  cudaFree(mag);
  cudaFree(spec);
  cudaFree(d_shifts);
  return st;
}

nrsense_status nrsense_phase_ramp(const float* coords_dev, nrsense_c64* y_dev, int64_t rows_total,
                                  int32_t n_coils, int32_t nseg, const int64_t* seg_off_host,
                                  const double* shifts_host, void* stream) {
  if (coords_dev == nullptr || y_dev == nullptr || seg_off_host == nullptr ||
      shifts_host == nullptr || n_coils < 1 || nseg < 1 || rows_total < 0)
    return NRSENSE_ERR_ARG;
  if (seg_off_host[0] < 0 || seg_off_host[nseg] > rows_total) return NRSENSE_ERR_ARG;
  for (int i = 0; i < nseg; ++i)
    if (seg_off_host[i + 1] < seg_off_host[i]) return NRSENSE_ERR_ARG;
  for (int i = 0; i < 3 * nseg; ++i)
    if (!std::isfinite(shifts_host[i])) return NRSENSE_ERR_ARG;
  const long long rows = seg_off_host[nseg] - seg_off_host[0];
  if (rows == 0) return NRSENSE_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  long long* d_off = nullptr;
  double* d_sh = nullptr;
  nrsense_status st = NRSENSE_OK;
  if (cudaMalloc(&d_off, size_t(nseg + 1) * sizeof(long long)) != cudaSuccess ||
      cudaMalloc(&d_sh, size_t(nseg) * 3 * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    st = NRSENSE_ERR_OOM;
  }
  if (st == NRSENSE_OK &&
      (cudaMemcpyAsync(d_off, seg_off_host, size_t(nseg + 1) * sizeof(long long),
                       cudaMemcpyHostToDevice, s) != cudaSuccess ||
       cudaMemcpyAsync(d_sh, shifts_host, size_t(nseg) * 3 * sizeof(double),
                       cudaMemcpyHostToDevice, s) != cudaSuccess))
    st = NRSENSE_ERR_CUDA;
  if (st == NRSENSE_OK) {
    phase_ramp_kernel<<<grid_for(rows), kThreads, 0, s>>>(
        coords_dev, reinterpret_cast<float2*>(y_dev), n_coils, d_off, nseg, d_sh);
    if (cudaGetLastError() != cudaSuccess) st = NRSENSE_ERR_CUDA;
  }
  // the segment tables live until the kernel has run
  if (cudaStreamSynchronize(s) != cudaSuccess && st == NRSENSE_OK) st = NRSENSE_ERR_CUDA;
  cudaFree(d_off);
  cudaFree(d_sh);
  return st;
}

nrsense_status nrsense_kmeans(const double* points_host, int64_t n, int32_t k, int32_t max_iter,
                              int32_t* labels_host, double* centres_host, double* inertia_host,
                              int32_t* iters_host, int32_t* reference_host) {
  if (points_host == nullptr || labels_host == nullptr || centres_host == nullptr || n < 1 ||
      k < 1 || k > n || max_iter < 1)
    return NRSENSE_ERR_ARG;
  for (int64_t i = 0; i < 3 * n; ++i)
    if (!std::isfinite(points_host[i])) return NRSENSE_ERR_ARG;
  const double* P = points_host;
  double mean[3] = {0, 0, 0};
  for (int64_t i = 0; i < n; ++i)
    for (int a = 0; a < 3; ++a) mean[a] += P[3 * i + a];
  for (int a = 0; a < 3; ++a) mean[a] /= double(n);
  double S[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  for (int64_t i = 0; i < n; ++i)
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) S[a][b] += (P[3 * i + a] - mean[a]) * (P[3 * i + b] - mean[b]);
  double v[3];
  top_eigenvector(S, v);
  std::vector<double> proj(static_cast<size_t>(n));
  for (int64_t i = 0; i < n; ++i)
    proj[size_t(i)] = (P[3 * i] - mean[0]) * v[0] + (P[3 * i + 1] - mean[1]) * v[1] +
                      (P[3 * i + 2] - mean[2]) * v[2];
  std::vector<int64_t> order(static_cast<size_t>(n));
  std::iota(order.begin(), order.end(), int64_t(0));
  std::stable_sort(order.begin(), order.end(),
                   [&](int64_t a, int64_t b) { return proj[size_t(a)] < proj[size_t(b)]; });
  std::vector<double> C(size_t(3 * k));
  for (int j = 0; j < k; ++j) {
    const int64_t idx = order[size_t(int64_t((j + 0.5) * double(n) / double(k)))];
    for (int a = 0; a < 3; ++a) C[size_t(3 * j + a)] = P[3 * idx + a];
  }
  std::vector<int32_t> lab(static_cast<size_t>(n), -1), nl(static_cast<size_t>(n));
  int it = 0;
  while (it < max_iter) {
    for (int64_t i = 0; i < n; ++i) {
      int bj = 0;
      double bd = 0.0;
      for (int j = 0; j < k; ++j) {
        double d = 0.0;
        for (int a = 0; a < 3; ++a) {
          const double e = P[3 * i + a] - C[size_t(3 * j + a)];
          d += e * e;
        }
        if (j == 0 || d < bd) {
          bd = d;
          bj = j;
        }
      }
      nl[size_t(i)] = bj;
    }
    ++it;
    if (nl == lab) break;
    lab = nl;
    std::vector<double> sum(size_t(3 * k), 0.0);
    std::vector<int64_t> cnt(size_t(k), 0);
    for (int64_t i = 0; i < n; ++i) {
      const int j = lab[size_t(i)];
      cnt[size_t(j)] += 1;
      for (int a = 0; a < 3; ++a) sum[size_t(3 * j + a)] += P[3 * i + a];
    }
    for (int j = 0; j < k; ++j)
      if (cnt[size_t(j)] > 0)
        for (int a = 0; a < 3; ++a) C[size_t(3 * j + a)] = sum[size_t(3 * j + a)] / double(cnt[size_t(j)]);
  }
  double inertia = 0.0;
  std::vector<double> var(size_t(k), 0.0);
  std::vector<int64_t> cnt(size_t(k), 0);
  for (int64_t i = 0; i < n; ++i) {
    const int j = lab[size_t(i)];
    double d = 0.0;
    for (int a = 0; a < 3; ++a) {
      const double e = P[3 * i + a] - C[size_t(3 * j + a)];
      d += e * e;
    }
    inertia += d;
    var[size_t(j)] += d;
    cnt[size_t(j)] += 1;
  }
  int ref = -1;
  double bv = 0.0;
  for (int j = 0; j < k; ++j) {
    if (cnt[size_t(j)] == 0) continue;
    const double vj = var[size_t(j)] / double(cnt[size_t(j)]);
    if (ref < 0 || vj < bv) {
      ref = j;
      bv = vj;
    }
  }
  std::memcpy(labels_host, lab.data(), size_t(n) * sizeof(int32_t));
  std::memcpy(centres_host, C.data(), size_t(3 * k) * sizeof(double));
  if (inertia_host) *inertia_host = inertia;
  if (iters_host) *iters_host = it;
  if (reference_host) *reference_host = ref;
  return NRSENSE_OK;
}

}  // extern "C"
