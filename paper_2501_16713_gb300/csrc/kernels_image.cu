// Image-space gridding kernels: the T_j half of the operator (section
// "Image-space Gridding", forward diagram F -> 1/C* -> Z -> F^H -> B_j^(i)
// and adjoint diagram P_j^(i) -> F -> Z^H -> 1/C -> F^H).  The FFTs are cuFFT
// calls issued by apply.cu; these kernels do the deapodization, zero-padding,
// cropping and the Backprojection Core B_j^(i) at displaced voxel positions.
#include "plan_internal.h"

namespace nrs {

namespace {

// FFT-order index n in [0, N) -> signed frequency k in [-N/2, N/2).
__device__ __forceinline__ int freq_of(int n, int N) { return n < (N >> 1) ? n : n - N; }

// K1: U[k mod G] = X[k] / (C3(k/G) * N^3) for k in K_N^3 (steps 1/C* and Z of
// the forward diagram; the 1/N^3 belongs to the F^H step that follows).
__global__ void deapod_pad_kernel(Geo g, const float* __restrict__ dtab,
                                  const float2* __restrict__ xhat, float2* __restrict__ upad,
                                  float scale) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= g.nvox) return;
  const int i2 = int(idx % g.n2);
  const long long r = idx / g.n2;
  const int i1 = int(r % g.n1);
  const int i0 = int(r / g.n1);
  const int k0 = freq_of(i0, g.n0), k1 = freq_of(i1, g.n1), k2 = freq_of(i2, g.n2);
  const float w = dtab[k0 + (g.n0 >> 1)] * dtab[g.n0 + k1 + (g.n1 >> 1)] *
                  dtab[g.n0 + g.n1 + k2 + (g.n2 >> 1)] * scale;
  const int p0 = k0 < 0 ? k0 + g.g0 : k0;
  const int p1 = k1 < 0 ? k1 + g.g1 : k1;
  const int p2 = k2 < 0 ? k2 + g.g2 : k2;
  const float2 v = xhat[idx];
  upad[((long long)p0 * g.g1 + p1) * g.g2 + p2] = make_float2(v.x * w, v.y * w);
}

// K4: X[k] = Ufreq[k mod G] / (C3(k/G) * N^3) for k in K_N^3 (steps Z^H and 1/C
// of the adjoint diagram; the 1/N^3 belongs to the preceding F step).
__global__ void crop_deapod_kernel(Geo g, const float* __restrict__ dtab,
                                   const float2* __restrict__ ufreq, float2* __restrict__ xhat,
                                   float scale) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= g.nvox) return;
  const int i2 = int(idx % g.n2);
  const long long r = idx / g.n2;
  const int i1 = int(r % g.n1);
  const int i0 = int(r / g.n1);
  const int k0 = freq_of(i0, g.n0), k1 = freq_of(i1, g.n1), k2 = freq_of(i2, g.n2);
  const float w = dtab[k0 + (g.n0 >> 1)] * dtab[g.n0 + k1 + (g.n1 >> 1)] *
                  dtab[g.n0 + g.n1 + k2 + (g.n2 >> 1)] * scale;
  const int p0 = k0 < 0 ? k0 + g.g0 : k0;
  const int p1 = k1 < 0 ? k1 + g.g1 : k1;
  const int p2 = k2 < 0 ? k2 + g.g2 : k2;
  const float2 v = ufreq[((long long)p0 * g.g1 + p1) * g.g2 + p2];
  xhat[idx] = make_float2(v.x * w, v.y * w);
}

// K2: m_j[n] = sum_taps c3(sigma (n + d_j[n]) - g) u[g mod G] for every phase
// (Backprojection Core B_j^(i) at the displaced voxel positions of the
// displacement-field equation).  One thread per voxel, all phases: the
// phases' taps of one voxel are close, so they share L1/L2 lines.
template <int W, bool RAT>
__global__ void __launch_bounds__(256) interp_image_kernel(Geo g, KernelCoefs kc, int P,
                                                           const float* __restrict__ disp,
                                                           const float2* __restrict__ u,
                                                           float2* __restrict__ m) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= g.nvox) return;
  const int i2 = int(idx % g.n2);
  const long long r = idx / g.n2;
  const int i1 = int(r % g.n1);
  const int i0 = int(r / g.n1);
  const float sg = float(g.osf);
  // RAT (sigma = G / N not an integer, g.osf == 0): sigma n = (G n) div N +
  // r / N exactly, r = (G n) mod N; the rest of the decomposition in FP64
  int ip0 = 0, ip1 = 0, ip2 = 0;
  double fr0 = 0.0, fr1 = 0.0, fr2 = 0.0, sr0 = 0.0, sr1 = 0.0, sr2 = 0.0;
  if constexpr (RAT) {
    ip0 = int((long long)g.g0 * i0 / g.n0);
    ip1 = int((long long)g.g1 * i1 / g.n1);
    ip2 = int((long long)g.g2 * i2 / g.n2);
    fr0 = double((long long)g.g0 * i0 - (long long)ip0 * g.n0) / g.n0;
    fr1 = double((long long)g.g1 * i1 - (long long)ip1 * g.n1) / g.n1;
    fr2 = double((long long)g.g2 * i2 - (long long)ip2 * g.n2) / g.n2;
    sr0 = double(g.g0) / g.n0;
    sr1 = double(g.g1) / g.n1;
    sr2 = double(g.g2) / g.n2;
  }
  for (int j = 0; j < P; ++j) {
    const float* dj = disp + (long long)j * 3 * g.nvox;
    float f0, f1, f2;
    int b0, b1, b2;
    if constexpr (!RAT) {
      // exact decomposition of q = sigma*n + sigma*d into first tap and fraction
      const float s0 = sg * __ldg(dj + idx);
      const float s1 = sg * __ldg(dj + g.nvox + idx);
      const float s2 = sg * __ldg(dj + 2 * g.nvox + idx);
      const float fl0 = floorf(s0), fl1 = floorf(s1), fl2 = floorf(s2);
      f0 = s0 - fl0;
      f1 = s1 - fl1;
      f2 = s2 - fl2;
      b0 = wrap_any(g.osf * i0 + int(fl0) - (W / 2 - 1), g.g0);
      b1 = wrap_any(g.osf * i1 + int(fl1) - (W / 2 - 1), g.g1);
      b2 = wrap_any(g.osf * i2 + int(fl2) - (W / 2 - 1), g.g2);
    } else {
      const double s0 = fr0 + sr0 * double(__ldg(dj + idx));
      const double s1 = fr1 + sr1 * double(__ldg(dj + g.nvox + idx));
      const double s2 = fr2 + sr2 * double(__ldg(dj + 2 * g.nvox + idx));
      const double fl0 = floor(s0), fl1 = floor(s1), fl2 = floor(s2);
      f0 = float(s0 - fl0);
      f1 = float(s1 - fl1);
      f2 = float(s2 - fl2);
      b0 = wrap_any(ip0 + int(fl0) - (W / 2 - 1), g.g0);
      b1 = wrap_any(ip1 + int(fl1) - (W / 2 - 1), g.g1);
      b2 = wrap_any(ip2 + int(fl2) - (W / 2 - 1), g.g2);
    }
    float w0[W], w1[W], w2[W];
    kernel_weights<W>(f0, kc, w0);
    kernel_weights<W>(f1, kc, w1);
    kernel_weights<W>(f2, kc, w2);
    int x2[W];
#pragma unroll
    for (int t = 0; t < W; ++t) x2[t] = wrap_once(b2 + t, g.g2);
    float2 aw = make_float2(0.f, 0.f);
#pragma unroll
    for (int t0 = 0; t0 < W; ++t0) {
      const long long row0 = (long long)wrap_once(b0 + t0, g.g0) * g.g1;
#pragma unroll
      for (int t1 = 0; t1 < W; ++t1) {
        const float w01 = w0[t0] * w1[t1];
        const float2* rowp = u + (row0 + wrap_once(b1 + t1, g.g1)) * g.g2;
        float2 rw = make_float2(0.f, 0.f);
#pragma unroll
        for (int t2 = 0; t2 < W; ++t2) {
          const float2 v = __ldg(rowp + x2[t2]);
          rw = __ffma2_rn(make_float2(w2[t2], w2[t2]), v, rw);  // each part as fmaf
        }
        aw = __ffma2_rn(make_float2(w01, w01), rw, aw);
      }
    }
    m[(long long)j * g.nvox + idx] = aw;
  }
}

__global__ void axpby_kernel(long long n, const float2* __restrict__ x, float a,
                             float2* __restrict__ y, float b) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float2 xv = x[i], yv = y[i];
  y[i] = make_float2(fmaf(a, xv.x, b * yv.x), fmaf(a, xv.y, b * yv.y));
}

__global__ void copy_phases_kernel(long long nvox, int P, const float2* __restrict__ x,
                                   float2* __restrict__ m) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= nvox) return;
  const float2 v = x[i];
  for (int j = 0; j < P; ++j) m[(long long)j * nvox + i] = v;
}

__global__ void sum_phases_kernel(long long nvox, int P, const float2* __restrict__ m,
                                  float2* __restrict__ x) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= nvox) return;
  float2 a = m[i];
  for (int j = 1; j < P; ++j) {
    const float2 v = m[(long long)j * nvox + i];
    a.x += v.x;
    a.y += v.y;
  }
  x[i] = a;
}

inline unsigned blocks_for(long long n, int threads) {
  return unsigned((n + threads - 1) / threads);
}

}  // namespace

int launch_deapod_pad(const Geo& g, const float* deapod, const nrsense_c64* xhat,
                       nrsense_c64* upad, cudaStream_t s) {
  deapod_pad_kernel<<<blocks_for(g.nvox, 256), 256, 0, s>>>(
      g, deapod, reinterpret_cast<const float2*>(xhat), reinterpret_cast<float2*>(upad),
      float(1.0 / double(g.nvox)));
  return 1;
}

int launch_crop_deapod(const Geo& g, const float* deapod, const nrsense_c64* ufreq,
                        nrsense_c64* xhat, cudaStream_t s) {
  crop_deapod_kernel<<<blocks_for(g.nvox, 256), 256, 0, s>>>(
      g, deapod, reinterpret_cast<const float2*>(ufreq), reinterpret_cast<float2*>(xhat),
      float(1.0 / double(g.nvox)));
  return 1;
}

int launch_interp_image(const Geo& g, int W, const KernelCoefs& kc, int P,
                         const float* disp, const nrsense_c64* u, nrsense_c64* m,
                         cudaStream_t s) {
  const auto* up = reinterpret_cast<const float2*>(u);
  auto* mp = reinterpret_cast<float2*>(m);
  const unsigned nb = blocks_for(g.nvox, 256);
  const bool rat = g.osf == 0;  // sigma not an integer: its own instantiation
  if (W == 4) {
    if (rat)
      interp_image_kernel<4, true><<<nb, 256, 0, s>>>(g, kc, P, disp, up, mp);
    else
      interp_image_kernel<4, false><<<nb, 256, 0, s>>>(g, kc, P, disp, up, mp);
  } else {
    if (rat)
      interp_image_kernel<6, true><<<nb, 256, 0, s>>>(g, kc, P, disp, up, mp);
    else
      interp_image_kernel<6, false><<<nb, 256, 0, s>>>(g, kc, P, disp, up, mp);
  }
  return 1;
}

int launch_axpby(long long n, const nrsense_c64* x, float a, nrsense_c64* y, float b,
                  cudaStream_t s) {
  axpby_kernel<<<blocks_for(n, 256), 256, 0, s>>>(n, reinterpret_cast<const float2*>(x), a,
                                                  reinterpret_cast<float2*>(y), b);
  return 1;
}

int launch_copy_phases(const Geo& g, int P, const nrsense_c64* x, nrsense_c64* m,
                        cudaStream_t s) {
  copy_phases_kernel<<<blocks_for(g.nvox, 256), 256, 0, s>>>(
      g.nvox, P, reinterpret_cast<const float2*>(x), reinterpret_cast<float2*>(m));
  return 1;
}

int launch_sum_phases(const Geo& g, int P, const nrsense_c64* m, nrsense_c64* x,
                       cudaStream_t s) {
  sum_phases_kernel<<<blocks_for(g.nvox, 256), 256, 0, s>>>(
      g.nvox, P, reinterpret_cast<const float2*>(m), reinterpret_cast<float2*>(x));
  return 1;
}

}  // namespace nrs
