// k-space half of the nonrigid SENSE operator: coil sensitivities S and
// inverse k-space gridding G_j (section "k-space Gridding", inverse gridding
// diagram 1/c* -> Z -> F -> B^(k)) and the elementwise ends of k-space
// gridding G_j^H (F^H -> Z^H -> 1/c, then S^H).  Grids hold all C coils
// interleaved ([G^3][C], coil fastest) so that one tap of one sample is one
// contiguous C*8-byte read.
#include "plan_internal.h"

namespace nrs {

namespace {

// centred index n' = i - N/2 placed on the periodic G grid
__device__ __forceinline__ int centred_pos(int i, int N, int G) {
  const int c = i - (N >> 1);
  return c < 0 ? c + G : c;
}

// K5: v_{j,c}[n'] = S_c[n] m_j[n] / C3(n'/G) written into the centred N^3 block
// of the zero-padded coil grids (steps S, 1/c* and Z).
__global__ void coil_fanout_pad_kernel(Geo g, int C, const float* __restrict__ dtab,
                                       const float2* __restrict__ smaps,  // [nvox][C]
                                       const float2* __restrict__ m,
                                       float2* __restrict__ xpad) {         // [G^3][C]
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= g.nvox * C) return;
  const long long idx = t / C;
  const int c = int(t - idx * C);
  const int i2 = int(idx % g.n2);
  const long long r = idx / g.n2;
  const int i1 = int(r % g.n1);
  const int i0 = int(r / g.n1);
  const float w = dtab[i0] * dtab[g.n0 + i1] * dtab[g.n0 + g.n1 + i2];
  const float2 mv = m[idx];
  const float2 sv = smaps[t];
  const float2 v = make_float2((sv.x * mv.x - sv.y * mv.y) * w, (sv.x * mv.y + sv.y * mv.x) * w);
  const long long p = ((long long)centred_pos(i0, g.n0, g.g0) * g.g1 + centred_pos(i1, g.n1, g.g1)) *
                          g.g2 + centred_pos(i2, g.n2, g.g2);
  xpad[p * C + c] = v;
}

// Stage variant of K5 without S: coil images v (C, N^3) -> padded grids.
__global__ void image_to_padded_kernel(Geo g, int C, const float* __restrict__ dtab,
                                       const float2* __restrict__ v,  // [C][nvox]
                                       float2* __restrict__ xpad) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= g.nvox * C) return;
  const long long idx = t / C;
  const int c = int(t - idx * C);
  const int i2 = int(idx % g.n2);
  const long long r = idx / g.n2;
  const int i1 = int(r % g.n1);
  const int i0 = int(r / g.n1);
  const float w = dtab[i0] * dtab[g.n0 + i1] * dtab[g.n0 + g.n1 + i2];
  const float2 vv = v[(long long)c * g.nvox + idx];
  const long long p = ((long long)centred_pos(i0, g.n0, g.g0) * g.g1 + centred_pos(i1, g.n1, g.g1)) *
                          g.g2 + centred_pos(i2, g.n2, g.g2);
  xpad[p * C + c] = make_float2(vv.x * w, vv.y * w);
}

// K6: y_{j,s,c} = sum_taps c3(q_s - g) X_{j,c}[g] (Backprojection Core B^(k)).
// Thread = (sorted sample, group of CPT coils); coordinates are read once per
// thread and all CPT coils of a tap come from one contiguous load.
template <int W, int CPT>
__global__ void __launch_bounds__(256) interp_kspace_kernel(
    Geo g, KernelCoefs kc, int C, long long M, const float4* __restrict__ qs,
    const int32_t* __restrict__ perm, const float2* __restrict__ grid, float2* __restrict__ y) {
  const int tps = C / CPT;
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= M * tps) return;
  const long long s = t / tps;
  const int cg = int(t - s * tps);
  const float4 q = __ldg(qs + s);
  int b0, b1, b2;
  unpack_base(__float_as_uint(q.w), b0, b1, b2);
  float w0[W], w1[W], w2[W];
  kernel_weights<W>(q.x, kc, w0);
  kernel_weights<W>(q.y, kc, w1);
  kernel_weights<W>(q.z, kc, w2);
  int x2[W];
#pragma unroll
  for (int k = 0; k < W; ++k) x2[k] = wrap_once(b2 + k, g.g2);
  float acc[2 * CPT];
#pragma unroll
  for (int i = 0; i < 2 * CPT; ++i) acc[i] = 0.f;
  const float2* gbase = grid + cg * CPT;
#pragma unroll
  for (int t0 = 0; t0 < W; ++t0) {
    const long long row0 = (long long)wrap_once(b0 + t0, g.g0) * g.g1;
#pragma unroll
    for (int t1 = 0; t1 < W; ++t1) {
      const float w01 = w0[t0] * w1[t1];
      const long long row = (row0 + wrap_once(b1 + t1, g.g1)) * g.g2;
#pragma unroll
      for (int t2 = 0; t2 < W; ++t2) {
        const float w = w01 * w2[t2];
        const float2* p = gbase + (row + x2[t2]) * C;
        if constexpr (CPT == 4) {
          const float4 a = __ldg(reinterpret_cast<const float4*>(p));
          const float4 b = __ldg(reinterpret_cast<const float4*>(p) + 1);
          acc[0] = fmaf(w, a.x, acc[0]); acc[1] = fmaf(w, a.y, acc[1]);
          acc[2] = fmaf(w, a.z, acc[2]); acc[3] = fmaf(w, a.w, acc[3]);
          acc[4] = fmaf(w, b.x, acc[4]); acc[5] = fmaf(w, b.y, acc[5]);
          acc[6] = fmaf(w, b.z, acc[6]); acc[7] = fmaf(w, b.w, acc[7]);
        } else if constexpr (CPT == 2) {
          const float4 a = __ldg(reinterpret_cast<const float4*>(p));
          acc[0] = fmaf(w, a.x, acc[0]); acc[1] = fmaf(w, a.y, acc[1]);
          acc[2] = fmaf(w, a.z, acc[2]); acc[3] = fmaf(w, a.w, acc[3]);
        } else {
          const float2 a = __ldg(p);
          acc[0] = fmaf(w, a.x, acc[0]); acc[1] = fmaf(w, a.y, acc[1]);
        }
      }
    }
  }
  float2* out = y + (long long)__ldg(perm + s) * C + cg * CPT;
  if constexpr (CPT == 4) {
    reinterpret_cast<float4*>(out)[0] = make_float4(acc[0], acc[1], acc[2], acc[3]);
    reinterpret_cast<float4*>(out)[1] = make_float4(acc[4], acc[5], acc[6], acc[7]);
  } else if constexpr (CPT == 2) {
    reinterpret_cast<float4*>(out)[0] = make_float4(acc[0], acc[1], acc[2], acc[3]);
  } else {
    out[0] = make_float2(acc[0], acc[1]);
  }
}

// K8: w_j[n] = sum_c conj(S_c[n]) Xt_c[n' mod G] / C3(n'/G) (steps Z^H, 1/c of
// k-space gridding, then S^H).
__global__ void crop_coilsum_kernel(Geo g, int C, const float* __restrict__ dtab,
                                    const float2* __restrict__ smaps,  // [nvox][C]
                                    const float2* __restrict__ xg,     // [G^3][C]
                                    float2* __restrict__ w) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= g.nvox) return;
  const int i2 = int(idx % g.n2);
  const long long r = idx / g.n2;
  const int i1 = int(r % g.n1);
  const int i0 = int(r / g.n1);
  const float dk = dtab[i0] * dtab[g.n0 + i1] * dtab[g.n0 + g.n1 + i2];
  const long long p = ((long long)centred_pos(i0, g.n0, g.g0) * g.g1 + centred_pos(i1, g.n1, g.g1)) *
                          g.g2 + centred_pos(i2, g.n2, g.g2);
  const float2* xs = xg + p * C;
  const float2* ss = smaps + idx * C;
  float ar = 0.f, ai = 0.f;
  for (int c = 0; c < C; ++c) {
    const float2 s = __ldg(ss + c);
    const float2 v = __ldg(xs + c);
    ar = fmaf(s.x, v.x, fmaf(s.y, v.y, ar));
    ai = fmaf(s.x, v.y, fmaf(-s.y, v.x, ai));
  }
  w[idx] = make_float2(ar * dk, ai * dk);
}

// Stage variant of K8 without S^H: padded grids -> coil images (C, N^3).
__global__ void crop_to_coils_kernel(Geo g, int C, const float* __restrict__ dtab,
                                     const float2* __restrict__ xg, float2* __restrict__ v) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= g.nvox * C) return;
  const long long idx = t / C;
  const int c = int(t - idx * C);
  const int i2 = int(idx % g.n2);
  const long long r = idx / g.n2;
  const int i1 = int(r % g.n1);
  const int i0 = int(r / g.n1);
  const float dk = dtab[i0] * dtab[g.n0 + i1] * dtab[g.n0 + g.n1 + i2];
  const long long p = ((long long)centred_pos(i0, g.n0, g.g0) * g.g1 + centred_pos(i1, g.n1, g.g1)) *
                          g.g2 + centred_pos(i2, g.n2, g.g2);
  const float2 x = xg[p * C + c];
  v[(long long)c * g.nvox + idx] = make_float2(x.x * dk, x.y * dk);
}

inline unsigned blocks_for(long long n, int threads) {
  return unsigned((n + threads - 1) / threads);
}

template <int W>
int interp_dispatch(const Geo& g, const KernelCoefs& kc, int C, const PointSet& ps,
                     const float2* grid, float2* y, cudaStream_t s) {
  if (ps.npts == 0) return 0;
  if (C % 4 == 0) {
    const long long n = ps.npts * (C / 4);
    interp_kspace_kernel<W, 4><<<blocks_for(n, 256), 256, 0, s>>>(g, kc, C, ps.npts, ps.qs,
                                                                   ps.perm, grid, y);
  } else if (C % 2 == 0) {
    const long long n = ps.npts * (C / 2);
    interp_kspace_kernel<W, 2><<<blocks_for(n, 256), 256, 0, s>>>(g, kc, C, ps.npts, ps.qs,
                                                                   ps.perm, grid, y);
  } else {
    const long long n = ps.npts * C;
    interp_kspace_kernel<W, 1><<<blocks_for(n, 256), 256, 0, s>>>(g, kc, C, ps.npts, ps.qs,
                                                                   ps.perm, grid, y);
  }
  return 1;
}

}  // namespace

int launch_coil_fanout_pad(const Geo& g, int C, const float* deapod,
                            const nrsense_c64* smaps, const nrsense_c64* m,
                            nrsense_c64* xpad, cudaStream_t s) {
  coil_fanout_pad_kernel<<<blocks_for(g.nvox * C, 256), 256, 0, s>>>(
      g, C, deapod, reinterpret_cast<const float2*>(smaps), reinterpret_cast<const float2*>(m),
      reinterpret_cast<float2*>(xpad));
  return 1;
}

int launch_image_to_padded(const Geo& g, int C, const float* deapod,
                            const nrsense_c64* v, nrsense_c64* xpad, cudaStream_t s) {
  image_to_padded_kernel<<<blocks_for(g.nvox * C, 256), 256, 0, s>>>(
      g, C, deapod, reinterpret_cast<const float2*>(v), reinterpret_cast<float2*>(xpad));
  return 1;
}

int launch_interp_kspace(const Geo& g, int W, const KernelCoefs& kc, int C,
                          const PointSet& ps, const nrsense_c64* grid, nrsense_c64* y,
                          cudaStream_t s) {
  const auto* gp = reinterpret_cast<const float2*>(grid);
  auto* yp = reinterpret_cast<float2*>(y);
  return W == 4 ? interp_dispatch<4>(g, kc, C, ps, gp, yp, s)
                : interp_dispatch<6>(g, kc, C, ps, gp, yp, s);
}

int launch_crop_coilsum(const Geo& g, int C, const float* deapod,
                         const nrsense_c64* smaps, const nrsense_c64* xg,
                         nrsense_c64* w, cudaStream_t s) {
  crop_coilsum_kernel<<<blocks_for(g.nvox, 256), 256, 0, s>>>(
      g, C, deapod, reinterpret_cast<const float2*>(smaps), reinterpret_cast<const float2*>(xg),
      reinterpret_cast<float2*>(w));
  return 1;
}

int launch_crop_to_coils(const Geo& g, int C, const float* deapod,
                          const nrsense_c64* xg, nrsense_c64* v, cudaStream_t s) {
  crop_to_coils_kernel<<<blocks_for(g.nvox * C, 256), 256, 0, s>>>(
      g, C, deapod, reinterpret_cast<const float2*>(xg), reinterpret_cast<float2*>(v));
  return 1;
}

}  // namespace nrs
