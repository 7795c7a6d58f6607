// Allocation-free FP64 inner product of two complex vectors.
//
// This is a variant of the CG solver's inner-product kernel (solver.cu) for
// callers that cannot allocate device memory at all: code that may not call
// cudaMalloc (for example a process whose device memory is owned entirely by
// another allocator or a fixed pool, or a real-time loop where an allocation
// could block), and that therefore can neither create a plan nor let the
// library allocate scratch.  The caller passes the two input vectors and a
// device pointer for the two-double result; the per-block partial sums live
// in a fixed array in this file, so the call itself allocates nothing.  The
// paper has no counterpart to this entry point.
#include <mutex>

#include "plan_internal.h"

namespace {

constexpr int kNaThreads = 256;
constexpr int kNaPerThread = 16;
constexpr int kNaChunk = kNaThreads * kNaPerThread;  // elements per block (4096)
constexpr int kNaMaxBlocks = 16384;                  // partial pairs the scratch holds

static_assert((long long)kNaMaxBlocks * kNaChunk == NRSENSE_DOT_NOALLOC_MAX_N,
              "capacity in the header must match the scratch array");

// Per-block partial sums (real, imaginary), 256 KB on every GPU that loads the
// library, held until the process exits.  Every call overwrites the slots it
// uses before reading them, so nothing needs clearing between calls.
static __device__ __align__(256) double g_noalloc_partials[2 * kNaMaxBlocks];

constexpr int kMaxDevices = 64;
double* g_partials_addr[kMaxDevices] = {};  // device address of the array, per device
std::mutex g_setup_mutex;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block b sums conj(x_i) y_i over i in [b * kNaChunk, (b + 1) * kNaChunk) in FP64.
__global__ void __launch_bounds__(kNaThreads) noalloc_dot_partial(const float2* __restrict__ x,
                                                                  const float2* __restrict__ y,
                                                                  long long n,
                                                                  double* __restrict__ partials) {
  __shared__ double s_re[kNaThreads / 32], s_im[kNaThreads / 32];
  const long long base = (long long)blockIdx.x * kNaChunk;
  double re = 0.0, im = 0.0;
#pragma unroll 4
  for (int k = 0; k < kNaPerThread; ++k) {
    const long long i = base + (long long)k * kNaThreads + threadIdx.x;
    if (i < n) {
      const float2 a = x[i], b = y[i];
      re = fma((double)a.x, (double)b.x, fma((double)a.y, (double)b.y, re));
      im = fma((double)a.x, (double)b.y, fma(-(double)a.y, (double)b.x, im));
    }
  }
  re = warp_sum(re);
  im = warp_sum(im);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    s_re[warp] = re;
    s_im[warp] = im;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double tr = 0.0, ti = 0.0;
    for (int w = 0; w < kNaThreads / 32; ++w) {
      tr += s_re[w];
      ti += s_im[w];
    }
    partials[2 * blockIdx.x] = tr;
    partials[2 * blockIdx.x + 1] = ti;
  }
}

// Sum the nb partial pairs in block order (deterministic) into out[0..1].
__global__ void __launch_bounds__(kNaThreads) noalloc_dot_final(const double* __restrict__ partials,
                                                                int nb, double* __restrict__ out) {
  __shared__ double s_re[kNaThreads / 32], s_im[kNaThreads / 32];
  double re = 0.0, im = 0.0;
  for (int b = threadIdx.x; b < nb; b += kNaThreads) {
    re += partials[2 * b];
    im += partials[2 * b + 1];
  }
  re = warp_sum(re);
  im = warp_sum(im);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    s_re[warp] = re;
    s_im[warp] = im;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double tr = 0.0, ti = 0.0;
    for (int w = 0; w < kNaThreads / 32; ++w) {
      tr += s_re[w];
      ti += s_im[w];
    }
    out[0] = tr;
    out[1] = ti;
  }
}

// Device address of the scratch array on the current device, looked up once
// per device (with that device current) and cached for the life of the
// process.  The cache does not survive a cudaDeviceReset of that device: the
// module is loaded again afterwards and the array may move.
nrsense_status partials_address(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return NRSENSE_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return NRSENSE_ERR_ARG;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (g_partials_addr[dev] == nullptr) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_partials) != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return NRSENSE_ERR_CUDA;
    }
    g_partials_addr[dev] = static_cast<double*>(p);
  }
  *out = g_partials_addr[dev];
  return NRSENSE_OK;
}

}  // namespace

extern "C" nrsense_status nrsense_dot_noalloc(const nrsense_c64* x_dev, const nrsense_c64* y_dev,
                                              int64_t n, double* out_dev, void* stream) {
  if (x_dev == nullptr || y_dev == nullptr || out_dev == nullptr || n < 0) return NRSENSE_ERR_ARG;
  if (n > NRSENSE_DOT_NOALLOC_MAX_N) return NRSENSE_ERR_ARG;  // beyond the fixed scratch
  // an error left by earlier, unrelated work is reported as such, before
  // anything is launched, instead of being taken for a failure of this call
  if (cudaPeekAtLastError() != cudaSuccess) return NRSENSE_ERR_CUDA;
  double* partials = nullptr;
  const nrsense_status st = partials_address(&partials);
  if (st != NRSENSE_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int nb = int((n + kNaChunk - 1) / kNaChunk);
  if (nb > 0)
    noalloc_dot_partial<<<nb, kNaThreads, 0, s>>>(reinterpret_cast<const float2*>(x_dev),
                                                  reinterpret_cast<const float2*>(y_dev), n,
                                                  partials);
  noalloc_dot_final<<<1, kNaThreads, 0, s>>>(partials, nb, out_dev);
  return cudaGetLastError() == cudaSuccess ? NRSENSE_OK : NRSENSE_ERR_CUDA;
}
