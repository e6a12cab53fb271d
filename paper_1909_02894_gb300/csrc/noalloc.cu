// Norm reduction that allocates no device memory.
//
// dirac_observables reduces through a partial-sums buffer that the context allocates.
// Some callers cannot allocate device memory at the point where they need a norm:
// services whose device memory is entirely owned by another allocator or by a fixed
// arena reserved up front, and latency-critical loops that cannot afford
// cudaMalloc/cudaFree's implicit device synchronisation. For them, dirac_norms_noalloc does the same FP64
// reduction with its partial sums in a file-scope device array that exists for as long
// as the library is loaded (on every GPU that loads it).
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/dirac.h"
#include "internal.h"

namespace {

constexpr int kThreads = 256;
// Block count cap of the reduction. Blocks stride over the grid, so any grid the
// library accepts (up to 4096 x 4096 points) fits; the scratch is 2048 x 2 doubles
// (32 KiB) per device.
constexpr int kMaxBlocks = 2048;
constexpr int kMaxN = 4096;

// Per-block partial sums {sum |psi|^2, sum w |psi|^2}. Every call overwrites exactly the
// entries it later reads, so nothing needs clearing between calls; calls that overlap
// on the GPU (different streams, no ordering) share this array and race.
static __device__ __align__(256) double g_noalloc_partials[kMaxBlocks * 2];

std::mutex g_mu;
double* g_addr[64] = {nullptr};  // device address of g_noalloc_partials, per device

__device__ inline double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

__device__ inline void block_sum2(double a, double b, double* out) {
  __shared__ double sh[2][kThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  a = warp_sum(a);
  b = warp_sum(b);
  if (lane == 0) {
    sh[0][wid] = a;
    sh[1][wid] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s0 = 0.0, s1 = 0.0;
    for (int i = 0; i < kThreads / 32; ++i) {
      s0 += sh[0][i];
      s1 += sh[1][i];
    }
    out[0] = s0;
    out[1] = s1;
  }
}

// psi: [2][n] complex128; weight: [n] or null (weight 1).
__global__ void __launch_bounds__(kThreads) k_norm_partials(const double2* psi,
                                                            const double* weight, size_t n,
                                                            double* partials) {
  double s = 0.0, sw = 0.0;
  for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (size_t)gridDim.x * blockDim.x) {
    const double2 a = psi[k], b = psi[n + k];
    const double d = a.x * a.x + a.y * a.y + b.x * b.x + b.y * b.y;
    s += d;
    sw += (weight ? weight[k] : 1.0) * d;
  }
  block_sum2(s, sw, partials + 2 * (size_t)blockIdx.x);
}

__global__ void __launch_bounds__(kThreads) k_norm_final(const double* partials, int blocks,
                                                         double scale, double* out) {
  double s = 0.0, sw = 0.0;
  for (int b = threadIdx.x; b < blocks; b += blockDim.x) {
    s += partials[2 * b];
    sw += partials[2 * b + 1];
  }
  __shared__ double r[2];
  block_sum2(s, sw, r);
  __syncthreads();
  if (threadIdx.x == 0) {
    out[0] = scale * r[0];
    out[1] = scale * r[1];
  }
}

}  // namespace

extern "C" dirac_status dirac_norms_noalloc(const double* psi, const double* weight, int nx,
                                            int ny, double ax, double ay, double* out,
                                            void* cuda_stream) {
  if (!psi || !out) {
    dgb::set_global_error("dirac_norms_noalloc: psi and out must be device pointers");
    return DIRAC_EINVAL;
  }
  if (nx < 16 || ny < 16 || nx > kMaxN || ny > kMaxN || (nx & (nx - 1)) || (ny & (ny - 1))) {
    dgb::set_global_error(
        "dirac_norms_noalloc: nx and ny must be powers of two in [16, 4096] (the static "
        "scratch is sized for at most 4096 x 4096 points)");
    return DIRAC_EINVAL;
  }
  if (!(ax > 0.0) || !(ay > 0.0)) {
    dgb::set_global_error("dirac_norms_noalloc: domain half-widths must be positive");
    return DIRAC_EINVAL;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= 64) {
    dgb::set_global_error("dirac_norms_noalloc: no usable current device");
    return DIRAC_ECUDA;
  }
  double* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
      // The array's name is only a host-side stand-in; kernels need its device address,
      // looked up once per device with that device current.
      e = cudaGetSymbolAddress((void**)&g_addr[dev], g_noalloc_partials);
      if (e != cudaSuccess) {
        g_addr[dev] = nullptr;
        dgb::set_global_error(std::string("dirac_norms_noalloc: cudaGetSymbolAddress: ") +
                              cudaGetErrorString(e));
        return DIRAC_ECUDA;
      }
    }
    scratch = g_addr[dev];
  }
  // A launch error left by earlier work on this thread would otherwise surface below as
  // this call's own; report it without clearing it, and launch nothing.
  e = cudaPeekAtLastError();
  if (e != cudaSuccess) {
    dgb::set_global_error(std::string("dirac_norms_noalloc: an earlier CUDA error is pending "
                                      "on this thread (left in place): ") +
                          cudaGetErrorString(e));
    return DIRAC_ECUDA;
  }
  const size_t n = (size_t)nx * ny;
  size_t blocks = (n + kThreads - 1) / kThreads;
  if (blocks > (size_t)kMaxBlocks) blocks = kMaxBlocks;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  k_norm_partials<<<(unsigned)blocks, kThreads, 0, st>>>(reinterpret_cast<const double2*>(psi),
                                                         weight, n, scratch);
  const double scale = (2.0 * ax / nx) * (2.0 * ay / ny);
  k_norm_final<<<1, kThreads, 0, st>>>(scratch, (int)blocks, scale, out);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    dgb::set_global_error(std::string("dirac_norms_noalloc: launch: ") + cudaGetErrorString(e));
    return DIRAC_ECUDA;
  }
  return DIRAC_OK;
}
