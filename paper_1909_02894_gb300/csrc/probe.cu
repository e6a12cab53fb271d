// Measured arithmetic peaks of the device: the denominators of the ALU-bound rooflines.
//
// Each thread runs eight independent fused multiply-add chains (enough to cover the FMA
// latency) over a fixed number of iterations; eight 256-thread blocks per SM fill every
// warp slot. The kernel is timed with CUDA events after a warm-up launch, with the
// iteration count scaled so that the timed launch takes a few milliseconds. The chains'
// results go to a file-scope device variable only when they take an impossible value, so
// the compiler keeps the arithmetic and nothing is allocated.
#include <cuda_runtime.h>

#include <string>

#include "../../include/dirac.h"
#include "internal.h"

namespace {

__device__ double g_probe_sink;

template <typename T>
__global__ void __launch_bounds__(256) k_fma_chains(int iters, T a, T b) {
  T x[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) x[i] = T(threadIdx.x + i) * T(1e-3);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = fma(x[i], a, b);
  }
  T s = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += x[i];
  if (s == T(-12345.678)) g_probe_sink = (double)s;
}

// The same with packed FP32 pairs (fma.rn.f32x2, sm_100 and later): two FMAs per
// instruction.
__global__ void __launch_bounds__(256) k_fma2_chains(int iters, float a, float b) {
  unsigned long long x[8], av, bv;
  asm("mov.b64 %0, {%1, %1};" : "=l"(av) : "f"(a));
  asm("mov.b64 %0, {%1, %1};" : "=l"(bv) : "f"(b));
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const float lo = (float)(threadIdx.x + i) * 1e-3f, hi = lo + 0.5f;
    asm("mov.b64 %0, {%1, %2};" : "=l"(x[i]) : "f"(lo), "f"(hi));
  }
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i)
      asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(x[i]) : "l"(av), "l"(bv));
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    float lo, hi;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(x[i]));
    s += lo + hi;
  }
  if (s == -12345.678f) g_probe_sink = (double)s;
}

cudaError_t launch_probe(int kind, int blocks, int iters, cudaStream_t st) {
  if (kind == 0)
    k_fma_chains<double><<<blocks, 256, 0, st>>>(iters, 0.999999, 1e-7);
  else if (kind == 1)
    k_fma_chains<float><<<blocks, 256, 0, st>>>(iters, 0.999999f, 1e-7f);
  else
    k_fma2_chains<<<blocks, 256, 0, st>>>(iters, 0.999999f, 1e-7f);
  return cudaGetLastError();
}

}  // namespace

extern "C" dirac_status dirac_measure_alu_peak(int kind, double* tflops, void* cuda_stream) {
  if (!tflops || kind < 0 || kind > 2) {
    dgb::set_global_error("dirac_measure_alu_peak: kind must be 0, 1 or 2 and tflops non-NULL");
    return DIRAC_EINVAL;
  }
  *tflops = 0.0;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaStream_t st = (cudaStream_t)cuda_stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  const int blocks = 8 * sms;
  int iters = 256;
  float ms = 0.f;
  // scale the iteration count until one launch takes at least 2 ms (bounded doubling)
  for (int round = 0; round < 16 && e == cudaSuccess; ++round) {
    e = launch_probe(kind, blocks, iters, st);  // warm-up at this size
    if (e == cudaSuccess) e = cudaEventRecord(e0, st);
    if (e == cudaSuccess) e = launch_probe(kind, blocks, iters, st);
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess || ms >= 2.0f || iters >= (1 << 24)) break;
    iters *= 2;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess) {
    dgb::set_global_error(std::string("dirac_measure_alu_peak: ") + cudaGetErrorString(e));
    return DIRAC_ECUDA;
  }
  const double fmas = (double)blocks * 256.0 * (double)iters * 8.0 * (kind == 2 ? 2.0 : 1.0);
  *tflops = 2.0 * fmas / ((double)ms * 1e-3) / 1e12;
  return DIRAC_OK;
}
