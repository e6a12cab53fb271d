// Launch logic of the fused line pass, instantiated once per precision.
#pragma once
#include <cuda_runtime.h>

#include "internal.h"

namespace dgb {

template <typename T, int L, int LPC, int MODE>
static cudaError_t launch_one(const LinePassArgs<T>& a, cudaStream_t st) {
  using Gm = Geo<T, L, LPC>;
  if (a.n_lines % Gm::GL != 0 || a.n_lines < Gm::GL) return cudaErrorInvalidValue;
  auto kern = line_pass_kernel<T, L, LPC, MODE>;
  // Function attributes are per device; set them once per device for this kernel.
  static bool configured[64] = {false};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (!configured[dev]) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Gm::SMEM);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    configured[dev] = true;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(a.n_lines / LPC, 1, 1);
  cfg.blockDim = dim3(Gm::THREADS, 1, 1);
  cfg.dynamicSmemBytes = Gm::SMEM;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  if (Gm::CS > 1) {
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = Gm::CS;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
  }
  return cudaLaunchKernelEx(&cfg, kern, a);
}

// Two CTA shapes per line length: opt 0 (about 256 threads) and opt 1 (512 threads);
// lines of 128 points or fewer use 16 lines per CTA, 4096-point lines one line of 512
// threads.
template <typename T, int MODE>
static cudaError_t dispatch(const LinePassArgs<T>& a, int opt, cudaStream_t st) {
  const bool big = (MODE == MODE_STEP) && opt != 0;
  switch (a.L) {
    case 16: return launch_one<T, 16, 16, MODE>(a, st);
    case 32: return launch_one<T, 32, 16, MODE>(a, st);
    case 64: return launch_one<T, 64, 16, MODE>(a, st);
    case 128: return launch_one<T, 128, 16, MODE>(a, st);
    case 4096: return launch_one<T, 4096, 1, MODE>(a, st);
    default: break;
  }
  if constexpr (MODE == MODE_STEP) {
    if (big) {
      switch (a.L) {
        case 256: return launch_one<T, 256, 16, MODE>(a, st);
        case 512: return launch_one<T, 512, 8, MODE>(a, st);
        case 1024: return launch_one<T, 1024, 4, MODE>(a, st);
        case 2048: return launch_one<T, 2048, 2, MODE>(a, st);
        default: return cudaErrorInvalidValue;
      }
    }
  }
  switch (a.L) {
    case 256: return launch_one<T, 256, 8, MODE>(a, st);
    case 512: return launch_one<T, 512, 4, MODE>(a, st);
    case 1024: return launch_one<T, 1024, 2, MODE>(a, st);
    case 2048: return launch_one<T, 2048, 1, MODE>(a, st);
    default: return cudaErrorInvalidValue;
  }
}

template <typename T>
cudaError_t launch_line_pass(const LinePassArgs<T>& a, int mode, int opt, cudaStream_t st) {
  if (mode == MODE_DERIV) return dispatch<T, MODE_DERIV>(a, 0, st);
  return dispatch<T, MODE_STEP>(a, opt, st);
}

}  // namespace dgb
