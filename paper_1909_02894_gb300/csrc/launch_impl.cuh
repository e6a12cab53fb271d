// Launch logic of the fused line pass, instantiated once per precision.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <string.h>

#include "internal.h"
#include "persist_pass.cuh"

namespace dgb {

// Elements per thread: FP32 lines of 256 points or more use E = 8 (radix-8 passes; the
// FFT state of a thread fits the 64-register budget of 1024 threads per SM without
// spilling), and so do 64- and 128-point lines in both precisions (twice the threads per
// line: a small grid's pass is bound by the latency of each warp's dependent chain, and
// halving the chain measured 0.086 -> 0.050 ms per 128^2 complex128 step); the other
// lengths use E = 16.
template <typename T>
constexpr int radix_e(int L) {
  return ((sizeof(T) == 4 && L >= 256) || L == 64 || L == 128) ? 8 : 16;
}
// The other radix schedule the autotuner may choose (0: none): FP32 lines of 256..4096
// points in radix-16 passes, FP64 lines of 256..2048 points in radix-8 passes.
template <typename T>
constexpr int radix_alt(int L) {
  return L < 256 ? 0 : sizeof(T) == 4 ? (L <= 4096 ? 16 : 0) : (L <= 2048 ? 8 : 0);
}

template <typename T, int L, int LPC, int MODE, int E = radix_e<T>(L)>
static cudaError_t launch_one(const LinePassArgs<T>& a, cudaStream_t st) {
  using Gm = Geo<T, L, LPC, E>;
  if (a.n_lines % Gm::GL != 0 || a.n_lines < Gm::GL) return cudaErrorInvalidValue;
  auto kern = line_pass_kernel<T, L, LPC, E, MODE>;
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
  cfg.gridDim = dim3((a.inst ? a.inst_capacity : 1) * (a.n_lines / LPC), 1, 1);
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

// Two CTA shapes per line length (opt 0 smaller, opt 1 larger; lines of 32 points or
// fewer and 4096-point lines have one). Lines per CTA, by precision:
//   FP32 (E = 8 from 256 points): 256: 4|8, 512: 2|4, 1024: 1|2, 2048: 1|2, 4096: 1
//     (256|512 threads, 512|1024 at 2048, 1024 at 4096)
//   FP64 (E = 16 from 256 points): 256: 1|2, 512: 2|4, 1024: 1|2, 2048: 1|2, 4096: 1 (32..512 threads).
//     The FP64 pass is bound by the FP64 units and its CTAs hold 128-162 registers per
//     thread, so few CTAs fit an SM: small CTAs keep all 152 SMs evenly loaded. Measured on
//     the strained-graphene grids (ms per step, opt 0 | opt 1): 256^2 0.096 | 0.096,
//     512^2 0.203 | 0.199, 1024^2 0.741 | 0.886, 2048^2 3.61 | 3.20; the shapes used before
//     (256: 8|16, 512: 4|8, 1024: 2|4) took 0.180 | 0.350, 0.199 | 0.387, 0.885 | 0.832.
//   both: 64 and 128 points (E = 8) 2|16 lines per CTA, 16 and 32 points 16. Measured
//     (ms per step, opt 0 | opt 1): complex128 64^2 0.045 | 0.078, 128^2 0.050 | 0.168;
//     complex64 64^2 0.0156 | 0.0146, 128^2 0.0166 | 0.0187.
template <typename T, int MODE>
static cudaError_t dispatch(const LinePassArgs<T>& a, int opt, cudaStream_t st) {
  constexpr bool F = sizeof(T) == 4;
  const bool big = (MODE == MODE_STEP) && opt != 0;
  if constexpr (MODE == MODE_STEP) {
    // 64- and 128-point lines: 2 lines per CTA as the smaller shape (one or two warps; a
    // small grid then spreads over 8x as many CTAs), 16 as the larger
    if (!big) {
      switch (a.L) {
        case 64: return launch_one<T, 64, 2, MODE>(a, st);
        case 128: return launch_one<T, 128, 2, MODE>(a, st);
        default: break;
      }
    }
  }
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
        case 256: return launch_one<T, 256, F ? 8 : 2, MODE>(a, st);
        case 512: return launch_one<T, 512, 4, MODE>(a, st);
        case 1024: return launch_one<T, 1024, 2, MODE>(a, st);
        case 2048: return launch_one<T, 2048, 2, MODE>(a, st);
        default: return cudaErrorInvalidValue;
      }
    }
  }
  switch (a.L) {
    case 256: return launch_one<T, 256, F ? 4 : 1, MODE>(a, st);
    case 512: return launch_one<T, 512, 2, MODE>(a, st);
    case 1024: return launch_one<T, 1024, 1, MODE>(a, st);
    case 2048: return launch_one<T, 2048, 1, MODE>(a, st);
    default: return cudaErrorInvalidValue;
  }
}

static int sm_count() {
  static int cached[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
  if (!cached[dev]) cudaDeviceGetAttribute(&cached[dev], cudaDevAttrMultiProcessorCount, dev);
  return cached[dev];
}

// Tensor map of a transposed complex64 output out[rows][n_lines] (16-byte points) as a 2D
// float tensor of 4 n_lines x rows, with boxes of 4 x 256 (one point of 256 rows): a
// staged 4096-point line is 16 such boxes. The encoder is taken from the driver at the
// first call.
static cudaError_t out_tensor_map(CUtensorMap* m, void* out, int n_lines, int rows) {
  using Encode = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                              const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                              const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                              CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  static const Encode encode = []() -> Encode {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return nullptr;
    return reinterpret_cast<Encode>(fn);
  }();
  if (!encode) return cudaErrorNotSupported;
  if (n_lines < 1 || rows % 256 != 0 || (reinterpret_cast<uintptr_t>(out) & 15))
    return cudaErrorInvalidValue;
  const cuuint64_t dims[2] = {(cuuint64_t)4 * (cuuint64_t)n_lines, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)n_lines * 16};  // bytes between rows
  const cuuint32_t box[2] = {4, 256};
  const cuuint32_t elem_strides[2] = {1, 1};
  const CUresult r = encode(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, out, dims, strides, box,
                            elem_strides, CU_TENSOR_MAP_INTERLEAVE_NONE,
                            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// Persistent prefetching variant (complex64 step mode, 256..4096-point lines): one
// 1024-thread CTA per SM (clusters of 2 for 4096-point lines), as
// many as can be resident, at most one per group of 4096 points.
template <int L>
static cudaError_t launch_persist(const LinePassArgs<float>& a, cudaStream_t st) {
  using PG = PGeo<float, L>;
  // one U field per pass: the U landing zone holds either the load-side or the
  // store-side matrices (batched launches keep the same rule per instance)
  if (!a.err || a.n_lines % PG::GL != 0 || (a.u_load && a.u_store) || a.beta_im) return cudaErrorInvalidValue;
  auto kern = a.inst ? line_pass_persistent<float, L, true> : line_pass_persistent<float, L, false>;
  static int max_clusters[2][64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  cudaLaunchConfig_t cfg = {};
  cfg.blockDim = dim3(PG::THREADS, 1, 1);
  cfg.dynamicSmemBytes = PG::SMEM;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = PG::CS;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int& cached = max_clusters[a.inst ? 1 : 0][dev];
  if (!cached) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PG::SMEM);
    if (e != cudaSuccess) return e;
    cfg.gridDim = dim3(PG::CS * 64, 1, 1);
    int n = 0;
    e = cudaOccupancyMaxActiveClusters(&n, kern, &cfg);
    if (e != cudaSuccess) return e;
    if (n <= 0) return cudaErrorInvalidConfiguration;
    cached = n;
  }
  const int groups = (a.inst ? a.inst_capacity : 1) * (a.n_lines / PG::LPI);
  int clusters = cached;
  if (clusters > groups / PG::CS) clusters = groups / PG::CS;
  cfg.gridDim = dim3(clusters * PG::CS, 1, 1);
  CUtensorMap tmap;
  memset(&tmap, 0, sizeof(tmap));
  if (L == 4096 && !a.inst && !a.store_normal) {  // the tensor stores of the output tiles
    e = out_tensor_map(&tmap, a.out, a.n_lines, L);
    if (e != cudaSuccess) return e;
  }
  return cudaLaunchKernelEx(&cfg, kern, a, groups, a.err, tmap);
}

// The alternative radix schedule (radix_alt), opt 3 the smaller and opt 4 the larger of two
// CTA shapes (about 256 and 512 threads; 4096-point FP32 lines and 2048-point FP64 lines
// have one, 512 threads). Its twiddle table (a.tw_alt) has the layout of that radix.
template <typename T>
static cudaError_t dispatch_alt(const LinePassArgs<T>& a0, int opt, cudaStream_t st) {
  if (!a0.tw_alt) return cudaErrorInvalidValue;
  LinePassArgs<T> a = a0;
  a.tw = a0.tw_alt;
  const bool big = opt == 4;
  constexpr int M = MODE_STEP;
  if constexpr (sizeof(T) == 4) {  // radix 16: 2 L / 16 threads per line
    switch (a.L) {
      case 256: return big ? launch_one<T, 256, 16, M, 16>(a, st) : launch_one<T, 256, 8, M, 16>(a, st);
      case 512: return big ? launch_one<T, 512, 8, M, 16>(a, st) : launch_one<T, 512, 4, M, 16>(a, st);
      case 1024: return big ? launch_one<T, 1024, 4, M, 16>(a, st) : launch_one<T, 1024, 2, M, 16>(a, st);
      case 2048: return big ? launch_one<T, 2048, 2, M, 16>(a, st) : launch_one<T, 2048, 1, M, 16>(a, st);
      case 4096: return launch_one<T, 4096, 1, M, 16>(a, st);
      default: return cudaErrorInvalidValue;
    }
  } else {  // radix 8: 2 L / 8 threads per line
    switch (a.L) {
      case 256: return big ? launch_one<T, 256, 8, M, 8>(a, st) : launch_one<T, 256, 4, M, 8>(a, st);
      case 512: return big ? launch_one<T, 512, 4, M, 8>(a, st) : launch_one<T, 512, 2, M, 8>(a, st);
      case 1024: return big ? launch_one<T, 1024, 2, M, 8>(a, st) : launch_one<T, 1024, 1, M, 8>(a, st);
      case 2048: return launch_one<T, 2048, 1, M, 8>(a, st);
      default: return cudaErrorInvalidValue;
    }
  }
}

template <typename T>
cudaError_t launch_line_pass(const LinePassArgs<T>& a, int mode, int opt, cudaStream_t st) {
  if (mode == MODE_DERIV) return dispatch<T, MODE_DERIV>(a, 0, st);
  if (opt == 3 || opt == 4) {
    if (radix_alt<T>(a.L) == 0) return cudaErrorInvalidValue;
    return dispatch_alt<T>(a, opt, st);
  }
  if constexpr (sizeof(T) == 4) {
    if (opt == 2) {
      switch (a.L) {
        case 256: return launch_persist<256>(a, st);
        case 512: return launch_persist<512>(a, st);
        case 1024: return launch_persist<1024>(a, st);
        case 2048: return launch_persist<2048>(a, st);
        case 4096: return launch_persist<4096>(a, st);
        default: break;
      }
    }
  }
  return dispatch<T, MODE_STEP>(a, opt >= 1 ? 1 : 0, st);
}

// Batched tick launch (complex64, square grids, 256..2048-point lines): every step of
// the tick in one persistent launch, one 1024-thread CTA per SM, work items from a
// queue with per-instance dependencies (see line_pass_persistent). a.inst, a.n_inst and
// the tick fields describe the whole tick; a.tw serves both passes (equal line lengths).
template <int L>
static cudaError_t launch_persist_tick(const LinePassArgs<float>& a, cudaStream_t st) {
  using PG = PGeo<float, L>;
  if constexpr (PG::CS != 1) {
    return cudaErrorInvalidValue;
  } else {
    if (!a.err || !a.inst || !a.n_inst || !a.tick_queue || !a.tick_done || a.tick_k < 1 ||
        a.tick_k > PG::TICK_K_MAX ||
        a.n_lines != L || a.n_lines % PG::GL != 0 || a.beta_im)
      return cudaErrorInvalidValue;
    auto kern = line_pass_persistent<float, L, true, true>;
    static int max_blocks[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!max_blocks[dev]) {
      e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PG::SMEM);
      if (e != cudaSuccess) return e;
      int per_sm = 0;
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, PG::THREADS, PG::SMEM);
      if (e != cudaSuccess) return e;
      if (per_sm <= 0) return cudaErrorInvalidConfiguration;
      max_blocks[dev] = per_sm * sm_count();
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(max_blocks[dev], 1, 1);
    cfg.blockDim = dim3(PG::THREADS, 1, 1);
    cfg.dynamicSmemBytes = PG::SMEM;
    cfg.stream = st;
    CUtensorMap tmap;
    memset(&tmap, 0, sizeof(tmap));
    return cudaLaunchKernelEx(&cfg, kern, a, 0, a.err, tmap);
  }
}

template <typename T>
cudaError_t launch_line_pass_tick(const LinePassArgs<T>& a, cudaStream_t st) {
  if constexpr (sizeof(T) == 4) {
    switch (a.L) {
      case 256: return launch_persist_tick<256>(a, st);
      case 512: return launch_persist_tick<512>(a, st);
      case 1024: return launch_persist_tick<1024>(a, st);
      case 2048: return launch_persist_tick<2048>(a, st);
      default: break;
    }
  }
  return cudaErrorInvalidValue;
}

template <typename T>
int line_pass_radix(int L) { return radix_e<T>(L); }
template <typename T>
int line_pass_radix_alt(int L) { return radix_alt<T>(L); }

}  // namespace dgb
