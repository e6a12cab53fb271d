// Launch logic of the fused line pass, instantiated once per precision.
#pragma once
#include <cuda_runtime.h>

#include "internal.h"

namespace dgb {

template <typename T>
constexpr int elems_per_thread() { return sizeof(T) == 4 ? 16 : 8; }
// Lines gathered per transposed-store segment: 8 x 16 B (c64) or 4 x 32 B (c128) = 128 B.
template <typename T>
constexpr int seg_lines() { return sizeof(T) == 4 ? 8 : 4; }

inline int ilog2(int v) {
  int l = 0;
  while ((1 << l) < v) ++l;
  return l;
}

template <typename T>
LaunchShape line_pass_shape(int L, int n_lines, int threads_req) {
  constexpr int E = elems_per_thread<T>();
  LaunchShape s{};
  s.tpl = L / E;
  const int thr = threads_req > 0 ? threads_req : 256;
  int lpc = thr / s.tpl;
  if (lpc < 1) lpc = 1;
  while (lpc & (lpc - 1)) lpc &= lpc - 1;  // power of two
  if (lpc > n_lines) lpc = n_lines;
  const int G = seg_lines<T>();
  s.cs = lpc >= G ? 1 : G / lpc;
  while (s.cs > 1 && lpc * s.cs > n_lines) s.cs >>= 1;
  s.lpc = lpc;
  const int l = ilog2(L), e = ilog2(E);
  s.npass = (l + e - 1) / e;
  s.rl = 1 << (l - (s.npass - 1) * e);
  const int plen = Pad<T>::len(L);
  s.line_stride = 2 * plen + (s.tpl < 16 ? (((s.tpl - 2 * plen) % 16) + 16) % 16 : 0);
  const size_t fft_bytes = (size_t)lpc * s.line_stride * sizeof(Cx<T>);
  const size_t stage_bytes = (size_t)lpc * (L + 1) * sizeof(Q4<T>);
  s.smem = fft_bytes > stage_bytes ? fft_bytes : stage_bytes;
  s.threads = lpc * s.tpl;
  s.blocks = n_lines / lpc;
  return s;
}

template <typename T, int MODE>
static cudaError_t launch_mode(const LinePassArgs<T>& a0, int threads_req, cudaStream_t st) {
  constexpr int E = elems_per_thread<T>();
  LinePassArgs<T> a = a0;
  const LaunchShape s = line_pass_shape<T>(a.L, a.n_lines, threads_req);
  if (s.threads > 512 || s.threads < 1 || a.n_lines % (s.lpc * s.cs) != 0)
    return cudaErrorInvalidConfiguration;
  a.lpc = s.lpc;
  a.cs = s.cs;
  auto kern = line_pass_kernel<T, E, MODE>;
  // The dynamic shared-memory limit is a per-device function attribute; remember what was
  // set for each device so the hot loop does not repeat the call.
  static size_t configured[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (s.smem > 48 * 1024 && s.smem > configured[dev]) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)s.smem);
    if (e != cudaSuccess) return e;
    configured[dev] = s.smem;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(s.blocks, 1, 1);
  cfg.blockDim = dim3(s.threads, 1, 1);
  cfg.dynamicSmemBytes = s.smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  if (s.cs > 1) {
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = s.cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
  }
  return cudaLaunchKernelEx(&cfg, kern, a, s.npass, s.rl, s.line_stride);
}

template <typename T>
cudaError_t launch_line_pass(const LinePassArgs<T>& a, int mode, int threads_req,
                             cudaStream_t st) {
  if (mode == MODE_DERIV) return launch_mode<T, MODE_DERIV>(a, threads_req, st);
  return launch_mode<T, MODE_STEP>(a, threads_req, st);
}

}  // namespace dgb
