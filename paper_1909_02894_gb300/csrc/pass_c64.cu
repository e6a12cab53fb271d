// Fused line pass, complex64 state (FP32 arithmetic, FP64-derived tables).
#include "launch_impl.cuh"

namespace dgb {
template cudaError_t launch_line_pass<float>(const LinePassArgs<float>&, int, int, cudaStream_t);
template int line_pass_radix<float>(int);
template int line_pass_radix_alt<float>(int);
template cudaError_t launch_line_pass_tick<float>(const LinePassArgs<float>&, cudaStream_t);

// Debug builds: reads and clears this translation unit's index-check flag (0 otherwise).
int dgb_debug_flag_c64() {
#if DIRAC_DEBUG
  int v = 0;
  if (cudaMemcpyFromSymbol(&v, g_dbg_bounds, sizeof(int)) != cudaSuccess) return 1;
  if (v) {
    const int z = 0;
    cudaMemcpyToSymbol(g_dbg_bounds, &z, sizeof(int));
  }
  return v;
#else
  return 0;
#endif
}
}  // namespace dgb
