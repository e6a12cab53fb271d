// Fused line pass, complex128 state (FP64 arithmetic).
#include "launch_impl.cuh"

namespace dgb {
template cudaError_t launch_line_pass<double>(const LinePassArgs<double>&, int, int, cudaStream_t);
template int line_pass_radix<double>(int);
template int line_pass_radix_alt<double>(int);
template cudaError_t launch_line_pass_tick<double>(const LinePassArgs<double>&, cudaStream_t);

// Debug builds: reads and clears this translation unit's index-check flag (0 otherwise).
int dgb_debug_flag_c128() {
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
