// Fused line pass, complex64 state (FP32 arithmetic, FP64-derived tables).
#include "launch_impl.cuh"

namespace dgb {
template cudaError_t launch_line_pass<float>(const LinePassArgs<float>&, int, int, cudaStream_t);
template int line_pass_radix<float>(int);
template int line_pass_radix_alt<float>(int);
template cudaError_t launch_line_pass_tick<float>(const LinePassArgs<float>&, cudaStream_t);
}  // namespace dgb
