// Fused line pass, complex128 state (FP64 arithmetic).
#include "launch_impl.cuh"

namespace dgb {
template cudaError_t launch_line_pass<double>(const LinePassArgs<double>&, int, int, cudaStream_t);
template int line_pass_radix<double>(int);
template int line_pass_radix_alt<double>(int);
template cudaError_t launch_line_pass_tick<double>(const LinePassArgs<double>&, cudaStream_t);
}  // namespace dgb
