// Fused line pass, complex128 state (FP64 arithmetic).
#include "launch_impl.cuh"

namespace dgb {
template cudaError_t launch_line_pass<double>(const LinePassArgs<double>&, int, int, cudaStream_t);
template int line_pass_radix<double>(int);
}  // namespace dgb
