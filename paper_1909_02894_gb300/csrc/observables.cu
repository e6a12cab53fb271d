// State conversion between the ABI's [2][n] complex128 layout and the internal
// point-interleaved layout, and the FP64 observable reductions.
#include "internal.h"

namespace dgb {

static const int TPB = 256;

template <typename T>
__global__ void k_pack(const double* src, Q4<T>* psi, size_t n) {
  const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const double2 a = reinterpret_cast<const double2*>(src)[k];
  const double2 b = reinterpret_cast<const double2*>(src)[n + k];
  psi[k] = {(T)a.x, (T)a.y, (T)b.x, (T)b.y};
}

template <typename T>
__global__ void k_unpack(const Q4<T>* psi, double* dst, size_t n) {
  const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const Q4<T> p = psi[k];
  reinterpret_cast<double2*>(dst)[k] = make_double2((double)p.x, (double)p.y);
  reinterpret_cast<double2*>(dst)[n + k] = make_double2((double)p.z, (double)p.w);
}

template <typename T>
cudaError_t launch_pack(const double* src, Q4<T>* psi, size_t n, cudaStream_t st) {
  k_pack<T><<<(unsigned)((n + TPB - 1) / TPB), TPB, 0, st>>>(src, psi, n);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_unpack(const Q4<T>* psi, double* dst, size_t n, cudaStream_t st) {
  k_unpack<T><<<(unsigned)((n + TPB - 1) / TPB), TPB, 0, st>>>(psi, dst, n);
  return cudaGetLastError();
}

int observables_blocks(size_t n) {
  size_t b = (n + TPB - 1) / TPB;
  return (int)(b < 2048 ? b : 2048);
}

__device__ inline double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Block-level deterministic sum of 4 values per thread into out[0..3] (thread 0 writes).
__device__ inline void block_sum4(double (&v)[4], double* out) {
  __shared__ double sh[4][TPB / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const double s = warp_sum(v[c]);
    if (lane == 0) sh[c][wid] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int c = 0; c < 4; ++c) {
      double s = 0.0;
      for (int i = 0; i < TPB / 32; ++i) s += sh[c][i];
      out[c] = s;
    }
  }
}

// norm, norm_gamma and the energy density w psi^dagger H psi with
// H psi = -i a1 sigma_x (dx + Omx psi) - i a2 sigma_y (dy + Omy psi) + meff sigma_z psi,
// accumulated in FP64 (a grid-stride loop per block, fixed block count: deterministic).
template <typename T>
__global__ void __launch_bounds__(TPB) k_observables(
    const Q4<T>* psi, const Q4<T>* dx, const Q4<T>* dy, const double* a1, const double* a2,
    const double* meff, const double* w, const double* omx, const double* omy,
    const double* V, const double* Ax, const double* Ay, size_t n, double* density,
    double* partials) {
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (size_t)gridDim.x * blockDim.x) {
    const Q4<T> p = psi[k];
    const double p1r = p.x, p1i = p.y, p2r = p.z, p2i = p.w;
    const double d = p1r * p1r + p1i * p1i + p2r * p2r + p2i * p2i;
    if (density) density[k] = d;
    const double wk = w[k];
    acc[0] += d;
    acc[1] += wk * d;
    if (dx) {
      const Q4<T> gx = dx[k], gy = dy[k];
      const double ox = omx[k], oy = omy[k], A1 = a1[k], A2 = a2[k], me = meff[k];
      // phi_x = dx + Omx psi, phi_y = dy + Omy psi (components 1 and 2)
      const double fx1r = gx.x + ox * p1r, fx1i = gx.y + ox * p1i;
      const double fx2r = gx.z + ox * p2r, fx2i = gx.w + ox * p2i;
      const double fy1r = gy.x + oy * p1r, fy1i = gy.y + oy * p1i;
      const double fy2r = gy.z + oy * p2r, fy2i = gy.w + oy * p2i;
      // h1 = -i a1 phx2 - a2 phy2 + me p1 ; h2 = -i a1 phx1 + a2 phy1 - me p2
      double h1r = A1 * fx2i - A2 * fy2r + me * p1r;
      double h1i = -A1 * fx2r - A2 * fy2i + me * p1i;
      double h2r = A1 * fx1i + A2 * fy1r - me * p2r;
      double h2i = -A1 * fx1r + A2 * fy1i - me * p2i;
      // static potentials: + V psi - (a1 Ax sigma_x + a2 Ay sigma_y) psi
      const double vk = V ? V[k] : 0.0, xk = Ax ? A1 * Ax[k] : 0.0, yk = Ay ? A2 * Ay[k] : 0.0;
      h1r += vk * p1r - xk * p2r - yk * p2i;
      h1i += vk * p1i - xk * p2i + yk * p2r;
      h2r += vk * p2r - xk * p1r + yk * p1i;
      h2i += vk * p2i - xk * p1i - yk * p1r;
      // conj(p1) h1 + conj(p2) h2
      acc[2] += wk * (p1r * h1r + p1i * h1i + p2r * h2r + p2i * h2i);
      acc[3] += wk * (p1r * h1i - p1i * h1r + p2r * h2i - p2i * h2r);
    }
  }
  block_sum4(acc, partials + 4 * (size_t)blockIdx.x);
}

template <typename T>
cudaError_t launch_observables(const Q4<T>* psi, const Q4<T>* dx, const Q4<T>* dy,
                               const double* a1, const double* a2, const double* meff,
                               const double* w, const double* omx, const double* omy,
                               const double* V, const double* Ax, const double* Ay,
                               size_t n, double* density, double* partials, int blocks,
                               cudaStream_t st) {
  k_observables<T><<<blocks, TPB, 0, st>>>(psi, dx, dy, a1, a2, meff, w, omx, omy, V, Ax, Ay,
                                           n, density, partials);
  return cudaGetLastError();
}

__global__ void __launch_bounds__(TPB) k_reduce_partials(const double* partials, int blocks,
                                                         double scale, double* result) {
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int b = threadIdx.x; b < blocks; b += blockDim.x)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[c] += partials[4 * (size_t)b + c];
  __shared__ double out[4];
  block_sum4(acc, out);
  __syncthreads();
  if (threadIdx.x < 4) result[threadIdx.x] = scale * out[threadIdx.x];
}

cudaError_t launch_reduce_partials(const double* partials, int blocks, double scale,
                                   double* result, cudaStream_t st) {
  k_reduce_partials<<<1, TPB, 0, st>>>(partials, blocks, scale, result);
  return cudaGetLastError();
}

#define INST(T)                                                                               \
  template cudaError_t launch_pack<T>(const double*, Q4<T>*, size_t, cudaStream_t);          \
  template cudaError_t launch_unpack<T>(const Q4<T>*, double*, size_t, cudaStream_t);        \
  template cudaError_t launch_observables<T>(const Q4<T>*, const Q4<T>*, const Q4<T>*,       \
                                             const double*, const double*, const double*,    \
                                             const double*, const double*, const double*,    \
                                             const double*, const double*, const double*,    \
                                             size_t, double*, double*, int, cudaStream_t);
INST(float)
INST(double)
#undef INST

}  // namespace dgb
