// Pointwise kernels of the unsplit polynomial scheme (Sec. 4.2 eq. op_split_poly, Sec. 5
// eq. poly): the middle step applies sum_q a_q P_q(dt A) with
//   A psi = - sum_j b^j sigma_j [[d_j]] psi,   b^j = a^j / S^j (Sec. 3),
// where the spectral derivatives come from the derivative-mode line passes and the rest
// is one combine kernel per operator application.
#include <cuda_runtime.h>
#include <math.h>

#include "internal.h"

namespace dgb {

namespace {
constexpr int TPB = 256;
unsigned blocks_for(size_t n) { return (unsigned)((n + TPB - 1) / TPB); }
}  // namespace

// psi <- U psi at every point of the normal layout
template <typename T>
__global__ void k_apply_u(Q4<T>* psi, const Q4<T>* u, size_t n) {
  const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) psi[k] = apply_u(u[k], psi[k]);
}

// psi <- U psi for a general complex U stored as two Q4 per point (deviation from I):
// (d00, u01), (u10, d11)
template <typename T>
__global__ void k_apply_ug(Q4<T>* psi, const Q4<T>* ug, size_t n) {
  const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const Q4<T> p = psi[k], r0 = ug[2 * k], r1 = ug[2 * k + 1];
  // row 0: d00 psi1 + u01 psi2; row 1: u10 psi1 + d11 psi2 (complex), added to psi
  const T a = p.x, b = p.y, c = p.z, d = p.w;
  psi[k] = {a + (r0.x * a - r0.y * b + r0.z * c - r0.w * d),
            b + (r0.x * b + r0.y * a + r0.z * d + r0.w * c),
            c + (r1.x * a - r1.y * b + r1.z * c - r1.w * d),
            d + (r1.x * b + r1.y * a + r1.z * d + r1.w * c)};
}

// S = b1 sigma_x dx + b2 sigma_y dy with sigma_x (u, v) = (v, u), sigma_y (u, v) =
// (-i v, i u); out = alpha S + beta prev; acc += gamma out.
// b^j complex with complex stretching (sxinv_im, syinv_im not null).
template <typename T>
__global__ void k_unsplit_combine(const Q4<T>* dx, const Q4<T>* dy, const double* a1,
                                  const double* a2, const double* sxinv, const double* syinv,
                                  const double* sxinv_im, const double* syinv_im, int nx,
                                  int ny, T ar, T ai, const Q4<T>* prev, T beta, T gr, T gi,
                                  Q4<T>* out, Q4<T>* acc) {
  const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= (size_t)nx * ny) return;
  const int j = (int)(k / nx), i = (int)(k - (size_t)j * nx);
  const T b1 = (T)(a1[k] * sxinv[i]), b2 = (T)(a2[k] * syinv[j]);
  const T b1i = sxinv_im ? (T)(a1[k] * sxinv_im[i]) : T(0);
  const T b2i = syinv_im ? (T)(a2[k] * syinv_im[j]) : T(0);
  const Q4<T> x = dx[k], y = dy[k];
  // sigma_x dx = (dx2, dx1), sigma_y dy = (-i dy2, i dy1), times complex b
  const T t1r = y.w, t1i = -y.z, t2r = -y.y, t2i = y.x;  // sigma_y dy components
  const T s1r = (b1 * x.z - b1i * x.w) + (b2 * t1r - b2i * t1i);
  const T s1i = (b1 * x.w + b1i * x.z) + (b2 * t1i + b2i * t1r);
  const T s2r = (b1 * x.x - b1i * x.y) + (b2 * t2r - b2i * t2i);
  const T s2i = (b1 * x.y + b1i * x.x) + (b2 * t2i + b2i * t2r);
  Q4<T> o = {ar * s1r - ai * s1i, ar * s1i + ai * s1r, ar * s2r - ai * s2i, ar * s2i + ai * s2r};
  if (prev) {
    const Q4<T> p = prev[k];
    o.x += beta * p.x;
    o.y += beta * p.y;
    o.z += beta * p.z;
    o.w += beta * p.w;
  }
  out[k] = o;
  if (acc) {
    Q4<T> s = acc[k];
    s.x += gr * o.x - gi * o.y;
    s.y += gr * o.y + gi * o.x;
    s.z += gr * o.z - gi * o.w;
    s.w += gr * o.w + gi * o.z;
    acc[k] = s;
  }
}

// out = c in (complex c)
template <typename T>
__global__ void k_scale(Q4<T>* out, const Q4<T>* in, T cr, T ci, size_t n) {
  const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const Q4<T> v = in[k];
  out[k] = {cr * v.x - ci * v.y, cr * v.y + ci * v.x, cr * v.z - ci * v.w, cr * v.w + ci * v.z};
}

// Per-block maxima of |b1| and |b2| (grid-stride), partials[2 b], partials[2 b + 1].
__global__ void k_max_b(const double* a1, const double* a2, const double* sxinv,
                        const double* syinv, const double* sxinv_im, const double* syinv_im,
                        int nx, int ny, double* partials) {
  __shared__ double m1[TPB], m2[TPB];
  double x1 = 0.0, x2 = 0.0;
  const size_t n = (size_t)nx * ny;
  for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(k / nx), i = (int)(k - (size_t)j * nx);
    x1 = fmax(x1, fabs(a1[k]) * hypot(sxinv[i], sxinv_im ? sxinv_im[i] : 0.0));
    x2 = fmax(x2, fabs(a2[k]) * hypot(syinv[j], syinv_im ? syinv_im[j] : 0.0));
  }
  m1[threadIdx.x] = x1;
  m2[threadIdx.x] = x2;
  __syncthreads();
  for (int s = TPB / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) {
      m1[threadIdx.x] = fmax(m1[threadIdx.x], m1[threadIdx.x + s]);
      m2[threadIdx.x] = fmax(m2[threadIdx.x], m2[threadIdx.x + s]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = m1[0];
    partials[2 * blockIdx.x + 1] = m2[0];
  }
}

// ---- Krylov building blocks (Scheme I): FP64 accumulation of complex inner products
// <V_i, w> = sum conj(V_i) w over both components; block (x, i) writes its partial sum
// of vector i to partials[2 (i gridDim.x + x)], fixed grid so the sum order is fixed.
template <typename T>
__global__ void k_multi_dot(const Q4<T>* const* V, const Q4<T>* w, size_t n, double* partials) {
  __shared__ double sr[TPB], si[TPB];
  const Q4<T>* v = V[blockIdx.y];
  double ar = 0.0, ai = 0.0;
  for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (size_t)gridDim.x * blockDim.x) {
    const Q4<T> a = v[k], b = w[k];
    ar += (double)a.x * b.x + (double)a.y * b.y + (double)a.z * b.z + (double)a.w * b.w;
    ai += (double)a.x * b.y - (double)a.y * b.x + (double)a.z * b.w - (double)a.w * b.z;
  }
  sr[threadIdx.x] = ar;
  si[threadIdx.x] = ai;
  __syncthreads();
  for (int s = TPB / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) {
      sr[threadIdx.x] += sr[threadIdx.x + s];
      si[threadIdx.x] += si[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const size_t o = 2 * ((size_t)blockIdx.y * gridDim.x + blockIdx.x);
    partials[o] = sr[0];
    partials[o + 1] = si[0];
  }
}

// out += sum_i c_i V_i (c complex, coef[2 i], coef[2 i + 1]; FP64 coefficients)
template <typename T>
__global__ void k_multi_axpy(Q4<T>* out, const Q4<T>* const* V, const double* coef, int count,
                             size_t n) {
  const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  Q4<T> o = out[k];
  for (int i = 0; i < count; ++i) {
    const T cr = (T)coef[2 * i], ci = (T)coef[2 * i + 1];
    const Q4<T> v = V[i][k];
    o.x += cr * v.x - ci * v.y;
    o.y += cr * v.y + ci * v.x;
    o.z += cr * v.z - ci * v.w;
    o.w += cr * v.w + ci * v.z;
  }
  out[k] = o;
}

// out = a x + b y (real a, b)
template <typename T>
__global__ void k_axpby(Q4<T>* out, T a, const Q4<T>* x, T b, const Q4<T>* y, size_t n) {
  const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const Q4<T> p = x[k], q = y[k];
  out[k] = {a * p.x + b * q.x, a * p.y + b * q.y, a * p.z + b * q.z, a * p.w + b * q.w};
}

template <typename T>
cudaError_t launch_multi_dot(const Q4<T>* const* V, int count, const Q4<T>* w, size_t n,
                             double* partials, int n_blocks, cudaStream_t st) {
  k_multi_dot<T><<<dim3(n_blocks, count), TPB, 0, st>>>(V, w, n, partials);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_multi_axpy(Q4<T>* out, const Q4<T>* const* V, const double* coef, int count,
                              size_t n, cudaStream_t st) {
  k_multi_axpy<T><<<blocks_for(n), TPB, 0, st>>>(out, V, coef, count, n);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_axpby(Q4<T>* out, double a, const Q4<T>* x, double b, const Q4<T>* y,
                         size_t n, cudaStream_t st) {
  k_axpby<T><<<blocks_for(n), TPB, 0, st>>>(out, (T)a, x, (T)b, y, n);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_apply_ug(Q4<T>* psi, const Q4<T>* ug, size_t n, cudaStream_t st) {
  k_apply_ug<T><<<blocks_for(n), TPB, 0, st>>>(psi, ug, n);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_apply_u(Q4<T>* psi, const Q4<T>* u, size_t n, cudaStream_t st) {
  k_apply_u<T><<<blocks_for(n), TPB, 0, st>>>(psi, u, n);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_unsplit_combine(const Q4<T>* dx, const Q4<T>* dy, const double* a1,
                                   const double* a2, const double* sxinv, const double* syinv,
                                   const double* sxinv_im, const double* syinv_im, int nx,
                                   int ny, double ar, double ai, const Q4<T>* prev,
                                   double beta, double gr, double gi, Q4<T>* out, Q4<T>* acc,
                                   cudaStream_t st) {
  k_unsplit_combine<T><<<blocks_for((size_t)nx * ny), TPB, 0, st>>>(
      dx, dy, a1, a2, sxinv, syinv, sxinv_im, syinv_im, nx, ny, (T)ar, (T)ai, prev, (T)beta,
      (T)gr, (T)gi, out, acc);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_scale(Q4<T>* out, const Q4<T>* in, double cr, double ci, size_t n,
                         cudaStream_t st) {
  k_scale<T><<<blocks_for(n), TPB, 0, st>>>(out, in, (T)cr, (T)ci, n);
  return cudaGetLastError();
}

cudaError_t launch_max_b(const double* a1, const double* a2, const double* sxinv,
                         const double* syinv, const double* sxinv_im, const double* syinv_im,
                         int nx, int ny, double* partials, int n_blocks, cudaStream_t st) {
  k_max_b<<<n_blocks, TPB, 0, st>>>(a1, a2, sxinv, syinv, sxinv_im, syinv_im, nx, ny, partials);
  return cudaGetLastError();
}

// Bessel functions J_0(x) .. J_n(x), x >= 0, by downward recurrence from an order well
// above max(n, x) (where the minimal solution dominates), J_{k-1} = (2k/x) J_k - J_{k+1},
// normalised by the Neumann sum J_0 + 2 (J_2 + J_4 + ...) = 1. Returns false for bad input.
bool bessel_j_series(double x, int n, double* out) {
  if (!(x >= 0.0) || n < 0) return false;
  for (int k = 0; k <= n; ++k) out[k] = 0.0;
  if (x == 0.0) {
    out[0] = 1.0;
    return true;
  }
  const double big = fmax((double)n, x);
  int top = (int)(big + 50.0 + 6.0 * sqrt(big));
  if (top % 2) ++top;
  double hi = 0.0, mid = 1e-300, norm = 0.0;
  for (int k = top; k > 0; --k) {
    const double lo = 2.0 * k / x * mid - hi;  // J_{k-1} (unnormalised)
    hi = mid;
    mid = lo;
    const int idx = k - 1;
    if (fabs(mid) > 1e200) {
      hi *= 1e-200;
      mid *= 1e-200;
      norm *= 1e-200;
      for (int t = 0; t <= n; ++t) out[t] *= 1e-200;
    }
    if (idx <= n) out[idx] = mid;
    if (idx > 0 && idx % 2 == 0) norm += 2.0 * mid;
  }
  norm += mid;
  for (int k = 0; k <= n; ++k) out[k] /= norm;
  return true;
}

#define INST(T)                                                                              \
  template cudaError_t launch_apply_u<T>(Q4<T>*, const Q4<T>*, size_t, cudaStream_t);        \
  template cudaError_t launch_apply_ug<T>(Q4<T>*, const Q4<T>*, size_t, cudaStream_t);       \
  template cudaError_t launch_unsplit_combine<T>(                                            \
      const Q4<T>*, const Q4<T>*, const double*, const double*, const double*, const double*, \
      const double*, const double*, int, int, double, double, const Q4<T>*, double, double,  \
      double, Q4<T>*, Q4<T>*, cudaStream_t);                                                 \
  template cudaError_t launch_scale<T>(Q4<T>*, const Q4<T>*, double, double, size_t,         \
                                       cudaStream_t);                                        \
  template cudaError_t launch_multi_dot<T>(const Q4<T>* const*, int, const Q4<T>*, size_t,    \
                                           double*, int, cudaStream_t);                      \
  template cudaError_t launch_multi_axpy<T>(Q4<T>*, const Q4<T>* const*, const double*, int,  \
                                            size_t, cudaStream_t);                           \
  template cudaError_t launch_axpby<T>(Q4<T>*, double, const Q4<T>*, double, const Q4<T>*,   \
                                       size_t, cudaStream_t);
INST(float)
INST(double)
#undef INST

}  // namespace dgb
