// FP64 precompute on the device: coefficient fields, spin connection, absorbing-layer
// profile, half-step matrices and the per-axis FFT/k-space tables. Runs at context
// creation (and, for U and the k-space tables, whenever dt changes); never per step.
#include <math.h>

#include "internal.h"

namespace dgb {

static const int TPB = 256;
static inline int nblocks(size_t n) { return (int)((n + TPB - 1) / TPB); }

// Sec. 2.2 with a diagonal static metric: a^j = c sqrt(g00/g_jj), meff = m c^2 sqrt(g00),
// w = sqrt(g11 g22/g00) (sqrt|g| g^00, eq. l2gamma). The spin connection needs the
// derivative of ln(w a^j) (covariant) or of ln g00 (the printed 2D form).
__global__ void k_metric_fields(const double* g00, const double* g11, const double* g22, int n,
                                double c, double mass, int conn, double* a1, double* a2,
                                double* meff, double* w, Q4<double>* logs) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const double G00 = g00 ? g00[k] : 1.0, G11 = g11 ? g11[k] : 1.0, G22 = g22 ? g22[k] : 1.0;
  const double A1 = c * sqrt(G00 / G11), A2 = c * sqrt(G00 / G22);
  const double Wt = sqrt(G11 * G22 / G00);
  a1[k] = A1;
  a2[k] = A2;
  meff[k] = mass * c * c * sqrt(G00);
  w[k] = Wt;
  double f1, f2;
  if (conn == 1) {
    f1 = f2 = log(G00);
  } else {
    f1 = log(Wt * A1);
    f2 = log(Wt * A2);
  }
  logs[k] = {f1, 0.0, f2, 0.0};
}

cudaError_t launch_metric_fields(const double* g00, const double* g11, const double* g22,
                                 int n, double c, double mass, int conn, double* a1,
                                 double* a2, double* meff, double* w, Q4<double>* logs,
                                 cudaStream_t st) {
  k_metric_fields<<<nblocks(n), TPB, 0, st>>>(g00, g11, g22, n, c, mass, conn, a1, a2, meff,
                                              w, logs);
  return cudaGetLastError();
}

// Omega_x = fac Re d_x f1, Omega_y = fac Re d_y f2 (the real part drops the purely
// imaginary Nyquist term of a real field's spectral derivative).
__global__ void k_omega(const Q4<double>* dxT, const Q4<double>* dy, int nx, int ny, double fac,
                        double* omx, double* omy) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nx * ny) return;
  const int j = k / nx, i = k - j * nx;
  omx[k] = fac * dxT[(size_t)i * ny + j].x;
  omy[k] = fac * dy[k].z;
}

cudaError_t launch_omega(const Q4<double>* dxT, const Q4<double>* dy, int nx, int ny,
                         double fac, double* omx, double* omy, cudaStream_t st) {
  k_omega<<<nblocks((size_t)nx * ny), TPB, 0, st>>>(dxT, dy, nx, ny, fac, omx, omy);
  return cudaGetLastError();
}

// Sec. 3: S = 1 + Sigma~ (theta = 0) on the outer `width` points of each side. The depth
// into the layer is measured from the layer's inner edge on the grid: e = (width - i) h on
// the left (so the point x_0 = -a is exactly at |x| = L) and e = (i - n + width) h on the
// right; with s = e - delta (delta = width h) the six profiles are
// s0 e^2, s0 e^3, -s0/s, s0/s^2, -s0/s - s0/delta, s0/s^2 - s0/delta^2.
// Where a singular profile is infinite, 1/S = 0.
__global__ void k_pml(int n, double a, int width, int type, double sigma0, double theta,
                      double* sinv, double* sinv_im) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double r = 1.0, ri = 0.0;
  if (width > 0 && (i <= width || i >= n - width)) {
    const double h = 2.0 * a / n;
    const double depth = (i <= width) ? (double)(width - i) * h : (double)(i - n + width) * h;
    const double delta = width * h;
    const double s = depth - delta;
    double sig = 0.0;
    bool inf = false;
    switch (type) {
      case 1: sig = sigma0 * depth * depth; break;
      case 2: sig = sigma0 * depth * depth * depth; break;
      case 3: inf = (s == 0.0); if (!inf) sig = -sigma0 / s; break;
      case 4: inf = (s == 0.0); if (!inf) sig = sigma0 / (s * s); break;
      case 5: inf = (s == 0.0); if (!inf) sig = -sigma0 / s - sigma0 / delta; break;
      case 6: inf = (s == 0.0); if (!inf) sig = sigma0 / (s * s) - sigma0 / (delta * delta); break;
      default: break;
    }
    if (sinv_im) {  // S = 1 + exp(i theta) Sigma~, 1/S = conj(S) / |S|^2
      const double sr = 1.0 + cos(theta) * sig, si = sin(theta) * sig;
      const double m = sr * sr + si * si;
      r = inf ? 0.0 : sr / m;
      ri = inf ? 0.0 : -si / m;
    } else {
      r = inf ? 0.0 : 1.0 / (1.0 + sig);
    }
  }
  sinv[i] = r;
  if (sinv_im) sinv_im[i] = ri;
}

cudaError_t launch_pml(int n, double a, int width, int type, double sigma0, double theta,
                       double* sinv, double* sinv_im, cudaStream_t st) {
  k_pml<<<nblocks(n), TPB, 0, st>>>(n, a, width, type, sigma0, theta, sinv, sinv_im);
  return cudaGetLastError();
}

template <typename T>
__global__ void k_beta(const double* a1, const double* a2, const double* sxinv,
                       const double* syinv, const double* sxinv_im, const double* syinv_im,
                       int nx, int ny, T* beta1, T* beta2T, T* beta1_im, T* beta2T_im) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nx * ny) return;
  const int j = k / nx, i = k - j * nx;
  beta1[k] = (T)(a1[k] * sxinv[i] - 1.0);
  beta2T[(size_t)i * ny + j] = (T)(a2[k] * syinv[j] - 1.0);
  if (beta1_im) {  // complex stretching: imaginary parts of b - 1
    beta1_im[k] = (T)(a1[k] * sxinv_im[i]);
    beta2T_im[(size_t)i * ny + j] = (T)(a2[k] * syinv_im[j]);
  }
}

template <typename T>
cudaError_t launch_beta(const double* a1, const double* a2, const double* sxinv,
                        const double* syinv, const double* sxinv_im, const double* syinv_im,
                        int nx, int ny, T* beta1, T* beta2T, T* beta1_im, T* beta2T_im,
                        cudaStream_t st) {
  k_beta<T><<<nblocks((size_t)nx * ny), TPB, 0, st>>>(a1, a2, sxinv, syinv, sxinv_im, syinv_im,
                                                      nx, ny, beta1, beta2T, beta1_im,
                                                      beta2T_im);
  return cudaGetLastError();
}

// exp(v.sigma) = C(z) I + S(z) v.sigma with z = v.v (Sec. 4.1 eq. exp_dirac in the
// complex-argument form), C = cosh sqrt z, S = sinh sqrt z / sqrt z; here v1, v2 are real
// and v3 = -i dt/2 meff, so z is real. Returns (C - 1, S v1, S v2, -dt/2 meff S) with C - 1
// written as a squared half-angle sine to keep it accurate when z is small.
__device__ inline void pauli_exp(double v1, double v2, double hm, double* out) {
  const double z = v1 * v1 + v2 * v2 - hm * hm;
  double cm1, S;
  if (fabs(z) < 1e-8) {
    cm1 = z * (0.5 + z * (1.0 / 24.0 + z * (1.0 / 720.0)));
    S = 1.0 + z * (1.0 / 6.0 + z * (1.0 / 120.0 + z * (1.0 / 5040.0)));
  } else if (z > 0.0) {
    const double r = sqrt(z);
    const double sh = sinh(0.5 * r);
    cm1 = 2.0 * sh * sh;
    S = sinh(r) / r;
  } else {
    const double r = sqrt(-z);
    const double sn = sin(0.5 * r);
    cm1 = -2.0 * sn * sn;
    S = sin(r) / r;
  }
  out[0] = cm1;
  out[1] = S * v1;
  out[2] = S * v2;
  out[3] = -hm * S;
}

template <typename T>
__global__ void k_halfstep(const double* a1, const double* a2, const double* meff,
                           const double* omx, const double* omy, int nx, int ny, double dt,
                           Q4<T>* u_n, Q4<T>* u_t, Q4<T>* u2_t, Q4<T>* u2_n) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nx * ny) return;
  const int j = k / nx, i = k - j * nx;
  // exponent -i dt/2 (meff sigma_z + F), F = -i (a1 Omx sigma_x + a2 Omy sigma_y)
  const double v1 = -0.5 * dt * a1[k] * omx[k];
  const double v2 = -0.5 * dt * a2[k] * omy[k];
  const double hm = 0.5 * dt * meff[k];
  double u[4], u2[4];
  pauli_exp(v1, v2, hm, u);
  pauli_exp(2.0 * v1, 2.0 * v2, 2.0 * hm, u2);
  const Q4<T> U = {(T)u[0], (T)u[1], (T)u[2], (T)u[3]};
  const Q4<T> U2 = {(T)u2[0], (T)u2[1], (T)u2[2], (T)u2[3]};
  u_n[k] = U;
  u_t[(size_t)i * ny + j] = U;
  u2_t[(size_t)i * ny + j] = U2;
  if (u2_n) u2_n[k] = U2;
}

// ---- half step with static potentials: a general complex 2x2 matrix per point
struct Z {  // FP64 complex for the per-point exponential
  double r, i;
};
__device__ inline Z zmul(Z a, Z b) { return {a.r * b.r - a.i * b.i, a.r * b.i + a.i * b.r}; }
__device__ inline Z zadd(Z a, Z b) { return {a.r + b.r, a.i + b.i}; }
__device__ inline Z zscale(Z a, double s) { return {a.r * s, a.i * s}; }
__device__ inline Z zdiv(Z a, Z b) {
  const double d = b.r * b.r + b.i * b.i;
  return {(a.r * b.r + a.i * b.i) / d, (a.i * b.r - a.r * b.i) / d};
}
__device__ inline Z zsqrt(Z a) {  // principal root, no cancellation
  const double m = hypot(a.r, a.i);
  if (m == 0.0) return {0.0, 0.0};
  if (a.r >= 0.0) {
    const double t = sqrt(0.5 * (m + a.r));
    return {t, a.i / (2.0 * t)};
  }
  const double t = sqrt(0.5 * (m - a.r));
  return {fabs(a.i) / (2.0 * t), copysign(t, a.i)};
}
__device__ inline Z zsinh(Z a) { return {sinh(a.r) * cos(a.i), cosh(a.r) * sin(a.i)}; }

// exp(v.sigma) - I = (C - 1) I + S v.sigma with z = v.v complex, C - 1 = 2 sinh^2(r/2),
// S = sinh(r)/r, r = sqrt(z) (series for small z); then times the scalar phase
// exp(i phi): U - I = e (C - 1 + S v.sigma) + (e - 1) I with e - 1 = -2 sin^2(phi/2) + i sin phi.
// Output the four entries minus the identity: d00, u01, u10, d11.
__device__ inline void pauli_exp_general(Z v1, Z v2, Z v3, double phi, Z* d) {
  const Z z = zadd(zadd(zmul(v1, v1), zmul(v2, v2)), zmul(v3, v3));
  Z cm1, S;
  if (hypot(z.r, z.i) < 1e-8) {
    const Z z2 = zmul(z, z);
    cm1 = zadd(zscale(z, 0.5), zscale(z2, 1.0 / 24.0));
    S = zadd({1.0, 0.0}, zadd(zscale(z, 1.0 / 6.0), zscale(z2, 1.0 / 120.0)));
  } else {
    const Z r = zsqrt(z);
    const Z sh = zsinh(zscale(r, 0.5));
    cm1 = zscale(zmul(sh, sh), 2.0);
    S = zdiv(zsinh(r), r);
  }
  // v.sigma = [[v3, v1 - i v2], [v1 + i v2, -v3]]
  const Z iv2 = {-v2.i, v2.r};
  Z m00 = zadd(cm1, zmul(S, v3));
  Z m01 = zmul(S, {v1.r - iv2.r, v1.i - iv2.i});
  Z m10 = zmul(S, {v1.r + iv2.r, v1.i + iv2.i});
  Z m11 = zadd(cm1, zscale(zmul(S, v3), -1.0));
  const double sh2 = sin(0.5 * phi);
  const Z em1 = {-2.0 * sh2 * sh2, sin(phi)};  // e^{i phi} - 1
  const Z e = {1.0 + em1.r, em1.i};
  d[0] = zadd(zmul(e, m00), em1);
  d[1] = zmul(e, m01);
  d[2] = zmul(e, m10);
  d[3] = zadd(zmul(e, m11), em1);
}

// U and U^2 with potentials (normal layout), two Q4 per point:
// (d00.re, d00.im, u01.re, u01.im), (u10.re, u10.im, d11.re, d11.im).
template <typename T>
__global__ void k_halfstep_general(const double* a1, const double* a2, const double* meff,
                                   const double* omx, const double* omy, const double* V,
                                   const double* Ax, const double* Ay, size_t n, double dt,
                                   Q4<T>* ug, Q4<T>* ug2) {
  const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  // exponent -i dt/2 [meff sigma_z + F], F = -i sum_j a^j Omega_j sigma_j
  //   - sum_j a^j A_j sigma_j + V I
  const Z v1 = {-0.5 * dt * a1[k] * omx[k], Ax ? 0.5 * dt * a1[k] * Ax[k] : 0.0};
  const Z v2 = {-0.5 * dt * a2[k] * omy[k], Ay ? 0.5 * dt * a2[k] * Ay[k] : 0.0};
  const Z v3 = {0.0, -0.5 * dt * meff[k]};
  const double phi = V ? -0.5 * dt * V[k] : 0.0;
  Z d[4];
  pauli_exp_general(v1, v2, v3, phi, d);
  ug[2 * k] = {(T)d[0].r, (T)d[0].i, (T)d[1].r, (T)d[1].i};
  ug[2 * k + 1] = {(T)d[2].r, (T)d[2].i, (T)d[3].r, (T)d[3].i};
  pauli_exp_general(zscale(v1, 2.0), zscale(v2, 2.0), zscale(v3, 2.0), 2.0 * phi, d);
  ug2[2 * k] = {(T)d[0].r, (T)d[0].i, (T)d[1].r, (T)d[1].i};
  ug2[2 * k + 1] = {(T)d[2].r, (T)d[2].i, (T)d[3].r, (T)d[3].i};
}

template <typename T>
cudaError_t launch_halfstep_general(const double* a1, const double* a2, const double* meff,
                                    const double* omx, const double* omy, const double* V,
                                    const double* Ax, const double* Ay, int nx, int ny,
                                    double dt, Q4<T>* ug, Q4<T>* ug2, cudaStream_t st) {
  const size_t n = (size_t)nx * ny;
  k_halfstep_general<T><<<nblocks(n), TPB, 0, st>>>(a1, a2, meff, omx, omy, V, Ax, Ay, n, dt,
                                                    ug, ug2);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_halfstep(const double* a1, const double* a2, const double* meff,
                            const double* omx, const double* omy, int nx, int ny, double dt,
                            Q4<T>* u_n, Q4<T>* u_t, Q4<T>* u2_t, Q4<T>* u2_n,
                            cudaStream_t st) {
  k_halfstep<T><<<nblocks((size_t)nx * ny), TPB, 0, st>>>(a1, a2, meff, omx, omy, nx, ny, dt,
                                                          u_n, u_t, u2_t, u2_n);
  return cudaGetLastError();
}

// hi/lo split of an FP64 value into the table type.
template <typename T>
__device__ inline void split(double v, T* hi, T* lo) {
  const T h = (T)v;
  *hi = h;
  *lo = (T)(v - (double)h);
}

// Per-pass twiddle blocks (layout in line_pass.cuh, tw_offset) for E elements per
// thread: for every pass after the first, span NS (E, E^2, ...) and radix R (E, or the
// remaining radix for the last pass), entries [(t - 1) NS + k] = exp(-2 pi i t k/(NS R)).
// Computed in FP64.
template <typename T>
__global__ void k_twiddles(int n, int e, Cx<T>* tw) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= n) return;
  int log2n = 0, log2e = 0;
  while ((1 << log2n) < n) ++log2n;
  while ((1 << log2e) < e) ++log2e;
  const int npass = (log2n + log2e - 1) / log2e;
  int off = 0, ns = e;
  for (int p = 1; p < npass; ++p, ns *= e) {
    const int r = (p + 1 == npass) ? (1 << (log2n - (npass - 1) * log2e)) : e;
    const int cnt = (r - 1) * ns;
    if (m < off + cnt) {
      const int t = (m - off) / ns + 1, k = (m - off) % ns;
      double s, c;
      sincospi(2.0 * (double)t * k / ((double)ns * r), &s, &c);
      tw[m] = {(T)c, (T)(-s)};
      return;
    }
    off += cnt;
  }
  tw[m] = {(T)1, (T)0};  // unused entries
}

template <typename T>
cudaError_t launch_twiddles(int n, int e, Cx<T>* tw, cudaStream_t st) {
  k_twiddles<T><<<nblocks(n), TPB, 0, st>>>(n, e, tw);
  return cudaGetLastError();
}

// Sec. 5: FFT index q -> p = q (q < n/2) or q - n, xi = p pi / a. In the eigenbasis of
// sigma the step multiplier exp(-i dt xi sigma) - I has eigenvalues (cos - 1) -+ i sin;
// the table holds (cos - 1, sin) scaled by 1/(2n): the inverse FFT's 1/n and the 1/2 of
// the return from the (unnormalised) eigenbasis.
template <typename T>
__global__ void k_step_mult(int n, double a, double dt, Q4<T>* mult) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  const int p = q < n / 2 ? q : q - n;
  const double th = dt * (p * (M_PI / a));
  const double hs = sin(0.5 * th);
  const double cm1 = -hs * hs / n;
  const double sn = 0.5 * sin(th) / n;
  Q4<T> r;
  split<T>(cm1, &r.x, &r.y);
  split<T>(sn, &r.z, &r.w);
  mult[q] = r;
}

template <typename T>
cudaError_t launch_step_mult(int n, double a, double dt, Q4<T>* mult, cudaStream_t st) {
  k_step_mult<T><<<nblocks(n), TPB, 0, st>>>(n, a, dt, mult);
  return cudaGetLastError();
}

constexpr bool perm1024_is_a_permutation() {
  bool seen[1024] = {};
  for (int k = 0; k < 1024; ++k) {
    const int p = perm1024(k);
    if (p < 0 || p >= 1024 || seen[p]) return false;
    seen[p] = true;
  }
  return true;
}
static_assert(perm1024_is_a_permutation(), "perm1024 must map 0..1023 onto itself");

// dst[perm1024(q)] = src[q] for the 1024 entries of a 1024-point step table
template <typename T>
__global__ void k_perm1024(const Q4<T>* __restrict__ src, Q4<T>* __restrict__ dst) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < 1024) dst[perm1024(q)] = src[q];
}

template <typename T>
cudaError_t launch_perm1024(const Q4<T>* src, Q4<T>* dst, cudaStream_t st) {
  k_perm1024<T><<<nblocks(1024), TPB, 0, st>>>(src, dst);
  return cudaGetLastError();
}

template <typename T>
__global__ void k_deriv_mult(int n, double a, Q4<T>* mult) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  const int p = q < n / 2 ? q : q - n;
  Q4<T> r;
  r.x = r.y = (T)0;
  split<T>(p * (M_PI / a) / n, &r.z, &r.w);
  mult[q] = r;
}

template <typename T>
cudaError_t launch_deriv_mult(int n, double a, Q4<T>* mult, cudaStream_t st) {
  k_deriv_mult<T><<<nblocks(n), TPB, 0, st>>>(n, a, mult);
  return cudaGetLastError();
}

// 32 x 32 tiles through shared memory; one padding column avoids bank conflicts.
template <typename T>
__global__ void k_transpose(const Q4<T>* in, Q4<T>* out, int rows, int cols) {
  __shared__ Q4<T> tile[32][33];
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
    const int r = r0 + dy, c = c0 + threadIdx.x;
    if (r < rows && c < cols) tile[dy][threadIdx.x] = in[(size_t)r * cols + c];
  }
  __syncthreads();
  for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
    const int c = c0 + dy, r = r0 + threadIdx.x;
    if (r < rows && c < cols) out[(size_t)c * rows + r] = tile[threadIdx.x][dy];
  }
}

template <typename T>
cudaError_t launch_transpose(const Q4<T>* in, Q4<T>* out, int rows, int cols, cudaStream_t st) {
  dim3 grid((cols + 31) / 32, (rows + 31) / 32);
  k_transpose<T><<<grid, dim3(32, 8), 0, st>>>(in, out, rows, cols);
  return cudaGetLastError();
}

#define INST(T)                                                                              \
  template cudaError_t launch_beta<T>(const double*, const double*, const double*,          \
                                      const double*, const double*, const double*, int, int, \
                                      T*, T*, T*, T*, cudaStream_t);        \
  template cudaError_t launch_halfstep<T>(const double*, const double*, const double*,      \
                                          const double*, const double*, int, int, double,    \
                                          Q4<T>*, Q4<T>*, Q4<T>*, Q4<T>*, cudaStream_t);     \
  template cudaError_t launch_halfstep_general<T>(                                            \
      const double*, const double*, const double*, const double*, const double*,             \
      const double*, const double*, const double*, int, int, double, Q4<T>*, Q4<T>*,         \
      cudaStream_t);                                                                         \
  template cudaError_t launch_twiddles<T>(int, int, Cx<T>*, cudaStream_t);                    \
  template cudaError_t launch_step_mult<T>(int, double, double, Q4<T>*, cudaStream_t);        \
  template cudaError_t launch_perm1024<T>(const Q4<T>*, Q4<T>*, cudaStream_t);                \
  template cudaError_t launch_deriv_mult<T>(int, double, Q4<T>*, cudaStream_t);               \
  template cudaError_t launch_transpose<T>(const Q4<T>*, Q4<T>*, int, int, cudaStream_t);
INST(float)
INST(double)
#undef INST

}  // namespace dgb
