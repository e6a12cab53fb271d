/*
 * FP64 CPU oracle for "Numerical Scheme II" of arXiv:1909.02894 in 2D (two-component
 * spinor, Pauli matrices sigma_x, sigma_y, sigma_z as in Sec. 6).
 *
 * TEST INFRASTRUCTURE: plain, slow and written to be checked against the paper by eye.
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg use it; the
 * product path never does. No code is shared with the CUDA path.
 *
 * One time step (Sec. 4.2 eq. op_split_curved; Sec. 5.2 eq. poly_mod, rem2,
 * second_scheme), taken in this order and never merged:
 *   S1  psi <- U psi,  U = exp(-i dt/2 [meff sigma_z + F]),  F = -i sum_j a^j Omega_j sigma_j
 *   S2  for each row:    Xi = F_x^-1[ exp(-i dt xi sigma_x) F_x psi ];  psi <- b1 Xi + (1-b1) psi
 *   S3  for each column: Xi = F_y^-1[ exp(-i dt xi sigma_y) F_y psi ];  psi <- b2 Xi + (1-b2) psi
 *   S4  psi <- U psi
 * with b^j = a^j / S^j (Sec. 5.2: PML by replacing a^i with a^i/S^i).  The exponential
 * exp(-i dt xi Lambda) of eq. second_scheme in the alpha^i eigenbasis equals
 * exp(-i dt xi sigma_j) in the original basis because Pi Lambda Pi^dagger = sigma_j.
 *
 * Parity status: every function is pinned by the oracle tests. The absorbing-layer
 * profile is checked point by point against the Sec. 3 closed forms (all six types,
 * theta = 0 and theta != 0); the covariant spin connection by the Hermiticity of w H
 * (a real weighted energy) and by a dense Hamiltonian on a tiny curved grid.
 */
#include "dirac_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

static const double PI = 3.14159265358979323846264338327950288;

static int is_pow2(int n) { return n >= 2 && (n & (n - 1)) == 0; }

int oracle_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

int oracle_set_threads(int n) {
  if (n < 1) return -1;
#ifdef _OPENMP
  omp_set_num_threads(n);
#endif
  return 0;
}

/* ---------------------------------------------------------------------------------
 * Sec. 5: DFT pair. With x_k = -a + k h, h = 2a/N and xi_p = p pi / a the phase
 * exp(-i xi_p (x_k + a)) is exp(-2 pi i p k / N), so the forward sum is the standard
 * DFT; the inverse carries 1/N.  Iterative radix-2 Cooley-Tukey with each twiddle
 * evaluated directly from cos/sin of its own angle.
 * ------------------------------------------------------------------------------- */
int oracle_fft(int n, cplx *x, int inverse) {
  if (!is_pow2(n) && n != 1) return -1;
  if (n == 1) return 0;
  /* bit-reversal permutation */
  for (int i = 1, j = 0; i < n; i++) {
    int bit = n >> 1;
    for (; j & bit; bit >>= 1) j ^= bit;
    j ^= bit;
    if (i < j) {
      cplx t = x[i];
      x[i] = x[j];
      x[j] = t;
    }
  }
  const double sgn = inverse ? 1.0 : -1.0;
  for (int len = 2; len <= n; len <<= 1) {
    int half = len >> 1;
    for (int start = 0; start < n; start += len) {
      for (int k = 0; k < half; k++) {
        double ang = sgn * 2.0 * PI * (double)k / (double)len;
        cplx w = cos(ang) + I * sin(ang);
        cplx u = x[start + k];
        cplx v = w * x[start + k + half];
        x[start + k] = u + v;
        x[start + k + half] = u - v;
      }
    }
  }
  if (inverse) {
    double s = 1.0 / (double)n;
    for (int i = 0; i < n; i++) x[i] *= s;
  }
  return 0;
}

/* xi_p for FFT index q: p = q for q < N/2, p = q - N otherwise (p in [-N/2, N/2)). */
static double xi_of(int q, int n, double a) {
  int p = (q < n / 2) ? q : q - n;
  return (double)p * PI / a;
}

static int check_params(const oracle_params *p) {
  if (!p) return -1;
  if (!is_pow2(p->nx) || !is_pow2(p->ny)) return -1;
  if (!(p->ax > 0.0) || !(p->ay > 0.0)) return -1;
  if (p->pml_wx < 0 || p->pml_wy < 0) return -1;
  if (p->pml_wx >= p->nx / 2 || p->pml_wy >= p->ny / 2) return -1;
  if ((p->pml_wx > 0 || p->pml_wy > 0) && (p->pml_type < 1 || p->pml_type > 6)) return -1;
  return 0;
}

/* Gather line `line` along `axis` of a [ny][nx] complex field into buf. */
static void get_line(const oracle_params *p, int axis, int line, const cplx *f, cplx *buf) {
  if (axis == 0) {
    for (int i = 0; i < p->nx; i++) buf[i] = f[(size_t)line * p->nx + i];
  } else {
    for (int j = 0; j < p->ny; j++) buf[j] = f[(size_t)j * p->nx + line];
  }
}

static void put_line(const oracle_params *p, int axis, int line, cplx *f, const cplx *buf) {
  if (axis == 0) {
    for (int i = 0; i < p->nx; i++) f[(size_t)line * p->nx + i] = buf[i];
  } else {
    for (int j = 0; j < p->ny; j++) f[(size_t)j * p->nx + line] = buf[j];
  }
}

/* Sec. 5 eq. "trick": [[d_i]] psi = F_i^-1 [ i xi F_i psi ] along one axis. */
int oracle_deriv(const oracle_params *p, int axis, const cplx *in, cplx *out) {
  if (check_params(p) || (axis != 0 && axis != 1) || !in || !out) return -1;
  const int n = axis == 0 ? p->nx : p->ny;
  const int lines = axis == 0 ? p->ny : p->nx;
  const double a = axis == 0 ? p->ax : p->ay;
  if (in != out) memcpy(out, in, sizeof(cplx) * (size_t)p->nx * p->ny);
#pragma omp parallel
  {
    cplx *buf = malloc(sizeof(cplx) * (size_t)n);
#pragma omp for
    for (int l = 0; l < lines; l++) {
      get_line(p, axis, l, out, buf);
      oracle_fft(n, buf, 0);
      for (int q = 0; q < n; q++) buf[q] *= I * xi_of(q, n, a);
      oracle_fft(n, buf, 1);
      put_line(p, axis, l, out, buf);
    }
    free(buf);
  }
  return 0;
}

/* ---------------------------------------------------------------------------------
 * Sec. 3: absorbing layer. S(x) = 1 + exp(i theta) Sigma~(x), Sigma~ = Sigma(|x| - L)
 * on L* <= |x| <= L and 0 inside, with L = a, L* = a - width h, delta = L - L*.
 * The depth into the layer e = |x| - L* is taken from the integer grid index so that
 * the grid point x_0 = -a sits exactly at |x| = L (where the singular types III-VI
 * blow up: b = a/S is then 0).  In terms of s = |x| - L = e - delta the profiles are
 * I: s0 (s+delta)^2, II: s0 (s+delta)^3, III: -s0/s, IV: s0/s^2, V: -s0/s - s0/delta,
 * VI: s0/s^2 - s0/delta^2.
 * Returns 1/S (complex) for grid index i along an axis.
 * ------------------------------------------------------------------------------- */
static cplx pml_inv_S(const oracle_params *p, int axis, int i) {
  const int n = axis == 0 ? p->nx : p->ny;
  const int wdt = axis == 0 ? p->pml_wx : p->pml_wy;
  const double a = axis == 0 ? p->ax : p->ay;
  if (wdt <= 0) return 1.0;
  const double h = 2.0 * a / (double)n;
  double e;
  if (i <= wdt)
    e = (double)(wdt - i) * h;
  else if (i >= n - wdt)
    e = (double)(i - (n - wdt)) * h;
  else
    return 1.0;
  const double delta = (double)wdt * h;
  const double s = e - delta; /* in [-delta, 0] */
  const double s0 = p->sigma0;
  double sig;
  switch (p->pml_type) {
    case 1: sig = s0 * e * e; break;
    case 2: sig = s0 * e * e * e; break;
    case 3: if (s == 0.0) return 0.0; sig = -s0 / s; break;
    case 4: if (s == 0.0) return 0.0; sig = s0 / (s * s); break;
    case 5: if (s == 0.0) return 0.0; sig = -s0 / s - s0 / delta; break;
    case 6: if (s == 0.0) return 0.0; sig = s0 / (s * s) - s0 / (delta * delta); break;
    default: sig = 0.0;
  }
  cplx S = 1.0 + cexp(I * p->theta) * sig;
  return 1.0 / S;
}

static double gval(const double *g, size_t k) { return g ? g[k] : 1.0; }

/* ---------------------------------------------------------------------------------
 * Coefficients of the 2D Hamiltonian H = -i sum_j a^j sigma_j (d_j + Omega_j)
 * + meff sigma_z for a diagonal static metric (Sec. 2.2 with eq. alpha_form):
 *   a^j = c sqrt(g00/g_jj),  meff = m c^2 sqrt(g00),  w = sqrt(g11 g22 / g00)
 * (w = sqrt|g| g^00, the weight of the l2_gamma norm, eq. l2gamma).
 * Spin connection:
 *   covariant: Omega_j = 1/2 d_j ln(w a^j) -- the choice for which sum w |psi|^2 is
 *              conserved by the continuous equation (d_j(w a^j) = 2 w a^j Omega_j);
 *   paper_2d:  Omega_j = 1/2 d_j Phi with g00 = exp(2 Phi), as printed for the
 *              conformal example of Experiment 3: 1/4 d_j ln g00;
 *   none:      Omega_j = 0.
 * d_j is the spectral derivative of the sampled field; for a real field its Nyquist
 * term is purely imaginary and only the real part is kept.
 * ------------------------------------------------------------------------------- */
int oracle_coefficients(const oracle_params *p, const double *g00, const double *g11,
                        const double *g22, double *a1, double *a2, double *meff,
                        double *w, double *omx, double *omy, cplx *b1, cplx *b2) {
  if (check_params(p)) return -1;
  const int nx = p->nx, ny = p->ny;
  const size_t np = (size_t)nx * ny;
  for (size_t k = 0; k < np; k++) {
    double G00 = gval(g00, k), G11 = gval(g11, k), G22 = gval(g22, k);
    if (!(G00 > 0.0) || !(G11 > 0.0) || !(G22 > 0.0)) return -2;
  }
  double *A1 = malloc(sizeof(double) * np), *A2 = malloc(sizeof(double) * np);
  double *W = malloc(sizeof(double) * np);
  cplx *f1 = malloc(sizeof(cplx) * np), *f2 = malloc(sizeof(cplx) * np);
  cplx *d1 = malloc(sizeof(cplx) * np), *d2 = malloc(sizeof(cplx) * np);
  for (size_t k = 0; k < np; k++) {
    double G00 = gval(g00, k), G11 = gval(g11, k), G22 = gval(g22, k);
    A1[k] = p->c * sqrt(G00 / G11);
    A2[k] = p->c * sqrt(G00 / G22);
    W[k] = sqrt(G11 * G22 / G00);
    if (p->conn == ORACLE_CONN_PAPER_2D) {
      f1[k] = log(G00);
      f2[k] = log(G00);
    } else {
      f1[k] = log(W[k] * A1[k]);
      f2[k] = log(W[k] * A2[k]);
    }
  }
  if (p->conn != ORACLE_CONN_NONE) {
    oracle_deriv(p, 0, f1, d1);
    oracle_deriv(p, 1, f2, d2);
  }
  const double fac = p->conn == ORACLE_CONN_PAPER_2D ? 0.25 : 0.5;
  for (int j = 0; j < ny; j++) {
    for (int i = 0; i < nx; i++) {
      size_t k = (size_t)j * nx + i;
      if (a1) a1[k] = A1[k];
      if (a2) a2[k] = A2[k];
      if (meff) meff[k] = p->mass * p->c * p->c * sqrt(gval(g00, k));
      if (w) w[k] = W[k];
      if (omx) omx[k] = p->conn == ORACLE_CONN_NONE ? 0.0 : fac * creal(d1[k]);
      if (omy) omy[k] = p->conn == ORACLE_CONN_NONE ? 0.0 : fac * creal(d2[k]);
      if (b1) b1[k] = A1[k] * pml_inv_S(p, 0, i);
      if (b2) b2[k] = A2[k] * pml_inv_S(p, 1, j);
    }
  }
  free(A1); free(A2); free(W); free(f1); free(f2); free(d1); free(d2);
  return 0;
}

/* ---------------------------------------------------------------------------------
 * Sec. 4.1 eq. exp_dirac, for the 2x2 exponent M = -i dt/2 (meff sigma_z + F) with
 * F = -i (a1 Omx sigma_x + a2 Omy sigma_y):  M = v . sigma with
 * v = (-dt/2 a1 Omx, -dt/2 a2 Omy, -i dt/2 meff).  Since (v.sigma)^2 = (v.v) I for any
 * complex v, exp(M) = C(z) I + S(z) M with z = v.v, C(z) = cosh(sqrt z) and
 * S(z) = sinh(sqrt z)/sqrt z (their even power series for small |z|).  For real G
 * this is the printed cos|G| + i(...)/|G| sin|G| form.
 * ------------------------------------------------------------------------------- */
static void exp_pauli(cplx v1, cplx v2, cplx v3, cplx u[4]) {
  cplx z = v1 * v1 + v2 * v2 + v3 * v3;
  cplx C, S;
  if (cabs(z) < 1e-8) {
    C = 1.0 + z / 2.0 + z * z / 24.0 + z * z * z / 720.0;
    S = 1.0 + z / 6.0 + z * z / 120.0 + z * z * z / 5040.0;
  } else {
    cplx r = csqrt(z);
    C = ccosh(r);
    S = csinh(r) / r;
  }
  /* v.sigma = [[v3, v1 - i v2], [v1 + i v2, -v3]] */
  u[0] = C + S * v3;
  u[1] = S * (v1 - I * v2);
  u[2] = S * (v1 + I * v2);
  u[3] = C - S * v3;
}

int oracle_half_step(const oracle_params *p, const double *g00, const double *g11,
                     const double *g22, double dt, cplx *u) {
  if (check_params(p) || !u) return -1;
  const size_t np = (size_t)p->nx * p->ny;
  double *a1 = malloc(sizeof(double) * np), *a2 = malloc(sizeof(double) * np);
  double *me = malloc(sizeof(double) * np);
  double *ox = malloc(sizeof(double) * np), *oy = malloc(sizeof(double) * np);
  int rc = oracle_coefficients(p, g00, g11, g22, a1, a2, me, NULL, ox, oy, NULL, NULL);
  if (rc == 0) {
    for (size_t k = 0; k < np; k++) {
      /* exponent -i dt/2 [meff sigma_z + F], F = -i sum_j a^j Omega_j sigma_j
       *   - sum_j a^j A_j sigma_j + V I  (the potentials: a scalar phase and an imaginary
       *   part of v_1, v_2) */
      cplx v1 = -0.5 * dt * a1[k] * ox[k];
      cplx v2 = -0.5 * dt * a2[k] * oy[k];
      cplx v3 = -0.5 * I * dt * me[k];
      if (p->Ax) v1 += 0.5 * I * dt * a1[k] * p->Ax[k];
      if (p->Ay) v2 += 0.5 * I * dt * a2[k] * p->Ay[k];
      exp_pauli(v1, v2, v3, &u[4 * k]);
      if (p->V) {
        const cplx ph = cexp(-0.5 * I * dt * p->V[k]);
        for (int t = 0; t < 4; t++) u[4 * k + t] *= ph;
      }
    }
  }
  free(a1); free(a2); free(me); free(ox); free(oy);
  return rc;
}

/* S1 / S4: psi <- U psi at every point. */
static void apply_U(const oracle_params *p, const cplx *u, cplx *psi) {
  const size_t np = (size_t)p->nx * p->ny;
  cplx *p1 = psi, *p2 = psi + np;
  for (size_t k = 0; k < np; k++) {
    cplx a = p1[k], b = p2[k];
    p1[k] = u[4 * k + 0] * a + u[4 * k + 1] * b;
    p2[k] = u[4 * k + 2] * a + u[4 * k + 3] * b;
  }
}

/* S2 (axis 0, sigma_x) or S3 (axis 1, sigma_y), Sec. 5.2 eq. second_scheme:
 *   Xi = F^-1 [ exp(-i dt xi sigma_j) F psi ],  psi <- b Xi + (1 - b) psi,
 * exp(-i t sigma_x) = [[cos t, -i sin t], [-i sin t, cos t]],
 * exp(-i t sigma_y) = [[cos t, -sin t], [sin t, cos t]]. */
static void directional_substep(const oracle_params *p, int axis, double dt,
                                const cplx *b, cplx *psi) {
  const int n = axis == 0 ? p->nx : p->ny;
  const int lines = axis == 0 ? p->ny : p->nx;
  const double a = axis == 0 ? p->ax : p->ay;
  const size_t np = (size_t)p->nx * p->ny;
#pragma omp parallel
  {
    cplx *x1 = malloc(sizeof(cplx) * n), *x2 = malloc(sizeof(cplx) * n);
    cplx *o1 = malloc(sizeof(cplx) * n), *o2 = malloc(sizeof(cplx) * n);
    cplx *bl = malloc(sizeof(cplx) * n);
#pragma omp for
    for (int l = 0; l < lines; l++) {
      get_line(p, axis, l, psi, o1);
      get_line(p, axis, l, psi + np, o2);
      get_line(p, axis, l, b, bl);
      memcpy(x1, o1, sizeof(cplx) * n);
      memcpy(x2, o2, sizeof(cplx) * n);
      oracle_fft(n, x1, 0);
      oracle_fft(n, x2, 0);
      for (int q = 0; q < n; q++) {
        double t = dt * xi_of(q, n, a);
        double cs = cos(t), sn = sin(t);
        cplx h1 = x1[q], h2 = x2[q];
        if (axis == 0) {
          x1[q] = cs * h1 - I * sn * h2;
          x2[q] = -I * sn * h1 + cs * h2;
        } else {
          x1[q] = cs * h1 - sn * h2;
          x2[q] = sn * h1 + cs * h2;
        }
      }
      oracle_fft(n, x1, 1);
      oracle_fft(n, x2, 1);
      for (int k = 0; k < n; k++) {
        x1[k] = bl[k] * x1[k] + (1.0 - bl[k]) * o1[k];
        x2[k] = bl[k] * x2[k] + (1.0 - bl[k]) * o2[k];
      }
      put_line(p, axis, l, psi, x1);
      put_line(p, axis, l, psi + np, x2);
    }
    free(x1); free(x2); free(o1); free(o2); free(bl);
  }
}

int oracle_run(const oracle_params *p, const double *g00, const double *g11,
               const double *g22, double dt, long n_steps, cplx *psi) {
  return oracle_run_scheme(p, g00, g11, g22, dt, n_steps, ORACLE_SCHEME_II, psi);
}

int oracle_run_scheme(const oracle_params *p, const double *g00, const double *g11,
                      const double *g22, double dt, long n_steps, int scheme, cplx *psi) {
  if (check_params(p) || !psi || n_steps < 0 || !(dt > 0.0)) return -1;
  if (scheme != ORACLE_SCHEME_II && scheme != ORACLE_SCHEME_II_SYMMETRIC) return -1;
  const size_t np = (size_t)p->nx * p->ny;
  cplx *u = malloc(sizeof(cplx) * 4 * np);
  cplx *b1 = malloc(sizeof(cplx) * np), *b2 = malloc(sizeof(cplx) * np);
  int rc = oracle_half_step(p, g00, g11, g22, dt, u);
  if (rc == 0)
    rc = oracle_coefficients(p, g00, g11, g22, NULL, NULL, NULL, NULL, NULL, NULL, b1, b2);
  if (rc == 0) {
    for (long s = 0; s < n_steps; s++) {
      apply_U(p, u, psi);                              /* S1 */
      if (scheme == ORACLE_SCHEME_II) {
        directional_substep(p, 0, dt, b1, psi);        /* S2 */
        directional_substep(p, 1, dt, b2, psi);        /* S3 */
      } else {
        directional_substep(p, 0, 0.5 * dt, b1, psi);  /* x over dt/2 */
        directional_substep(p, 1, dt, b2, psi);        /* y over dt   */
        directional_substep(p, 0, 0.5 * dt, b1, psi);  /* x over dt/2 */
      }
      apply_U(p, u, psi);                              /* S4 */
    }
  }
  free(u); free(b1); free(b2);
  return rc;
}

/* ---------------------------------------------------------------------------------
 * Unsplit middle step (Sec. 4.2 eq. op_split_poly, Sec. 5 eq. poly). The operator is
 * A psi = - sum_j b^j sigma_j [[d_j]] psi with sigma_x (u, v) = (v, u) and
 * sigma_y (u, v) = (-i v, i u); d is scratch of 2 np points.
 * ------------------------------------------------------------------------------- */
static void apply_A(const oracle_params *p, const cplx *b1, const cplx *b2, const cplx *in,
                    cplx *out, cplx *d) {
  const size_t np = (size_t)p->nx * p->ny;
  oracle_deriv(p, 0, in, d);
  oracle_deriv(p, 0, in + np, d + np);
  for (size_t k = 0; k < np; k++) {
    out[k] = -b1[k] * d[np + k];
    out[np + k] = -b1[k] * d[k];
  }
  oracle_deriv(p, 1, in, d);
  oracle_deriv(p, 1, in + np, d + np);
  for (size_t k = 0; k < np; k++) {
    out[k] += -b2[k] * (-I * d[np + k]);
    out[np + k] += -b2[k] * (I * d[k]);
  }
}

int oracle_apply_A(const oracle_params *p, const double *g00, const double *g11,
                   const double *g22, const cplx *in, cplx *out) {
  if (check_params(p) || !in || !out || in == out) return -1;
  const size_t np = (size_t)p->nx * p->ny;
  cplx *b1 = malloc(sizeof(cplx) * np), *b2 = malloc(sizeof(cplx) * np);
  cplx *d = malloc(sizeof(cplx) * 2 * np);
  int rc = oracle_coefficients(p, g00, g11, g22, NULL, NULL, NULL, NULL, NULL, NULL, b1, b2);
  if (rc == 0) apply_A(p, b1, b2, in, out, d);
  free(b1); free(b2); free(d);
  return rc;
}

/* J_0 .. J_n by Miller's backward recurrence J_{k-1} = (2k/x) J_k - J_{k+1}, started far
 * above max(n, x) and normalised with J_0 + 2 sum_k J_2k = 1. */
int oracle_bessel_j(double x, int n, double *j) {
  if (!(x >= 0.0) || n < 0 || !j) return -1;
  for (int k = 0; k <= n; k++) j[k] = 0.0;
  if (x == 0.0) {
    j[0] = 1.0;
    return 0;
  }
  int m = (n > (int)x ? n : (int)x) + 40 + (int)sqrt(40.0 * (n + x));
  m += m & 1;
  double up = 0.0, cur = 1e-280, sum = 0.0;
  for (int k = m; k >= 1; k--) {
    const double low = (2.0 * k / x) * cur - up;  /* J_{k-1} up to a common factor */
    up = cur;
    cur = low;
    if (fabs(cur) > 1e250) {  /* rescale everything kept so far */
      cur *= 1e-250;
      up *= 1e-250;
      sum *= 1e-250;
      for (int t = 0; t <= n; t++) j[t] *= 1e-250;
    }
    if (k - 1 <= n) j[k - 1] = cur;
    if (k - 1 >= 2 && (k - 1) % 2 == 0) sum += 2.0 * cur;
  }
  sum += cur;  /* J_0 */
  for (int k = 0; k <= n; k++) j[k] /= sum;
  return 0;
}

static double poly_bound(const oracle_params *p, const cplx *b1, const cplx *b2, double dt) {
  const size_t np = (size_t)p->nx * p->ny;
  double m1 = 0.0, m2 = 0.0;
  for (size_t k = 0; k < np; k++) {
    if (cabs(b1[k]) > m1) m1 = cabs(b1[k]);
    if (cabs(b2[k]) > m2) m2 = cabs(b2[k]);
  }
  const double hx = 2.0 * p->ax / p->nx, hy = 2.0 * p->ay / p->ny;
  return dt * (m1 * PI / hx + m2 * PI / hy);
}

int oracle_run_poly(const oracle_params *p, const double *g00, const double *g11,
                    const double *g22, double dt, long n_steps, int family, int order,
                    cplx *psi) {
  if (check_params(p) || !psi || n_steps < 0 || !(dt > 0.0)) return -1;
  if ((family != ORACLE_POLY_TAYLOR && family != ORACLE_POLY_CHEBYSHEV) || order < 1 ||
      order > 256)
    return -1;
  const size_t np = (size_t)p->nx * p->ny, n2 = 2 * np;
  cplx *u = malloc(sizeof(cplx) * 4 * np);
  cplx *b1 = malloc(sizeof(cplx) * np), *b2 = malloc(sizeof(cplx) * np);
  cplx *t0 = malloc(sizeof(cplx) * n2), *t1 = malloc(sizeof(cplx) * n2);
  cplx *t2 = malloc(sizeof(cplx) * n2), *acc = malloc(sizeof(cplx) * n2);
  cplx *d = malloc(sizeof(cplx) * n2);
  double *jq = malloc(sizeof(double) * (order + 1));
  int rc = oracle_half_step(p, g00, g11, g22, dt, u);
  if (rc == 0)
    rc = oracle_coefficients(p, g00, g11, g22, NULL, NULL, NULL, NULL, NULL, NULL, b1, b2);
  const double R = rc == 0 ? poly_bound(p, b1, b2, dt) : 0.0;
  if (rc == 0 && family == ORACLE_POLY_CHEBYSHEV) rc = oracle_bessel_j(R, order, jq);
  for (long s = 0; rc == 0 && s < n_steps; s++) {
    apply_U(p, u, psi);
    if (family == ORACLE_POLY_TAYLOR) {
      /* acc = sum_q (dt A)^q / q! psi, term by term */
      memcpy(acc, psi, sizeof(cplx) * n2);
      memcpy(t0, psi, sizeof(cplx) * n2);
      for (int q = 1; q <= order; q++) {
        apply_A(p, b1, b2, t0, t1, d);
        for (size_t k = 0; k < n2; k++) {
          t0[k] = (dt / q) * t1[k];
          acc[k] += t0[k];
        }
      }
    } else {
      /* phi_0 = psi, phi_1 = B psi, phi_{q+1} = 2 B phi_q - phi_{q-1}, B = (i dt / R) A;
       * acc = sum_q c_q phi_q with c_q = (2 - delta_q0) (-i)^q J_q(R) */
      cplx cq = 1.0;  /* (-i)^q */
      memcpy(t0, psi, sizeof(cplx) * n2);
      for (size_t k = 0; k < n2; k++) acc[k] = jq[0] * t0[k];
      apply_A(p, b1, b2, t0, t1, d);
      for (size_t k = 0; k < n2; k++) t1[k] *= I * dt / R;
      cq *= -I;
      for (size_t k = 0; k < n2; k++) acc[k] += 2.0 * cq * jq[1] * t1[k];
      for (int q = 2; q <= order; q++) {
        apply_A(p, b1, b2, t1, t2, d);
        cq *= -I;
        for (size_t k = 0; k < n2; k++) {
          t2[k] = 2.0 * (I * dt / R) * t2[k] - t0[k];
          acc[k] += 2.0 * cq * jq[q] * t2[k];
        }
        cplx *t = t0;
        t0 = t1;
        t1 = t2;
        t2 = t;
      }
    }
    memcpy(psi, acc, sizeof(cplx) * n2);
    apply_U(p, u, psi);
  }
  free(u); free(b1); free(b2); free(t0); free(t1); free(t2); free(acc); free(d); free(jq);
  return rc;
}

/* ---------------------------------------------------------------------------------
 * Scheme I (Sec. 5.1 eq. cn): G psi* = G~ psi, G = I - (dt/2) A, G~ = I + (dt/2) A,
 * solved by restarted GMRES with modified Gram-Schmidt and Givens rotations.
 * ------------------------------------------------------------------------------- */
static cplx zdot(const cplx *a, const cplx *b, size_t n) { /* sum conj(a) b */
  cplx s = 0.0;
  for (size_t k = 0; k < n; k++) s += conj(a[k]) * b[k];
  return s;
}

/* out = in + sgn (dt/2) A in */
static void apply_G(const oracle_params *p, const cplx *b1, const cplx *b2, double sgn,
                    double dt, const cplx *in, cplx *out, cplx *d) {
  const size_t n2 = 2 * (size_t)p->nx * p->ny;
  apply_A(p, b1, b2, in, out, d);
  for (size_t k = 0; k < n2; k++) out[k] = in[k] + sgn * 0.5 * dt * out[k];
}

static int cn_solve(const oracle_params *p, const cplx *b1, const cplx *b2, double dt,
                    const cplx *rhs, cplx *x, double tol, int m, int max_restarts,
                    long *iters) {
  const size_t n2 = 2 * (size_t)p->nx * p->ny;
  cplx *V = malloc(sizeof(cplx) * n2 * (size_t)(m + 1));
  cplx *w = malloc(sizeof(cplx) * n2), *d = malloc(sizeof(cplx) * n2);
  cplx *H = calloc((size_t)(m + 1) * m, sizeof(cplx));
  cplx *cs = malloc(sizeof(cplx) * m), *sn = malloc(sizeof(cplx) * m);
  cplx *g = malloc(sizeof(cplx) * (m + 1)), *y = malloc(sizeof(cplx) * m);
  const double bnorm = sqrt(creal(zdot(rhs, rhs, n2)));
  int rc = -2;
  for (int cycle = 0; cycle <= max_restarts; cycle++) {
    apply_G(p, b1, b2, -1.0, dt, x, w, d);
    for (size_t k = 0; k < n2; k++) w[k] = rhs[k] - w[k];
    const double beta = sqrt(creal(zdot(w, w, n2)));
    if (beta <= tol * bnorm || beta == 0.0) {
      rc = 0;
      break;
    }
    if (cycle == max_restarts) break;
    for (size_t k = 0; k < n2; k++) V[k] = w[k] / beta;
    for (int i = 0; i <= m; i++) g[i] = 0.0;
    g[0] = beta;
    int kdim = 0;
    for (int j = 0; j < m; j++) {
      cplx *vj = V + (size_t)j * n2, *vn = V + (size_t)(j + 1) * n2;
      apply_G(p, b1, b2, -1.0, dt, vj, vn, d);
      for (int i = 0; i <= j; i++) {
        const cplx *vi = V + (size_t)i * n2;
        const cplx h = zdot(vi, vn, n2);
        H[(size_t)i * m + j] = h;
        for (size_t k = 0; k < n2; k++) vn[k] -= h * vi[k];
      }
      const double hn = sqrt(creal(zdot(vn, vn, n2)));
      H[(size_t)(j + 1) * m + j] = hn;
      if (hn > 0.0)
        for (size_t k = 0; k < n2; k++) vn[k] /= hn;
      /* earlier rotations on column j, then a new one zeroing H[j+1][j] */
      for (int i = 0; i < j; i++) {
        const cplx a = H[(size_t)i * m + j], b = H[(size_t)(i + 1) * m + j];
        H[(size_t)i * m + j] = conj(cs[i]) * a + conj(sn[i]) * b;
        H[(size_t)(i + 1) * m + j] = -sn[i] * a + cs[i] * b;
      }
      const cplx a = H[(size_t)j * m + j], b = H[(size_t)(j + 1) * m + j];
      const double r = sqrt(creal(a * conj(a)) + creal(b * conj(b)));
      cs[j] = r > 0.0 ? a / r : 1.0;
      sn[j] = r > 0.0 ? b / r : 0.0;
      H[(size_t)j * m + j] = r;
      H[(size_t)(j + 1) * m + j] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = conj(cs[j]) * g[j];
      kdim = j + 1;
      if (iters) (*iters)++;
      if (cabs(g[j + 1]) <= tol * bnorm) break;
    }
    /* back substitution H y = g, then x += V y */
    for (int i = kdim - 1; i >= 0; i--) {
      cplx sacc = g[i];
      for (int t = i + 1; t < kdim; t++) sacc -= H[(size_t)i * m + t] * y[t];
      y[i] = sacc / H[(size_t)i * m + i];
    }
    for (int i = 0; i < kdim; i++) {
      const cplx *vi = V + (size_t)i * n2;
      for (size_t k = 0; k < n2; k++) x[k] += y[i] * vi[k];
    }
  }
  free(V); free(w); free(d); free(H); free(cs); free(sn); free(g); free(y);
  return rc;
}

int oracle_run_cn(const oracle_params *p, const double *g00, const double *g11,
                  const double *g22, double dt, long n_steps, double tol, int restart,
                  int max_restarts, long *iters, cplx *psi) {
  if (check_params(p) || !psi || n_steps < 0 || !(dt > 0.0) || !(tol > 0.0) || restart < 1 ||
      restart > 1000 || max_restarts < 0)
    return -1;
  const size_t np = (size_t)p->nx * p->ny, n2 = 2 * np;
  cplx *u = malloc(sizeof(cplx) * 4 * np);
  cplx *b1 = malloc(sizeof(cplx) * np), *b2 = malloc(sizeof(cplx) * np);
  cplx *rhs = malloc(sizeof(cplx) * n2), *d = malloc(sizeof(cplx) * n2);
  if (iters) *iters = 0;
  int rc = oracle_half_step(p, g00, g11, g22, dt, u);
  if (rc == 0)
    rc = oracle_coefficients(p, g00, g11, g22, NULL, NULL, NULL, NULL, NULL, NULL, b1, b2);
  for (long s = 0; rc == 0 && s < n_steps; s++) {
    apply_U(p, u, psi);
    apply_G(p, b1, b2, +1.0, dt, psi, rhs, d);  /* G~ psi */
    rc = cn_solve(p, b1, b2, dt, rhs, psi, tol, restart, max_restarts, iters);
    if (rc == 0) apply_U(p, u, psi);
  }
  free(u); free(b1); free(b2); free(rhs); free(d);
  return rc;
}

/* ---------------------------------------------------------------------------------
 * Observables. norm = hx hy sum |psi|^2 (the discrete l2 norm of Prop. 5.3),
 * norm_gamma = hx hy sum w |psi|^2 (eq. l2gamma with the weight sqrt|g| g^00),
 * density = |psi_1|^2 + |psi_2|^2 (Sec. 6.2), and the energy
 * hx hy sum w psi^dagger H psi with H = -i sum_j a^j sigma_j ([[d_j]] + Omega_j)
 * + meff sigma_z (no absorbing layer) + V - sum_j a^j A_j sigma_j (static potentials, when
 * given), reported as real and imaginary parts.
 * ------------------------------------------------------------------------------- */
int oracle_observables(const oracle_params *p, const double *g00, const double *g11,
                       const double *g22, const cplx *psi, double *obs, double *density) {
  if (check_params(p) || !psi || !obs) return -1;
  const int nx = p->nx, ny = p->ny;
  const size_t np = (size_t)nx * ny;
  const double hx = 2.0 * p->ax / nx, hy = 2.0 * p->ay / ny;
  double *a1 = malloc(sizeof(double) * np), *a2 = malloc(sizeof(double) * np);
  double *me = malloc(sizeof(double) * np), *w = malloc(sizeof(double) * np);
  double *ox = malloc(sizeof(double) * np), *oy = malloc(sizeof(double) * np);
  cplx *dx1 = malloc(sizeof(cplx) * np), *dx2 = malloc(sizeof(cplx) * np);
  cplx *dy1 = malloc(sizeof(cplx) * np), *dy2 = malloc(sizeof(cplx) * np);
  int rc = oracle_coefficients(p, g00, g11, g22, a1, a2, me, w, ox, oy, NULL, NULL);
  if (rc == 0) {
    const cplx *p1 = psi, *p2 = psi + np;
    oracle_deriv(p, 0, p1, dx1);
    oracle_deriv(p, 0, p2, dx2);
    oracle_deriv(p, 1, p1, dy1);
    oracle_deriv(p, 1, p2, dy2);
    double nrm = 0.0, nrg = 0.0;
    cplx en = 0.0;
    for (size_t k = 0; k < np; k++) {
      double d = creal(p1[k] * conj(p1[k])) + creal(p2[k] * conj(p2[k]));
      if (density) density[k] = d;
      nrm += d;
      nrg += w[k] * d;
      /* phi_j = [[d_j]] psi + Omega_j psi */
      cplx fx1 = dx1[k] + ox[k] * p1[k], fx2 = dx2[k] + ox[k] * p2[k];
      cplx fy1 = dy1[k] + oy[k] * p1[k], fy2 = dy2[k] + oy[k] * p2[k];
      /* -i a1 sigma_x phi_x: sigma_x (u, v) = (v, u) */
      cplx h1 = -I * a1[k] * fx2, h2 = -I * a1[k] * fx1;
      /* -i a2 sigma_y phi_y: sigma_y (u, v) = (-i v, i u) */
      h1 += -I * a2[k] * (-I * fy2);
      h2 += -I * a2[k] * (I * fy1);
      /* meff sigma_z psi */
      h1 += me[k] * p1[k];
      h2 += -me[k] * p2[k];
      /* static potentials: + V psi - a1 Ax sigma_x psi - a2 Ay sigma_y psi */
      if (p->V) {
        h1 += p->V[k] * p1[k];
        h2 += p->V[k] * p2[k];
      }
      if (p->Ax) {
        h1 += -a1[k] * p->Ax[k] * p2[k];
        h2 += -a1[k] * p->Ax[k] * p1[k];
      }
      if (p->Ay) {
        h1 += -a2[k] * p->Ay[k] * (-I * p2[k]);
        h2 += -a2[k] * p->Ay[k] * (I * p1[k]);
      }
      en += w[k] * (conj(p1[k]) * h1 + conj(p2[k]) * h2);
    }
    obs[0] = hx * hy * nrm;
    obs[1] = hx * hy * nrg;
    obs[2] = hx * hy * creal(en);
    obs[3] = hx * hy * cimag(en);
  }
  free(a1); free(a2); free(me); free(w); free(ox); free(oy);
  free(dx1); free(dx2); free(dy1); free(dy2);
  return rc;
}

/* ---------------------------------------------------------------------------------
 * Constant coefficients: with g constant the spin connection vanishes, U is the
 * constant exp(-i dt/2 meff sigma_z), and a plane wave exp(i xi.(x + a)) times a
 * 2-vector A is mapped by every sub-step to the same plane wave times
 *   K_j = a^j exp(-i dt xi_j sigma_j) + (1 - a^j) I        (eq. second_scheme),
 * so one step is T = U K_y K_x U and n steps are T^n (repeated products).
 * ------------------------------------------------------------------------------- */
static void mat2_mul(const cplx A[4], const cplx B[4], cplx C[4]) {
  cplx c0 = A[0] * B[0] + A[1] * B[2];
  cplx c1 = A[0] * B[1] + A[1] * B[3];
  cplx c2 = A[2] * B[0] + A[3] * B[2];
  cplx c3 = A[2] * B[1] + A[3] * B[3];
  C[0] = c0; C[1] = c1; C[2] = c2; C[3] = c3;
}

int oracle_modes_evolve(const oracle_params *p, double g00, double g11, double g22,
                        double dt, long n_steps, int n_modes, const int *qx,
                        const int *qy, const cplx *amps, int n_pts, const int *ix,
                        const int *iy, cplx *out) {
  return oracle_modes_evolve_scheme(p, g00, g11, g22, dt, n_steps, ORACLE_SCHEME_II, n_modes,
                                    qx, qy, amps, n_pts, ix, iy, out);
}

int oracle_modes_evolve_scheme(const oracle_params *p, double g00, double g11, double g22,
                               double dt, long n_steps, int scheme, int n_modes,
                               const int *qx, const int *qy, const cplx *amps, int n_pts,
                               const int *ix, const int *iy, cplx *out) {
  if (check_params(p) || p->pml_wx || p->pml_wy) return -1;
  if (scheme != ORACLE_SCHEME_II && scheme != ORACLE_SCHEME_II_SYMMETRIC) return -1;
  if (!(g00 > 0.0 && g11 > 0.0 && g22 > 0.0) || n_steps < 0) return -1;
  const double a1 = p->c * sqrt(g00 / g11), a2 = p->c * sqrt(g00 / g22);
  const double me = p->mass * p->c * p->c * sqrt(g00);
  cplx U[4];
  exp_pauli(0.0, 0.0, -0.5 * I * dt * me, U);
  for (int s = 0; s < n_pts; s++) out[2 * s] = out[2 * s + 1] = 0.0;
  for (int m = 0; m < n_modes; m++) {
    if (qx[m] < 0 || qx[m] >= p->nx || qy[m] < 0 || qy[m] >= p->ny) return -1;
    /* the x sub-step runs over dt (Scheme II) or twice over dt/2 around y (symmetric) */
    const double hx_dt = scheme == ORACLE_SCHEME_II ? dt : 0.5 * dt;
    double tx = hx_dt * xi_of(qx[m], p->nx, p->ax), ty = dt * xi_of(qy[m], p->ny, p->ay);
    cplx Kx[4] = {a1 * cos(tx) + (1.0 - a1), -I * a1 * sin(tx), -I * a1 * sin(tx),
                  a1 * cos(tx) + (1.0 - a1)};
    cplx Ky[4] = {a2 * cos(ty) + (1.0 - a2), -a2 * sin(ty), a2 * sin(ty),
                  a2 * cos(ty) + (1.0 - a2)};
    cplx T[4], tmp[4];
    mat2_mul(Kx, U, tmp);
    mat2_mul(Ky, tmp, T);
    if (scheme == ORACLE_SCHEME_II_SYMMETRIC) {
      mat2_mul(Kx, T, tmp);
      memcpy(T, tmp, sizeof(T));
    }
    mat2_mul(U, T, T);
    cplx v0 = amps[2 * m], v1 = amps[2 * m + 1];
    for (long s = 0; s < n_steps; s++) {
      cplx w0 = T[0] * v0 + T[1] * v1;
      cplx w1 = T[2] * v0 + T[3] * v1;
      v0 = w0;
      v1 = w1;
    }
    const double hx = 2.0 * p->ax / p->nx, hy = 2.0 * p->ay / p->ny;
    const double kx = xi_of(qx[m], p->nx, p->ax), ky = xi_of(qy[m], p->ny, p->ay);
    for (int s = 0; s < n_pts; s++) {
      /* x_i + a = i h */
      cplx e = cexp(I * (kx * (ix[s] * hx) + ky * (iy[s] * hy)));
      out[2 * s] += v0 * e;
      out[2 * s + 1] += v1 * e;
    }
  }
  return 0;
}
