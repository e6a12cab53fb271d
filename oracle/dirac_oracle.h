/*
 * FP64 CPU oracle for the direction-split explicit pseudospectral step ("Numerical
 * Scheme II") of Antoine, Fillion-Gourdeau, Lorin and McLean, "Pseudospectral
 * computational methods for the time-dependent Dirac equation in static curved
 * spaces" (arXiv:1909.02894), 2D, two-component spinor.
 *
 * TEST INFRASTRUCTURE. Only the test suite, the smoke check and the CPU-baseline leg of
 * the benchmark may load this library. The product path never calls it. It shares no
 * code, header, table or constant with the CUDA path.
 *
 * Array conventions: real fields are [ny][nx] doubles, x fastest. A spinor is
 * [2][ny][nx] double complex (interleaved re, im), component-major.
 * Every function returns 0 on success and a negative value on invalid arguments.
 *
 * Parity status: every function below is pinned by the oracle tests, including the
 * absorbing-layer profile (point by point against the Sec. 3 closed forms) and the
 * covariant spin connection (w H Hermitian: the weighted energy is real; a dense
 * curved-space Hamiltonian on a tiny grid).
 */
#ifndef DIRAC_ORACLE_H
#define DIRAC_ORACLE_H

#include <complex.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORACLE_CONN_COVARIANT = 0, ORACLE_CONN_PAPER_2D = 1, ORACLE_CONN_NONE = 2 };

typedef struct {
  int nx, ny;          /* powers of two (Sec. 5 needs N even; the radix-2 FFT needs 2^k) */
  double ax, ay;       /* domain [-ax, ax) x [-ay, ay)                                   */
  double mass, c;      /* m and the speed of light                                       */
  int conn;            /* spin-connection reading, ORACLE_CONN_*                         */
  int pml_wx, pml_wy;  /* absorbing-layer width in grid points per side, 0 = none        */
  int pml_type;        /* 1..6 = the paper's types I..VI (Sec. 3)                        */
  double sigma0, theta;
  /* static electromagnetic potentials (Sec. 2, the F of the curved-space Hamiltonian):
   * [ny][nx] fields, NULL = 0. V is the scalar potential energy, entering H as + V I;
   * Ax, Ay are the vector potential times the charge, entering H as
   * - sum_j a^j A_j sigma_j (from alpha.(-i grad - e A)). They act through U only. */
  const double *V, *Ax, *Ay;
} oracle_params;

/* Forward DFT psi~_p = sum_k psi_k exp(-2 pi i p k / n), inverse with 1/n (Sec. 5). */
int oracle_fft(int n, double complex *x, int inverse);

/* Spectral derivative [[d_axis]] of a complex [ny][nx] field (Sec. 5, eq. "trick"). */
int oracle_deriv(const oracle_params *p, int axis, const double complex *in,
                 double complex *out);

/* Coefficient fields (each [ny][nx]): a1, a2, meff, w, omega_x, omega_y (real) and
 * b1 = a1/S1, b2 = a2/S2 (complex; real when theta = 0). NULL g means g = 1. */
int oracle_coefficients(const oracle_params *p, const double *g00, const double *g11,
                        const double *g22, double *a1, double *a2, double *meff,
                        double *w, double *omx, double *omy, double complex *b1,
                        double complex *b2);

/* Half-step matrix U = exp(-i dt/2 [meff sigma_z + F]) per point as 4 complex entries
 * [u00, u01, u10, u11] per point: out is [ny][nx][4] double complex. */
int oracle_half_step(const oracle_params *p, const double *g00, const double *g11,
                     const double *g22, double dt, double complex *u);

enum { ORACLE_SCHEME_II = 0, ORACLE_SCHEME_II_SYMMETRIC = 1 };

/* n_steps of Scheme II from psi (in place): U, x-substep, y-substep, U per step. */
int oracle_run(const oracle_params *p, const double *g00, const double *g11,
               const double *g22, double dt, long n_steps, double complex *psi);

/* The same with a choice of sub-step order: ORACLE_SCHEME_II as printed (Sec. 5.2), or
 * its symmetric (Strang) ordering U, x-substep over dt/2, y-substep over dt, x-substep
 * over dt/2, U per step: the symmetric decomposition of Sec. 3 (eq. op_flat) applied to
 * the direction split as well. */
int oracle_run_scheme(const oracle_params *p, const double *g00, const double *g11,
                      const double *g22, double dt, long n_steps, int scheme,
                      double complex *psi);

/* The unsplit middle-step operator of Sec. 4.2 (eqs. op_split_cn, op_split_poly) with
 * alpha(x) = a(x).alpha (eq. alpha_form), the absorbing layer's a^j -> b^j = a^j/S^j
 * (Sec. 3) and the spectral derivative (eq. trick):
 *   A psi = - sum_j b^j sigma_j [[d_j]] psi      (in, out: [2][ny][nx]; may not alias). */
int oracle_apply_A(const oracle_params *p, const double *g00, const double *g11,
                   const double *g22, const double complex *in, double complex *out);

/* Bessel functions J_0(x) .. J_n(x) (x >= 0), the Chebyshev coefficients of exp. */
int oracle_bessel_j(double x, int n, double *j);

enum { ORACLE_POLY_TAYLOR = 0, ORACLE_POLY_CHEBYSHEV = 1 };

/* n_steps of the polynomial scheme (Sec. 5, eq. poly): U, then
 * psi <- sum_q a_q P_q(dt A) psi (degree `order`), then U. TAYLOR: a_q P_q(z) = z^q / q!.
 * CHEBYSHEV: with H = i dt A and a bound R >= |spectrum of H| (R = dt sum_j max|b^j| pi/h_j),
 * exp(dt A) = exp(-i H) ~ sum_q (2 - delta_q0) (-i)^q J_q(R) T_q(H / R). */
int oracle_run_poly(const oracle_params *p, const double *g00, const double *g11,
                    const double *g22, double dt, long n_steps, int family, int order,
                    double complex *psi);

/* n_steps of the Crank-Nicolson scheme (Scheme I, Sec. 5.1 eq. cn): U, then
 * G psi* = G~ psi with G = I - (dt/2) A, G~ = I + (dt/2) A (A as in oracle_apply_A), then
 * U. The linear system is solved by restarted GMRES (Sec. 5.1 names Krylov solvers) with
 * modified Gram-Schmidt in FP64, from psi as initial guess, until the residual is below
 * tol times |G~ psi|. iters (may be NULL) receives the total Arnoldi steps.
 * Returns -2 if a solve does not converge within max_restarts cycles of `restart`. */
int oracle_run_cn(const oracle_params *p, const double *g00, const double *g11,
                  const double *g22, double dt, long n_steps, double tol, int restart,
                  int max_restarts, long *iters, double complex *psi);

/* obs = {norm, norm_gamma, energy_re, energy_im}; density may be NULL. */
int oracle_observables(const oracle_params *p, const double *g00, const double *g11,
                       const double *g22, const double complex *psi, double *obs,
                       double *density);

/* Constant coefficients (scalar g00, g11, g22, no absorbing layer): each plane wave
 * is an eigenfunction of every sub-step, so the scheme's result after n_steps is a
 * per-mode 2x2 matrix power. modes: qx[k], qy[k] FFT indices and amps[2k], amps[2k+1]
 * the two components; evaluated at grid points (ix[s], iy[s]) into out[2s], out[2s+1]. */
int oracle_modes_evolve(const oracle_params *p, double g00, double g11, double g22,
                        double dt, long n_steps, int n_modes, const int *qx,
                        const int *qy, const double complex *amps, int n_pts,
                        const int *ix, const int *iy, double complex *out);
/* The same for either sub-step order (ORACLE_SCHEME_*). */
int oracle_modes_evolve_scheme(const oracle_params *p, double g00, double g11, double g22,
                               double dt, long n_steps, int scheme, int n_modes,
                               const int *qx, const int *qy, const double complex *amps,
                               int n_pts, const int *ix, const int *iy, double complex *out);

/* Number of OpenMP threads the oracle uses (1 without OpenMP). */
int oracle_threads(void);

/* Sets the number of OpenMP threads for later calls (n >= 1; ignored without OpenMP). */
int oracle_set_threads(int n);

#ifdef __cplusplus
}
#endif
#endif
