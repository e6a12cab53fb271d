// Internal declarations shared by the library's translation units (not part of the ABI).
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <string>

#include "common.cuh"
#include "line_pass.cuh"

namespace dgb {

// Sets the text that dirac_last_error(NULL) returns (errors without a context).
void set_global_error(const std::string& msg);

// Enqueues one fused line pass (MODE_STEP or MODE_DERIV). opt selects the CTA shape:
// 0 = about 256 threads per CTA, 1 = 512 threads, 2 = the persistent prefetching
// variant (complex64 step mode, lines of 256..4096 points; otherwise as 1).
template <typename T>
cudaError_t launch_line_pass(const LinePassArgs<T>& a, int mode, int opt, cudaStream_t st);
// Every step of a batch tick of one class in one persistent launch (complex64, square
// grids, 256..2048-point lines; cudaErrorInvalidValue otherwise).
template <typename T>
cudaError_t launch_line_pass_tick(const LinePassArgs<T>& a, cudaStream_t st);
// Elements per thread (8 or 16) the line pass uses for line length L; the twiddle table
// of that axis must be built for the same value.
template <typename T>
int line_pass_radix(int L);
// The alternative radix schedule the autotuner may pick for lines of L points (0: none);
// launch options 3 and 4 run it, with a twiddle table of that radix in tw_alt.
template <typename T>
int line_pass_radix_alt(int L);
// Debug builds (-DDIRAC_DEBUG=1): read and clear the index-check flags of the line-pass
// translation units; nonzero when a check failed. Always 0 in release builds.
int dgb_debug_flag_c64();
int dgb_debug_flag_c128();
inline int dgb_debug_bounds() { return dgb_debug_flag_c64() | dgb_debug_flag_c128(); }

// ---- FP64 precompute (precompute.cu)
// a1, a2, meff, w and the two log fields (packed as a complex128 spinor (f1, f2)) from the
// metric; g == nullptr means 1.
cudaError_t launch_metric_fields(const double* g00, const double* g11, const double* g22,
                                 int n, double c, double mass, int conn, double* a1,
                                 double* a2, double* meff, double* w, Q4<double>* logs,
                                 cudaStream_t st);
// Omega_x, Omega_y (normal layout) from the x derivative (transposed layout [nx][ny]) and
// the y derivative (normal layout) of the log fields.
cudaError_t launch_omega(const Q4<double>* dxT, const Q4<double>* dy, int nx, int ny,
                         double fac, double* omx, double* omy, cudaStream_t st);
// 1/S for grid indices of one axis (Sec. 3 profiles), S = 1 + exp(i theta) Sigma~: the real
// part into sinv and, if sinv_im is not null, the imaginary part (else theta must be 0).
cudaError_t launch_pml(int n, double a, int width, int type, double sigma0, double theta,
                       double* sinv, double* sinv_im, cudaStream_t st);
// beta1 = a1/S1 - 1 (normal layout), beta2T = a2/S2 - 1 (transposed layout), in T; with
// complex stretching (sxinv_im, syinv_im not null) the imaginary parts go to beta1_im,
// beta2T_im.
template <typename T>
cudaError_t launch_beta(const double* a1, const double* a2, const double* sxinv,
                        const double* syinv, const double* sxinv_im, const double* syinv_im,
                        int nx, int ny, T* beta1, T* beta2T, T* beta1_im, T* beta2T_im,
                        cudaStream_t st);
// Half-step matrices for dt: U (normal layout), U and U^2 (transposed layout) and, if
// u2_n is not null, U^2 in the normal layout, stored as (c0 - 1, c1, c2, c3) in T.
template <typename T>
cudaError_t launch_halfstep(const double* a1, const double* a2, const double* meff,
                            const double* omx, const double* omy, int nx, int ny, double dt,
                            Q4<T>* u_n, Q4<T>* u_t, Q4<T>* u2_t, Q4<T>* u2_n,
                            cudaStream_t st);
// Per-axis tables: per-pass twiddle blocks (layout in line_pass.cuh); step multipliers
// ((cos(dt xi) - 1)/n, sin(dt xi)/n) as hi/lo pairs; derivative multipliers xi/n.
template <typename T>
cudaError_t launch_twiddles(int n, int e, Cx<T>* tw, cudaStream_t st);
template <typename T>
cudaError_t launch_step_mult(int n, double a, double dt, Q4<T>* mult, cudaStream_t st);
template <typename T>
cudaError_t launch_perm1024(const Q4<T>* src, Q4<T>* dst, cudaStream_t st);
template <typename T>
cudaError_t launch_deriv_mult(int n, double a, Q4<T>* mult, cudaStream_t st);

// Half step with static potentials: general complex U and U^2 per point (normal layout,
// two Q4 per point holding U - I: (d00, u01), (u10, d11)); V, Ax, Ay may be null (0).
template <typename T>
cudaError_t launch_halfstep_general(const double* a1, const double* a2, const double* meff,
                                    const double* omx, const double* omy, const double* V,
                                    const double* Ax, const double* Ay, int nx, int ny,
                                    double dt, Q4<T>* ug, Q4<T>* ug2, cudaStream_t st);
// psi <- U psi for such a general U.
template <typename T>
cudaError_t launch_apply_ug(Q4<T>* psi, const Q4<T>* ug, size_t n, cudaStream_t st);

// ---- unsplit polynomial scheme (unsplit.cu)
// psi <- U psi at every point (normal layout).
template <typename T>
cudaError_t launch_apply_u(Q4<T>* psi, const Q4<T>* u, size_t n, cudaStream_t st);
// out = alpha (b1 sigma_x dx + b2 sigma_y dy) + beta prev (prev may be null); acc +=
// gamma out (acc may be null); b^j = a^j / S^j from the FP64 fields (complex when the
// imaginary parts of 1/S are given); all normal layout.
template <typename T>
cudaError_t launch_unsplit_combine(const Q4<T>* dx, const Q4<T>* dy, const double* a1,
                                   const double* a2, const double* sxinv, const double* syinv,
                                   const double* sxinv_im, const double* syinv_im, int nx,
                                   int ny, double ar, double ai, const Q4<T>* prev,
                                   double beta, double gr, double gi, Q4<T>* out, Q4<T>* acc,
                                   cudaStream_t st);
// out = c in.
template <typename T>
cudaError_t launch_scale(Q4<T>* out, const Q4<T>* in, double cr, double ci, size_t n,
                         cudaStream_t st);
// Per-block maxima of |b1|, |b2| into partials[2 * n_blocks].
cudaError_t launch_max_b(const double* a1, const double* a2, const double* sxinv,
                         const double* syinv, const double* sxinv_im, const double* syinv_im,
                         int nx, int ny, double* partials, int n_blocks, cudaStream_t st);
// Krylov building blocks (Scheme I). Partial inner products <V_i, w> (i < count) in
// FP64: partials[2 (i n_blocks + b)] (re, im) per block b; V is a device array of count
// pointers.
template <typename T>
cudaError_t launch_multi_dot(const Q4<T>* const* V, int count, const Q4<T>* w, size_t n,
                             double* partials, int n_blocks, cudaStream_t st);
// out += sum_i coef_i V_i with complex FP64 coef (device array of 2 count doubles).
template <typename T>
cudaError_t launch_multi_axpy(Q4<T>* out, const Q4<T>* const* V, const double* coef, int count,
                              size_t n, cudaStream_t st);
// out = a x + b y.
template <typename T>
cudaError_t launch_axpby(Q4<T>* out, double a, const Q4<T>* x, double b, const Q4<T>* y,
                         size_t n, cudaStream_t st);
// J_0(x) .. J_n(x) into out[0..n] (host, FP64); false for x < 0 or n < 0.
bool bessel_j_series(double x, int n, double* out);

// Tiled transpose of a [rows][cols] array of Q4<T> into [cols][rows].
template <typename T>
cudaError_t launch_transpose(const Q4<T>* in, Q4<T>* out, int rows, int cols, cudaStream_t st);

// ---- state conversion and observables (observables.cu)
// psi[k] = (p1[k], p2[k]) from a [2][n] complex128 array, and back.
template <typename T>
cudaError_t launch_pack(const double* src, Q4<T>* psi, size_t n, cudaStream_t st);
template <typename T>
cudaError_t launch_unpack(const Q4<T>* psi, double* dst, size_t n, cudaStream_t st);
// Per-block FP64 partial sums {norm, norm_gamma, e_re, e_im} into partials[blocks][4]
// and the density map (if not null). dx and dy may be null (no energy); the static
// potentials V, Ax, Ay may be null (0).
template <typename T>
cudaError_t launch_observables(const Q4<T>* psi, const Q4<T>* dx, const Q4<T>* dy,
                               const double* a1, const double* a2, const double* meff,
                               const double* w, const double* omx, const double* omy,
                               const double* V, const double* Ax, const double* Ay,
                               size_t n, double* density, double* partials, int blocks,
                               cudaStream_t st);
cudaError_t launch_reduce_partials(const double* partials, int blocks, double scale,
                                   double* result, cudaStream_t st);
int observables_blocks(size_t n);

}  // namespace dgb
