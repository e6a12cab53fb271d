/*
 * dirac.h -- C ABI of the GB300 (sm_103a) implementation of the direction-split explicit
 * pseudospectral step ("Numerical Scheme II", Sec. 5.2) for the 2D time-dependent Dirac
 * equation in a static curved space, from Antoine, Fillion-Gourdeau, Lorin, McLean,
 * "Pseudospectral computational methods for the time-dependent Dirac equation in static
 * curved spaces" (arXiv:1909.02894).
 *
 * The problem (Sec. 2.2, Sec. 5, Sec. 6 for the 2D two-component form):
 *   i d_t psi = H psi,  H = -i sum_{j=x,y} a^j(x) sigma_j (d_j + Omega_j(x)) + meff(x) sigma_z
 * on the periodic grid x_k = -a + k h, h = 2a/N (Sec. 5), with a diagonal static metric
 * ds^2 = g00 dt^2 - g11 dx^2 - g22 dy^2 giving a^j = c sqrt(g00/g_jj),
 * meff = m c^2 sqrt(g00), and absorbing layers that replace a^j by b^j = a^j / S^j(x^j)
 * (Sec. 3, and Sec. 5.2 "replacing a^i by a^i/S^i").
 *
 * One time step dt (Sec. 4.2 eq. op_split_curved with Sec. 5.2 eq. poly_mod and
 * second_scheme):
 *   S1  psi <- U psi,  U = exp(-i dt/2 [meff sigma_z + F]),  F = -i sum_j a^j Omega_j sigma_j
 *   S2  rows:    Xi = F_x^-1[exp(-i dt xi sigma_x) F_x psi],  psi <- b^1 Xi + (1 - b^1) psi
 *   S3  columns: Xi = F_y^-1[exp(-i dt xi sigma_y) F_y psi],  psi <- b^2 Xi + (1 - b^2) psi
 *   S4  psi <- U psi
 *
 * Conventions shared by every call:
 *   - Real fields are [ny][nx] doubles, x fastest (the paper's vector ordering, App. C).
 *   - A spinor crossing the ABI is [2][ny][nx] complex128 (interleaved re, im), component
 *     major, in both precisions; DIRAC_C64 contexts convert on the device.
 *   - The caller owns every array it passes; create/set_state copy what they need, so the
 *     caller may free its arrays when the call returns. The context owns all of its device
 *     memory until dirac_destroy.
 *   - Every call returns a dirac_status; no exception or exit crosses the ABI.
 *     dirac_last_error() gives the detail of the last failure on a context.
 *   - Calls on one context are not thread-safe; distinct contexts are independent.
 */
#ifndef DIRAC_H
#define DIRAC_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dirac_ctx dirac_ctx;
typedef struct dirac_batch dirac_batch;

typedef enum {
  DIRAC_OK = 0,
  DIRAC_EINVAL = 1,       /* invalid argument (sizes, pointers, non-positive g, dt <= 0) */
  DIRAC_ENOMEM = 2,       /* device or host allocation failed                           */
  DIRAC_EUNSUPPORTED = 3, /* valid but outside this build (e.g. theta != 0 in complex64) */
  DIRAC_ECUDA = 4,        /* a CUDA runtime call failed                                   */
  DIRAC_ETIMEOUT = 5,     /* a bounded device wait ran out                                */
  DIRAC_ENONFINITE = 6,   /* the state holds NaN or Inf                                   */
  DIRAC_ESTATE = 7,       /* call out of order (e.g. step before set_state)               */
  DIRAC_ENOCONV = 8       /* Scheme I: the Krylov solver did not reach its tolerance      */
} dirac_status;

typedef enum { DIRAC_C64 = 0, DIRAC_C128 = 1 } dirac_precision;

/* Order of the sub-steps within one time step (Sec. 5.2, Scheme II): SCHEME_II is the
 * printed order U, x, y, U (first order in time, Prop. 5.2); SCHEME_II_SYMMETRIC runs the
 * x sub-step twice over dt/2 around the y sub-step (U, x/2, y, x/2, U): the symmetric
 * (Strang) decomposition the paper's time discretization uses in flat space (Sec. 3,
 * eq. op_flat) carried over to the direction split; second order in time in flat space. The symmetric order costs three line passes per step. */
typedef enum {
  DIRAC_SCHEME_II = 0,
  DIRAC_SCHEME_II_SYMMETRIC = 1,
  /* The polynomial scheme (Sec. 4.2 eq. op_split_poly, Sec. 5 eq. poly): U, then the
   * unsplit middle step psi <- sum_q a_q P_q(dt A) psi with A = -sum_j b^j sigma_j [[d_j]]
   * (eq. alpha_form; b^j = a^j/S^j), then U. TAYLOR: a_q P_q(z) = z^q/q!. CHEBYSHEV:
   * exp(dt A) = exp(-i H), H = i dt A, expanded as sum_q (2 - delta_q0) (-i)^q J_q(R)
   * T_q(H/R) with R = dt sum_j max|b^j| pi/h_j. Explicit, hence only conditionally stable
   * (Sec. 5: Taylor is usually unstable); the degree is set by dirac_set_poly_degree.
   * Each term costs two derivative passes, a transpose and a pointwise combine. */
  DIRAC_SCHEME_POLY_TAYLOR = 2,
  DIRAC_SCHEME_POLY_CHEBYSHEV = 3,
  /* Scheme I (Sec. 5.1 eq. cn): U, then G psi* = G~ psi with G = I + dt/2 alpha.[[grad]]
   * = I - dt/2 A and G~ = I + dt/2 A (A as above), then U. The linear system is solved by
   * restarted GMRES (Sec. 5.1: "a Krylov iteration solver") from psi, with FP64 inner
   * products and Hessenberg arithmetic; see dirac_set_krylov. Unconditionally stable in
   * flat space (a Cayley transform, Prop. 5.1), second order in time there. */
  DIRAC_SCHEME_CRANK_NICOLSON = 4
} dirac_scheme;

/* Spin connection Omega_j (Sec. 2.2). COVARIANT: Omega_j = 1/2 d_j ln(w a^j) with
 * w = sqrt(g11 g22 / g00) (= sqrt|g| g^00, the weight of the conserved norm, eq. l2gamma).
 * PAPER_2D: Omega_j = 1/2 d_j Phi with g00 = exp(2 Phi), as printed for Experiment 3.
 * NONE: Omega_j = 0. d_j is the spectral derivative of the sampled field (eq. trick),
 * real part. */
typedef enum { DIRAC_CONN_COVARIANT = 0, DIRAC_CONN_PAPER_2D = 1, DIRAC_CONN_NONE = 2 } dirac_connection;

/* Grid sizes: powers of two, 16 <= nx, ny <= 4096 (Sec. 5 needs N even). */
typedef struct { int nx, ny; } dirac_grid;

/* Domain [-ax, ax) x [-ay, ay), ax, ay > 0 (Sec. 5). */
typedef struct { double ax, ay; } dirac_domain;

/* Diagonal static metric (eq. alpha_form needs alpha^j = a^j(x) alpha^j). Host arrays
 * [ny][nx], entries > 0; a NULL pointer means the constant 1. g12 = 0. */
typedef struct {
  const double *g00, *g11, *g22;
  dirac_connection conn;
} dirac_metric;

/* Absorbing layer (Sec. 3): width_x/width_y grid points per side (0 = none, < N/2),
 * type 1..6 = the paper's profiles I..VI, sigma0 = Sigma_0, theta = stretching angle.
 * theta != 0 (S = 1 + exp(i theta) Sigma~) makes b complex: supported in complex128 (the
 * passes add i Im(b - 1) D); complex64 contexts return DIRAC_EUNSUPPORTED, as do batches
 * of such contexts. */
typedef struct {
  int width_x, width_y;
  int type;
  double sigma0, theta;
} dirac_absorber;

/* Observables (Sec. 2.2 eq. l2gamma, Prop. 5.3's discrete l2 norm, Sec. 6.2 density):
 *   norm       = hx hy sum |psi|^2
 *   norm_gamma = hx hy sum w |psi|^2
 *   energy     = hx hy sum w Re(psi^dagger H psi), energy_imag its imaginary part,
 *                with H as above without absorbing layers.
 * All reductions are accumulated in FP64. */
typedef struct {
  double norm, norm_gamma, energy, energy_imag;
} dirac_obs;

/* Creates a context: validates the arguments, copies the metric to the device and
 * precomputes a^j, meff, w, Omega_j, b^j and the layer profile in FP64 on the GPU.
 * metric may be NULL (flat space), absorber may be NULL (no layer). c > 0, mass real.
 * cuda_stream: a cudaStream_t to launch on, or NULL for a stream the context creates.
 * On success *out holds the context; on failure *out is NULL. */
dirac_status dirac_create(const dirac_grid *grid, const dirac_domain *domain,
                          const dirac_metric *metric, double mass, double c,
                          const dirac_absorber *absorber, dirac_precision precision,
                          void *cuda_stream, dirac_ctx **out);

/* Sets the state from psi, [2][ny][nx] complex128. on_device = 0: psi is host memory,
 * copied before return; on_device = 1: psi is device memory, read on the context's
 * stream (the caller keeps it alive until the stream reaches this point). */
dirac_status dirac_set_state(dirac_ctx *ctx, const double *psi, int on_device);

/* Writes the state to psi_out, [2][ny][nx] complex128, host (on_device = 0, returns when
 * the copy is done) or device (on_device = 1, enqueued on the context's stream). */
dirac_status dirac_get_state(dirac_ctx *ctx, double *psi_out, int on_device);

/* Advances the state by n_steps steps of size dt (n_steps >= 0, dt > 0), enqueued on the
 * context's stream without host synchronisation. Consecutive steps merge the trailing
 * U of one step with the leading U of the next (U U, the same matrix in closed form).
 * A new dt recomputes U and the k-space phase tables in FP64 first. */
dirac_status dirac_step(dirac_ctx *ctx, long n_steps, double dt);

/* Computes the observables (synchronises the stream). density_or_NULL, if not NULL, is a
 * host [ny][nx] array that receives |psi_1|^2 + |psi_2|^2. Returns DIRAC_ENONFINITE
 * (after filling *out) if the norm is not finite. */
dirac_status dirac_observables(dirac_ctx *ctx, dirac_obs *out, double *density_or_NULL);

/* Blocks until all work enqueued on the context's stream has finished. Returns
 * DIRAC_ETIMEOUT if a bounded wait inside a kernel ran out since the last check (the
 * state is then not valid); dirac_get_state to the host and dirac_observables check the
 * same flag. */
dirac_status dirac_synchronize(dirac_ctx *ctx);

/* Text of the last error on ctx (or of the last failed dirac_create when ctx is NULL).
 * The string stays valid until the next call on the same context. */
const char *dirac_last_error(const dirac_ctx *ctx);

/* Releases the context and all its device memory. NULL is allowed. */
void dirac_destroy(dirac_ctx *ctx);

/* Selects the time-step scheme of later dirac_step calls (dirac_scheme; the default is
 * DIRAC_SCHEME_II). The symmetric order needs two more device arrays (x-pass multipliers
 * for dt/2 and U^2 in the normal layout), allocated on the next dirac_step. Contexts
 * with another scheme than DIRAC_SCHEME_II cannot join a batch (dirac_batch_submit returns
 * DIRAC_EUNSUPPORTED). DIRAC_EINVAL for other values. */
dirac_status dirac_set_scheme(dirac_ctx *ctx, int scheme);

/* Static electromagnetic potentials (Sec. 2: the F of the curved-space Hamiltonian),
 * host [ny][nx] FP64 arrays copied by the call; NULL means 0 (all NULL removes them).
 * V is the scalar potential energy, entering H as + V I; Ax, Ay are the vector potential
 * times the charge, entering H as - sum_j a^j A_j sigma_j (from alpha.(-i grad - e A)).
 * They act through the half-step matrix U, which becomes a general complex 2x2 matrix per
 * point, applied by its own pointwise kernel (U before the first pass of a call, U^2
 * between steps, U after the last) instead of inside the line passes. The energy that
 * dirac_observables reports includes them (H gains V - sum_j a^j A_j sigma_j). Contexts
 * with potentials cannot join a batch. DIRAC_EINVAL for non-finite values. */
dirac_status dirac_set_potentials(dirac_ctx *ctx, const double *V, const double *Ax,
                                  const double *Ay);

/* Degree N_p of the polynomial schemes' middle step (1..256; default 8). The polynomial
 * schemes use three more state-sized device arrays, allocated on the next dirac_step.
 * DIRAC_EINVAL for other values. */
dirac_status dirac_set_poly_degree(dirac_ctx *ctx, int degree);

/* Krylov solver of Scheme I: relative residual tolerance tol (|G~ psi - G psi*| <= tol
 * |G~ psi|; 0 = default: 1e-14 for complex128, 3e-7 for complex64), Krylov dimension
 * `restart` (1..100, default 20; restart + 1 state-sized device arrays, allocated on the
 * next dirac_step) and at most max_restarts restarts per step (default 100). A step whose
 * solve does not converge returns DIRAC_ENOCONV and leaves the state invalid. */
dirac_status dirac_set_krylov(dirac_ctx *ctx, double tol, int restart, int max_restarts);

/* Total Arnoldi steps of Scheme I on this context since its creation. */
long dirac_krylov_iterations(const dirac_ctx *ctx);

/* CTA shape of the two fused passes (each pass: FFT along a line, k-space multiply,
 * inverse FFT, combine, transposed store): 256 selects the smaller and 512 the larger of
 * the pass's two shapes for its line length (complex64: about 256 and 512 threads per
 * CTA; complex128: 1 to 4 lines per CTA, 32 to 512 threads), 1024 the persistent
 * prefetching variant (complex64, lines of 256..4096 points; one CTA per SM streams the
 * next lines into shared memory while it transforms the current ones); 0 = the default
 * (complex64: persistent for lines of 1024 points or more, the smaller shape for 128-
 * and 256-point lines, else the larger; complex128: the smaller shape for 1024-point
 * lines and lines of 128 points or fewer, else the larger). 64- and 128-point lines take
 * 2 or 16 lines per CTA; lines of 32 points or fewer and 4096-point lines have one shape
 * only. 256 or 512 plus
 * DIRAC_LAUNCH_ALT_RADIX selects the other radix schedule of the FFT passes, where the line
 * length has one: complex64 lines of 256..4096 points in radix-16 instead of radix-8
 * passes, complex128 lines of 256..2048 points in radix-8 instead of radix-16 passes, each
 * with its own lines-per-CTA pair (about 256 | 512 threads); elsewhere the flag is ignored.
 * Used by the autotuner. DIRAC_EINVAL for other values. */
#define DIRAC_LAUNCH_ALT_RADIX 0x10000
dirac_status dirac_set_launch(dirac_ctx *ctx, int threads_x_pass, int threads_y_pass);

/* Autotuner: times every CTA shape and radix schedule of the x and the y pass (the
 * dirac_set_launch values; reps launches each, CUDA
 * events on the context's stream, output to scratch memory so the state is unchanged),
 * applies the fastest with dirac_set_launch and returns it in *threads_x, *threads_y.
 * The state must be set; synchronises the stream. */
dirac_status dirac_autotune(dirac_ctx *ctx, int reps, int *threads_x, int *threads_y);

/* Test hook for failure detection: in the next dirac_step -- or, for a context submitted
 * to a batch, in the first tick that steps it -- the persistent pass's bulk-copy waits
 * expect 16 bytes that never arrive, so each wait runs out after its bound (about 1.5 s),
 * the kernel returns early and the next synchronising call (dirac_synchronize, or
 * dirac_batch_poll / dirac_batch_synchronize) reports DIRAC_ETIMEOUT; the context stays
 * usable (set the state again). No effect on the other launch shapes. */
dirac_status dirac_test_timeout_next_step(dirac_ctx *ctx);

/* Host-side fault injection for failure-detection tests (no GPU fault involved): with the
 * environment variable DIRAC_FAULT=alloc:N (N >= 1) set when dirac_create runs, the N-th
 * device allocation of that context fails as if the device were out of memory; the call
 * frees everything it had allocated and returns DIRAC_ENOMEM, and later contexts (created
 * without the variable) are unaffected. Any other value, or none, disables it. */

/* Number of kernel launches this context has enqueued so far (for accounting). */
long dirac_launch_count(const dirac_ctx *ctx);

/* Device bytes a context of this size and precision can hold (state, coefficients,
 * half-step matrices, host-transfer staging, observables scratch). 0 for bad input. */
size_t dirac_footprint_bytes(const dirac_grid *grid, dirac_precision precision);

/* ---- Batched stepping of many independent contexts (any mix of grid sizes).
 * Contexts of the same grid size form a class; one tick advances every active context
 * by up to steps_per_tick steps: per step and class, one x-pass and one y-pass launch
 * over all of that class's active contexts. With the environment variable
 * DIRAC_BATCH_TICK=1 set at dirac_batch_create, a class of square complex64 grids with
 * 256..2048-point lines whose passes run the persistent pass takes its whole tick in ONE
 * persistent launch instead: work items (step, pass, context, line group) come from a
 * queue, and each waits -- bounded, DIRAC_ETIMEOUT when the bound runs out -- until the
 * context's previous pass is finished (the same results; 4-8% slower per class on the
 * 256-instance mix, hence not the default). The classes run on parallel branches of a
 * CUDA graph captured once per class layout and replayed. Each context computes
 * exactly what dirac_step(ctx, n_steps, dt) computes (Sec. 5.2 Scheme II); a submitted
 * context belongs to the batch until it is released and must not be stepped, read or
 * destroyed meanwhile. Contexts must have the batch's precision. */

/* Creates a batch with a device-memory budget (bytes of dirac_footprint_bytes summed
 * over the submitted contexts), on cuda_stream (NULL = a stream of its own). */
dirac_status dirac_batch_create(size_t hbm_budget_bytes, dirac_precision precision,
                                void *cuda_stream, int steps_per_tick, dirac_batch **out);

/* Admits a context (its state must be set) for n_steps steps of size dt; *slot receives
 * its handle. DIRAC_ENOMEM when the budget would be exceeded (retry after a release). */
dirac_status dirac_batch_submit(dirac_batch *batch, dirac_ctx *inst, long n_steps, double dt,
                                int *slot);

/* Enqueues n_ticks ticks (host returns after enqueueing; the tables of one tick are
 * prepared while the previous one runs). */
dirac_status dirac_batch_run(dirac_batch *batch, int n_ticks);

/* *done = 1 once every step of the slot's context has finished on the device.
 * DIRAC_ETIMEOUT if a bounded device wait ran out in a batched pass: every context in the
 * batch at that moment is then marked failed (its state is not valid), stops stepping,
 * and its poll keeps returning DIRAC_ETIMEOUT until it is released; the batch itself keeps
 * working for contexts submitted afterwards (set their state again first). */
dirac_status dirac_batch_poll(dirac_batch *batch, int slot, int *done);

/* Returns the slot (and its budget); a context still running is cancelled after the
 * steps already enqueued. The context is the caller's again. */
dirac_status dirac_batch_release(dirac_batch *batch, int slot);

/* Waits for all enqueued ticks; DIRAC_ETIMEOUT as for dirac_batch_poll. */
dirac_status dirac_batch_synchronize(dirac_batch *batch);

/* Number of contexts still stepping. */
int dirac_batch_active(const dirac_batch *batch);

/* Kernels the batch has enqueued (each kernel node of a replayed tick graph counts). */
long dirac_batch_launch_count(const dirac_batch *batch);

/* Batch autotuner: for every class (contexts of one grid size) with contexts still
 * stepping, times each CTA shape of its x and y passes launched over all of those
 * contexts at once (reps launches per shape, CUDA events on the batch's stream) and keeps
 * the fastest for the class's later ticks. The timed launches read the states and write
 * only the contexts' second state buffers, which hold nothing between steps, so no state
 * changes. Call between ticks (it synchronises the batch's stream); DIRAC_EINVAL for
 * reps < 1, DIRAC_ETIMEOUT if a bounded device wait ran out. */
dirac_status dirac_batch_autotune(dirac_batch *batch, int reps);

/* The CTA shapes, in dirac_set_launch terms (256, 512, 1024 threads, possibly with
 * DIRAC_LAUNCH_ALT_RADIX), that the class of
 * nx x ny contexts runs in this batch: the autotuner's choice, else the batch default
 * (complex64 lines of 256 points or more: the persistent pass; otherwise 512).
 * DIRAC_EINVAL if the batch has no such class. */
dirac_status dirac_batch_launch_shape(const dirac_batch *batch, int nx, int ny, int *threads_x,
                                      int *threads_y);

const char *dirac_batch_last_error(const dirac_batch *batch);

/* Waits for enqueued work and frees the batch (not the contexts). NULL is allowed. */
void dirac_batch_destroy(dirac_batch *batch);

/* Norms of a device spinor without allocating device memory. The paper has no
 * counterpart: this serves callers that cannot call cudaMalloc where they need a norm --
 * services whose device memory all belongs to another allocator or to a fixed arena
 * reserved up front (a further cudaMalloc would fail or break their accounting), and
 * loops that cannot afford cudaMalloc/cudaFree's implicit device synchronisation.
 *   psi:    device [2][ny][nx] complex128 (the ABI spinor layout), read only
 *   weight: device [ny][nx] doubles (e.g. w = sqrt(g11 g22 / g00)), or NULL for weight 1
 *   out:    device pointer to 2 doubles, receives {hx hy sum |psi|^2, hx hy sum w |psi|^2}
 *   cuda_stream: the stream to enqueue on (NULL = the default stream); nothing is
 *   synchronised, out is valid once the stream reaches this point.
 * Sizes: nx, ny powers of two in [16, 4096]; larger grids return DIRAC_EINVAL with a
 * message in dirac_last_error(NULL). The partial sums live in a 32 KiB file-scope device
 * array that every GPU loading the library holds until exit; the first call on a device
 * looks up its device address (make that first call before any stream capture on that
 * device). All calls share the array: calls that overlap on the GPU race, so order them
 * on one stream or synchronise between them. Every call overwrites the partial sums it
 * reads, so no clearing is needed. If a launch error of earlier, unrelated work is still
 * pending on the calling thread, the call returns DIRAC_ECUDA without launching and
 * leaves that error in place for its owner. */
dirac_status dirac_norms_noalloc(const double *psi, const double *weight, int nx, int ny,
                                 double ax, double ay, double *out, void *cuda_stream);

/* Measurement helper (no counterpart in the paper): the device's fused multiply-add
 * throughput, the denominator of the ALU-bound rooflines of the benchmark. kind 0: FP64
 * FMA, 1: FP32 FMA, 2: FP32 packed pairs (two FMAs per fma.rn.f32x2 instruction).
 * Launches eight 256-thread blocks per SM, each thread running eight independent FMA
 * chains, on cuda_stream (NULL = the default stream), timed with CUDA events over one
 * launch of at least 2 ms after a warm-up; *tflops receives 2 x FMAs / s / 1e12.
 * Synchronises the stream; allocates nothing. DIRAC_EINVAL for another kind or a NULL
 * tflops (message in dirac_last_error(NULL)), DIRAC_ECUDA if a launch fails. */
dirac_status dirac_measure_alu_peak(int kind, double *tflops, void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif
