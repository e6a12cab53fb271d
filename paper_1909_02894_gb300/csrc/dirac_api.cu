// C ABI of the Scheme II library: context management and the host side of each call.
// Every numerical step runs in the kernels of this library; the host only validates,
// allocates, enqueues and copies.
#include <cuda_runtime.h>
#include <math.h>

#include <cstdio>
#include <cstdlib>
#include <complex>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/dirac.h"
#include "ctx.h"
#include "internal.h"

using namespace dgb;



static thread_local std::string g_create_error;

namespace dgb {
void set_global_error(const std::string& msg) { g_create_error = msg; }
}  // namespace dgb

static size_t npts(const dirac_ctx* c) { return (size_t)c->nx * c->ny; }

static dirac_status fail(dirac_ctx* c, dirac_status s, const std::string& msg) {
  if (c) c->err = msg;
  else g_create_error = msg;
  return s;
}

static dirac_status cuda_fail(dirac_ctx* c, cudaError_t e, const char* where) {
  std::string m = std::string(where) + ": " + cudaGetErrorString(e);
  return fail(c, e == cudaErrorMemoryAllocation ? DIRAC_ENOMEM : DIRAC_ECUDA, m);
}

#define CK(call, where)                                   \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, where); \
  } while (0)

static bool pow2_in(int n, int lo, int hi) { return n >= lo && n <= hi && (n & (n - 1)) == 0; }

// Failure-detection test hook read at creation: DIRAC_FAULT=alloc:N (N >= 1) makes the
// N-th device allocation of the new context fail with cudaErrorMemoryAllocation, so the
// creation returns DIRAC_ENOMEM after freeing what it had allocated. Anything else: off.
static int fault_alloc_from_env() {
  const char* f = getenv("DIRAC_FAULT");
  if (!f || strncmp(f, "alloc:", 6) != 0) return 0;
  char* end = nullptr;
  const long n = strtol(f + 6, &end, 10);
  return (end && *end == '\0' && n >= 1 && n < (1L << 30)) ? (int)n : 0;
}

static cudaError_t dalloc(dirac_ctx* ctx, void** p, size_t bytes) {
  if (ctx->fault_alloc_at > 0 && ++ctx->n_allocs == ctx->fault_alloc_at) {
    // injected failure: nothing is allocated, the caller unwinds as for a real one
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  cudaError_t e = cudaMalloc(p, bytes);
  if (e == cudaSuccess) ctx->allocs.push_back(*p);
  return e;
}

static void free_all(dirac_ctx* ctx) {
  for (void* p : ctx->allocs) cudaFree(p);
  ctx->allocs.clear();
}

// ------------------------------------------------------------------ precision dispatch
// launch option for a pass from the dirac_set_launch preference (0 = default)
static int pass_opt(const dirac_ctx* ctx, int shape, int L) {
  if (shape & DIRAC_LAUNCH_ALT_RADIX) {  // validated by dirac_set_launch
    const int threads = shape & ~DIRAC_LAUNCH_ALT_RADIX;
    if (ctx->prec == DIRAC_C64 ? line_pass_radix_alt<float>(L) : line_pass_radix_alt<double>(L))
      return threads == 256 ? 3 : 4;
    shape = threads;  // this line length has no alternative radix: the default one
  }
  const int threads = shape;
  if (threads == 256) return 0;
  if (threads == 512) return 1;
  if (threads == 1024) return 2;
  // Default, by measurement on the strained-graphene grids: complex64 the persistent
  // prefetching pass for lines of 1024 points or more, the smaller shape for 128- and
  // 256-point lines (0.016 against 0.018 ms per 256^2 step, 0.0166 against 0.0187 per
  // 128^2), else the larger; complex128 the smaller shape for 1024-point lines (one line
  // per CTA: 1024 CTAs spread over the SMs to within one line, 0.74 against 0.89 ms per
  // 1024^2 step) and for lines of 128 points or fewer (0.050 against 0.168 ms per 128^2
  // step), else the larger.
  if (ctx->prec == DIRAC_C64) return L >= 1024 ? 2 : (L == 256 || L == 128) ? 0 : 1;
  return (L == 1024 || L <= 128) ? 0 : 1;
}

// Reads and clears the device error flag (after the stream has been synchronised).
static dirac_status device_error(dirac_ctx* ctx) {
  int flag = 0;
  cudaError_t e = cudaMemcpy(&flag, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "read device error flag");
  if (DIRAC_DEBUG && dgb_debug_bounds())
    return fail(ctx, DIRAC_ECUDA, "debug build: an index check of a line pass failed");
  if (flag) {
    cudaMemset(ctx->d_err, 0, sizeof(int));
    if (flag == 2)  // the 4096-point pass's staging tile (never expected)
      return fail(ctx, DIRAC_ECUDA, "a line pass found its shared-memory staging tile "
                                    "misaligned for tensor stores; the state is not valid");
    return fail(ctx, DIRAC_ETIMEOUT, "a bounded device wait ran out; the state is not valid");
  }
  return DIRAC_OK;
}

template <typename T>
static LinePassArgs<T> pass_args(dirac_ctx* ctx, int axis) {
  LinePassArgs<T> a{};
  a.err = ctx->d_err;
  a.L = axis == 0 ? ctx->nx : ctx->ny;
  a.n_lines = axis == 0 ? ctx->ny : ctx->nx;
  a.sigma = axis;
  a.tw = (const Cx<T>*)(axis == 0 ? ctx->tw_x : ctx->tw_y);
  a.tw_alt = (const Cx<T>*)(axis == 0 ? ctx->tw_x_alt : ctx->tw_y_alt);
  return a;
}

template <typename T>
static dirac_status tables_for_dt(dirac_ctx* ctx, double dt) {
  cudaStream_t st = ctx->stream;
  const bool sym = ctx->scheme == DIRAC_SCHEME_II_SYMMETRIC;
  const bool need_u2n = ctx->scheme != DIRAC_SCHEME_II;  // U^2 applied in the normal layout
  if (sym && !ctx->mult_xh)
    CK(dalloc(ctx, &ctx->mult_xh, ctx->nx * sizeof(Q4<T>)), "allocate tables");
  if (sym && ctx->mult_px && !ctx->mult_pxh)
    CK(dalloc(ctx, &ctx->mult_pxh, ctx->nx * sizeof(Q4<T>)), "allocate tables");
  if (need_u2n && !ctx->u_identity && !ctx->u2_n)
    CK(dalloc(ctx, &ctx->u2_n, npts(ctx) * sizeof(Q4<T>)), "allocate half-step");
  if (!ctx->u_identity) {
    CK(launch_halfstep<T>(ctx->a1, ctx->a2, ctx->meff, ctx->omx, ctx->omy, ctx->nx, ctx->ny, dt,
                          (Q4<T>*)ctx->u_n, (Q4<T>*)ctx->u_t, (Q4<T>*)ctx->u2_t,
                          need_u2n ? (Q4<T>*)ctx->u2_n : nullptr, st),
       "half-step matrices");
    ctx->launches += 1;
  }
  if (ctx->has_pot) {
    if (!ctx->ug) CK(dalloc(ctx, &ctx->ug, 2 * npts(ctx) * sizeof(Q4<T>)), "allocate half-step");
    if (!ctx->ug2) CK(dalloc(ctx, &ctx->ug2, 2 * npts(ctx) * sizeof(Q4<T>)), "allocate half-step");
    CK(launch_halfstep_general<T>(ctx->a1, ctx->a2, ctx->meff, ctx->omx, ctx->omy,
                                  ctx->pot_use[0] ? ctx->pot_v : nullptr,
                                  ctx->pot_use[1] ? ctx->pot_ax : nullptr,
                                  ctx->pot_use[2] ? ctx->pot_ay : nullptr, ctx->nx, ctx->ny, dt,
                                  (Q4<T>*)ctx->ug, (Q4<T>*)ctx->ug2, st),
       "half-step matrices with potentials");
    ctx->launches += 1;
  }
  CK(launch_step_mult<T>(ctx->nx, ctx->ax, dt, (Q4<T>*)ctx->mult_x, st), "x multipliers");
  CK(launch_step_mult<T>(ctx->ny, ctx->ay, dt, (Q4<T>*)ctx->mult_y, st), "y multipliers");
  ctx->launches += 2;
  if (sym) {
    CK(launch_step_mult<T>(ctx->nx, ctx->ax, 0.5 * dt, (Q4<T>*)ctx->mult_xh, st),
       "x multipliers (dt/2)");
    ctx->launches += 1;
  }
  // the same tables in the 1024-point persistent pass's order
  const void* perm_src[3] = {ctx->mult_x, ctx->mult_y, ctx->mult_xh};
  void* perm_dst[3] = {ctx->mult_px, ctx->mult_py, ctx->mult_pxh};
  for (int t = 0; t < 3; ++t) {
    if (!perm_dst[t]) continue;
    CK(launch_perm1024<T>((const Q4<T>*)perm_src[t], (Q4<T>*)perm_dst[t], st), "multiplier order");
    ctx->launches += 1;
  }
  ctx->dt_cached = dt;
  return DIRAC_OK;
}

// psi <- U psi (squared = false) or U^2 psi in the normal layout, outside the passes: the
// general matrices when potentials are set, else the real-form ones (none when U = I).
template <typename T>
static dirac_status apply_half(dirac_ctx* ctx, void* psi, bool squared) {
  const size_t np = npts(ctx);
  if (ctx->has_pot) {
    CK(launch_apply_ug<T>((Q4<T>*)psi, (const Q4<T>*)(squared ? ctx->ug2 : ctx->ug), np,
                          ctx->stream),
       "half step");
  } else if (!ctx->u_identity) {
    CK(launch_apply_u<T>((Q4<T>*)psi, (const Q4<T>*)(squared ? ctx->u2_n : ctx->u_n), np,
                         ctx->stream),
       "half step");
  } else {
    return DIRAC_OK;
  }
  ctx->launches += 1;
  return DIRAC_OK;
}

// Symmetric order: x over dt/2 (normal -> transposed), y over dt (transposed -> normal),
// x over dt/2 (normal -> normal, into the other buffer); U on the first x pass's load,
// U^2 / U on the last x pass's store. The state alternates between the two buffers and
// ends in ctx->psi.
template <typename T>
static dirac_status step_symmetric(dirac_ctx* ctx, long n) {
  LinePassArgs<T> ax = pass_args<T>(ctx, 0), ay = pass_args<T>(ctx, 1);
  ax.mult = (const Q4<T>*)ctx->mult_xh;
  ax.mult_perm = (const Q4<T>*)ctx->mult_pxh;
  ax.beta = (const T*)ctx->beta1;
  ax.beta_im = (const T*)ctx->beta1_im;
  ay.mult = (const Q4<T>*)ctx->mult_y;
  ay.mult_perm = (const Q4<T>*)ctx->mult_py;
  ay.beta = (const T*)ctx->beta2T;
  ay.beta_im = (const T*)ctx->beta2T_im;
  ax.test_extra_tx = ay.test_extra_tx = ctx->test_timeout_next;
  ctx->test_timeout_next = 0;
  void* cur = ctx->psi;
  void* oth = ctx->psiT;
  const int opt_x = pass_opt(ctx, ctx->threads_x, ctx->nx);
  const int opt_y = pass_opt(ctx, ctx->threads_y, ctx->ny);
  const bool fused = !ctx->has_pot;  // potentials: U applied by its own kernel
  if (!fused) {
    dirac_status r = apply_half<T>(ctx, cur, false);
    if (r != DIRAC_OK) return r;
  }
  for (long s = 0; s < n; ++s) {
    LinePassArgs<T> a1 = ax, a3 = ax;
    a1.in = (const Q4<T>*)cur;
    a1.out = (Q4<T>*)oth;
    a1.u_load = (fused && s == 0 && !ctx->u_identity) ? (const Q4<T>*)ctx->u_n : nullptr;
    ay.in = (const Q4<T>*)oth;
    ay.out = (Q4<T>*)cur;
    a3.in = (const Q4<T>*)cur;
    a3.out = (Q4<T>*)oth;
    a3.store_normal = 1;
    a3.u_store = (!fused || ctx->u_identity)
                     ? nullptr
                     : (const Q4<T>*)(s + 1 == n ? ctx->u_n : ctx->u2_n);
    CK(launch_line_pass<T>(a1, MODE_STEP, opt_x, ctx->stream), "x pass (dt/2)");
    CK(launch_line_pass<T>(ay, MODE_STEP, opt_y, ctx->stream), "y pass");
    CK(launch_line_pass<T>(a3, MODE_STEP, opt_x, ctx->stream), "x pass (dt/2, rows)");
    ctx->launches += 3;
    if (!fused) {
      dirac_status r = apply_half<T>(ctx, oth, s + 1 < n);
      if (r != DIRAC_OK) return r;
    }
    void* t = cur;
    cur = oth;
    oth = t;
  }
  if (cur != ctx->psi) {  // the two state buffers trade names
    ctx->psiT = ctx->psi;
    ctx->psi = cur;
  }
  return DIRAC_OK;
}

// out = alpha S(in) + beta prev, acc += gamma out, with S(in) = sum_j b^j sigma_j [[d_j]] in
// (so dt A = -dt S): x derivative (row pass, rows back in place), transpose, y derivative
// (transposed store back to rows), pointwise combine. psiT, scratch1, scratch2 are scratch.
template <typename T>
static dirac_status unsplit_apply(dirac_ctx* ctx, const void* in, void* out, double ar,
                                  double ai, const void* prev, double beta, double gr,
                                  double gi, void* acc) {
  cudaStream_t st = ctx->stream;
  LinePassArgs<T> ax = pass_args<T>(ctx, 0), ay = pass_args<T>(ctx, 1);
  ax.in = (const Q4<T>*)in;
  ax.out = (Q4<T>*)ctx->scratch1;
  ax.mult = (const Q4<T>*)ctx->dmult_x;
  ax.store_normal = 1;
  CK(launch_line_pass<T>(ax, MODE_DERIV, 0, st), "x derivative");
  CK(launch_transpose<T>((const Q4<T>*)in, (Q4<T>*)ctx->psiT, ctx->ny, ctx->nx, st), "transpose");
  ay.in = (const Q4<T>*)ctx->psiT;
  ay.out = (Q4<T>*)ctx->scratch2;
  ay.mult = (const Q4<T>*)ctx->dmult_y;
  CK(launch_line_pass<T>(ay, MODE_DERIV, 0, st), "y derivative");
  CK(launch_unsplit_combine<T>((const Q4<T>*)ctx->scratch1, (const Q4<T>*)ctx->scratch2, ctx->a1,
                               ctx->a2, ctx->sxinv, ctx->syinv, ctx->sxinv_im, ctx->syinv_im,
                               ctx->nx, ctx->ny, ar, ai,
                               (const Q4<T>*)prev, beta, gr, gi, (Q4<T>*)out, (Q4<T>*)acc, st),
     "combine");
  ctx->launches += 4;
  return DIRAC_OK;
}

#define CKS(x)                       \
  do {                               \
    dirac_status s_ = (x);           \
    if (s_ != DIRAC_OK) return s_;   \
  } while (0)

// The polynomial scheme (eq. poly): U, the middle step, U per step, with U^2 between
// consecutive steps of a call. Four state-sized buffers (the state and pool[0..2]) rotate:
// the middle step's sum becomes the new state.
template <typename T>
static dirac_status step_poly(dirac_ctx* ctx, long n, double dt) {
  cudaStream_t st = ctx->stream;
  const size_t np = npts(ctx), bytes = np * sizeof(Q4<T>);
  for (void*& p : ctx->pool)
    if (!p) CK(dalloc(ctx, &p, bytes), "allocate polynomial terms");
  if (!ctx->scratch1) CK(dalloc(ctx, &ctx->scratch1, bytes), "scratch");
  if (!ctx->scratch2) CK(dalloc(ctx, &ctx->scratch2, bytes), "scratch");
  const int N = ctx->poly_degree;
  const bool cheb = ctx->scheme == DIRAC_SCHEME_POLY_CHEBYSHEV;
  std::vector<double> jq(N + 1, 0.0);
  double R = 0.0;
  if (cheb) {
    if (ctx->bmax[0] < 0.0) {  // max |b^j| over the grid, once per context
      const int nb = 256;
      double* part = nullptr;
      CK(dalloc(ctx, (void**)&part, 2 * nb * sizeof(double)), "scratch");
      CK(launch_max_b(ctx->a1, ctx->a2, ctx->sxinv, ctx->syinv, ctx->sxinv_im, ctx->syinv_im,
                      ctx->nx, ctx->ny, part, nb, st),
         "max b");
      std::vector<double> h(2 * nb);
      CK(cudaMemcpyAsync(h.data(), part, 2 * nb * sizeof(double), cudaMemcpyDeviceToHost, st),
         "max b");
      CK(cudaStreamSynchronize(st), "max b");
      ctx->bmax[0] = ctx->bmax[1] = 0.0;
      for (int b = 0; b < nb; ++b) {
        ctx->bmax[0] = fmax(ctx->bmax[0], h[2 * b]);
        ctx->bmax[1] = fmax(ctx->bmax[1], h[2 * b + 1]);
      }
      ctx->launches += 1;
    }
    const double hx = 2.0 * ctx->ax / ctx->nx, hy = 2.0 * ctx->ay / ctx->ny;
    R = dt * (ctx->bmax[0] * M_PI / hx + ctx->bmax[1] * M_PI / hy);
    if (!(R > 0.0) || !bessel_j_series(R, N, jq.data()))
      return fail(ctx, DIRAC_EINVAL, "no Chebyshev bound for this grid and dt");
  }
  for (long s = 0; s < n; ++s) {
    if (s == 0) CKS(apply_half<T>(ctx, ctx->psi, false));
    void* bufs[4] = {ctx->psi, ctx->pool[0], ctx->pool[1], ctx->pool[2]};
    void* acc = bufs[3];
    if (!cheb) {
      // acc = sum_q (dt A)^q / q! psi; (dt/q) A t = -(dt/q) S(t)
      CK(cudaMemcpyAsync(acc, bufs[0], bytes, cudaMemcpyDeviceToDevice, st), "copy");
      void *cur = bufs[0], *nxt = bufs[1], *spare = bufs[2];
      for (int q = 1; q <= N; ++q) {
        CKS(unsplit_apply<T>(ctx, cur, nxt, -dt / q, 0.0, nullptr, 0.0, 1.0, 0.0, acc));
        cur = nxt;
        nxt = (cur == bufs[1]) ? spare : bufs[1];
      }
    } else {
      // phi_0 = psi, phi_1 = B phi_0, phi_{q+1} = 2 B phi_q - phi_{q-1} with
      // B = (i dt / R) A = -(i dt / R) S; acc = sum_q (2 - delta_q0) (-i)^q J_q(R) phi_q
      CK(launch_scale<T>((Q4<T>*)acc, (const Q4<T>*)bufs[0], jq[0], 0.0, np, st), "scale");
      ctx->launches += 1;
      static const double pr[4] = {1.0, 0.0, -1.0, 0.0}, pi_[4] = {0.0, -1.0, 0.0, 1.0};
      void *prev = bufs[0], *cur = bufs[1], *spare = bufs[2];
      if (N >= 1)
        CKS(unsplit_apply<T>(ctx, prev, cur, 0.0, -dt / R, nullptr, 0.0, 2.0 * pr[1] * jq[1],
                             2.0 * pi_[1] * jq[1], acc));
      for (int q = 2; q <= N; ++q) {
        CKS(unsplit_apply<T>(ctx, cur, spare, 0.0, -2.0 * dt / R, prev, -1.0,
                             2.0 * pr[q & 3] * jq[q], 2.0 * pi_[q & 3] * jq[q], acc));
        void* t = prev;
        prev = cur;
        cur = spare;
        spare = t;
      }
    }
    // the sum is the new state; the other three buffers become the pool
    int k = 0;
    for (void* b : bufs)
      if (b != acc) ctx->pool[k++] = b;
    ctx->psi = acc;
    CKS(apply_half<T>(ctx, ctx->psi, s + 1 < n));
  }
  return DIRAC_OK;
}

// ---- Scheme I (eq. cn): U, G psi* = G~ psi by restarted GMRES, U (U^2 between steps).
// G v = v - dt/2 A v = v + dt/2 S(v), G~ v = v - dt/2 S(v) (S as in unsplit_apply).
constexpr int kKrylovBlocks = 304;

// <V_i, w> for i < count, V = the device pointer array starting at slot first.
template <typename T>
static dirac_status krylov_dots(dirac_ctx* ctx, int first, int count, const void* w,
                                std::vector<std::complex<double>>& out) {
  cudaStream_t st = ctx->stream;
  CK(launch_multi_dot<T>((const Q4<T>* const*)(ctx->k_vptr + first), count, (const Q4<T>*)w,
                         npts(ctx), ctx->k_partials, kKrylovBlocks, st),
     "inner products");
  std::vector<double> h(2 * (size_t)kKrylovBlocks * count);
  CK(cudaMemcpyAsync(h.data(), ctx->k_partials, h.size() * sizeof(double),
                     cudaMemcpyDeviceToHost, st),
     "inner products");
  CK(cudaStreamSynchronize(st), "inner products");
  out.assign(count, 0.0);
  for (int i = 0; i < count; ++i) {
    double re = 0.0, im = 0.0;
    for (int b = 0; b < kKrylovBlocks; ++b) {
      re += h[2 * ((size_t)i * kKrylovBlocks + b)];
      im += h[2 * ((size_t)i * kKrylovBlocks + b) + 1];
    }
    out[i] = {re, im};
  }
  ctx->launches += 1;
  return DIRAC_OK;
}

// out += sum_i c_i V_{first + i}
template <typename T>
static dirac_status krylov_combine(dirac_ctx* ctx, void* out, int first,
                                   const std::vector<std::complex<double>>& c) {
  std::vector<double> h(2 * c.size());
  for (size_t i = 0; i < c.size(); ++i) {
    h[2 * i] = c[i].real();
    h[2 * i + 1] = c[i].imag();
  }
  CK(cudaMemcpyAsync(ctx->k_coef, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice,
                     ctx->stream),
     "coefficients");
  CK(launch_multi_axpy<T>((Q4<T>*)out, (const Q4<T>* const*)(ctx->k_vptr + first), ctx->k_coef,
                          (int)c.size(), npts(ctx), ctx->stream),
     "combination");
  ctx->launches += 1;
  return DIRAC_OK;
}

template <typename T>
static dirac_status step_cn(dirac_ctx* ctx, long n, double dt) {
  cudaStream_t st = ctx->stream;
  const size_t np = npts(ctx), bytes = np * sizeof(Q4<T>);
  const int m = ctx->krylov_m;
  const double tol = ctx->krylov_tol > 0.0 ? ctx->krylov_tol : (sizeof(T) == 8 ? 1e-14 : 3e-7);
  // buffers: basis V_0..V_m, the right-hand side, the pointer table (basis, then rhs)
  while ((int)ctx->kv.size() < m + 1) {
    void* p = nullptr;
    CK(dalloc(ctx, &p, bytes), "allocate Krylov basis");
    ctx->kv.push_back(p);
  }
  if (!ctx->k_rhs) CK(dalloc(ctx, &ctx->k_rhs, bytes), "allocate Krylov basis");
  if (!ctx->scratch1) CK(dalloc(ctx, &ctx->scratch1, bytes), "scratch");
  if (!ctx->scratch2) CK(dalloc(ctx, &ctx->scratch2, bytes), "scratch");
  if (!ctx->k_partials)
    CK(dalloc(ctx, (void**)&ctx->k_partials, 2 * (size_t)kKrylovBlocks * 102 * sizeof(double)),
       "scratch");
  if (!ctx->k_coef) CK(dalloc(ctx, (void**)&ctx->k_coef, 2 * 102 * sizeof(double)), "scratch");
  if (!ctx->k_vptr) CK(dalloc(ctx, (void**)&ctx->k_vptr, 102 * sizeof(void*)), "scratch");
  {
    std::vector<void*> table(ctx->kv.begin(), ctx->kv.begin() + m + 1);
    table.push_back(ctx->k_rhs);
    CK(cudaMemcpy(ctx->k_vptr, table.data(), table.size() * sizeof(void*), cudaMemcpyHostToDevice),
       "pointer table");
  }
  using cd = std::complex<double>;
  std::vector<cd> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), y(m), h, h2;
  for (long s = 0; s < n; ++s) {
    if (s == 0) CKS(apply_half<T>(ctx, ctx->psi, false));
    void* x = ctx->psi;
    CKS(unsplit_apply<T>(ctx, x, ctx->k_rhs, -0.5 * dt, 0.0, x, 1.0, 0.0, 0.0, nullptr));
    CKS(krylov_dots<T>(ctx, m + 1, 1, ctx->k_rhs, h));
    const double bnorm = sqrt(h[0].real());
    bool converged = false;
    for (int cycle = 0; cycle <= ctx->krylov_restarts && !converged; ++cycle) {
      // r = rhs - G x into V_0
      void* v0 = ctx->kv[0];
      CKS(unsplit_apply<T>(ctx, x, v0, 0.5 * dt, 0.0, x, 1.0, 0.0, 0.0, nullptr));
      CK(launch_axpby<T>((Q4<T>*)v0, 1.0, (const Q4<T>*)ctx->k_rhs, -1.0, (const Q4<T>*)v0, np, st),
         "residual");
      CKS(krylov_dots<T>(ctx, 0, 1, v0, h));
      const double beta = sqrt(fmax(h[0].real(), 0.0));
      if (beta <= tol * bnorm || beta == 0.0) {
        converged = true;
        break;
      }
      if (cycle == ctx->krylov_restarts) break;
      CK(launch_scale<T>((Q4<T>*)v0, (const Q4<T>*)v0, 1.0 / beta, 0.0, np, st), "normalise");
      std::fill(g.begin(), g.end(), cd(0.0));
      g[0] = beta;
      int kdim = 0;
      for (int j = 0; j < m; ++j) {
        void* w = ctx->kv[j + 1];
        CKS(unsplit_apply<T>(ctx, ctx->kv[j], w, 0.5 * dt, 0.0, ctx->kv[j], 1.0, 0.0, 0.0,
                             nullptr));
        // classical Gram-Schmidt, twice
        CKS(krylov_dots<T>(ctx, 0, j + 1, w, h));
        std::vector<cd> neg(j + 1);
        for (int i = 0; i <= j; ++i) neg[i] = -h[i];
        CKS(krylov_combine<T>(ctx, w, 0, neg));
        CKS(krylov_dots<T>(ctx, 0, j + 1, w, h2));
        for (int i = 0; i <= j; ++i) {
          neg[i] = -h2[i];
          h[i] += h2[i];
        }
        CKS(krylov_combine<T>(ctx, w, 0, neg));
        std::vector<cd> nn;
        CKS(krylov_dots<T>(ctx, j + 1, 1, w, nn));
        const double hn = sqrt(fmax(nn[0].real(), 0.0));
        if (hn > 0.0)
          CK(launch_scale<T>((Q4<T>*)w, (const Q4<T>*)w, 1.0 / hn, 0.0, np, st), "normalise");
        for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = h[i];
        H[(size_t)(j + 1) * m + j] = hn;
        for (int i = 0; i < j; ++i) {  // earlier Givens rotations on column j
          const cd a = H[(size_t)i * m + j], b = H[(size_t)(i + 1) * m + j];
          H[(size_t)i * m + j] = std::conj(cs[i]) * a + std::conj(sn[i]) * b;
          H[(size_t)(i + 1) * m + j] = -sn[i] * a + cs[i] * b;
        }
        const cd a = H[(size_t)j * m + j], b = H[(size_t)(j + 1) * m + j];
        const double r = sqrt(std::norm(a) + std::norm(b));
        cs[j] = r > 0.0 ? a / r : cd(1.0);
        sn[j] = r > 0.0 ? b / r : cd(0.0);
        H[(size_t)j * m + j] = r;
        H[(size_t)(j + 1) * m + j] = 0.0;
        g[j + 1] = -sn[j] * g[j];
        g[j] = std::conj(cs[j]) * g[j];
        kdim = j + 1;
        ctx->krylov_iters += 1;
        if (std::abs(g[j + 1]) <= tol * bnorm || hn == 0.0) break;
      }
      for (int i = kdim - 1; i >= 0; --i) {  // H y = g, then x += V y
        cd acc = g[i];
        for (int t = i + 1; t < kdim; ++t) acc -= H[(size_t)i * m + t] * y[t];
        y[i] = acc / H[(size_t)i * m + i];
      }
      CKS(krylov_combine<T>(ctx, x, 0, std::vector<cd>(y.begin(), y.begin() + kdim)));
      ctx->launches += 3;
    }
    if (!converged) return fail(ctx, DIRAC_ENOCONV, "Scheme I: GMRES did not converge");
    CKS(apply_half<T>(ctx, ctx->psi, s + 1 < n));
  }
  return DIRAC_OK;
}

template <typename T>
static dirac_status step_impl(dirac_ctx* ctx, long n, double dt) {
  if (dt != ctx->dt_cached) {
    dirac_status s = tables_for_dt<T>(ctx, dt);
    if (s != DIRAC_OK) return s;
  }
  if (ctx->scheme == DIRAC_SCHEME_II_SYMMETRIC) return step_symmetric<T>(ctx, n);
  if (ctx->scheme == DIRAC_SCHEME_POLY_TAYLOR || ctx->scheme == DIRAC_SCHEME_POLY_CHEBYSHEV)
    return step_poly<T>(ctx, n, dt);
  if (ctx->scheme == DIRAC_SCHEME_CRANK_NICOLSON) return step_cn<T>(ctx, n, dt);
  LinePassArgs<T> ax = pass_args<T>(ctx, 0), ay = pass_args<T>(ctx, 1);
  ax.in = (const Q4<T>*)ctx->psi;
  ax.out = (Q4<T>*)ctx->psiT;
  ax.mult = (const Q4<T>*)ctx->mult_x;
  ax.mult_perm = (const Q4<T>*)ctx->mult_px;
  ax.beta = (const T*)ctx->beta1;
  ax.beta_im = (const T*)ctx->beta1_im;
  ay.in = (const Q4<T>*)ctx->psiT;
  ay.out = (Q4<T>*)ctx->psi;
  ay.mult = (const Q4<T>*)ctx->mult_y;
  ay.mult_perm = (const Q4<T>*)ctx->mult_py;
  ay.beta = (const T*)ctx->beta2T;
  ay.beta_im = (const T*)ctx->beta2T_im;
  ax.test_extra_tx = ay.test_extra_tx = ctx->test_timeout_next;
  ctx->test_timeout_next = 0;
  const bool fused = !ctx->has_pot;  // potentials: U applied by its own kernel
  if (!fused) CKS(apply_half<T>(ctx, ctx->psi, false));
  for (long s = 0; s < n; ++s) {
    ax.u_load = (fused && s == 0 && !ctx->u_identity) ? (const Q4<T>*)ctx->u_n : nullptr;
    ax.u_store = nullptr;
    CK(launch_line_pass<T>(ax, MODE_STEP, pass_opt(ctx, ctx->threads_x, ctx->nx), ctx->stream),
       "x pass");
    ay.u_load = nullptr;
    ay.u_store = (!fused || ctx->u_identity) ? nullptr
                                             : (const Q4<T>*)(s + 1 == n ? ctx->u_t : ctx->u2_t);
    CK(launch_line_pass<T>(ay, MODE_STEP, pass_opt(ctx, ctx->threads_y, ctx->ny), ctx->stream),
       "y pass");
    ctx->launches += 2;
    if (!fused) CKS(apply_half<T>(ctx, ctx->psi, s + 1 < n));
  }
  return DIRAC_OK;
}

// Spectral derivatives of the state: dx (normal layout) into scratch1, dy into scratch2.
// Uses psiT as the transposed intermediate.
template <typename T>
static dirac_status state_derivatives(dirac_ctx* ctx) {
  cudaStream_t st = ctx->stream;
  LinePassArgs<T> ax = pass_args<T>(ctx, 0), ay = pass_args<T>(ctx, 1);
  // y derivative: transpose psi -> scratch1 ([nx][ny]); derivative pass stores it back
  // transposed, i.e. in the normal layout, into scratch2.
  CK(launch_transpose<T>((const Q4<T>*)ctx->psi, (Q4<T>*)ctx->scratch1, ctx->ny, ctx->nx, st),
     "transpose");
  ay.in = (const Q4<T>*)ctx->scratch1;
  ay.out = (Q4<T>*)ctx->scratch2;
  ay.mult = (const Q4<T>*)ctx->dmult_y;
  CK(launch_line_pass<T>(ay, MODE_DERIV, 0, st), "y derivative");
  // x derivative: psi -> psiT (transposed), then back to the normal layout in scratch1.
  ax.in = (const Q4<T>*)ctx->psi;
  ax.out = (Q4<T>*)ctx->psiT;
  ax.mult = (const Q4<T>*)ctx->dmult_x;
  CK(launch_line_pass<T>(ax, MODE_DERIV, 0, st), "x derivative");
  CK(launch_transpose<T>((const Q4<T>*)ctx->psiT, (Q4<T>*)ctx->scratch1, ctx->nx, ctx->ny, st),
     "transpose");
  ctx->launches += 4;
  return DIRAC_OK;
}

template <typename T>
static dirac_status observables_impl(dirac_ctx* ctx, dirac_obs* out, double* density_host) {
  cudaStream_t st = ctx->stream;
  const size_t n = npts(ctx);
  if (!ctx->scratch1) {
    CK(dalloc(ctx, &ctx->scratch1, n * sizeof(Q4<T>)), "scratch");
    CK(dalloc(ctx, &ctx->scratch2, n * sizeof(Q4<T>)), "scratch");
  }
  dirac_status s = state_derivatives<T>(ctx);
  if (s != DIRAC_OK) return s;
  if (density_host && !ctx->density) CK(dalloc(ctx, (void**)&ctx->density, n * sizeof(double)), "density");
  const int blocks = observables_blocks(n);
  CK(launch_observables<T>((const Q4<T>*)ctx->psi, (const Q4<T>*)ctx->scratch1,
                           (const Q4<T>*)ctx->scratch2, ctx->a1, ctx->a2, ctx->meff, ctx->w,
                           ctx->omx, ctx->omy, ctx->pot_use[0] ? ctx->pot_v : nullptr,
                           ctx->pot_use[1] ? ctx->pot_ax : nullptr,
                           ctx->pot_use[2] ? ctx->pot_ay : nullptr, n,
                           density_host ? ctx->density : nullptr, ctx->partials, blocks, st),
     "observables");
  const double hxhy = (2.0 * ctx->ax / ctx->nx) * (2.0 * ctx->ay / ctx->ny);
  CK(launch_reduce_partials(ctx->partials, blocks, hxhy, ctx->result, st), "reduce");
  ctx->launches += 2;
  double r[4];
  CK(cudaMemcpyAsync(r, ctx->result, sizeof(r), cudaMemcpyDeviceToHost, st), "copy result");
  if (density_host)
    CK(cudaMemcpyAsync(density_host, ctx->density, n * sizeof(double), cudaMemcpyDeviceToHost, st),
       "copy density");
  CK(cudaStreamSynchronize(st), "synchronize");
  {
    dirac_status de = device_error(ctx);
    if (de != DIRAC_OK) return de;
  }
  out->norm = r[0];
  out->norm_gamma = r[1];
  out->energy = r[2];
  out->energy_imag = r[3];
  if (!isfinite(r[0]) || !isfinite(r[1]) || !isfinite(r[2]) || !isfinite(r[3]))
    return fail(ctx, DIRAC_ENONFINITE, "the state holds non-finite values");
  return DIRAC_OK;
}

template <typename T>
static dirac_status create_impl(dirac_ctx* ctx, const double* g_host[3]) {
  cudaStream_t st = ctx->stream;
  const size_t n = npts(ctx);
  const int nx = ctx->nx, ny = ctx->ny;
  // FP64 fields
  double** f64[] = {&ctx->a1, &ctx->a2, &ctx->meff, &ctx->w, &ctx->omx, &ctx->omy};
  for (double** p : f64) CK(dalloc(ctx, (void**)p, n * sizeof(double)), "allocate fields");
  CK(dalloc(ctx, (void**)&ctx->sxinv, nx * sizeof(double)), "allocate layer");
  CK(dalloc(ctx, (void**)&ctx->syinv, ny * sizeof(double)), "allocate layer");
  const bool complex_layer =
      ctx->abs.theta != 0.0 && (ctx->abs.width_x > 0 || ctx->abs.width_y > 0);
  if (complex_layer) {
    CK(dalloc(ctx, (void**)&ctx->sxinv_im, nx * sizeof(double)), "allocate layer");
    CK(dalloc(ctx, (void**)&ctx->syinv_im, ny * sizeof(double)), "allocate layer");
  }
  // state, coefficient fields, tables
  CK(dalloc(ctx, &ctx->psi, n * sizeof(Q4<T>)), "allocate state");
  CK(dalloc(ctx, &ctx->psiT, n * sizeof(Q4<T>)), "allocate state");
  CK(dalloc(ctx, &ctx->beta1, n * sizeof(T)), "allocate coefficients");
  CK(dalloc(ctx, &ctx->beta2T, n * sizeof(T)), "allocate coefficients");
  if (complex_layer) {
    CK(dalloc(ctx, &ctx->beta1_im, n * sizeof(T)), "allocate coefficients");
    CK(dalloc(ctx, &ctx->beta2T_im, n * sizeof(T)), "allocate coefficients");
  }
  if (!ctx->u_identity) {
    CK(dalloc(ctx, &ctx->u_n, n * sizeof(Q4<T>)), "allocate half-step");
    CK(dalloc(ctx, &ctx->u_t, n * sizeof(Q4<T>)), "allocate half-step");
    CK(dalloc(ctx, &ctx->u2_t, n * sizeof(Q4<T>)), "allocate half-step");
  }
  CK(dalloc(ctx, &ctx->tw_x, nx * sizeof(Cx<T>)), "allocate tables");
  CK(dalloc(ctx, &ctx->tw_y, ny * sizeof(Cx<T>)), "allocate tables");
  if (line_pass_radix_alt<T>(nx))
    CK(dalloc(ctx, &ctx->tw_x_alt, nx * sizeof(Cx<T>)), "allocate tables");
  if (line_pass_radix_alt<T>(ny))
    CK(dalloc(ctx, &ctx->tw_y_alt, ny * sizeof(Cx<T>)), "allocate tables");
  CK(dalloc(ctx, &ctx->mult_x, nx * sizeof(Q4<T>)), "allocate tables");
  CK(dalloc(ctx, &ctx->mult_y, ny * sizeof(Q4<T>)), "allocate tables");
  if (sizeof(T) == 4 && nx == 1024)  // the 1024-point persistent pass's table order
    CK(dalloc(ctx, &ctx->mult_px, nx * sizeof(Q4<T>)), "allocate tables");
  if (sizeof(T) == 4 && ny == 1024)
    CK(dalloc(ctx, &ctx->mult_py, ny * sizeof(Q4<T>)), "allocate tables");
  CK(dalloc(ctx, &ctx->dmult_x, nx * sizeof(Q4<T>)), "allocate tables");
  CK(dalloc(ctx, &ctx->dmult_y, ny * sizeof(Q4<T>)), "allocate tables");
  CK(dalloc(ctx, (void**)&ctx->staging, 2 * n * 2 * sizeof(double)), "allocate staging");
  CK(dalloc(ctx, (void**)&ctx->partials, 4 * sizeof(double) * observables_blocks(n)), "allocate");
  CK(dalloc(ctx, (void**)&ctx->result, 4 * sizeof(double)), "allocate");
  CK(dalloc(ctx, (void**)&ctx->d_err, sizeof(int)), "allocate");
  CK(cudaMemsetAsync(ctx->d_err, 0, sizeof(int), st), "clear error flag");

  // metric upload: the staging buffer holds the three fields during creation
  double* gdev[3] = {nullptr, nullptr, nullptr};
  for (int f = 0; f < 3; ++f) {
    if (g_host[f]) {
      gdev[f] = ctx->staging + (size_t)f * n;
      CK(cudaMemcpyAsync(gdev[f], g_host[f], n * sizeof(double), cudaMemcpyHostToDevice, st),
         "upload metric");
    }
  }
  // The log fields and their derivatives use psi/psiT-sized scratch in FP64.
  void *logs = nullptr, *logsT = nullptr, *dxT = nullptr, *dy = nullptr;
  CK(cudaMallocAsync(&logs, n * sizeof(Q4<double>), st), "allocate precompute scratch");
  CK(cudaMallocAsync(&logsT, n * sizeof(Q4<double>), st), "allocate precompute scratch");
  CK(cudaMallocAsync(&dxT, n * sizeof(Q4<double>), st), "allocate precompute scratch");
  CK(cudaMallocAsync(&dy, n * sizeof(Q4<double>), st), "allocate precompute scratch");
  CK(launch_metric_fields(gdev[0], gdev[1], gdev[2], (int)n, ctx->c, ctx->mass, ctx->conn,
                          ctx->a1, ctx->a2, ctx->meff, ctx->w, (Q4<double>*)logs, st),
     "metric fields");
  ctx->launches += 1;
  if (ctx->conn == DIRAC_CONN_NONE) {
    CK(cudaMemsetAsync(ctx->omx, 0, n * sizeof(double), st), "zero connection");
    CK(cudaMemsetAsync(ctx->omy, 0, n * sizeof(double), st), "zero connection");
  } else {
    // FP64 spectral derivatives with the same fused line pass (derivative mode)
    void *tx = nullptr, *ty = nullptr, *mx = nullptr, *my = nullptr;
    CK(cudaMallocAsync(&tx, nx * sizeof(Cx<double>), st), "allocate");
    CK(cudaMallocAsync(&ty, ny * sizeof(Cx<double>), st), "allocate");
    CK(cudaMallocAsync(&mx, nx * sizeof(Q4<double>), st), "allocate");
    CK(cudaMallocAsync(&my, ny * sizeof(Q4<double>), st), "allocate");
    CK(launch_twiddles<double>(nx, line_pass_radix<double>(nx), (Cx<double>*)tx, st), "twiddles");
    CK(launch_twiddles<double>(ny, line_pass_radix<double>(ny), (Cx<double>*)ty, st), "twiddles");
    CK(launch_deriv_mult<double>(nx, ctx->ax, (Q4<double>*)mx, st), "derivative table");
    CK(launch_deriv_mult<double>(ny, ctx->ay, (Q4<double>*)my, st), "derivative table");
    LinePassArgs<double> d{};
    d.L = nx; d.n_lines = ny; d.sigma = 0; d.tw = (const Cx<double>*)tx;
    d.mult = (const Q4<double>*)mx; d.in = (const Q4<double>*)logs; d.out = (Q4<double>*)dxT;
    CK(launch_line_pass<double>(d, MODE_DERIV, 0, st), "x derivative of log fields");
    CK(launch_transpose<double>((const Q4<double>*)logs, (Q4<double>*)logsT, ny, nx, st),
       "transpose");
    d.L = ny; d.n_lines = nx; d.sigma = 1; d.tw = (const Cx<double>*)ty;
    d.mult = (const Q4<double>*)my; d.in = (const Q4<double>*)logsT; d.out = (Q4<double>*)dy;
    CK(launch_line_pass<double>(d, MODE_DERIV, 0, st), "y derivative of log fields");
    const double fac = ctx->conn == DIRAC_CONN_PAPER_2D ? 0.25 : 0.5;
    CK(launch_omega((const Q4<double>*)dxT, (const Q4<double>*)dy, nx, ny, fac, ctx->omx,
                    ctx->omy, st),
       "spin connection");
    ctx->launches += 8;
    CK(cudaFreeAsync(tx, st), "free"); CK(cudaFreeAsync(ty, st), "free");
    CK(cudaFreeAsync(mx, st), "free"); CK(cudaFreeAsync(my, st), "free");
  }
  CK(cudaFreeAsync(logs, st), "free"); CK(cudaFreeAsync(logsT, st), "free");
  CK(cudaFreeAsync(dxT, st), "free"); CK(cudaFreeAsync(dy, st), "free");
  // absorbing layer and b - 1
  CK(launch_pml(nx, ctx->ax, ctx->abs.width_x, ctx->abs.type, ctx->abs.sigma0, ctx->abs.theta,
                ctx->sxinv, ctx->sxinv_im, st),
     "layer x");
  CK(launch_pml(ny, ctx->ay, ctx->abs.width_y, ctx->abs.type, ctx->abs.sigma0, ctx->abs.theta,
                ctx->syinv, ctx->syinv_im, st),
     "layer y");
  CK(launch_beta<T>(ctx->a1, ctx->a2, ctx->sxinv, ctx->syinv, ctx->sxinv_im, ctx->syinv_im, nx,
                    ny, (T*)ctx->beta1, (T*)ctx->beta2T, (T*)ctx->beta1_im,
                    (T*)ctx->beta2T_im, st),
     "b - 1");
  CK(launch_twiddles<T>(nx, line_pass_radix<T>(nx), (Cx<T>*)ctx->tw_x, st), "twiddles");
  CK(launch_twiddles<T>(ny, line_pass_radix<T>(ny), (Cx<T>*)ctx->tw_y, st), "twiddles");
  if (ctx->tw_x_alt)
    CK(launch_twiddles<T>(nx, line_pass_radix_alt<T>(nx), (Cx<T>*)ctx->tw_x_alt, st), "twiddles");
  if (ctx->tw_y_alt)
    CK(launch_twiddles<T>(ny, line_pass_radix_alt<T>(ny), (Cx<T>*)ctx->tw_y_alt, st), "twiddles");
  CK(launch_deriv_mult<T>(nx, ctx->ax, (Q4<T>*)ctx->dmult_x, st), "derivative table");
  CK(launch_deriv_mult<T>(ny, ctx->ay, (Q4<T>*)ctx->dmult_y, st), "derivative table");
  ctx->launches += 7;
  CK(cudaStreamSynchronize(st), "create");
  ctx->dt_cached = 0.0;
  return DIRAC_OK;
}

// ------------------------------------------------------------------ library-internal
dirac_status dgb_tables_for_dt(dirac_ctx* ctx, double dt) {
  return ctx->prec == DIRAC_C64 ? tables_for_dt<float>(ctx, dt) : tables_for_dt<double>(ctx, dt);
}

int dgb_pass_opt(const dirac_ctx* ctx, int threads, int L) { return pass_opt(ctx, threads, L); }

// Device bytes a context of this size holds at most (creation, state, half-step
// matrices, staging for host transfers, observables scratch and density).
size_t dgb_footprint_bytes(int nx, int ny, dirac_precision prec) {
  const size_t n = (size_t)nx * ny;
  const size_t r = prec == DIRAC_C64 ? 4 : 8, q4 = 4 * r;
  size_t per_point = 6 * sizeof(double)   // a1, a2, meff, w, omx, omy
                     + 2 * q4             // psi, psiT
                     + 2 * r              // b - 1 (both layouts)
                     + 3 * q4             // U (two layouts), U^2
                     + 4 * sizeof(double) // staging (complex128 spinor)
                     + 2 * q4             // observables scratch
                     + sizeof(double);    // density
  size_t per_line = (size_t)(nx + ny) * (sizeof(double) + 3 * q4);
  return n * per_point + per_line + 4 * sizeof(double) * 2048 + 4096;
}

// Times every CTA shape of one pass (reps launches each, CUDA events on the context's
// stream) with its output in scratch memory, so the state is untouched; returns the
// fastest shape (threads value for dirac_set_launch).
template <typename T>
static dirac_status tune_pass(dirac_ctx* ctx, int axis, int reps, int* best, float* best_ms) {
  LinePassArgs<T> a = pass_args<T>(ctx, axis);
  a.in = (const Q4<T>*)ctx->psi;  // any data of the pass's shape: the time does not depend on it
  a.out = (Q4<T>*)ctx->scratch1;
  a.mult = (const Q4<T>*)(axis == 0 ? ctx->mult_x : ctx->mult_y);
  a.mult_perm = (const Q4<T>*)(axis == 0 ? ctx->mult_px : ctx->mult_py);
  a.beta = (const T*)(axis == 0 ? ctx->beta1 : ctx->beta2T);
  a.u_store = (axis == 1 && !ctx->u_identity) ? (const Q4<T>*)ctx->u2_t : nullptr;
  const int L = a.L;
  const int options[5] = {256, 512, 1024, 256 | DIRAC_LAUNCH_ALT_RADIX,
                          512 | DIRAC_LAUNCH_ALT_RADIX};
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0), "tune");
  CK(cudaEventCreate(&e1), "tune");
  *best = 0;
  *best_ms = 1e30f;
  for (int t : options) {
    if (t == 1024 && !(sizeof(T) == 4 && L >= 256)) continue;  // persistent: complex64 only
    if ((t & DIRAC_LAUNCH_ALT_RADIX) && !line_pass_radix_alt<T>(L)) continue;
    const int opt = pass_opt(ctx, t, L);
    cudaError_t e = cudaSuccess;
    for (int w = 0; w < 2 && e == cudaSuccess; ++w) e = launch_line_pass<T>(a, MODE_STEP, opt, ctx->stream);
    if (e == cudaSuccess) e = cudaEventRecord(e0, ctx->stream);
    for (int r = 0; r < reps && e == cudaSuccess; ++r) e = launch_line_pass<T>(a, MODE_STEP, opt, ctx->stream);
    if (e == cudaSuccess) e = cudaEventRecord(e1, ctx->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      return cuda_fail(ctx, e, "autotune");
    }
    ctx->launches += reps + 2;
    if (ms < *best_ms) {
      *best_ms = ms;
      *best = t;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *best_ms /= reps;
  return DIRAC_OK;
}

template <typename T>
static dirac_status autotune_impl(dirac_ctx* ctx, int reps, int* tx, int* ty) {
  if (!ctx->scratch1) {
    CK(dalloc(ctx, &ctx->scratch1, npts(ctx) * sizeof(Q4<T>)), "scratch");
    CK(dalloc(ctx, &ctx->scratch2, npts(ctx) * sizeof(Q4<T>)), "scratch");
  }
  if (ctx->dt_cached == 0.0) {
    dirac_status s = tables_for_dt<T>(ctx, 0.01);
    if (s != DIRAC_OK) return s;
  }
  float mx, my;
  dirac_status s = tune_pass<T>(ctx, 0, reps, tx, &mx);
  if (s == DIRAC_OK) s = tune_pass<T>(ctx, 1, reps, ty, &my);
  if (s != DIRAC_OK) return s;
  ctx->threads_x = *tx;
  ctx->threads_y = *ty;
  return DIRAC_OK;
}

// ------------------------------------------------------------------------ the ABI
extern "C" {

dirac_status dirac_create(const dirac_grid* grid, const dirac_domain* domain,
                          const dirac_metric* metric, double mass, double c,
                          const dirac_absorber* absorber, dirac_precision precision,
                          void* cuda_stream, dirac_ctx** out) {
  if (!out) return fail(nullptr, DIRAC_EINVAL, "out is NULL");
  *out = nullptr;
  if (!grid || !domain) return fail(nullptr, DIRAC_EINVAL, "grid and domain are required");
  if (!pow2_in(grid->nx, 16, 4096) || !pow2_in(grid->ny, 16, 4096))
    return fail(nullptr, DIRAC_EINVAL, "nx and ny must be powers of two in [16, 4096]");
  if (!(domain->ax > 0.0) || !(domain->ay > 0.0) || !isfinite(domain->ax) || !isfinite(domain->ay))
    return fail(nullptr, DIRAC_EINVAL, "domain half-widths must be positive and finite");
  if (!(c > 0.0) || !isfinite(c) || !isfinite(mass))
    return fail(nullptr, DIRAC_EINVAL, "c must be positive and mass finite");
  if (precision != DIRAC_C64 && precision != DIRAC_C128)
    return fail(nullptr, DIRAC_EINVAL, "unknown precision");
  dirac_absorber ab = {0, 0, 1, 1.0, 0.0};
  if (absorber) {
    ab = *absorber;
    if (ab.width_x < 0 || ab.width_y < 0 || ab.width_x >= grid->nx / 2 ||
        ab.width_y >= grid->ny / 2)
      return fail(nullptr, DIRAC_EINVAL, "absorber widths must be in [0, N/2)");
    if ((ab.width_x > 0 || ab.width_y > 0) && (ab.type < 1 || ab.type > 6))
      return fail(nullptr, DIRAC_EINVAL, "absorber type must be 1..6");
    if (!isfinite(ab.sigma0) || ab.sigma0 < 0.0 || !isfinite(ab.theta))
      return fail(nullptr, DIRAC_EINVAL, "absorber sigma0 must be >= 0 and theta finite");
    if (ab.theta != 0.0 && (ab.width_x > 0 || ab.width_y > 0) && precision != DIRAC_C128)
      return fail(nullptr, DIRAC_EUNSUPPORTED,
                  "complex stretching (theta != 0) needs complex128 (a complex b)");
  }
  int conn = DIRAC_CONN_COVARIANT;
  const double* g_host[3] = {nullptr, nullptr, nullptr};
  if (metric) {
    conn = metric->conn;
    if (conn < 0 || conn > 2) return fail(nullptr, DIRAC_EINVAL, "unknown connection mode");
    g_host[0] = metric->g00;
    g_host[1] = metric->g11;
    g_host[2] = metric->g22;
    const size_t n = (size_t)grid->nx * grid->ny;
    for (int f = 0; f < 3; ++f) {
      if (!g_host[f]) continue;
      for (size_t k = 0; k < n; ++k) {
        const double v = g_host[f][k];
        if (!(v > 0.0) || !isfinite(v))
          return fail(nullptr, DIRAC_EINVAL, "metric entries must be positive and finite");
      }
    }
  }
  dirac_ctx* ctx = new (std::nothrow) dirac_ctx();
  if (!ctx) return fail(nullptr, DIRAC_ENOMEM, "host allocation failed");
  ctx->nx = grid->nx;
  ctx->ny = grid->ny;
  ctx->ax = domain->ax;
  ctx->ay = domain->ay;
  ctx->mass = mass;
  ctx->c = c;
  ctx->prec = precision;
  ctx->conn = conn;
  ctx->abs = ab;
  ctx->u_identity = (mass == 0.0 && conn == DIRAC_CONN_NONE);
  ctx->fault_alloc_at = fault_alloc_from_env();
  cudaGetDevice(&ctx->device);
  if (cuda_stream) {
    ctx->stream = (cudaStream_t)cuda_stream;
  } else {
    cudaError_t e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      dirac_status s = cuda_fail(nullptr, e, "create stream");
      delete ctx;
      return s;
    }
    ctx->own_stream = true;
  }
  dirac_status s = precision == DIRAC_C64 ? create_impl<float>(ctx, g_host)
                                          : create_impl<double>(ctx, g_host);
  if (s != DIRAC_OK) {
    g_create_error = ctx->err;
    dirac_destroy(ctx);
    return s;
  }
  *out = ctx;
  return DIRAC_OK;
}

dirac_status dirac_set_state(dirac_ctx* ctx, const double* psi, int on_device) {
  if (!ctx) return fail(nullptr, DIRAC_EINVAL, "ctx is NULL");
  if (!psi) return fail(ctx, DIRAC_EINVAL, "psi is NULL");
  const size_t n = npts(ctx);
  const double* src = psi;
  if (!on_device) {
    CK(cudaMemcpyAsync(ctx->staging, psi, 4 * n * sizeof(double), cudaMemcpyHostToDevice,
                       ctx->stream),
       "upload state");
    src = ctx->staging;
  }
  if (ctx->prec == DIRAC_C64)
    CK(launch_pack<float>(src, (Q4<float>*)ctx->psi, n, ctx->stream), "pack state");
  else
    CK(launch_pack<double>(src, (Q4<double>*)ctx->psi, n, ctx->stream), "pack state");
  ctx->launches += 1;
  if (!on_device) CK(cudaStreamSynchronize(ctx->stream), "upload state");
  ctx->state_set = true;
  return DIRAC_OK;
}

dirac_status dirac_get_state(dirac_ctx* ctx, double* psi_out, int on_device) {
  if (!ctx) return fail(nullptr, DIRAC_EINVAL, "ctx is NULL");
  if (!psi_out) return fail(ctx, DIRAC_EINVAL, "psi_out is NULL");
  if (!ctx->state_set) return fail(ctx, DIRAC_ESTATE, "no state has been set");
  const size_t n = npts(ctx);
  double* dst = on_device ? psi_out : ctx->staging;
  if (ctx->prec == DIRAC_C64)
    CK(launch_unpack<float>((const Q4<float>*)ctx->psi, dst, n, ctx->stream), "unpack state");
  else
    CK(launch_unpack<double>((const Q4<double>*)ctx->psi, dst, n, ctx->stream), "unpack state");
  ctx->launches += 1;
  if (!on_device) {
    CK(cudaMemcpyAsync(psi_out, ctx->staging, 4 * n * sizeof(double), cudaMemcpyDeviceToHost,
                       ctx->stream),
       "download state");
    CK(cudaStreamSynchronize(ctx->stream), "download state");
    return device_error(ctx);
  }
  return DIRAC_OK;
}

dirac_status dirac_step(dirac_ctx* ctx, long n_steps, double dt) {
  if (!ctx) return fail(nullptr, DIRAC_EINVAL, "ctx is NULL");
  if (n_steps < 0) return fail(ctx, DIRAC_EINVAL, "n_steps must be >= 0");
  if (!(dt > 0.0) || !isfinite(dt)) return fail(ctx, DIRAC_EINVAL, "dt must be positive");
  if (!ctx->state_set) return fail(ctx, DIRAC_ESTATE, "set_state must come before step");
  if (n_steps == 0) return DIRAC_OK;
  return ctx->prec == DIRAC_C64 ? step_impl<float>(ctx, n_steps, dt)
                                : step_impl<double>(ctx, n_steps, dt);
}

dirac_status dirac_observables(dirac_ctx* ctx, dirac_obs* out, double* density_or_NULL) {
  if (!ctx) return fail(nullptr, DIRAC_EINVAL, "ctx is NULL");
  if (!out) return fail(ctx, DIRAC_EINVAL, "out is NULL");
  if (!ctx->state_set) return fail(ctx, DIRAC_ESTATE, "no state has been set");
  return ctx->prec == DIRAC_C64 ? observables_impl<float>(ctx, out, density_or_NULL)
                                : observables_impl<double>(ctx, out, density_or_NULL);
}

dirac_status dirac_synchronize(dirac_ctx* ctx) {
  if (!ctx) return fail(nullptr, DIRAC_EINVAL, "ctx is NULL");
  CK(cudaStreamSynchronize(ctx->stream), "synchronize");
  return device_error(ctx);
}

const char* dirac_last_error(const dirac_ctx* ctx) {
  return ctx ? ctx->err.c_str() : g_create_error.c_str();
}

void dirac_destroy(dirac_ctx* ctx) {
  if (!ctx) return;
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  free_all(ctx);
  if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
}

dirac_status dirac_set_scheme(dirac_ctx* ctx, int scheme) {
  if (!ctx) return fail(nullptr, DIRAC_EINVAL, "ctx is NULL");
  if (scheme < DIRAC_SCHEME_II || scheme > DIRAC_SCHEME_CRANK_NICOLSON)
    return fail(ctx, DIRAC_EINVAL, "unknown scheme");
  if (scheme != ctx->scheme) {
    ctx->scheme = scheme;
    ctx->dt_cached = 0.0;  // the tables of the new order are made on the next step
  }
  return DIRAC_OK;
}

dirac_status dirac_set_potentials(dirac_ctx* ctx, const double* V, const double* Ax,
                                  const double* Ay) {
  if (!ctx) return fail(nullptr, DIRAC_EINVAL, "ctx is NULL");
  const size_t n = npts(ctx);
  const double* src[3] = {V, Ax, Ay};
  double** dst[3] = {&ctx->pot_v, &ctx->pot_ax, &ctx->pot_ay};
  for (int f = 0; f < 3; ++f)
    if (src[f])
      for (size_t k = 0; k < n; ++k)
        if (!isfinite(src[f][k])) return fail(ctx, DIRAC_EINVAL, "potentials must be finite");
  for (int f = 0; f < 3; ++f) {
    ctx->pot_use[f] = src[f] != nullptr;
    if (!src[f]) continue;  // an earlier buffer stays allocated for a later call
    if (!*dst[f]) {
      void* p = nullptr;
      if (dalloc(ctx, &p, n * sizeof(double)) != cudaSuccess)
        return fail(ctx, DIRAC_ENOMEM, "allocate potentials");
      *dst[f] = (double*)p;
    }
    cudaError_t e = cudaMemcpy(*dst[f], src[f], n * sizeof(double), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "copy potentials");
  }
  ctx->has_pot = V || Ax || Ay;
  ctx->dt_cached = 0.0;  // the half-step matrices are made again on the next step
  return DIRAC_OK;
}

dirac_status dirac_set_poly_degree(dirac_ctx* ctx, int degree) {
  if (!ctx) return fail(nullptr, DIRAC_EINVAL, "ctx is NULL");
  if (degree < 1 || degree > 256) return fail(ctx, DIRAC_EINVAL, "degree must be 1..256");
  ctx->poly_degree = degree;
  return DIRAC_OK;
}

dirac_status dirac_set_krylov(dirac_ctx* ctx, double tol, int restart, int max_restarts) {
  if (!ctx) return fail(nullptr, DIRAC_EINVAL, "ctx is NULL");
  if (!(tol >= 0.0) || !isfinite(tol) || restart < 1 || restart > 100 || max_restarts < 0)
    return fail(ctx, DIRAC_EINVAL, "tol >= 0, restart in 1..100, max_restarts >= 0");
  ctx->krylov_tol = tol;
  ctx->krylov_m = restart;
  ctx->krylov_restarts = max_restarts;
  return DIRAC_OK;
}

long dirac_krylov_iterations(const dirac_ctx* ctx) { return ctx ? ctx->krylov_iters : 0; }

dirac_status dirac_set_launch(dirac_ctx* ctx, int threads_x_pass, int threads_y_pass) {
  if (!ctx) return fail(nullptr, DIRAC_EINVAL, "ctx is NULL");
  const int t[2] = {threads_x_pass, threads_y_pass};
  for (int k = 0; k < 2; ++k) {
    const int th = t[k] & ~DIRAC_LAUNCH_ALT_RADIX;
    const bool alt = (t[k] & DIRAC_LAUNCH_ALT_RADIX) != 0;
    if ((th != 0 && th != 256 && th != 512 && th != 1024) || (alt && th != 256 && th != 512))
      return fail(ctx, DIRAC_EINVAL,
                  "shape must be 0 (default), 256, 512 or 1024, or 256 or 512 plus "
                  "DIRAC_LAUNCH_ALT_RADIX");
  }
  ctx->threads_x = threads_x_pass;
  ctx->threads_y = threads_y_pass;
  return DIRAC_OK;
}

long dirac_launch_count(const dirac_ctx* ctx) { return ctx ? ctx->launches : 0; }

dirac_status dirac_test_timeout_next_step(dirac_ctx* ctx) {
  if (!ctx) return fail(nullptr, DIRAC_EINVAL, "ctx is NULL");
  ctx->test_timeout_next = 16;
  return DIRAC_OK;
}

dirac_status dirac_autotune(dirac_ctx* ctx, int reps, int* threads_x, int* threads_y) {
  if (!ctx) return fail(nullptr, DIRAC_EINVAL, "ctx is NULL");
  if (!threads_x || !threads_y || reps < 1) return fail(ctx, DIRAC_EINVAL, "bad arguments");
  if (!ctx->state_set) return fail(ctx, DIRAC_ESTATE, "set_state must come before autotune");
  return ctx->prec == DIRAC_C64 ? autotune_impl<float>(ctx, reps, threads_x, threads_y)
                                : autotune_impl<double>(ctx, reps, threads_x, threads_y);
}

size_t dirac_footprint_bytes(const dirac_grid* grid, dirac_precision precision) {
  if (!grid || grid->nx <= 0 || grid->ny <= 0) return 0;
  return dgb_footprint_bytes(grid->nx, grid->ny, precision);
}

}  // extern "C"
