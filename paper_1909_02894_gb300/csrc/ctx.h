// Definition of the opaque context (library-internal; shared by the ABI and the batch).
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/dirac.h"

struct dirac_ctx {
  int nx = 0, ny = 0;
  double ax = 0, ay = 0, mass = 0, c = 1;
  dirac_precision prec = DIRAC_C64;
  int conn = 0;
  dirac_absorber abs = {0, 0, 1, 1.0, 0.0};
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int device = 0;
  bool u_identity = false;  // no mass and no connection: U = I exactly

  // FP64 fields in the normal layout [ny][nx]
  double *a1 = nullptr, *a2 = nullptr, *meff = nullptr, *w = nullptr, *omx = nullptr,
         *omy = nullptr;
  double *sxinv = nullptr, *syinv = nullptr;
  double *sxinv_im = nullptr, *syinv_im = nullptr;  // complex stretching (theta != 0)
  // state and per-pass coefficients in the state precision
  void *psi = nullptr, *psiT = nullptr;
  void *beta1 = nullptr, *beta2T = nullptr;
  void *beta1_im = nullptr, *beta2T_im = nullptr;  // complex stretching: Im(b - 1)
  void *u_n = nullptr, *u_t = nullptr, *u2_t = nullptr;
  void *tw_x_alt = nullptr, *tw_y_alt = nullptr;  // twiddles of the alternative radix
  void *tw_x = nullptr, *tw_y = nullptr, *mult_x = nullptr, *mult_y = nullptr,
       *dmult_x = nullptr, *dmult_y = nullptr;
  double* staging = nullptr;  // [2][ny][nx] complex128 for host transfers
  void *scratch1 = nullptr, *scratch2 = nullptr;
  double *partials = nullptr, *result = nullptr, *density = nullptr;

  int scheme = DIRAC_SCHEME_II;
  int poly_degree = 8;
  void* pool[3] = {nullptr, nullptr, nullptr};  // polynomial schemes: term buffers
  double bmax[2] = {-1.0, -1.0};                // max |b1|, |b2| (Chebyshev bound)
  // static potentials (device FP64 [ny][nx], null = 0) and the general half-step matrices
  double *pot_v = nullptr, *pot_ax = nullptr, *pot_ay = nullptr;
  bool pot_use[3] = {false, false, false};  // V, Ax, Ay set
  bool has_pot = false;
  void *ug = nullptr, *ug2 = nullptr;  // U and U^2, two Q4 per point
  // Scheme I: Krylov solver settings and buffers
  double krylov_tol = 0.0;  // 0 = precision default
  int krylov_m = 20, krylov_restarts = 100;
  long krylov_iters = 0;
  std::vector<void*> kv;            // basis V_0 .. V_m (state-sized)
  void* k_rhs = nullptr;            // G~ psi
  void** k_vptr = nullptr;          // device copy of the basis pointers
  double* k_partials = nullptr;     // inner-product partial sums
  double* k_coef = nullptr;         // combination coefficients (device)
  // complex64 axes of 1024 points: the step tables (x at dt and dt/2, y) in the order of
  // perm1024, for the 1024-point persistent pass
  void *mult_px = nullptr, *mult_py = nullptr, *mult_pxh = nullptr;
  void *mult_xh = nullptr, *u2_n = nullptr;  // symmetric order: x multipliers at dt/2,
                                             // U^2 in the normal layout
  int* d_err = nullptr;       // device error flag written by bounded waits
  double dt_cached = 0.0;
  bool state_set = false;
  int threads_x = 0, threads_y = 0;
  unsigned test_timeout_next = 0;  // test hook: next dirac_step's waits run out
  // Host-side fault injection (DIRAC_FAULT=alloc:N at creation): the N-th device
  // allocation of this context fails as if the device were out of memory; 0 = off.
  int fault_alloc_at = 0;
  int n_allocs = 0;
  long launches = 0;
  std::string err;
  std::vector<void*> allocs;
};

// Library-internal helpers implemented in dirac_api.cu.
dirac_status dgb_tables_for_dt(dirac_ctx* ctx, double dt);
size_t dgb_footprint_bytes(int nx, int ny, dirac_precision prec);
// Launch option (0, 1, 2 = persistent) for a pass of line length L.
int dgb_pass_opt(const dirac_ctx* ctx, int threads, int L);
