// Fused line pass: one direction of one Scheme II step for a block of lines.
//
// For every line (a row of the input array, length L):
//   forward FFT along the line -> k-space multiply -> inverse FFT -> pointwise epilogue
//   -> store TRANSPOSED (out[i][line]).
// Two passes make a step: the x pass reads psi[ny][nx] and writes psiT[nx][ny]; the
// y pass reads psiT and writes psi back. Both therefore read whole contiguous lines.
//
// Step mode (Sec. 5.2 eq. second_scheme). In the eigenbasis of sigma_j the k-space
// operator exp(-i dt xi sigma_j) is diagonal: phi_+- = psi_1 +- psi_2 (sigma_x) or
// psi_1 -+ i psi_2 (sigma_y) are multiplied by exp(-+ i dt xi). Each eigencomponent is a
// scalar FFT -> multiply -> inverse FFT chain, computed by its own thread:
//   D_+- = F^-1[ (exp(-+ i dt xi) - 1) / (2L) F phi_+- ]
//   D    = (D_+ + D_-, D_+ - D_-)  (sigma_x)   or   (D_+ + D_-, i (D_+ - D_-))  (sigma_y)
//   psi_new = psi + D + (b - 1) D,  optionally followed by U psi_new
// which equals b Xi + (1 - b) psi with Xi = F^-1[exp(-i dt xi sigma_j) F psi]; writing it
// as a deviation from identity keeps FP32 rounding proportional to |exp(..) - 1|.
// Derivative mode (Sec. 5 eq. trick): out_c = F^-1[ i xi / L  F psi_c ] per component.
//
// FFT: radix-E Stockham autosort (E = 8 or 16 elements per thread). Thread (j, c) of a
// line holds elements j + m L/E (m < E) of component c; that index set is the input of
// the first pass and the output of the last one for any radix sequence, so the global
// load, the k-space multiply and the epilogue happen in registers and only the passes in
// between go through shared memory. L and E are template parameters: all index
// arithmetic folds.
#pragma once
#include <cooperative_groups.h>

#include "common.cuh"

namespace dgb {

namespace cg = cooperative_groups;

enum { MODE_STEP = 0, MODE_DERIV = 1 };

// Per-instance pointers of a batched launch (several simulations of the same grid size
// in one launch); the twiddle table is shared (it depends only on the line length).
template <typename T>
struct InstPtrs {
  const Q4<T>* in;
  Q4<T>* out;
  const T* beta;
  const Q4<T>* u_load;
  const Q4<T>* u_store;
  const Q4<T>* mult;
  const Q4<T>* mult_perm;  // see LinePassArgs
  unsigned test_extra_tx;  // test hook of this instance (see LinePassArgs); 0 normally
};

template <typename T>
struct LinePassArgs {
  const Q4<T>* in;      // [n_lines][L] spinor points
  Q4<T>* out;           // [L][n_lines] spinor points (transposed)
  int L;                // line length = FFT size (power of two, 16..4096)
  int n_lines;          // lines in the input = row length of the output
  int sigma;            // 0: sigma_x (x pass), 1: sigma_y (y pass)
  const Cx<T>* tw;      // per-pass twiddles, see tw_offset (at most L entries)
  const Cx<T>* tw_alt;  // the same for the alternative radix schedule (or nullptr)
  const Q4<T>* mult;    // per k index q: step ((cos - 1) hi, lo, sin hi, lo) / (2L);
                        // derivative (0, 0, xi hi, xi lo) / L
  const Q4<T>* mult_perm;  // 1024-point lines: the step table with entry q at perm1024(q),
                           // read by the 1024-point persistent pass; or nullptr
  const T* beta;        // b - 1 per input point, or nullptr (b = 1)
  const T* beta_im;     // imaginary part of b - 1 (complex stretching), or nullptr
  const Q4<T>* u_load;  // U applied to psi when it is read, or nullptr
  const Q4<T>* u_store; // U applied to psi_new before the store, or nullptr
  int* err;             // device error flag (persistent variant: bounded-wait timeouts)
  const InstPtrs<T>* inst;  // batched launch: per-instance pointers (overrides the above)
  const int* n_inst;        // batched launch: number of active instances (device memory)
  int inst_capacity;        // batched launch: table entries (host side, sizes the grid)
  unsigned test_extra_tx;   // test hook: bytes a bulk copy never delivers (0 normally);
                            // makes the persistent pass's bounded wait run out
  int store_normal;         // 0 = out is [L][n_lines] (transposed store), 1 = out is
                            // [n_lines][L] like `in` (out must not alias in)
  // Batched tick launch (the persistent pass runs every step of a tick in one launch):
  // inst is then the tick's table [tick_k steps][2 passes][inst_capacity], n_inst the
  // active count per step; work items are taken from *tick_queue (zero at launch) and
  // tick_done[i] counts the finished line groups of instance slot i (zero at launch).
  int tick_k;
  int* tick_queue;
  int* tick_done;
};

// Batched launches: a block (or group) of lines belongs to instance `k`; take that
// instance's pointers.
template <typename T>
__device__ __forceinline__ void bind_instance(LinePassArgs<T>& a, int k) {
  const InstPtrs<T> p = a.inst[k];
  a.in = p.in;
  a.out = p.out;
  a.beta = p.beta;
  a.u_load = p.u_load;
  a.u_store = p.u_store;
  a.mult = p.mult;
  a.mult_perm = p.mult_perm;
  a.test_extra_tx = p.test_extra_tx;
}

// Read-only cached loads of the table types.
__device__ __forceinline__ Cx<float> ldg_cx(const Cx<float>* p) {
  const float2 v = __ldg(reinterpret_cast<const float2*>(p));
  return {v.x, v.y};
}
__device__ __forceinline__ Cx<double> ldg_cx(const Cx<double>* p) {
  const double2 v = __ldg(reinterpret_cast<const double2*>(p));
  return {v.x, v.y};
}
__device__ __forceinline__ Q4<float> ldg_q4(const Q4<float>* p) {
  const float4 v = __ldg(reinterpret_cast<const float4*>(p));
  return {v.x, v.y, v.z, v.w};
}
__device__ __forceinline__ Q4<double> ldg_q4(const Q4<double>* p) {
  const double2 a = __ldg(reinterpret_cast<const double2*>(p));
  const double2 b = __ldg(reinterpret_cast<const double2*>(p) + 1);
  return {a.x, a.y, b.x, b.y};
}

// ---------------------------------------------------------------- small DFTs
// Complex additions whose operands need no swap of real and imaginary parts go through
// cadd_p / csub_p: for complex64 one packed-pair instruction (add/sub.rn.f32x2) instead
// of two, with identical results. Additions of a value times +-i keep the scalar form,
// where the swap and sign fold into the operands.
template <typename T, bool INV>
__device__ __forceinline__ void dft2(Cx<T>& a, Cx<T>& b) {
  const Cx<T> t = a;
  a = cadd_p(t, b);
  b = csub_p(t, b);
}

template <typename T, bool INV>
__device__ __forceinline__ void dft4(Cx<T>& x0, Cx<T>& x1, Cx<T>& x2, Cx<T>& x3) {
  const Cx<T> a = cadd_p(x0, x2), b = csub_p(x0, x2), c = cadd_p(x1, x3), d = csub_p(x1, x3);
  const Cx<T> jd = INV ? mul_i(d) : mul_mi(d);
  x0 = cadd_p(a, c);
  x2 = csub_p(a, c);
  x1 = cadd(b, jd);
  x3 = csub(b, jd);
}

// multiply by exp(-+ 2 pi i M / 16) (forward: minus); cos/sin of pi M / 8 as constants
template <typename T, bool INV, int M>
__device__ __forceinline__ Cx<T> w16(Cx<T> a) {
  constexpr double c = (M == 1) ? 0.92387953251128675613 : (M == 2) ? 0.70710678118654752440
                     : (M == 3) ? 0.38268343236508977173 : (M == 6) ? -0.70710678118654752440
                     : (M == 9) ? -0.92387953251128675613 : 0.0;
  constexpr double s = (M == 1) ? 0.38268343236508977173 : (M == 2) ? 0.70710678118654752440
                     : (M == 3) ? 0.92387953251128675613 : (M == 6) ? 0.70710678118654752440
                     : (M == 9) ? -0.38268343236508977173 : 0.0;
  if constexpr (M == 0) return a;
  if constexpr (M == 4) return INV ? mul_i(a) : mul_mi(a);
  const Cx<T> w = {T(c), INV ? T(s) : T(-s)};
  return cmul(a, w);
}

template <typename T, bool INV>
__device__ __forceinline__ void dft8(Cx<T> (&x)[8]) {
  Cx<T> e0 = x[0], e1 = x[2], e2 = x[4], e3 = x[6];
  Cx<T> o0 = x[1], o1 = x[3], o2 = x[5], o3 = x[7];
  dft4<T, INV>(e0, e1, e2, e3);
  dft4<T, INV>(o0, o1, o2, o3);
  o1 = w16<T, INV, 2>(o1);
  o2 = w16<T, INV, 4>(o2);
  o3 = w16<T, INV, 6>(o3);
  x[0] = cadd_p(e0, o0); x[4] = csub_p(e0, o0);
  x[1] = cadd_p(e1, o1); x[5] = csub_p(e1, o1);
  x[2] = cadd(e2, o2); x[6] = csub(e2, o2);
  x[3] = cadd_p(e3, o3); x[7] = csub_p(e3, o3);
}

// Radix-16 butterfly with an optional input twiddle tw[(t - 1) step] on element t
// (t >= 1; tw points at the thread's k within its pass block and step = NS), loaded just
// before the inner DFT4 that consumes it so that only four twiddles are live at a time.
template <typename T, bool INV, bool TW>
__device__ __forceinline__ void dft16(Cx<T> (&x)[16], const Cx<T>* __restrict__ tw = nullptr,
                                      int step = 0) {
  // 16 = 4 x 4: inner DFT4 over n1 of x[4 n1 + n2], twiddle W16^(n2 k1), outer DFT4.
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) {
    if constexpr (TW) {
#pragma unroll
      for (int n1 = 0; n1 < 4; ++n1) {
        const int t = 4 * n1 + n2;
        if (t == 0) continue;
        const Cx<T> w = ldg_cx(tw + (t - 1) * step);
        x[t] = INV ? cmulc(x[t], w) : cmul(x[t], w);
      }
      asm volatile("" ::: "memory");
    }
    dft4<T, INV>(x[n2], x[n2 + 4], x[n2 + 8], x[n2 + 12]);
  }
  x[5] = w16<T, INV, 1>(x[5]);
  x[9] = w16<T, INV, 2>(x[9]);
  x[13] = w16<T, INV, 3>(x[13]);
  x[6] = w16<T, INV, 2>(x[6]);
  x[10] = w16<T, INV, 4>(x[10]);
  x[14] = w16<T, INV, 6>(x[14]);
  x[7] = w16<T, INV, 3>(x[7]);
  x[11] = w16<T, INV, 6>(x[11]);
  x[15] = w16<T, INV, 9>(x[15]);
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) dft4<T, INV>(x[4 * k1], x[4 * k1 + 1], x[4 * k1 + 2], x[4 * k1 + 3]);
  // x[4 k1 + k2] holds y[k1 + 4 k2]
  Cx<T> y[16];
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1)
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) y[k1 + 4 * k2] = x[4 * k1 + k2];
#pragma unroll
  for (int i = 0; i < 16; ++i) x[i] = y[i];
}

template <typename T, int R, bool INV>
__device__ __forceinline__ void dftR(Cx<T> (&x)[R]) {
  if constexpr (R == 2) {
    dft2<T, INV>(x[0], x[1]);
  } else if constexpr (R == 4) {
    dft4<T, INV>(x[0], x[1], x[2], x[3]);
  } else if constexpr (R == 8) {
    dft8<T, INV>(x);
  } else {
    dft16<T, INV, false>(x);
  }
}

// ------------------------------------------------------------- geometry
__host__ __device__ constexpr int ilog2c(int v) { return v <= 1 ? 0 : 1 + ilog2c(v >> 1); }

// Twiddle table layout: the passes after the first (span NS = E, E^2, ...) each own a
// block [(t - 1) NS + k] = exp(-2 pi i t k / (NS R)), t = 1..R-1, k < NS, so that the
// lanes of a warp (consecutive k) read consecutive entries. Every pass but the last has
// radix E; the block of span NS starts after the (E - 1) NS' entries of each earlier span.
__host__ __device__ constexpr int tw_offset(int NS, int E) {
  return NS <= E ? 0 : tw_offset(NS / E, E) + (E - 1) * (NS / E);
}

// Compile-time launch geometry for line length L, LPC lines per CTA and E elements per
// thread. Shared memory per line: two components of P = L + L/E padded slots (one pad slot
// per E keeps the strided Stockham writes conflict-free), the second component offset by
// half a 128-B bank row (a few short lines take other offsets) so that the two threads of
// a point pair never collide, plus a small line pad for short lines. A CPU model of every
// access pattern (all L, both precisions, E = 8 and 16, 256..1024 threads) finds no bank
// conflicts with these offsets.
template <typename T, int L, int E>
struct SmemPlan {
  static constexpr int B = sizeof(T) == 4 ? 16 : 8;  // slots per 128 B
  static constexpr bool F = sizeof(T) == 4;
  static constexpr int CM = (E == 16) ? ((!F && L == 32) ? 2 : B / 2)
                                      : ((L == 16) ? 2 : (F && L == 32) ? 4 : B / 2);
  static constexpr int EXTRA = (E == 16 && F && L == 32) ? 2 : (E == 16 && F && L == 64) ? 4 : 0;
};

template <typename T, int L_, int LPC_, int E_>
struct Geo {
  static constexpr int L = L_;
  static constexpr int LPC = LPC_;
  static constexpr int E = E_;                  // elements per thread
  static constexpr int SH = ilog2c(E);          // pad one slot every E slots
  static constexpr int J = L / E;               // index groups per line
  static constexpr int TPL = 2 * J;             // threads per line (two components)
  static constexpr int THREADS = LPC * TPL;
  static constexpr int B = SmemPlan<T, L, E>::B;
  static constexpr int P = L + L / E;
  static constexpr int CM = SmemPlan<T, L, E>::CM;
  static constexpr int COMP = P + (((CM - P % B) % B) + B) % B;
  static constexpr int STRIDE = 2 * COMP + SmemPlan<T, L, E>::EXTRA;
  // Lines gathered per output segment: 4 (64 B complex64, 128 B complex128), 2 for
  // 4096-point lines. A cluster of 4 CTAs packs the GPCs better than 8 and measured faster
  // at 1024..2048 points; 4096-point lines run one CTA per SM, where only 36 clusters of 4
  // (144 CTAs) but 76 clusters of 2 (every SM) are resident: clusters of 2 measured 6-7%
  // faster at 4096^2 in both precisions.
  static constexpr int G = L == 4096 ? 2 : 4;
  static constexpr int CS = LPC >= G ? 1 : G / LPC;   // CTAs per cluster
  static constexpr int GL = LPC * CS;                  // lines gathered per output segment
  static constexpr int LOG2L = ilog2c(L);
  static constexpr int NPASS = (LOG2L + SH - 1) / SH;
  static constexpr int RL = 1 << (LOG2L - (NPASS - 1) * SH);
  static constexpr size_t FFT_BYTES = (size_t)LPC * STRIDE * sizeof(Cx<T>);
  static constexpr size_t STAGE_BYTES = (size_t)LPC * (L + 1) * sizeof(Q4<T>);
  static constexpr size_t SMEM = FFT_BYTES > STAGE_BYTES ? FFT_BYTES : STAGE_BYTES;
  static constexpr int NIT = (L / CS) * GL / THREADS;  // transposed-store items per thread
  static_assert((L & (L - 1)) == 0 && L >= 16, "L must be a power of two >= 16");
  static_assert(E == 8 || E == 16, "E must be 8 or 16");
  static_assert(THREADS <= 1024, "at most 1024 threads per CTA");
  static_assert((L / CS) * GL == NIT * THREADS && NIT % 2 == 0, "store items must divide");
};

template <int E>
__device__ __forceinline__ int spad(int i) { return i + (i >> ilog2c(E)); }

// ------------------------------------------------------------- Stockham passes
// Butterfly u (u < E/R) works on index s = j + u L/E and elements v[u + t E/R]
// (t < R): twiddle by W_{NS R}^{t k} with k = s mod NS (from the pass's table block),
// then the R-point DFT.
template <typename T, int L, int E, int R, int NS, bool INV>
__device__ __forceinline__ void pass_compute(Cx<T> (&v)[E], int j, const Cx<T>* __restrict__ tw) {
  constexpr int NB = E / R, J = L / E;
#pragma unroll
  for (int u = 0; u < NB; ++u) {
    Cx<T> x[R];
#pragma unroll
    for (int t = 0; t < R; ++t) x[t] = v[u + t * NB];
    if constexpr (NS > 1 && R == 16) {
      const int k = (j + u * J) & (NS - 1);
      dft16<T, INV, true>(x, tw + tw_offset(NS, E) + k, NS);
    } else {
      if constexpr (NS > 1) {
        const int k = (j + u * J) & (NS - 1);
        const Cx<T>* twk = tw + tw_offset(NS, E) + k;
        if constexpr (sizeof(T) == 4 && (R == 8 || R == 4)) {
          // FP32 radix-8/4: W^k, W^2k and W^4k from the table, the others as products of
          // two or three of them (at most two extra roundings per twiddle)
          Cx<T> w[8];
          w[1] = ldg_cx(twk);
          w[2] = ldg_cx(twk + NS);
          w[3] = cmul(w[1], w[2]);
          if constexpr (R == 8) {
            w[4] = ldg_cx(twk + 3 * NS);
            w[5] = cmul(w[4], w[1]);
            w[6] = cmul(w[4], w[2]);
            w[7] = cmul(w[4], w[3]);
          }
#pragma unroll
          for (int t = 1; t < R; ++t) x[t] = INV ? cmulc(x[t], w[t]) : cmul(x[t], w[t]);
        } else {
#pragma unroll
          for (int t = 1; t < R; ++t) {
            const Cx<T> w = ldg_cx(twk + (t - 1) * NS);
            x[t] = INV ? cmulc(x[t], w) : cmul(x[t], w);
          }
        }
      }
      dftR<T, R, INV>(x);
    }
#pragma unroll
    for (int t = 0; t < R; ++t) v[u + t * NB] = x[t];
  }
}

// Output (u, t) of a pass goes to index (s - k) R + k + t NS (padded).
template <typename T, int L, int E, int R, int NS>
__device__ __forceinline__ void pass_store(const Cx<T> (&v)[E], Cx<T>* buf, int j) {
  constexpr int NB = E / R, J = L / E;
#pragma unroll
  for (int u = 0; u < NB; ++u) {
    const int s = j + u * J;
    const int k = s & (NS - 1);
    const int base = spad<E>((s - k) * R + k);
#pragma unroll
    for (int t = 0; t < R; ++t) {
      // NS = 1 only in the first pass (radix E, base a multiple of E + 1 slots); there the
      // t-th output is the next slot. NS a multiple of E adds NS + NS/E slots per step.
      const int o = (NS == 1) ? base + t : base + t * (NS + NS / E);
      if (dbg_in(o, L + L / E)) buf[o] = v[u + t * NB];
    }
  }
}

template <typename T, int L, int E>
__device__ __forceinline__ void pass_load(Cx<T> (&v)[E], const Cx<T>* buf, int j) {
  constexpr int J = L / E;
  if constexpr (J % E == 0) {
    const int b = spad<E>(j);
#pragma unroll
    for (int m = 0; m < E; ++m) {
      const int o = b + m * (J + J / E);
      v[m] = dbg_in(o, L + L / E) ? buf[o] : Cx<T>{T(0), T(0)};
    }
  } else {
#pragma unroll
    for (int m = 0; m < E; ++m) {
      const int o = spad<E>(j + m * J);
      v[m] = dbg_in(o, L + L / E) ? buf[o] : Cx<T>{T(0), T(0)};
    }
  }
}

template <typename T, int L, int E, bool INV, int P = 0, int NS = 1>
__device__ __forceinline__ void fft_passes(Cx<T> (&v)[E], Cx<T>* buf, int j, const Cx<T>* tw) {
  constexpr int SH = ilog2c(E);
  constexpr int LOG2L = ilog2c(L);
  constexpr int NPASS = (LOG2L + SH - 1) / SH;
  constexpr int RL = 1 << (LOG2L - (NPASS - 1) * SH);
  constexpr int R = (P + 1 == NPASS) ? RL : E;
  pass_compute<T, L, E, R, NS, INV>(v, j, tw);
  if constexpr (P + 1 < NPASS) {
    __syncthreads();  // everyone has finished reading the buffer
    pass_store<T, L, E, R, NS>(v, buf, j);
    __syncthreads();
    pass_load<T, L, E>(v, buf, j);
    fft_passes<T, L, E, INV, P + 1, NS * R>(v, buf, j, tw);
  }
}

// ------------------------------------------------------------------ the kernel
// Occupancy target: FP32 radix-8 CTAs fill 1024 threads per SM at <= 64 registers (the
// E = 8 state fits without spilling); FP32 radix-16 CTAs 512 threads per SM at <= 128
// registers; FP64 CTAs take up to 128 registers (the FP64 path is ALU bound).
template <typename T, int THREADS, int E>
struct MinBlocks {
  static constexpr int want = sizeof(T) == 4 ? (E == 8 ? 1024 : 512) / THREADS : 1;
  static constexpr int value = want < 1 ? 1 : want;
};

// Row c of U psi for U = [[c0 + i c3, c1 - i c2], [c1 + i c2, c0 - i c3]] stored as
// u = (c0 - 1, c1, c2, c3): own = psi_c, oth = psi_(1-c).
template <typename T>
__device__ __forceinline__ Cx<T> apply_u_row(const Q4<T>& u, Cx<T> own, Cx<T> oth, int c) {
  const T s3 = c ? -u.w : u.w, s2 = c ? u.z : -u.z;
  // own + (c0-1) own + i s3 own + (c1 + i s2) oth
  const T re = u.x * own.re - s3 * own.im + u.y * oth.re - s2 * oth.im;
  const T im = u.x * own.im + s3 * own.re + u.y * oth.im + s2 * oth.re;
  return {own.re + re, own.im + im};
}

template <typename T>
__device__ __forceinline__ Cx<T> shfl_pair(Cx<T> v) {
  return {__shfl_xor_sync(0xffffffffu, v.re, 1), __shfl_xor_sync(0xffffffffu, v.im, 1)};
}

template <typename T, int L, int LPC, int E, int MODE>
__global__ void __launch_bounds__(Geo<T, L, LPC, E>::THREADS,
                                  MinBlocks<T, Geo<T, L, LPC, E>::THREADS, E>::value)
    line_pass_kernel(LinePassArgs<T> a) {
  using Gm = Geo<T, L, LPC, E>;
  constexpr int J = Gm::J;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Cx<T>* smem = reinterpret_cast<Cx<T>*>(smem_raw);

  // batched launch: blocks of one instance are consecutive (whole clusters), and blocks
  // past the active instances leave at once (together with their cluster)
  int blk = blockIdx.x;
  if (a.inst) {
    const int per_inst = a.n_lines / LPC;
    const int k = blk / per_inst;
    if (k >= *a.n_inst) return;
    bind_instance(a, k);
    blk -= k * per_inst;
  }
  const int tid = threadIdx.x;
  const int lcta = tid / Gm::TPL;
  const int r = tid - lcta * Gm::TPL;
  const int c = r & 1;        // eigencomponent (step) or component (derivative)
  const int j = r >> 1;
  const size_t row = (size_t)(blk * LPC + lcta) * L;
  Cx<T>* buf = smem + lcta * Gm::STRIDE + c * Gm::COMP;
  const T sg = c ? T(-1) : T(1);
  // component c of point gi (the pair of threads reads one 2x8-B / 2x16-B point together)
  const Cx<T>* in_c = reinterpret_cast<const Cx<T>*>(a.in) + c;

  Cx<T> v[E];
  // ---- load psi at j + m L/E and form this thread's component
#pragma unroll
  for (int m = 0; m < E; ++m) {
    if ((m & 3) == 0) asm volatile("" ::: "memory");
    const size_t gi = row + j + m * J;
    Cx<T> own = dbg_in(gi, (size_t)a.n_lines * L) ? in_c[2 * gi] : Cx<T>{T(0), T(0)};
    if constexpr (MODE == MODE_STEP) {
      Cx<T> oth = shfl_pair(own);
      if (a.u_load) {
        const Q4<T> u = ldg_q4(a.u_load + gi);
        own = apply_u_row(u, own, oth, c);
        oth = shfl_pair(own);
      }
      const Cx<T> p1 = c ? oth : own, p2 = c ? own : oth;
      if (a.sigma == 0) v[m] = {p1.re + sg * p2.re, p1.im + sg * p2.im};
      else v[m] = {p1.re + sg * p2.im, p1.im - sg * p2.re};
    } else {
      v[m] = own;
    }
  }

  fft_passes<T, L, E, false>(v, buf, j, a.tw);

  // ---- k-space multiply at q = j + m L/E (the table carries the inverse FFT's scale)
#pragma unroll
  for (int m = 0; m < E; ++m) {
    if ((m & 3) == 0) asm volatile("" ::: "memory");
    const Q4<T> q = ldg_q4(a.mult + j + m * J);
    const T vr = v[m].re, vi = v[m].im;
    if constexpr (MODE == MODE_DERIV) {
      if constexpr (sizeof(T) == 4) {
        v[m] = {-(q.z * vi + q.w * vi), q.z * vr + q.w * vr};
      } else {
        v[m] = {-q.z * vi, q.z * vr};
      }
    } else {
      // eigenvalue +1 (c = 0): exp(-i th) - 1 = (cos - 1) - i sin; -1 (c = 1): + i sin
      const T sh = -sg * q.z, sl = -sg * q.w;
      if constexpr (sizeof(T) == 4) {
        v[m] = {q.x * vr + ((q.y * vr - sl * vi) - sh * vi),
                q.x * vi + ((q.y * vi + sl * vr) + sh * vr)};
      } else {
        v[m] = {q.x * vr - sh * vi, q.x * vi + sh * vr};
      }
    }
  }

  {
    // The inverse FFT's index and twiddle-address arithmetic equals the forward one's;
    // an opaque copy of j and buf makes the compiler recompute it instead of keeping
    // every pass's values live across the k-space multiply (which spilled).
    int j2 = j;
    Cx<T>* buf2 = buf;
    asm volatile("" : "+r"(j2), "+l"(buf2));
    fft_passes<T, L, E, true>(v, buf2, j2, a.tw);
  }

  // ---- epilogue into the staging buffer [lcta][i] (line stride L + 1 points); thread c
  // writes component c of each point
  __syncthreads();  // the FFT buffers are free again
  Q4<T>* stage = reinterpret_cast<Q4<T>*>(smem_raw);
  Cx<T>* my_stage = reinterpret_cast<Cx<T>*>(stage + (size_t)lcta * (L + 1)) + c;
#pragma unroll
  for (int m = 0; m < E; ++m) {
    if ((m & 3) == 0) asm volatile("" ::: "memory");
    const int i = j + m * J;
    if constexpr (MODE == MODE_STEP) {
      const size_t gi = row + i;
      // D_c from the two eigencomponents: sigma_x (D+ + D-, D+ - D-),
      // sigma_y (D+ + D-, i (D+ - D-))
      const Cx<T> oth = shfl_pair(v[m]);
      const Cx<T> dp = c ? oth : v[m], dm = c ? v[m] : oth;
      Cx<T> d;
      if (c == 0) d = cadd_p(dp, dm);
      else d = a.sigma == 0 ? csub_p(dp, dm) : mul_i(csub_p(dp, dm));
      const bool gi_ok = dbg_in(gi, (size_t)a.n_lines * L);
      Cx<T> p = gi_ok ? in_c[2 * gi] : Cx<T>{T(0), T(0)};
      if (a.u_load && gi_ok) p = apply_u_row(ldg_q4(a.u_load + gi), p, shfl_pair(p), c);
      const T bm1 = (a.beta && gi_ok) ? a.beta[gi] : T(0);
      // (p + d) + (b - 1) d
      Cx<T> o = cfma_p(bm1, d, cadd_p(p, d));
      if (a.beta_im) {  // complex b - 1: add i Im(b - 1) d
        const T bi = gi_ok ? a.beta_im[gi] : T(0);
        o = {o.re - bi * d.im, o.im + bi * d.re};
      }
      if (a.u_store && gi_ok) o = apply_u_row(ldg_q4(a.u_store + gi), o, shfl_pair(o), c);
      if (a.store_normal) {
        if (gi_ok) reinterpret_cast<Cx<T>*>(a.out)[2 * gi + c] = o;
      }
      else if (dbg_in(i, L + 1)) my_stage[2 * i] = o;
    } else {
      if (a.store_normal) {
        if (dbg_in(row + i, (size_t)a.n_lines * L))
          reinterpret_cast<Cx<T>*>(a.out)[2 * (row + i) + c] = v[m];
      }
      else if (dbg_in(i, L + 1)) my_stage[2 * i] = v[m];
    }
  }

  // ---- transposed store: the cluster's GL lines go out as contiguous segments
  // out[i][line0 .. line0 + GL); CTA rank q writes rows i of its L/CS slice. Remote
  // (DSMEM) reads are issued in two rounds of four before the matching global stores.
  constexpr int CS = Gm::CS, GL = Gm::GL, ROWS = L / CS;
  int rank = 0;
  if constexpr (CS > 1) {
    rank = (int)cg::this_cluster().block_rank();
    cg::this_cluster().sync();
  } else {
    __syncthreads();
  }
  const int line0 = (blk / CS) * GL;
  const int i0 = rank * ROWS;
  constexpr int HALF = Gm::NIT / 2;
  // (a normal-layout store happened in the epilogue)
  if (!a.store_normal) {
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    Q4<T> val[HALF];
#pragma unroll
    for (int q = 0; q < HALF; ++q) {
      const int it = tid + (h * HALF + q) * Gm::THREADS;
      const int g = it % GL;
      const int i = i0 + it / GL;
      const int owner = g / LPC;
      const Q4<T>* src = stage;
      if constexpr (CS > 1) {
        if (owner != rank) src = cg::this_cluster().map_shared_rank(stage, owner);
      }
      const size_t si = (size_t)(g - owner * LPC) * (L + 1) + i;
      val[q] = dbg_in(si, (size_t)LPC * (L + 1)) ? src[si] : Q4<T>{T(0), T(0), T(0), T(0)};
    }
#pragma unroll
    for (int q = 0; q < HALF; ++q) {
      const int it = tid + (h * HALF + q) * Gm::THREADS;
      const int g = it % GL;
      const int i = i0 + it / GL;
      if (dbg_in((size_t)i * a.n_lines + line0 + g, (size_t)a.n_lines * L))
        a.out[(size_t)i * a.n_lines + line0 + g] = val[q];
    }
  }
  }
  if constexpr (CS > 1) cg::this_cluster().sync();
}

}  // namespace dgb
