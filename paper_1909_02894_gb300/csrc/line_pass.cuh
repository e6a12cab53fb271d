// Fused line pass: one direction of one Scheme II step for a block of lines.
//
// For every line (a row of the input array, length L) and both spinor components:
//   forward FFT along the line  ->  k-space multiply  ->  inverse FFT  ->  pointwise
//   epilogue  ->  store TRANSPOSED (out[i][line]).
// Two passes make a step: the x pass reads psi[ny][nx] and writes psiT[nx][ny]; the
// y pass reads psiT and writes psi back. Both therefore read whole contiguous lines.
//
// Step mode (Sec. 5.2 eq. second_scheme, written as a deviation from identity):
//   D = F^-1[ (exp(-i dt xi sigma_j) - I) / L  F psi ]      (unnormalised inverse FFT)
//   psi_new = psi + b D = psi + D + (b - 1) D,  then optionally U psi_new
// which equals b Xi + (1 - b) psi with Xi = F^-1[exp(-i dt xi sigma_j) F psi].
// Derivative mode (Sec. 5 eq. trick): out = F^-1[ i xi / L  F psi ] per component.
//
// FFT: radix-E Stockham autosort in registers with shared-memory exchanges between
// passes. Thread j of a line holds elements j + m L/E (m < E) of both components; that
// index set is the input of the first pass and the output of the last one for any
// radix sequence, so the global load, the k-space multiply and the global store all
// happen in registers.
#pragma once
#include <cooperative_groups.h>

#include "common.cuh"

namespace dgb {

namespace cg = cooperative_groups;

enum { MODE_STEP = 0, MODE_DERIV = 1 };

template <typename T>
struct LinePassArgs {
  const Q4<T>* in;      // [n_lines][L] spinor points
  Q4<T>* out;           // [L][n_lines] spinor points (transposed)
  int L;                // line length = FFT size (power of two, >= 16)
  int n_lines;          // lines in the input = row length of the output
  int sigma;            // 0: sigma_x (x pass), 1: sigma_y (y pass)
  const Cx<T>* tw;      // tw[m] = exp(-2 pi i m / L), m < L
  const Q4<T>* mult;    // per k index q: step (c-1 hi, c-1 lo, s hi, s lo) / L;
                        // derivative (0, 0, xi hi, xi lo) / L
  const T* beta;        // b - 1 per input point, or nullptr (b = 1)
  const Q4<T>* u_load;  // U applied to psi when it is read, or nullptr
  const Q4<T>* u_store; // U applied to psi_new before the store, or nullptr
  int lpc;              // lines per CTA
  int cs;               // CTAs per cluster (1 = no cluster)
};

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
template <typename T, bool INV>
__device__ __forceinline__ void dft2(Cx<T>& a, Cx<T>& b) {
  Cx<T> t = a;
  a = cadd(t, b);
  b = csub(t, b);
}

template <typename T, bool INV>
__device__ __forceinline__ void dft4(Cx<T>& x0, Cx<T>& x1, Cx<T>& x2, Cx<T>& x3) {
  Cx<T> a = cadd(x0, x2), b = csub(x0, x2), c = cadd(x1, x3), d = csub(x1, x3);
  Cx<T> jd = INV ? mul_i(d) : mul_mi(d);
  x0 = cadd(a, c);
  x2 = csub(a, c);
  x1 = cadd(b, jd);
  x3 = csub(b, jd);
}

// multiply by exp(-+ 2 pi i m / 16) (forward: minus)
template <typename T, bool INV, int M>
__device__ __forceinline__ Cx<T> w16(Cx<T> a) {
  constexpr double PI = 3.14159265358979323846264338327950288;
  // cos and sin of pi M / 8 folded at compile time
  constexpr double c = (M == 0) ? 1.0 : (M == 1) ? 0.92387953251128675613 : (M == 2) ? 0.70710678118654752440
                     : (M == 3) ? 0.38268343236508977173 : (M == 4) ? 0.0 : (M == 6) ? -0.70710678118654752440
                     : (M == 9) ? -0.92387953251128675613 : 0.0;
  constexpr double s = (M == 0) ? 0.0 : (M == 1) ? 0.38268343236508977173 : (M == 2) ? 0.70710678118654752440
                     : (M == 3) ? 0.92387953251128675613 : (M == 4) ? 1.0 : (M == 6) ? 0.70710678118654752440
                     : (M == 9) ? -0.38268343236508977173 : 0.0;
  (void)PI;
  if (M == 0) return a;
  if (M == 4) return INV ? mul_i(a) : mul_mi(a);
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
  x[0] = cadd(e0, o0); x[4] = csub(e0, o0);
  x[1] = cadd(e1, o1); x[5] = csub(e1, o1);
  x[2] = cadd(e2, o2); x[6] = csub(e2, o2);
  x[3] = cadd(e3, o3); x[7] = csub(e3, o3);
}

template <typename T, bool INV>
__device__ __forceinline__ void dft16(Cx<T> (&x)[16]) {
  // 16 = 4 x 4: inner DFT4 over n1 of x[4 n1 + n2], twiddle W16^(n2 k1), outer DFT4.
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) dft4<T, INV>(x[n2], x[n2 + 4], x[n2 + 8], x[n2 + 12]);
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
    dft16<T, INV>(x);
  }
}

// Shared-memory padding: one slot every PADK complex slots keeps the strided Stockham
// writes free of bank conflicts (8-byte slots: 16 per 128 B; 16-byte slots: 8).
template <typename T>
struct Pad {
  static constexpr int K = (sizeof(T) == 4) ? 16 : 8;
  static constexpr int SH = (sizeof(T) == 4) ? 4 : 3;
  __device__ __forceinline__ static int idx(int i) { return i + (i >> SH); }
  __host__ __device__ static int len(int L) { return L + L / K; }
};

// One radix-R Stockham pass on the registers of one thread (both components):
// butterfly u (u < E/R) works on index s = j + u L/E, reads v[u + t E/R] (t < R),
// twiddles by W_{Ns R}^{t k} with k = s mod Ns and applies the R-point DFT.
template <typename T, int E, int R, bool INV>
__device__ __forceinline__ void stockham_pass(Cx<T> (&v1)[E], Cx<T> (&v2)[E], int j, int L,
                                              int Ns, const Cx<T>* __restrict__ tw) {
  constexpr int NB = E / R;
#pragma unroll
  for (int u = 0; u < NB; ++u) {
    const int s = j + u * (L / E);
    const int k = s & (Ns - 1);
    Cx<T> x1[R], x2[R];
#pragma unroll
    for (int t = 0; t < R; ++t) {
      x1[t] = v1[u + t * NB];
      x2[t] = v2[u + t * NB];
    }
    if (Ns > 1) {
      const int step = k * (L / (Ns * R));
#pragma unroll
      for (int t = 1; t < R; ++t) {
        const Cx<T> w = ldg_cx(tw + t * step);
        if (INV) {
          x1[t] = cmulc(x1[t], w);
          x2[t] = cmulc(x2[t], w);
        } else {
          x1[t] = cmul(x1[t], w);
          x2[t] = cmul(x2[t], w);
        }
      }
    }
    dftR<T, R, INV>(x1);
    dftR<T, R, INV>(x2);
#pragma unroll
    for (int t = 0; t < R; ++t) {
      v1[u + t * NB] = x1[t];
      v2[u + t * NB] = x2[t];
    }
  }
}

// Write the outputs of a radix-R pass to shared memory: output of (u, t) goes to
// (s - k) R + k + t Ns.
template <typename T, int E, int R>
__device__ __forceinline__ void stockham_store(const Cx<T> (&v1)[E], const Cx<T> (&v2)[E],
                                               Cx<T>* b1, Cx<T>* b2, int j, int L, int Ns) {
  constexpr int NB = E / R;
#pragma unroll
  for (int u = 0; u < NB; ++u) {
    const int s = j + u * (L / E);
    const int k = s & (Ns - 1);
    const int base = (s - k) * R + k;
#pragma unroll
    for (int t = 0; t < R; ++t) {
      const int o = Pad<T>::idx(base + t * Ns);
      b1[o] = v1[u + t * NB];
      b2[o] = v2[u + t * NB];
    }
  }
}

template <typename T, int E, bool INV>
__device__ __forceinline__ void run_pass(int R, Cx<T> (&v1)[E], Cx<T> (&v2)[E], int j, int L,
                                         int Ns, const Cx<T>* tw) {
  if constexpr (E == 16) {
    if (R == 16) { stockham_pass<T, E, 16, INV>(v1, v2, j, L, Ns, tw); return; }
  }
  if (R == 8) { stockham_pass<T, E, 8, INV>(v1, v2, j, L, Ns, tw); return; }
  if (R == 4) { stockham_pass<T, E, 4, INV>(v1, v2, j, L, Ns, tw); return; }
  stockham_pass<T, E, 2, INV>(v1, v2, j, L, Ns, tw);
}

template <typename T, int E>
__device__ __forceinline__ void run_store(int R, const Cx<T> (&v1)[E], const Cx<T> (&v2)[E],
                                          Cx<T>* b1, Cx<T>* b2, int j, int L, int Ns) {
  if constexpr (E == 16) {
    if (R == 16) { stockham_store<T, E, 16>(v1, v2, b1, b2, j, L, Ns); return; }
  }
  if (R == 8) { stockham_store<T, E, 8>(v1, v2, b1, b2, j, L, Ns); return; }
  if (R == 4) { stockham_store<T, E, 4>(v1, v2, b1, b2, j, L, Ns); return; }
  stockham_store<T, E, 2>(v1, v2, b1, b2, j, L, Ns);
}

template <typename T, int E>
__device__ __forceinline__ void smem_load(Cx<T> (&v1)[E], Cx<T> (&v2)[E], const Cx<T>* b1,
                                          const Cx<T>* b2, int j, int L) {
#pragma unroll
  for (int m = 0; m < E; ++m) {
    const int o = Pad<T>::idx(j + m * (L / E));
    v1[m] = b1[o];
    v2[m] = b2[o];
  }
}

// Full FFT (forward or inverse, unnormalised) of the E-element register sets of a line.
// On entry v holds elements j + m L/E of the input; on exit the same indices of the
// output. Passes: radix E first, then the remaining radix rl last; each pass but the last
// goes through shared memory (b1, b2 per component). With the small radix last and the
// padded layout every shared-memory access pattern is free of bank conflicts.
template <typename T, int E, bool INV>
__device__ __forceinline__ void line_fft(Cx<T> (&v1)[E], Cx<T> (&v2)[E], Cx<T>* b1, Cx<T>* b2,
                                         int j, int L, int npass, int rl, const Cx<T>* tw) {
  int Ns = 1;
  for (int p = 0; p < npass; ++p) {
    const int R = (p + 1 == npass) ? rl : E;
    run_pass<T, E, INV>(R, v1, v2, j, L, Ns, tw);
    if (p + 1 < npass) {
      __syncthreads();  // everyone has finished reading the buffer
      run_store<T, E>(R, v1, v2, b1, b2, j, L, Ns);
      __syncthreads();
      smem_load<T, E>(v1, v2, b1, b2, j, L);
    }
    Ns *= R;
  }
}

// ------------------------------------------------------------------ the kernel
template <typename T, int E, int MODE>
__global__ void __launch_bounds__(512) line_pass_kernel(LinePassArgs<T> a, int npass, int rl,
                                                        int line_stride) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Cx<T>* smem = reinterpret_cast<Cx<T>*>(smem_raw);

  const int L = a.L;
  const int tpl = L / E;                 // threads per line
  const int tid = threadIdx.x;
  const int lcta = tid / tpl;            // line within the CTA
  const int j = tid - lcta * tpl;
  const int line = blockIdx.x * a.lpc + lcta;
  const size_t row = (size_t)line * L;

  Cx<T>* b1 = smem + (size_t)lcta * line_stride;
  Cx<T>* b2 = b1 + Pad<T>::len(L);

  Cx<T> v1[E], v2[E];
  // ---- load psi (both components) for elements j + m L/E
#pragma unroll
  for (int m = 0; m < E; ++m) {
    const size_t gi = row + j + m * (L / E);
    Q4<T> p = a.in[gi];
    if (MODE == MODE_STEP && a.u_load) p = apply_u(a.u_load[gi], p);
    v1[m] = {p.x, p.y};
    v2[m] = {p.z, p.w};
  }

  line_fft<T, E, false>(v1, v2, b1, b2, j, L, npass, rl, a.tw);

  // ---- k-space multiply at q = j + m L/E (the multiplier carries 1/L)
#pragma unroll
  for (int m = 0; m < E; ++m) {
    const int q = j + m * (L / E);
    const Q4<T> c = ldg_q4(a.mult + q);
    const Cx<T> x1 = v1[m], x2 = v2[m];
    if (MODE == MODE_DERIV) {
      // i xi x, xi = c.z + c.w
      v1[m] = {-(c.z * x1.im + c.w * x1.im), c.z * x1.re + c.w * x1.re};
      v2[m] = {-(c.z * x2.im + c.w * x2.im), c.z * x2.re + c.w * x2.re};
    } else if (a.sigma == 0) {
      // (c-1) x - i s sigma_x x:  d1 = (c-1) x1 - i s x2,  d2 = (c-1) x2 - i s x1
      v1[m] = {c.x * x1.re + (c.y * x1.re + (c.z * x2.im + c.w * x2.im)),
               c.x * x1.im + (c.y * x1.im - (c.z * x2.re + c.w * x2.re))};
      v2[m] = {c.x * x2.re + (c.y * x2.re + (c.z * x1.im + c.w * x1.im)),
               c.x * x2.im + (c.y * x2.im - (c.z * x1.re + c.w * x1.re))};
    } else {
      // (c-1) x - i s sigma_y x:  d1 = (c-1) x1 - s x2,  d2 = (c-1) x2 + s x1
      v1[m] = {c.x * x1.re + (c.y * x1.re - (c.z * x2.re + c.w * x2.re)),
               c.x * x1.im + (c.y * x1.im - (c.z * x2.im + c.w * x2.im))};
      v2[m] = {c.x * x2.re + (c.y * x2.re + (c.z * x1.re + c.w * x1.re)),
               c.x * x2.im + (c.y * x2.im + (c.z * x1.im + c.w * x1.im))};
    }
  }

  line_fft<T, E, true>(v1, v2, b1, b2, j, L, npass, rl, a.tw);

  // ---- epilogue into the staging buffer [lcta][i] (line stride L + 1 points)
  __syncthreads();  // FFT buffers are free again
  Q4<T>* stage = reinterpret_cast<Q4<T>*>(smem_raw);
  Q4<T>* my_stage = stage + (size_t)lcta * (L + 1);
#pragma unroll
  for (int m = 0; m < E; ++m) {
    const int i = j + m * (L / E);
    Q4<T> o;
    if (MODE == MODE_STEP) {
      const size_t gi = row + i;
      Q4<T> p = a.in[gi];
      if (a.u_load) p = apply_u(a.u_load[gi], p);
      const T bm1 = a.beta ? a.beta[gi] : T(0);
      o.x = (p.x + v1[m].re) + bm1 * v1[m].re;
      o.y = (p.y + v1[m].im) + bm1 * v1[m].im;
      o.z = (p.z + v2[m].re) + bm1 * v2[m].re;
      o.w = (p.w + v2[m].im) + bm1 * v2[m].im;
      if (a.u_store) o = apply_u(a.u_store[gi], o);
    } else {
      o = {v1[m].re, v1[m].im, v2[m].re, v2[m].im};
    }
    my_stage[i] = o;
  }

  // ---- transposed store: the cluster's G = lpc * cs lines go out as contiguous
  // segments out[i][line0 .. line0 + G); CTA rank c writes rows i of its L/cs slice.
  const int G = a.lpc * a.cs;
  const int rank = (a.cs > 1) ? (int)cg::this_cluster().block_rank() : 0;
  if (a.cs > 1) cg::this_cluster().sync(); else __syncthreads();
  const int line0 = (blockIdx.x / a.cs) * G;
  const int rows = L / a.cs;
  const int i0 = rank * rows;
  const int items = rows * G;
  for (int it = tid; it < items; it += blockDim.x) {
    const int g = it % G;
    const int i = i0 + it / G;
    const int owner = g / a.lpc;
    const Q4<T>* src = stage;
    if (a.cs > 1 && owner != rank) src = cg::this_cluster().map_shared_rank(stage, owner);
    const Q4<T> val = src[(size_t)(g - owner * a.lpc) * (L + 1) + i];
    a.out[(size_t)i * a.n_lines + line0 + g] = val;
  }
  if (a.cs > 1) cg::this_cluster().sync();
}

}  // namespace dgb
