// Persistent, prefetching variant of the fused line pass (complex64 step mode).
//
// One 1024-thread CTA per SM loops over groups of lines, 4096 points per group (LPI =
// 4096 / L lines). While it transforms group g, thread 0 has already started a bulk
// asynchronous copy of group g + gridDim.x's spinor rows into the other half of a
// double buffer in shared memory (completion counted on an mbarrier) and an L2 bulk
// prefetch of that group's b - 1 and U rows. The FFT, k-space multiply, inverse FFT and
// epilogue are those of line_pass_kernel (eigencomponent per thread, radix-8 passes);
// the spinor values for the load and for the epilogue come from shared memory, so the
// only global-memory latency left in a group's critical path is the L2 hit of its b - 1
// and U values. The output leaves in the transposed layout as LPI-line segments.
//
// Every wait on an mbarrier is bounded: if one runs out, the CTA records an error code
// in *err, waits (bounded) for the copy it issued itself and returns.
#pragma once
#include "line_pass.cuh"

namespace dgb {

template <typename T, int L>
struct PGeo {
  static constexpr int E = 8;
  static constexpr int THREADS = 1024;
  static constexpr int TPL = 2 * L / E;
  static constexpr int LPI = THREADS / TPL;  // lines per group
  using G = Geo<T, L, LPI, E>;               // FFT buffer plan (padded, conflict-free)
  static constexpr size_t F_BYTES = ((G::SMEM + 127) / 128) * 128;
  static constexpr size_t PSI_BYTES = (size_t)LPI * L * sizeof(Q4<T>);
  static constexpr size_t SMEM = F_BYTES + 2 * PSI_BYTES + 2 * sizeof(uint64_t);
  static_assert(sizeof(T) == 4, "persistent pass is complex64 only");
  static_assert(G::THREADS == THREADS, "group must fill the CTA");
  static_assert(SMEM <= 227 * 1024, "shared memory budget");
};

constexpr int kWaitTries = 1 << 22;
constexpr int kErrTimeout = 1;

template <typename T, int L>
__global__ void __launch_bounds__(1024, 1)
    line_pass_persistent(LinePassArgs<T> a, int n_groups, int* __restrict__ err) {
  using PG = PGeo<T, L>;
  using Gm = typename PG::G;
  constexpr int E = PG::E, J = L / E, LPI = PG::LPI;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  Cx<T>* fbuf = reinterpret_cast<Cx<T>*>(smem_raw);
  Q4<T>* psi_buf[2] = {reinterpret_cast<Q4<T>*>(smem_raw + PG::F_BYTES),
                       reinterpret_cast<Q4<T>*>(smem_raw + PG::F_BYTES + PG::PSI_BYTES)};
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw + PG::F_BYTES + 2 * PG::PSI_BYTES);

  const int tid = threadIdx.x;
  const int lcta = tid / PG::TPL;
  const int r = tid - lcta * PG::TPL;
  const int c = r & 1;
  const int j = r >> 1;
  Cx<T>* buf = fbuf + lcta * Gm::STRIDE + c * Gm::COMP;
  const T sg = c ? T(-1) : T(1);
  constexpr uint32_t GROUP_BYTES = (uint32_t)(LPI * L * sizeof(Q4<T>));
  constexpr uint32_t BETA_BYTES = (uint32_t)(LPI * L * sizeof(T));
  constexpr uint32_t U_BYTES = GROUP_BYTES;

  auto issue = [&](int g, int slot) {
    const size_t first = (size_t)g * LPI * L;
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(&bars[slot], GROUP_BYTES);
    bulk_copy_g2s(psi_buf[slot], a.in + first, GROUP_BYTES, &bars[slot]);
    if (a.beta) bulk_prefetch_l2(a.beta + first, BETA_BYTES);
    if (a.u_store) bulk_prefetch_l2(a.u_store + first, U_BYTES);
    if (a.u_load) bulk_prefetch_l2(a.u_load + first, U_BYTES);
  };

  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (tid == 0 && (int)blockIdx.x < n_groups) issue(blockIdx.x, 0);

  int it = 0;
  for (int g = blockIdx.x; g < n_groups; g += gridDim.x, ++it) {
    const int b = it & 1;
    const bool has_next = g + (int)gridDim.x < n_groups;
    if (tid == 0 && has_next) issue(g + gridDim.x, b ^ 1);

    const bool ok = mbar_wait_bounded(&bars[b], (it >> 1) & 1, kWaitTries);
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        atomicExch(err, kErrTimeout);
        if (has_next) mbar_wait_bounded(&bars[b ^ 1], ((it + 1) >> 1) & 1, kWaitTries);
      }
      return;
    }

    const size_t row = ((size_t)g * LPI + lcta) * L;
    const Cx<T>* src_c = reinterpret_cast<const Cx<T>*>(psi_buf[b] + (size_t)lcta * L) + c;
    Cx<T> v[E];
#pragma unroll
    for (int m = 0; m < E; ++m) {
      const int i = j + m * J;
      Cx<T> own = src_c[2 * i];
      Cx<T> oth = shfl_pair(own);
      if (a.u_load) {
        own = apply_u_row(ldg_q4(a.u_load + row + i), own, oth, c);
        oth = shfl_pair(own);
      }
      const Cx<T> p1 = c ? oth : own, p2 = c ? own : oth;
      if (a.sigma == 0) v[m] = {p1.re + sg * p2.re, p1.im + sg * p2.im};
      else v[m] = {p1.re + sg * p2.im, p1.im - sg * p2.re};
    }

    fft_passes<T, L, E, false>(v, buf, j, a.tw);
#pragma unroll
    for (int m = 0; m < E; ++m) {
      if ((m & 3) == 0) asm volatile("" ::: "memory");
      const Q4<T> q = ldg_q4(a.mult + j + m * J);
      const T vr = v[m].re, vi = v[m].im;
      const T sh = -sg * q.z, sl = -sg * q.w;
      v[m] = {q.x * vr + ((q.y * vr - sl * vi) - sh * vi),
              q.x * vi + ((q.y * vi + sl * vr) + sh * vr)};
    }
    fft_passes<T, L, E, true>(v, buf, j, a.tw);

    __syncthreads();  // the FFT buffer becomes the staging buffer
    Q4<T>* stage = reinterpret_cast<Q4<T>*>(smem_raw);
    Cx<T>* my_stage = reinterpret_cast<Cx<T>*>(stage + (size_t)lcta * (L + 1)) + c;
#pragma unroll
    for (int m = 0; m < E; ++m) {
      if ((m & 3) == 0) asm volatile("" ::: "memory");
      const int i = j + m * J;
      const size_t gi = row + i;
      const Cx<T> oth = shfl_pair(v[m]);
      const Cx<T> dp = c ? oth : v[m], dm = c ? v[m] : oth;
      Cx<T> d;
      if (c == 0) d = cadd(dp, dm);
      else d = a.sigma == 0 ? csub(dp, dm) : mul_i(csub(dp, dm));
      Cx<T> p = src_c[2 * i];
      if (a.u_load) p = apply_u_row(ldg_q4(a.u_load + gi), p, shfl_pair(p), c);
      const T bm1 = a.beta ? a.beta[gi] : T(0);
      Cx<T> o = {(p.re + d.re) + bm1 * d.re, (p.im + d.im) + bm1 * d.im};
      if (a.u_store) o = apply_u_row(ldg_q4(a.u_store + gi), o, shfl_pair(o), c);
      my_stage[2 * i] = o;
    }
    __syncthreads();
    // transposed store: out[i][g LPI .. g LPI + LPI)
    const int line0 = g * LPI;
    constexpr int NIT = LPI * L / PG::THREADS;
    Q4<T> val[NIT];
#pragma unroll
    for (int q = 0; q < NIT; ++q) {
      const int itm = tid + q * PG::THREADS;
      val[q] = stage[(size_t)(itm % LPI) * (L + 1) + itm / LPI];
    }
#pragma unroll
    for (int q = 0; q < NIT; ++q) {
      const int itm = tid + q * PG::THREADS;
      a.out[(size_t)(itm / LPI) * a.n_lines + line0 + itm % LPI] = val[q];
    }
    __syncthreads();  // staging and psi_buf[b] are free for the next group
  }
}

}  // namespace dgb
