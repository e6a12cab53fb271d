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
// and U values. The output leaves in the transposed layout as segments of LPI lines; for
// 4096-point lines the CTAs run as clusters of 4 that gather their staged lines through
// distributed shared memory into 4-line segments.
//
// Every wait on an mbarrier is bounded: if one runs out, the CTA records an error code
// in *err, stops issuing copies and transforming, keeps taking part in the cluster
// barriers until its peers finish (so none of them waits forever), waits (bounded) for
// the copy it issued itself and returns.
#pragma once
#include "line_pass.cuh"

namespace dgb {

template <typename T, int L>
struct PGeo {
  static constexpr int E = 8;
  static constexpr int THREADS = 1024;
  static constexpr int TPL = 2 * L / E;
  static constexpr int LPI = THREADS / TPL;  // lines per group
  // CTAs per cluster: 4 for 4096-point lines (64-B output segments measured faster than
  // 16-B ones); shorter lines write LPI-line segments without a cluster (the cluster
  // barriers cost more than they saved at 2048 points).
  static constexpr int CS = L == 4096 ? 4 : 1;
  static constexpr int GL = LPI * CS;               // lines per output segment
  using G = Geo<T, L, LPI, E>;               // FFT buffer plan (padded, conflict-free)
  static constexpr size_t F_BYTES = ((G::SMEM + 127) / 128) * 128;
  static constexpr size_t PSI_BYTES = (size_t)LPI * L * sizeof(Q4<T>);
  static constexpr size_t SMEM = F_BYTES + 2 * PSI_BYTES + 2 * sizeof(uint64_t);
  static_assert(sizeof(T) == 4, "persistent pass is complex64 only");
  static_assert(G::THREADS == THREADS, "group must fill the CTA");
  static_assert(SMEM <= 227 * 1024, "shared memory budget");
};

constexpr uint64_t kWaitNs = 1500000000ull;  // 1.5 s: a copy of 64 KB takes microseconds
constexpr int kErrTimeout = 1;

// BATCH: the launch covers several instances (a0.inst); otherwise every pointer stays a
// kernel parameter, which the compiler reads from the constant bank instead of keeping
// in registers.
template <typename T, int L, bool BATCH>
__global__ void __launch_bounds__(1024, 1)
    line_pass_persistent(const LinePassArgs<T> a0, int n_groups, int* __restrict__ err) {
  using PG = PGeo<T, L>;
  using Gm = typename PG::G;
  constexpr int E = PG::E, J = L / E, LPI = PG::LPI, CS = PG::CS, GL = PG::GL;
  extern __shared__ __align__(128) unsigned char psmem[];
  Cx<T>* fbuf = reinterpret_cast<Cx<T>*>(psmem);
  Q4<T>* psi_buf[2] = {reinterpret_cast<Q4<T>*>(psmem + PG::F_BYTES),
                       reinterpret_cast<Q4<T>*>(psmem + PG::F_BYTES + PG::PSI_BYTES)};
  uint64_t* bars = reinterpret_cast<uint64_t*>(psmem + PG::F_BYTES + 2 * PG::PSI_BYTES);

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
  // cluster geometry: super-group s = lines [s GL, s GL + GL); CTA rank q owns group s CS + q
  int rank = 0;
  if constexpr (CS > 1) rank = (int)cg::this_cluster().block_rank();
  const int cluster_id = blockIdx.x / CS, n_clusters = gridDim.x / CS;

  // batched launch: groups of instance k are [k gpi, (k + 1) gpi)
  const int gpi = a0.n_lines / LPI;
  if constexpr (BATCH) n_groups = *a0.n_inst * gpi;
  const int n_super = n_groups / CS;
  auto args_of = [&](int grp, size_t* first) {
    if constexpr (BATCH) {
      LinePassArgs<T> x = a0;
      const int k = grp / gpi;
      bind_instance(x, k);
      *first = (size_t)(grp - k * gpi) * LPI * L;
      return x;
    } else {
      *first = (size_t)grp * LPI * L;
      return a0;
    }
  };
  auto issue = [&](int grp, int slot) {
    size_t first;
    const LinePassArgs<T> x = args_of(grp, &first);
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(&bars[slot], GROUP_BYTES + a0.test_extra_tx);
    bulk_copy_g2s(psi_buf[slot], x.in + first, GROUP_BYTES, &bars[slot]);
    if (x.beta) bulk_prefetch_l2(x.beta + first, BETA_BYTES);
    if (x.u_store) bulk_prefetch_l2(x.u_store + first, U_BYTES);
    if (x.u_load) bulk_prefetch_l2(x.u_load + first, U_BYTES);
  };

  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (tid == 0 && cluster_id < n_super) issue(cluster_id * CS + rank, 0);

  bool failed = false;      // uniform across the CTA
  int pending = -1;         // slot of a copy issued and not yet waited for (after a failure)
  uint32_t pending_par = 0; // the phase parity that copy completes
  int it = 0;
  for (int s = cluster_id; s < n_super; s += n_clusters, ++it) {
    const int b = it & 1;
    const int g = s * CS + rank;
    const bool has_next = s + n_clusters < n_super;
    if (!failed) {
      if (tid == 0 && has_next) issue((s + n_clusters) * CS + rank, b ^ 1);
      const bool ok = mbar_wait_bounded(&bars[b], (it >> 1) & 1, kWaitNs);
      if (__syncthreads_or(!ok)) {
        failed = true;
        if (tid == 0) atomicExch(err, kErrTimeout);
        pending = has_next ? (b ^ 1) : -1;
        pending_par = ((it + 1) >> 1) & 1;
      }
    }
    size_t gfirst;
    const LinePassArgs<T> a = args_of(g, &gfirst);
    if (!failed) {
      const size_t row = gfirst + (size_t)lcta * L;
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
      // The inverse FFT's index and twiddle-address arithmetic equals the forward one's;
      // an opaque copy of j and buf makes the compiler recompute it instead of keeping
      // every pass's values live across the k-space multiply (which spilled).
      int j2 = j;
      Cx<T>* buf2 = buf;
      asm volatile("" : "+r"(j2), "+l"(buf2));
      fft_passes<T, L, E, true>(v, buf2, j2, a.tw);

      __syncthreads();  // the FFT buffer becomes the staging buffer
      Q4<T>* stage = reinterpret_cast<Q4<T>*>(psmem);
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
    }
    // ---- transposed store of the super-group: out[i][s GL .. s GL + GL); CTA rank q
    // writes rows i of its L/CS slice, reading the owners' staging buffers
    if constexpr (CS > 1) cg::this_cluster().sync(); else __syncthreads();
    if (!failed) {
      const Q4<T>* stage = reinterpret_cast<const Q4<T>*>(psmem);
      const int line0 = (int)(gfirst / L) - rank * LPI;
      const int i0 = rank * (L / CS);
      constexpr int NIT = (L / CS) * GL / PG::THREADS;
      Q4<T> val[NIT];
      if constexpr (CS > 1) {
        // gather through distributed shared memory: 32-bit shared::cluster addresses
        const uint32_t local = smem_u32(stage);
#pragma unroll
        for (int q = 0; q < NIT; ++q) {
          const int itm = tid + q * PG::THREADS;
          const int gg = itm % GL, owner = gg / LPI;
          const uint32_t off = (uint32_t)(((gg - owner * LPI) * (L + 1) + i0 + itm / GL) * sizeof(Q4<T>));
          val[q] = ld_dsmem_q4<T>(mapa_shared(local, owner) + off);
        }
      } else {
#pragma unroll
        for (int q = 0; q < NIT; ++q) {
          const int itm = tid + q * PG::THREADS;
          val[q] = stage[(size_t)(itm % GL) * (L + 1) + i0 + itm / GL];
        }
      }
#pragma unroll
      for (int q = 0; q < NIT; ++q) {
        const int itm = tid + q * PG::THREADS;
        a.out[(size_t)(i0 + itm / GL) * a.n_lines + line0 + itm % GL] = val[q];
      }
    }
    // staging and psi_buf[b] are free for the next super-group once every CTA of the
    // cluster has finished reading
    if constexpr (CS > 1) cg::this_cluster().sync(); else __syncthreads();
  }
  if (failed && tid == 0 && pending >= 0) mbar_wait_bounded(&bars[pending], pending_par, kWaitNs);
}

}  // namespace dgb
