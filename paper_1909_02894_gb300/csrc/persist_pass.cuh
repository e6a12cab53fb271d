// Persistent, prefetching variant of the fused line pass (complex64 step mode).
//
// One 1024-thread CTA per SM loops over groups of lines, 4096 points per group (LPI =
// 4096 / L lines). Shared memory holds three regions: the FFT buffer (also the staging
// buffer of the transposed store), a spinor landing zone and a b - 1 / U landing zone.
// Thread 0 fills both landing zones with bulk asynchronous copies whose completion is
// counted on one mbarrier each:
//   * spinor rows of group g + 1 are requested as soon as every thread has read group g's
//     rows (right after the load), so they arrive while group g is transformed. Each
//     thread parks its own component of its points (needed again by the epilogue) in
//     tensor memory, which frees the zone that early;
//   * b - 1 and U rows of group g + 1 are requested once group g's epilogue has used the
//     zone, and arrive during group g + 1's transforms.
// So a group's critical path holds no global-memory load but the k-space multipliers and
// twiddles (cached tables). The FFT, k-space multiply, inverse FFT and epilogue are those
// of line_pass_kernel (eigencomponent per thread, radix-8 passes). The output leaves in
// the transposed layout as segments of LPI lines. 4096-point lines run as clusters of 2
// CTAs (adjacent lines): in single-instance launches each CTA stages its finished line in
// shared memory and thread 0 writes it with asynchronous tensor stores (one point per
// row, 256 rows per box), which drain while the next group loads and transforms; the two
// CTAs write the two 16-byte halves of each 32-byte sector at about the same time.
// Batched launches gather the two staged lines through distributed shared memory into
// 32-byte segments and store them from registers. 4096- and 1024-point lines run FFTs
// whose exchanges go through tensor memory (fft4096_swap, fft1024_swap); the other
// lengths run the Stockham passes.
//
// Every wait on an mbarrier is bounded: if one runs out, the CTA records an error code
// in *err, stops issuing copies and transforming, keeps taking part in the cluster
// barriers until its peers finish (so none of them waits forever), waits (bounded) for
// the copies it issued itself, frees its tensor memory and returns.
#pragma once
#include <cuda.h>  // CUtensorMap

#include "line_pass.cuh"

namespace dgb {

template <typename T, int L>
struct PGeo {
  static constexpr int E = 8;
  static constexpr int THREADS = 1024;
  static constexpr int TPL = 2 * L / E;
  static constexpr int LPI = THREADS / TPL;  // lines per group
  // CTAs per cluster: 2 for 4096-point lines (adjacent lines run together). Batched
  // launches gather their output into 32-byte (one DRAM sector) segments of the 2 lines;
  // single-instance launches write each CTA's line with tensor stores, and the two halves
  // of each sector arrive at about the same time. Clusters of 2 keep every SM busy (76 x 2
  // CTAs resident on 152 SMs; clusters of 4 fit only 36 x 4) and measured faster than both
  // clusters of 4 (64-B segments) and no cluster (16-B register stores). Shorter lines
  // write LPI-line segments without a cluster (the cluster barriers cost more than they
  // saved at 2048 points).
  static constexpr int CS = L == 4096 ? 2 : 1;
  static constexpr int GL = LPI * CS;               // lines per output segment
  using G = Geo<T, L, LPI, E>;               // FFT buffer plan (padded, conflict-free)
  // 4096-point lines run the digit-swap FFT (fft4096_swap): unpadded component buffers,
  // which also hold the staging buffer of L + 1 points
  static constexpr bool SWAP = L == 4096;
  // 1024-point lines run fft1024_swap: line l of the group on the 8 warps of tensor-memory
  // lane quarter l; warp-local exchange buffers of XQ elements per (component, lane bit 1)
  // group with rows of XP (conflict free for the 8-byte accesses of both directions)
  static constexpr bool SWAP1K = L == 1024;
  static constexpr int XP = 9, XQ = 76;
  static constexpr size_t XBUF_BYTES = (size_t)(THREADS / 32) * 4 * XQ * sizeof(Cx<T>);
  // The 4096-point path pads its staging buffer and its b - 1 / U zones after every 512
  // points (1 point, 4 floats, 1 matrix), so that the two threads of a point pair, which
  // work on points 512 k apart in the epilogue, reach different banks.
  static constexpr int PAD_EVERY = 512;
  static constexpr size_t STAGE_POINTS = SWAP ? L + L / PAD_EVERY : L + 1;
  // Row pitch (points) of the staging buffer between lines: the transposed store gathers
  // the same point of the LPI lines in consecutive lanes, so rows LPI apart in 16-byte
  // slots of a 128-byte bank row must differ: pitch = 8 / LPI modulo 8 (any odd pitch for
  // 16 lines).
  static constexpr int SPITCH = SWAP ? L + 1 : L + (LPI <= 8 ? 8 / LPI : 1);
  static constexpr size_t F_RAW =
      SWAP ? ((size_t)2 * L * sizeof(Cx<T>) > STAGE_POINTS * sizeof(Q4<T>)
                  ? (size_t)2 * L * sizeof(Cx<T>) : STAGE_POINTS * sizeof(Q4<T>))
      : SWAP1K ? (XBUF_BYTES > (size_t)LPI * SPITCH * sizeof(Q4<T>)
                      ? XBUF_BYTES : (size_t)LPI * SPITCH * sizeof(Q4<T>))
           : G::SMEM;
  static constexpr size_t F_BYTES = ((F_RAW + 127) / 128) * 128;
  static constexpr size_t PSI_BYTES = (size_t)LPI * L * sizeof(Q4<T>);
  static constexpr size_t BETA_BYTES = (size_t)LPI * L * sizeof(T);
  static constexpr size_t U_BYTES = PSI_BYTES;
  static constexpr int CHUNKS = SWAP ? L / PAD_EVERY : 1;  // bulk copies per b - 1 / U row
  static constexpr size_t BETA_CHUNK = BETA_BYTES / CHUNKS, U_CHUNK = U_BYTES / CHUNKS;
  static constexpr size_t BETA_PITCH = BETA_CHUNK + (SWAP ? 4 * sizeof(T) : 0);
  static constexpr size_t U_PITCH = U_CHUNK + (SWAP ? sizeof(Q4<T>) : 0);
  static constexpr size_t OFF_PSI = F_BYTES;
  static constexpr size_t OFF_BETA = OFF_PSI + PSI_BYTES;
  static constexpr size_t OFF_U = OFF_BETA + CHUNKS * BETA_PITCH;
  static constexpr size_t OFF_BAR = OFF_U + CHUNKS * U_PITCH;
  static constexpr size_t OFF_T3 = OFF_BAR + 32;  // two mbarriers + tensor-memory address
  // pass-3 twiddles of the digit-swap FFT: 8 warp slices x 8 entries (the 7 powers, a pad)
  static constexpr size_t OFF_T2 = OFF_T3 + 64 * sizeof(Cx<T>);
  // W_128^(u t) (t = 1..7 rows of 16) of the 1024-point FFT
  static constexpr size_t OFF_ITEM = OFF_T2 + (SWAP1K ? 128 : 0) * sizeof(Cx<T>);
  // batched tick: a ring of three work items (5 ints each) and the item offsets of the
  // tick's steps (at most TICK_K_MAX + 1)
  static constexpr int TICK_K_MAX = 1024;
  static constexpr size_t OFF_TPRE = OFF_ITEM + 16 * sizeof(int);
  static constexpr size_t SMEM = OFF_TPRE + (TICK_K_MAX + 1) * sizeof(int);
  // tensor memory: 8 warps share each lane quarter; per warp slice s = warp / 4 the
  // parked spinor values take columns [16 s, 16 s + 16); the digit-swap FFT adds an
  // exchange region of 128 columns and 32 twiddle columns per slice
  static constexpr uint32_t T_PARK = 0, T_X = 128, T_TW = 256, T_X2 = 384;
  static constexpr uint32_t TMEM_COLS = (SWAP || SWAP1K) ? 512 : 128;
  static_assert(sizeof(T) == 4, "persistent pass is complex64 only");
  static_assert(G::THREADS == THREADS, "group must fill the CTA");
  static_assert(SMEM <= 227 * 1024, "shared memory budget");
  static_assert(SWAP || F_BYTES >= (size_t)LPI * SPITCH * sizeof(Q4<T>), "staging buffer");
  static_assert(SMEM > 227 * 1024 / 2, "one CTA per SM (the tensor-memory allocation relies on it)");
  static_assert(THREADS / 32 / 4 * 2 * E == 128, "tensor-memory layout");
  static_assert(BETA_PITCH % 16 == 0 && U_PITCH % 16 == 0 && OFF_BAR % 16 == 0, "bulk copy");
  // positions in the padded staging buffer / b - 1 zone / U zone of point i of a line
  static __device__ __forceinline__ int spos(int i) { return SWAP ? i + i / PAD_EVERY : i; }
  // The same for point j + m L/E with 0 <= j < L/E: in the padded 4096-point layout
  // L/E = PAD_EVERY, so that point's padding is m slots (no division at run time).
  static __device__ __forceinline__ int spos_jm(int j, int m) {
    return SWAP ? j + m * (L / E + 1) : j + m * (L / E);
  }
  static __device__ __forceinline__ int bpos_jm(int j, int m) {
    return SWAP ? j + m * (L / E + 4) : j + m * (L / E);
  }
  static __device__ __forceinline__ int upos_jm(int j, int m) { return spos_jm(j, m); }
  static_assert(!SWAP || L / E == PAD_EVERY, "padding every L/E points");
  // entries of the landing zones and of the staging buffer (debug index checks)
  static constexpr size_t PSI_N = (size_t)LPI * L;
  static constexpr size_t BETA_N = CHUNKS * BETA_PITCH / sizeof(T);
  static constexpr size_t U_N = CHUNKS * U_PITCH / sizeof(Q4<T>);
  static constexpr size_t STAGE_N = SWAP ? STAGE_POINTS : (size_t)LPI * SPITCH;
};

constexpr uint64_t kWaitNs = 1500000000ull;  // 1.5 s: a copy of 64 KB takes microseconds
constexpr int kErrTimeout = 1;
constexpr int kErrAlign = 2;  // the staging tile of the tensor stores is not 128-B aligned

// ---- digit-swap FFT of 4096 points (forward, or inverse without the 1/N scale)
//
// Index n = d0 + 8 d1 + 64 d2 + 512 d3 (octal digits). Thread j (512 per component line)
// holds 8 elements in registers; its index j = 16 w + lane / 2 puts j's top three bits in
// the warp slice w / 4, the set of warps that share a tensor-memory lane quarter. The
// transform is a radix-8 decimation in frequency (four passes over d3, d2, d1, d0, each
// followed by the twiddles W_4096^(n' k0), W_512^(n'' k1), W_64^(d0 k2)); between passes
// the digit in registers trades places with a digit spread over the threads:
//   pass 1 (registers d3)  --tensor memory: registers <-> slice digit--
//   pass 2 (d2)            --shared memory: a general permutation--
//   pass 3 (d1)            --tensor memory--
//   pass 4 (d0)
// Input and output are both in natural order, element r of thread j at index j + 512 r,
// so only one of the three exchanges goes through shared memory.
// Shared-memory slot of element idx of component c: XOR of index bits 6, 9, 10, 11 into
// bits 0..3, and of 9 for the second component. 8-byte accesses are served per half-warp
// (8 points x 2 components); the write pattern (lanes vary bits 0..2 and c) and the read
// pattern (bits 9..11 and c) then reach 16 different bank pairs.
__device__ __forceinline__ int swz4096(int idx, int cx) {
  return idx ^ (((idx >> 6) & 1) | (((idx >> 9) & 7) << 1)) ^ cx;
}

// v[t] *= w^t for t = 1..7 (conjugate for the inverse), w^t = (f[2t - 2], f[2t - 1])
template <typename T, bool INV>
__device__ __forceinline__ void twiddle8(Cx<T> (&v)[8], const float (&f)[16]) {
#pragma unroll
  for (int t = 1; t < 8; ++t) {
    const Cx<T> w = {f[2 * t - 2], f[2 * t - 1]};
    v[t] = INV ? cmulc(v[t], w) : cmul(v[t], w);
  }
}

// registers <-> slice digit through tensor memory: thread (j mod 64, slice s) stores its
// 8 elements at columns x + 16 s + 2 r and reads element s of every slice's block;
// afterwards element r' comes from slice r'. `x` carries this warp's lane quarter.
template <typename T>
__device__ __forceinline__ void tmem_swap(Cx<T> (&v)[8], uint32_t x, int s, int q) {
  {
    float f[16];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      f[2 * r] = v[r].re;
      f[2 * r + 1] = v[r].im;
    }
    tmem_st16(x + 16u * (uint32_t)s, f);
  }
  tmem_wait_st();
  tmem_fence_before_sync();
  named_barrier(1 + q, 256);  // the 8 warps of this lane quarter
  tmem_fence_after_sync();
  float g[16];
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    float h[2];
    tmem_ld2(x + 16u * (uint32_t)r + 2u * (uint32_t)s, h);
    g[2 * r] = h[0];
    g[2 * r + 1] = h[1];
  }
  tmem_wait_ld_regs(g);
#pragma unroll
  for (int r = 0; r < 8; ++r) v[r] = {g[2 * r], g[2 * r + 1]};
}

// tws: this thread's pass-1 and pass-2 twiddles parked in tensor memory (w^1..w^7 of
// each, 16 columns apart); x: the exchange region; fc: this component's 4096-point shared
// buffer and cx its slot XOR (0 or 9, see swz4096); t3: the warp slice's pass-3 twiddles
// W_64^(d0 t), t = 1..7, in shared memory (one broadcast read each). pre: what precedes
// the first write of the shared buffer (0 nothing, 1 the wait of a split cluster barrier,
// 2 thread 0 waits until its bulk stores have read the buffer, then a CTA barrier).
template <typename T, bool INV>
__device__ __forceinline__ void fft4096_swap(Cx<T> (&v)[8], Cx<T>* fc, int cx, int j, int s,
                                             int q, uint32_t tws, uint32_t x,
                                             const Cx<T>* t3, int pre = 0) {
  {
    float t1[16];
    tmem_ld16(tws, t1);
    dft8<T, INV>(v);
    tmem_wait_ld_regs(t1);
    twiddle8<T, INV>(v, t1);
  }
  tmem_swap(v, x, s, q);
  {
    float t2[16];
    tmem_ld16(tws + 16u, t2);
    dft8<T, INV>(v);
    tmem_wait_ld_regs(t2);
    twiddle8<T, INV>(v, t2);
  }
  // registers k1, threads (d0, d1, k0)  ->  registers d1, threads (k0, k1, d0). The
  // swizzle of the written slots depends on r only through bit 0 (index bit 6) and that
  // of the read slots not at all, so both reduce to two bases and constant offsets:
  //   write r: swz(hi 512 + mid 8 + lo + 64 r) = wb[r & 1] + 64 r
  //   read r:  swz(lo 512 + mid 64 + hi + 8 r)  = rb[r & 1] + 8 r
  const int lo = j & 7, mid = (j >> 3) & 7, hi = j >> 6;
  const int wb0 = ((hi * 512 + mid * 8 + lo) ^ (hi << 1)) ^ cx, wb1 = wb0 ^ 1;
  const int m = ((mid & 1) | (lo << 1)) ^ cx;  // XOR applied to every read slot
  const int rbase = (lo * 512 + mid * 64 + hi) ^ (m & 7);
  const int m3 = (m >> 3) & 1;  // flips bit 3, the low bit of r's field
  const int rb0 = rbase + 8 * m3, rb1 = rbase - 8 * m3;
  // Earlier readers of the buffer have finished: the previous group's gather (the wait of
  // the split cluster barrier, pre = 1, or a barrier the caller passed), its bulk stores
  // (pre = 2) or the forward FFT (the barrier between the transforms).
  if (pre == 1) cluster_wait();
  if (pre == 2) {
    if (threadIdx.x == 0) bulk_wait_read_all();
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const int o = (r & 1 ? wb1 : wb0) + 64 * r;
    if (dbg_in(o, 4096)) fc[o] = v[r];
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const int o = (r & 1 ? rb1 : rb0) + 8 * r;
    v[r] = dbg_in(o, 4096) ? fc[o] : Cx<T>{T(0), T(0)};
  }
  dft8<T, INV>(v);
  {
    float f[16];
#pragma unroll
    for (int t = 1; t < 8; ++t) {
      const Cx<T> w = t3[t - 1];
      f[2 * t - 2] = w.re;
      f[2 * t - 1] = w.im;
    }
    f[14] = f[15] = 0.f;
    twiddle8<T, INV>(v, f);
  }
  tmem_swap(v, x, s, q);
  dft8<T, INV>(v);
}

// ---- 1024-point FFT, one line per tensor-memory lane quarter
//
// Line l of the group runs on the 8 warps of lane quarter l (warp & 3 == l). Thread
// (slice s = warp / 4, lane) holds component lane & 1 and of it the elements j + 128 r,
// r = 0..7, with j = 16 s + u, u = lane / 2 = u0 + 2 u1 (u0 = lane bit 1, u1 = lane bits
// 2..4). Forward, a decimation in frequency over n = j + 128 b:
//   DFT-8 over b (registers) -> k0, twiddle W_1024^(j k0);
//   tensor memory: registers <-> slice (registers s, slice k0);
//   DFT-8 over s -> k1, twiddle W_128^(u k1);
//   warp-local exchange through shared memory: registers <-> u1 (lanes k1, registers u1);
//   DFT-8 over u1 -> v1, twiddle W_16^(u0 v1);
//   DFT-2 over u0 (lane bit 1, shuffles) -> v0.
// Element r of thread (s, lane) is then frequency s + 8 (lane >> 2) + 64 r + 512 v0,
// v0 = (lane >> 1) & 1. The inverse runs the same steps backwards with conjugate twiddles
// and ends in natural order. Only the tensor-memory exchange synchronises warps (the 8 of
// the line's quarter); x is the exchange region (one for each direction), xw this warp's
// exchange buffer, t1 the thread's parked W_1024^(j t), t2 the W_128^(u t) table.
template <typename T, bool INV>
__device__ __forceinline__ void tw16_lane(Cx<T> (&v)[8], bool u0) {
  Cx<T> w[8];
  w[1] = w16<T, INV, 1>(v[1]);
  w[2] = w16<T, INV, 2>(v[2]);
  w[3] = w16<T, INV, 3>(v[3]);
  w[4] = w16<T, INV, 4>(v[4]);
  w[5] = w16<T, INV, 4>(w16<T, INV, 1>(v[5]));
  w[6] = w16<T, INV, 6>(v[6]);
  w[7] = w16<T, INV, 4>(w16<T, INV, 3>(v[7]));
#pragma unroll
  for (int r = 1; r < 8; ++r) v[r] = u0 ? w[r] : v[r];
}

template <typename T>
__device__ __forceinline__ void dft2_lane(Cx<T> (&v)[8], bool hi) {
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const Cx<T> p = {__shfl_xor_sync(0xffffffffu, v[r].re, 2),
                     __shfl_xor_sync(0xffffffffu, v[r].im, 2)};
    v[r] = cfma_p(hi ? T(-1) : T(1), v[r], p);  // p - v or v + p, exactly
  }
}

// registers <-> lane bits 2..4 among the 8 lanes of equal lane bits 0..1
template <typename T, int XP, int XQ>
__device__ __forceinline__ void warp_xchg(Cx<T> (&v)[8], Cx<T>* xw, int lane) {
  Cx<T>* g = xw + ((lane & 1) + 2 * ((lane >> 1) & 1)) * XQ;
  const int l3 = lane >> 2;
#pragma unroll
  for (int r = 0; r < 8; ++r)
    if (dbg_in(l3 * XP + r, XQ)) g[l3 * XP + r] = v[r];
  __syncwarp();
#pragma unroll
  for (int r = 0; r < 8; ++r)
    v[r] = dbg_in(r * XP + l3, XQ) ? g[r * XP + l3] : Cx<T>{T(0), T(0)};
}

template <typename T, bool INV, int XP, int XQ>
__device__ __forceinline__ void fft1024_swap(Cx<T> (&v)[8], Cx<T>* xw, int lane, int s, int q,
                                             uint32_t t1, uint32_t x, const Cx<T>* t2) {
  const bool u0 = (lane >> 1) & 1;
  const int u = lane >> 1;
  auto tw128 = [&]() {
    float f[16];
#pragma unroll
    for (int t = 1; t < 8; ++t) {
      const Cx<T> w = t2[(t - 1) * 16 + u];
      f[2 * t - 2] = w.re;
      f[2 * t - 1] = w.im;
    }
    f[14] = f[15] = 0.f;
    twiddle8<T, INV>(v, f);
  };
  if constexpr (!INV) {
    {
      float f[16];
      tmem_ld16(t1, f);
      dft8<T, false>(v);
      tmem_wait_ld_regs(f);
      twiddle8<T, false>(v, f);
    }
    tmem_swap(v, x, s, q);
    dft8<T, false>(v);
    tw128();
    warp_xchg<T, XP, XQ>(v, xw, lane);
    dft8<T, false>(v);
    tw16_lane<T, false>(v, u0);
    dft2_lane(v, u0);
  } else {
    dft2_lane(v, u0);
    tw16_lane<T, true>(v, u0);
    dft8<T, true>(v);
    __syncwarp();  // every lane has read the forward exchange
    warp_xchg<T, XP, XQ>(v, xw, lane);
    tw128();
    dft8<T, true>(v);
    tmem_swap(v, x, s, q);
    {
      float f[16];
      tmem_ld16(t1, f);
      tmem_wait_ld_regs(f);
      twiddle8<T, true>(v, f);
    }
    dft8<T, true>(v);
  }
}

// BATCH: the launch covers several instances (a0.inst); otherwise every pointer stays a
// kernel parameter, which the compiler reads from the constant bank instead of keeping
// in registers. Each instance has at most one of u_load / u_store (the U landing zone
// holds one matrix field).
// TICK (batched, square grids, no clusters): one launch runs every step of a batch tick.
// Work items -- (step k, pass p, instance slot i, line group) in that order -- are taken
// from a queue (*a0.tick_queue), two ahead of the one being worked on. Item (k, p, i) reads
// what the previous pass of slot i wrote and overwrites what it read, so its rows are
// requested only once all 2k + p earlier passes of slot i are finished:
// a0.tick_done[i] >= (2k + p) line groups per pass. Thread 0 checks that when the item is
// next (a counter value loaded early in the current iteration); if it is not yet true, the
// item is marked and, at the start of its iteration, the CTA publishes its previous group
// and thread 0 waits (a bounded spin, DIRAC_ETIMEOUT when it runs out). A finished group
// is published one iteration late, after the next group's inverse FFT: every thread
// fences its stores (long complete by then) before that CTA barrier, and thread 0 then
// adds 1 to tick_done[i] with release semantics. An item only waits on earlier items, held
// by running CTAs that publish before they wait, so every wait ends. A CTA that has failed
// keeps taking items and counting them done (without work), so that no other CTA waits on
// it.
// TST (single-instance 4096-point launches): each thread writes its finished points into
// the CTA's staged line (point i at slot i, no padding); after a CTA barrier thread 0
// writes it with 16 tensor stores (tmap_out: the output as a 2D float tensor of
// 4 n_lines x L, boxes of 4 x 256, one 16-byte point per row), or, for rows back in the
// input's layout, with one bulk store. Before the next group's first write into the shared
// buffer thread 0 waits until its stores have read the staged line. No cluster barrier:
// the CTAs of a cluster only run adjacent lines at the same time. Other launches take a
// zero tmap_out.
template <typename T, int L, bool BATCH, bool TICK = false>
__global__ void __launch_bounds__(1024, 1)
    line_pass_persistent(const LinePassArgs<T> a0, int n_groups, int* __restrict__ err,
                         const __grid_constant__ CUtensorMap tmap_out) {
  using PG = PGeo<T, L>;
  static_assert(!TICK || (BATCH && PG::CS == 1), "ticks run batched, without clusters");
  using Gm = typename PG::G;
  constexpr int E = PG::E, J = L / E, LPI = PG::LPI, CS = PG::CS, GL = PG::GL;
  constexpr bool TST = PG::SWAP && CS > 1 && !BATCH;
  constexpr int TBOX = 256;  // rows per tensor store
  static_assert(!TST || (LPI == 1 && (size_t)L * sizeof(Q4<T>) <= PG::F_BYTES), "staged line");
  extern __shared__ __align__(128) unsigned char psmem[];
  Cx<T>* fbuf = reinterpret_cast<Cx<T>*>(psmem);
  Q4<T>* psi_z = reinterpret_cast<Q4<T>*>(psmem + PG::OFF_PSI);
  T* beta_z = reinterpret_cast<T*>(psmem + PG::OFF_BETA);
  Q4<T>* u_z = reinterpret_cast<Q4<T>*>(psmem + PG::OFF_U);
  // [0] spinor copy, [1] b-1/U copy
  uint64_t* bars = reinterpret_cast<uint64_t*>(psmem + PG::OFF_BAR);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(psmem + PG::OFF_BAR + 2 * sizeof(uint64_t));
  Cx<T>* t3tab = reinterpret_cast<Cx<T>*>(psmem + PG::OFF_T3);
  Cx<T>* t2tab = reinterpret_cast<Cx<T>*>(psmem + PG::OFF_T2);

  const int tid = threadIdx.x;
  const int warp = tid >> 5;
  const int lane = tid & 31;
  Cx<T>* xw = reinterpret_cast<Cx<T>*>(psmem) + (size_t)warp * 4 * PG::XQ;
  // line within the group, component, and index j of the thread's first element; the
  // 1024-point FFT puts line l on lane quarter l (warps l, l + 4, ...)
  const int lcta = PG::SWAP1K ? (warp & 3) : tid / PG::TPL;
  const int c = PG::SWAP1K ? (lane & 1) : ((tid - lcta * PG::TPL) & 1);
  const int j = PG::SWAP1K ? 16 * (warp >> 2) + (lane >> 1) : (tid - lcta * PG::TPL) >> 1;
  Cx<T>* buf = fbuf + lcta * Gm::STRIDE + c * Gm::COMP;
  const T sg = c ? T(-1) : T(1);
  constexpr uint32_t GROUP_BYTES = (uint32_t)PG::PSI_BYTES;
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
  auto issue_psi_x = [&](const LinePassArgs<T>& x, size_t first) {  // thread 0
    if (!dbg_in(first + PG::PSI_N - 1, (size_t)x.n_lines * L)) first = 0;
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(&bars[0], GROUP_BYTES + x.test_extra_tx);
    bulk_copy_g2s(psi_z, x.in + first, GROUP_BYTES, &bars[0]);
  };
  auto issue_psi = [&](int grp) {  // thread 0
    size_t first;
    const LinePassArgs<T> x = args_of(grp, &first);
    issue_psi_x(x, first);
  };
  // thread 0; an empty request completes its phase at once
  auto issue_bu_x = [&](const LinePassArgs<T>& x, size_t first) {
    if (!dbg_in(first + PG::PSI_N - 1, (size_t)x.n_lines * L)) first = 0;
    const Q4<T>* usrc = x.u_load ? x.u_load : x.u_store;
    const uint32_t bytes =
        (x.beta ? (uint32_t)PG::BETA_BYTES : 0u) + (usrc ? (uint32_t)PG::U_BYTES : 0u);
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(&bars[1], bytes);
#pragma unroll
    for (int k = 0; k < PG::CHUNKS; ++k) {
      if (x.beta)
        bulk_copy_g2s(reinterpret_cast<unsigned char*>(beta_z) + k * PG::BETA_PITCH,
                      x.beta + first + k * (PG::BETA_CHUNK / sizeof(T)),
                      (uint32_t)PG::BETA_CHUNK, &bars[1]);
      if (usrc)
        bulk_copy_g2s(reinterpret_cast<unsigned char*>(u_z) + k * PG::U_PITCH,
                      usrc + first + k * (PG::U_CHUNK / sizeof(Q4<T>)), (uint32_t)PG::U_CHUNK,
                      &bars[1]);
    }
  };
  auto issue_bu = [&](int grp) {
    size_t first;
    const LinePassArgs<T> x = args_of(grp, &first);
    issue_bu_x(x, first);
  };

  // ---- batched tick: work item {k, p, i, gi, wait} (k < 0: none) broadcast through a
  // shared-memory ring, slot it % 3 for iteration it; tpre[k] = first item of step k
  int* s_item = reinterpret_cast<int*>(psmem + PG::OFF_ITEM);
  int* tpre = reinterpret_cast<int*>(psmem + PG::OFF_TPRE);
  auto tick_decode = [&](int t, int* out5) {  // thread 0: item number -> {k, p, i, gi, 0}
    out5[4] = 0;
    if (t >= tpre[a0.tick_k]) {
      out5[0] = -1;
      return;
    }
    int lo = 0, hi = a0.tick_k;  // tpre[lo] <= t < tpre[hi]
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (tpre[mid] <= t) lo = mid;
      else hi = mid;
    }
    t -= tpre[lo];
    const int per_pass = (tpre[lo + 1] - tpre[lo]) >> 1;
    const int p = t >= per_pass ? 1 : 0;
    t -= p * per_pass;
    const int i = t / gpi;
    out5[0] = lo;
    out5[1] = p;
    out5[2] = i;
    out5[3] = t - i * gpi;
  };
  auto tick_args = [&](const int* it4, size_t* first) {
    LinePassArgs<T> x = a0;
    x.inst = a0.inst + ((size_t)it4[0] * 2 + it4[1]) * a0.inst_capacity;
    bind_instance(x, it4[2]);
    x.sigma = it4[1];
    *first = (size_t)it4[3] * LPI * L;
    return x;
  };
  auto tick_ready = [&](const int* it4) {  // thread 0
    return ld_acquire_gpu(a0.tick_done + it4[2]) >= (2 * it4[0] + it4[1]) * gpi;
  };
  auto tick_wait = [&](const int* it4) {  // thread 0, bounded
    const uint64_t t0 = global_ns();
    while (!tick_ready(it4)) {
      if (global_ns() - t0 > kWaitNs) {
        atomicExch(err, kErrTimeout);
        return;
      }
    }
  };

  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    fence_mbar_init();
  }
  if constexpr (PG::SWAP) {
    // pass-3 twiddles W_64^(s t) (block of span 8 of the pass table: [(t - 1) 8 + s])
    if (tid < 56) {
      const int s3 = tid / 7, t = tid - s3 * 7 + 1;
      t3tab[s3 * 8 + t - 1] = ldg_cx(a0.tw + tw_offset(8, 8) + (t - 1) * 8 + s3);
    }
  }
  if constexpr (PG::SWAP1K) {
    // W_128^(u t) = W_1024^(8 u t), u < 16, t = 1..7, from the table's W_1024^k, k < 512
    if (tid < 112) {
      const int t = tid / 16 + 1, u = tid % 16, e = 8 * u * t;
      const Cx<T>* w0 = a0.tw + tw_offset(512, 8);
      const Cx<T> w = ldg_cx(w0 + (e & 511));
      t2tab[tid] = e < 512 ? w : Cx<T>{-w.re, -w.im};
    }
  }
  if constexpr (TICK) {
    // item offsets of the steps, then the first two items
    for (int k = tid; k < a0.tick_k; k += PG::THREADS) tpre[k + 1] = 2 * gpi * a0.n_inst[k];
    __syncthreads();
    if (tid == 0) {
      tpre[0] = 0;
      for (int k = 0; k < a0.tick_k; ++k) tpre[k + 1] += tpre[k];
      tick_decode(atomicAdd(a0.tick_queue, 1), s_item);
      tick_decode(atomicAdd(a0.tick_queue, 1), s_item + 5);
      s_item[4] = 1;  // the first item's rows are requested at its iteration
    }
  }
  if (warp == 0) tmem_alloc(tslot, PG::TMEM_COLS);
  tmem_fence_before_sync();
  __syncthreads();
  tmem_fence_after_sync();
  const uint32_t tbase = *tslot;
  const int quarter = warp & 3, slice = warp >> 2;
  const uint32_t tlane = tbase + ((32u * (uint32_t)quarter) << 16);  // this warp's lanes
  const uint32_t tpark = tlane + PG::T_PARK + 16u * (uint32_t)slice;
  if constexpr (PG::SWAP) {
    // passes 1 and 2 of the digit-swap FFT: W_4096^(j t) and W_512^((j mod 64) t) for
    // t = 1..7, from the pass table's blocks of span 512 and 64
#pragma unroll
    for (int p = 0; p < 2; ++p) {
      const Cx<T>* b = p == 0 ? a0.tw + tw_offset(512, 8) + j : a0.tw + tw_offset(64, 8) + (j & 63);
      const int span = p == 0 ? 512 : 64;
      float f[16];
#pragma unroll
      for (int t = 1; t < 8; ++t) {
        const Cx<T> w = ldg_cx(b + (t - 1) * span);
        f[2 * t - 2] = w.re;
        f[2 * t - 1] = w.im;
      }
      f[14] = f[15] = 0.f;
      tmem_st16(tlane + PG::T_TW + 32u * (uint32_t)slice + 16u * (uint32_t)p, f);
    }
    tmem_wait_st();
  }
  if constexpr (PG::SWAP1K) {
    // W_1024^(j t), t = 1..7, parked once per kernel (W_1024^(k + 512) = -W_1024^k)
    const Cx<T>* w0 = a0.tw + tw_offset(512, 8);
    float f[16];
#pragma unroll
    for (int t = 1; t < 8; ++t) {
      const int e = j * t;
      const Cx<T> w = ldg_cx(w0 + (e & 511));
      f[2 * t - 2] = e < 512 ? w.re : -w.re;
      f[2 * t - 1] = e < 512 ? w.im : -w.im;
    }
    f[14] = f[15] = 0.f;
    tmem_st16(tlane + PG::T_TW + 16u * (uint32_t)slice, f);
    tmem_wait_st();
  }
  // TICK: the instance slot of the previous group, not yet published (-1: none)
  int prev_i = -1;
  if constexpr (TICK) {
    if (tid == 0 && s_item[0] >= 0) {
      size_t f;
      const LinePassArgs<T> x = tick_args(s_item, &f);
      issue_bu_x(x, f);
    }
  } else {
    if (tid == 0 && cluster_id < n_super) {
      issue_psi(cluster_id * CS + rank);
      issue_bu(cluster_id * CS + rank);
    }
  }

  // transposed store: this thread's line within an output segment (THREADS is a multiple
  // of GL) and, for clusters, the shared::cluster address of that line in its owner's
  // staging buffer
  const int gline = tid % GL;
  uint32_t gsrc = 0;
  if constexpr (CS > 1) {
    const int owner = gline / LPI;
    gsrc = mapa_shared(smem_u32(psmem), (uint32_t)owner) +
           (uint32_t)((gline - owner * LPI) * PG::SPITCH * sizeof(Q4<T>));
  }
  bool failed = false;  // uniform across the CTA
  if constexpr (TST) {
    if (smem_u32(psmem) & 127u) {  // tensor stores read 128-B aligned boxes
      failed = true;
      if (tid == 0) atomicExch(err, kErrAlign);
    }
  }
  // copies requested / phases waited for, per mbarrier (uniform; at most one outstanding)
  const uint32_t first_issue =
      TICK ? (s_item[0] >= 0 ? 1u : 0u) : (cluster_id < n_super ? 1u : 0u);
  uint32_t issued[2] = {TICK ? 0u : first_issue, first_issue};
  uint32_t done[2] = {0u, 0u};
  int it = 0;
  // clusters with a gather (batched launches): the barrier after the transposed store is
  // split; its arrive ends an iteration and its wait comes just before the next write into
  // the staging area (the forward FFT's shared-memory exchange), so the load and the first
  // FFT passes overlap the peer's gather. pend: an arrive awaits its wait (uniform across
  // the cluster; never set on the TST path)
  bool pend = false;
  for (int s = cluster_id;; s += n_clusters, ++it) {
    // TICK: this iteration's item, the next one and the one after (thread 0 decodes it)
    int* cur = s_item + 5 * (it % 3);
    int* nxt = s_item + 5 * ((it + 1) % 3);
    int* nx2 = s_item + 5 * ((it + 2) % 3);
    if constexpr (TICK) {
      if (cur[0] < 0) break;
    } else {
      if (s >= n_super) break;
    }
    const uint32_t par = (uint32_t)it & 1u;
    const int g = s * CS + rank;
    const bool has_next = s + n_clusters < n_super;
    size_t gfirst;
    LinePassArgs<T> a;
    if constexpr (TICK) a = tick_args(cur, &gfirst);
    else a = args_of(g, &gfirst);
    int ticket = 0;     // TICK, thread 0: the queue position two items ahead
    int next_done = 0;  // TICK, thread 0: the next item's dependency counter, loaded early
    if constexpr (TICK) {
      if (failed) {  // no work: count the items done and keep taking them
        if (tid == 0) {
          if (prev_i >= 0) red_release_gpu_add(a0.tick_done + prev_i, 1);
          red_release_gpu_add(a0.tick_done + cur[2], 1);
          tick_decode(atomicAdd(a0.tick_queue, 1), nx2);
        }
        prev_i = -1;
        __syncthreads();
        continue;
      }
      if (cur[4]) {
        // the rows were not ready when this item became next: publish the previous group
        // (this item may depend on it), then wait for the item's dependencies
        if (prev_i >= 0) __threadfence();
        __syncthreads();
        if (tid == 0) {
          if (prev_i >= 0) red_release_gpu_add(a0.tick_done + prev_i, 1);
          tick_wait(cur);
          fence_proxy_async_global();  // the previous pass's stores before the bulk copy
          issue_psi_x(a, gfirst);
          issued[0] += 1;
        }
        prev_i = -1;
      }
      if (tid == 0) {
        ticket = atomicAdd(a0.tick_queue, 1);
        if (nxt[0] >= 0) next_done = ld_acquire_gpu(a0.tick_done + nxt[2]);
      }
    }
    Cx<T> v[E];
    Q4<T> o_out[TST ? E / 2 : 1];  // TST: this thread's finished points m = 4c .. 4c + 3
    const int lrow = lcta * L;  // this line's first point within the group
    if (!failed) {
      // a thread whose wait ran out reads whatever the zone holds; the barrier after the
      // load turns it into a failure of the whole CTA before anything is used
      bool ok = mbar_wait_bounded(&bars[0], par, kWaitNs);
      if (ok && a.u_load) ok = mbar_wait_bounded(&bars[1], par, kWaitNs);
      if constexpr (PG::SWAP) {
        // Both components of every point (a 16-byte read, shared by the pair); thread c
        // parks the full points m = 4c .. 4c + 3 of its 8, which it finishes in the epilogue.
        float park[2 * E];
#pragma unroll
        for (int mm = 0; mm < E / 2; ++mm) {
          Q4<T> pp[2];
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int m = mm + h * (E / 2);
            const int i = j + m * J;
            Q4<T> p = dbg_in(i, PG::PSI_N) ? psi_z[i] : Q4<T>{T(0), T(0), T(0), T(0)};
            if (a.u_load && dbg_in(PG::upos_jm(j, m), PG::U_N))
              p = apply_u(u_z[PG::upos_jm(j, m)], p);
            pp[h] = p;
            if (a.sigma == 0) v[m] = cfma_p(sg, Cx<T>{p.z, p.w}, Cx<T>{p.x, p.y});
            else v[m] = {p.x + sg * p.w, p.y - sg * p.z};
          }
          const Q4<T> mine = c ? pp[1] : pp[0];
          park[4 * mm] = mine.x;
          park[4 * mm + 1] = mine.y;
          park[4 * mm + 2] = mine.z;
          park[4 * mm + 3] = mine.w;
        }
        tmem_st16(tpark, park);
      } else {
        const Cx<T>* src_c = reinterpret_cast<const Cx<T>*>(psi_z + lrow) + c;
        float park[2 * E];
#pragma unroll
        for (int m = 0; m < E; ++m) {
          const int i = j + m * J;
          Cx<T> own = dbg_in(lrow + i, PG::PSI_N) ? src_c[2 * i] : Cx<T>{T(0), T(0)};
          Cx<T> oth = shfl_pair(own);
          if (a.u_load && dbg_in(lrow + i, PG::U_N)) {
            own = apply_u_row(u_z[lrow + i], own, oth, c);
            oth = shfl_pair(own);
          }
          park[2 * m] = own.re;
          park[2 * m + 1] = own.im;
          const Cx<T> p1 = c ? oth : own, p2 = c ? own : oth;
          if (a.sigma == 0) v[m] = {p1.re + sg * p2.re, p1.im + sg * p2.im};
          else v[m] = {p1.re + sg * p2.im, p1.im - sg * p2.re};
        }
        tmem_st16(tpark, park);
      }
      // the spinor zone has been read: request the next group's rows
      const bool bad = __syncthreads_or(!ok);
      if constexpr (TICK) {
        if (tid == 0) tick_decode(ticket, nx2);
      }
      if (bad) {
        failed = true;
        if (tid == 0) atomicExch(err, kErrTimeout);
        if constexpr (TICK) {  // count the previous group done (the results are void)
          if (tid == 0 && prev_i >= 0) red_release_gpu_add(a0.tick_done + prev_i, 1);
          prev_i = -1;
        }
      } else {
        done[0] += 1;
        if constexpr (TICK) {
          if (tid == 0 && nxt[0] >= 0) {
            if (next_done >= (2 * nxt[0] + nxt[1]) * gpi) {
              size_t f;
              const LinePassArgs<T> x = tick_args(nxt, &f);
              fence_proxy_async_global();  // the previous pass's stores before the copy
              issue_psi_x(x, f);
              issued[0] += 1;
            } else {
              nxt[4] = 1;  // requested at its iteration, after a wait
            }
          }
        } else if (has_next) {
          if (tid == 0) issue_psi((s + n_clusters) * CS + rank);
          issued[0] += 1;
        }
      }
    }
    if (!failed) {
      if constexpr (PG::SWAP) {
        // batched launches wait before the transform: inside it, the extra branch makes
        // the compiler spill the instance's pointers
        if constexpr (BATCH && CS > 1)
          if (pend) cluster_wait();
        fft4096_swap<T, false>(v, fbuf + c * L, 9 * c, j, slice, quarter,
                               tlane + PG::T_TW + 32u * (uint32_t)slice, tlane + PG::T_X,
                               t3tab + 8 * slice, TST ? 2 : (!BATCH && CS > 1 && pend) ? 1 : 0);
        pend = false;
      } else if constexpr (PG::SWAP1K) {
        fft1024_swap<T, false, PG::XP, PG::XQ>(v, xw, lane, slice, quarter,
                                               tlane + PG::T_TW + 16u * (uint32_t)slice,
                                               tlane + PG::T_X, t2tab);
      } else {
        fft_passes<T, L, E, false>(v, buf, j, a.tw);
      }
      // frequency of element m: j + m J, or for the 1024-point FFT
      // slice + 8 (lane >> 2) + 64 m + 512 ((lane >> 1) & 1)
      // (the 1024-point FFT reads the permuted table when there is one: the natural one puts
      // a warp's 16 entries 128 B apart, in the same banks of L1)
      const Q4<T>* mb = a.mult + j;
      int ks = J;
      if constexpr (PG::SWAP1K) {
        const int l4 = lane >> 2, v0 = (lane >> 1) & 1, sl = warp >> 2;
        mb = a.mult_perm ? a.mult_perm + (v0 * 64 + sl * 8 + l4) : a.mult + (sl + 8 * l4 + 512 * v0);
        ks = a.mult_perm ? 128 : 64;
      }
#pragma unroll
      for (int m = 0; m < E; ++m) {
        if constexpr (!PG::SWAP)
          if ((m & 3) == 0) asm volatile("" ::: "memory");  // at most 4 loads in flight
        const Q4<T> q = ldg_q4(mb + m * ks);
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
      if constexpr (PG::SWAP) {
        // the forward FFT's exchanges (tensor memory and shared memory) have been read by
        // every thread before the inverse FFT's overwrite them
        tmem_fence_before_sync();
        __syncthreads();
        tmem_fence_after_sync();
        fft4096_swap<T, true>(v, fbuf + c * L, 9 * c, j2, slice, quarter,
                              tlane + PG::T_TW + 32u * (uint32_t)slice, tlane + PG::T_X,
                              t3tab + 8 * slice);
      }
      else if constexpr (PG::SWAP1K)
        fft1024_swap<T, true, PG::XP, PG::XQ>(v, xw, lane, slice, quarter,
                                              tlane + PG::T_TW + 16u * (uint32_t)slice,
                                              tlane + PG::T_X2, t2tab);
      else
        fft_passes<T, L, E, true>(v, buf2, j2, a.tw);

      // b - 1 / U of this group; the barrier also frees the FFT buffer for staging (TICK:
      // and publishes the previous group, whose stores completed long ago)
      const bool ok = mbar_wait_bounded(&bars[1], par, kWaitNs);
      if constexpr (TICK) {
        if (prev_i >= 0) __threadfence();
      }
      const bool bad_bu = __syncthreads_or(!ok);
      if constexpr (TICK) {
        if (tid == 0 && prev_i >= 0) red_release_gpu_add(a0.tick_done + prev_i, 1);
        prev_i = -1;
      }
      if (bad_bu) {
        failed = true;
        if (tid == 0) atomicExch(err, kErrTimeout);
      } else {
        done[1] += 1;
        tmem_wait_st();
        Q4<T>* stage = reinterpret_cast<Q4<T>*>(psmem);
        if constexpr (TST) {
          // the pair's eigencomponents meet through a shuffle (the shared buffer holds the
          // staged line here); thread c finishes points m = 4c .. 4c + 3
          float pk[2 * E];
          tmem_ld16(tpark, pk);
          tmem_wait_ld_regs(pk);
#pragma unroll
          for (int mm = 0; mm < E / 2; ++mm) {
            const int m4 = 4 * c + mm;
            const Cx<T> snd = c ? v[mm] : v[mm + E / 2];  // the partner's points
            const Cx<T> mine = c ? v[mm + E / 2] : v[mm];
            const Cx<T> rcv = {__shfl_xor_sync(0xffffffffu, snd.re, 1),
                               __shfl_xor_sync(0xffffffffu, snd.im, 1)};
            const Cx<T> dp = c ? rcv : mine, dm = c ? mine : rcv;  // (D+, D-)
            const Cx<T> d1 = cadd_p(dp, dm);
            const Cx<T> dd2 = csub_p(dp, dm);
            const T bm1 = (a.beta && dbg_in(PG::bpos_jm(j, m4), PG::BETA_N))
                              ? beta_z[PG::bpos_jm(j, m4)] : T(0);
            const Cx<T> o1 = cfma_p(bm1, d1, cadd_p(Cx<T>{pk[4 * mm], pk[4 * mm + 1]}, d1));
            Cx<T> o2;
            if (a.sigma == 0) {
              o2 = cfma_p(bm1, dd2, cadd_p(Cx<T>{pk[4 * mm + 2], pk[4 * mm + 3]}, dd2));
            } else {
              const Cx<T> d2 = mul_i(dd2);
              o2 = {(pk[4 * mm + 2] + d2.re) + bm1 * d2.re, (pk[4 * mm + 3] + d2.im) + bm1 * d2.im};
            }
            Q4<T> o = {o1.re, o1.im, o2.re, o2.im};
            if (a.u_store && dbg_in(PG::upos_jm(j, m4), PG::U_N))
              o = apply_u(u_z[PG::upos_jm(j, m4)], o);
            o_out[mm] = o;
          }
        } else if constexpr (PG::SWAP) {
          // eigencomponent results of the pair meet in the staging buffer (the partner is
          // the neighbouring lane); thread c then finishes points m = 4c .. 4c + 3
          Cx<T>* stc = reinterpret_cast<Cx<T>*>(stage) + c;
#pragma unroll
          for (int m = 0; m < E; ++m)
            if (dbg_in(PG::spos_jm(j, m), PG::STAGE_N)) stc[2 * PG::spos_jm(j, m)] = v[m];
          __syncwarp();
          float pk[2 * E];
          tmem_ld16(tpark, pk);
          tmem_wait_ld_regs(pk);
#pragma unroll
          for (int mm = 0; mm < E / 2; ++mm) {
            const int m4 = 4 * c + mm;  // point j + m4 J
            const bool sp_ok = dbg_in(PG::spos_jm(j, m4), PG::STAGE_N);
            const Q4<T> dd = sp_ok ? stage[PG::spos_jm(j, m4)]  // (D+, D-)
                                   : Q4<T>{T(0), T(0), T(0), T(0)};
            const Cx<T> dp = {dd.x, dd.y}, dm = {dd.z, dd.w};
            const Cx<T> d1 = cadd_p(dp, dm);
            const Cx<T> dd2 = csub_p(dp, dm);
            const T bm1 = (a.beta && dbg_in(PG::bpos_jm(j, m4), PG::BETA_N))
                              ? beta_z[PG::bpos_jm(j, m4)] : T(0);
            // psi + D + (b - 1) D per component
            const Cx<T> o1 = cfma_p(bm1, d1, cadd_p(Cx<T>{pk[4 * mm], pk[4 * mm + 1]}, d1));
            Cx<T> o2;
            if (a.sigma == 0) {
              o2 = cfma_p(bm1, dd2, cadd_p(Cx<T>{pk[4 * mm + 2], pk[4 * mm + 3]}, dd2));
            } else {
              const Cx<T> d2 = mul_i(dd2);
              o2 = {(pk[4 * mm + 2] + d2.re) + bm1 * d2.re, (pk[4 * mm + 3] + d2.im) + bm1 * d2.im};
            }
            Q4<T> o = {o1.re, o1.im, o2.re, o2.im};
            if (a.u_store && dbg_in(PG::upos_jm(j, m4), PG::U_N))
              o = apply_u(u_z[PG::upos_jm(j, m4)], o);
            if (sp_ok) stage[PG::spos_jm(j, m4)] = o;
          }
        } else {
          Cx<T>* my_stage = reinterpret_cast<Cx<T>*>(stage + (size_t)lcta * PG::SPITCH) + c;
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            float pk[E];
            tmem_ld8(tpark + (uint32_t)(h * E), pk);
            tmem_wait_ld_regs(pk);
#pragma unroll
            for (int mm = 0; mm < E / 2; ++mm) {
              const int m = h * (E / 2) + mm;
              const int i = j + m * J;
              const Cx<T> oth = shfl_pair(v[m]);
              const Cx<T> dp = c ? oth : v[m], dm = c ? v[m] : oth;
              Cx<T> d;
              if (c == 0) d = cadd_p(dp, dm);
              else d = a.sigma == 0 ? csub_p(dp, dm) : mul_i(csub_p(dp, dm));
              const Cx<T> p = {pk[2 * mm], pk[2 * mm + 1]};
              const T bm1 = (a.beta && dbg_in(lrow + i, PG::BETA_N)) ? beta_z[lrow + i] : T(0);
              Cx<T> o = cfma_p(bm1, d, cadd_p(p, d));  // (p + d) + (b - 1) d
              if (a.u_store && dbg_in(lrow + i, PG::U_N))
                o = apply_u_row(u_z[lrow + i], o, shfl_pair(o), c);
              if (dbg_in((size_t)lcta * PG::SPITCH + i, PG::STAGE_N)) my_stage[2 * i] = o;
            }
          }
        }
      }
    }
    if constexpr (TST) {
      // ---- TST store: the staged line, then (after the barrier, which also frees the
      // b - 1 / U zone) the next rows requested and the line's stores issued
      if (!failed) {
#pragma unroll
        for (int mm = 0; mm < E / 2; ++mm) {
          const int i = j + (4 * c + mm) * J;
          if (dbg_in(i, (size_t)L)) reinterpret_cast<Q4<T>*>(psmem)[i] = o_out[mm];
        }
        fence_proxy_async_smem();  // the staging writes before the (async-proxy) stores
      }
      __syncthreads();
      if (!failed && has_next) {
        if (tid == 0) issue_bu((s + n_clusters) * CS + rank);
        issued[1] += 1;
      }
      if (!failed && tid == 0) {
        if (a.store_normal) {
          if (dbg_in(gfirst + L - 1, (size_t)a.n_lines * L))
            bulk_copy_s2g(a.out + gfirst, smem_u32(psmem), (uint32_t)(L * sizeof(Q4<T>)));
        } else {
          const int line = (int)(gfirst / L);
#pragma unroll
          for (int k = 0; k < L / TBOX; ++k)
            if (dbg_in(line, (size_t)a.n_lines))
              tma_store_2d(&tmap_out, smem_u32(psmem) + (uint32_t)(k * TBOX * sizeof(Q4<T>)),
                           4 * line, k * TBOX);
        }
        bulk_commit();
      }
      continue;
    }
    if constexpr (CS > 1) {
      if (pend) {  // no forward FFT ran in this iteration (failure)
        cluster_wait();
        pend = false;
      }
    }
    // ---- transposed store of the super-group: out[i][s GL .. s GL + GL); CTA rank q
    // writes rows i of its L/CS slice, reading the owners' staging buffers. The barrier
    // publishes the staging writes and tells thread 0 that the b - 1 / U zone is free.
    if constexpr (CS > 1) cg::this_cluster().sync(); else __syncthreads();
    if constexpr (TICK) {
      if (!failed && tid == 0 && nxt[0] >= 0) {
        size_t f;
        const LinePassArgs<T> x = tick_args(nxt, &f);
        issue_bu_x(x, f);
        issued[1] += 1;
      }
    } else if (!failed && has_next) {
      if (tid == 0) issue_bu((s + n_clusters) * CS + rank);
      issued[1] += 1;
    }
    if (!failed && a.store_normal) {
      // rows back in the input's layout: this CTA's own lines, contiguous
      const Q4<T>* stage = reinterpret_cast<const Q4<T>*>(psmem);
      constexpr int NIT = LPI * L / PG::THREADS;
#pragma unroll
      for (int q = 0; q < NIT; ++q) {
        const int idx = tid + q * PG::THREADS;
        const bool out_ok = dbg_in(gfirst + idx, (size_t)a.n_lines * L);
        if constexpr (PG::SWAP) {  // one line; the padding of idx is idx / PAD_EVERY
          const size_t si = tid + tid / PG::PAD_EVERY + q * (PG::THREADS + PG::THREADS / PG::PAD_EVERY);
          if (out_ok && dbg_in(si, PG::STAGE_N)) a.out[gfirst + idx] = stage[si];
        } else {
          const int l = idx / L, i = idx - l * L;
          const size_t si = (size_t)l * PG::SPITCH + PG::spos(i);
          if (out_ok && dbg_in(si, PG::STAGE_N)) a.out[gfirst + idx] = stage[si];
        }
      }
    } else if (!failed) {
      const Q4<T>* stage = reinterpret_cast<const Q4<T>*>(psmem);
      const int line0 = (int)(gfirst / L) - rank * LPI;
      const int i0 = rank * (L / CS);
      constexpr int NIT = (L / CS) * GL / PG::THREADS;
      // item q of this thread: line gg of the segment, row i0 + tid / GL + q RPI
      constexpr int RPI = PG::THREADS / GL;
      static_assert(PG::THREADS % GL == 0, "items per row");
      static_assert(!PG::SWAP || (RPI == PG::PAD_EVERY && (L / CS) % PG::PAD_EVERY == 0),
                    "the padding of row i0 + tid / GL + q RPI is i0 / PAD_EVERY + q");
      const int r0 = i0 + tid / GL;
      const int sp0 = PG::SWAP ? r0 + i0 / PG::PAD_EVERY : r0;  // staging slot of row r0
      constexpr int SPQ = PG::SWAP ? RPI + 1 : RPI;
      Q4<T> val[NIT];
      if constexpr (CS > 1) {
        // gather through distributed shared memory from the owner's staged line
#pragma unroll
        for (int q = 0; q < NIT; ++q)
          val[q] = dbg_in(sp0 + q * SPQ, PG::STAGE_N)
                       ? ld_dsmem_q4<T>(gsrc + (uint32_t)((sp0 + q * SPQ) * sizeof(Q4<T>)))
                       : Q4<T>{T(0), T(0), T(0), T(0)};
      } else {
#pragma unroll
        for (int q = 0; q < NIT; ++q)
          val[q] = dbg_in((size_t)gline * PG::SPITCH + sp0 + q * SPQ, PG::STAGE_N)
                       ? stage[(size_t)gline * PG::SPITCH + sp0 + q * SPQ]
                       : Q4<T>{T(0), T(0), T(0), T(0)};
      }
      Q4<T>* dst = a.out + (size_t)r0 * a.n_lines + line0 + gline;
      const size_t dstep = (size_t)RPI * a.n_lines;
#pragma unroll
      for (int q = 0; q < NIT; ++q)  // streaming stores: the next pass reads them once
        if (dbg_in(r0 + q * RPI, L) && dbg_in(line0 + gline, a.n_lines))
          __stcs(reinterpret_cast<float4*>(dst + q * dstep),
                 make_float4(val[q].x, val[q].y, val[q].z, val[q].w));
    }
    // the staging buffer is free for the next super-group once every CTA of the cluster
    // has read it (the loads have returned: the stores above consumed them), so the
    // arrive needs no release fence for the outstanding global stores
    if constexpr (CS > 1) {
      cluster_arrive_relaxed();
      pend = true;
    } else {
      __syncthreads();
      // TICK: this group is published in the next iteration (or after the loop)
      if constexpr (TICK) prev_i = cur[2];
    }
  }
  if constexpr (TICK) {
    if (prev_i >= 0) {
      __threadfence();
      __syncthreads();
      if (tid == 0) red_release_gpu_add(a0.tick_done + prev_i, 1);
    }
  }
  if constexpr (CS > 1) {
    // the peer may still be reading this CTA's staged lines
    if (pend) cluster_wait();
  }
  if constexpr (TST) {
    if (tid == 0) bulk_wait_all();  // the tile stays allocated until the stores are done
  }
  if (failed && tid == 0) {
    // at most one copy per mbarrier is outstanding: the last one requested
    for (int b = 0; b < 2; ++b)
      if (issued[b] > done[b]) mbar_wait_bounded(&bars[b], (issued[b] - 1u) & 1u, kWaitNs);
  }
  tmem_wait_st();
  tmem_fence_before_sync();
  __syncthreads();
  tmem_fence_after_sync();
  if (warp == 0) tmem_dealloc(tbase, PG::TMEM_COLS);
}

}  // namespace dgb
