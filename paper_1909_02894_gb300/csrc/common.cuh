// Shared device types and helpers for the Scheme II kernels (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

// Debug builds (nvcc -DDIRAC_DEBUG=1, see DIRAC_NVCC_EXTRA) check the index of each
// memory access of the line passes against its buffer: a failed check sets this
// translation unit's flag and the access is skipped (a load gives zero). Release builds
// compile the checks away.
#ifndef DIRAC_DEBUG
#define DIRAC_DEBUG 0
#endif

namespace dgb {

#if DIRAC_DEBUG
static __device__ int g_dbg_bounds = 0;
#endif
// true when idx < bound (always, in release builds)
__device__ __forceinline__ bool dbg_in(size_t idx, size_t bound) {
#if DIRAC_DEBUG
  if (idx >= bound) {
    atomicExch(&g_dbg_bounds, 1);
    return false;
  }
#endif
  return true;
}

// Complex number in registers / shared memory.
template <typename T>
struct __align__(2 * sizeof(T)) Cx {
  T re, im;
};

// Four reals: a spinor point (psi1.re, psi1.im, psi2.re, psi2.im), a half-step matrix
// (c0 - 1, c1, c2, c3), or a k-space multiplier (hi/lo pairs).
template <typename T>
struct __align__(4 * sizeof(T)) Q4 {
  T x, y, z, w;
};

template <typename T>
__device__ __forceinline__ Cx<T> cadd(Cx<T> a, Cx<T> b) { return {a.re + b.re, a.im + b.im}; }
template <typename T>
__device__ __forceinline__ Cx<T> csub(Cx<T> a, Cx<T> b) { return {a.re - b.re, a.im - b.im}; }
template <typename T>
__device__ __forceinline__ Cx<T> cmul(Cx<T> a, Cx<T> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
// a * conj(b)
template <typename T>
__device__ __forceinline__ Cx<T> cmulc(Cx<T> a, Cx<T> b) {
  return {a.re * b.re + a.im * b.im, a.im * b.re - a.re * b.im};
}
// ---- packed FP32 pairs (sm_100 and later): the (re, im) of a complex64 value in one
// 64-bit register pair, two FP32 operations per instruction, each rounded exactly like its
// scalar counterpart (add/sub/fma.rn.f32x2).
__device__ __forceinline__ unsigned long long pk2(float lo, float hi) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void upk2(unsigned long long r, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(r));
}
__device__ __forceinline__ unsigned long long add_f32x2(unsigned long long a,
                                                         unsigned long long b) {
  unsigned long long r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ unsigned long long sub_f32x2(unsigned long long a,
                                                         unsigned long long b) {
  unsigned long long r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
// a * b + c per lane
__device__ __forceinline__ unsigned long long fma_f32x2(unsigned long long a,
                                                         unsigned long long b,
                                                         unsigned long long c) {
  unsigned long long r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}
__device__ __forceinline__ unsigned long long pk2(Cx<float> a) { return pk2(a.re, a.im); }
__device__ __forceinline__ Cx<float> upk2(unsigned long long r) {
  Cx<float> a;
  upk2(r, a.re, a.im);
  return a;
}

// a + b and a - b: one packed instruction for complex64, the scalar pair otherwise.
// Building with -DDGB_PACKED_F32X2=0 keeps the scalar form for complex64 too (same results).
#ifndef DGB_PACKED_F32X2
#define DGB_PACKED_F32X2 1
#endif
template <typename T>
__device__ __forceinline__ Cx<T> cadd_p(Cx<T> a, Cx<T> b) { return cadd(a, b); }
template <typename T>
__device__ __forceinline__ Cx<T> csub_p(Cx<T> a, Cx<T> b) { return csub(a, b); }
// s * a + b with the same real s on both parts (a single fma.rn.f32x2 for complex64)
template <typename T>
__device__ __forceinline__ Cx<T> cfma_p(T s, Cx<T> a, Cx<T> b) {
  return {s * a.re + b.re, s * a.im + b.im};
}
#if DGB_PACKED_F32X2
template <>
__device__ __forceinline__ Cx<float> cadd_p<float>(Cx<float> a, Cx<float> b) {
  return upk2(add_f32x2(pk2(a), pk2(b)));
}
template <>
__device__ __forceinline__ Cx<float> csub_p<float>(Cx<float> a, Cx<float> b) {
  return upk2(sub_f32x2(pk2(a), pk2(b)));
}
template <>
__device__ __forceinline__ Cx<float> cfma_p<float>(float s, Cx<float> a, Cx<float> b) {
  return upk2(fma_f32x2(pk2(s, s), pk2(a), pk2(b)));
}
#endif

template <typename T>
__device__ __forceinline__ Cx<T> mul_i(Cx<T> a) { return {-a.im, a.re}; }
template <typename T>
__device__ __forceinline__ Cx<T> mul_mi(Cx<T> a) { return {a.im, -a.re}; }

// psi <- U psi with U = [[c0 + i c3, c1 - i c2], [c1 + i c2, c0 - i c3]] stored as
// u = (c0 - 1, c1, c2, c3): the deviation from the identity is applied and added, so a
// U close to I costs one rounding of psi.
template <typename T>
__device__ __forceinline__ Q4<T> apply_u(Q4<T> u, Q4<T> p) {
  const T ar = p.x, ai = p.y, br = p.z, bi = p.w;
  T d1r = u.x * ar - u.w * ai + u.y * br + u.z * bi;
  T d1i = u.x * ai + u.w * ar + u.y * bi - u.z * br;
  T d2r = u.x * br + u.w * bi + u.y * ar - u.z * ai;
  T d2i = u.x * bi - u.w * br + u.y * ai + u.z * ar;
  return {ar + d1r, ai + d1i, br + d2r, bi + d2i};
}

}  // namespace dgb

namespace dgb {

// ---- asynchronous bulk copies and mbarriers (sm_90+ PTX), used by the persistent pass
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// Orders this thread's earlier generic-proxy shared-memory accesses before later
// async-proxy operations on the same memory (bulk copies that write it, bulk and tensor
// stores that read it).
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
// Global -> shared bulk copy (16-B aligned addresses, size a multiple of 16) whose
// completion is counted on the mbarrier.
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes,
                                              uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void bulk_prefetch_l2(const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Bounded wait: gives up after limit_ns nanoseconds of wall time.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  uint64_t limit_ns) {
  const uint64_t t0 = global_ns();
  while (!mbar_try_wait(bar, parity))
    if (global_ns() - t0 > limit_ns) return false;
  return true;
}

// GPU-scope acquire load and release increment of a global counter (cross-CTA ordering of
// the batched tick's work items).
__device__ __forceinline__ int ld_acquire_gpu(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void red_release_gpu_add(int* p, int v) {
  asm volatile("red.release.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
// Orders this thread's earlier generic-proxy accesses of global memory before its later
// async-proxy (bulk copy) accesses.
__device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}

// Position of frequency k (< 1024) in the step-multiplier table of 1024-point lines that
// the 1024-point persistent pass reads: its digit-swap FFT leaves frequency
// s + 8 l4 + 64 m + 512 v0 in element m of the thread with warp slice s and lane bits
// l4 = lane >> 2, v0 = (lane >> 1) & 1, so the table is ordered (m, v0, s, l4) and the 16
// entries a warp reads for one m are two runs of 8 consecutive entries.
__host__ __device__ constexpr int perm1024(int k) {
  return ((k >> 6) & 7) * 128 + ((k >> 9) & 1) * 64 + (k & 7) * 8 + ((k >> 3) & 7);
}

// ---- asynchronous stores from shared memory (bulk-group completion)
// Tiled tensor store of one 2D box from shared memory (128-B aligned) to global memory,
// at element coordinates (x, y) of the tensor map; x times the element size a multiple of
// 16 bytes, neither coordinate negative.
__device__ __forceinline__ void tma_store_2d(const void* tmap, uint32_t smem, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%2, %3}], [%1];" ::"l"(tmap),
      "r"(smem), "r"(x), "r"(y)
      : "memory");
}
// Bulk store of `bytes` (a multiple of 16) from shared to global memory, both 16-B aligned.
__device__ __forceinline__ void bulk_copy_s2g(void* dst, uint32_t smem, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst),
               "r"(smem), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() {
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
// every committed bulk store of this thread has read its shared-memory source
__device__ __forceinline__ void bulk_wait_read_all() {
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
// every committed bulk store of this thread is complete
__device__ __forceinline__ void bulk_wait_all() {
  asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

// Address of the same shared-memory variable in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t mapa_shared(uint32_t addr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
  return r;
}
template <typename T>
__device__ __forceinline__ Q4<T> ld_dsmem_q4(uint32_t addr);
template <>
__device__ __forceinline__ Q4<float> ld_dsmem_q4<float>(uint32_t addr) {
  Q4<float> v;
  asm volatile("ld.shared::cluster.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "r"(addr)
               : "memory");
  return v;
}

// ---- tensor memory (tcgen05, sm_100a+) used as per-thread parking space. A CTA holds
// `cols` columns x 128 lanes of 32-bit cells; warp w reaches lanes 32 (w % 4) .. + 31
// (its lane quarter) with the 32x32b shapes, one lane per thread.
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t cols) {  // one warp
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   smem_u32(slot)),
               "r"(cols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t cols) {  // one warp
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(cols)
               : "memory");
}
__device__ __forceinline__ void tmem_fence_before_sync() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tmem_fence_after_sync() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// 16 consecutive columns of this thread's lane <- r[0..15]
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const float (&r)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
      "{%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16};" ::"r"(taddr),
      "f"(r[0]), "f"(r[1]), "f"(r[2]), "f"(r[3]), "f"(r[4]), "f"(r[5]), "f"(r[6]), "f"(r[7]),
      "f"(r[8]), "f"(r[9]), "f"(r[10]), "f"(r[11]), "f"(r[12]), "f"(r[13]), "f"(r[14]), "f"(r[15])
      : "memory");
}
// r[0..15] <- 16 consecutive columns of this thread's lane (complete after a wait)
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=f"(r[0]), "=f"(r[1]), "=f"(r[2]), "=f"(r[3]), "=f"(r[4]), "=f"(r[5]), "=f"(r[6]),
        "=f"(r[7]), "=f"(r[8]), "=f"(r[9]), "=f"(r[10]), "=f"(r[11]), "=f"(r[12]), "=f"(r[13]),
        "=f"(r[14]), "=f"(r[15])
      : "r"(taddr)
      : "memory");
}
// r[0..7] <- 8 consecutive columns of this thread's lane (complete after tmem_wait_ld)
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&r)[8]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=f"(r[0]), "=f"(r[1]), "=f"(r[2]), "=f"(r[3]), "=f"(r[4]), "=f"(r[5]), "=f"(r[6]),
        "=f"(r[7])
      : "r"(taddr)
      : "memory");
}
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const float (&r)[8]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr),
      "f"(r[0]), "f"(r[1]), "f"(r[2]), "f"(r[3]), "f"(r[4]), "f"(r[5]), "f"(r[6]), "f"(r[7])
      : "memory");
}
// r[0..1] <- 2 consecutive columns of this thread's lane (complete after tmem_wait_ld)
__device__ __forceinline__ void tmem_ld2(uint32_t taddr, float (&r)[2]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0, %1}, [%2];"
               : "=f"(r[0]), "=f"(r[1])
               : "r"(taddr)
               : "memory");
}
// Waits for this thread's tensor-memory loads; naming the destination registers as
// operands keeps every use of them after the wait.
__device__ __forceinline__ void tmem_wait_ld_regs(float (&r)[8]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+f"(r[0]), "+f"(r[1]), "+f"(r[2]), "+f"(r[3]), "+f"(r[4]), "+f"(r[5]),
                 "+f"(r[6]), "+f"(r[7])::"memory");
}
__device__ __forceinline__ void tmem_wait_ld_regs(float (&r)[16]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+f"(r[0]), "+f"(r[1]), "+f"(r[2]), "+f"(r[3]), "+f"(r[4]), "+f"(r[5]),
                 "+f"(r[6]), "+f"(r[7]), "+f"(r[8]), "+f"(r[9]), "+f"(r[10]), "+f"(r[11]),
                 "+f"(r[12]), "+f"(r[13]), "+f"(r[14]), "+f"(r[15])::"memory");
}
// Barrier over `count` threads (a multiple of 32) on hardware barrier `id` (1..15).
__device__ __forceinline__ void named_barrier(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}
__device__ __forceinline__ void tmem_wait_st() {
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
// Cluster barrier without release semantics: orders execution only (no wait for this
// thread's outstanding global stores); the wait side keeps acquire.
// split cluster barrier: arrive without release semantics, and the matching wait
__device__ __forceinline__ void cluster_arrive_relaxed() {
  asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() {
  asm volatile("barrier.cluster.wait.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_sync_relaxed() {
  asm volatile("barrier.cluster.arrive.relaxed.aligned;\n\tbarrier.cluster.wait.aligned;" :::
                   "memory");
}

}  // namespace dgb
