// Shared device types and helpers for the Scheme II kernels (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace dgb {

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
