// etd_coeffs.cuh - per-mode ETD coefficients and launch-ordering helpers shared by the FFT axis
// passes and the tensor-core transform passes.
//
// phi_1, phi_2 of Section 2.2 (phi_0(z) = e^z, phi_{k+1}(z) = (phi_k(z) - 1/k!)/z) evaluated at
// z = -zeta, zeta = tau * lambda >= 0 of one eigenmode, with E = exp(-zeta) supplied by a table.
#pragma once
#include <cuda_runtime.h>

namespace etd {

__host__ __device__ constexpr double inv_factorial(int n) {
  double f = 1.0;
  for (int k = 2; k <= n; ++k) f *= (double)k;
  return 1.0 / f;
}

// phi_2(z) = sum_{m>=0} z^m / (m+2)! by Horner, for |z| < 1 (truncation below the type's epsilon).
template <class T> __device__ __forceinline__ T phi2_series(T z) {
  constexpr int M = sizeof(T) == 4 ? 10 : 18;
  T p = (T)inv_factorial(M + 1);
#pragma unroll
  for (int m = M - 2; m >= 0; --m) p = p * z + (T)inv_factorial(m + 2);
  return p;
}

// phi_1(-zeta), phi_2(-zeta) for zeta >= 0 with E = exp(-zeta): series for zeta < 1, else the
// recurrence phi_{k+1} = (phi_k - 1/k!)/z, which has no cancellation there. rz = 1/zeta.
template <class T> __device__ __forceinline__ void phi12(T zeta, T E, T rz, T& p1, T& p2) {
  if (zeta < T(1)) {
    p2 = phi2_series<T>(-zeta);
    p1 = T(1) - zeta * p2;
  } else {
    p1 = (T(1) - E) * rz;
    p2 = (T(1) - p1) * rz;
  }
}
template <class T> __device__ __forceinline__ T phi1_only(T zeta, T E, T rz) {
  if (zeta < T(1)) return T(1) - zeta * phi2_series<T>(-zeta);
  return (T(1) - E) * rz;
}
// 1/zeta (zeta > 0 where it is used): one division per mode serves every phi of the mode.
template <class T> __device__ __forceinline__ T recip(T z) { return T(1) / z; }

// Hardware reciprocal approximation (one MUFU instruction, within 1 ulp; flushes denormals), for
// the tensor-core routes whose operand rounding is far coarser.
__device__ __forceinline__ float rcp_approx(float z) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(z));
  return r;
}

// Correctly rounded reciprocal (the same value as 1/z).
__device__ __forceinline__ float rcp_rn(float z) { return __frcp_rn(z); }
__device__ __forceinline__ double rcp_rn(double z) { return __drcp_rn(z); }

// Branch-free forms of phi12 / phi1_only: the series and the closed form are both evaluated and
// the one valid for zeta selected, so modes on both sides of zeta = 1 in one warp do not diverge
// and the chains of several modes interleave.
template <class T> __device__ __forceinline__ void phi12_sel(T zeta, T E, T& p1, T& p2) {
  const bool small = zeta < T(1);
  const T s2 = phi2_series<T>(small ? -zeta : T(0));
  const T rz = rcp_rn(small ? T(1) : zeta);
  const T c1 = (T(1) - E) * rz;
  p2 = small ? s2 : (T(1) - c1) * rz;
  p1 = small ? T(1) - zeta * s2 : c1;
}
template <class T> __device__ __forceinline__ T phi1_sel(T zeta, T E) {
  const bool small = zeta < T(1);
  const T s2 = phi2_series<T>(small ? -zeta : T(0));
  const T rz = rcp_rn(small ? T(1) : zeta);
  return small ? T(1) - zeta * s2 : (T(1) - E) * rz;
}

// The phi-function weights of one mode as the FFT pass epilogues evaluate them in type T (the
// per-mode path: 3D plans, and 2D plans without per-mode weight tables), from zeta = tau lambda >= 0 and
// E = e^{-zeta} as stored (products of per-axis factors): phi_1(-zeta), phi_2(-zeta) by the closed forms
// with one correctly rounded reciprocal rz = 1/zeta for zeta >= 1, and below by the series of phi_2 with
// phi_1 = 1 - zeta phi_2; the series runs only in warps holding such a mode (act: the calling lanes,
// every one of which votes with its own predicate).
template <class T>
__device__ __forceinline__ void stage_phi12(T zeta, T E, unsigned act, T& p1, T& p2, T& rz) {
  const bool small = zeta < T(1);
  rz = rcp_rn(small ? T(1) : zeta);
  p1 = (T(1) - E) * rz;
  p2 = (T(1) - p1) * rz;
  if (__any_sync(act, small)) {
    const T s2 = phi2_series<T>(small ? -zeta : T(0));
    p2 = small ? s2 : p2;
    p1 = small ? T(1) - zeta * s2 : p1;
  }
}
// c2 phi_1(-c2 zeta) with Ec = e^{-c2 zeta}: (1 - Ec) / zeta from rz for c2 zeta >= 1, the series below.
template <class T>
__device__ __forceinline__ T stage_phi1c(T zeta, T Ec, T c2, T rz, unsigned act) {
  const T zc = c2 * zeta;
  T t = (T(1) - Ec) * rz;
  const bool smc = zc < T(1);
  if (__any_sync(act, smc)) {
    const T s2c = phi2_series<T>(smc ? -zc : T(0));
    t = smc ? c2 * (T(1) - zc * s2c) : t;
  }
  return t;
}

// Programmatic dependent launch: wait until the previous kernel in the stream has completed and its
// writes are visible (a no-op when launched without the attribute), and let the next kernel start
// its prologue early. Every pass waits before its first read of a field.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void griddep_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory"); }

}  // namespace etd
