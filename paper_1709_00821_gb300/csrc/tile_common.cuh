// Device helpers shared by the tiled kernels (forward and adjoint): register-row loads and
// stores of K consecutive cells per lane, dynamic-index access into register arrays, the
// Eq. 15 pulse.
#pragma once

#include "rketd_internal.cuh"

namespace rketd {
namespace tile {

constexpr unsigned kFull = 0xffffffffu;

// Eq. 15, normalised by tau: amp ((t - t0)/tau) exp(-(t - t0)^2 / (2 tau^2)).
__device__ __forceinline__ double pulse(double t, double t0, double tau, double amp) {
  const double u = (t - t0) / tau;
  return amp * u * exp(-0.5 * u * u);
}

template <typename T, int K>
__device__ __forceinline__ T pick(const T (&r)[K], int i) {
  T v = T(0);
#pragma unroll
  for (int q = 0; q < K; ++q)
    if (q == i) v = r[q];
  return v;
}

template <typename T, int K>
__device__ __forceinline__ void put(T (&r)[K], int i, T v) {
#pragma unroll
  for (int q = 0; q < K; ++q)
    if (q == i) r[q] = v;
}

// Four consecutive values at p (16-byte aligned for float, 32 for double).
__device__ __forceinline__ void ld4(const float* p, float* r) {
  const float4 q = __ldg(reinterpret_cast<const float4*>(p));
  r[0] = q.x; r[1] = q.y; r[2] = q.z; r[3] = q.w;
}
__device__ __forceinline__ void ld4(const double* p, double* r) {
  const double2 q0 = __ldg(reinterpret_cast<const double2*>(p));
  const double2 q1 = __ldg(reinterpret_cast<const double2*>(p) + 1);
  r[0] = q0.x; r[1] = q0.y; r[2] = q1.x; r[3] = q1.y;
}
__device__ __forceinline__ void st4(float* p, const float* r) {
  *reinterpret_cast<float4*>(p) = make_float4(r[0], r[1], r[2], r[3]);
}
__device__ __forceinline__ void st4(double* p, const double* r) {
  reinterpret_cast<double2*>(p)[0] = make_double2(r[0], r[1]);
  reinterpret_cast<double2*>(p)[1] = make_double2(r[2], r[3]);
}

// K values of slab storage `base` at slab-local cells g0 .. g0+K-1; groups of four
// outside [0, hi) read as zero (g0 and hi are multiples of 4).
template <typename T, int K, bool MASK>
__device__ __forceinline__ void load_row(const T* __restrict__ base, int64_t g0, int64_t hi, T (&r)[K]) {
#pragma unroll
  for (int v = 0; v < K / 4; ++v) {
    const int64_t g = g0 + 4 * v;
    if (!MASK || (g >= 0 && g < hi)) {
      ld4(base + g, &r[4 * v]);
    } else {
      r[4 * v] = r[4 * v + 1] = r[4 * v + 2] = r[4 * v + 3] = T(0);
    }
  }
}

// Stores the slots whose tile-local index lies in [vlo, vhi).
template <typename T, int K>
__device__ __forceinline__ void store_row(T* __restrict__ base, int64_t g0, int li0, int vlo, int vhi,
                                          const T (&r)[K]) {
#pragma unroll
  for (int v = 0; v < K / 4; ++v) {
    const int li = li0 + 4 * v;
    if (li >= vlo && li + 4 <= vhi) {
      st4(base + g0 + 4 * v, &r[4 * v]);
    } else {
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (li + q >= vlo && li + q < vhi) base[g0 + 4 * v + q] = r[4 * v + q];
    }
  }
}


}  // namespace tile
}  // namespace rketd
