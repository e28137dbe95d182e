// Device helpers shared by the tiled kernels (forward and adjoint): register-row loads and
// stores of K consecutive cells per lane, dynamic-index access into register arrays, the
// Eq. 15 pulse.
#pragma once

#include <type_traits>

#include "rketd_internal.cuh"

namespace rketd {
namespace tile {

constexpr unsigned kFull = 0xffffffffu;

// Eq. 15, normalised by tau: amp ((t - t0)/tau) exp(-(t - t0)^2 / (2 tau^2)).
__device__ __forceinline__ double pulse(double t, double t0, double tau, double amp) {
  const double u = (t - t0) / tau;
  return amp * u * exp(-0.5 * u * u);
}

// The source values of one pass (steps n0 + 1 .. n0 + nsub, nsub <= 64), evaluated once per warp:
// lane l holds steps n0 + 1 + l and n0 + 33 + l. One FP64 pulse per lane and pass instead of one
// per step in the source lane (the FP64 pipe is narrow). Warp-uniform calls only.
template <typename T>
struct PassSource {
  T v0, v1;
};
template <typename T>
__device__ __forceinline__ PassSource<T> pass_source(int64_t n0, int nsub, double dt, double t0, double tau,
                                                     double amp, int lane) {
  PassSource<T> r{T(0), T(0)};
  if (lane < nsub) r.v0 = (T)pulse((double)(n0 + 1 + lane) * dt, t0, tau, amp);
  if (lane + 32 < nsub) r.v1 = (T)pulse((double)(n0 + 33 + lane) * dt, t0, tau, amp);
  return r;
}
// value of step n0 + 1 + t, all lanes (t warp-uniform)
template <typename T>
__device__ __forceinline__ T source_at(const PassSource<T>& p, int t) {
  return t < 32 ? __shfl_sync(kFull, p.v0, t) : __shfl_sync(kFull, p.v1, t - 32);
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

// The probes one lane samples in a pass, gathered once before the time loop: the first two in
// registers (slot among the lane's K cells, offset of the pass's first sample in the series
// buffer); a lane with more (rare: probes closer than K cells) reads the rest from the list.
struct LaneProbes {
  int n, s0, s1;
  int64_t o0, o1;
};
__device__ __forceinline__ LaneProbes lane_probes(const TileProbe* list, int begin, int count, int lane, int K,
                                                  int series_len, int series_pos) {
  LaneProbes r{0, 0, 0, 0, 0};
  for (int q = 0; q < count; ++q) {
    const TileProbe p = list[begin + q];
    if (lane != p.local / K) continue;
    const int64_t o = (int64_t)p.slot * series_len + series_pos;
    if (r.n == 0) {
      r.s0 = p.local % K;
      r.o0 = o;
    } else if (r.n == 1) {
      r.s1 = p.local % K;
      r.o1 = o;
    }
    ++r.n;
  }
  return r;
}

// Four consecutive values at p (16-byte aligned for float, 32 for double). NC: through the
// read-only (non-coherent) path, for data no thread writes during the kernel; otherwise from L2
// (ld.global.cg), for data that other warps of the same kernel write (the persistent step).
template <bool NC = true>
__device__ __forceinline__ void ld4(const float* p, float* r) {
  const float4 q = NC ? __ldg(reinterpret_cast<const float4*>(p)) : __ldcg(reinterpret_cast<const float4*>(p));
  r[0] = q.x; r[1] = q.y; r[2] = q.z; r[3] = q.w;
}
template <bool NC = true>
__device__ __forceinline__ void ld4(const double* p, double* r) {
  const double2 q0 = NC ? __ldg(reinterpret_cast<const double2*>(p)) : __ldcg(reinterpret_cast<const double2*>(p));
  const double2 q1 =
      NC ? __ldg(reinterpret_cast<const double2*>(p) + 1) : __ldcg(reinterpret_cast<const double2*>(p) + 1);
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
template <typename T, int K, bool MASK, bool NC = true>
__device__ __forceinline__ void load_row(const T* __restrict__ base, int64_t g0, int64_t hi, T (&r)[K]) {
#pragma unroll
  for (int v = 0; v < K / 4; ++v) {
    const int64_t g = g0 + 4 * v;
    if (!MASK || (g >= 0 && g < hi)) {
      ld4<NC>(base + g, &r[4 * v]);
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


// ---- packed FP32x2: two cells in one 64-bit register (lo = half A cell, hi = half B cell) ----
typedef unsigned long long f2;  // lo = cell of half A, hi = cell of half B

__device__ __forceinline__ f2 pk(float lo, float hi) {
  f2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ float lo_of(f2 v) {
  float l, h;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(l), "=f"(h) : "l"(v));
  return l;
}
__device__ __forceinline__ float hi_of(f2 v) {
  float l, h;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(l), "=f"(h) : "l"(v));
  return h;
}
__device__ __forceinline__ f2 sub2(f2 a, f2 b) {
  f2 d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) {
  f2 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ f2 add2(f2 a, f2 b) {
  f2 d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2 mul2(f2 a, f2 b) {
  f2 d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}


// element `slot` (0..K-1) of a pair array
template <int P>
__device__ __forceinline__ float pick2(const f2 (&r)[P], int slot) {
  const int p = slot < P ? slot : slot - P;
  float v = 0.f;
#pragma unroll
  for (int q = 0; q < P; ++q)
    if (q == p) v = slot < P ? lo_of(r[q]) : hi_of(r[q]);
  return v;
}
template <int P>
__device__ __forceinline__ void put2(f2 (&r)[P], int slot, float v) {
  const int p = slot < P ? slot : slot - P;
#pragma unroll
  for (int q = 0; q < P; ++q)
    if (q == p) r[q] = slot < P ? pk(v, hi_of(r[q])) : pk(lo_of(r[q]), v);
}
// element S (a constant) of a pair array, read and written
template <int S, int P>
__device__ __forceinline__ float pick2c(const f2 (&r)[P]) {
  if constexpr (S < P) return lo_of(r[S]);
  else return hi_of(r[S - P]);
}
template <int S, int P>
__device__ __forceinline__ void put2c(f2 (&r)[P], float v) {
  if constexpr (S < P) r[S] = pk(v, hi_of(r[S]));
  else r[S - P] = pk(lo_of(r[S - P]), v);
}
// f(std::integral_constant<int, slot>) for a slot 0 .. 2P-1 that is the same in every lane of the
// warp: one uniform branch to code with a constant slot, instead of a select over every pair
#define RKETD_SLOT_CASE(S) \
  case S:                  \
    if constexpr (S < 2 * P) f(std::integral_constant<int, S>{}); \
    break;
template <int P, typename F>
__device__ __forceinline__ void at_uniform_slot(int slot, F&& f) {
  static_assert(2 * P <= 16, "at most 16 cells per lane");
  switch (slot) {
    RKETD_SLOT_CASE(0) RKETD_SLOT_CASE(1) RKETD_SLOT_CASE(2) RKETD_SLOT_CASE(3)
    RKETD_SLOT_CASE(4) RKETD_SLOT_CASE(5) RKETD_SLOT_CASE(6) RKETD_SLOT_CASE(7)
    RKETD_SLOT_CASE(8) RKETD_SLOT_CASE(9) RKETD_SLOT_CASE(10) RKETD_SLOT_CASE(11)
    RKETD_SLOT_CASE(12) RKETD_SLOT_CASE(13) RKETD_SLOT_CASE(14) RKETD_SLOT_CASE(15)
    default: break;
  }
}
#undef RKETD_SLOT_CASE


template <int K, bool NC = true>
__device__ __forceinline__ void load_pairs(const float* __restrict__ p, f2 (&r)[K / 2], bool negate) {
  constexpr int P = K / 2;
  float t[K];
#pragma unroll
  for (int v = 0; v < K / 4; ++v) {
    const float4 q = NC ? __ldg(reinterpret_cast<const float4*>(p) + v) : __ldcg(reinterpret_cast<const float4*>(p) + v);
    t[4 * v] = q.x;
    t[4 * v + 1] = q.y;
    t[4 * v + 2] = q.z;
    t[4 * v + 3] = q.w;
  }
#pragma unroll
  for (int q = 0; q < P; ++q) r[q] = negate ? pk(-t[q], -t[P + q]) : pk(t[q], t[P + q]);
}

template <int K>
__device__ __forceinline__ void store_pairs(float* __restrict__ p, int li0, int vlo, int vhi, const f2 (&r)[K / 2]) {
  constexpr int P = K / 2;
  float t[K];
#pragma unroll
  for (int q = 0; q < P; ++q) {
    t[q] = lo_of(r[q]);
    t[P + q] = hi_of(r[q]);
  }
#pragma unroll
  for (int v = 0; v < K / 4; ++v) {
    const int li = li0 + 4 * v;
    if (li >= vlo && li + 4 <= vhi) {
      reinterpret_cast<float4*>(p)[v] = make_float4(t[4 * v], t[4 * v + 1], t[4 * v + 2], t[4 * v + 3]);
    } else {
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (li + q >= vlo && li + q < vhi) p[4 * v + q] = t[4 * v + q];
    }
  }
}

}  // namespace tile
}  // namespace rketd
