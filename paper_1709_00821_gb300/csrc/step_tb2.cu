// Interior tiled step for FP32 fields with two cells per packed FP32x2 register.
//
// Same tile, halo and arithmetic as k_tb<float, K, interior> (step_tb.cu), but each lane's K
// cells are split into halves A = [0, K/2) and B = [K/2, K) and cell A[p] shares a 64-bit
// register with cell B[p]. Shifting by one cell then maps pair p to pair p-1 (or p+1) for
// both halves at once, so every update is one add/sub/fma.rn.f32x2 per pair: half the issue
// slots of the scalar kernel for the same FP32 work (the kernel is issue-bound: the FP32
// pipe runs the pair in two cycles either way). Only the two pairs at the ends of a lane's
// range need a repack per half step. Every element is rounded exactly as in the scalar
// kernel (fma2 is two fused multiply-adds, sub2 two subtractions), so the fields are bitwise
// identical to the plain and scalar tiled kernels.
#include "rketd_internal.cuh"

#ifndef RKETD_TB_MINB
#define RKETD_TB_MINB 3
#endif

namespace rketd {
namespace {

constexpr unsigned kFull = 0xffffffffu;
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

__device__ __forceinline__ double pulse(double t, double t0, double tau, double amp) {
  const double u = (t - t0) / tau;
  return amp * u * exp(-0.5 * u * u);
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

template <int K>
__device__ __forceinline__ void load_pairs(const float* __restrict__ p, f2 (&r)[K / 2], bool negate) {
  constexpr int P = K / 2;
  float t[K];
#pragma unroll
  for (int v = 0; v < K / 4; ++v) {
    const float4 q = __ldg(reinterpret_cast<const float4*>(p) + v);
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

template <int K>
__global__ void __launch_bounds__(128, RKETD_TB_MINB) k_tb2(const StepArgs<float> a) {
  constexpr int P = K / 2;
  const int lane = threadIdx.x & 31;
  const int tid = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (tid >= a.n_tiles) return;  // uniform per warp
  const Tile tl = a.tiles[tid];
  const int s = tl.slab;
  const int64_t base = a.soff[s] + tl.start + lane * K;  // interior tile: every cell is in the slab
  const int li0 = lane * K;

  f2 e[P], h[P], jj[P], da[P], ncb[P], dj[P], bp[P], cc[P];
  load_pairs<K>(a.E_in + base, e, false);
  load_pairs<K>(a.H_in + base, h, false);
  load_pairs<K>(a.J_in + base, jj, false);  // carries cj J~
  load_pairs<K>(a.coef[kDa] + base, da, false);
  load_pairs<K>(a.coef[kCb] + base, ncb, true);
  load_pairs<K>(a.coef[kDj] + base, dj, false);
  load_pairs<K>(a.coef[kBp] + base, bp, false);
  load_pairs<K>(a.coef[kCc] + base, cc, false);
  const f2 nS = pk(-a.S, -a.S);
  const bool has_src = tl.src_local >= 0 && lane == tl.src_local / K;
  const int src_slot = tl.src_local % K;
  const bool extras = tl.src_local >= 0 || tl.probe_count > 0;

  for (int t = 0; t < a.nsub; ++t) {
    // Eq. 14 on pairs: the cell after pair p is pair p+1; after pair P-1 it is (B[0], next lane's A[0])
    const float nextA0 = __shfl_down_sync(kFull, lo_of(e[0]), 1);
    const f2 eLast = pk(hi_of(e[0]), nextA0);
#pragma unroll
    for (int p = 0; p < P; ++p) {
      const f2 en = (p + 1 < P) ? e[p + 1] : eLast;
      h[p] = fma2(nS, sub2(en, e[p]), h[p]);
    }
    // Eqs. 13 + 11: the cell before pair p is pair p-1; before pair 0 it is (previous lane's B[P-1], A[P-1])
    const float prevB = __shfl_up_sync(kFull, hi_of(h[P - 1]), 1);
    const f2 hFirst = pk(prevB, lo_of(h[P - 1]));
#pragma unroll
    for (int p = 0; p < P; ++p) {
      const f2 hp = p ? h[p - 1] : hFirst;
      const f2 dH = sub2(h[p], hp);
      const f2 en = e[p];
      f2 enew = fma2(da[p], en, en);
      enew = fma2(ncb[p], dH, enew);
      enew = sub2(enew, jj[p]);
      f2 jn = fma2(dj[p], jj[p], jj[p]);
      jn = fma2(bp[p], en, jn);
      jn = fma2(cc[p], enew, jn);
      e[p] = enew;
      jj[p] = jn;
    }
    if (extras) {
      if (has_src) {
        const double sv = pulse((double)(a.n0 + t + 1) * a.dt, a.t0, a.tau, a.amp);
        put2(e, src_slot, pick2(e, src_slot) + (float)sv);
      }
      for (int q = 0; q < (a.series ? tl.probe_count : 0); ++q) {
        const TileProbe tp = a.tprobes[tl.probe_begin + q];
        if (lane == tp.local / K)
          a.series[(int64_t)tp.slot * a.series_len + a.series_pos + t] = pick2(e, tp.local % K);
      }
    }
  }
  store_pairs<K>(a.E_out + base, li0, tl.vlo, tl.vhi, e);
  store_pairs<K>(a.H_out + base, li0, tl.vlo, tl.vhi, h);
  store_pairs<K>(a.J_out + base, li0, tl.vlo, tl.vhi, jj);
}

}  // namespace

cudaError_t launch_tb_pairs(const StepArgs<float>& a, int K, int wpb, cudaStream_t st) {
  if (a.n_tiles <= 0) return cudaSuccess;
  if (wpb < 1 || wpb > 4) return cudaErrorInvalidValue;
  const dim3 block(32 * wpb);
  const dim3 grid((a.n_tiles + wpb - 1) / wpb);
  switch (K) {
    case 8: k_tb2<8><<<grid, block, 0, st>>>(a); break;
    case 12: k_tb2<12><<<grid, block, 0, st>>>(a); break;
    case 16: k_tb2<16><<<grid, block, 0, st>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace rketd
