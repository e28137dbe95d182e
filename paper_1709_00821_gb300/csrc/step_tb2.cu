// Interior tiled step for FP32 fields with two cells per packed FP32x2 register.
//
// Same tile, halo and arithmetic as k_tb<float, K, interior> (step_tb.cu), but each lane's K
// cells are split into halves A = [0, K/2) and B = [K/2, K) and cell A[p] shares a 64-bit
// register with cell B[p]. Shifting by one cell then maps pair p to pair p-1 (or p+1) for
// both halves at once, so every update is one add/sub/fma.rn.f32x2 per pair: half the issue
// slots of the scalar kernel for the same FP32 work (the kernel is issue-bound: the FP32
// pipe runs the pair in two cycles either way). Only the two pairs at the ends of a lane's
// range need a repack per half step. Every element is rounded exactly as in the scalar
// kernel (fma2 is two fused multiply-adds, sub2 two subtractions, and so on), so the fields
// are bitwise identical to the plain and scalar tiled kernels. The current is the folded
// G of rketd_internal.cuh, updated as fold_e / fold_g do.
#include "rketd_internal.cuh"
#include "tile_common.cuh"

#ifndef RKETD_TB_MINB
#define RKETD_TB_MINB 3
#endif

namespace rketd {
namespace {

using namespace tile;
// XTRA: the tile list holds the tiles that sample a probe or whose loaded range contains their
// slab's source cell (the planner launches those few apart, so that the main launch carries no
// per-step branch for them).
template <int K, bool XTRA>
__global__ void __launch_bounds__(128, RKETD_TB_MINB) k_tb2(const StepArgs<float> a) {
  constexpr int P = K / 2;
  const int lane = threadIdx.x & 31;
  const int tid = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (tid >= a.n_tiles) return;  // uniform per warp
  const Tile tl = a.tiles[tid];
  const int s = tl.slab;
  const int64_t base = a.soff[s] + tl.start + lane * K;  // interior tile: every cell is in the slab
  const int li0 = lane * K;

  f2 e[P], h[P], g[P], cb[P], dj[P], bq[P], cq[P];
  load_pairs<K>(a.E_in + base, e, false);
  load_pairs<K>(a.H_in + base, h, false);
  load_pairs<K>(a.J_in + base, g, false);
  load_pairs<K>(a.coef[kCb] + base, cb, false);
  load_pairs<K>(a.coef[kDj] + base, dj, false);
  load_pairs<K>(a.coef[kBq] + base, bq, false);
  load_pairs<K>(a.coef[kCq] + base, cq, false);
  const f2 nS = pk(-a.S, -a.S);
  const bool has_src = XTRA && tl.src_local >= 0 && lane == tl.src_local / K;
  const int src_slot = tl.src_local % K;
  const LaneProbes lp = (XTRA && a.series)
                            ? lane_probes(a.tprobes, tl.probe_begin, tl.probe_count, lane, K, a.series_len, a.series_pos)
                            : LaneProbes{0, 0, 0, 0, 0};
  const bool tile_src = XTRA && tl.src_local >= 0;  // warp-uniform
  const PassSource<float> ps = tile_src ? pass_source<float>(a.n0, a.nsub, a.dt, a.t0, a.tau, a.amp, lane)
                                        : PassSource<float>{0.f, 0.f};

#pragma unroll 2
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
      const f2 enew = sub2(en, fma2(cb[p], dH, g[p]));
      g[p] = add2(g[p], fma2(cq[p], enew, fma2(bq[p], en, mul2(dj[p], g[p]))));
      e[p] = enew;
    }
    if constexpr (XTRA) {
      if (tile_src) {
        const float sv = source_at(ps, t);
        if (has_src) {
          put2(e, src_slot, pick2(e, src_slot) + sv);
          put2(g, src_slot, fmaf(-a.coef[kDa][base + src_slot], sv, pick2(g, src_slot)));
        }
      }
      if (lp.n > 0) {
        a.series[lp.o0 + t] = pick2(e, lp.s0);
        if (lp.n > 1) {
          a.series[lp.o1 + t] = pick2(e, lp.s1);
          for (int q = 0, m = 0; lp.n > 2 && q < tl.probe_count; ++q) {
            const TileProbe tp = a.tprobes[tl.probe_begin + q];
            if (lane == tp.local / K && m++ >= 2)
              a.series[(int64_t)tp.slot * a.series_len + a.series_pos + t] = pick2(e, tp.local % K);
          }
        }
      }
    }
  }
  store_pairs<K>(a.E_out + base, li0, tl.vlo, tl.vhi, e);
  store_pairs<K>(a.H_out + base, li0, tl.vlo, tl.vhi, h);
  store_pairs<K>(a.J_out + base, li0, tl.vlo, tl.vhi, g);
}

}  // namespace

cudaError_t launch_tb_pairs(const StepArgs<float>& a, int K, int wpb, cudaStream_t st, bool xtra) {
  if (a.n_tiles <= 0) return cudaSuccess;
  if (wpb < 1 || wpb > 4) return cudaErrorInvalidValue;
  const dim3 block(32 * wpb);
  const dim3 grid((a.n_tiles + wpb - 1) / wpb);
  switch (K) {
    case 8: xtra ? k_tb2<8, true><<<grid, block, 0, st>>>(a) : k_tb2<8, false><<<grid, block, 0, st>>>(a); break;
    case 12: xtra ? k_tb2<12, true><<<grid, block, 0, st>>>(a) : k_tb2<12, false><<<grid, block, 0, st>>>(a); break;
    case 16: xtra ? k_tb2<16, true><<<grid, block, 0, st>>>(a) : k_tb2<16, false><<<grid, block, 0, st>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace rketd
