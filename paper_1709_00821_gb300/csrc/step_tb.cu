// Temporally blocked 1D RKETD-FDTD step (Eqs. 14, 13, 11, 15, ends) on warp tiles.
//
// A warp owns 32*K consecutive cells of one slab, K per lane, kept in registers
// together with four per-cell update coefficients. One pass advances the tile by up
// to tb_steps leapfrog steps without leaving the registers: the only exchange between
// cells of different lanes is one shuffle per half step (E of the right neighbour for
// Eq. 14, H of the left neighbour for Eq. 12/13). A tile loads tb_steps cells of halo
// on each side; after t steps the outermost t cells of each side are stale, so the
// middle 32*K - 2*tb_steps cells are exact and are the only cells stored. Reads come from
// one copy of the fields and writes go to the other (ping-pong), so neighbouring tiles
// never see each other's writes within a pass.
//
// Two instantiations per (T, K): the interior kernel (every loaded cell is an interior
// cell of its slab, outside any CPML) carries no boundary code; the edge kernel handles
// cells outside the slab, the first-order Mur or PEC end cells and the CPML memories.
#include "rketd_internal.cuh"
#include "tile_common.cuh"

// Resident CTAs of 4 warps per SM the interior kernel is compiled for (register cap).
#ifndef RKETD_TB_MINB
#define RKETD_TB_MINB 3
#endif

namespace rketd {
namespace {

using namespace tile;

// XTRA: the tiles may sample a probe or hold their slab's source cell (always so for edge tiles
// and the recording recompute; the planner launches the few interior tiles that do apart from the
// rest, so that the main launch carries no per-step branch for them).
template <typename T, int K, bool EDGE, bool REC, bool XTRA>
__global__ void __launch_bounds__(128, EDGE ? 1 : RKETD_TB_MINB) k_tb(const StepArgs<T> a) {
  const int lane = threadIdx.x & 31;
  const int tid = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (tid >= a.n_tiles) return;  // uniform per warp
  const Tile tl = a.tiles[tid];
  const int s = tl.slab;
  const int64_t nz = a.nz[s];
  const int64_t soff = a.soff[s];
  const int64_t nzp = (nz + 31) & ~int64_t(31);  // storage extent of the slab
  const int li0 = lane * K;
  const int64_t g0 = tl.start + li0;  // slab-local cell of slot 0
  const T S = a.S;

  // jj carries the folded current G (rketd_internal.cuh): the E update subtracts it directly
  T e[K], h[K], jj[K], cb[K], dj[K], bq[K], cq[K];
  load_row<T, K, EDGE>(a.E_in + soff, g0, nzp, e);
  load_row<T, K, EDGE>(a.H_in + soff, g0, nzp, h);
  load_row<T, K, EDGE>(a.J_in + soff, g0, nzp, jj);
  load_row<T, K, EDGE>(a.coef[kCb] + soff, g0, nzp, cb);
  load_row<T, K, EDGE>(a.coef[kDj] + soff, g0, nzp, dj);
  load_row<T, K, EDGE>(a.coef[kBq] + soff, g0, nzp, bq);
  load_row<T, K, EDGE>(a.coef[kCq] + soff, g0, nzp, cq);
  const bool has_src = XTRA && tl.src_local >= 0 && lane == tl.src_local / K;
  const LaneProbes lp = (XTRA && a.series)
                            ? lane_probes(a.tprobes, tl.probe_begin, tl.probe_count, lane, K, a.series_len, a.series_pos)
                            : LaneProbes{0, 0, 0, 0, 0};
  const bool tile_src = XTRA && tl.src_local >= 0;  // warp-uniform
  const PassSource<T> ps =
      tile_src ? pass_source<T>(a.n0, a.nsub, a.dt, a.t0, a.tau, a.amp, lane) : PassSource<T>{T(0), T(0)};

  // Edge-tile bookkeeping (bit i = slot i).
  uint32_t mH = 0, mE = 0, mcH = 0, mcE = 0;
  T pE[EDGE ? K : 1], pH[EDGE ? K : 1];
  int i0 = -1, i1 = -1;  // slots of cells 0 and nz-1 in this lane
  const int nc = a.ncpml;
  const int64_t pbase = (int64_t)s * 2 * nc;
  if (EDGE) {
#pragma unroll
    for (int i = 0; i < K; ++i) {
      const int64_t g = g0 + i;
      const bool hasH = g >= 0 && g <= nz - 2;
      const bool intE = g >= 1 && g <= nz - 2;
      if (hasH) mH |= 1u << i;
      if (intE) mE |= 1u << i;
      pE[i] = T(0);
      pH[i] = T(0);
      if (a.bc >= 1) {  // CPML memories, or the split-field PML's nodes (no memory)
        if (intE && (g < nc || g > nz - 1 - nc)) {
          mcE |= 1u << i;
          if (a.bc == 1) pE[i] = a.psiE_in[pbase + (g < nc ? g : nc + (nz - 1 - g))];
        }
        if (hasH && (g < nc || g >= nz - 1 - nc)) {
          mcH |= 1u << i;
          if (a.bc == 1) pH[i] = a.psiH_in[pbase + (g < nc ? g : nc + (nz - 2 - g))];
        }
      }
      if (g == 0) i0 = i;
      if (g == nz - 1) i1 = i;
    }
  }

  // window cells this lane records (exact cells only): bit i = slot i
  uint32_t mrec = 0;
  if (REC) {
#pragma unroll
    for (int i = 0; i < K; ++i) {
      const int li = li0 + i;
      const int64_t g = g0 + i;
      if (li >= tl.vlo && li < tl.vhi && g >= a.rec_c0 && g < a.rec_c0 + a.rec_w) mrec |= 1u << i;
    }
  }

  for (int t = 0; t < a.nsub; ++t) {
    // ---- Eq. 14: H~_{k+1/2} -= S (E_{k+1} - E_k) (CPML: stretched difference + psi) ----
    const T eR = __shfl_down_sync(kFull, e[0], 1);
#pragma unroll
    for (int i = 0; i < K; ++i) {
      const T en = (i + 1 < K) ? e[i + 1] : eR;
      const T dE = en - e[i];
      if (!EDGE) {
        h[i] = fma(-S, dE, h[i]);
      } else if (mH & (1u << i)) {
        if (mcH & (1u << i)) {
          const int64_t g = g0 + i;
          const int ih = (int)(g < nc ? g : nz - 2 - g);
          if (a.bc == 2) {
            h[i] = pml_update(h[i], a.cpmlH[ih], a.cpmlH[nc + ih], dE);
          } else {
            const T db = a.cpmlH[ih], c = a.cpmlH[nc + ih], ki = a.cpmlH[2 * nc + ih];
            pH[i] = fma(db, pH[i], fma(c, dE, pH[i]));
            h[i] = fma(-S, fma(dE, ki, pH[i]), h[i]);
          }
        } else {
          h[i] = fma(-S, dE, h[i]);
        }
      }
    }
    // ---- Eqs. 13 + 11: E^{n+1} then J~^{n+1} ----
    const T hL = __shfl_up_sync(kFull, h[K - 1], 1);
    T e0o = T(0), e1o = T(0), eN1o = T(0), eN2o = T(0);
    if (EDGE) {
      const T eLo = __shfl_up_sync(kFull, e[K - 1], 1);
      if (i0 >= 0) {
        e0o = pick(e, i0);
        e1o = (i0 + 1 < K) ? pick(e, i0 + 1) : eR;
      }
      if (i1 >= 0) {
        eN1o = pick(e, i1);
        eN2o = (i1 > 0) ? pick(e, i1 - 1) : eLo;
      }
    }
#pragma unroll
    for (int i = 0; i < K; ++i) {
      const T hp = i ? h[i - 1] : hL;
      const T dH = h[i] - hp;
      T curl = dH;
      bool upd = true;
      if (EDGE) {
        upd = (mE >> i) & 1u;
        if (mcE & (1u << i)) {
          const int64_t g = g0 + i;
          const int d = (int)(g < nc ? g : nz - 1 - g);
          if (a.bc == 2) {  // split-field PML: vacuum, no current
            e[i] = pml_update(e[i], a.cpmlE[d], a.cpmlE[nc + 1 + d], dH);
            upd = false;
          } else {
            const T db = a.cpmlE[d], c = a.cpmlE[nc + 1 + d], ki = a.cpmlE[2 * (nc + 1) + d];
            pE[i] = fma(db, pE[i], fma(c, dH, pE[i]));
            curl = fma(dH, ki, pE[i]);
          }
        }
      }
      if (upd) {
        const T en = e[i];
        const T enew = fold_e(en, cb[i], curl, jj[i]);
        jj[i] = fold_g(jj[i], dj[i], bq[i], cq[i], en, enew);
        e[i] = enew;
      }
    }
    // ---- Eq. 15 soft source at t = (n+1) dt (and its fold into G) ----
    if (tile_src) {
      const T sv = source_at(ps, t);
      if (has_src) {
        const int sl = tl.src_local % K;
        put(e, sl, pick(e, sl) + sv);
        put(jj, sl, fma(-a.coef[kDa][soff + g0 + sl], sv, pick(jj, sl)));
      }
    }
    // ---- ends: first-order Mur or PEC ----
    if (EDGE) {
      const T eRn = __shfl_down_sync(kFull, e[0], 1);
      const T eLn = __shfl_up_sync(kFull, e[K - 1], 1);
      if (a.bc == 0) {
        if (i0 >= 0) {
          const T e1n = (i0 + 1 < K) ? pick(e, i0 + 1) : eRn;
          put(e, i0, fma(a.qmur, e1n - e0o, e1o));
        }
        if (i1 >= 0) {
          const T eN2n = (i1 > 0) ? pick(e, i1 - 1) : eLn;
          put(e, i1, fma(a.qmur, eN2n - eN1o, eN2o));
        }
      } else {
        if (i0 >= 0) put(e, i0, T(0));
        if (i1 >= 0) put(e, i1, T(0));
      }
    }
    // ---- probe samples (only the tile whose exact region holds the probe) ----
    if (XTRA && lp.n > 0) {
      a.series[lp.o0 + t] = pick(e, lp.s0);
      if (lp.n > 1) {
        a.series[lp.o1 + t] = pick(e, lp.s1);
        for (int p = 0, m = 0; lp.n > 2 && p < tl.probe_count; ++p) {
          const TileProbe tp = a.tprobes[tl.probe_begin + p];
          if (lane == tp.local / K && m++ >= 2)
            a.series[(int64_t)tp.slot * a.series_len + a.series_pos + t] = pick(e, tp.local % K);
        }
      }
    }
    // ---- window recording for the adjoint ----
    if (REC && mrec) {
      T* r = a.rec + ((int64_t)s * a.rec_len + a.rec_pos + t) * 3 * a.rec_w;
#pragma unroll
      for (int v = 0; v < K / 4; ++v) {
        const uint32_t m4 = (mrec >> (4 * v)) & 0xFu;
        const int64_t c = g0 + 4 * v - a.rec_c0;
        if (m4 == 0xFu && (c & 3) == 0) {  // whole aligned group: vector stores
          st4(r + c, &e[4 * v]);
          st4(r + a.rec_w + c, &h[4 * v]);
          st4(r + 2 * a.rec_w + c, &jj[4 * v]);
        } else if (m4) {
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            if (m4 & (1u << q)) {
              r[c + q] = e[4 * v + q];
              r[a.rec_w + c + q] = h[4 * v + q];
              r[2 * a.rec_w + c + q] = jj[4 * v + q];
            }
          }
        }
      }
    }
  }

  store_row<T, K>(a.E_out + soff, g0, li0, tl.vlo, tl.vhi, e);
  store_row<T, K>(a.H_out + soff, g0, li0, tl.vlo, tl.vhi, h);
  store_row<T, K>(a.J_out + soff, g0, li0, tl.vlo, tl.vhi, jj);
  if (EDGE && a.bc == 1) {
#pragma unroll
    for (int i = 0; i < K; ++i) {
      const int li = li0 + i;
      if (li < tl.vlo || li >= tl.vhi) continue;
      const int64_t g = g0 + i;
      if (mcE & (1u << i)) a.psiE_out[pbase + (g < nc ? g : nc + (nz - 1 - g))] = pE[i];
      if (mcH & (1u << i)) a.psiH_out[pbase + (g < nc ? g : nc + (nz - 2 - g))] = pH[i];
    }
  }
}

template <typename T, int K, bool REC = false>
cudaError_t launch_k(const StepArgs<T>& a, bool edge, int wpb, cudaStream_t st, bool xtra) {
  const dim3 block(32 * wpb);
  const dim3 grid((a.n_tiles + wpb - 1) / wpb);
  if (edge)
    k_tb<T, K, true, REC, true><<<grid, block, 0, st>>>(a);
  else if (REC || xtra)
    k_tb<T, K, false, REC, true><<<grid, block, 0, st>>>(a);
  else
    k_tb<T, K, false, false, false><<<grid, block, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace

template <>
cudaError_t launch_tb<float>(const StepArgs<float>& a, int K, bool edge, int wpb, cudaStream_t st, bool xtra) {
  if (a.n_tiles <= 0) return cudaSuccess;
  if (wpb < 1 || wpb > 4) return cudaErrorInvalidValue;
  switch (K) {
    case 4: return launch_k<float, 4>(a, edge, wpb, st, xtra);
    case 8: return launch_k<float, 8>(a, edge, wpb, st, xtra);
    case 12: return launch_k<float, 12>(a, edge, wpb, st, xtra);
    case 16: return launch_k<float, 16>(a, edge, wpb, st, xtra);
    default: return cudaErrorInvalidValue;
  }
}

template <>
cudaError_t launch_tb<double>(const StepArgs<double>& a, int K, bool edge, int wpb, cudaStream_t st, bool xtra) {
  if (a.n_tiles <= 0) return cudaSuccess;
  if (wpb < 1 || wpb > 4) return cudaErrorInvalidValue;
  switch (K) {
    case 4: return launch_k<double, 4>(a, edge, wpb, st, xtra);
    case 8: return launch_k<double, 8>(a, edge, wpb, st, xtra);
    default: return cudaErrorInvalidValue;
  }
}

template <>
cudaError_t launch_tb_rec<float>(const StepArgs<float>& a, int K, bool edge, int wpb, cudaStream_t st) {
  if (a.n_tiles <= 0) return cudaSuccess;
  if (wpb < 1 || wpb > 4) return cudaErrorInvalidValue;
  switch (K) {
    case 4: return launch_k<float, 4, true>(a, edge, wpb, st, true);
    case 8: return launch_k<float, 8, true>(a, edge, wpb, st, true);
    case 16: return launch_k<float, 16, true>(a, edge, wpb, st, true);
    default: return cudaErrorInvalidValue;
  }
}

template <>
cudaError_t launch_tb_rec<double>(const StepArgs<double>& a, int K, bool edge, int wpb, cudaStream_t st) {
  if (a.n_tiles <= 0) return cudaSuccess;
  if (wpb < 1 || wpb > 4) return cudaErrorInvalidValue;
  switch (K) {
    case 4: return launch_k<double, 4, true>(a, edge, wpb, st, true);
    case 8: return launch_k<double, 8, true>(a, edge, wpb, st, true);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace rketd
