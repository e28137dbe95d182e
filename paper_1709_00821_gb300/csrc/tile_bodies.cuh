// Bodies of the temporally blocked tile steps, one warp per tile: the scalar form (any precision,
// interior or edge tiles, window recording for the adjoint) and the packed FP32x2 interior form.
// The tiled kernels (step_tb.cu, step_tb2.cu) run one tile per warp and launch; the persistent
// batch step (step_persist.cu) runs many tiles of many passes per warp.
#pragma once

#include "rketd_internal.cuh"
#include "tile_common.cuh"

namespace rketd {
namespace tile {

// one value of state that the kernel may also write: a plain load (NC, the one-tile-per-launch
// kernels) or one from L2 (the persistent step, where other SMs write it between passes)
template <bool NC, typename T>
__device__ __forceinline__ T ldf(const T* p) {
  if constexpr (NC) return *p;
  else return __ldcg(p);
}

// The tiled step of one tile (step_tb.cu) for lane `lane` of the warp that owns it: interior or
// edge tile, optional window recording, optional probe/source code; n0 and spos and NC as for
// tb2_tile.
template <typename T, int K, bool EDGE, bool REC, bool XTRA, bool NC>
__device__ __forceinline__ void tb_tile(const StepArgs<T>& a, const Tile tl, int lane, int64_t n0, int spos) {
  const int s = tl.slab;
  const int64_t nz = a.nz[s];
  const int64_t soff = a.soff[s];
  const int64_t nzp = (nz + 31) & ~int64_t(31);  // storage extent of the slab
  const int li0 = lane * K;
  const int64_t g0 = tl.start + li0;  // slab-local cell of slot 0
  const T S = a.S;

  // jj carries the folded current G (rketd_internal.cuh): the E update subtracts it directly
  T e[K], h[K], jj[K], cb[K], dj[K], bq[K], cq[K];
  load_row<T, K, EDGE, NC>(a.E_in + soff, g0, nzp, e);
  load_row<T, K, EDGE, NC>(a.H_in + soff, g0, nzp, h);
  load_row<T, K, EDGE, NC>(a.J_in + soff, g0, nzp, jj);
  load_row<T, K, EDGE>(a.coef[kCb] + soff, g0, nzp, cb);
  load_row<T, K, EDGE>(a.coef[kDj] + soff, g0, nzp, dj);
  load_row<T, K, EDGE>(a.coef[kBq] + soff, g0, nzp, bq);
  load_row<T, K, EDGE>(a.coef[kCq] + soff, g0, nzp, cq);
  const bool has_src = XTRA && tl.src_local >= 0 && lane == tl.src_local / K;
  const LaneProbes lp = (XTRA && a.series)
                            ? lane_probes(a.tprobes, tl.probe_begin, tl.probe_count, lane, K, a.series_len, spos)
                            : LaneProbes{0, 0, 0, 0, 0};
  const bool tile_src = XTRA && tl.src_local >= 0;  // warp-uniform
  const PassSource<T> ps =
      tile_src ? pass_source<T>(n0, a.nsub, a.dt, a.t0, a.tau, a.amp, lane) : PassSource<T>{T(0), T(0)};

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
          if (a.bc == 1) pE[i] = ldf<NC>(a.psiE_in + pbase + (g < nc ? g : nc + (nz - 1 - g)));
        }
        if (hasH && (g < nc || g >= nz - 1 - nc)) {
          mcH |= 1u << i;
          if (a.bc == 1) pH[i] = ldf<NC>(a.psiH_in + pbase + (g < nc ? g : nc + (nz - 2 - g)));
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
            a.series[(int64_t)tp.slot * a.series_len + spos + t] = pick(e, tp.local % K);
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

// The interior tiled FP32 step of one tile (packed FP32x2 pairs; see step_tb2.cu), for lane
// `lane` of the warp that owns it: n0 is the step index at pass start, spos the pass's first
// column in the probe-series buffer. NC: fields through the read-only path (false in the
// persistent step, where other warps of the kernel write them).
//
// XTRA tiles may also hold a slab end (the planner's end tiles, first-order Mur ends): the tile
// that starts at cell 0, and the one whose last lane holds cell nz - 1 (in slot K - 4 .. K - 1,
// as the tile ends at round_up(nz, 4) - 1). They run the pair updates on every cell and then set
// the end cell's E by Mur's condition from the same values, in the same order and rounding, as the
// edge tiles (after the source, before the probes); the plain step never updates the end cells' G
// nor the H beyond cell nz - 2, so those are stored as loaded. The values the pair updates leave in
// the end cells and beyond nz - 1 reach no other cell: E there is overwritten every step, and G and
// H there feed only that E.
template <int K, bool XTRA, bool NC>
__device__ __forceinline__ void tb2_tile(const StepArgs<float>& a, const Tile tl, int lane, int64_t n0, int spos) {
  constexpr int P = K / 2;
  const int s = tl.slab;
  const int64_t base = a.soff[s] + tl.start + lane * K;  // interior tile: every cell is in the slab
  const int li0 = lane * K;

  f2 e[P], h[P], g[P], cb[P], dj[P], bq[P], cq[P];
  load_pairs<K, NC>(a.E_in + base, e, false);
  load_pairs<K, NC>(a.H_in + base, h, false);
  load_pairs<K, NC>(a.J_in + base, g, false);
  load_pairs<K>(a.coef[kCb] + base, cb, false);
  load_pairs<K>(a.coef[kDj] + base, dj, false);
  load_pairs<K>(a.coef[kBq] + base, bq, false);
  load_pairs<K>(a.coef[kCq] + base, cq, false);
  const f2 nS = pk(-a.S, -a.S);
  const bool has_src = XTRA && tl.src_local >= 0 && lane == tl.src_local / K;
  const int src_slot = tl.src_local % K;
  const LaneProbes lp = (XTRA && a.series)
                            ? lane_probes(a.tprobes, tl.probe_begin, tl.probe_count, lane, K, a.series_len, spos)
                            : LaneProbes{0, 0, 0, 0, 0};
  const bool tile_src = XTRA && tl.src_local >= 0;  // warp-uniform
  const PassSource<float> ps = tile_src ? pass_source<float>(n0, a.nsub, a.dt, a.t0, a.tau, a.amp, lane)
                                        : PassSource<float>{0.f, 0.f};
  // slab ends held (warp-uniform): cell 0 at lane 0, slot 0; cell nz - 1 at lane 31, slot sR
  bool endL = false;
  int sR = -1;
  float g0k = 0.f, gRk = 0.f, hRk = 0.f;  // their state that the step leaves as loaded
  if constexpr (XTRA) {
    endL = tl.start == 0;
    const int64_t r = a.nz[s] - 1 - tl.start - 31 * K;  // slot of cell nz - 1 in lane 31
    if (r >= K - 4 && r < K) sR = (int)r;
    if (endL) g0k = lo_of(g[0]);
    if (sR >= 0)
      at_uniform_slot<P>(sR, [&](auto S) {
        constexpr int q = decltype(S)::value;
        gRk = pick2c<q>(g);
        hRk = pick2c<q>(h);
      });
  }
  // the source cell's -da, which its fold into G takes every step
  const float nda = has_src ? -a.coef[kDa][base + src_slot] : 0.f;

#pragma unroll 2
  for (int t = 0; t < a.nsub; ++t) {
    // the end cells' E before this step (Mur's condition reads them)
    float e0o = 0.f, e1o = 0.f, eN1o = 0.f, eN2o = 0.f;
    if constexpr (XTRA) {
      if (endL) {
        e0o = lo_of(e[0]);
        e1o = lo_of(e[1]);
      }
      if (sR >= 0)
        at_uniform_slot<P>(sR, [&](auto S) {
          constexpr int q = decltype(S)::value;
          if constexpr (q >= 1) {
            eN1o = pick2c<q>(e);
            eN2o = pick2c<q - 1>(e);
          }
        });
    }
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
        if (has_src)
          at_uniform_slot<P>(src_slot, [&](auto S) {
            constexpr int q = decltype(S)::value;
            put2c<q>(e, pick2c<q>(e) + sv);
            put2c<q>(g, fmaf(nda, sv, pick2c<q>(g)));
          });
      }
      // first-order Mur ends
      if (endL && lane == 0) e[0] = pk(fmaf(a.qmur, lo_of(e[1]) - e0o, e1o), hi_of(e[0]));
      if (sR >= 0 && lane == 31)
        at_uniform_slot<P>(sR, [&](auto S) {
          constexpr int q = decltype(S)::value;
          if constexpr (q >= 1) put2c<q>(e, fmaf(a.qmur, pick2c<q - 1>(e) - eN1o, eN2o));
        });
      if (lp.n > 0) {
        a.series[lp.o0 + t] = pick2(e, lp.s0);
        if (lp.n > 1) {
          a.series[lp.o1 + t] = pick2(e, lp.s1);
          for (int q = 0, m = 0; lp.n > 2 && q < tl.probe_count; ++q) {
            const TileProbe tp = a.tprobes[tl.probe_begin + q];
            if (lane == tp.local / K && m++ >= 2)
              a.series[(int64_t)tp.slot * a.series_len + spos + t] = pick2(e, tp.local % K);
          }
        }
      }
    }
  }
  if constexpr (XTRA) {
    if (endL && lane == 0) g[0] = pk(g0k, hi_of(g[0]));
    if (sR >= 0 && lane == 31)
      at_uniform_slot<P>(sR, [&](auto S) {
        constexpr int q = decltype(S)::value;
        put2c<q>(g, gRk);
        put2c<q>(h, hRk);
      });
  }
  store_pairs<K>(a.E_out + base, li0, tl.vlo, tl.vhi, e);
  store_pairs<K>(a.H_out + base, li0, tl.vlo, tl.vhi, h);
  store_pairs<K>(a.J_out + base, li0, tl.vlo, tl.vhi, g);
}

}  // namespace tile
}  // namespace rketd
