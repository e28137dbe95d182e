// Resident 1D step: a whole slab lives in the registers of one thread-block cluster for a whole
// block of steps (Eqs. 14, 13, 11, 15, first-order Mur ends, probe samples), one launch per
// DFT block.
//
// The tiled kernels reload a slab from HBM every few steps; for a short slab (the paper's own
// problem: 2000 cells) that makes every step pay a launch and a load, and a few warps carry the
// whole run's latency. Here thread g of the cluster owns slab cells g K - pl .. g K - pl + K - 1
// for the whole launch. Cells cross a thread boundary only through one value each way per step:
//   - to the left neighbour thread: its first E (for the neighbour's last H update, Eq. 14);
//   - to the right neighbour thread: its last E and last H (the right neighbour recomputes that
//     H^{n+1/2} itself, with the same operations as its owner, so that its first E update
//     (Eq. 13) needs no second exchange).
// Inside a warp these go by shuffles; between warps and between the CTAs of the cluster, through
// double-buffered slots in the receiving warp's shared memory (distributed shared memory across
// CTAs), written before and read after one cluster barrier per step. The double buffer makes one
// barrier enough: a warp cannot write a slot again before every reader has passed the next barrier.
//
// The left padding pl (0 or 1) keeps cells 0, 1 and cells nz-2, nz-1 in one warp each, so the Mur
// ends need only shuffles. FP64 runs one warp per SM sub-partition (the FP64 units of this part are
// few per sub-partition, so the cells are spread over up to 16 SMs of the cluster); FP32 fits a
// slab of a few thousand cells in one CTA.
#include <cooperative_groups.h>

#include <type_traits>

#include "rketd_internal.cuh"
#include "tile_common.cuh"

namespace cg = cooperative_groups;

namespace rketd {
namespace {

using namespace tile;

constexpr int kResMaxWarps = 32;

// CL: the slab spans a cluster of several CTAs (distributed shared memory and a cluster barrier);
// otherwise one CTA (its own shared memory and a CTA barrier).
template <typename T, int K, int MAXT, bool CL>
__global__ void __launch_bounds__(MAXT) k_res(const StepArgs<T> a, int pl) {
  __shared__ T fromR[2][kResMaxWarps];     // E of the cell after the warp's last cell
  __shared__ T fromL[2][2][kResMaxWarps];  // E and H of the cell before the warp's first cell
  const int lane = threadIdx.x & 31, lw = threadIdx.x >> 5, NW = blockDim.x >> 5;
  const int rank = (int)blockIdx.x;  // the grid is one cluster
  const int NC = (int)gridDim.x;
  const int64_t gth = (int64_t)rank * blockDim.x + threadIdx.x;
  const int64_t c0 = gth * K - pl;  // slab cell of slot 0
  const int64_t nz = a.nz[0];
  const T S = a.S;

  T e[K], h[K], g[K], cb[K], dj[K], bq[K], cq[K];
  uint32_t mH = 0, mE = 0;
#pragma unroll
  for (int i = 0; i < K; ++i) {
    const int64_t c = c0 + i;
    const bool in = c >= 0 && c < nz;
    e[i] = in ? a.E_in[c] : T(0);
    h[i] = in ? a.H_in[c] : T(0);
    g[i] = in ? a.J_in[c] : T(0);
    cb[i] = in ? a.coef[kCb][c] : T(0);
    dj[i] = in ? a.coef[kDj][c] : T(0);
    bq[i] = in ? a.coef[kBq][c] : T(0);
    cq[i] = in ? a.coef[kCq][c] : T(0);
    if (c >= 0 && c <= nz - 2) mH |= 1u << i;
    if (c >= 1 && c <= nz - 2) mE |= 1u << i;
  }
  // ends (their pair partners are in this warp by the choice of pl)
  const int i0 = (c0 <= 0 && 0 < c0 + K) ? (int)(-c0) : -1;           // slot of cell 0
  const int i1 = (c0 <= nz - 1 && nz - 1 < c0 + K) ? (int)(nz - 1 - c0) : -1;  // slot of cell nz-1
  // source
  const int64_t src = a.src[0];
  const int is = (c0 <= src && src < c0 + K) ? (int)(src - c0) : -1;
  const T da_src = is >= 0 ? a.coef[kDa][src] : T(0);
  const bool src_warp = __any_sync(kFull, is >= 0);
  const bool end_warp = __any_sync(kFull, i0 >= 0 || i1 >= 0);
  // probes among this thread's cells (tprobes: local = slab cell, slot = probe index)
  int np = 0, ps0 = 0, ps1 = 0;
  int64_t po0 = 0, po1 = 0;
  for (int q = 0; q < a.total_probes; ++q) {
    const TileProbe p = a.tprobes[q];
    if (p.local < c0 || p.local >= c0 + K) continue;
    const int64_t o = (int64_t)p.slot * a.series_len + a.series_pos;
    if (np == 0) {
      ps0 = (int)(p.local - c0);
      po0 = o;
    } else {
      ps1 = (int)(p.local - c0);
      po1 = o;
    }
    ++np;
  }
  // neighbour warps: the receiving slots of the warp before and after this one
  const int64_t gw = gth >> 5, nwarps = (int64_t)NC * NW;
  const bool has_left = gw > 0, has_right = gw + 1 < nwarps;
  const int l_rank = lw > 0 ? rank : rank - 1, l_idx = lw > 0 ? lw - 1 : NW - 1;
  const int r_rank = lw + 1 < NW ? rank : rank + 1, r_idx = lw + 1 < NW ? lw + 1 : 0;

  T sv_lane = T(0);
  for (int t = 0; t < a.nsub; ++t) {
    const int b = t & 1;
    if (src_warp && (t & 31) == 0) {
      const int r = t + lane;
      sv_lane = r < a.nsub ? (T)pulse((double)(a.n0 + 1 + r) * a.dt, a.t0, a.tau, a.amp) : T(0);
    }
    // ---- exchange: first E to the left, last E and H to the right ----
    if constexpr (CL) {
      cg::cluster_group cl = cg::this_cluster();
      if (lane == 0 && has_left) *cl.map_shared_rank(&fromR[b][l_idx], l_rank) = e[0];
      if (lane == 31 && has_right) {
        *cl.map_shared_rank(&fromL[b][0][r_idx], r_rank) = e[K - 1];
        *cl.map_shared_rank(&fromL[b][1][r_idx], r_rank) = h[K - 1];
      }
    } else {
      if (lane == 0 && has_left) fromR[b][l_idx] = e[0];
      if (lane == 31 && has_right) {
        fromL[b][0][r_idx] = e[K - 1];
        fromL[b][1][r_idx] = h[K - 1];
      }
    }
    T eR = __shfl_down_sync(kFull, e[0], 1);
    T eL = __shfl_up_sync(kFull, e[K - 1], 1);
    T hLo = __shfl_up_sync(kFull, h[K - 1], 1);
    if constexpr (CL)
      cg::this_cluster().sync();
    else
      __syncthreads();
    if (lane == 31) eR = has_right ? fromR[b][lw] : T(0);
    if (lane == 0) {
      eL = has_left ? fromL[b][0][lw] : T(0);
      hLo = has_left ? fromL[b][1][lw] : T(0);
    }
    // ---- Eq. 14 (and the left neighbour's last H, by the same operations) ----
#pragma unroll
    for (int i = 0; i < K; ++i) {
      const T en = (i + 1 < K) ? e[i + 1] : eR;
      if (mH & (1u << i)) h[i] = fma(-S, en - e[i], h[i]);
    }
    const T hL = fma(-S, e[0] - eL, hLo);
    // ---- Eqs. 13 + 11 on the folded current (the end cells' old E kept for Mur) ----
    T e0o = T(0), e1o = T(0), eN1o = T(0), eN2o = T(0);
    if (end_warp) {
      if (i0 >= 0) {
        e0o = pick(e, i0);
        e1o = i0 + 1 < K ? pick(e, i0 + 1) : eR;
      }
      if (i1 >= 0) {
        eN1o = pick(e, i1);
        eN2o = i1 > 0 ? pick(e, i1 - 1) : eL;
      }
    }
#pragma unroll
    for (int i = 0; i < K; ++i) {
      const T hp = i ? h[i - 1] : hL;
      if (mE & (1u << i)) {
        const T enew = fold_e(e[i], cb[i], h[i] - hp, g[i]);
        g[i] = fold_g(g[i], dj[i], bq[i], cq[i], e[i], enew);
        e[i] = enew;
      }
    }
    // ---- Eq. 15 soft source and its fold into G ----
    if (src_warp) {
      const T sv = __shfl_sync(kFull, sv_lane, t & 31);
      if (is >= 0) {
        put(e, is, pick(e, is) + sv);
        put(g, is, fma(-da_src, sv, pick(g, is)));
      }
    }
    // ---- first-order Mur ends (partners by shuffle within the warp) ----
    if (end_warp) {
      const T nextNew = __shfl_down_sync(kFull, e[0], 1);
      const T prevNew = __shfl_up_sync(kFull, e[K - 1], 1);
      if (i0 >= 0) {
        const T e1n = i0 + 1 < K ? pick(e, i0 + 1) : nextNew;
        put(e, i0, fma(a.qmur, e1n - e0o, e1o));
      }
      if (i1 >= 0) {
        const T eN2n = i1 > 0 ? pick(e, i1 - 1) : prevNew;
        put(e, i1, fma(a.qmur, eN2n - eN1o, eN2o));
      }
    }
    // ---- probe samples ----
    if (np > 0) {
      a.series[po0 + t] = pick(e, ps0);
      if (np > 1) a.series[po1 + t] = pick(e, ps1);
      for (int q = 0, m = 0; np > 2 && q < a.total_probes; ++q) {  // rare: more probes in one thread
        const TileProbe p = a.tprobes[q];
        if (p.local >= c0 && p.local < c0 + K && m++ >= 2)
          a.series[(int64_t)p.slot * a.series_len + a.series_pos + t] = pick(e, (int)(p.local - c0));
      }
    }
  }
#pragma unroll
  for (int i = 0; i < K; ++i) {
    const int64_t c = c0 + i;
    if (c >= 0 && c < nz) {
      a.E_out[c] = e[i];
      a.H_out[c] = h[i];
      a.J_out[c] = g[i];
    }
  }
}

template <typename T, int K, int MAXT>
cudaError_t launch_k(const StepArgs<T>& a, int ctas, int threads, int pl, cudaStream_t st, bool query_only,
                     int* max_clusters) {
  if (threads > MAXT || threads % 32 || threads / 32 > kResMaxWarps) return cudaErrorInvalidValue;
  if (ctas == 1) {
    auto f1 = k_res<T, K, MAXT, false>;
    if (query_only) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(max_clusters, f1, threads, 0);
    f1<<<1, threads, 0, st>>>(a, pl);
    return cudaGetLastError();
  }
  auto fn = k_res<T, K, MAXT, true>;
  if (ctas > 8) {
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(ctas);
  cfg.blockDim = dim3(threads);
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = ctas;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  if (query_only) return cudaOccupancyMaxActiveClusters(max_clusters, fn, &cfg);
  return cudaLaunchKernelEx(&cfg, fn, a, pl);
}

}  // namespace

// K = cells per thread; query_only: report in *max_clusters how many such clusters fit at once
// (0: the shape cannot run) instead of launching.
template <typename T>
cudaError_t launch_resident(const StepArgs<T>& a, int K, int ctas, int threads, int pl, cudaStream_t st,
                            bool query_only, int* max_clusters) {
  if (ctas < 1 || ctas > 16) return cudaErrorInvalidValue;
  if constexpr (std::is_same<T, double>::value) {
    switch (K) {
      case 1: return launch_k<T, 1, 256>(a, ctas, threads, pl, st, query_only, max_clusters);
      case 2: return launch_k<T, 2, 256>(a, ctas, threads, pl, st, query_only, max_clusters);
      case 4: return launch_k<T, 4, 256>(a, ctas, threads, pl, st, query_only, max_clusters);
      case 8: return launch_k<T, 8, 128>(a, ctas, threads, pl, st, query_only, max_clusters);
      default: return cudaErrorInvalidValue;
    }
  } else {
  switch (K) {
    case 2: return launch_k<T, 2, 1024>(a, ctas, threads, pl, st, query_only, max_clusters);
    case 4: return launch_k<T, 4, 512>(a, ctas, threads, pl, st, query_only, max_clusters);
    case 8: return launch_k<T, 8, 256>(a, ctas, threads, pl, st, query_only, max_clusters);
    case 16: return launch_k<T, 16, 128>(a, ctas, threads, pl, st, query_only, max_clusters);
    default: return cudaErrorInvalidValue;
  }
  }
}
template cudaError_t launch_resident<float>(const StepArgs<float>&, int, int, int, int, cudaStream_t, bool, int*);
template cudaError_t launch_resident<double>(const StepArgs<double>&, int, int, int, int, cudaStream_t, bool, int*);

}  // namespace rketd
