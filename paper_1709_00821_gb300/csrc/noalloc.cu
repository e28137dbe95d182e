// rketd_advance_1d_noalloc: the temporally blocked single-slab step with all of its
// working memory in one fixed device array, for callers that cannot allocate device memory.
//
// Who needs it: code that runs where cudaMalloc is not allowed or not wanted -- a framework
// whose caching allocator owns the whole GPU and forbids allocations behind its back, or a
// real-time loop that cannot afford the device-wide synchronisation that cudaMalloc/cudaFree
// imply. Such callers pass their own input and output arrays; everything else the step needs
// (the per-cell update coefficients, two working copies of the fields for the ping-pong passes,
// the tile list) lives in g_noalloc_scratch below.
//
// The array is a file-scope __device__ variable, so every GPU that loads this library holds
// it (kNoallocScratchBytes) until the process exits, whether or not the entry point is used.
// All calls share it and it keeps what the last call left there, so each call rewrites every
// part it reads before reading it; two calls whose work overlaps on the GPU (different streams,
// or different host threads) would race on it and must be serialised by the caller.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "../../include/rketd.h"
#include "rketd_internal.cuh"

// Largest slab (E nodes) the fixed scratch array holds.
#ifndef RKETD_NOALLOC_MAX_NZ
#define RKETD_NOALLOC_MAX_NZ 131072
#endif

namespace rketd {
namespace {

constexpr int64_t kNoallocMaxNz = RKETD_NOALLOC_MAX_NZ;
constexpr int kNoallocMaxTiles = 4096;
constexpr int64_t kNoallocPad = ((kNoallocMaxNz + 31) / 32) * 32;
// 6 coefficient arrays + 2 x (E, H, J) in FP64, the tile list and a small slab table
constexpr size_t kNoallocScratchBytes =
    12 * kNoallocPad * sizeof(double) + kNoallocMaxTiles * sizeof(Tile) + 1024;

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

std::mutex g_setup_mutex;
void* g_scratch_addr[64] = {};  // device address of g_noalloc_scratch per device ordinal

rketd_status nfail(rketd_status st, const char* msg) {
  set_error_message(msg);
  return st;
}

// The tiling of one slab: interior tiles of K cells per lane cover [a, b) (W = 32K - 2T exact cells
// each, loaded range inside the guard cells [1, nz - 2]), narrow edge tiles of Ke cells per lane
// cover [0, a) and [b, nz). Computed once on the host; k_plan writes the same tiles on the device.
struct NoallocPlan {
  int64_t a = 0, n_int = 0, b = 0, n_edge = 0;
  int64_t j_src0 = 0, j_src1 = 0;  // interior tiles whose loaded range holds the source cell
};

// Tile shapes of the entry point (the tiled step's defaults): cells per lane and steps per pass.
constexpr int noalloc_K(bool f64) { return f64 ? 8 : 16; }
constexpr int noalloc_T(bool f64) { return f64 ? 4 : 32; }

NoallocPlan noalloc_plan(int64_t nz, int64_t src, int K, int Ke, int T) {
  NoallocPlan p;
  const int64_t L = 32 * K, W = L - 2 * T, We = 32 * Ke - 2 * T;
  const int64_t hi_guard = nz - 2;
  p.a = ((1 + T + 3) / 4) * 4;
  if (p.a - T + L - 1 <= hi_guard) p.n_int = (hi_guard - (p.a - T + L - 1)) / W + 1;
  if (p.n_int == 0) p.a = 0;
  p.b = p.a + p.n_int * W;
  p.n_edge = (p.a + We - 1) / We + (nz - p.b + We - 1) / We;
  // tile j loads [a + jW - T, a + jW - T + L): it holds src when d - L < jW <= d, d = src - a + T
  const int64_t d = src - p.a + T;
  if (p.n_int && d >= 0) {
    p.j_src0 = d - L + 1 > 0 ? (d - L + 1 + W - 1) / W : 0;
    p.j_src1 = std::min<int64_t>(p.n_int, d / W + 1);
    if (p.j_src1 < p.j_src0) p.j_src1 = p.j_src0;
  }
  return p;
}

// One tile loading [v0 - T, v0 - T + Lt) and holding [v0, v1) exactly.
__host__ __device__ inline Tile noalloc_tile(int64_t v0, int64_t v1, int Lt, int T, int64_t src) {
  Tile t;
  t.slab = 0;
  t.start = v0 - T;
  t.vlo = T;
  t.vhi = (int32_t)(T + (v1 - v0));
  const int64_t sl = src - t.start;
  t.src_local = (sl >= 0 && sl < Lt) ? (int32_t)sl : -1;
  t.probe_begin = 0;
  t.probe_count = 0;
  t.adj_begin = 0;
  t.adj_count = 0;
  return t;
}

// The tile list of a NoallocPlan in launch order: interior tiles without the source, then those
// with it, then the edge tiles. Returns the count. The device writes it (k_plan), and
// rketd_noalloc_tiles_1d hands the same list to the host for checking.
__host__ __device__ inline int noalloc_tiles(const NoallocPlan& pl, int64_t nz, int64_t src, int K, int Ke, int T,
                                             Tile* tiles) {
  const int L = 32 * K, W = L - 2 * T, Le = 32 * Ke, We = Le - 2 * T;
  int n = 0;
  for (int64_t j = 0; j < pl.n_int; ++j)
    if (j < pl.j_src0 || j >= pl.j_src1) tiles[n++] = noalloc_tile(pl.a + j * W, pl.a + (j + 1) * W, L, T, src);
  for (int64_t j = pl.j_src0; j < pl.j_src1; ++j)
    tiles[n++] = noalloc_tile(pl.a + j * W, pl.a + (j + 1) * W, L, T, src);
  for (int64_t v = 0; v < pl.a; v += We) tiles[n++] = noalloc_tile(v, v + We < pl.a ? v + We : pl.a, Le, T, src);
  for (int64_t v = pl.b; v < nz; v += We) tiles[n++] = noalloc_tile(v, v + We < nz ? v + We : nz, Le, T, src);
  return n;
}

// Writes the tile list and the slab table (soff = 0, off = 0, nz, src). One thread.
__global__ void k_plan(Tile* tiles, int64_t* table, int64_t nz, int64_t src, int K, int Ke, int T, NoallocPlan pl) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  table[0] = 0;
  table[1] = 0;
  table[2] = nz;
  table[3] = src;
  noalloc_tiles(pl, nz, src, K, Ke, T, tiles);
}

// Caller's SI fields -> normalised working copy (E~ = E, H~ = eta0 H, folded current
// G = cj (dt/eps0) J - da E), with the padding cells zeroed; and back.
template <typename T>
__global__ void k_in(const T* E, const T* H, const T* J, const T* cj, const T* da, T* Es, T* Hs, T* Js, int64_t nz,
                     int64_t nzp, double hs, double js) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= nzp) return;
  Es[k] = k < nz ? E[k] : T(0);
  Hs[k] = k < nz - 1 ? (T)((double)H[k] * hs) : T(0);
  Js[k] = k < nz ? (T)((double)J[k] * js * (double)cj[k] - (double)da[k] * (double)E[k]) : T(0);
}

template <typename T>
__global__ void k_out(const T* Es, const T* Hs, const T* Js, const T* cj, const T* da, T* E, T* H, T* J, int64_t nz,
                      double hs, double js) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= nz) return;
  E[k] = Es[k];
  if (k < nz - 1) H[k] = (T)((double)Hs[k] * hs);
  J[k] = (T)(((double)Js[k] + (double)da[k] * (double)Es[k]) / (double)cj[k] * js);
}

template <typename T>
rketd_status advance(void* base, const rketd_grid1d* g, int64_t nz, const double* wp2, const double* nu,
                     int64_t src, const rketd_pulse* p, int64_t n0, int64_t nsteps, T* E, T* H, T* J,
                     cudaStream_t st) {
  const int64_t nzp = ((nz + 31) / 32) * 32;
  unsigned char* q = (unsigned char*)base;
  T* coef[kNumCoef];
  for (int k = 0; k < kNumCoef; ++k) coef[k] = (T*)(q + (size_t)k * kNoallocPad * sizeof(double));
  T* fld[2][3];
  for (int b = 0; b < 2; ++b)
    for (int f = 0; f < 3; ++f) fld[b][f] = (T*)(q + (size_t)(6 + 3 * b + f) * kNoallocPad * sizeof(double));
  Tile* tiles = (Tile*)(q + 12 * kNoallocPad * sizeof(double));
  int64_t* table = (int64_t*)(tiles + kNoallocMaxTiles);

  const int K = noalloc_K(sizeof(T) == 8), TS = noalloc_T(sizeof(T) == 8), Ke = 4;
  const double S = g->dt / (g->dz * std::sqrt(kMu0 * kEps0));
  const double eta0 = std::sqrt(kMu0 / kEps0);
  const NoallocPlan pl = noalloc_plan(nz, src, K, Ke, TS);
  const int64_t n_int = pl.n_int, n_edge = pl.n_edge, n_src = pl.j_src1 - pl.j_src0;
  if (n_int + n_edge > kNoallocMaxTiles) return nfail(RKETD_EINVAL, "noalloc: too many tiles");

  cudaError_t e;
  k_plan<<<1, 32, 0, st>>>(tiles, table, nz, src, K, Ke, TS, pl);
  if ((e = cudaGetLastError()) != cudaSuccess) return nfail(RKETD_ECUDA, cudaGetErrorString(e));
  void* cptr[kNumCoef];
  for (int k = 0; k < kNumCoef; ++k) cptr[k] = coef[k];
  // table layout: soff[0] = 0, off[0] = 0, nz[0], src[0]
  e = launch_coeffs(sizeof(T) == 8 ? 1 : 0, wp2, nu, table, table + 1, table + 2, 1, nzp, g->dt, S, cptr, st,
                    g->scheme);
  if (e != cudaSuccess) return nfail(RKETD_ECUDA, cudaGetErrorString(e));
  const unsigned blocks = (unsigned)((nzp + 255) / 256);
  k_in<T><<<blocks, 256, 0, st>>>(E, H, J, coef[kCj], coef[kDa], fld[0][0], fld[0][1], fld[0][2], nz, nzp, eta0,
                                  g->dt / kEps0);
  if ((e = cudaGetLastError()) != cudaSuccess) return nfail(RKETD_ECUDA, cudaGetErrorString(e));

  StepArgs<T> s{};
  for (int k = 0; k < kNumCoef; ++k) s.coef[k] = coef[k];
  s.soff = table;
  s.nz = table + 2;
  s.src = table + 3;
  s.bc = 0;
  s.ncpml = 0;
  s.S = (T)S;
  s.qmur = (T)((S - 1.0) / (S + 1.0));
  s.dt = g->dt;
  s.tau = p->tau;
  s.t0 = p->t0;
  s.amp = p->amp;
  s.series = nullptr;
  s.series_len = 1;
  s.tprobes = nullptr;
  int cur = 0;
  for (int64_t done = 0; done < nsteps;) {
    const int nsub = (int)(nsteps - done < TS ? nsteps - done : TS);
    s.E_in = fld[cur][0];
    s.H_in = fld[cur][1];
    s.J_in = fld[cur][2];
    s.E_out = fld[1 - cur][0];
    s.H_out = fld[1 - cur][1];
    s.J_out = fld[1 - cur][2];
    s.n0 = n0 + done;
    s.nsub = nsub;
    s.series_pos = 0;
    s.tiles = tiles;
    s.n_tiles = (int)(n_int - n_src);
    if (s.n_tiles && (e = launch_tb<T>(s, K, false, 2, st, false)) != cudaSuccess)
      return nfail(RKETD_ECUDA, cudaGetErrorString(e));
    s.tiles = tiles + (n_int - n_src);
    s.n_tiles = (int)n_src;
    if (n_src && (e = launch_tb<T>(s, K, false, 2, st, true)) != cudaSuccess)
      return nfail(RKETD_ECUDA, cudaGetErrorString(e));
    s.tiles = tiles + n_int;
    s.n_tiles = (int)n_edge;
    if (n_edge && (e = launch_tb<T>(s, Ke, true, 2, st, true)) != cudaSuccess)
      return nfail(RKETD_ECUDA, cudaGetErrorString(e));
    cur = 1 - cur;
    done += nsub;
  }
  k_out<T><<<(unsigned)((nz + 255) / 256), 256, 0, st>>>(fld[cur][0], fld[cur][1], fld[cur][2], coef[kCj],
                                                         coef[kDa], E, H, J, nz, 1.0 / eta0, kEps0 / g->dt);
  if ((e = cudaGetLastError()) != cudaSuccess) return nfail(RKETD_ECUDA, cudaGetErrorString(e));
  return RKETD_OK;
}

}  // namespace
}  // namespace rketd

using namespace rketd;

extern "C" rketd_status rketd_advance_1d_noalloc(const rketd_grid1d* grid, int64_t nz, const double* wp2,
                                                const double* nu, int64_t src_cell, const rketd_pulse* pulse,
                                                int64_t n0, int64_t nsteps, void* E, void* H, void* J,
                                                void* stream) {
  set_error_message("");
  if (!grid || !pulse || !wp2 || !nu || !E || !H || !J) return nfail(RKETD_EINVAL, "noalloc: NULL argument");
  if (nz < 8) return nfail(RKETD_EINVAL, "noalloc: nz must be >= 8");
  if (nz > kNoallocMaxNz)
    return nfail(RKETD_EINVAL, "noalloc: nz exceeds the fixed scratch capacity of 131072 cells");
  if (nsteps < 0 || n0 < 0) return nfail(RKETD_EINVAL, "noalloc: negative step count or index");
  if (grid->bc != RKETD_BC_MUR1) return nfail(RKETD_EUNSUPPORTED, "noalloc: only first-order Mur ends");
  if (grid->scheme != RKETD_SCHEME_RKETD && grid->scheme != RKETD_SCHEME_ETD1)
    return nfail(grid->scheme == RKETD_SCHEME_ETD2 ? RKETD_EUNSUPPORTED : RKETD_EINVAL,
                 "noalloc: scheme must be RKETD (Eq. 11) or ETD1 (Eq. 9)");
  if (grid->prec != RKETD_F32 && grid->prec != RKETD_F64) return nfail(RKETD_EINVAL, "noalloc: bad precision");
  if (!(grid->dz > 0) || !(grid->dt > 0) || !std::isfinite(grid->dz) || !std::isfinite(grid->dt))
    return nfail(RKETD_EINVAL, "noalloc: dz and dt must be finite and > 0");
  if (!(grid->dt / (grid->dz * std::sqrt(kMu0 * kEps0)) <= 1.0))
    return nfail(RKETD_ECOURANT, "noalloc: Courant number exceeds 1");
  if (src_cell < 1 || src_cell > nz - 2) return nfail(RKETD_EINVAL, "noalloc: source cell outside the interior");
  if (!(pulse->tau > 0)) return nfail(RKETD_EINVAL, "noalloc: pulse tau must be > 0");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return nfail(RKETD_ECUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= 64) return nfail(RKETD_EUNSUPPORTED, "noalloc: device ordinal >= 64");
  void* base;
  {
    // First call on each device: resolve the device address of the scratch array with that
    // device current (the host-side symbol is only a stand-in, not a device address).
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
      void* ptr = nullptr;
      e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
      if (e != cudaSuccess || !ptr) return nfail(RKETD_ECUDA, cudaGetErrorString(e));
      g_scratch_addr[dev] = ptr;
    }
    base = g_scratch_addr[dev];
  }
  cudaStream_t st = (cudaStream_t)stream;
  if (nsteps == 0) return RKETD_OK;
  if (grid->prec == RKETD_F64)
    return advance<double>(base, grid, nz, wp2, nu, src_cell, pulse, n0, nsteps, (double*)E, (double*)H, (double*)J, st);
  return advance<float>(base, grid, nz, wp2, nu, src_cell, pulse, n0, nsteps, (float*)E, (float*)H, (float*)J, st);
}

extern "C" rketd_status rketd_noalloc_tiles_1d(int32_t prec, int64_t nz, int64_t src_cell, int64_t* rows, int64_t cap,
                                              int64_t* n_tiles, int64_t* launch_counts) {
  set_error_message("");
  if (!n_tiles || !launch_counts || (cap > 0 && !rows) || cap < 0) return nfail(RKETD_EINVAL, "NULL argument");
  if (prec != RKETD_F32 && prec != RKETD_F64) return nfail(RKETD_EINVAL, "bad precision");
  if (nz < 8 || nz > kNoallocMaxNz) return nfail(RKETD_EINVAL, "nz must be in [8, 131072]");
  if (src_cell < 1 || src_cell > nz - 2) return nfail(RKETD_EINVAL, "source cell outside the interior");
  const bool f64 = prec == RKETD_F64;
  const int K = noalloc_K(f64), T = noalloc_T(f64), Ke = 4;
  const NoallocPlan pl = noalloc_plan(nz, src_cell, K, Ke, T);
  const int64_t n_src = pl.j_src1 - pl.j_src0;
  launch_counts[0] = pl.n_int - n_src;
  launch_counts[1] = n_src;
  launch_counts[2] = pl.n_edge;
  *n_tiles = pl.n_int + pl.n_edge;
  if (*n_tiles > kNoallocMaxTiles) return nfail(RKETD_EINVAL, "too many tiles");
  std::vector<Tile> t((size_t)*n_tiles);
  const int n = noalloc_tiles(pl, nz, src_cell, K, Ke, T, t.data());
  if (n != *n_tiles) return nfail(RKETD_EINVAL, "tile count differs from the plan");
  for (int64_t i = 0; i < n && i < cap; ++i) {
    int64_t* r = rows + 5 * i;
    r[0] = t[i].start;
    r[1] = t[i].vlo;
    r[2] = t[i].vhi;
    r[3] = t[i].src_local;
    r[4] = 32 * (i < pl.n_int ? K : Ke);
  }
  return RKETD_OK;
}
