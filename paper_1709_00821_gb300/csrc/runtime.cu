// Host runtime behind include/rketd.h: validation, device memory, tile planning, the
// step loop (plain or temporally blocked passes, DFT block folds), state files and the
// variant autotuner. Everything numeric runs in the kernels of the other files.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/rketd.h"
#include "rketd_internal.cuh"

using namespace rketd;

namespace {

thread_local std::string g_err;

// injected allocation failure (a test hook): -1 disarmed, else the successful allocations left
std::mutex g_alloc_mu;
int64_t g_alloc_fail_after = -1;
int64_t g_alloc_count = 0;

bool alloc_should_fail() {
  std::lock_guard<std::mutex> lk(g_alloc_mu);
  ++g_alloc_count;
  if (g_alloc_fail_after < 0) return false;
  if (g_alloc_fail_after == 0) {
    g_alloc_fail_after = -1;
    return true;
  }
  --g_alloc_fail_after;
  return false;
}

template <typename T>
__global__ void k_finite(const T* __restrict__ p, int64_t n, int* flag) {
  bool bad = false;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    bad |= !isfinite(p[i]);
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flag, 1);
}

rketd_status fail(rketd_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return st;
}

rketd_status cuda_fail(cudaError_t e, const char* what) {
  if (e == cudaErrorMemoryAllocation) return fail(RKETD_ENOMEM, "%s: %s", what, cudaGetErrorString(e));
  return fail(RKETD_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(call, what)                                  \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return cuda_fail(e_, what);  \
  } while (0)

int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

}  // namespace

void rketd::set_error_message(const char* msg) { g_err = msg ? msg : ""; }

cudaError_t rketd::device_alloc(void** p, size_t bytes) {
  *p = nullptr;
  if (alloc_should_fail()) return cudaErrorMemoryAllocation;
  return cudaMalloc(p, bytes);
}

cudaError_t rketd::device_alloc_async(void** p, size_t bytes, cudaStream_t st) {
  *p = nullptr;
  if (alloc_should_fail()) return cudaErrorMemoryAllocation;
  return cudaMallocAsync(p, bytes, st);
}

cudaError_t rketd::launch_finite_scan(bool f64, const void* p, int64_t n, int* flag, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const unsigned blocks = (unsigned)std::min<int64_t>((n + 255) / 256, 152 * 8);
  if (f64)
    k_finite<double><<<blocks, 256, 0, st>>>((const double*)p, n, flag);
  else
    k_finite<float><<<blocks, 256, 0, st>>>((const float*)p, n, flag);
  return cudaGetLastError();
}

struct rketd_ctx {
  int32_t n_slabs = 0;
  int prec = 0;
  size_t esz = 4;
  rketd_grid1d grid{};
  rketd_pulse pulse{};
  int n_probes = 0, n_freq = 0;
  std::vector<double> freq;
  std::vector<int64_t> nz, soff, off, src, probe_cell;
  int64_t n_store = 0, n_cells = 0;
  double S = 0, qmur = 0;
  cudaStream_t stream = nullptr;
  rketd_options opt{};
  bool auto_variant = false;  // variant 0 was asked for: resident where it applies, else tiled

  // device memory
  std::vector<void*> allocs;
  void* E[2] = {nullptr, nullptr};
  void* H[2] = {nullptr, nullptr};
  void* J[2] = {nullptr, nullptr};
  int cur = 0;
  void* coef[kNumCoef] = {};
  // Eq. 10 recursion only: E^{n-1} and its weights ep, gp in the E and G updates
  void* Ep = nullptr;
  void* ext[2] = {nullptr, nullptr};
  double* wp2_d = nullptr;
  double* nu_d = nullptr;
  int64_t* soff_d = nullptr;
  int64_t* off_d = nullptr;
  int64_t* nz_d = nullptr;
  int64_t* src_d = nullptr;
  int32_t* cell_slab_d = nullptr;
  void* psiE[2] = {nullptr, nullptr};
  void* psiH[2] = {nullptr, nullptr};
  int64_t n_psi = 0;
  void* cpmlE = nullptr;
  void* cpmlH = nullptr;
  int64_t* probe_index_d = nullptr;
  double* freq_d = nullptr;
  void* series = nullptr;
  void* tw = nullptr;
  double* Xr = nullptr;
  double* Xi = nullptr;
  double* Xtmp = nullptr;  // [2][P*nf] for spectra with pending samples
  double* rot = nullptr;   // [nf][2] exp(-j 2 pi f m0 dt) of the fold being added
  int total_probes = 0;

  // tiles for the current (K, tb_steps)
  std::vector<Tile> tiles_h;
  Tile* adj_tiles_d = nullptr;  // [interior off-window][interior on-window][edge] for the adjoint
  int adj_n_plain = 0, adj_n_win = 0;
  int64_t adj_w_lo = -1, adj_w_hi = -1;
  Tile* tiles_d = nullptr;
  TileProbe* tprobes_d = nullptr;
  int n_interior = 0, n_edge = 0;
  int n_int_xtra = 0;  // the last n_int_xtra interior tiles sample a probe or load a source cell
  int tiles_K = 0, tiles_T = 0;
  bool tiles_ends = false;  // the plan has end tiles (build_tile_plan)
  bool in_ckpt = false;     // inside rketd_forward_ckpt

  // persistent variant: per tile, the neighbours it waits for (CSR), its last finished pass, the
  // work counter, the status word and the two passes' step arguments
  int* dep_off_d = nullptr;
  int* dep_idx_d = nullptr;
  int* done_d = nullptr;
  int* work_d = nullptr;
  int* err_d = nullptr;
  StepArgs<float>* sa_d = nullptr;
  int persist_grid = 0;
  int wait_limit = 1 << 22;
  int64_t persist_cells = 0;  // exact cells of all tiles (timing)

  // resident variant: cluster shape, left padding, probe list (slab cell, probe index)
  bool res_ok = false;
  int res_K = 0, res_ctas = 0, res_threads = 0, res_pl = 0;
  TileProbe* res_probes_d = nullptr;

  int64_t step = 0;
  int64_t launches = 0;

  // the edge-tile kernel runs on a side stream, overlapping the interior kernel; the probe and
  // source tiles (forward) or the window tiles (adjoint) on a second one, so that these two
  // latency-bound launches of few warps also overlap each other
  cudaStream_t side = nullptr, side2 = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr, join2 = nullptr;

  // adjoint: checkpoints of the forward run and the reverse-sweep buffers
  int64_t ckpt_steps = 0;  // steps of the checkpointed forward run (0 = none)
  int32_t ckpt_every = 0;
  void* ckpt = nullptr;    // [n_ckpt][3][n_store]
  int64_t n_ckpt = 0;
  void* lam[6] = {};       // adjoint E, H, J (two copies each)
  void* recF = nullptr;
  void* recA = nullptr;
  // a second set of segment records: the gradient sums of one segment run on gstream while the
  // next segment is recomputed and swept on the main and side streams
  void* recF2 = nullptr;
  void* recA2 = nullptr;
  void* seeds2 = nullptr;    // the loss seeds of the next segment, made ahead on gstream
  void* tw_seed2 = nullptr;
  cudaStream_t gstream = nullptr;
  cudaEvent_t ev_adj = nullptr, ev_grad[2] = {nullptr, nullptr}, ev_seed = nullptr;
  void* seeds = nullptr;
  void* tw_seed = nullptr;
  double* gX = nullptr;    // [2][P*nf]
  double* gacc = nullptr;  // [5][n_slabs][w]
  int64_t rec_cap = 0;     // window width the record buffers were sized for

  // captured whole rketd_step calls, keyed by (start step, steps, buffer parity)
  struct GraphEntry {
    int64_t s0, n;
    int cur_in, cur_out;
    int64_t launches;
    int K, T;
    cudaGraphExec_t exec;
  };
  std::vector<GraphEntry> graphs;
  cudaStream_t cap = nullptr;  // capture/replay stream, forked from and joined to `stream`
  cudaEvent_t cap_in = nullptr, cap_out = nullptr;

  // optional CUDA-event timing of the interior tiled kernel (the dominant kernel)
  bool timing = false;
  std::vector<cudaEvent_t> ev;  // pairs: start, stop
  size_t ev_used = 0;
  double t_ms = 0, t_cells = 0;
  int64_t t_launches = 0;

  ~rketd_ctx() {
    for (GraphEntry& g : graphs) cudaGraphExecDestroy(g.exec);
    if (adj_tiles_d) cudaFree(adj_tiles_d);
    if (cap_in) cudaEventDestroy(cap_in);
    if (cap_out) cudaEventDestroy(cap_out);
    if (cap) cudaStreamDestroy(cap);
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
    if (fork) cudaEventDestroy(fork);
    if (join) cudaEventDestroy(join);
    if (join2) cudaEventDestroy(join2);
    if (side) cudaStreamDestroy(side);
    if (side2) cudaStreamDestroy(side2);
    if (ev_adj) cudaEventDestroy(ev_adj);
    if (ev_seed) cudaEventDestroy(ev_seed);
    for (cudaEvent_t e : ev_grad)
      if (e) cudaEventDestroy(e);
    if (gstream) cudaStreamDestroy(gstream);
    for (void* p : allocs) cudaFree(p);
    if (tiles_d) cudaFree(tiles_d);
    if (tprobes_d) cudaFree(tprobes_d);
    if (dep_off_d) cudaFree(dep_off_d);
    if (dep_idx_d) cudaFree(dep_idx_d);
    if (done_d) cudaFree(done_d);
    if (res_probes_d) cudaFree(res_probes_d);
  }

  rketd_status alloc(void** p, size_t bytes, const char* what) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = device_alloc(p, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return cuda_fail(e, what);
    }
    allocs.push_back(*p);
    return RKETD_OK;
  }
  int pos() const { return (int)(step % opt.dft_block); }
};

namespace {

bool finite_pos(double x) { return std::isfinite(x) && x > 0; }

rketd_status check_options(const rketd_options& o, int prec) {
  if (o.variant < 0 || o.variant > 4) return fail(RKETD_EINVAL, "options.variant must be 0, 1, 2, 3 or 4");
  if (o.variant == 4 && (prec != 0 || o.fp32_pairs == 2))
    return fail(RKETD_EUNSUPPORTED, "the persistent variant runs FP32 fields with packed pairs");
  if (o.res_ctas < 0 || o.res_ctas > 16) return fail(RKETD_EINVAL, "res_ctas must be 0..16");
  if (o.res_threads < 0 || o.res_threads % 32 || o.res_threads > (prec == 1 ? 256 : 1024))
    return fail(RKETD_EINVAL, "res_threads must be a multiple of 32, at most 1024 (FP32) or 256 (FP64)");
  if (o.res_cells != 0 && (prec == 1 ? (o.res_cells != 1 && o.res_cells != 2 && o.res_cells != 4 && o.res_cells != 8)
                                     : (o.res_cells != 2 && o.res_cells != 4 && o.res_cells != 8 && o.res_cells != 16)))
    return fail(RKETD_EINVAL, "res_cells must be 1, 2, 4 or 8 (FP64) or 2, 4, 8 or 16 (FP32)");
  if (prec == 0 && o.cells_per_lane != 0 && o.cells_per_lane != 8 && o.cells_per_lane != 12 &&
      o.cells_per_lane != 16)
    return fail(RKETD_EUNSUPPORTED, "FP32 cells_per_lane must be 8, 12 or 16");
  if (prec == 1 && o.cells_per_lane != 0 && o.cells_per_lane != 4 && o.cells_per_lane != 8)
    return fail(RKETD_EUNSUPPORTED, "FP64 cells_per_lane must be 4 or 8");
  if (o.tb_steps != 0 && (o.tb_steps < 4 || o.tb_steps > 64 || o.tb_steps % 4))
    return fail(RKETD_EINVAL, "tb_steps must be a multiple of 4 in [4, 64]");
  if (o.warps_per_block < 0 || o.warps_per_block > 4) return fail(RKETD_EINVAL, "warps_per_block must be 1..4");
  if (o.dft_block < 0) return fail(RKETD_EINVAL, "dft_block must be >= 0");
  if (o.fp32_pairs < 0 || o.fp32_pairs > 2) return fail(RKETD_EINVAL, "fp32_pairs must be 0, 1 or 2");
  if (o.use_graphs < 0 || o.use_graphs > 2) return fail(RKETD_EINVAL, "use_graphs must be 0, 1 or 2");
  return RKETD_OK;
}

void fill_auto(rketd_options& o, int prec) {
  if (o.variant == 0) o.variant = 2;  // the resident variant is chosen over this at creation where it applies
  if (o.cells_per_lane == 0) o.cells_per_lane = prec == 1 ? 8 : 16;
  if (o.tb_steps == 0) o.tb_steps = prec == 1 ? 4 : 32;
  // a tile must keep at least 32 exact cells
  while (32 * o.cells_per_lane - 2 * o.tb_steps < 32 && o.tb_steps > 4) o.tb_steps -= 4;
  if (o.warps_per_block == 0) o.warps_per_block = prec == 1 ? 2 : 1;
  if (o.dft_block == 0) o.dft_block = 512;
  o.dft_block = (int32_t)round_up(o.dft_block, o.tb_steps);
}

// Cells per lane of the edge-tile kernel: narrow tiles keep the boundary code cheap.
int edge_cells_per_lane(int T) { return 32 * 4 - 2 * T >= 32 ? 4 : 8; }

// The tile lists of one plan: interior tiles (those without a probe or a source cell first), then
// edge tiles, in launch order; the tile-probe list they index.
struct TilePlan {
  std::vector<Tile> tiles;
  std::vector<TileProbe> probes;
  int n_interior = 0, n_int_xtra = 0, n_edge = 0;
};

// Builds the warp tiles for (K, T) on the host. Per slab, interior tiles of W = 32K - 2T exact
// cells cover the middle: their loaded range (T cells of halo each side) stays inside
// [max(1, ncpml), nz - 2 - ncpml], so the interior kernel needs no boundary code; one more
// interior tile, shifted left to end at that guard, takes the cells after the last whole one.
// Narrow edge tiles (Ke cells per lane) cover the two ends, where the Mur/PEC cells, the CPML
// and cells outside the slab live. Every cell is exact in exactly one tile.
// ends (first-order Mur ends, FP32 pairs): in slabs of more than 2 (32K - T) cells, two end tiles of the
// interior width take the ends instead of the edge tiles. The left one loads [0, 32K) and holds
// [0, 32K - T) exactly (no halo is needed beside the Mur cell); the right one starts at
// round_up(nz, 4) - 32K (so its copies stay 16-byte aligned and inside the slab's storage) and
// holds its cells from T on, up to nz - 1. They are the only interior-width tiles that load cell 0
// or cell nz - 1, which is how the kernel tells them apart; they run with the probe/source tiles.
// The interior tiles between them are planned as above, with the last one shifted left to end
// where the right end tile's exact cells begin.
rketd_status build_tile_plan(int n_slabs, const int64_t* nzs, const int64_t* srcs, int n_probes,
                             const int64_t* probe_cell, int64_t nc, int K, int T, bool ends, TilePlan& out) {
  const int L = 32 * K;
  const int W = L - 2 * T;
  const int Ke = edge_cells_per_lane(T);
  const int Le = 32 * Ke;
  const int We = Le - 2 * T;
  if (W < 4 || We < 4) return fail(RKETD_EINVAL, "tile of %d cells cannot hold %d steps of halo", L, T);
  std::vector<Tile> interior, edge;
  std::vector<TileProbe> tp_int, tp_edge;
  // a tile loading [start, start + Lt) and storing the exact cells [vstart, vend)
  auto add_at = [&](int s, int64_t start, int64_t vstart, int64_t vend, int Lt, bool is_edge) -> rketd_status {
    Tile t{};
    t.slab = s;
    t.start = start;
    t.vlo = (int32_t)(vstart - start);
    t.vhi = (int32_t)(vend - start);
    const int64_t sl = srcs[s] - t.start;
    t.src_local = (sl >= 0 && sl < Lt) ? (int32_t)sl : -1;
    std::vector<TileProbe>& tps = is_edge ? tp_edge : tp_int;
    t.probe_begin = (int32_t)tps.size();
    for (int p = 0; p < n_probes; ++p) {
      const int64_t cell = probe_cell[(size_t)s * n_probes + p];
      const int64_t loc = cell - t.start;
      if (loc >= t.vlo && loc < t.vhi) tps.push_back({(int32_t)loc, s * n_probes + p});
    }
    t.probe_count = (int32_t)tps.size() - t.probe_begin;
    if (t.probe_count > kMaxTileProbes) return fail(RKETD_EINVAL, "more than %d probes in one tile", kMaxTileProbes);
    // probes anywhere in the loaded range (the adjoint seeds every copy of a probe cell)
    t.adj_begin = (int32_t)tps.size();
    for (int p = 0; p < n_probes; ++p) {
      const int64_t cell = probe_cell[(size_t)s * n_probes + p];
      const int64_t loc = cell - t.start;
      if (loc >= 0 && loc < Lt) tps.push_back({(int32_t)loc, s * n_probes + p});
    }
    t.adj_count = (int32_t)tps.size() - t.adj_begin;
    (is_edge ? edge : interior).push_back(t);
    return RKETD_OK;
  };
  auto add = [&](int s, int64_t vstart, int64_t vend, int Lt, bool is_edge) -> rketd_status {
    return add_at(s, vstart - T, vstart, vend, Lt, is_edge);
  };
  for (int s = 0; s < n_slabs; ++s) {
    const int64_t nz = nzs[s];
    rketd_status st;
    if (ends && nc == 0) {
      const int64_t aL = L - T;                  // the left end tile's exact cells: [0, aL)
      const int64_t sR = round_up(nz, 4) - L;    // the right end tile loads [sR, sR + L)
      if (sR + 2 * T - L >= 1) {                 // room for the shifted interior tile
        const int64_t hi = sR + T;               // interior tiles: exact [aL, hi)
        if ((st = add_at(s, 0, 0, aL, L, false))) return st;
        int64_t v = aL;
        for (; v + W <= hi; v += W)
          if ((st = add(s, v, v + W, L, false))) return st;
        if (v < hi && (st = add_at(s, hi - (L - T), v, hi, L, false))) return st;
        if ((st = add_at(s, sR, hi, nz, L, false))) return st;
        continue;
      }
    }
    const int64_t lo_guard = std::max<int64_t>(1, nc);
    const int64_t hi_guard = nz - 2 - nc;
    int64_t a = round_up(lo_guard + T, 4);
    int64_t n_int = 0;
    if (a - T + L - 1 <= hi_guard) n_int = (hi_guard - (a - T + L - 1)) / W + 1;
    if (n_int == 0) a = 0;
    int64_t b = a + n_int * W;
    for (int64_t v = 0; v < a; v += We)
      if ((st = add(s, v, std::min<int64_t>(v + We, a), Le, true))) return st;
    for (int64_t j = 0; j < n_int; ++j)
      if ((st = add(s, a + j * W, a + (j + 1) * W, L, false))) return st;
    // One more interior tile, shifted left as far as the guard needs (start a multiple of 4), takes
    // over the cells after b that it holds exactly: the narrow edge tiles, several times dearer per
    // cell, then only cover the last T + ncpml + a few cells.
    if (n_int > 0) {
      const int64_t st4 = ((hi_guard - L + 1) / 4) * 4;
      const int64_t e_end = st4 + L - T;
      if (st4 >= lo_guard && e_end > b) {
        if ((st = add_at(s, st4, b, e_end, L, false))) return st;
        b = e_end;
      }
    }
    for (int64_t v = b; v < nz; v += We)
      if ((st = add(s, v, std::min<int64_t>(v + We, nz), Le, true))) return st;
  }
  for (Tile& t : edge) {
    t.probe_begin += (int32_t)tp_int.size();
    t.adj_begin += (int32_t)tp_int.size();
  }
  // interior tiles that sample a probe, load a source cell or hold a slab end go last: they run
  // the kernel with that code, the others a kernel without a per-step branch for it
  auto plain_tile = [&](const Tile& t) {
    return t.src_local < 0 && t.probe_count == 0 && t.start != 0 && t.start + L - 1 < nzs[t.slab] - 1;
  };
  std::stable_partition(interior.begin(), interior.end(), plain_tile);
  out.n_int_xtra = 0;
  for (const Tile& t : interior) out.n_int_xtra += !plain_tile(t);
  out.n_interior = (int)interior.size();
  out.n_edge = (int)edge.size();
  out.tiles = interior;
  out.tiles.insert(out.tiles.end(), edge.begin(), edge.end());
  out.probes = tp_int;
  out.probes.insert(out.probes.end(), tp_edge.begin(), tp_edge.end());
  return RKETD_OK;
}

// Plans the tiles for (K, T) and uploads the lists.
// Persistent variant: for every tile, the tiles of its slab that it must wait for before a pass
// (those whose exact cells its loaded range reads, and those whose loaded range reads the exact
// cells it writes, itself included), as a CSR list; the flags, counter, status word and argument
// room of the launch; the grid (resident one-warp blocks).
rketd_status plan_persist(rketd_ctx* c, int K, int T) {
  const std::vector<Tile>& t = c->tiles_h;
  const int n = (int)t.size();
  const int Ke = edge_cells_per_lane(T);
  struct R { int64_t l0, l1, e0, e1; int j; };
  std::vector<std::vector<R>> by_slab(c->n_slabs);
  int64_t cells = 0;
  for (int j = 0; j < n; ++j) {
    const int64_t w = 32LL * (j < c->n_interior ? K : Ke);
    by_slab[t[j].slab].push_back({t[j].start, t[j].start + w, t[j].start + t[j].vlo, t[j].start + t[j].vhi, j});
    cells += t[j].vhi - t[j].vlo;
  }
  std::vector<std::vector<int>> deps(n);
  for (auto& v : by_slab) {
    std::sort(v.begin(), v.end(), [](const R& x, const R& y) { return x.l0 < y.l0; });
    const int m = (int)v.size();
    const int64_t wmax = 32LL * std::max(K, Ke);  // widest loaded range
    int lo = 0;
    for (int a = 0; a < m; ++a) {
      // only tiles whose loaded range starts within (l0 - wmax, l1) can overlap tile a
      while (lo < m && v[lo].l0 <= v[a].l0 - wmax) ++lo;
      for (int b = lo; b < m && v[b].l0 < v[a].l1; ++b) {
        const bool raw = v[b].e0 < v[a].l1 && v[a].l0 < v[b].e1;  // a reads b's exact cells
        const bool war = v[b].l0 < v[a].e1 && v[a].e0 < v[b].l1;  // b read what a writes
        if (raw || war) deps[v[a].j].push_back(v[b].j);
      }
    }
  }
  std::vector<int> off(n + 1, 0), idx;
  for (int j = 0; j < n; ++j) {
    off[j + 1] = off[j] + (int)deps[j].size();
    idx.insert(idx.end(), deps[j].begin(), deps[j].end());
  }
  if (c->dep_off_d) cudaFree(c->dep_off_d);
  if (c->dep_idx_d) cudaFree(c->dep_idx_d);
  if (c->done_d) cudaFree(c->done_d);
  c->dep_off_d = c->dep_idx_d = c->done_d = nullptr;
  CK(device_alloc((void**)&c->dep_off_d, sizeof(int) * (n + 1)), "tile dependencies");
  CK(device_alloc((void**)&c->dep_idx_d, sizeof(int) * std::max<size_t>(1, idx.size())), "tile dependencies");
  CK(device_alloc((void**)&c->done_d, sizeof(int) * std::max(1, n)), "tile flags");
  CK(cudaMemcpy(c->dep_off_d, off.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice), "tile dependencies");
  if (!idx.empty())
    CK(cudaMemcpy(c->dep_idx_d, idx.data(), sizeof(int) * idx.size(), cudaMemcpyHostToDevice), "tile dependencies");
  if (!c->work_d) {
    void* p = nullptr;
    rketd_status st = c->alloc(&p, 2 * sizeof(int), "persistent counters");
    if (st) return st;
    c->work_d = (int*)p;
    c->err_d = c->work_d + 1;
    CK(cudaMemset(c->work_d, 0, 2 * sizeof(int)), "persistent counters");
    st = c->alloc(&p, 2 * sizeof(StepArgs<float>), "persistent arguments");
    if (st) return st;
    c->sa_d = (StepArgs<float>*)p;
  }
  c->persist_grid = persist_capacity(K, Ke);
  if (c->persist_grid <= 0) return fail(RKETD_ECUDA, "persistent step: no resident capacity");
  c->persist_cells = cells;
  return RKETD_OK;
}

// Whether the tiled and persistent forward steps plan end tiles (build_tile_plan): FP32 pairs with
// first-order Mur ends. The checkpointed run and the adjoint keep the edge tiles.
bool fwd_end_tiles(const rketd_ctx* c) {
  return c->prec != RKETD_F64 && (c->opt.variant == 2 || c->opt.variant == 4) && c->opt.fp32_pairs != 2 &&
         c->opt.cells_per_lane % 4 == 0 && c->grid.bc == RKETD_BC_MUR1 && !c->in_ckpt;
}

rketd_status plan_tiles(rketd_ctx* c, int K, int T, bool ends = false) {
  const int64_t nc = c->grid.bc != RKETD_BC_MUR1 ? c->grid.cpml_cells : 0;
  TilePlan plan;
  rketd_status st0 = build_tile_plan(c->n_slabs, c->nz.data(), c->src.data(), c->n_probes, c->probe_cell.data(), nc,
                                     K, T, ends, plan);
  if (st0) return st0;
  const std::vector<Tile>& all = plan.tiles;
  const std::vector<TileProbe>& tps = plan.probes;
  c->tiles_h = all;
  c->adj_w_lo = c->adj_w_hi = -1;  // the adjoint's tile order is rebuilt on next use
  // captured graphs point at the old tile lists
  for (auto& g : c->graphs) cudaGraphExecDestroy(g.exec);
  c->graphs.clear();
  if (c->tiles_d) cudaFree(c->tiles_d);
  if (c->tprobes_d) cudaFree(c->tprobes_d);
  c->tiles_d = nullptr;
  c->tprobes_d = nullptr;
  CK(device_alloc((void**)&c->tiles_d, sizeof(Tile) * std::max<size_t>(1, all.size())), "tile list");
  CK(device_alloc((void**)&c->tprobes_d, sizeof(TileProbe) * std::max<size_t>(1, tps.size())), "tile probes");
  CK(cudaMemcpy(c->tiles_d, all.data(), sizeof(Tile) * all.size(), cudaMemcpyHostToDevice), "tile upload");
  if (!tps.empty())
    CK(cudaMemcpy(c->tprobes_d, tps.data(), sizeof(TileProbe) * tps.size(), cudaMemcpyHostToDevice),
       "tile probe upload");
  c->n_interior = plan.n_interior;
  c->n_int_xtra = plan.n_int_xtra;
  c->n_edge = plan.n_edge;
  c->tiles_K = K;
  c->tiles_T = T;
  c->tiles_ends = ends;
  if (c->opt.variant == 4) return plan_persist(c, K, T);
  return RKETD_OK;
}

// Shape of the resident variant for this context (single Mur slab, not the Eq. 10 recursion): the
// first instantiated shape (cells per thread K, CTA size) whose cluster of at most 16 CTAs holds the
// slab. FP64 prefers few cells per thread over many CTAs of 128 threads (a warp per SM sub-partition,
// whose FP64 units are few); FP32 prefers 2 cells per thread in CTAs of up to 1024 threads (its
// steps are latency-bound: many short warps beat few long ones). Options
// res_cells / res_threads / res_ctas override. The shape is kept only if it can be scheduled.
// Returns RKETD_EUNSUPPORTED (with the reason) where it does not apply.
rketd_status plan_resident(rketd_ctx* c) {
  c->res_ok = false;
  if (c->n_slabs != 1 || c->grid.bc != RKETD_BC_MUR1 || c->grid.scheme == RKETD_SCHEME_ETD2)
    return fail(RKETD_EUNSUPPORTED, "the resident variant takes one slab with first-order Mur ends (Eq. 11 or 9)");
  const int64_t nz = c->nz[0];
  const bool f64 = c->prec == RKETD_F64;
  // instantiated shapes: cells per thread and the largest CTA for it, in order of preference
  struct Shape { int K, max_threads, default_threads; };
  const Shape s64[] = {{1, 256, 128}, {2, 256, 128}, {4, 256, 128}, {8, 128, 128}};
  const Shape s32[] = {{2, 1024, 1024}, {4, 512, 512}, {8, 256, 256}, {16, 128, 128}};
  const Shape* shapes = f64 ? s64 : s32;
  int K = 0, ctas = 0, pl = 0, threads = 0;
  for (int q = 0; q < 4 && !K; ++q) {
    const Shape sh = shapes[q];
    if (c->opt.res_cells && c->opt.res_cells != sh.K) continue;
    if (c->opt.res_threads > sh.max_threads) continue;
    const int k = sh.K;
    const int p = ((nz - 1) % (32 * k) == 0) ? 1 : 0;  // keeps cells nz-2, nz-1 in one warp
    int th = c->opt.res_threads ? c->opt.res_threads : sh.default_threads;
    int n = c->opt.res_ctas ? c->opt.res_ctas : (int)((nz + p + (int64_t)th * k - 1) / ((int64_t)th * k));
    if (!c->opt.res_threads && n == 1)  // one CTA: no more threads than the slab needs
      th = (int)std::min<int64_t>(th, round_up((nz + p + k - 1) / k, 32));
    if (n >= 1 && n <= 16 && (int64_t)n * th * k >= nz + p) {
      K = k;
      ctas = n;
      pl = p;
      threads = th;
    }
  }
  if (!K) return fail(RKETD_EUNSUPPORTED, "slab of %lld cells does not fit the resident variant's shapes", (long long)nz);
  int max_clusters = 0;
  const StepArgs<double> q64{};
  const StepArgs<float> q32{};
  cudaError_t e = f64 ? launch_resident<double>(q64, K, ctas, threads, pl, c->stream, true, &max_clusters)
                      : launch_resident<float>(q32, K, ctas, threads, pl, c->stream, true, &max_clusters);
  if (e != cudaSuccess || max_clusters < 1) {
    cudaGetLastError();
    return fail(RKETD_EUNSUPPORTED, "a cluster of %d CTAs x %d threads cannot be scheduled", ctas, threads);
  }
  if (!c->res_probes_d && c->n_probes) {
    std::vector<TileProbe> pr(c->n_probes);
    for (int p = 0; p < c->n_probes; ++p) pr[p] = {(int32_t)c->probe_cell[p], p};
    CK(device_alloc((void**)&c->res_probes_d, sizeof(TileProbe) * pr.size()), "probe list");
    CK(cudaMemcpy(c->res_probes_d, pr.data(), sizeof(TileProbe) * pr.size(), cudaMemcpyHostToDevice), "probe list");
  }
  c->res_K = K;
  c->res_ctas = ctas;
  c->res_threads = threads;
  c->res_pl = pl;
  c->res_ok = true;
  return RKETD_OK;
}

template <typename T>
StepArgs<T> make_args(rketd_ctx* c, int in, int out) {
  StepArgs<T> a{};
  a.E_in = (const T*)c->E[in];
  a.H_in = (const T*)c->H[in];
  a.J_in = (const T*)c->J[in];
  a.E_out = (T*)c->E[out];
  a.H_out = (T*)c->H[out];
  a.J_out = (T*)c->J[out];
  for (int k = 0; k < kNumCoef; ++k) a.coef[k] = (const T*)c->coef[k];
  a.soff = c->soff_d;
  a.nz = c->nz_d;
  a.src = c->src_d;
  a.Ep = (T*)c->Ep;
  a.ep = (const T*)c->ext[0];
  a.gp = (const T*)c->ext[1];
  a.psiE_in = (const T*)c->psiE[in];
  a.psiH_in = (const T*)c->psiH[in];
  a.psiE_out = (T*)c->psiE[out];
  a.psiH_out = (T*)c->psiH[out];
  a.cpmlE = (const T*)c->cpmlE;
  a.cpmlH = (const T*)c->cpmlH;
  a.ncpml = c->grid.bc != RKETD_BC_MUR1 ? c->grid.cpml_cells : 0;
  a.bc = c->grid.bc;
  a.S = (T)c->S;
  a.qmur = (T)c->qmur;
  a.dt = c->grid.dt;
  a.tau = c->pulse.tau;
  a.t0 = c->pulse.t0;
  a.amp = c->pulse.amp;
  a.n0 = c->step;
  a.series = (T*)c->series;
  a.series_len = c->opt.dft_block;
  a.series_pos = c->pos();
  a.total_probes = c->total_probes;
  return a;
}

// DFT of the first n buffered columns into (Xr, Xi), first sample index m0. The twiddle table holds
// exp(-j 2 pi f t dt) for t = 0 .. dft_block-1 (built at creation); the fold's sums are rotated by
// exp(-j 2 pi f m0 dt).
template <typename T>
rketd_status dft_block(rketd_ctx* c, int n, int64_t m0, double* Xr, double* Xi) {
  if (c->total_probes == 0 || n == 0) return RKETD_OK;
  CK(launch_dft_rotation(c->freq_d, c->n_freq, c->grid.dt, m0, c->rot, c->stream), "dft rotation");
  CK(launch_dft<T>((const T*)c->series, c->opt.dft_block, n, (const T*)c->tw, c->total_probes, c->n_freq, Xr,
                   Xi, c->stream, c->rot),
     "dft");
  c->launches += 2;
  return RKETD_OK;
}

rketd_status harvest_timing(rketd_ctx* c) {
  for (size_t i = 0; i + 1 < c->ev_used; i += 2) {
    CK(cudaEventSynchronize(c->ev[i + 1]), "timing event");
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, c->ev[i], c->ev[i + 1]), "timing event");
    c->t_ms += ms;
  }
  c->ev_used = 0;
  return RKETD_OK;
}

rketd_status timing_event(rketd_ctx* c, cudaEvent_t* out) {
  if (c->ev_used == c->ev.size()) {
    if (c->ev.size() >= 8192) {
      rketd_status st = harvest_timing(c);
      if (st) return st;
    } else {
      for (int i = 0; i < 256; ++i) {
        cudaEvent_t e;
        CK(cudaEventCreate(&e), "timing event");
        c->ev.push_back(e);
      }
    }
  }
  *out = c->ev[c->ev_used++];
  return RKETD_OK;
}

template <typename T>
rketd_status step_impl(rketd_ctx* c, int64_t nsteps) {
  const int B = c->opt.dft_block;
  while (nsteps > 0) {
    const int pos = c->pos();
    if (c->opt.variant == 1) {
      StepArgs<T> a = make_args<T>(c, c->cur, c->cur);
      a.nsub = 1;
      if (c->n_slabs > 1 && !c->cell_slab_d) {
        void* p;
        rketd_status st = c->alloc(&p, sizeof(int32_t) * c->n_store, "cell-to-slab map");
        if (st) return st;
        std::vector<int32_t> m(c->n_store);
        for (int s = 0; s < c->n_slabs; ++s) {
          const int64_t end = s + 1 < c->n_slabs ? c->soff[s + 1] : c->n_store;
          for (int64_t i = c->soff[s]; i < end; ++i) m[i] = s;
        }
        CK(cudaMemcpy(p, m.data(), sizeof(int32_t) * c->n_store, cudaMemcpyHostToDevice), "cell-to-slab upload");
        c->cell_slab_d = (int32_t*)p;
      }
      CK(launch_plain_step<T>(a, c->n_slabs > 1 ? c->cell_slab_d : nullptr, c->n_store, c->probe_index_d,
                              c->stream),
         "plain step");
      c->launches += 2 + (c->total_probes > 0);
      c->step += 1;
      nsteps -= 1;
    } else if (c->opt.variant == 3) {
      if (!c->res_ok) {
        rketd_status st = plan_resident(c);
        if (st) return st;
      }
      const int nsub = (int)std::min<int64_t>(nsteps, (int64_t)(B - pos));
      StepArgs<T> a = make_args<T>(c, c->cur, 1 - c->cur);
      a.nsub = nsub;
      a.tprobes = c->res_probes_d;
      cudaEvent_t e0 = nullptr, e1 = nullptr;
      if (c->timing) {
        rketd_status st = timing_event(c, &e0);
        if (!st) st = timing_event(c, &e1);
        if (st) return st;
        CK(cudaEventRecord(e0, c->stream), "timing event");
      }
      CK(launch_resident<T>(a, c->res_K, c->res_ctas, c->res_threads, c->res_pl, c->stream, false, nullptr),
         "resident step");
      c->launches += 1;
      if (c->timing) {
        CK(cudaEventRecord(e1, c->stream), "timing event");
        c->t_launches += 1;
        c->t_cells += (double)c->nz[0] * nsub;
      }
      c->cur = 1 - c->cur;
      c->step += nsub;
      nsteps -= nsub;
    } else if (c->opt.variant == 4) {
      // persistent: every whole pass left in this DFT block (or in the call) in one launch
      const int K = c->opt.cells_per_lane, TS = c->opt.tb_steps;
      if (c->tiles_K != K || c->tiles_T != TS || c->tiles_ends != fwd_end_tiles(c) || !c->done_d) {
        rketd_status st = plan_tiles(c, K, TS, fwd_end_tiles(c));
        if (st) return st;
      }
      const int nsub = (int)std::min<int64_t>({(int64_t)TS, nsteps, (int64_t)(B - pos)});
      const int n_pass = nsub == TS ? (int)std::min<int64_t>((B - pos) / TS, nsteps / TS) : 1;
      StepArgs<T> a0 = make_args<T>(c, c->cur, 1 - c->cur);
      StepArgs<T> a1 = make_args<T>(c, 1 - c->cur, c->cur);
      for (StepArgs<T>* a : {&a0, &a1}) {
        a->nsub = nsub;
        a->tprobes = c->tprobes_d;
        a->tiles = c->tiles_d;
        a->n_tiles = (int)c->tiles_h.size();
        a->n0 = a0.n0;
        a->series_pos = a0.series_pos;
      }
      PersistCtl pc{};
      pc.n_tiles = (int)c->tiles_h.size();
      pc.n_main = c->n_interior - c->n_int_xtra;
      pc.n_xtra = c->n_int_xtra;
      pc.n_pass = n_pass;
      pc.nsub = nsub;
      pc.dep_off = c->dep_off_d;
      pc.dep_idx = c->dep_idx_d;
      pc.done = c->done_d;
      pc.work = c->work_d;
      pc.err = c->err_d;
      pc.wait_limit = c->wait_limit;
      CK(cudaMemsetAsync(c->done_d, 0xff, sizeof(int) * std::max(1, pc.n_tiles), c->stream), "tile flags");
      CK(cudaMemsetAsync(c->work_d, 0, sizeof(int), c->stream), "work counter");
      const int grid = (int)std::min<int64_t>(c->persist_grid, ((int64_t)n_pass * pc.n_tiles + 7) / 8);
      cudaEvent_t e0 = nullptr, e1 = nullptr;
      if (c->timing) {
        rketd_status st = timing_event(c, &e0);
        if (!st) st = timing_event(c, &e1);
        if (st) return st;
        CK(cudaEventRecord(e0, c->stream), "timing event");
      }
      CK(launch_persist(c->sa_d, *reinterpret_cast<const StepArgs<float>*>(&a0),
                        *reinterpret_cast<const StepArgs<float>*>(&a1), pc, K, edge_cells_per_lane(TS), grid,
                        c->stream),
         "persistent step");
      c->launches += 2;
      if (c->timing) {
        CK(cudaEventRecord(e1, c->stream), "timing event");
        c->t_launches += 1;
        c->t_cells += (double)c->persist_cells * nsub * n_pass;
      }
      c->cur = (c->cur + n_pass) & 1;
      c->step += (int64_t)nsub * n_pass;
      nsteps -= (int64_t)nsub * n_pass;
    } else {
      const int K = c->opt.cells_per_lane, TS = c->opt.tb_steps;
      if (c->tiles_K != K || c->tiles_T != TS || c->tiles_ends != fwd_end_tiles(c)) {
        rketd_status st = plan_tiles(c, K, TS, fwd_end_tiles(c));
        if (st) return st;
      }
      const int nsub = (int)std::min<int64_t>({(int64_t)TS, nsteps, (int64_t)(B - pos)});
      StepArgs<T> a = make_args<T>(c, c->cur, 1 - c->cur);
      a.nsub = nsub;
      a.tprobes = c->tprobes_d;
      // Edge tiles first, on the high-priority side stream, so their few long-running warps
      // start before the interior grid fills the GPU, then the interior tiles with a probe or a
      // source cell; joined back after the main interior launch.
      const bool fp32p = std::is_same<T, float>::value && c->opt.fp32_pairs != 2 && K % 4 == 0;
      const int n_main = c->n_interior - c->n_int_xtra;
      const bool forked = n_main && (c->n_edge || c->n_int_xtra);
      const bool forked2 = forked && c->n_edge && c->n_int_xtra;
      cudaStream_t side = forked ? c->side : c->stream;
      cudaStream_t side2 = forked2 ? c->side2 : side;
      if (forked) {
        CK(cudaEventRecord(c->fork, c->stream), "fork");
        CK(cudaStreamWaitEvent(c->side, c->fork, 0), "fork");
        if (forked2) CK(cudaStreamWaitEvent(c->side2, c->fork, 0), "fork");
      }
      if (c->n_edge) {
        a.tiles = c->tiles_d + c->n_interior;
        a.n_tiles = c->n_edge;
        CK(launch_tb<T>(a, edge_cells_per_lane(TS), true, 2, side, true), "tiled step (edge)");
        c->launches += 1;
      }
      if (c->n_int_xtra) {
        a.tiles = c->tiles_d + n_main;
        a.n_tiles = c->n_int_xtra;
        if (fp32p) {
          CK(launch_tb_pairs(*reinterpret_cast<const StepArgs<float>*>(&a), K, c->opt.warps_per_block, side2, true),
             "tiled step (probe and source tiles, FP32 pairs)");
        } else {
          CK(launch_tb<T>(a, K, false, c->opt.warps_per_block, side2, true), "tiled step (probe and source tiles)");
        }
        c->launches += 1;
      }
      if (forked) CK(cudaEventRecord(c->join, c->side), "join");
      if (forked2) CK(cudaEventRecord(c->join2, c->side2), "join");
      a.tiles = c->tiles_d;
      a.n_tiles = n_main;
      if (a.n_tiles) {
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (c->timing) {
          rketd_status st = timing_event(c, &e0);
          if (!st) st = timing_event(c, &e1);
          if (st) return st;
          CK(cudaEventRecord(e0, c->stream), "timing event");
        }
        if (fp32p) {
          CK(launch_tb_pairs(*reinterpret_cast<const StepArgs<float>*>(&a), K, c->opt.warps_per_block, c->stream,
                             false),
             "tiled step (interior, FP32 pairs)");
        } else {
          CK(launch_tb<T>(a, K, false, c->opt.warps_per_block, c->stream, false), "tiled step (interior)");
        }
        c->launches += 1;
        if (c->timing) {
          CK(cudaEventRecord(e1, c->stream), "timing event");
          c->t_launches += 1;
          c->t_cells += (double)a.n_tiles * (32 * K - 2 * TS) * nsub;
        }
      }
      if (forked) CK(cudaStreamWaitEvent(c->stream, c->join, 0), "join");
      if (forked2) CK(cudaStreamWaitEvent(c->stream, c->join2, 0), "join");
      c->cur = 1 - c->cur;
      c->step += nsub;
      nsteps -= nsub;
    }
    if (c->pos() == 0) {
      rketd_status st = dft_block<T>(c, B, c->step - B + 1, c->Xr, c->Xi);
      if (st) return st;
    }
  }
  return RKETD_OK;
}

rketd_status validate_and_copy(rketd_ctx* c, int32_t n_slabs, const int64_t* nz, const rketd_grid1d* grid,
                               const double* wp2, const double* nu, const int64_t* src_cell,
                               const rketd_pulse* pulse, const int64_t* probe_cell, const rketd_dft* dft,
                               const rketd_options* opt) {
  if (n_slabs < 1) return fail(RKETD_EINVAL, "n_slabs must be >= 1");
  if (!nz || !grid || !wp2 || !nu || !src_cell || !pulse) return fail(RKETD_EINVAL, "NULL argument");
  if (!finite_pos(grid->dz) || !finite_pos(grid->dt)) return fail(RKETD_EINVAL, "dz and dt must be finite and > 0");
  if (grid->prec != RKETD_F32 && grid->prec != RKETD_F64) return fail(RKETD_EINVAL, "prec must be F32 or F64");
  if (grid->bc != RKETD_BC_MUR1 && grid->bc != RKETD_BC_CPML && grid->bc != RKETD_BC_PML)
    return fail(RKETD_EINVAL, "bc must be MUR1, CPML or PML");
  if (grid->scheme < RKETD_SCHEME_RKETD || grid->scheme > RKETD_SCHEME_ETD2)
    return fail(RKETD_EINVAL, "scheme must be RKETD (Eq. 11), ETD1 (Eq. 9) or ETD2 (Eq. 10)");
  const double S = grid->dt / (grid->dz * std::sqrt(kMu0 * kEps0));
  if (!(S <= 1.0)) return fail(RKETD_ECOURANT, "Courant number c dt/dz = %.17g exceeds 1", S);
  if (!finite_pos(pulse->tau) || !std::isfinite(pulse->t0) || !std::isfinite(pulse->amp))
    return fail(RKETD_EINVAL, "pulse tau must be > 0, t0 and amp finite");
  const int nc = grid->bc != RKETD_BC_MUR1 ? grid->cpml_cells : 0;
  if (grid->bc == RKETD_BC_PML) {
    if (grid->cpml_cells < 1) return fail(RKETD_EINVAL, "cpml_cells must be >= 1");
    if (!finite_pos(grid->cpml_m) || !std::isfinite(grid->cpml_sigma_max))
      return fail(RKETD_EINVAL, "PML grading parameters out of range");
  }
  if (grid->bc == RKETD_BC_CPML) {
    if (grid->cpml_cells < 1) return fail(RKETD_EINVAL, "cpml_cells must be >= 1");
    if (!finite_pos(grid->cpml_m) || !std::isfinite(grid->cpml_sigma_max) || !(grid->cpml_kappa_max >= 1.0) ||
        !(grid->cpml_alpha_max >= 0.0))
      return fail(RKETD_EINVAL, "CPML grading parameters out of range");
  }
  const int np = dft ? dft->n_probes : 0;
  const int nf = dft ? dft->n_freq : 0;
  if (np < 0 || (np > 0 && (nf < 1 || !dft->freq_hz || !probe_cell)))
    return fail(RKETD_EINVAL, "probes need n_freq >= 1, freq_hz and probe_cell");
  c->n_slabs = n_slabs;
  c->prec = grid->prec;
  c->esz = grid->prec == RKETD_F64 ? 8 : 4;
  c->grid = *grid;
  if (grid->bc != RKETD_BC_MUR1 && !(grid->cpml_sigma_max > 0))
    c->grid.cpml_sigma_max = 0.8 * (grid->cpml_m + 1) / (std::sqrt(kMu0 / kEps0) * grid->dz);
  c->pulse = *pulse;
  c->n_probes = np;
  c->n_freq = np > 0 ? nf : 0;
  for (int f = 0; f < c->n_freq; ++f) {
    if (!std::isfinite(dft->freq_hz[f]) || dft->freq_hz[f] < 0) return fail(RKETD_EINVAL, "frequencies must be >= 0");
    c->freq.push_back(dft->freq_hz[f]);
  }
  c->S = S;
  c->qmur = (S - 1.0) / (S + 1.0);
  int64_t o = 0, so = 0;
  for (int s = 0; s < n_slabs; ++s) {
    if (nz[s] < 8) return fail(RKETD_EINVAL, "slab %d: nz = %lld < 8", s, (long long)nz[s]);
    if (nc && 2 * (int64_t)nc + 4 > nz[s]) return fail(RKETD_EINVAL, "slab %d: CPML thicker than the grid", s);
    const int64_t sc = src_cell[s];
    if (sc < std::max<int64_t>(1, nc) || sc > nz[s] - 1 - std::max(1, nc))
      return fail(RKETD_EINVAL, "slab %d: source cell %lld outside the interior", s, (long long)sc);
    for (int p = 0; p < np; ++p) {
      const int64_t pc = probe_cell[(size_t)s * np + p];
      if (pc < nc || pc > nz[s] - 1 - nc || pc < 0 || pc >= nz[s])
        return fail(RKETD_EINVAL, "slab %d: probe cell %lld outside the grid or inside the CPML", s, (long long)pc);
      c->probe_cell.push_back(pc);
    }
    c->nz.push_back(nz[s]);
    c->off.push_back(o);
    c->soff.push_back(so);
    c->src.push_back(sc);
    o += nz[s];
    so += round_up(nz[s], 32);
  }
  c->n_cells = o;
  c->n_store = so;
  for (int64_t i = 0; i < o; ++i) {
    if (!(wp2[i] >= 0) || !std::isfinite(wp2[i])) return fail(RKETD_EINVAL, "wp2[%lld] must be finite and >= 0", (long long)i);
    if (!(nu[i] >= 0) || !std::isfinite(nu[i])) return fail(RKETD_EINVAL, "nu[%lld] must be finite and >= 0", (long long)i);
  }
  if (grid->bc == RKETD_BC_PML)  // the split-field PML layers are vacuum
    for (int s = 0; s < n_slabs; ++s)
      for (int64_t k = 0; k < nz[s]; ++k)
        if ((k < nc || k > nz[s] - 1 - nc) && wp2[c->off[s] + k] != 0.0)
          return fail(RKETD_EINVAL, "slab %d: plasma (wp2 > 0) at cell %lld inside the PML layer", s, (long long)k);
  c->total_probes = n_slabs * np;
  rketd_options op{};
  rketd_default_options(&op);
  if (opt) op = *opt;
  rketd_status st = check_options(op, c->prec);
  if (st) return st;
  c->auto_variant = op.variant == 0;
  if (grid->scheme == RKETD_SCHEME_ETD2) {
    // E^{n-1} is one more carried array: the plain (one step per launch) kernels carry it
    if (op.variant == 2 || op.variant == 3 || op.variant == 4)
      return fail(RKETD_EUNSUPPORTED, "the Eq. 10 recursion (ETD2) runs on the plain variant only");
    op.variant = 1;
  }
  fill_auto(op, c->prec);
  c->opt = op;
  return RKETD_OK;
}

rketd_status zero_state(rketd_ctx* c) {
  const size_t fb = c->esz * c->n_store;
  for (int b = 0; b < 2; ++b) {
    CK(cudaMemsetAsync(c->E[b], 0, fb, c->stream), "memset E");
    CK(cudaMemsetAsync(c->H[b], 0, fb, c->stream), "memset H");
    CK(cudaMemsetAsync(c->J[b], 0, fb, c->stream), "memset J");
    if (c->n_psi) {
      CK(cudaMemsetAsync(c->psiE[b], 0, c->esz * c->n_psi, c->stream), "memset psi");
      CK(cudaMemsetAsync(c->psiH[b], 0, c->esz * c->n_psi, c->stream), "memset psi");
    }
  }
  if (c->Ep) CK(cudaMemsetAsync(c->Ep, 0, fb, c->stream), "memset E^{n-1}");
  if (c->total_probes) {
    const size_t xb = sizeof(double) * c->total_probes * c->n_freq;
    CK(cudaMemsetAsync(c->Xr, 0, xb, c->stream), "memset X");
    CK(cudaMemsetAsync(c->Xi, 0, xb, c->stream), "memset X");
  }
  if (c->err_d) CK(cudaMemsetAsync(c->err_d, 0, sizeof(int), c->stream), "status word");
  c->cur = 0;
  c->step = 0;
  return RKETD_OK;
}

rketd_status update_coeffs(rketd_ctx* c) {
  CK(launch_coeffs(c->prec, c->wp2_d, c->nu_d, c->soff_d, c->off_d, c->nz_d, c->n_slabs, c->n_store, c->grid.dt,
                   c->S, c->coef, c->stream, c->grid.scheme, c->ext),
     "coefficient kernel");
  c->launches += 1;
  return RKETD_OK;
}

// rketd_step through a CUDA graph: a call with the same start step, step count, buffer parity
// and tile shape as an earlier one replays that call's captured launches (a whole run from a
// reset, for example); otherwise the call is captured on the internal stream and kept (up to
// 8 graphs). The internal stream is ordered after and before the context's stream by events,
// so capture works whatever stream the context was given.
rketd_status step_graph(rketd_ctx* c, int64_t nsteps) {
  const int K = c->opt.variant == 3 ? -1 : c->opt.cells_per_lane, TS = c->opt.tb_steps;
  if (c->opt.variant == 3) {
    if (!c->res_ok) {
      rketd_status st = plan_resident(c);
      if (st) return st;
    }
  } else if (c->tiles_K != K || c->tiles_T != TS || c->tiles_ends != fwd_end_tiles(c)) {
    rketd_status st = plan_tiles(c, K, TS, fwd_end_tiles(c));
    if (st) return st;
  }
  if (!c->cap) {
    CK(cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking), "graph stream");
    CK(cudaEventCreateWithFlags(&c->cap_in, cudaEventDisableTiming), "graph event");
    CK(cudaEventCreateWithFlags(&c->cap_out, cudaEventDisableTiming), "graph event");
  }
  CK(cudaEventRecord(c->cap_in, c->stream), "graph fork");
  CK(cudaStreamWaitEvent(c->cap, c->cap_in, 0), "graph fork");
  rketd_ctx::GraphEntry* hit = nullptr;
  for (auto& g : c->graphs)
    if (g.s0 == c->step && g.n == nsteps && g.cur_in == c->cur && g.K == K && g.T == TS) hit = &g;
  if (!hit) {
    cudaStream_t user = c->stream;
    const int64_t s0 = c->step, l0 = c->launches;
    const int cur0 = c->cur;
    c->stream = c->cap;
    CK(cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal), "graph capture");
    rketd_status st = c->prec == RKETD_F64 ? step_impl<double>(c, nsteps) : step_impl<float>(c, nsteps);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(c->cap, &graph);
    c->stream = user;
    if (st || e != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      if (!st) st = cuda_fail(e, "graph capture");
      return st;
    }
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(e, "graph instantiate");
    if (c->graphs.size() >= 8) {
      cudaGraphExecDestroy(c->graphs.front().exec);
      c->graphs.erase(c->graphs.begin());
    }
    c->graphs.push_back({s0, nsteps, cur0, c->cur, c->launches - l0, K, TS, exec});
    hit = &c->graphs.back();
    // step_impl advanced the host-side state while recording; the replay below does the work
    c->step = s0;
    c->cur = cur0;
    c->launches = l0;
  }
  CK(cudaGraphLaunch(hit->exec, c->cap), "graph launch");
  CK(cudaEventRecord(c->cap_out, c->cap), "graph join");
  CK(cudaStreamWaitEvent(c->stream, c->cap_out, 0), "graph join");
  c->step += nsteps;
  c->cur = hit->cur_out;
  c->launches += hit->launches;
  return RKETD_OK;
}

}  // namespace

extern "C" {

void rketd_default_options(rketd_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof *o);
  o->use_graphs = 0;
}

const char* rketd_last_error(void) { return g_err.c_str(); }

const char* rketd_version(void) { return "rketd-gb300 0.1 (sm_103a)"; }

rketd_status rketd_create_batch_1d(int32_t n_slabs, const int64_t* nz, const rketd_grid1d* grid, const double* wp2,
                                   const double* nu, const int64_t* src_cell, const rketd_pulse* pulse,
                                   const int64_t* probe_cell, const rketd_dft* dft, const rketd_options* opt,
                                   void* stream, rketd_ctx** out) {
  g_err.clear();
  if (!out) return fail(RKETD_EINVAL, "out is NULL");
  *out = nullptr;
  rketd_ctx* c = new (std::nothrow) rketd_ctx();
  if (!c) return fail(RKETD_ENOMEM, "host allocation");
  rketd_status st = validate_and_copy(c, n_slabs, nz, grid, wp2, nu, src_cell, pulse, probe_cell, dft, opt);
  if (st) {
    delete c;
    return st;
  }
  c->stream = (cudaStream_t)stream;
  auto cleanup = [&](rketd_status s) {
    delete c;
    return s;
  };
  int prio_lo = 0, prio_hi = 0;
  cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
  if (cudaStreamCreateWithPriority(&c->side, cudaStreamNonBlocking, prio_hi) != cudaSuccess ||
      cudaStreamCreateWithPriority(&c->side2, cudaStreamNonBlocking, prio_hi) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->join, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->join2, cudaEventDisableTiming) != cudaSuccess)
    return cleanup(cuda_fail(cudaGetLastError(), "side stream"));
  const size_t fb = c->esz * c->n_store;
  for (int b = 0; b < 2; ++b) {
    if ((st = c->alloc(&c->E[b], fb, "E"))) return cleanup(st);
    if ((st = c->alloc(&c->H[b], fb, "H"))) return cleanup(st);
    if ((st = c->alloc(&c->J[b], fb, "J"))) return cleanup(st);
  }
  for (int k = 0; k < kNumCoef; ++k)
    if ((st = c->alloc(&c->coef[k], fb, "coefficients"))) return cleanup(st);
  if (c->grid.scheme == RKETD_SCHEME_ETD2) {
    if ((st = c->alloc(&c->Ep, fb, "E^{n-1}"))) return cleanup(st);
    for (int k = 0; k < 2; ++k)
      if ((st = c->alloc(&c->ext[k], fb, "coefficients"))) return cleanup(st);
  }
  void* p;
  if ((st = c->alloc(&p, sizeof(double) * c->n_cells, "wp2"))) return cleanup(st);
  c->wp2_d = (double*)p;
  if ((st = c->alloc(&p, sizeof(double) * c->n_cells, "nu"))) return cleanup(st);
  c->nu_d = (double*)p;
  const size_t sb = sizeof(int64_t) * n_slabs;
  if ((st = c->alloc(&p, sb, "slab table"))) return cleanup(st);
  c->soff_d = (int64_t*)p;
  if ((st = c->alloc(&p, sb, "slab table"))) return cleanup(st);
  c->off_d = (int64_t*)p;
  if ((st = c->alloc(&p, sb, "slab table"))) return cleanup(st);
  c->nz_d = (int64_t*)p;
  if ((st = c->alloc(&p, sb, "slab table"))) return cleanup(st);
  c->src_d = (int64_t*)p;
  const int nc = c->grid.bc != RKETD_BC_MUR1 ? c->grid.cpml_cells : 0;
  if (nc && c->grid.bc == RKETD_BC_PML) {
    if ((st = c->alloc(&c->cpmlE, c->esz * 2 * (nc + 1), "PML table"))) return cleanup(st);
    if ((st = c->alloc(&c->cpmlH, c->esz * 2 * nc, "PML table"))) return cleanup(st);
  } else if (nc) {
    c->n_psi = (int64_t)n_slabs * 2 * nc;
    for (int b = 0; b < 2; ++b) {
      if ((st = c->alloc(&c->psiE[b], c->esz * c->n_psi, "CPML memory"))) return cleanup(st);
      if ((st = c->alloc(&c->psiH[b], c->esz * c->n_psi, "CPML memory"))) return cleanup(st);
    }
    if ((st = c->alloc(&c->cpmlE, c->esz * 3 * (nc + 1), "CPML table"))) return cleanup(st);
    if ((st = c->alloc(&c->cpmlH, c->esz * 3 * nc, "CPML table"))) return cleanup(st);
  }
  if (c->total_probes) {
    const int P = c->total_probes, nf = c->n_freq, B = c->opt.dft_block;
    if ((st = c->alloc(&p, sizeof(int64_t) * P, "probe index"))) return cleanup(st);
    c->probe_index_d = (int64_t*)p;
    if ((st = c->alloc(&p, sizeof(double) * nf, "frequencies"))) return cleanup(st);
    c->freq_d = (double*)p;
    if ((st = c->alloc(&c->series, c->esz * (size_t)P * B, "probe series"))) return cleanup(st);
    if ((st = c->alloc(&c->tw, c->esz * 2 * (size_t)B * nf, "twiddles"))) return cleanup(st);
    if ((st = c->alloc(&p, sizeof(double) * (size_t)P * nf, "spectra"))) return cleanup(st);
    c->Xr = (double*)p;
    if ((st = c->alloc(&p, sizeof(double) * (size_t)P * nf, "spectra"))) return cleanup(st);
    c->Xi = (double*)p;
    if ((st = c->alloc(&p, sizeof(double) * 2 * (size_t)P * nf, "spectra"))) return cleanup(st);
    c->Xtmp = (double*)p;
    if ((st = c->alloc(&p, sizeof(double) * 2 * (size_t)nf, "dft rotation"))) return cleanup(st);
    c->rot = (double*)p;
    std::vector<int64_t> pi(P);
    for (int s = 0; s < n_slabs; ++s)
      for (int q = 0; q < c->n_probes; ++q) pi[s * c->n_probes + q] = c->soff[s] + c->probe_cell[s * c->n_probes + q];
    if (cudaMemcpy(c->probe_index_d, pi.data(), sizeof(int64_t) * P, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(c->freq_d, c->freq.data(), sizeof(double) * nf, cudaMemcpyHostToDevice) != cudaSuccess)
      return cleanup(cuda_fail(cudaGetLastError(), "probe upload"));
    // twiddles exp(-j 2 pi f t dt), t = 0 .. dft_block-1, shared by every fold
    cudaError_t e = c->prec == RKETD_F64
                        ? launch_twiddles<double>(c->freq_d, nf, c->grid.dt, 0, B, (double*)c->tw, c->stream)
                        : launch_twiddles<float>(c->freq_d, nf, c->grid.dt, 0, B, (float*)c->tw, c->stream);
    if (e != cudaSuccess) return cleanup(cuda_fail(e, "twiddles"));
    c->launches += 1;
  }
  if (cudaMemcpy(c->soff_d, c->soff.data(), sb, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(c->off_d, c->off.data(), sb, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(c->nz_d, c->nz.data(), sb, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(c->src_d, c->src.data(), sb, cudaMemcpyHostToDevice) != cudaSuccess)
    return cleanup(cuda_fail(cudaGetLastError(), "slab table upload"));
  // padding cells of the coefficient arrays must hold finite values: zero everything first
  for (int k = 0; k < kNumCoef; ++k)
    if (cudaMemsetAsync(c->coef[k], 0, fb, c->stream) != cudaSuccess) return cleanup(cuda_fail(cudaGetLastError(), "memset"));
  for (int k = 0; k < 2; ++k)
    if (c->ext[k] && cudaMemsetAsync(c->ext[k], 0, fb, c->stream) != cudaSuccess)
      return cleanup(cuda_fail(cudaGetLastError(), "memset"));
  if (nc) {
    cudaError_t e = c->grid.bc == RKETD_BC_PML
                        ? launch_pml_tables(c->prec, nc, c->grid.dt, c->S, c->grid.cpml_m, c->grid.cpml_sigma_max,
                                            c->cpmlE, c->cpmlH, c->stream)
                        : launch_cpml_tables(c->prec, nc, c->grid.dt, c->grid.cpml_m, c->grid.cpml_sigma_max,
                                             c->grid.cpml_kappa_max, c->grid.cpml_alpha_max, c->cpmlE, c->cpmlH,
                                             c->stream);
    if (e != cudaSuccess) return cleanup(cuda_fail(e, "CPML tables"));
    c->launches += 1;
  }
  if ((st = zero_state(c))) return cleanup(st);
  if ((st = rketd_set_medium(c, wp2, nu, 0))) return cleanup(st);
  // resident variant: where asked for, or under auto where it applies
  if (c->opt.variant == 3 || (c->auto_variant && c->opt.variant == 2)) {
    st = plan_resident(c);
    if (st == RKETD_OK) {
      c->opt.variant = 3;
    } else if (c->opt.variant == 3) {
      return cleanup(st);
    } else {
      g_err.clear();
    }
  }
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return cleanup(cuda_fail(cudaGetLastError(), "create"));
  *out = c;
  return RKETD_OK;
}

rketd_status rketd_create_1d(int64_t nz, const rketd_grid1d* grid, const double* wp2, const double* nu,
                             int64_t src_cell, const rketd_pulse* pulse, const int64_t* probe_cell,
                             const rketd_dft* dft, const rketd_options* opt, void* stream, rketd_ctx** out) {
  return rketd_create_batch_1d(1, &nz, grid, wp2, nu, &src_cell, pulse, probe_cell, dft, opt, stream, out);
}

rketd_status rketd_set_medium(rketd_ctx* c, const double* wp2, const double* nu, int32_t on_device) {
  if (!c || !wp2 || !nu) return fail(RKETD_EINVAL, "NULL argument");
  const size_t b = sizeof(double) * c->n_cells;
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  CK(cudaMemcpyAsync(c->wp2_d, wp2, b, kind, c->stream), "medium upload");
  CK(cudaMemcpyAsync(c->nu_d, nu, b, kind, c->stream), "medium upload");
  // The state carries the folded current G = cj J~ - da E; J~ stays unchanged across the medium
  // change. The old cj and da are parked in the other (unused) ping-pong copies of J and H.
  void* old_cj = c->J[1 - c->cur];
  void* old_da = c->H[1 - c->cur];
  CK(cudaMemcpyAsync(old_cj, c->coef[kCj], c->esz * c->n_store, cudaMemcpyDeviceToDevice, c->stream), "medium");
  CK(cudaMemcpyAsync(old_da, c->coef[kDa], c->esz * c->n_store, cudaMemcpyDeviceToDevice, c->stream), "medium");
  rketd_status st = update_coeffs(c);
  if (st) return st;
  CK(launch_rescale(c->prec, c->J[c->cur], c->E[c->cur], c->coef[kCj], old_cj, c->coef[kDa], old_da, c->n_store,
                    c->stream),
     "current rescale");
  c->launches += 1;
  return RKETD_OK;
}

rketd_status rketd_reset(rketd_ctx* c) {
  if (!c) return fail(RKETD_EINVAL, "NULL context");
  return zero_state(c);
}

rketd_status rketd_step(rketd_ctx* c, int64_t nsteps) {
  if (!c) return fail(RKETD_EINVAL, "NULL context");
  if (nsteps < 0) return fail(RKETD_EINVAL, "nsteps < 0");
  if (nsteps == 0) return RKETD_OK;
  const bool graphs =
      c->opt.use_graphs != 2 && !c->timing && (c->opt.variant == 2 || c->opt.variant == 3 || c->opt.variant == 4);
  if (!graphs) return c->prec == RKETD_F64 ? step_impl<double>(c, nsteps) : step_impl<float>(c, nsteps);
  return step_graph(c, nsteps);
}

rketd_status rketd_sync(rketd_ctx* c) {
  if (!c) return fail(RKETD_EINVAL, "NULL context");
  CK(cudaStreamSynchronize(c->stream), "stream synchronize");
  CK(cudaGetLastError(), "device error");
  if (c->err_d) {
    int e = 0;
    CK(cudaMemcpy(&e, c->err_d, sizeof(int), cudaMemcpyDeviceToHost), "status word");
    if (e) return fail(RKETD_ETIMEOUT, "a wait of the persistent step gave up; fields are not valid");
  }
  return RKETD_OK;
}

rketd_status rketd_set_wait_limit(rketd_ctx* c, int32_t polls) {
  if (!c) return fail(RKETD_EINVAL, "NULL context");
  c->wait_limit = polls < 0 ? (1 << 22) : polls;
  for (auto& g : c->graphs) cudaGraphExecDestroy(g.exec);  // the limit is a launch argument
  c->graphs.clear();
  return RKETD_OK;
}

int64_t rketd_step_index(const rketd_ctx* c) { return c ? c->step : -1; }

int64_t rketd_launch_count(const rketd_ctx* c) { return c ? c->launches : -1; }

rketd_status rketd_check_finite(rketd_ctx* c) {
  if (!c) return fail(RKETD_EINVAL, "NULL context");
  int* flag = nullptr;
  CK(device_alloc_async((void**)&flag, sizeof(int), c->stream), "finite scan");
  rketd_status st = RKETD_OK;
  cudaError_t e = cudaMemsetAsync(flag, 0, sizeof(int), c->stream);
  const bool f64 = c->prec == RKETD_F64;
  const void* arrs[6] = {c->E[c->cur], c->H[c->cur], c->J[c->cur], c->Ep, c->psiE[c->cur], c->psiH[c->cur]};
  const int64_t lens[6] = {c->n_store, c->n_store, c->n_store, c->Ep ? c->n_store : 0, c->psiE[c->cur] ? c->n_psi : 0,
                           c->psiH[c->cur] ? c->n_psi : 0};
  for (int q = 0; q < 6 && e == cudaSuccess; ++q) e = launch_finite_scan(f64, arrs[q], lens[q], flag, c->stream);
  const int64_t nx = (int64_t)c->total_probes * c->n_freq;
  if (e == cudaSuccess && nx) e = launch_finite_scan(true, c->Xr, nx, flag, c->stream);
  if (e == cudaSuccess && nx) e = launch_finite_scan(true, c->Xi, nx, flag, c->stream);
  int h = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
  cudaFreeAsync(flag, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(e, "finite scan");
  if (h) st = fail(RKETD_ENUMERIC, "a field, CPML memory or spectrum holds NaN or Inf");
  return st;
}

rketd_status rketd_debug_fail_alloc(int64_t after) {
  std::lock_guard<std::mutex> lk(g_alloc_mu);
  g_alloc_fail_after = after < 0 ? -1 : after;
  return RKETD_OK;
}

int64_t rketd_debug_alloc_count(void) {
  std::lock_guard<std::mutex> lk(g_alloc_mu);
  return g_alloc_count;
}

rketd_status rketd_get_fields(rketd_ctx* c, int32_t slab, double* E, double* H, double* J) {
  if (!c) return fail(RKETD_EINVAL, "NULL context");
  if (slab < 0 || slab >= c->n_slabs) return fail(RKETD_EINVAL, "slab index out of range");
  const int64_t nz = c->nz[slab];
  double* tmp;
  CK(device_alloc_async((void**)&tmp, sizeof(double) * 3 * nz, c->stream), "field staging");
  const double hs = 1.0 / std::sqrt(kMu0 / kEps0);
  const double js = kEps0 / c->grid.dt;
  cudaError_t e = launch_gather_fields(c->prec, c->E[c->cur], c->H[c->cur], c->J[c->cur], c->coef[kCj],
                                       c->coef[kDa], c->soff[slab], nz, hs, js, tmp, tmp + nz, tmp + 2 * nz,
                                       c->stream);
  c->launches += 1;
  if (e == cudaSuccess && E) e = cudaMemcpyAsync(E, tmp, sizeof(double) * nz, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess && H)
    e = cudaMemcpyAsync(H, tmp + nz, sizeof(double) * (nz - 1), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess && J)
    e = cudaMemcpyAsync(J, tmp + 2 * nz, sizeof(double) * nz, cudaMemcpyDeviceToHost, c->stream);
  cudaFreeAsync(tmp, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(e, "get_fields");
  return RKETD_OK;
}

rketd_status rketd_get_spectra_device(rketd_ctx* c, double* re, double* im) {
  if (!c || !re || !im) return fail(RKETD_EINVAL, "NULL argument");
  const size_t n = (size_t)c->total_probes * c->n_freq;
  if (n == 0) return RKETD_OK;
  CK(cudaMemcpyAsync(re, c->Xr, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream), "spectra copy");
  CK(cudaMemcpyAsync(im, c->Xi, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream), "spectra copy");
  const int pending = c->pos();
  if (pending) {
    rketd_status st = c->prec == RKETD_F64 ? dft_block<double>(c, pending, c->step - pending + 1, re, im)
                                          : dft_block<float>(c, pending, c->step - pending + 1, re, im);
    if (st) return st;
  }
  return RKETD_OK;
}

rketd_status rketd_get_spectra(rketd_ctx* c, double* re, double* im) {
  if (!c || !re || !im) return fail(RKETD_EINVAL, "NULL argument");
  const size_t n = (size_t)c->total_probes * c->n_freq;
  if (n == 0) return RKETD_OK;
  rketd_status st = rketd_get_spectra_device(c, c->Xtmp, c->Xtmp + n);
  if (st) return st;
  CK(cudaMemcpyAsync(re, c->Xtmp, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream), "spectra D2H");
  CK(cudaMemcpyAsync(im, c->Xtmp + n, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream), "spectra D2H");
  CK(cudaStreamSynchronize(c->stream), "spectra sync");
  return RKETD_OK;
}

rketd_status rketd_rt(const double* tr, const double* ti, const double* ir, const double* ii, int32_t n,
                      double* Rr, double* Ri, double* Tr, double* Ti) {
  if (!tr || !ti || !ir || !ii || n < 1) return fail(RKETD_EINVAL, "invalid arguments");
  // probe 0 = reflection (tot - inc)/inc, probe 1 = transmission tot/inc; arrays are [2][n]
  for (int f = 0; f < n; ++f) {
    for (int p = 0; p < 2; ++p) {
      double* Or = p == 0 ? Rr : Tr;
      double* Oi = p == 0 ? Ri : Ti;
      if (!Or || !Oi) continue;
      const double ar = p == 0 ? tr[f] - ir[f] : tr[n + f];
      const double ai = p == 0 ? ti[f] - ii[f] : ti[n + f];
      const double br = ir[p * n + f], bi = ii[p * n + f];
      const double d = br * br + bi * bi;
      if (!(d > 0)) return fail(RKETD_ENUMERIC, "incident spectrum is zero at frequency %d", f);
      Or[f] = (ar * br + ai * bi) / d;
      Oi[f] = (ai * br - ar * bi) / d;
    }
  }
  return RKETD_OK;
}

}  // extern "C"

namespace {

// Version 2: the current is stored as the folded G = cj J~ - da E (version 1 held cj J~).
// Version 3: the header names the current recursion; the Eq. 10 recursion adds E^{n-1}.
constexpr int32_t kStateVersion = 3;

struct StateHeader {
  char magic[8];
  int32_t version, prec, n_slabs, n_probes, n_freq, dft_block;
  int64_t n_store, n_psi, step;
  int32_t scheme, pad;
};

bool write_dev(FILE* f, const void* dev, size_t bytes, cudaStream_t st) {
  if (!bytes) return true;
  std::vector<char> h(bytes);
  if (cudaMemcpyAsync(h.data(), dev, bytes, cudaMemcpyDeviceToHost, st) != cudaSuccess) return false;
  if (cudaStreamSynchronize(st) != cudaSuccess) return false;
  return fwrite(h.data(), 1, bytes, f) == bytes;
}

bool read_dev(FILE* f, void* dev, size_t bytes, cudaStream_t st) {
  if (!bytes) return true;
  std::vector<char> h(bytes);
  if (fread(h.data(), 1, bytes, f) != bytes) return false;
  if (cudaMemcpyAsync(dev, h.data(), bytes, cudaMemcpyHostToDevice, st) != cudaSuccess) return false;
  return cudaStreamSynchronize(st) == cudaSuccess;
}

StateHeader header_of(const rketd_ctx* c) {
  StateHeader h{};
  std::memcpy(h.magic, "RKETDST1", 8);
  h.version = kStateVersion;
  h.prec = c->prec;
  h.n_slabs = c->n_slabs;
  h.n_probes = c->n_probes;
  h.n_freq = c->n_freq;
  h.dft_block = c->opt.dft_block;
  h.n_store = c->n_store;
  h.n_psi = c->n_psi;
  h.step = c->step;
  h.scheme = c->grid.scheme;
  return h;
}

}  // namespace

extern "C" {

rketd_status rketd_save_state(rketd_ctx* c, const char* path) {
  if (!c || !path) return fail(RKETD_EINVAL, "NULL argument");
  CK(cudaStreamSynchronize(c->stream), "save_state sync");
  FILE* f = fopen(path, "wb");
  if (!f) return fail(RKETD_EIO, "cannot open %s for writing", path);
  const StateHeader h = header_of(c);
  const size_t fb = c->esz * c->n_store, pb = c->esz * c->n_psi;
  const size_t xb = sizeof(double) * c->total_probes * c->n_freq;
  const size_t sb = c->esz * (size_t)c->total_probes * c->opt.dft_block;
  bool ok = fwrite(&h, sizeof h, 1, f) == 1 && write_dev(f, c->E[c->cur], fb, c->stream) &&
            write_dev(f, c->H[c->cur], fb, c->stream) && write_dev(f, c->J[c->cur], fb, c->stream) &&
            (!pb || (write_dev(f, c->psiE[c->cur], pb, c->stream) && write_dev(f, c->psiH[c->cur], pb, c->stream))) &&
            (!xb || (write_dev(f, c->Xr, xb, c->stream) && write_dev(f, c->Xi, xb, c->stream) &&
                     write_dev(f, c->series, sb, c->stream))) &&
            (!c->Ep || write_dev(f, c->Ep, fb, c->stream));
  ok = (fclose(f) == 0) && ok;
  if (!ok) return fail(RKETD_EIO, "writing %s failed", path);
  return RKETD_OK;
}

rketd_status rketd_load_state(rketd_ctx* c, const char* path) {
  if (!c || !path) return fail(RKETD_EINVAL, "NULL argument");
  FILE* f = fopen(path, "rb");
  if (!f) return fail(RKETD_EIO, "cannot open %s", path);
  StateHeader h{};
  const StateHeader want = header_of(c);
  if (fread(&h, sizeof h, 1, f) != 1 || std::memcmp(h.magic, want.magic, 8) || h.version != kStateVersion) {
    fclose(f);
    return fail(RKETD_EIO, "%s is not an RKETD state file", path);
  }
  if (h.prec != want.prec || h.n_slabs != want.n_slabs || h.n_probes != want.n_probes || h.n_freq != want.n_freq ||
      h.dft_block != want.dft_block || h.n_store != want.n_store || h.n_psi != want.n_psi || h.step < 0 ||
      h.scheme != want.scheme) {
    fclose(f);
    return fail(RKETD_EINVAL, "%s was saved from a context of a different shape", path);
  }
  CK(cudaStreamSynchronize(c->stream), "load_state sync");
  c->cur = 0;
  const size_t fb = c->esz * c->n_store, pb = c->esz * c->n_psi;
  const size_t xb = sizeof(double) * c->total_probes * c->n_freq;
  const size_t sb = c->esz * (size_t)c->total_probes * c->opt.dft_block;
  bool ok = read_dev(f, c->E[0], fb, c->stream) && read_dev(f, c->H[0], fb, c->stream) &&
            read_dev(f, c->J[0], fb, c->stream) &&
            (!pb || (read_dev(f, c->psiE[0], pb, c->stream) && read_dev(f, c->psiH[0], pb, c->stream))) &&
            (!xb || (read_dev(f, c->Xr, xb, c->stream) && read_dev(f, c->Xi, xb, c->stream) &&
                     read_dev(f, c->series, sb, c->stream))) &&
            (!c->Ep || read_dev(f, c->Ep, fb, c->stream));
  fclose(f);
  if (!ok) return fail(RKETD_EIO, "reading %s failed", path);
  c->step = h.step;
  return RKETD_OK;
}

rketd_status rketd_autotune(rketd_ctx* c, int32_t passes) {
  if (!c) return fail(RKETD_EINVAL, "NULL context");
  if (passes < 1) return fail(RKETD_EINVAL, "passes must be >= 1");
  if (c->grid.scheme == RKETD_SCHEME_ETD2)
    return fail(RKETD_EUNSUPPORTED, "the autotuner times the tiled variant, which the Eq. 10 recursion does not run on");
  CK(cudaStreamSynchronize(c->stream), "autotune sync");
  // save the state
  const size_t fb = c->esz * c->n_store, pb = c->esz * c->n_psi;
  const size_t xb = sizeof(double) * c->total_probes * c->n_freq;
  const size_t sb = c->esz * (size_t)c->total_probes * c->opt.dft_block;
  std::vector<std::pair<void*, size_t>> saved;
  auto save = [&](void* src, size_t bytes) -> rketd_status {
    void* d = nullptr;
    if (!bytes) { saved.push_back({nullptr, 0}); return RKETD_OK; }
    CK(device_alloc(&d, bytes), "autotune save");
    saved.push_back({d, bytes});
    CK(cudaMemcpyAsync(d, src, bytes, cudaMemcpyDeviceToDevice, c->stream), "autotune save");
    return RKETD_OK;
  };
  void* srcs[8] = {c->E[c->cur], c->H[c->cur], c->J[c->cur], c->psiE[c->cur], c->psiH[c->cur], c->Xr, c->Xi, c->series};
  size_t sizes[8] = {fb, fb, fb, pb, pb, xb, xb, sb};
  rketd_status st = RKETD_OK;
  for (int i = 0; i < 8 && !st; ++i) st = save(srcs[i], sizes[i]);
  const int64_t step0 = c->step;
  const int cur0 = c->cur;
  const rketd_options opt0 = c->opt;
  std::vector<std::array<int, 3>> cands;
  const std::vector<int> Ks32 = {8, 12, 16}, Ks64 = {4, 8};
  const int Ts[] = {8, 16, 24, 32, 48, 64};
  for (int K : (c->prec == RKETD_F64 ? Ks64 : Ks32))
    for (int T : Ts)
      for (int w : {1, 2, 4})
        if (32 * K - 2 * T >= 64 && opt0.dft_block % T == 0) cands.push_back({K, T, w});
  float best_ms = 1e30f;
  rketd_options best = opt0;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (!st && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
    st = cuda_fail(cudaGetLastError(), "autotune events");
  const int64_t nsteps = (int64_t)passes * 64;
  // a persistent context tunes the persistent step's tile shape; any other the tiled variant's
  const int tuned = opt0.variant == 4 ? 4 : 2;
  for (size_t i = 0; i < cands.size() && !st; ++i) {
    c->opt.variant = tuned;
    c->opt.use_graphs = 2;
    c->opt.cells_per_lane = cands[i][0];
    c->opt.tb_steps = cands[i][1];
    c->opt.warps_per_block = cands[i][2];
    st = rketd_step(c, cands[i][1]);  // warm-up and tile planning
    if (st) break;
    if (cudaEventRecord(e0, c->stream) != cudaSuccess) { st = cuda_fail(cudaGetLastError(), "autotune"); break; }
    st = rketd_step(c, nsteps);
    if (st) break;
    if (cudaEventRecord(e1, c->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
      st = cuda_fail(cudaGetLastError(), "autotune");
      break;
    }
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best_ms) {
      best_ms = ms;
      best = c->opt;
    }
  }
  // the resident variant, where it applies, is one more candidate
  if (!st && tuned == 2 && c->n_slabs == 1 && c->grid.bc == RKETD_BC_MUR1 && c->grid.scheme != RKETD_SCHEME_ETD2) {
    c->opt = opt0;
    c->opt.variant = 3;
    c->opt.use_graphs = 2;
    if (plan_resident(c) == RKETD_OK) {
      st = rketd_step(c, 64);  // warm-up
      if (!st && cudaEventRecord(e0, c->stream) != cudaSuccess) st = cuda_fail(cudaGetLastError(), "autotune");
      if (!st) st = rketd_step(c, nsteps);
      if (!st && (cudaEventRecord(e1, c->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess))
        st = cuda_fail(cudaGetLastError(), "autotune");
      float ms = 0;
      if (!st && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms < best_ms) {
        best_ms = ms;
        best = c->opt;
      }
    } else {
      g_err.clear();
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  // restore the state
  c->opt = st ? opt0 : best;
  c->opt.use_graphs = opt0.use_graphs;
  c->step = step0;
  c->cur = cur0;
  void* dsts[8] = {c->E[c->cur], c->H[c->cur], c->J[c->cur], c->psiE[c->cur], c->psiH[c->cur], c->Xr, c->Xi, c->series};
  for (size_t i = 0; i < saved.size(); ++i) {
    if (saved[i].first) {
      cudaMemcpyAsync(dsts[i], saved[i].first, saved[i].second, cudaMemcpyDeviceToDevice, c->stream);
      cudaStreamSynchronize(c->stream);
      cudaFree(saved[i].first);
    }
  }
  return st;
}

rketd_status rketd_forward_ckpt(rketd_ctx* c, int64_t nsteps, int32_t ckpt_every) {
  if (!c) return fail(RKETD_EINVAL, "NULL context");
  if (nsteps < 1 || ckpt_every < 1) return fail(RKETD_EINVAL, "nsteps and ckpt_every must be >= 1");
  if (c->grid.bc != RKETD_BC_MUR1) return fail(RKETD_EUNSUPPORTED, "the adjoint supports first-order Mur ends only");
  if (c->grid.scheme != RKETD_SCHEME_RKETD)
    return fail(RKETD_EUNSUPPORTED, "the adjoint differentiates the Eq. 11 recursion only");
  if (c->opt.variant == 3 || c->opt.variant == 4) c->opt.variant = 2;  // the checkpointed run and the adjoint use the tiled kernels
  if (c->opt.variant != 2) return fail(RKETD_EUNSUPPORTED, "the adjoint runs on the tiled variant");
  const int64_t n_ckpt = (nsteps + ckpt_every - 1) / ckpt_every;
  const size_t fb = c->esz * c->n_store;
  if (n_ckpt != c->n_ckpt) {
    if (c->ckpt) {
      cudaFree(c->ckpt);
      c->allocs.erase(std::find(c->allocs.begin(), c->allocs.end(), c->ckpt));
      c->ckpt = nullptr;
    }
    rketd_status st = c->alloc(&c->ckpt, 3 * fb * n_ckpt, "checkpoints");
    if (st) return st;
    c->n_ckpt = n_ckpt;
  }
  rketd_status st = zero_state(c);
  if (st) return st;
  for (int64_t j = 0; j < n_ckpt; ++j) {
    char* dst = (char*)c->ckpt + 3 * fb * j;
    CK(cudaMemcpyAsync(dst, c->E[c->cur], fb, cudaMemcpyDeviceToDevice, c->stream), "checkpoint");
    CK(cudaMemcpyAsync(dst + fb, c->H[c->cur], fb, cudaMemcpyDeviceToDevice, c->stream), "checkpoint");
    CK(cudaMemcpyAsync(dst + 2 * fb, c->J[c->cur], fb, cudaMemcpyDeviceToDevice, c->stream), "checkpoint");
    // direct launches: every segment starts at a different step, so per-call graphs would not repeat
    const int64_t n = std::min<int64_t>(ckpt_every, nsteps - j * ckpt_every);
    c->in_ckpt = true;  // the edge-tile plan that the adjoint's recompute mirrors
    st = c->prec == RKETD_F64 ? step_impl<double>(c, n) : step_impl<float>(c, n);
    c->in_ckpt = false;
    if (st) return st;
  }
  c->ckpt_steps = nsteps;
  c->ckpt_every = ckpt_every;
  return RKETD_OK;
}

}  // extern "C"

namespace {

template <typename T>
rketd_status adjoint_impl(rketd_ctx* c, int64_t w_lo, int64_t w_hi, double* grad_wp2, double* grad_nu) {
  const int64_t N = c->ckpt_steps, C = c->ckpt_every;
  const int K = c->opt.cells_per_lane, TS = c->opt.tb_steps, Ke = edge_cells_per_lane(TS);
  // recorded rows start 4 cells before the window (its left neighbour, needed for dH, at index 3)
  // and have a width that is a multiple of 4, so that whole aligned groups are stored as vectors
  const int64_t nwin = w_hi - w_lo;
  const int64_t rw = ((nwin + 4 + 3) / 4) * 4;
  const int64_t r0 = w_lo - 4;
  const size_t fb = c->esz * c->n_store;
  const int P = c->total_probes, nf = c->n_freq;
  if (c->tiles_K != K || c->tiles_T != TS || c->tiles_ends) {
    rketd_status st = plan_tiles(c, K, TS);
    if (st) return st;
  }
  rketd_status st;
  if (c->adj_w_lo != w_lo || c->adj_w_hi != w_hi || !c->adj_tiles_d) {
    // interior tiles whose exact cells miss the recorded cells run the plain kernels
    std::vector<Tile> plain, win;
    for (int i = 0; i < c->n_interior; ++i) {
      const Tile& t = c->tiles_h[i];
      const int64_t v0 = t.start + t.vlo, v1 = t.start + t.vhi;
      // (tiles that load a source cell run the recording kernel, which has the source code)
      (t.src_local < 0 && (v1 <= w_lo - 4 || v0 >= w_lo - 4 + ((w_hi - w_lo + 7) / 4) * 4) ? plain : win)
          .push_back(t);
    }
    std::vector<Tile> order = plain;
    order.insert(order.end(), win.begin(), win.end());
    order.insert(order.end(), c->tiles_h.begin() + c->n_interior, c->tiles_h.end());
    if (c->adj_tiles_d) cudaFree(c->adj_tiles_d);
    c->adj_tiles_d = nullptr;
    CK(device_alloc((void**)&c->adj_tiles_d, sizeof(Tile) * std::max<size_t>(1, order.size())), "adjoint tiles");
    CK(cudaMemcpy(c->adj_tiles_d, order.data(), sizeof(Tile) * order.size(), cudaMemcpyHostToDevice), "adjoint tiles");
    c->adj_n_plain = (int)plain.size();
    c->adj_n_win = (int)win.size();
    c->adj_w_lo = w_lo;
    c->adj_w_hi = w_hi;
  }
  const Tile* t_plain = c->adj_tiles_d;
  const Tile* t_win = c->adj_tiles_d + c->adj_n_plain;
  const Tile* t_edge = t_win + c->adj_n_win;
  // window tiles on the side stream, edge tiles on the second side stream
  auto fork = [&]() -> rketd_status {
    CK(cudaEventRecord(c->fork, c->stream), "fork");
    CK(cudaStreamWaitEvent(c->side, c->fork, 0), "fork");
    CK(cudaStreamWaitEvent(c->side2, c->fork, 0), "fork");
    return RKETD_OK;
  };
  auto join = [&]() -> rketd_status {
    CK(cudaEventRecord(c->join, c->side), "join");
    CK(cudaEventRecord(c->join2, c->side2), "join");
    CK(cudaStreamWaitEvent(c->stream, c->join, 0), "join");
    CK(cudaStreamWaitEvent(c->stream, c->join2, 0), "join");
    return RKETD_OK;
  };
  if (!c->lam[0])
    for (int i = 0; i < 6; ++i)
      if ((st = c->alloc(&c->lam[i], fb, "adjoint fields"))) return st;
  if (!c->gstream) {
    int lo = 0, hi = 0;
    CK(cudaDeviceGetStreamPriorityRange(&lo, &hi), "gradient stream");
    CK(cudaStreamCreateWithPriority(&c->gstream, cudaStreamNonBlocking, lo), "gradient stream");
    CK(cudaEventCreateWithFlags(&c->ev_adj, cudaEventDisableTiming), "gradient events");
    CK(cudaEventCreateWithFlags(&c->ev_seed, cudaEventDisableTiming), "gradient events");
    for (cudaEvent_t& e : c->ev_grad) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "gradient events");
  }
  if (rw > c->rec_cap) {
    for (void** p : {&c->recF, &c->recA, &c->recF2, &c->recA2, &c->seeds, &c->tw_seed, &c->seeds2, &c->tw_seed2,
                     (void**)&c->gacc}) {
      if (*p) {
        cudaFree(*p);
        c->allocs.erase(std::find(c->allocs.begin(), c->allocs.end(), *p));
        *p = nullptr;
      }
    }
    if ((st = c->alloc(&c->recF, c->esz * (size_t)c->n_slabs * (C + 1) * 3 * rw, "adjoint records"))) return st;
    if ((st = c->alloc(&c->recA, c->esz * (size_t)c->n_slabs * C * 2 * rw, "adjoint records"))) return st;
    if ((st = c->alloc(&c->recF2, c->esz * (size_t)c->n_slabs * (C + 1) * 3 * rw, "adjoint records"))) return st;
    if ((st = c->alloc(&c->recA2, c->esz * (size_t)c->n_slabs * C * 2 * rw, "adjoint records"))) return st;
    if ((st = c->alloc(&c->seeds, c->esz * (size_t)std::max(P, 1) * C, "adjoint seeds"))) return st;
    if ((st = c->alloc(&c->tw_seed, c->esz * 2 * (size_t)C * std::max(nf, 1), "adjoint twiddles"))) return st;
    if ((st = c->alloc(&c->seeds2, c->esz * (size_t)std::max(P, 1) * C, "adjoint seeds"))) return st;
    if ((st = c->alloc(&c->tw_seed2, c->esz * 2 * (size_t)C * std::max(nf, 1), "adjoint twiddles"))) return st;
    void* g;
    if ((st = c->alloc(&g, sizeof(double) * 5 * (size_t)c->n_slabs * nwin, "gradient sums"))) return st;
    c->gacc = (double*)g;
    c->rec_cap = rw;
  }
  for (int i = 0; i < 6; ++i) CK(cudaMemsetAsync(c->lam[i], 0, fb, c->stream), "adjoint init");
  CK(cudaMemsetAsync(c->gacc, 0, sizeof(double) * 5 * (size_t)c->n_slabs * nwin, c->stream), "adjoint init");
  int lcur = 0;
  const int64_t n_seg = (N + C - 1) / C;
  // loss seeds for the samples after steps n0 .. n0+L-1 of a segment, made on the gradient
  // stream one segment ahead of the transposed sweep that reads them (two buffers)
  auto make_seeds = [&](int64_t seg) -> rketd_status {
    if (P == 0 || seg < 0) return RKETD_OK;
    const int64_t m0 = seg * C;
    const int Ls = (int)std::min<int64_t>(C, N - m0);
    const int b = (int)((n_seg - 1 - seg) & 1);
    T* tw = (T*)(b ? c->tw_seed2 : c->tw_seed);
    CK(launch_twiddles<T>(c->freq_d, nf, c->grid.dt, m0 + 1, Ls, tw, c->gstream), "seed twiddles");
    CK(launch_seeds<T>(c->gX, c->gX + (size_t)P * nf, tw, P, nf, Ls, (T*)(b ? c->seeds2 : c->seeds), Ls, c->gstream),
       "seeds");
    CK(cudaEventRecord(c->ev_seed, c->gstream), "seeds done");
    c->launches += 2;
    return RKETD_OK;
  };
  CK(cudaEventRecord(c->ev_adj, c->stream), "adjoint inputs");
  CK(cudaStreamWaitEvent(c->gstream, c->ev_adj, 0), "adjoint inputs");
  if ((st = make_seeds(n_seg - 1))) return st;
  for (int64_t seg = n_seg - 1; seg >= 0; --seg) {
    const int64_t n0 = seg * C;
    const int L = (int)std::min<int64_t>(C, N - n0);
    // record set of this segment; the gradient sums of the segment that used it last must be done
    const int rb = (int)((n_seg - 1 - seg) & 1);
    void* recF = rb ? c->recF2 : c->recF;
    void* recA = rb ? c->recA2 : c->recA;
    if (n_seg - 1 - seg >= 2) CK(cudaStreamWaitEvent(c->stream, c->ev_grad[rb], 0), "record reuse");
    // restore the checkpoint and recompute the segment, recording the window
    const char* src = (const char*)c->ckpt + 3 * fb * seg;
    CK(cudaMemcpyAsync(c->E[0], src, fb, cudaMemcpyDeviceToDevice, c->stream), "restore");
    CK(cudaMemcpyAsync(c->H[0], src + fb, fb, cudaMemcpyDeviceToDevice, c->stream), "restore");
    CK(cudaMemcpyAsync(c->J[0], src + 2 * fb, fb, cudaMemcpyDeviceToDevice, c->stream), "restore");
    c->cur = 0;
    CK(launch_rec_init<T>((const T*)c->E[0], (const T*)c->H[0], (const T*)c->J[0], c->soff_d, c->nz_d, c->n_slabs, r0,
                          (int)rw, L + 1, (T*)recF, c->stream),
       "record init");
    c->launches += 1;
    for (int done = 0; done < L;) {
      const int nsub = std::min(TS, L - done);
      c->step = n0 + done;
      StepArgs<T> a = make_args<T>(c, c->cur, 1 - c->cur);
      a.nsub = nsub;
      a.series = nullptr;
      a.tprobes = c->tprobes_d;
      a.rec = (T*)recF;
      a.rec_c0 = r0;
      a.rec_w = (int)rw;
      a.rec_len = L + 1;
      a.rec_pos = done + 1;
      if ((st = fork())) return st;
      // window and edge tiles (recording) on the side stream, the rest with the plain kernels
      a.tiles = t_win;
      a.n_tiles = c->adj_n_win;
      CK(launch_tb_rec<T>(a, K, false, 2, c->side), "recompute (window)");
      a.tiles = t_edge;
      a.n_tiles = c->n_edge;
      CK(launch_tb_rec<T>(a, Ke, true, 2, c->side2), "recompute (edge)");
      a.tiles = t_plain;
      a.n_tiles = c->adj_n_plain;
      if (std::is_same<T, float>::value && c->opt.fp32_pairs != 2 && K % 4 == 0) {
        CK(launch_tb_pairs(*reinterpret_cast<const StepArgs<float>*>(&a), K, c->opt.warps_per_block, c->stream,
                           false),
           "recompute (interior)");
      } else {
        CK(launch_tb<T>(a, K, false, c->opt.warps_per_block, c->stream, false), "recompute (interior)");
      }
      if ((st = join())) return st;
      c->launches += 3;
      c->cur = 1 - c->cur;
      done += nsub;
    }
    // this segment's loss seeds (made on the gradient stream)
    const T* seeds = (const T*)(rb ? c->seeds2 : c->seeds);
    if (P > 0) CK(cudaStreamWaitEvent(c->stream, c->ev_seed, 0), "seeds ready");
    // transposed passes from the end of the segment back to its start
    for (int hi = L; hi > 0;) {
      const int nsub = std::min(TS, hi);
      AdjArgs<T> a{};
      a.lE_in = (const T*)c->lam[3 * lcur];
      a.lH_in = (const T*)c->lam[3 * lcur + 1];
      a.lJ_in = (const T*)c->lam[3 * lcur + 2];
      a.lE_out = (T*)c->lam[3 * (1 - lcur)];
      a.lH_out = (T*)c->lam[3 * (1 - lcur) + 1];
      a.lJ_out = (T*)c->lam[3 * (1 - lcur) + 2];
      for (int k = 0; k < kNumCoef; ++k) a.coef[k] = (const T*)c->coef[k];
      a.soff = c->soff_d;
      a.nz = c->nz_d;
      a.S = (T)c->S;
      a.qmur = (T)c->qmur;
      a.nsub = nsub;
      a.n_hi = n0 + hi;
      a.seg_n0 = n0;
      a.seeds = seeds;
      a.seed_len = L;
      a.tprobes = c->tprobes_d;
      a.rec = (T*)recA;
      a.rec_c0 = r0;
      a.rec_w = (int)rw;
      a.rec_len = L;
      if ((st = fork())) return st;
      a.tiles = t_win;
      a.n_tiles = c->adj_n_win;
      CK(launch_adj<T>(a, K, false, 2, c->side), "adjoint (window)");
      a.tiles = t_edge;
      a.n_tiles = c->n_edge;
      CK(launch_adj<T>(a, Ke, true, 2, c->side2), "adjoint (edge)");
      a.tiles = t_plain;
      a.n_tiles = c->adj_n_plain;
      a.rec = nullptr;
      if (std::is_same<T, float>::value && c->opt.fp32_pairs != 2 && K % 4 == 0) {
        CK(launch_adj_pairs(*reinterpret_cast<const AdjArgs<float>*>(&a), K, c->opt.warps_per_block, c->stream),
           "adjoint (interior, FP32 pairs)");
      } else {
        CK(launch_adj<T>(a, K, false, 2, c->stream), "adjoint (interior)");
      }
      if ((st = join())) return st;
      c->launches += 3;
      lcur = 1 - lcur;
      hi -= nsub;
    }
    // the segment's gradient sums on the gradient stream (in segment order, so the FP64 totals
    // add up in the same order as on one stream), overlapping the next segment
    const GradSource gs{c->src_d, w_lo, n0, c->grid.dt, c->pulse.t0, c->pulse.tau, c->pulse.amp};
    CK(cudaEventRecord(c->ev_adj, c->stream), "segment done");
    CK(cudaStreamWaitEvent(c->gstream, c->ev_adj, 0), "segment done");
    CK(launch_grad_accum<T>((const T*)recF, (const T*)recA, c->n_slabs, (int)rw, (int)nwin, L, L + 1, gs, c->gacc,
                            c->gstream),
       "gradient sums");
    CK(cudaEventRecord(c->ev_grad[rb], c->gstream), "gradient sums done");
    c->launches += 1;
    if ((st = make_seeds(seg - 1))) return st;
  }
  CK(cudaEventRecord(c->ev_adj, c->gstream), "gradient sums done");
  CK(cudaStreamWaitEvent(c->stream, c->ev_adj, 0), "gradient sums done");
  CK(cudaMemsetAsync(grad_wp2, 0, sizeof(double) * c->n_cells, c->stream), "gradient init");
  CK(cudaMemsetAsync(grad_nu, 0, sizeof(double) * c->n_cells, c->stream), "gradient init");
  CK(launch_grad_chain(c->gacc, c->wp2_d, c->nu_d, c->off_d, c->n_slabs, w_lo, (int)nwin, c->grid.dt, c->S,
                       grad_wp2, grad_nu, c->stream),
     "chain rule");
  c->launches += 1;
  c->step = -1;  // the fields hold a recomputed intermediate state
  return RKETD_OK;
}

}  // namespace

extern "C" {

rketd_status rketd_adjoint(rketd_ctx* c, const double* dL_dX_re, const double* dL_dX_im, int64_t w_lo, int64_t w_hi,
                           double* grad_wp2, double* grad_nu) {
  if (!c || !dL_dX_re || !dL_dX_im || !grad_wp2 || !grad_nu) return fail(RKETD_EINVAL, "NULL argument");
  if (c->ckpt_steps < 1) return fail(RKETD_EINVAL, "no checkpointed forward run: call rketd_forward_ckpt first");
  int64_t nz_min = c->nz[0];
  for (int64_t v : c->nz) nz_min = std::min(nz_min, v);
  if (w_lo < 4 || w_hi <= w_lo || w_hi > nz_min - 1)
    return fail(RKETD_EINVAL, "window [%lld, %lld) must lie inside [4, nz - 1) of every slab", (long long)w_lo,
                (long long)w_hi);
  const int P = c->total_probes, nf = c->n_freq;
  if (P > 0) {
    if (!c->gX) {
      void* p;
      rketd_status st = c->alloc(&p, sizeof(double) * 2 * (size_t)P * nf, "loss gradient");
      if (st) return st;
      c->gX = (double*)p;
    }
    const size_t b = sizeof(double) * (size_t)P * nf;
    CK(cudaMemcpyAsync(c->gX, dL_dX_re, b, cudaMemcpyDefault, c->stream), "loss gradient upload");
    CK(cudaMemcpyAsync(c->gX + (size_t)P * nf, dL_dX_im, b, cudaMemcpyDefault, c->stream), "loss gradient upload");
  }
  return c->prec == RKETD_F64 ? adjoint_impl<double>(c, w_lo, w_hi, grad_wp2, grad_nu)
                              : adjoint_impl<float>(c, w_lo, w_hi, grad_wp2, grad_nu);
}

rketd_status rketd_kernel_timing(rketd_ctx* c, int32_t enable) {
  if (!c) return fail(RKETD_EINVAL, "NULL context");
  CK(cudaStreamSynchronize(c->stream), "timing sync");
  c->ev_used = 0;
  c->t_ms = 0;
  c->t_cells = 0;
  c->t_launches = 0;
  c->timing = enable != 0;
  return RKETD_OK;
}

rketd_status rketd_get_kernel_timing(rketd_ctx* c, double* ms, int64_t* launches, double* cell_updates) {
  if (!c) return fail(RKETD_EINVAL, "NULL context");
  rketd_status st = harvest_timing(c);
  if (st) return st;
  if (ms) *ms = c->t_ms;
  if (launches) *launches = c->t_launches;
  if (cell_updates) *cell_updates = c->t_cells;
  return RKETD_OK;
}

rketd_status rketd_get_options(const rketd_ctx* c, rketd_options* o) {
  if (!c || !o) return fail(RKETD_EINVAL, "NULL argument");
  *o = c->opt;
  return RKETD_OK;
}

rketd_status rketd_destroy(rketd_ctx* c) {
  if (!c) return RKETD_OK;
  cudaStreamSynchronize(c->stream);
  delete c;
  return RKETD_OK;
}

rketd_status rketd_plan_tiles_1d(int32_t n_slabs, const int64_t* nz, const int64_t* src_cell, int32_t n_probes,
                                 const int64_t* probe_cell, int32_t cpml_cells, int32_t cells_per_lane,
                                 int32_t tb_steps, int32_t end_tiles, int64_t* rows, int64_t cap,
                                 int64_t* n_tiles) {
  if (!nz || !src_cell || !n_tiles || (n_probes > 0 && !probe_cell) || (cap > 0 && !rows))
    return fail(RKETD_EINVAL, "NULL argument");
  if (n_slabs < 1 || n_probes < 0 || cpml_cells < 0 || cap < 0) return fail(RKETD_EINVAL, "bad count");
  if (cells_per_lane < 4 || cells_per_lane > kMaxCells || cells_per_lane % 4)
    return fail(RKETD_EINVAL, "cells_per_lane must be a multiple of 4 in [4, %d]", kMaxCells);
  if (tb_steps < 4 || tb_steps > 64 || tb_steps % 4) return fail(RKETD_EINVAL, "tb_steps must be a multiple of 4 in [4, 64]");
  for (int s = 0; s < n_slabs; ++s) {
    if (nz[s] < 8) return fail(RKETD_EINVAL, "slab %d: nz must be >= 8", s);
    if (src_cell[s] < 1 || src_cell[s] > nz[s] - 2) return fail(RKETD_EINVAL, "slab %d: source cell outside", s);
    for (int p = 0; p < n_probes; ++p) {
      const int64_t q = probe_cell[(size_t)s * n_probes + p];
      if (q < 0 || q >= nz[s]) return fail(RKETD_EINVAL, "slab %d: probe %d outside", s, p);
    }
  }
  TilePlan plan;
  rketd_status st = build_tile_plan(n_slabs, nz, src_cell, n_probes, probe_cell, cpml_cells, cells_per_lane, tb_steps,
                                    end_tiles != 0, plan);
  if (st) return st;
  *n_tiles = (int64_t)plan.tiles.size();
  const int64_t Lint = 32 * cells_per_lane, Ledge = 32 * edge_cells_per_lane(tb_steps);
  for (int64_t i = 0; i < (int64_t)plan.tiles.size() && i < cap; ++i) {
    const Tile& t = plan.tiles[i];
    const bool is_edge = i >= plan.n_interior;
    const int64_t kind = is_edge ? 2 : (i >= plan.n_interior - plan.n_int_xtra ? 1 : 0);
    int64_t* r = rows + 8 * i;
    r[0] = t.slab;
    r[1] = t.start;
    r[2] = t.vlo;
    r[3] = t.vhi;
    r[4] = kind;
    r[5] = t.src_local;
    r[6] = t.probe_count;
    r[7] = is_edge ? Ledge : Lint;
  }
  return RKETD_OK;
}

}  // extern "C"
