// Internal declarations shared by the library's translation units.
//
// Normalised variables used on the device (all slabs of a context share dz, dt):
//   E~ = E,  H~ = eta0 H,  J~ = (dt / eps0) J,  S = dt / (dz sqrt(mu0 eps0)),
// so that Eq. 14 reads H~ -= S (E_{k+1} - E_k) and Eq. 12 reads
//   E^{n+1} = E^n - S (H~_{k+1/2} - H~_{k-1/2}) - (J~^{n+1} + J~^n) / 2.
// With x = nu dt, w = wp^2 dt^2, a = e^{-x}, phi1 = (1 - a)/x, phi2 = (a - 1 + x)/x^2,
// Eq. 11 becomes J~^{n+1} = a J~^n + w phi1 E^n + w phi2 (E^{n+1} - E^n) and Eq. 12 with it
// substituted, solved for E^{n+1}, is (D = 1 + w phi2 / 2)
//   E^{n+1} = E^n + da E^n - cb (H~_{k+1/2} - H~_{k-1/2}) - cj J~^n,
//   da = -(w phi1 / 2)/D,  cb = S/D,  cj = (1 + a)/(2 D),
//   J~^{n+1} = J~^n + dj J~^n + bp E^n + cc E^{n+1},  dj = a - 1,  bp = w (phi1 - phi2),  cc = w phi2.
// The six per-cell coefficients are kept as deviations (da, dj) or small terms so that
// FP32 storage keeps their relative accuracy.
//
// The device state carries, in place of J~, the folded current
//   G = cj J~ - da E        (cj = (1 + a)/(2D) in (0, 1]),
// the part of the E update that does not depend on the new curl. Substituting it,
//   E^{n+1} = E^n - (cb (H~_{k+1/2} - H~_{k-1/2}) + G^n),
//   G^{n+1} = G^n + dj G^n + bq E^n + cq E^{n+1},
//   bq = cj bp + da a = w (phi1 - (1 + a) phi2)/(2D),   cq = cj cc - da = w (phi1 + (1 + a) phi2)/(2D),
// the same discrete map in exact arithmetic (expand G^{n+1} + da E^{n+1}). In finite precision it
// matters: E and G are each rounded once per step at their own magnitude, after the small terms
// have been summed, so that da E and dj G (down to 1e-7 of E and G on plasma slabs) are not
// rounded away on their own every step; and E takes two operations instead of three. The soft
// source adds s to E^{n+1} after G^{n+1} is formed, so the source cell also takes G -= da s.
// kBq and kCq hold bq and cq; da and cj stay for converting G back to J (fields out, medium
// changes, the no-allocation entry point) and for the adjoint's chain rule.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace rketd {

constexpr double kEps0 = 8.8541878128e-12;
constexpr double kMu0 = 1.25663706212e-6;
constexpr int kMaxCells = 32;   // largest cells-per-lane instantiated
constexpr int kMaxTileProbes = 8;

enum CoefIndex { kDa = 0, kCb = 1, kCj = 2, kDj = 3, kBq = 4, kCq = 5, kNumCoef = 6 };

// E and G update of one interior cell (the folded form above). The G update sums its three small
// terms before adding G: G grows far beyond its per-step increment where the current has a large
// low-frequency part, and adding the terms to G one at a time would round each of them against G
// (in FP64 that alone moved the transmission spectrum of the 8000-step slab by 3e-12). The sum
// starts from dj G and bq E, which do not wait for E', so only one fma and the add follow E'.
template <typename T>
__device__ __forceinline__ T fold_e(T e, T cb, T curl, T g) {
  return e - fma(cb, curl, g);
}
template <typename T>
__device__ __forceinline__ T fold_g(T g, T dj, T bq, T cq, T e, T enew) {
  return g + fma(cq, enew, fma(bq, e, dj * g));
}

// One warp tile of the temporally blocked step: 32*K consecutive cells of one slab,
// loaded from `start` (slab-local, may be negative); after a pass of up to tb_steps
// steps the cells [vlo, vhi) (tile-local) are exact and are the only ones stored.
struct Tile {
  int32_t slab;
  int32_t src_local;    // tile-local index of the source cell, -1 if not loaded
  int64_t start;
  int32_t vlo, vhi;
  int32_t probe_begin;  // into the tile-probe list: probes in [vlo, vhi) (sampled here)
  int32_t probe_count;
  int32_t adj_begin;    // into the tile-probe list: probes anywhere in the loaded range
  int32_t adj_count;    // (the adjoint injects its seeds into every copy of a probe cell)
};

struct TileProbe {
  int32_t local;  // tile-local cell index (inside [vlo, vhi))
  int32_t slot;   // index into the probe-series buffer (slab * n_probes + p)
};

// Everything a step kernel needs; passed by value.
template <typename T>
struct StepArgs {
  const T* E_in;
  const T* H_in;
  const T* J_in;
  T* E_out;
  T* H_out;
  T* J_out;
  const T* coef[kNumCoef];
  const int64_t* soff;    // [n_slabs] storage offset of each slab
  const int64_t* nz;      // [n_slabs]
  const int64_t* src;     // [n_slabs] source cell
  // Eq. 10 recursion only (plain kernels): E^{n-1} (updated in place) and its weights in E' and G'
  T* Ep;
  const T* ep;
  const T* gp;
  // CPML (bc == 1): compact memories [n_slabs][2 ends][ncpml] for E and H nodes; the split-field
  // PML (bc == 2) uses cpmlE [2][ncpml+1] and cpmlH [2][ncpml] as its (da, c) tables, no memories
  const T* psiE_in;
  const T* psiH_in;
  T* psiE_out;
  T* psiH_out;
  const T* cpmlE;   // [3][ncpml+1] b, c, 1/kappa by E-node depth d = 0..ncpml
  const T* cpmlH;   // [3][ncpml]   b, c, 1/kappa by H-node depth index i (depth i + 1/2)
  int32_t ncpml;
  int32_t bc;
  T S;
  T qmur;
  // source (Eq. 15)
  double dt, tau, t0, amp;
  int64_t n0;           // step index at pass start (fields hold E^{n0})
  int32_t nsub;         // steps in this pass
  // probe series buffer [slot][series_len], written at column series_pos + t
  T* series;
  int32_t series_len;
  int32_t series_pos;
  // tiles
  const Tile* tiles;
  const TileProbe* tprobes;
  int32_t n_tiles;
  int32_t total_probes;
  // window recording (adjoint recompute): after each step the state (E, H, G) of cells
  // [rec_c0, rec_c0 + rec_w) of every slab goes to rec[slab][slot][3][rec_w], slot = rec_pos + t
  T* rec;
  int64_t rec_c0;
  int32_t rec_w;
  int32_t rec_len;
  int32_t rec_pos;
};

// The reverse (adjoint) step on the same tiles. lambda = (lE, lH, lJ) is the adjoint of
// (E, H~, G); a pass takes the adjoint from after step n_hi - 1 back to before step
// n_hi - nsub. seeds[slot][seed_len] holds dL/dE at probe `slot` for the sample that follows
// step n (column n - seg_n0). Window cells [rec_c0, rec_c0 + rec_w) record, for each step,
// mu = lE + cq lJ and lJ (both after the step) to rec[slab][n - seg_n0][2][rec_w].
template <typename T>
struct AdjArgs {
  const T* lE_in;
  const T* lH_in;
  const T* lJ_in;
  T* lE_out;
  T* lH_out;
  T* lJ_out;
  const T* coef[kNumCoef];
  const int64_t* soff;
  const int64_t* nz;
  T S;
  T qmur;
  int32_t nsub;
  int64_t n_hi;
  int64_t seg_n0;
  const T* seeds;
  int32_t seed_len;
  const Tile* tiles;
  const TileProbe* tprobes;
  int32_t n_tiles;
  T* rec;
  int64_t rec_c0;
  int32_t rec_w;
  int32_t rec_len;
};

// Sets the message rketd_last_error() returns on this thread (defined with the runtime).
void set_error_message(const char* msg);

// Every device allocation of the contexts goes through these: cudaMalloc / cudaMallocAsync,
// unless a test armed an injected failure (rketd_debug_fail_alloc), which is then reported as
// cudaErrorMemoryAllocation without touching the device.
cudaError_t device_alloc(void** p, size_t bytes);
cudaError_t device_alloc_async(void** p, size_t bytes, cudaStream_t st);

// ORs 1 into *flag if any of n values (FP64 if f64, else FP32) is NaN or infinite. Async.
cudaError_t launch_finite_scan(bool f64, const void* p, int64_t n, int* flag, cudaStream_t st);

// ---- launchers (defined in the .cu files) ----
// scheme: 0 = Eq. 11, 1 = Eq. 9, 2 = Eq. 10 (then ext[0], ext[1] receive ep and gp, the weights of
// E^{n-1} in the E and G updates; see coeffs.cu)
cudaError_t launch_coeffs(int prec, const double* wp2, const double* nu, const int64_t* soff,
                          const int64_t* off, const int64_t* nz, int n_slabs, int64_t n_store,
                          double dt, double S, void* const coef[kNumCoef], cudaStream_t st, int scheme = 0,
                          void* const ext[2] = nullptr);
cudaError_t launch_cpml_tables(int prec, int ncpml, double dt, double m, double smax, double kmax,
                               double amax, void* cpmlE, void* cpmlH, cudaStream_t st);
// split-field PML tables: E [2][n+1] and H [2][n] rows (e^{-x} - 1, S phi1(x)) by depth
cudaError_t launch_pml_tables(int prec, int n, double dt, double S, double m, double smax, void* tabE, void* tabH,
                              cudaStream_t st);

// split-field PML update of one node: x' = e^{-s} x - S phi1 D = x - (c D - da x), small terms first
template <typename T>
__device__ __forceinline__ T pml_update(T x, T da, T c, T d) {
  return x - fma(c, d, -da * x);
}

// Tiled step over a.tiles. Interior tiles (edge = false) that sample a probe or whose loaded range
// holds their slab's source cell need xtra = true; the others run a kernel without that code.
template <typename T>
cudaError_t launch_tb(const StepArgs<T>& a, int K, bool edge, int warps_per_block, cudaStream_t st, bool xtra);

// forward tiles that also record the window state (scalar kernel, template REC = true)
template <typename T>
cudaError_t launch_tb_rec(const StepArgs<T>& a, int K, bool edge, int warps_per_block, cudaStream_t st);

// adjoint pass over the tiles (adjoint.cu)
template <typename T>
cudaError_t launch_adj(const AdjArgs<T>& a, int K, bool edge, int warps_per_block, cudaStream_t st);
// adjoint pass, FP32 interior tiles off the window, packed FP32x2 pairs (no recording)
cudaError_t launch_adj_pairs(const AdjArgs<float>& a, int K, int warps_per_block, cudaStream_t st);
// seeds[slot][t] = sum_f (gXr cos - gXi sin)(2 pi f (m0 + t) dt) from a twiddle table tw[t][f]
template <typename T>
cudaError_t launch_seeds(const double* gXr, const double* gXi, const T* tw, int P, int nf, int n, T* seeds,
                         int seed_len, cudaStream_t st);
// The source of each slab, for the gradient sums of one segment (steps n0 ..): slab-local
// source cells, the window start and the pulse
struct GradSource {
  const int64_t* cell;
  int64_t w_lo;
  int64_t n0;
  double dt, t0, tau, amp;
};
// g[5][slab][w] += per-window-cell sums over one segment of the recorded forward and adjoint values
template <typename T>
cudaError_t launch_grad_accum(const T* recF, const T* recA, int n_slabs, int rec_w, int nwin, int L, int recF_len,
                              const GradSource& src, double* g, cudaStream_t st);
// chain rule: grad_wp2, grad_nu of window cells from g and d(coefficient)/d(wp2, nu)
cudaError_t launch_grad_chain(const double* g, const double* wp2, const double* nu, const int64_t* off,
                              int n_slabs, int64_t w_lo, int w, double dt, double S, double* grad_wp2,
                              double* grad_nu, cudaStream_t st);
// copies the window cells of the current state into recF slot 0
template <typename T>
cudaError_t launch_rec_init(const T* E, const T* H, const T* J, const int64_t* soff, const int64_t* nz, int n_slabs,
                            int64_t c0, int w, int rec_len, T* rec, cudaStream_t st);

// Resident step (step_resident.cu): a single slab held by one cluster of `ctas` CTAs of `threads`
// threads, K cells per thread, pl cells of left padding; a.nsub steps in one launch, first-order Mur
// ends; a.tprobes lists the probes as (slab cell, probe index). query_only: *max_clusters receives how
// many such clusters can be resident at once (0: the shape cannot run), nothing is launched.
template <typename T>
cudaError_t launch_resident(const StepArgs<T>& a, int K, int ctas, int threads, int pl, cudaStream_t st,
                            bool query_only, int* max_clusters);

// FP32 interior tiles with two cells per packed FP32x2 register (step_tb2.cu); xtra as for launch_tb
cudaError_t launch_tb_pairs(const StepArgs<float>& a, int K, int warps_per_block, cudaStream_t st, bool xtra);

// Persistent tiled step (step_persist.cu): n_pass passes of nsub steps over the whole tile list in
// one launch. Tile list order: [0, n_main) interior, [n_main, n_main + n_xtra) interior tiles with a
// probe or a source cell, then edge tiles (Ke cells per lane).
struct PersistCtl {
  int n_tiles, n_main, n_xtra;
  int n_pass, nsub;
  const int* dep_off;  // [n_tiles + 1]: tiles whose cells tile j reads or whose reads it overwrites
  const int* dep_idx;
  int* done;           // [n_tiles]: last pass finished, -1 at launch start
  int* work;           // work-item counter, 0 at launch start
  int* err;            // status word: 1 = a wait gave up
  int wait_limit;      // polls per wait (<= 0: every wait gives up at once)
};
// Resident one-warp blocks of the persistent kernel on this device (0 if unknown).
int persist_capacity(int K, int Ke);
// a0 / a1: the step arguments of even / odd passes (buffers swapped), n0 and series_pos of pass 0;
// sa_d: device room for both.
cudaError_t launch_persist(StepArgs<float>* sa_d, const StepArgs<float>& a0, const StepArgs<float>& a1,
                           const PersistCtl& pc, int K, int Ke, int grid, cudaStream_t st);

template <typename T>
cudaError_t launch_plain_step(const StepArgs<T>& a, const int32_t* cell_slab, int64_t n_store,
                              const int64_t* probe_index, cudaStream_t st);

template <typename T>
cudaError_t launch_twiddles(const double* freq, int n_freq, double dt, int64_t m0, int n_samples,
                            T* tw, cudaStream_t st);
template <typename T>
cudaError_t launch_dft(const T* series, int series_len, int n_samples, const T* tw, int total_probes,
                       int n_freq, double* X_re, double* X_im, cudaStream_t st, const double* rot = nullptr);
// rot[f] = exp(-j 2 pi f m0 dt), FP64 [n_freq][2]
cudaError_t launch_dft_rotation(const double* freq, int n_freq, double dt, int64_t m0, double* rot, cudaStream_t st);

// Device state of one slab to SI: E, H = H~ h_scale, J = (G + da E)/cj j_scale
cudaError_t launch_gather_fields(int prec, const void* E, const void* H, const void* G, const void* cj,
                                 const void* da, int64_t off, int64_t nz, double h_scale, double j_scale, double* Eo,
                                 double* Ho, double* Jo, cudaStream_t st);
// Medium change: G <- cj_new (G + da_old E)/cj_old - da_new E elementwise over n cells, so that
// J~ stays as it was while the coefficients change
cudaError_t launch_rescale(int prec, void* G, const void* E, const void* cj_new, const void* cj_old,
                           const void* da_new, const void* da_old, int64_t n, cudaStream_t st);

}  // namespace rketd
