/*
 * rketd.h -- C ABI of the GB300 (sm_103a) RKETD-FDTD library.
 *
 * The library advances the 1D Yee/RKETD scheme for an unmagnetized Drude plasma
 * (Xiong et al., "The Electromagnetic Waves Propagation in Unmagnetized Plasma
 * Media Using Parallelized FDTD", arXiv:1709.00821):
 *   Eq. 14  H update:  H^{n+1/2}_{k+1/2} = H^{n-1/2}_{k+1/2} - dt/(mu0 dz) (E^n_{k+1} - E^n_k)
 *   Eq. 12  E update driven by the time-averaged plasma current (J^{n+1} + J^n)/2
 *   Eq. 11  RKETD current recursion J^{n+1} = e^{-nu dt} J^n + ... (E^n, E^{n+1})
 *   Eq. 13  Eq. 11 substituted into Eq. 12 and solved for E^{n+1} (read with the
 *           common denominator on every term; the printed form drops it on two)
 *   Eq. 15  Gaussian-derivative soft source, tau = 15 dt in the paper's run
 * with first-order Mur or CPML ends and a running DFT at probe cells from which
 * the reflection and transmission spectra of Sec. IV.B follow.
 *
 * Conventions for every call:
 *  - Quantities at the ABI are SI: m, s, V/m, A/m, A/m^2, rad^2/s^2, 1/s, Hz.
 *  - Every call returns an rketd_status; no call aborts or throws across the ABI.
 *    On failure rketd_last_error() returns a message (thread-local, valid until
 *    the next call on the same thread).
 *  - Host arrays passed in are read during the call only (copied); the caller
 *    keeps ownership. Output host arrays are written during the call.
 *  - Device pointers passed in are borrowed: they must stay valid until the call's
 *    work on the context's stream has completed (rketd_sync).
 *  - A context owns the device memory it allocates (fields, coefficients, DFT
 *    state) and releases it in rketd_destroy. Work is queued on the CUDA stream
 *    given at creation (NULL = legacy default stream).
 *  - A context must not be used from two threads at once.
 */
#ifndef RKETD_H
#define RKETD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  RKETD_OK = 0,
  RKETD_EINVAL = 1,       /* invalid argument (sizes, cells, physical parameters) */
  RKETD_ECOURANT = 2,     /* c0 dt / dz > 1: the explicit leapfrog is unstable */
  RKETD_ENOMEM = 3,       /* device or host allocation failed */
  RKETD_ECUDA = 4,        /* a CUDA runtime call failed; message has the CUDA error */
  RKETD_ETIMEOUT = 5,     /* a bounded device-side wait gave up */
  RKETD_EUNSUPPORTED = 6, /* option combination not provided by this build */
  RKETD_ENUMERIC = 7,     /* non-finite value seen in the fields or spectra */
  RKETD_EIO = 8           /* state file could not be read or written */
} rketd_status;

typedef enum { RKETD_F32 = 0, RKETD_F64 = 1 } rketd_prec;
typedef enum { RKETD_BC_MUR1 = 0, RKETD_BC_CPML = 1, RKETD_BC_PML = 2 } rketd_bc;
/* Recursion for the plasma current over one step (Sec. II, from the exact solution Eq. 7):
 *   RKETD_SCHEME_RKETD  Eq. 11: F = eps0 wp^2 E interpolated linearly between t_n and t_{n+1};
 *                       Eq. 12 is then solved for E^{n+1} (Eq. 13). Second order. The default.
 *   RKETD_SCHEME_ETD1   Eq. 9: F held at F_n over the step. First order. J^{n+1} is explicit and
 *                       Eq. 12 gives E^{n+1} directly.
 *   RKETD_SCHEME_ETD2   Eq. 10 read literally: F extrapolated from F_{n-1} and F_n over the step.
 *                       Second order and explicit, but it needs E^{n-1}: the state carries one more
 *                       array, and the step runs on the plain variant only (variant 0 selects it;
 *                       the tiled variant returns RKETD_EUNSUPPORTED).
 * The adjoint (rketd_forward_ckpt/rketd_adjoint) and the allocation-free entry point take
 * RKETD_SCHEME_RKETD (and, for the latter, RKETD_SCHEME_ETD1) only. */
typedef enum { RKETD_SCHEME_RKETD = 0, RKETD_SCHEME_ETD1 = 1, RKETD_SCHEME_ETD2 = 2 } rketd_scheme;

/* Grid shared by every slab of a context. Courant number S = dt / (dz sqrt(mu0 eps0))
 * must satisfy 0 < S <= 1 (1D leapfrog stability); S is evaluated with
 * eps0 = 8.8541878128e-12 F/m and mu0 = 1.25663706212e-6 H/m.
 * prec: RKETD_F64 keeps fields, coefficients and DFT sums in FP64. RKETD_F32
 * keeps fields in FP32, derives the update coefficients in FP64 and stores them
 * as FP32 deviations from their vacuum values, and accumulates the DFT in
 * compensated FP32 per block of samples added into FP64 totals.
 * bc: RKETD_BC_MUR1 = first-order Mur at both ends; RKETD_BC_CPML = convolutional
 * PML of cpml_cells cells at both ends backed by PEC walls, with grading
 * sigma = sigma_max rho^m, kappa = 1 + (kappa_max - 1) rho^m, alpha = alpha_max (1 - rho)
 * in relative depth rho; sigma_max <= 0 selects 0.8 (m + 1)/(eta0 dz).
 * RKETD_BC_PML = the paper's split-field PML (Sec. III; 5 cells in Sec. IV.B) of cpml_cells cells
 * at both ends backed by PEC walls. In 1D only the z-split field exists, so the layer is one graded
 * conductivity sigma on E with the matched magnetic conductivity sigma mu0/eps0 on H, advanced by
 * exponential differencing: E' = e^{-x} E - (1 - e^{-x})/(sigma dz) dH, x = sigma dt/eps0, and the
 * same for H. sigma = sigma_max rho^m as above (kappa_max, alpha_max unused). The layers must be
 * vacuum (wp2 = 0 there, else RKETD_EINVAL). */
typedef struct {
  double dz, dt;
  int32_t prec;          /* rketd_prec */
  int32_t bc;            /* rketd_bc */
  int32_t cpml_cells;
  int32_t scheme;        /* rketd_scheme; 0 = Eq. 11 */
  double cpml_m, cpml_sigma_max, cpml_kappa_max, cpml_alpha_max;
} rketd_grid1d;

/* Eq. 15 soft source added to E^{n+1} at the source cell after the E update:
 * s(t) = amp * ((t - t0)/tau) * exp(-(t - t0)^2 / (2 tau^2)), t = (n+1) dt.
 * The paper uses tau = 15 dt and a delay of 5 tau. */
typedef struct {
  double tau, t0, amp;
} rketd_pulse;

/* Running DFT X_p(f) = sum_{m>=1} E_p^m exp(-j 2 pi f m dt) at n_probes cells per slab
 * (Sec. IV.B computes R and T by an FFT of the probe series; the sum is the same
 * transform evaluated at the requested frequencies). */
typedef struct {
  int32_t n_probes;     /* per slab, >= 0 */
  int32_t n_freq;       /* >= 1 when n_probes > 0 */
  const double* freq_hz;  /* [n_freq], host, copied */
} rketd_dft;

/* Execution options. Zero-initialise and set what you need; rketd_default_options()
 * fills the defaults. */
typedef struct {
  int32_t variant;      /* 0 = auto (resident where it applies, else tiled; plain for the Eq. 10
                           recursion), 1 = plain (paper structure: one H kernel and one E+J kernel per
                           step), 2 = temporally blocked warp tiles, 3 = resident: a single
                           Mur-terminated slab held in the registers of one thread-block cluster (up
                           to 16 CTAs) for a whole DFT block of steps per launch, for slabs of up to
                           16384 (FP64) or 32768 (FP32) cells; RKETD_EUNSUPPORTED where it does not
                           apply; 4 = persistent (FP32 only): the tiles of variant 2, every pass of a
                           DFT block in one launch whose resident warps take (pass, tile) work items
                           in order and wait (bounded) only for their slab's neighbouring tiles of
                           the previous pass; results bitwise those of variant 2. The checkpointed
                           forward run and the adjoint use the tiled kernels. */
  int32_t cells_per_lane;  /* K for the tiled kernel: 8, 12 or 16 (F32), 4 or 8 (F64); 0 = auto */
  int32_t tb_steps;     /* leapfrog steps per tiled pass (4..64, multiple of 4); 0 = auto */
  int32_t warps_per_block; /* warps per CTA of the tiled kernel, 1..4; 0 = auto */
  int32_t dft_block;    /* probe samples buffered between DFT folds (multiple of tb_steps); 0 = auto */
  int32_t use_graphs;   /* 0 = auto (on), 1 = on, 2 = off: rketd_step calls that repeat an earlier
                           call's start step, step count and buffer parity replay its CUDA graph */
  int32_t fp32_pairs;   /* FP32 interior tiles: 0 = auto (packed FP32x2 pairs), 1 = pairs, 2 = scalar */
  int32_t res_ctas;     /* resident variant: CTAs of the cluster, 1..16; 0 = auto */
  int32_t res_threads;  /* resident variant: threads per CTA, a multiple of 32, <= 1024 (FP32) or 256
                           (FP64); 0 = auto */
  int32_t res_cells;    /* resident variant: cells per thread, 2, 4, 8 or 16 (FP32), 1, 2, 4 or 8 (FP64)
                           (at most 1024, 512, 256, 128 threads with 2, 4, 8, 16 FP32 cells; 256 threads
                           with up to 4 FP64 cells, 128 with 8); 0 = auto */
  int32_t reserved[2];
} rketd_options;

typedef struct rketd_ctx rketd_ctx;

/* Fills *opt with the defaults (every field 0 = auto). */
void rketd_default_options(rketd_options* opt);

/*
 * Creates a context for n_slabs independent 1D problems advanced together
 * (the paper's single slab is n_slabs = 1).
 *   nz[s]        E nodes of slab s (>= 8); H nodes are k+1/2, k = 0..nz-2
 *   wp2, nu      concatenated per-cell plasma frequency squared (rad^2/s^2, >= 0)
 *                and collision frequency (1/s, >= 0), slab after slab, host FP64
 *   src_cell[s]  soft-source cell of slab s, 1 <= cell <= nz-2 (outside the CPML)
 *   probe_cell   [n_slabs * dft->n_probes] probe cells, 0 <= cell < nz (outside the CPML)
 *   stream       cudaStream_t for all work of this context (may be NULL)
 * The coefficient precompute (RKETD exponentials in FP64) runs on the device.
 * Errors: RKETD_EINVAL, RKETD_ECOURANT, RKETD_ENOMEM, RKETD_ECUDA. *out is NULL on error.
 */
rketd_status rketd_create_batch_1d(int32_t n_slabs, const int64_t* nz, const rketd_grid1d* grid,
                                   const double* wp2, const double* nu, const int64_t* src_cell,
                                   const rketd_pulse* pulse, const int64_t* probe_cell,
                                   const rketd_dft* dft, const rketd_options* opt, void* stream,
                                   rketd_ctx** out);

/* Single-slab convenience form of rketd_create_batch_1d. */
rketd_status rketd_create_1d(int64_t nz, const rketd_grid1d* grid, const double* wp2, const double* nu,
                             int64_t src_cell, const rketd_pulse* pulse, const int64_t* probe_cell,
                             const rketd_dft* dft, const rketd_options* opt, void* stream,
                             rketd_ctx** out);

/* Replaces the medium (same layout as at creation) and recomputes the update
 * coefficients on the device. on_device = 0: wp2/nu are host FP64 arrays (copied
 * host->device on the stream); 1: device FP64 arrays (read on the stream). Fields
 * are not touched. */
rketd_status rketd_set_medium(rketd_ctx* ctx, const double* wp2, const double* nu, int32_t on_device);

/* Zeroes fields, CPML memories and DFT sums and sets the step index to 0 (async). */
rketd_status rketd_reset(rketd_ctx* ctx);

/* Queues nsteps leapfrog steps (Eqs. 14, 13, 11, 15, ends, DFT) on the stream. Async;
 * device-side problems surface at rketd_sync. */
rketd_status rketd_step(rketd_ctx* ctx, int64_t nsteps);

/* Waits for the stream and reports any device-side error; RKETD_ETIMEOUT if a wait of the
 * persistent variant gave up since the last reset. */
rketd_status rketd_sync(rketd_ctx* ctx);

/* Current step index n (fields hold E^n, H^{n-1/2}, J^n). */
int64_t rketd_step_index(const rketd_ctx* ctx);

/* Copies slab s's fields to host FP64 SI arrays (any may be NULL): E[nz], H[nz-1], J[nz].
 * Synchronises the stream. */
rketd_status rketd_get_fields(rketd_ctx* ctx, int32_t slab, double* E, double* H, double* J);

/* Copies the DFT sums to host: re/im [n_slabs][n_probes][n_freq] (FP64). Synchronises. */
rketd_status rketd_get_spectra(rketd_ctx* ctx, double* re, double* im);

/* Same as rketd_get_spectra into device FP64 arrays (async on the stream). */
rketd_status rketd_get_spectra_device(rketd_ctx* ctx, double* re, double* im);

/* Host helper for Sec. IV.B: from total-field and incident (vacuum-run) spectra at
 * the reflection probe (index 0) and transmission probe (index 1) of one slab,
 * R = (X_R^tot - X_R^inc)/X_R^inc and T = X_T^tot / X_T^inc, each [n_freq]. */
rketd_status rketd_rt(const double* tot_re, const double* tot_im, const double* inc_re,
                      const double* inc_im, int32_t n_freq, double* R_re, double* R_im, double* T_re,
                      double* T_im);

/* Resets the context and runs nsteps steps from rest (as rketd_reset + rketd_step), keeping
 * a copy of the full state every ckpt_every steps for rketd_adjoint. First-order Mur ends
 * and the tiled variant only (RKETD_EUNSUPPORTED otherwise). The spectra of the run are
 * available as after rketd_step. */
rketd_status rketd_forward_ckpt(rketd_ctx* ctx, int64_t nsteps, int32_t ckpt_every);

/*
 * Discrete adjoint of the last rketd_forward_ckpt run (the transpose of Eqs. 14, 13, 11 and
 * the Mur ends, step by step in reverse): gradients of a loss L(X) of the probe spectra with
 * respect to the plasma frequency squared and the collision frequency of every cell in
 * [w_lo, w_hi) of every slab (the trainable window; 4 <= w_lo < w_hi <= nz - 1).
 *   dL_dX_re/im   dL/dRe X and dL/dIm X, [n_slabs][n_probes][n_freq] FP64, host or device
 *   grad_wp2/nu   device FP64 [total cells, concatenated as wp2], caller-owned; cells
 *                 outside the window are set to 0
 * Each checkpoint segment is recomputed forward while the window states are recorded, then
 * transposed on the same tiles; the per-step products are summed per segment (FP32 sums for
 * FP32 fields, added into FP64 totals) and taken to (wp2, nu) by the derivatives of the update
 * coefficients in FP64. Leaves the fields in an intermediate state (rketd_reset before reuse).
 * Async on the stream.
 */
rketd_status rketd_adjoint(rketd_ctx* ctx, const double* dL_dX_re, const double* dL_dX_im, int64_t w_lo,
                           int64_t w_hi, double* grad_wp2, double* grad_nu);

/* Saves / restores the full state (fields, CPML memories, DFT sums, step index) to a
 * versioned binary file. A run resumed from a saved state is bitwise identical to
 * an uninterrupted one with the same options. Synchronises. */
rketd_status rketd_save_state(rketd_ctx* ctx, const char* path);
rketd_status rketd_load_state(rketd_ctx* ctx, const char* path);

/* Times the tiled variants on this context for about `passes` passes each and keeps
 * the fastest (the state is saved and restored around the trials). Synchronises. */
rketd_status rketd_autotune(rketd_ctx* ctx, int32_t passes);

/* Options in use (after auto selection). */
rketd_status rketd_get_options(const rketd_ctx* ctx, rketd_options* opt);

/* Enables (1) or disables (0) CUDA-event timing of every launch of the interior tiled
 * step kernel (the kernel that carries almost all the work) on the context's stream, and
 * clears the totals. Synchronises. */
rketd_status rketd_kernel_timing(rketd_ctx* ctx, int32_t enable);

/* Totals since rketd_kernel_timing: summed device time (ms), launches, and exact
 * cell-updates done by those launches (halo recomputation not counted). Synchronises. */
rketd_status rketd_get_kernel_timing(rketd_ctx* ctx, double* ms, int64_t* launches, double* cell_updates);

/* Number of kernel launches this context has issued (graph replays count their nodes). */
int64_t rketd_launch_count(const rketd_ctx* ctx);

/*
 * Host-only view of the 1D tile plan that rketd_step builds for a batch of slabs, with no
 * device work (the library need not find a GPU). The paper has no counterpart: it lets tests
 * and tools check the temporally blocked tiling without running it.
 *   n_slabs, nz[n_slabs], src_cell[n_slabs], n_probes, probe_cell[n_slabs * n_probes]
 *                   as for rketd_create_batch_1d (slab-local cells)
 *   cpml_cells      CPML cells per end (0 for first-order Mur ends)
 *   cells_per_lane  K, a multiple of 4 in [4, 32]; tb_steps: T, a multiple of 4 in [4, 64]
 *   end_tiles       nonzero: the plan of the tiled FP32-pair step with first-order Mur ends
 *                   (cpml_cells 0), where slabs of more than 2 (32K - T) cells have their two
 *                   ends held by interior-width tiles of kind 1 (the left one loads [0, 32K),
 *                   the right one ends at round_up(nz, 4) - 1) instead of edge tiles
 *   rows            caller-owned int64 array of cap rows of 8, written in launch order: slab, start
 *                   (slab-local first loaded cell, may be negative for edge tiles), vlo, vhi (the
 *                   exact cells stored are start + [vlo, vhi)), kind (0 interior tile, 1 interior
 *                   tile that samples a probe, loads the source cell or holds a slab end, 2 edge
 *                   tile), src_local (the
 *                   source cell minus start if loaded, else -1), probe_count (probes among the exact
 *                   cells), loaded cells (32 K, or 32 Ke for edge tiles)
 *   cap             rows available; n_tiles receives the tile count even when it exceeds cap
 * Returns RKETD_EINVAL for NULL pointers, counts or shapes outside these ranges, cells outside
 * their slab, or a tile too narrow for its halo.
 */
rketd_status rketd_plan_tiles_1d(int32_t n_slabs, const int64_t* nz, const int64_t* src_cell, int32_t n_probes,
                                 const int64_t* probe_cell, int32_t cpml_cells, int32_t cells_per_lane,
                                 int32_t tb_steps, int32_t end_tiles, int64_t* rows, int64_t cap,
                                 int64_t* n_tiles);

/*
 * Advances one Mur-terminated 1D slab by nsteps steps without allocating any memory.
 * The paper has no counterpart: it exists for callers that must not allocate device
 * memory -- a framework whose caching allocator owns the GPU and forbids allocations behind
 * its back, or a loop that cannot afford the device-wide synchronisation of cudaMalloc/cudaFree.
 * It runs the tiled step of rketd_step (default tile shapes; FP32 interior tiles in the scalar
 * form, bitwise equal to the default packed pairs; no probes or DFT) and keeps
 * its working memory (update coefficients, the two working copies of the fields, the tile list)
 * in one fixed array of about 12.7 MB that the library reserves on every GPU it is loaded on,
 * from load until process exit.
 *   grid          dz, dt, prec (RKETD_F32 or RKETD_F64); bc must be RKETD_BC_MUR1; scheme
 *                 RKETD_SCHEME_RKETD or RKETD_SCHEME_ETD1 (RKETD_SCHEME_ETD2: RKETD_EUNSUPPORTED)
 *   nz            E nodes, 8 <= nz <= 131072 (larger is rejected with RKETD_EINVAL)
 *   wp2, nu       device FP64 arrays [nz] (rad^2/s^2, 1/s), read on the stream. They must be
 *                 finite and >= 0: this call does not check them (they are never copied to the
 *                 host), and a negative or non-finite value makes the fields grow or turn to NaN
 *   src_cell      1 <= src_cell <= nz-2; pulse as for rketd_create_1d
 *   n0            step index of the given fields (they hold E^n0, H^{n0-1/2}, J^n0)
 *   E, J          device arrays [nz], H [nz-1], SI, FP32 or FP64 as grid->prec; read and
 *                 overwritten in place with the state at step n0 + nsteps
 *   stream        cudaStream_t (NULL = legacy default stream)
 * The first call on each device looks up the device address of the fixed array (with that
 * device current) and keeps it for the life of the process; make that first call before any
 * stream capture. A device reset (cudaDeviceReset, or destroying and recreating the primary
 * context) while the library stays loaded leaves that address stale: do not use this entry
 * point after one. Every call reuses the same array, so calls whose GPU work overlaps (other
 * streams, other host threads) race and must be serialised by the caller. Async on the stream;
 * errors from argument checks are returned at once, device errors surface at the next
 * synchronisation.
 */
rketd_status rketd_advance_1d_noalloc(const rketd_grid1d* grid, int64_t nz, const double* wp2, const double* nu,
                                      int64_t src_cell, const rketd_pulse* pulse, int64_t n0, int64_t nsteps,
                                      void* E, void* H, void* J, void* stream);

/*
 * The tile list rketd_advance_1d_noalloc builds on the device for a slab, computed on the host by
 * the same code, so that callers and tests can check its coverage without a GPU (host only, no
 * CUDA call).
 *   prec          RKETD_F32 or RKETD_F64 (they use different tile shapes)
 *   nz, src_cell  as for rketd_advance_1d_noalloc (8 <= nz <= 131072, 1 <= src_cell <= nz-2)
 *   rows          caller-owned int64 array of cap rows of 5, in launch order: start (first loaded
 *                 cell), vlo, vhi (the exact cells are start + [vlo, vhi)), src_local (the source
 *                 cell minus start if loaded, else -1), loaded cells
 *   n_tiles       receives the tile count even when it exceeds cap
 *   launch_counts receives [3]: the tiles of the three launches of a pass, in order (interior
 *                 tiles without the source cell, interior tiles that load it, edge tiles)
 * Returns RKETD_EINVAL for NULL pointers or arguments outside these ranges.
 */
rketd_status rketd_noalloc_tiles_1d(int32_t prec, int64_t nz, int64_t src_cell, int64_t* rows, int64_t cap,
                                    int64_t* n_tiles, int64_t* launch_counts);

/* Persistent variant (options.variant = 4): polls of each wait of a tile for its neighbours'
 * previous pass before it gives up (0: every wait gives up at once, a test of the failure path;
 * < 0 restores the default of 2^22, with a 64 ns pause between polls). A wait that gives up lets
 * the tile go on and sets the context's status word: the next rketd_sync returns RKETD_ETIMEOUT
 * (the fields are then not valid) until rketd_reset clears it. No effect on the other variants. */
rketd_status rketd_set_wait_limit(rketd_ctx* ctx, int32_t polls);

/* Scans the state (E, H and the carried current of every slab, E^{n-1} for Eq. 10, CPML memories)
 * and the spectra for NaN or infinite values: RKETD_ENUMERIC if any is found, else RKETD_OK.
 * Input validation admits only finite parameters, but a finite input can still overflow (a source
 * amplitude near the largest double, say); this is the check for that. Synchronises. */
rketd_status rketd_check_finite(rketd_ctx* ctx);

/* Test hooks for the failure paths, process-wide, no effect unless called.
 * rketd_debug_fail_alloc: the next `after` device allocations made by the library succeed and
 * the one after them fails as if the device were out of memory, so the call that made it returns
 * RKETD_ENOMEM (creation calls release what they had allocated and leave *out NULL); after < 0
 * disarms. rketd_debug_alloc_count: device allocations the library has attempted so far. */
rketd_status rketd_debug_fail_alloc(int64_t after);
int64_t rketd_debug_alloc_count(void);

/* Releases the context and its device memory. NULL is accepted. */
rketd_status rketd_destroy(rketd_ctx* ctx);

/* ---------------------------------------------------------------------------------------
 * 3D Yee RKETD-FDTD: the paper's stated generalisation of the 1D scheme to 2D/3D (Sec. IV.B
 * closing remarks, Sec. V). Eqs. 14, 12, 11 and 13 applied component by component on a Yee
 * grid of nx x ny x nz cells with cell size d; arrays are [k][j][i] (x fastest).
 * Yee positions: Ex (i+1/2, j, k), Ey (i, j+1/2, k), Ez (i, j, k+1/2),
 *                Hx (i, j+1/2, k+1/2), Hy (i+1/2, j, k+1/2), Hz (i+1/2, j+1/2, k).
 * Boundaries: CPML of npml cells (grading as rketd_grid1d) on every face, backed by PEC
 * walls, or periodic in x and y with CPML along z only. Sources: a total-field/scattered-
 * field box fed by an auxiliary 1D vacuum line (Ex-polarised plane wave along +z, the Eq. 15
 * pulse injected on that line, first-order Mur ends), and/or an Eq. 15 soft sheet source
 * added to Ex on one z plane. Materials: each E component takes the Drude material at its own
 * position; mat[cell] packs the material indices (0..3, 0 = vacuum) of Ex, Ey, Ez of that
 * cell in bits 0-1, 2-3 and 4-5. Probes sample Ex; their running DFT is as rketd_dft.
 * ------------------------------------------------------------------------------------- */
typedef struct {
  int32_t nx, ny, nz;    /* cells per axis, >= 4 (and room for the CPML: > 2 (npml + 2)) */
  int32_t prec;          /* rketd_prec: F32 fields (FP64-derived coefficients) or F64 */
  double d, dt;          /* cell size (m) and time step (s); c0 dt / d <= 1/sqrt(3) */
  int32_t periodic_xy;   /* 1: periodic x and y, CPML along z only; 0: CPML on all faces */
  int32_t npml;          /* CPML cells per face, >= 1 */
  double pml_m, pml_sigma_max, pml_kappa_max, pml_alpha_max; /* as rketd_grid1d */
  int32_t tfsf;          /* 1: TF/SF box active */
  int32_t box[6];        /* i0, i1, j0, j1, k0, k1: the total-field region (outside the CPML) */
  int32_t sheet_k;       /* >= 0: soft sheet source on Ex at this z plane; -1: none */
  int32_t inc_off;       /* incident line index of plane k is k + inc_off (>= 2) */
  int32_t inc_len;       /* incident line length, >= nz + 2 inc_off */
  int32_t inc_src;       /* incident line source index, 1 <= inc_src < inc_off */
  int32_t variant;       /* 0 = auto (staged where it applies, else fused), 1 = plain (paper
                            structure: an H kernel and an E+J kernel per step, fields in place),
                            2 = fused (one kernel per step, step-n state in, step-n+1 state out:
                            twice the E/H memory), 3 = staged (fused, with the step-n planes
                            brought into shared memory by TMA copies; CPML on every face,
                            nx a multiple of 16 and each CPML memory array under 2^31 entries,
                            else RKETD_EUNSUPPORTED) */
} rketd_grid3d;

typedef struct rketd_ctx3d rketd_ctx3d;

/*
 * Creates a 3D context and zeroes its state.
 *   mat          host [nz][ny][nx] packed material bytes (copied)
 *   n_mat        1..4 materials; mat_wp2/mat_nu [n_mat] (entry 0 must be vacuum: wp2 = 0)
 *   pulse        Eq. 15 pulse of the incident line and of the sheet source
 *   probes       host [n_probes][3] (i, j, k) of the Ex samples; dft as for the 1D calls
 *   stream       cudaStream_t for all work of this context (NULL = legacy default stream)
 * Memory: 9 field arrays of nx ny nz values, one material byte per cell, CPML memories only
 * in the face slabs. Errors: RKETD_EINVAL, RKETD_ECOURANT, RKETD_ENOMEM, RKETD_ECUDA;
 * *out is NULL on error.
 */
rketd_status rketd_create_3d(const rketd_grid3d* grid, const uint8_t* mat, int32_t n_mat, const double* mat_wp2,
                             const double* mat_nu, const rketd_pulse* pulse, int32_t n_probes, const int32_t* probes,
                             const rketd_dft* dft, void* stream, rketd_ctx3d** out);

/* Zeroes fields, CPML memories, the incident line and the DFT sums; step index 0 (async). */
rketd_status rketd_reset_3d(rketd_ctx3d* ctx);

/* Queues nsteps steps: H (+CPML, TF/SF), incident H, E and J (+CPML, TF/SF, sheet),
 * incident E, probe samples; the DFT is folded every 512 samples. Both variants give the
 * same arithmetic, operation by operation. Async. */
rketd_status rketd_step_3d(rketd_ctx3d* ctx, int64_t nsteps);

/* Copies one component to a host FP64 SI array [nz][ny][nx]: which = 0..8 for Ex, Ey, Ez,
 * Hx, Hy, Hz, Jx, Jy, Jz. Synchronises. */
rketd_status rketd_get_field_3d(rketd_ctx3d* ctx, int32_t which, double* out);

/* Copies the DFT sums to host: re/im [n_probes][n_freq] (FP64), samples not yet folded
 * included. Synchronises. */
rketd_status rketd_get_spectra_3d(rketd_ctx3d* ctx, double* re, double* im);

/* Waits for the context's stream; RKETD_ETIMEOUT if a bounded wait of the staged form gave
 * up (its fields are then not valid). */
rketd_status rketd_sync_3d(rketd_ctx3d* ctx);

/* Sets the number of z planes (1..4096) one thread block advances per step (default 64).
 * A tuning knob: results do not depend on it. */
rketd_status rketd_kernel_chunk_3d(rketd_ctx3d* ctx, int32_t k_chunk);

/* Test hook: the staged form's compute threads give up waiting for a staged copy after `polls`
 * polls of its mbarrier (0: at once; < 0 restores the default of 2^20). A block whose wait gave up
 * stops, lets the copies it issued land (those waits keep the full bound), and the next
 * rketd_sync_3d returns RKETD_ETIMEOUT; rketd_reset_3d clears the status. No effect on the fused
 * and plain forms. */
rketd_status rketd_set_wait_limit_3d(rketd_ctx3d* ctx, int32_t polls);

/* Work of the staged form per kind of work item, in tile-planes (32 x 8 cells of one z plane):
 * [0] boundary tiles reaching the x and y CPML, [1] interior tiles in the middle z range, [2]
 * interior tiles in the z CPML slabs and at the TF/SF z faces or the sheet, [3] boundary tiles
 * reaching the x CPML only, [4] the y CPML only, [5] only TF/SF x/y faces. All 0 for the fused and
 * plain forms. Host only. */
rketd_status rketd_work_3d(const rketd_ctx3d* ctx, int64_t tile_planes[6]);

/* As rketd_check_finite, for the 3D fields (E, H, J) and spectra. Synchronises. */
rketd_status rketd_check_finite_3d(rketd_ctx3d* ctx);

/* Number of kernel launches this context has issued. */
int64_t rketd_launch_count_3d(const rketd_ctx3d* ctx);

/* Releases the 3D context and its device memory. NULL is accepted. */
rketd_status rketd_destroy_3d(rketd_ctx3d* ctx);

/* ---------------------------------------------------------------------------------------
 * 2D RKETD-FDTD (fields uniform along z): the paper's stated generalisation (Sec. IV.B closing
 * remarks, Sec. V) of the 1D scheme, Eqs. 14, 12, 11 and 13 applied to the 2D curl, in two
 * polarisations on an nx x ny Yee grid of cell size d; arrays are [j][i] (x fastest).
 *   RKETD_TMZ: Ez (i, j), Hx (i, j+1/2), Hy (i+1/2, j), current Jz;
 *   RKETD_TEZ: Hz (i+1/2, j+1/2), Ex (i+1/2, j), Ey (i, j+1/2), currents Jx, Jy.
 * Every E component of cell (i, j) takes the Drude material mat[j][i] (0..n_mat-1, 0 = vacuum).
 * Boundaries: first-order Mur on the E components tangential to the y faces (rows 0 and ny-1);
 * periodic x, or first-order Mur on those tangential to the x faces (columns 0 and nx-1). Source:
 * a soft line source on row src_j adding profile[i] s(t) to Ez (TMz) or Ex (TEz) after the E
 * update (s the Eq. 15 pulse), on the nodes the update advances (with Mur x ends TEz has no Ex at
 * column nx-1, position nx-1/2: it stays 0, and a probe there reads 0); with periodic x and profile[i] = cos(2 pi m i / nx) it launches one
 * transverse Fourier mode, which meets a y-layered medium at oblique incidence. Probes sample Ez
 * (TMz) or Ex (TEz); running DFT as rketd_dft. The step is the paper's two-kernel structure (an H
 * kernel, then an E+J kernel with the source and the ends), fields in place.
 * ------------------------------------------------------------------------------------- */
typedef enum { RKETD_TMZ = 0, RKETD_TEZ = 1 } rketd_pol2d;

typedef struct {
  int32_t nx, ny;        /* cells per axis, >= 4 */
  int32_t prec;          /* rketd_prec */
  int32_t pol;           /* rketd_pol2d */
  double d, dt;          /* cell size (m), time step (s); c0 dt / d <= 1/sqrt(2) */
  int32_t periodic_x;    /* 1: periodic in x; 0: first-order Mur at the x faces */
  int32_t src_j;         /* source row, 1 <= src_j <= ny-2 */
} rketd_grid2d;

typedef struct rketd_ctx2d rketd_ctx2d;

/*
 * Creates a 2D context and zeroes its state.
 *   mat           host [ny][nx] material indices (copied); n_mat 1..16 materials, mat_wp2/mat_nu
 *                 [n_mat] (entry 0 must be vacuum), finite and >= 0
 *   profile       host [nx] source weights per column (copied)
 *   probes        host [n_probes][2] (i, j) cells; dft as for the 1D calls
 *   stream        cudaStream_t for all work of this context (NULL = legacy default stream)
 * Errors: RKETD_EINVAL, RKETD_ECOURANT, RKETD_ENOMEM, RKETD_ECUDA; *out is NULL on error.
 */
rketd_status rketd_create_2d(const rketd_grid2d* grid, const uint8_t* mat, int32_t n_mat, const double* mat_wp2,
                             const double* mat_nu, const double* profile, const rketd_pulse* pulse, int32_t n_probes,
                             const int32_t* probes, const rketd_dft* dft, void* stream, rketd_ctx2d** out);

/* Zeroes the fields and the DFT sums; step index 0 (async). */
rketd_status rketd_reset_2d(rketd_ctx2d* ctx);

/* Queues nsteps steps (H, E and J with the source and the Mur ends, probe samples; the DFT is
 * folded every 512 samples). Async. */
rketd_status rketd_step_2d(rketd_ctx2d* ctx, int64_t nsteps);

/* Waits for the context's stream and reports any device-side error. */
rketd_status rketd_sync_2d(rketd_ctx2d* ctx);

/* Copies one component to a host FP64 SI array [ny][nx]: which = 0..3 for TMz (Ez, Hx, Hy, Jz),
 * 0..4 for TEz (Ex, Ey, Hz, Jx, Jy). Synchronises. */
rketd_status rketd_get_field_2d(rketd_ctx2d* ctx, int32_t which, double* out);

/* Copies the DFT sums to host: re/im [n_probes][n_freq] (FP64), pending samples included. Synchronises. */
rketd_status rketd_get_spectra_2d(rketd_ctx2d* ctx, double* re, double* im);

/* Number of kernel launches this context has issued. */
int64_t rketd_launch_count_2d(const rketd_ctx2d* ctx);

/* As rketd_check_finite, for the 2D fields, currents and spectra. Synchronises. */
rketd_status rketd_check_finite_2d(rketd_ctx2d* ctx);

/* Releases the 2D context and its device memory. NULL is accepted. */
rketd_status rketd_destroy_2d(rketd_ctx2d* ctx);

/* Message for the last failing call on this thread ("" if none). */
const char* rketd_last_error(void);

/* Library version string. */
const char* rketd_version(void);

#ifdef __cplusplus
}
#endif

#endif /* RKETD_H */
