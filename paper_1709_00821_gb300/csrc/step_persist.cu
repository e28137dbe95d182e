// Persistent tiled step of a ragged batch (FP32): every pass of a run of passes, over all slabs,
// in one launch.
//
// The tile plan of the tiled variant is kept: interior tiles of 32 K cells per warp (packed
// FP32x2 pairs), the interior tiles that sample a probe or load a source cell, and the narrow
// edge tiles, each advancing nsub leapfrog steps per pass between the two copies of the fields.
// Instead of three launches per pass, a grid of resident one-warp blocks takes (pass, tile) work
// items in pass-major order from a global counter, a few at a time. A tile of pass p may start
// once the tiles of its slab whose cells it reads, and those that read the cells it writes, have
// finished pass p - 1 (each tile publishes the last pass it finished; the planner lists those
// neighbours for every tile). No grid-wide barrier is needed, and slabs do not wait for one
// another. Work is taken in order by running warps only, and every dependency of an item lies
// earlier in that order, so the waits always end; each is still bounded (a wait that gives up sets
// the status word, which the next synchronisation reports, and the tile goes on so that nothing
// hangs). Fields are read through L2 (other warps of the launch write them), the coefficients
// through the read-only path. The arithmetic is the tiled kernels' (tile_bodies.cuh), so the
// results are bitwise those of the tiled variant.
#include "rketd_internal.cuh"
#include "tile_bodies.cuh"

namespace rketd {
namespace {

using namespace tile;

constexpr int kGrab = 2;  // work items a warp takes per counter update (8 and 32 measured slower)

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Every lane waits for each neighbour of tile j to have finished pass `need` (bounded polls);
// false if a wait gave up (wait_limit <= 0: at once). Once any wait of the launch has given up
// (status word set) the others give up at their next poll, so that a launch whose results are
// already void ends quickly. (Reading all the neighbours' flags at once, one per lane, followed by
// a fence in every lane, measured 2.6 % slower.)
__device__ __forceinline__ bool wait_deps(const PersistCtl& pc, int j, int need) {
  if (pc.wait_limit <= 0) return false;
  const int d1 = pc.dep_off[j + 1];
  for (int d = pc.dep_off[j]; d < d1; ++d) {
    const int* flag = pc.done + pc.dep_idx[d];
    for (int it = 0; ld_acquire(flag) < need; ++it) {
      if (it >= pc.wait_limit || ld_acquire(pc.err)) return false;
      __nanosleep(64);
    }
  }
  return true;
}

// The tile bodies as calls of their own (not inlined into the work loop), so that each is
// compiled as in its one-tile-per-launch kernel.
template <int K, bool XTRA>
__device__ __noinline__ void tb2_call(const StepArgs<float>& a, const Tile tl, int lane, int64_t n0, int spos) {
  tb2_tile<K, XTRA, false>(a, tl, lane, n0, spos);
}
template <int KE>
__device__ __noinline__ void edge_call(const StepArgs<float>& a, const Tile tl, int lane, int64_t n0, int spos) {
  tb_tile<float, KE, true, false, true, false>(a, tl, lane, n0, spos);
}

template <int K, int KE>
__global__ void __launch_bounds__(32, 12) k_persist(const StepArgs<float>* __restrict__ sa, const PersistCtl pc) {
  const int lane = threadIdx.x;
  const int total = pc.n_pass * pc.n_tiles;
  for (;;) {
    int w0 = 0;
    if (lane == 0) w0 = atomicAdd(pc.work, kGrab);
    w0 = __shfl_sync(0xffffffffu, w0, 0);
    if (w0 >= total) break;
    const int w1 = min(w0 + kGrab, total);
    for (int w = w0; w < w1; ++w) {
      // within a pass: the probe/source tiles and the edge tiles first, then the plain interior
      // tiles, so that the latency-bound short lists are done early and the next pass's first
      // tiles, which border them, seldom wait
      const int pass = w / pc.n_tiles, q = w - pass * pc.n_tiles;
      const int j = q + pc.n_main < pc.n_tiles ? q + pc.n_main : q + pc.n_main - pc.n_tiles;
      if (pass > 0 && !wait_deps(pc, j, pass - 1) && lane == 0) atomicExch(pc.err, 1);
      const StepArgs<float>& a = sa[pass & 1];
      const Tile tl = a.tiles[j];
      const int64_t n0 = a.n0 + (int64_t)pass * pc.nsub;
      const int spos = a.series_pos + pass * pc.nsub;
      if (j < pc.n_main)
        tb2_call<K, false>(a, tl, lane, n0, spos);
      else if (j < pc.n_main + pc.n_xtra)
        tb2_call<K, true>(a, tl, lane, n0, spos);
      else
        edge_call<KE>(a, tl, lane, n0, spos);
      // the tile's stores (every lane) are visible device-wide before its flag
      __threadfence();
      __syncwarp();
      if (lane == 0) st_release(pc.done + j, pass);
    }
  }
}

__global__ void k_set_args(StepArgs<float> a0, StepArgs<float> a1, StepArgs<float>* out) {
  out[0] = a0;
  out[1] = a1;
}

template <int K, int KE>
cudaError_t go(StepArgs<float>* sa_d, const StepArgs<float>& a0, const StepArgs<float>& a1, const PersistCtl& pc,
               int grid, cudaStream_t st) {
  k_set_args<<<1, 1, 0, st>>>(a0, a1, sa_d);
  k_persist<K, KE><<<grid, 32, 0, st>>>(sa_d, pc);
  return cudaGetLastError();
}

template <int K, int KE>
int capacity() {
  int dev = 0, n_sm = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_persist<K, KE>, 32, 0) != cudaSuccess)
    return 0;
  return n_sm * per_sm;
}

}  // namespace

int persist_capacity(int K, int Ke) {
  if (Ke == 4) {
    if (K == 8) return capacity<8, 4>();
    if (K == 12) return capacity<12, 4>();
    if (K == 16) return capacity<16, 4>();
  } else if (Ke == 8) {
    if (K == 8) return capacity<8, 8>();
    if (K == 12) return capacity<12, 8>();
    if (K == 16) return capacity<16, 8>();
  }
  return 0;
}

cudaError_t launch_persist(StepArgs<float>* sa_d, const StepArgs<float>& a0, const StepArgs<float>& a1,
                           const PersistCtl& pc, int K, int Ke, int grid, cudaStream_t st) {
  if (grid <= 0 || pc.n_pass <= 0 || pc.n_tiles <= 0) return cudaErrorInvalidValue;
  if (Ke == 4) {
    if (K == 8) return go<8, 4>(sa_d, a0, a1, pc, grid, st);
    if (K == 12) return go<12, 4>(sa_d, a0, a1, pc, grid, st);
    if (K == 16) return go<16, 4>(sa_d, a0, a1, pc, grid, st);
  } else if (Ke == 8) {
    if (K == 8) return go<8, 8>(sa_d, a0, a1, pc, grid, st);
    if (K == 12) return go<12, 8>(sa_d, a0, a1, pc, grid, st);
    if (K == 16) return go<16, 8>(sa_d, a0, a1, pc, grid, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace rketd
