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
#include "tile_bodies.cuh"

// Resident CTAs of 4 warps per SM the interior kernel is compiled for (register cap).
#ifndef RKETD_TB_MINB
#define RKETD_TB_MINB 3
#endif
// Resident CTAs of 4 warps per SM the FP32 edge kernel with 4 cells per lane is compiled for: 4
// (126 registers, no spills, 16 warps per SM instead of 12). Its tiles are latency-bound, and the
// extra warps made a pass of the 4096-slab batch 2.2% shorter.
#ifndef RKETD_TB_EDGE_MINB
#define RKETD_TB_EDGE_MINB 4
#endif

namespace rketd {
namespace {

using namespace tile;

// XTRA: the tiles may sample a probe or hold their slab's source cell (always so for edge tiles
// and the recording recompute; the planner launches the few interior tiles that do apart from the
// rest, so that the main launch carries no per-step branch for them).
template <typename T, int K, bool EDGE, bool REC, bool XTRA>
__global__ void __launch_bounds__(128, EDGE ? (sizeof(T) == 4 && K == 4 ? RKETD_TB_EDGE_MINB : 1) : RKETD_TB_MINB)
    k_tb(const StepArgs<T> a) {
  const int lane = threadIdx.x & 31;
  const int tid = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (tid >= a.n_tiles) return;  // uniform per warp
  tb_tile<T, K, EDGE, REC, XTRA, true>(a, a.tiles[tid], lane, a.n0, a.series_pos);
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
