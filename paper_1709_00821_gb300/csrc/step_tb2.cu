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
#include "tile_bodies.cuh"

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
  const int lane = threadIdx.x & 31;
  const int tid = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (tid >= a.n_tiles) return;  // uniform per warp
  tb2_tile<K, XTRA, true>(a, a.tiles[tid], lane, a.n0, a.series_pos);
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
