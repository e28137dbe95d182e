// Running DFT at the probe cells, X_p(f) += sum_m E_p^m exp(-j 2 pi f m dt), the
// transform behind the R(f)/T(f) spectra of Sec. IV.B, folded in blocks: the step
// kernels buffer the probe samples and one launch accumulates every (probe, frequency) pair,
// its samples split over the warps of a block, against a twiddle table (phases from FP64
// arguments reduced modulo 2 pi, no rotation recurrence). The 1D contexts build the table
// once, for sample offsets 0..B-1, and multiply each block's sums by exp(-j 2 pi f m0 dt) of
// the block's first sample m0 (one small launch per fold, in FP64); the 3D contexts build the
// table per block with the absolute sample indices. FP64 fields accumulate in FP64; FP32 fields accumulate each chunk of samples with
// compensated (Kahan) FP32 sums whose results are added to FP64 totals.
#include "rketd_internal.cuh"

namespace rketd {
namespace {

template <typename T>
__global__ void k_twiddles(const double* __restrict__ freq, int n_freq, double dt, int64_t m0, int n,
                           T* __restrict__ tw) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)n * n_freq) return;
  const int t = (int)(idx / n_freq);
  const int f = (int)(idx % n_freq);
  // phase / pi = 2 f m dt, reduced to [0, 2)
  double x = 2.0 * freq[f] * dt * (double)(m0 + t);
  x = x - 2.0 * floor(0.5 * x);
  double sn, cs;
  sincospi(x, &sn, &cs);
  tw[2 * idx] = (T)cs;
  tw[2 * idx + 1] = (T)(-sn);
}

// One block per (32 consecutive frequencies, probe): lane = frequency, the block's warps split the
// samples into contiguous chunks (so a fold of a few probes still spreads over many warps), and the
// warps' partial sums are added in warp order (deterministic: no atomics). FP32 samples accumulate each
// chunk with compensated (Kahan) FP32 sums; the chunk results are combined in FP64.
constexpr int kDftMaxWarps = 16;

// rot[f] = exp(-j 2 pi f m0 dt) in FP64 (phase reduced modulo 2 pi from an FP64 argument).
__global__ void k_rot(const double* __restrict__ freq, int n_freq, double dt, int64_t m0, double* __restrict__ rot) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= n_freq) return;
  double x = 2.0 * freq[f] * dt * (double)m0;
  x = x - 2.0 * floor(0.5 * x);
  double sn, cs;
  sincospi(x, &sn, &cs);
  rot[2 * f] = cs;
  rot[2 * f + 1] = -sn;
}

// rot == nullptr: the table tw holds exp(-j 2 pi f m dt) for the block's own sample indices m. Otherwise
// tw holds exp(-j 2 pi f t dt) for t = 0.. and the block's sum is multiplied by rot[f] = exp(-j 2 pi f m0 dt).
template <typename T>
__global__ void __launch_bounds__(32 * kDftMaxWarps) k_dft(const T* __restrict__ series, int len, int n,
                                                            const T* __restrict__ tw, int P, int nf,
                                                            double* __restrict__ Xr, double* __restrict__ Xi,
                                                            const double* __restrict__ rot) {
  __shared__ double part[kDftMaxWarps][2][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, W = blockDim.x >> 5;
  const int f = blockIdx.x * 32 + lane;
  const int chunk = (n + W - 1) / W;
  const int t0 = w * chunk, t1 = min(n, t0 + chunk);
  for (int p = blockIdx.y; p < P; p += gridDim.y) {
    const T* e = series + (int64_t)p * len;
    double ar = 0.0, ai = 0.0;
    if (f < nf) {
      if constexpr (sizeof(T) == 8) {
        for (int t = t0; t < t1; ++t) {
          const double v = e[t];
          ar = fma(v, tw[2 * ((int64_t)t * nf + f)], ar);
          ai = fma(v, tw[2 * ((int64_t)t * nf + f) + 1], ai);
        }
      } else {
        float sr = 0.f, cr = 0.f, si = 0.f, ci = 0.f;  // Kahan sums and compensations
        for (int t = t0; t < t1; ++t) {
          const float v = e[t];
          const float yr = v * tw[2 * ((int64_t)t * nf + f)] - cr;
          const float tr = sr + yr;
          cr = (tr - sr) - yr;
          sr = tr;
          const float yi = v * tw[2 * ((int64_t)t * nf + f) + 1] - ci;
          const float ti = si + yi;
          ci = (ti - si) - yi;
          si = ti;
        }
        ar = (double)sr - (double)cr;
        ai = (double)si - (double)ci;
      }
    }
    part[w][0][lane] = ar;
    part[w][1][lane] = ai;
    __syncthreads();
    if (w == 0 && f < nf) {
      double sr = 0.0, si = 0.0;
      for (int q = 0; q < W; ++q) {
        sr += part[q][0][lane];
        si += part[q][1][lane];
      }
      if (rot) {
        const double c = rot[2 * f], d = rot[2 * f + 1];  // (c + j d)(sr + j si)
        const double r = c * sr - d * si;
        si = c * si + d * sr;
        sr = r;
      }
      Xr[(int64_t)p * nf + f] += sr;
      Xi[(int64_t)p * nf + f] += si;
    }
    __syncthreads();
  }
}

// Device state to SI: E as is, H = H~/eta0, J = (G + da E)/cj * eps0/dt (G the folded current).
template <typename T>
__global__ void k_gather(const T* __restrict__ E, const T* __restrict__ H, const T* __restrict__ G,
                         const T* __restrict__ cj, const T* __restrict__ da, int64_t off, int64_t nz, double hs,
                         double js, double* Eo, double* Ho, double* Jo) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= nz) return;
  const double e = (double)E[off + k];
  if (Eo) Eo[k] = e;
  if (Ho && k < nz - 1) Ho[k] = (double)H[off + k] * hs;
  if (Jo) Jo[k] = ((double)G[off + k] + (double)da[off + k] * e) / (double)cj[off + k] * js;
}

}  // namespace

template <typename T>
cudaError_t launch_twiddles(const double* freq, int n_freq, double dt, int64_t m0, int n_samples, T* tw,
                            cudaStream_t st) {
  const int64_t total = (int64_t)n_samples * n_freq;
  if (total <= 0) return cudaSuccess;
  k_twiddles<T><<<(unsigned)((total + 255) / 256), 256, 0, st>>>(freq, n_freq, dt, m0, n_samples, tw);
  return cudaGetLastError();
}
template cudaError_t launch_twiddles<float>(const double*, int, double, int64_t, int, float*, cudaStream_t);
template cudaError_t launch_twiddles<double>(const double*, int, double, int64_t, int, double*, cudaStream_t);

template <typename T>
cudaError_t launch_dft(const T* series, int len, int n, const T* tw, int P, int nf, double* Xr, double* Xi,
                       cudaStream_t st, const double* rot) {
  if (P <= 0 || n <= 0) return cudaSuccess;
  // a warp per 64 samples or more, up to kDftMaxWarps; blocks over (frequency chunk, probe)
  int W = (n + 63) / 64;
  W = W < 1 ? 1 : (W > kDftMaxWarps ? kDftMaxWarps : W);
  const dim3 grid((nf + 31) / 32, P < 65535 ? P : 65535);
  k_dft<T><<<grid, 32 * W, 0, st>>>(series, len, n, tw, P, nf, Xr, Xi, rot);
  return cudaGetLastError();
}
template cudaError_t launch_dft<float>(const float*, int, int, const float*, int, int, double*, double*,
                                       cudaStream_t, const double*);
template cudaError_t launch_dft<double>(const double*, int, int, const double*, int, int, double*, double*,
                                        cudaStream_t, const double*);

cudaError_t launch_dft_rotation(const double* freq, int n_freq, double dt, int64_t m0, double* rot, cudaStream_t st) {
  if (n_freq <= 0) return cudaSuccess;
  k_rot<<<(n_freq + 127) / 128, 128, 0, st>>>(freq, n_freq, dt, m0, rot);
  return cudaGetLastError();
}

cudaError_t launch_gather_fields(int prec, const void* E, const void* H, const void* G, const void* cj,
                                 const void* da, int64_t off, int64_t nz, double hs, double js, double* Eo, double* Ho,
                                 double* Jo, cudaStream_t st) {
  const unsigned blocks = (unsigned)((nz + 255) / 256);
  if (prec == 1)
    k_gather<double><<<blocks, 256, 0, st>>>((const double*)E, (const double*)H, (const double*)G, (const double*)cj,
                                             (const double*)da, off, nz, hs, js, Eo, Ho, Jo);
  else
    k_gather<float><<<blocks, 256, 0, st>>>((const float*)E, (const float*)H, (const float*)G, (const float*)cj,
                                            (const float*)da, off, nz, hs, js, Eo, Ho, Jo);
  return cudaGetLastError();
}

}  // namespace rketd
