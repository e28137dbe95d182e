// Running DFT at the probe cells, X_p(f) += sum_m E_p^m exp(-j 2 pi f m dt), the
// transform behind the R(f)/T(f) spectra of Sec. IV.B, folded in blocks: the step
// kernels buffer the probe samples, then one launch builds the block's twiddle table
// (phases from FP64 arguments reduced modulo 2 pi, no rotation recurrence) and one
// launch accumulates every (probe, frequency) pair. FP64 fields accumulate in FP64;
// FP32 fields accumulate each block with compensated (Kahan) FP32 sums whose result
// is added to FP64 totals.
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

__global__ void k_dft64(const double* __restrict__ series, int len, int n, const double* __restrict__ tw,
                        int P, int nf, double* __restrict__ Xr, double* __restrict__ Xi) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= nf) return;
  for (int p = blockIdx.y; p < P; p += gridDim.y) {
    const double* e = series + (int64_t)p * len;
    double ar = 0.0, ai = 0.0;
    for (int t = 0; t < n; ++t) {
      const double v = e[t];
      ar = fma(v, tw[2 * ((int64_t)t * nf + f)], ar);
      ai = fma(v, tw[2 * ((int64_t)t * nf + f) + 1], ai);
    }
    Xr[(int64_t)p * nf + f] += ar;
    Xi[(int64_t)p * nf + f] += ai;
  }
}

__global__ void k_dft32(const float* __restrict__ series, int len, int n, const float* __restrict__ tw,
                        int P, int nf, double* __restrict__ Xr, double* __restrict__ Xi) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= nf) return;
  for (int p = blockIdx.y; p < P; p += gridDim.y) {
    const float* e = series + (int64_t)p * len;
    float sr = 0.f, cr = 0.f, si = 0.f, ci = 0.f;  // Kahan sums and compensations
    for (int t = 0; t < n; ++t) {
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
    Xr[(int64_t)p * nf + f] += (double)sr - (double)cr;
    Xi[(int64_t)p * nf + f] += (double)si - (double)ci;
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

template <>
cudaError_t launch_dft<double>(const double* series, int len, int n, const double* tw, int P, int nf,
                               double* Xr, double* Xi, cudaStream_t st) {
  if (P <= 0 || n <= 0) return cudaSuccess;
  const int threads = nf >= 128 ? 128 : ((nf + 31) / 32) * 32;
  const dim3 grid((nf + threads - 1) / threads, P < 65535 ? P : 65535);
  k_dft64<<<grid, threads, 0, st>>>(series, len, n, tw, P, nf, Xr, Xi);
  return cudaGetLastError();
}
template <>
cudaError_t launch_dft<float>(const float* series, int len, int n, const float* tw, int P, int nf,
                              double* Xr, double* Xi, cudaStream_t st) {
  if (P <= 0 || n <= 0) return cudaSuccess;
  const int threads = nf >= 128 ? 128 : ((nf + 31) / 32) * 32;
  const dim3 grid((nf + threads - 1) / threads, P < 65535 ? P : 65535);
  k_dft32<<<grid, threads, 0, st>>>(series, len, n, tw, P, nf, Xr, Xi);
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
