// Per-cell RKETD update coefficients (Eqs. 11-13, and the Eq. 9 / Eq. 10 recursions) and CPML
// grading tables, in FP64 on the device (layout and the folded current G = cj J~ - da E are
// described in rketd_internal.cuh).
// The FP32 path stores the same FP64 results rounded once to FP32; every coefficient is a
// deviation from its vacuum value or a small term, so rounding keeps its relative accuracy
// (a = e^{-nu dt} itself would lose most of a - 1 in FP32).
#include "rketd_internal.cuh"

namespace rketd {
namespace {

// phi1(x) = (1 - e^{-x})/x and phi2(x) = (e^{-x} - 1 + x)/x^2 (x = nu dt), the integrals that
// take the exact solution Eq. 7 with F interpolated linearly over the step to Eq. 11, and
// psi = phi1 - (1 + e^{-x}) phi2 of the folded current's bq.
// Below x = 0.5 all are Taylor polynomials of degree 20 (coefficients (-1)^k/(k+1)!,
// (-1)^k/(k+2)! and, for (phi1 - 2 phi2)/x, (-1)^(k+1) (k+1)/(k+3)!) evaluated by Horner's rule;
// the first omitted term is below 1e-27. From x = 0.5 up, expm1 keeps 1 - e^{-x} exact to rounding.
// Taylor coefficients of the three series (c1: phi1, c2: phi2, c3: (phi1 - 2 phi2)/x), each from the
// previous by one division in FP64, evaluated at compile time (the same operations as at run time,
// without ~60 FP64 divisions per cell on a part with few FP64 units).
struct PhiSeries {
  double c1[21], c2[21], c3[21];
};
__host__ __device__ constexpr PhiSeries phi_series() {
  PhiSeries t{};
  t.c1[0] = 1.0;
  t.c2[0] = 0.5;
  t.c3[0] = -1.0 / 6.0;  // k = 1 term of the sum for phi1 - 2 phi2, divided by x
  for (int k = 1; k <= 20; ++k) {
    t.c1[k] = -t.c1[k - 1] / (double)(k + 1);
    t.c2[k] = -t.c2[k - 1] / (double)(k + 2);
    t.c3[k] = -t.c3[k - 1] * (double)(k + 1) / ((double)k * (double)(k + 3));
  }
  return t;
}

__device__ void phi12(double x, double& p1, double& p2, double& psi) {
  if (x < 0.5) {
    // psi = phi1 - (1 + a) phi2 = (phi1 - 2 phi2) + x phi1 phi2 (1 + a = 2 - x phi1), where
    // phi1 - 2 phi2 = x sum_{k>=1} (-1)^k k/(k+2)! x^{k-1}: no cancellation as x -> 0 (psi ~ x/3)
    constexpr PhiSeries t = phi_series();
    double r1 = t.c1[20], r2 = t.c2[20], r3 = t.c3[20];
#pragma unroll
    for (int k = 19; k >= 0; --k) {
      r1 = fma(r1, x, t.c1[k]);
      r2 = fma(r2, x, t.c2[k]);
      r3 = fma(r3, x, t.c3[k]);
    }
    p1 = r1;
    p2 = r2;
    psi = x * (r3 + r1 * r2);
  } else {
    const double em = expm1(-x);
    p1 = -em / x;
    p2 = (x + em) / (x * x);
    psi = p1 - (2.0 + em) * p2;
  }
}

// scheme 0 (Eq. 11, J~' = a J~ + w phi2 E' + w (phi1 - phi2) E): D = 1 + w phi2/2, the coefficients of
// rketd_internal.cuh. scheme 1 (Eq. 9, J~' = a J~ + w phi1 E): explicit, D = 1, so da = -w phi1/2,
// cb = S, cj = (1 + a)/2 and bq = cq = w phi1/2. scheme 2 (Eq. 10, J~' = a J~ + w (phi1 + phi2) E
// - w phi2 E^{n-1}): D = 1, da = -w (phi1 + phi2)/2, bq = cq = w (phi1 + phi2)/2, and the E^{n-1}
// term enters E' as +ep E^{n-1} and G' as +gp E^{n-1}, ep = w phi2/2, gp = -(1 + a) w phi2/2
// (G' = cj J~' - da E' with G = cj J~ - da E, as for the other schemes).
template <typename T>
__global__ void k_coeffs(const double* __restrict__ wp2, const double* __restrict__ nu,
                         const int64_t* __restrict__ soff, const int64_t* __restrict__ off,
                         const int64_t* __restrict__ nz, int n_slabs, int64_t n_store, double dt,
                         double S, int scheme, T* __restrict__ da, T* __restrict__ cb, T* __restrict__ cj,
                         T* __restrict__ dj, T* __restrict__ bq, T* __restrict__ cq, T* __restrict__ ep,
                         T* __restrict__ gp) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_store;
       i += (int64_t)gridDim.x * blockDim.x) {
    // slab owning storage cell i: last s with soff[s] <= i
    int lo = 0, hi = n_slabs - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (soff[mid] <= i) lo = mid; else hi = mid - 1;
    }
    const int64_t k = i - soff[lo];
    double w = 0.0, x = 0.0;
    if (k < nz[lo]) {
      w = wp2[off[lo] + k] * dt * dt;
      x = nu[off[lo] + k] * dt;
    }
    double p1, p2, psi;
    phi12(x, p1, p2, psi);
    const double em = expm1(-x);  // a - 1
    // End cells are set by the boundary condition, never by Eq. 12, and carry no current:
    // da = 0 there makes G = cj J~ hold for them too (the step kernels do not read da).
    const bool end = k == 0 || k == nz[lo] - 1;
    dj[i] = (T)em;
    if (scheme == 0) {
      const double D = 1.0 + 0.5 * w * p2;
      const double h = 0.5 * w / D;
      da[i] = end ? T(0) : (T)(-h * p1);
      cb[i] = (T)(S / D);
      cj[i] = (T)(0.5 * (2.0 + em) / D);  // (1 + a)/(2D)
      bq[i] = (T)(h * psi);                     // cj bp + da a
      cq[i] = (T)(h * (p1 + (2.0 + em) * p2));  // cj cc - da
    } else {
      const double h = 0.5 * w;
      const double f = scheme == 1 ? p1 : p1 + p2;  // the E^n weight of J~' is w f
      da[i] = end ? T(0) : (T)(-h * f);
      cb[i] = (T)S;
      cj[i] = (T)(0.5 * (2.0 + em));
      bq[i] = (T)(h * f);
      cq[i] = (T)(h * f);
      if (scheme == 2) {
        ep[i] = end ? T(0) : (T)(h * p2);
        gp[i] = end ? T(0) : (T)(-(2.0 + em) * h * p2);
      }
    }
  }
}

// CPML (Roden-Gedney) b, c and 1/kappa against depth. E nodes: depth d = 0..n cells from
// the outer wall, rho = (n - d)/n; H nodes: depth i + 1/2, rho = (n - i - 1/2)/n.
// sigma = smax rho^m, kappa = 1 + (kmax - 1) rho^m, alpha = amax (1 - rho),
// b = exp(-(sigma/kappa + alpha) dt/eps0), c = sigma (b - 1)/(sigma kappa + kappa^2 alpha).
template <typename T>
__global__ void k_cpml(int n, double dt, double m, double smax, double kmax, double amax,
                       T* __restrict__ tabE, T* __restrict__ tabH) {
  const int i = threadIdx.x;
  for (int which = 0; which < 2; ++which) {
    const int count = which == 0 ? n + 1 : n;
    if (i >= count) continue;
    const double rho = which == 0 ? (double)(n - i) / n : ((double)n - i - 0.5) / n;
    const double pm = pow(rho, m);
    const double sigma = smax * pm;
    const double kap = 1.0 + (kmax - 1.0) * pm;
    const double alpha = amax * (1.0 - rho);
    // the memory's decay b = e^{-(sigma/kappa + alpha) dt / eps0} lies within 1e-5 of 1 near the
    // inner interface: it is kept as db = b - 1 (expm1 in FP64), so that an FP32 copy keeps full
    // relative accuracy, and the update reads psi' = psi + db psi + c dv
    const double db = expm1(-(sigma / kap + alpha) * dt / kEps0);
    const double den = sigma * kap + kap * kap * alpha;
    const double c = (sigma > 0.0 && den > 0.0) ? sigma * db / den : 0.0;
    T* tab = which == 0 ? tabE : tabH;
    tab[i] = (T)db;
    tab[count + i] = (T)c;
    tab[2 * count + i] = (T)(1.0 / kap);
  }
}

// Split-field PML (the paper's boundary) per depth: E nodes d = 0..n (rho = (n - d)/n), H nodes
// i + 1/2 (rho = (n - i - 1/2)/n); sigma = smax rho^m, x = sigma dt/eps0 (sigma* dt/mu0 for H with the
// matched sigma*), the update x' = e^{-x} x - S phi1(x) D on normalised fields: stored as
// da = e^{-x} - 1 (expm1) and c = S phi1(x), rows [da | c].
template <typename T>
__global__ void k_pml(int n, double dt, double S, double m, double smax, T* __restrict__ tabE,
                      T* __restrict__ tabH) {
  const int i = threadIdx.x;
  for (int which = 0; which < 2; ++which) {
    const int count = which == 0 ? n + 1 : n;
    if (i >= count) continue;
    const double rho = which == 0 ? (double)(n - i) / n : ((double)n - i - 0.5) / n;
    const double x = smax * pow(rho, m) * dt / kEps0;
    double p1, p2, psi;
    phi12(x, p1, p2, psi);
    T* tab = which == 0 ? tabE : tabH;
    tab[i] = (T)expm1(-x);
    tab[count + i] = (T)(S * p1);
  }
}

}  // namespace

cudaError_t launch_pml_tables(int prec, int n, double dt, double S, double m, double smax, void* tabE, void* tabH,
                              cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int threads = ((n + 1 + 31) / 32) * 32;
  if (prec == 1)
    k_pml<double><<<1, threads, 0, st>>>(n, dt, S, m, smax, (double*)tabE, (double*)tabH);
  else
    k_pml<float><<<1, threads, 0, st>>>(n, dt, S, m, smax, (float*)tabE, (float*)tabH);
  return cudaGetLastError();
}

cudaError_t launch_coeffs(int prec, const double* wp2, const double* nu, const int64_t* soff,
                          const int64_t* off, const int64_t* nz, int n_slabs, int64_t n_store,
                          double dt, double S, void* const coef[kNumCoef], cudaStream_t st, int scheme,
                          void* const ext[2]) {
  const int threads = 256;
  int64_t blocks = (n_store + threads - 1) / threads;
  if (blocks > 152 * 64) blocks = 152 * 64;
  if (blocks < 1) blocks = 1;
  if (scheme < 0 || scheme > 2 || (scheme == 2 && (!ext || !ext[0] || !ext[1]))) return cudaErrorInvalidValue;
  void* e0 = scheme == 2 ? ext[0] : nullptr;
  void* e1 = scheme == 2 ? ext[1] : nullptr;
  if (prec == 1) {
    k_coeffs<double><<<(unsigned)blocks, threads, 0, st>>>(
        wp2, nu, soff, off, nz, n_slabs, n_store, dt, S, scheme, (double*)coef[0], (double*)coef[1],
        (double*)coef[2], (double*)coef[3], (double*)coef[4], (double*)coef[5], (double*)e0, (double*)e1);
  } else {
    k_coeffs<float><<<(unsigned)blocks, threads, 0, st>>>(
        wp2, nu, soff, off, nz, n_slabs, n_store, dt, S, scheme, (float*)coef[0], (float*)coef[1],
        (float*)coef[2], (float*)coef[3], (float*)coef[4], (float*)coef[5], (float*)e0, (float*)e1);
  }
  return cudaGetLastError();
}

cudaError_t launch_cpml_tables(int prec, int ncpml, double dt, double m, double smax, double kmax,
                               double amax, void* cpmlE, void* cpmlH, cudaStream_t st) {
  if (ncpml <= 0) return cudaSuccess;
  const int threads = ((ncpml + 1 + 31) / 32) * 32;
  if (prec == 1)
    k_cpml<double><<<1, threads, 0, st>>>(ncpml, dt, m, smax, kmax, amax, (double*)cpmlE, (double*)cpmlH);
  else
    k_cpml<float><<<1, threads, 0, st>>>(ncpml, dt, m, smax, kmax, amax, (float*)cpmlE, (float*)cpmlH);
  return cudaGetLastError();
}

}  // namespace rketd

namespace rketd {
namespace {
template <typename T>
__global__ void k_rescale(T* G, const T* E, const T* cj_new, const T* cj_old, const T* da_new, const T* da_old,
                          int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  // cj_old = 0: no coefficients yet (the first medium of a new context, state all zero)
  if (i >= n || cj_old[i] == T(0)) return;
  // J~ = (G + da E)/cj is kept across the change; G' = cj' J~ - da' E
  const double e = (double)E[i];
  const double jt = ((double)G[i] + (double)da_old[i] * e) / (double)cj_old[i];
  G[i] = (T)((double)cj_new[i] * jt - (double)da_new[i] * e);
}
}  // namespace

cudaError_t launch_rescale(int prec, void* G, const void* E, const void* cj_new, const void* cj_old,
                           const void* da_new, const void* da_old, int64_t n, cudaStream_t st) {
  const unsigned blocks = (unsigned)((n + 255) / 256);
  if (prec == 1)
    k_rescale<double><<<blocks, 256, 0, st>>>((double*)G, (const double*)E, (const double*)cj_new,
                                              (const double*)cj_old, (const double*)da_new, (const double*)da_old, n);
  else
    k_rescale<float><<<blocks, 256, 0, st>>>((float*)G, (const float*)E, (const float*)cj_new, (const float*)cj_old,
                                             (const float*)da_new, (const float*)da_old, n);
  return cudaGetLastError();
}
}  // namespace rketd
