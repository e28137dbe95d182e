// The paper's two-kernel structure (Sec. III): an H-update kernel then an E-update
// kernel per time step, one cell per thread, fields in global memory. Here the E kernel
// also advances the current (Eq. 11 needs E^n and E^{n+1} of the same cell, so it stays in
// a register), adds the Eq. 15 source and applies the end conditions; a third small kernel
// copies the probe samples. This is the streaming form (one HBM pass per step) that the
// temporally blocked kernel is measured against, and the form that runs the Eq. 10 recursion
// (whose E^{n-1} is one more array, updated in place).
#include "rketd_internal.cuh"

namespace rketd {
namespace {

__device__ __forceinline__ double pulse(double t, double t0, double tau, double amp) {
  const double u = (t - t0) / tau;
  return amp * u * exp(-0.5 * u * u);
}

// slab of storage cell i: cell_slab lookup for batches, slab 0 otherwise
__device__ __forceinline__ int slab_of(const int32_t* cell_slab, int64_t i) {
  return cell_slab ? cell_slab[i] : 0;
}

// H update of storage cell i (slab s, slab-local cell k)
template <typename T>
__device__ __forceinline__ void h_cell(const StepArgs<T>& a, int64_t i, int s, int64_t k, int64_t nz) {
  if (k > nz - 2) return;  // H nodes k+1/2, k = 0..nz-2
  T* H = a.H_out;
  const T dE = a.E_in[i + 1] - a.E_in[i];
  const int nc = a.ncpml;
  if (a.bc == 2 && (k < nc || k >= nz - 1 - nc)) {  // split-field PML
    const int ih = (int)(k < nc ? k : nz - 2 - k);
    H[i] = pml_update(H[i], a.cpmlH[ih], a.cpmlH[nc + ih], dE);
  } else if (a.bc == 1 && (k < nc || k >= nz - 1 - nc)) {
    const int ih = (int)(k < nc ? k : nz - 2 - k);
    const int64_t pi = (int64_t)s * 2 * nc + (k < nc ? k : nc + (nz - 2 - k));
    const T db = a.cpmlH[ih], c = a.cpmlH[nc + ih], ki = a.cpmlH[2 * nc + ih];
    const T po = a.psiH_out[pi];
    const T psi = fma(db, po, fma(c, dE, po));
    a.psiH_out[pi] = psi;
    H[i] = fma(-a.S, fma(dE, ki, psi), H[i]);
  } else {
    H[i] = fma(-a.S, dE, H[i]);
  }
}

// E and current update of storage cell i (slab s, slab-local cell k), with the source and the ends
template <typename T>
__device__ __forceinline__ void ej_cell(const StepArgs<T>& a, int64_t i, int s, int64_t k, int64_t nz) {
  if (k < 1 || k > nz - 2) return;  // interior E nodes; the end cells are set below
  T* E = a.E_out;
  T* J = a.J_out;
  const T dH = a.H_in[i] - a.H_in[i - 1];
  T curl = dH;
  const int nc = a.ncpml;
  if (a.bc == 2 && (k < nc || k > nz - 1 - nc)) {  // split-field PML: vacuum, no current, no source
    const int d = (int)(k < nc ? k : nz - 1 - k);
    const T enew = pml_update(E[i], a.cpmlE[d], a.cpmlE[nc + 1 + d], dH);
    if (k == 1) E[i - 1] = T(0);
    if (k == nz - 2) E[i + 1] = T(0);
    E[i] = enew;
    return;
  }
  if (a.bc == 1 && (k < nc || k > nz - 1 - nc)) {
    const int d = (int)(k < nc ? k : nz - 1 - k);
    const int64_t pi = (int64_t)s * 2 * nc + (k < nc ? k : nc + (nz - 1 - k));
    const T db = a.cpmlE[d], c = a.cpmlE[nc + 1 + d], ki = a.cpmlE[2 * (nc + 1) + d];
    const T po = a.psiE_out[pi];
    const T psi = fma(db, po, fma(c, dH, po));
    a.psiE_out[pi] = psi;
    curl = fma(dH, ki, psi);
  }
  // J holds the folded current G (rketd_internal.cuh)
  const T en = E[i];
  const T go = J[i];
  T enew, gn;
  if (a.Ep == nullptr) {
    enew = fold_e(en, a.coef[kCb][i], curl, go);
    gn = fold_g(go, a.coef[kDj][i], a.coef[kBq][i], a.coef[kCq][i], en, enew);
  } else {
    // Eq. 10 read literally: E^{n-1} enters both updates (its small terms summed first, as above)
    const T pv = a.Ep[i];
    enew = en - fma(a.coef[kCb][i], curl, fma(-a.ep[i], pv, go));
    gn = go + fma(a.gp[i], pv, fma(a.coef[kCq][i], enew, fma(a.coef[kBq][i], en, a.coef[kDj][i] * go)));
    a.Ep[i] = en;
  }
  if (k == a.src[s]) {
    const T sv = (T)pulse((double)(a.n0 + 1) * a.dt, a.t0, a.tau, a.amp);
    enew += sv;
    gn = fma(-a.coef[kDa][i], sv, gn);
  }
  J[i] = gn;
  // The thread of cell 1 owns cell 0 and the thread of cell nz-2 owns cell nz-1: Mur needs
  // E_1^n and E_1^{n+1}, which only this thread has (cells are updated in place).
  if (k == 1) {
    if (a.bc == 0) {
      const T e0 = E[i - 1];
      E[i - 1] = fma(a.qmur, enew - e0, en);
    } else {
      E[i - 1] = T(0);
    }
  }
  if (k == nz - 2) {
    if (a.bc == 0) {
      const T eN = E[i + 1];
      E[i + 1] = fma(a.qmur, enew - eN, en);
    } else {
      E[i + 1] = T(0);
    }
  }
  E[i] = enew;
}

// Vectorised streaming kernels: each thread takes kV consecutive storage cells (slabs start at
// multiples of 32 cells, so a group never straddles two slabs and its 16-byte loads are aligned).
// One FP32 cell per thread kept too few bytes in flight to cover the HBM latency (the H kernel ran at
// 30% of the copy bandwidth); kV cells per thread issue wide loads. A group whose cells are all plain
// interior cells (no end cell or its Mur owner, no CPML or PML layer, no source, and in FP32 not the
// Eq. 10 recursion) takes the vector path; any other group updates cell by cell through h_cell /
// ej_cell.
// The per-cell operations are the same on both paths.
constexpr int kV = 4;

template <typename T>
struct Vec4 {
  T v[4];
};
__device__ __forceinline__ Vec4<float> ldv(const float* p) {
  const float4 q = *reinterpret_cast<const float4*>(p);
  return {{q.x, q.y, q.z, q.w}};
}
__device__ __forceinline__ Vec4<double> ldv(const double* p) {
  const double2 q0 = reinterpret_cast<const double2*>(p)[0];
  const double2 q1 = reinterpret_cast<const double2*>(p)[1];
  return {{q0.x, q0.y, q1.x, q1.y}};
}
__device__ __forceinline__ void stv(float* p, const Vec4<float>& r) {
  *reinterpret_cast<float4*>(p) = make_float4(r.v[0], r.v[1], r.v[2], r.v[3]);
}
__device__ __forceinline__ void stv(double* p, const Vec4<double>& r) {
  reinterpret_cast<double2*>(p)[0] = make_double2(r.v[0], r.v[1]);
  reinterpret_cast<double2*>(p)[1] = make_double2(r.v[2], r.v[3]);
}

template <typename T>
__global__ void __launch_bounds__(256) k_plain_h(const StepArgs<T> a, const int32_t* __restrict__ cell_slab,
                                                 int64_t n_store) {
  const int64_t i0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) * kV;
  if (i0 >= n_store) return;
  const int s = slab_of(cell_slab, i0);
  const int64_t k0 = i0 - a.soff[s];
  const int64_t nz = a.nz[s];
  const int nc = a.ncpml;
  const bool layers = a.bc != 0 && (k0 < nc || k0 + kV - 1 >= nz - 1 - nc);
  if (k0 + kV - 1 <= nz - 2 && !layers) {
    const Vec4<T> e = ldv(a.E_in + i0);
    const T e4 = a.E_in[i0 + kV];
    Vec4<T> h = ldv(a.H_out + i0);
#pragma unroll
    for (int q = 0; q < kV; ++q) h.v[q] = fma(-a.S, (q + 1 < kV ? e.v[q + 1] : e4) - e.v[q], h.v[q]);
    stv(a.H_out + i0, h);
    return;
  }
  for (int q = 0; q < kV && k0 + q < nz; ++q) h_cell(a, i0 + q, s, k0 + q, nz);
}

template <typename T>
__global__ void __launch_bounds__(256) k_plain_ej(const StepArgs<T> a, const int32_t* __restrict__ cell_slab,
                                                  int64_t n_store) {
  const int64_t i0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) * kV;
  if (i0 >= n_store) return;
  const int s = slab_of(cell_slab, i0);
  const int64_t k0 = i0 - a.soff[s];
  const int64_t nz = a.nz[s];
  const int nc = a.ncpml;
  const int64_t src = a.src[s];
  // plain cells: 2 <= k <= nz - 3 (cells 1 and nz - 2 also set the Mur/PEC end cells), outside the layers
  // (the Eq. 10 recursion takes the vector path in FP64 only: measured on a 2^24-cell slab, its FP32
  // vector form ran the E kernel at a third of the copy rate, slower than cell by cell)
  const bool plain = k0 >= 2 && k0 + kV - 1 <= nz - 3 && !(a.bc != 0 && (k0 < nc || k0 + kV - 1 > nz - 1 - nc)) &&
                     !(src >= k0 && src < k0 + kV) && (a.Ep == nullptr || sizeof(T) == 8);
  if (plain) {
    const Vec4<T> h = ldv(a.H_in + i0);
    const T hm = a.H_in[i0 - 1];
    Vec4<T> e = ldv(a.E_out + i0), g = ldv(a.J_out + i0);
    const Vec4<T> cb = ldv(a.coef[kCb] + i0), dj = ldv(a.coef[kDj] + i0), bq = ldv(a.coef[kBq] + i0),
                  cq = ldv(a.coef[kCq] + i0);
    if (a.Ep == nullptr) {
#pragma unroll
      for (int q = 0; q < kV; ++q) {
        const T dH = h.v[q] - (q ? h.v[q - 1] : hm);
        const T en = e.v[q];
        const T enew = fold_e(en, cb.v[q], dH, g.v[q]);
        g.v[q] = fold_g(g.v[q], dj.v[q], bq.v[q], cq.v[q], en, enew);
        e.v[q] = enew;
      }
    } else {  // Eq. 10: the operations of ej_cell, E^{n-1} and its weights read as vectors too
      Vec4<T> pv = ldv(a.Ep + i0);
      const Vec4<T> ep = ldv(a.ep + i0), gp = ldv(a.gp + i0);
#pragma unroll
      for (int q = 0; q < kV; ++q) {
        const T dH = h.v[q] - (q ? h.v[q - 1] : hm);
        const T en = e.v[q], go = g.v[q];
        const T enew = en - fma(cb.v[q], dH, fma(-ep.v[q], pv.v[q], go));
        g.v[q] = go + fma(gp.v[q], pv.v[q], fma(cq.v[q], enew, fma(bq.v[q], en, dj.v[q] * go)));
        pv.v[q] = en;
        e.v[q] = enew;
      }
      stv(a.Ep + i0, pv);
    }
    stv(a.E_out + i0, e);
    stv(a.J_out + i0, g);
    return;
  }
  for (int q = 0; q < kV && k0 + q < nz; ++q) ej_cell(a, i0 + q, s, k0 + q, nz);
}

template <typename T>
__global__ void k_probe_gather(const T* __restrict__ E, const int64_t* __restrict__ probe_index, int n,
                               T* __restrict__ series, int series_len, int pos) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < n) series[(int64_t)p * series_len + pos] = E[probe_index[p]];
}

}  // namespace

template <typename T>
cudaError_t launch_plain_step(const StepArgs<T>& a, const int32_t* cell_slab, int64_t n_store,
                              const int64_t* probe_index, cudaStream_t st) {
  const int threads = 256;
  const unsigned blocks = (unsigned)((n_store / kV + threads - 1) / threads);
  k_plain_h<T><<<blocks, threads, 0, st>>>(a, cell_slab, n_store);
  k_plain_ej<T><<<blocks, threads, 0, st>>>(a, cell_slab, n_store);
  if (a.total_probes > 0)
    k_probe_gather<T><<<(a.total_probes + 127) / 128, 128, 0, st>>>(a.E_out, probe_index, a.total_probes,
                                                                    a.series, a.series_len, a.series_pos);
  return cudaGetLastError();
}

template cudaError_t launch_plain_step<float>(const StepArgs<float>&, const int32_t*, int64_t,
                                              const int64_t*, cudaStream_t);
template cudaError_t launch_plain_step<double>(const StepArgs<double>&, const int32_t*, int64_t,
                                               const int64_t*, cudaStream_t);

}  // namespace rketd
