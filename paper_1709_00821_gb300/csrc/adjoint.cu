// Discrete adjoint of the tiled step, for gradients of a loss of the probe spectra with
// respect to the per-cell plasma frequency squared and collision frequency.
//
// Device step (rketd_internal.cuh), per interior cell, with the folded current G = cj J~ - da E:
//   H'_k = H_k - S (E_{k+1} - E_k)
//   E'_k = E_k - cb (H'_k - H'_{k-1}) - G_k,   G'_k = G_k + dj G_k + bq E_k + cq E'_k
// then the source (E' += s, and G' -= da s at the source cell: both additive) and the
// first-order Mur ends. Its transpose, from the adjoint (lE, lH, lJ) of (E, H~, G) after the
// step, with mu_k = lE_k + cq_k lJ_k:
//   Mur:      lE_1 += q lE_0, pre-step E_0 gets -q lE_0, pre-step E_1 gets lE_0, lE_0 = 0 (mirror)
//   E and G:  lJ_k <- lJ_k + dj_k lJ_k - mu_k,  lE_k <- mu_k + bq_k lJ_k
//   H:        lH'_k = lH_k - cb_k mu_k + cb_{k+1} mu_{k+1}
//             lE_k += S (lH'_k - lH'_{k-1}),  lH_k <- lH'_k
// The loss enters through the DFT: dL/dE_p^m = sum_f (dL/dRe X cos - dL/dIm X sin)(2 pi f m dt),
// injected at the probe cells before each transposed step. Coefficient gradients per step:
//   d/d(cb) = -mu (H_k - H_{k-1})^{n+1/2}, d/d(dj) = lJ G^n, d/d(bq) = lJ E^n,
//   d/d(cq) = lJ E'^{n+1} (before the source), and at the source cell d/d(da) = -s^{n+1} lJ
//   (lJ, mu after the step),
// summed over steps from values recorded at the window cells, then taken to (wp2, nu) by the
// derivatives of the coefficients (FP64; bq and cq through da, dj and the paper's bp, cc).
#include "rketd_internal.cuh"
#include "tile_common.cuh"

namespace rketd {
namespace {

using namespace tile;

template <typename T, int K, bool EDGE>
__global__ void __launch_bounds__(128, EDGE ? 1 : 2) k_adj(const AdjArgs<T> a) {
  const int lane = threadIdx.x & 31;
  const int tid = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (tid >= a.n_tiles) return;
  const Tile tl = a.tiles[tid];
  const int s = tl.slab;
  const int64_t nz = a.nz[s];
  const int64_t soff = a.soff[s];
  const int64_t nzp = (nz + 31) & ~int64_t(31);
  const int li0 = lane * K;
  const int64_t g0 = tl.start + li0;
  const T S = a.S;

  T le[K], lh[K], lj[K], cb[K], dj[K], bq[K], cq[K];
  load_row<T, K, EDGE>(a.lE_in + soff, g0, nzp, le);
  load_row<T, K, EDGE>(a.lH_in + soff, g0, nzp, lh);
  load_row<T, K, EDGE>(a.lJ_in + soff, g0, nzp, lj);
  load_row<T, K, EDGE>(a.coef[kCb] + soff, g0, nzp, cb);
  load_row<T, K, EDGE>(a.coef[kDj] + soff, g0, nzp, dj);
  load_row<T, K, EDGE>(a.coef[kBq] + soff, g0, nzp, bq);
  load_row<T, K, EDGE>(a.coef[kCq] + soff, g0, nzp, cq);

  uint32_t mH = 0, mE = 0, mrec = 0;
  int i0 = -1, i1 = -1;
#pragma unroll
  for (int i = 0; i < K; ++i) {
    const int64_t g = g0 + i;
    const int li = li0 + i;
    if (!EDGE || (g >= 0 && g <= nz - 2)) mH |= 1u << i;
    if (!EDGE || (g >= 1 && g <= nz - 2)) mE |= 1u << i;
    if (EDGE && g == 0) i0 = i;
    if (EDGE && g == nz - 1) i1 = i;
    if (a.rec && li >= tl.vlo && li < tl.vhi && g >= a.rec_c0 && g < a.rec_c0 + a.rec_w) mrec |= 1u << i;
    if (EDGE && !(g >= 0 && g < nz)) {  // cells outside the slab carry no adjoint
      le[i] = lh[i] = lj[i] = T(0);
    }
    if (EDGE && g == nz - 1) lh[i] = T(0);  // H node nz-1/2 does not exist
  }

  for (int t = a.nsub - 1; t >= 0; --t) {
    const int64_t n = a.n_hi - a.nsub + t;  // transposing step n -> n+1
    const int col = (int)(n - a.seg_n0);
    // ---- loss seeds at every copy of a probe cell ----
    for (int p = 0; p < tl.adj_count; ++p) {
      const TileProbe tp = a.tprobes[tl.adj_begin + p];
      if (lane == tp.local / K) {
        const int sl = tp.local % K;
        put(le, sl, pick(le, sl) + a.seeds[(int64_t)tp.slot * a.seed_len + col]);
      }
    }
    // ---- Mur ends (transposed) ----
    T pre0 = T(0), pre1 = T(0), preN1 = T(0), preN2 = T(0);  // contributions to pre-step E
    if (EDGE) {
      if (i0 >= 0) {
        const T l0 = pick(le, i0);
        put(le, i0 + 1, pick(le, i0 + 1) + a.qmur * l0);  // cell 1 is in this lane (slot of cell 0 <= K-4)
        pre0 = -a.qmur * l0;
        pre1 = l0;
        put(le, i0, T(0));
      }
      // cell nz-2 may sit in the previous lane: send q lE_{nz-1} there
      T lN1 = T(0);
      if (i1 >= 0) {
        lN1 = pick(le, i1);
        preN1 = -a.qmur * lN1;
        preN2 = lN1;
        put(le, i1, T(0));
        if (i1 > 0) put(le, i1 - 1, pick(le, i1 - 1) + a.qmur * lN1);
      }
      const T fromR = __shfl_down_sync(kFull, (i1 == 0) ? a.qmur * lN1 : T(0), 1);
      le[K - 1] += fromR;
    }
    // ---- E and J (transposed) ----
    T mu[K], nu_[K];
#pragma unroll
    for (int i = 0; i < K; ++i) {
      const bool upd = !EDGE || ((mE >> i) & 1u);
      mu[i] = upd ? fma(cq[i], lj[i], le[i]) : T(0);
    }
    if (mrec) {  // record (mu, lJ) of the window cells, whole aligned groups as vectors
      T* r = a.rec + ((int64_t)s * a.rec_len + col) * 2 * a.rec_w;
#pragma unroll
      for (int v = 0; v < K / 4; ++v) {
        const uint32_t m4 = (mrec >> (4 * v)) & 0xFu;
        const int64_t c = g0 + 4 * v - a.rec_c0;
        if (m4 == 0xFu && (c & 3) == 0) {
          st4(r + c, &mu[4 * v]);
          st4(r + a.rec_w + c, &lj[4 * v]);
        } else if (m4) {
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            if (m4 & (1u << q)) {
              r[c + q] = mu[4 * v + q];
              r[a.rec_w + c + q] = lj[4 * v + q];
            }
          }
        }
      }
    }
#pragma unroll
    for (int i = 0; i < K; ++i) {
      const bool upd = !EDGE || ((mE >> i) & 1u);
      const T m = mu[i];
      nu_[i] = cb[i] * m;
      if (upd) {
        const T ljo = lj[i];
        // the carried lJ is added last, as G in the forward step, so that dj lJ (a few ulp of
        // it) is not rounded away on its own
        lj[i] = ljo - fma(-dj[i], ljo, m);
        le[i] = fma(bq[i], ljo, m);
      } else {
        le[i] = T(0);
      }
    }
    // ---- H (transposed): lH'_k = lH_k - nu_k + nu_{k+1} ----
    const T nuR = __shfl_down_sync(kFull, nu_[0], 1);
#pragma unroll
    for (int i = 0; i < K; ++i) {
      const T nr = (i + 1 < K) ? nu_[i + 1] : nuR;
      if (!EDGE || ((mH >> i) & 1u)) lh[i] = lh[i] - nu_[i] + nr;
    }
    const T lhL = __shfl_up_sync(kFull, lh[K - 1], 1);
#pragma unroll
    for (int i = 0; i < K; ++i) {
      const T hp = i ? lh[i - 1] : lhL;
      if (EDGE) {
        const int64_t g = g0 + i;
        if (g >= 0 && g < nz) {
          const T hk = ((mH >> i) & 1u) ? lh[i] : T(0);
          const T hkm = (g >= 1) ? hp : T(0);
          le[i] = fma(S, hk - hkm, le[i]);
        }
      } else {
        le[i] = fma(S, lh[i] - hp, le[i]);
      }
    }
    if (EDGE) {
      if (i0 >= 0) {
        put(le, i0, pick(le, i0) + pre0);
        put(le, i0 + 1, pick(le, i0 + 1) + pre1);
      }
      if (i1 >= 0) put(le, i1, pick(le, i1) + preN1);
      const T toL = __shfl_down_sync(kFull, (i1 == 0) ? preN2 : T(0), 1);
      if (i1 > 0) put(le, i1 - 1, pick(le, i1 - 1) + preN2);
      le[K - 1] += toL;
    }
  }
  store_row<T, K>(a.lE_out + soff, g0, li0, tl.vlo, tl.vhi, le);
  store_row<T, K>(a.lH_out + soff, g0, li0, tl.vlo, tl.vhi, lh);
  store_row<T, K>(a.lJ_out + soff, g0, li0, tl.vlo, tl.vhi, lj);
}

// FP32 interior tiles off the window, two cells per packed FP32x2 register (halves A/B of each
// lane's range, as in the forward k_tb2): every element is rounded as in k_adj.
template <int K>
__global__ void __launch_bounds__(128, 3) k_adj2(const AdjArgs<float> a) {
  constexpr int P = K / 2;
  const int lane = threadIdx.x & 31;
  const int tid = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (tid >= a.n_tiles) return;
  const Tile tl = a.tiles[tid];
  const int64_t base = a.soff[tl.slab] + tl.start + lane * K;
  const int li0 = lane * K;
  f2 le[P], lh[P], lj[P], cb[P], ndj[P], bq[P], cq[P];
  load_pairs<K>(a.lE_in + base, le, false);
  load_pairs<K>(a.lH_in + base, lh, false);
  load_pairs<K>(a.lJ_in + base, lj, false);
  load_pairs<K>(a.coef[kCb] + base, cb, false);
  load_pairs<K>(a.coef[kDj] + base, ndj, true);
  load_pairs<K>(a.coef[kBq] + base, bq, false);
  load_pairs<K>(a.coef[kCq] + base, cq, false);
  const f2 S2 = pk(a.S, a.S);
  for (int t = a.nsub - 1; t >= 0; --t) {
    const int col = (int)(a.n_hi - a.nsub + t - a.seg_n0);
    for (int p = 0; p < tl.adj_count; ++p) {
      const TileProbe tp = a.tprobes[tl.adj_begin + p];
      if (lane == tp.local / K) {
        const int sl = tp.local % K;
        put2(le, sl, pick2(le, sl) + a.seeds[(int64_t)tp.slot * a.seed_len + col]);
      }
    }
    f2 nu[P];
#pragma unroll
    for (int p = 0; p < P; ++p) {
      const f2 m = fma2(cq[p], lj[p], le[p]);
      const f2 ljo = lj[p];
      lj[p] = sub2(ljo, fma2(ndj[p], ljo, m));
      le[p] = fma2(bq[p], ljo, m);
      nu[p] = mul2(cb[p], m);
    }
    // lH'_k = (lH_k - nu_k) + nu_{k+1}; the cell after pair P-1 is (B[0], next lane's A[0])
    const float nextA0 = __shfl_down_sync(kFull, lo_of(nu[0]), 1);
    const f2 nuLast = pk(hi_of(nu[0]), nextA0);
#pragma unroll
    for (int p = 0; p < P; ++p) lh[p] = add2(sub2(lh[p], nu[p]), (p + 1 < P) ? nu[p + 1] : nuLast);
    // lE_k += S (lH'_k - lH'_{k-1}); the cell before pair 0 is (previous lane's B[P-1], A[P-1])
    const float prevB = __shfl_up_sync(kFull, hi_of(lh[P - 1]), 1);
    const f2 lhFirst = pk(prevB, lo_of(lh[P - 1]));
#pragma unroll
    for (int p = 0; p < P; ++p) le[p] = fma2(S2, sub2(lh[p], p ? lh[p - 1] : lhFirst), le[p]);
  }
  store_pairs<K>(a.lE_out + base, li0, tl.vlo, tl.vhi, le);
  store_pairs<K>(a.lH_out + base, li0, tl.vlo, tl.vhi, lh);
  store_pairs<K>(a.lJ_out + base, li0, tl.vlo, tl.vhi, lj);
}

template <typename T, int K>
cudaError_t launch_a(const AdjArgs<T>& a, bool edge, int wpb, cudaStream_t st) {
  const dim3 block(32 * wpb);
  const dim3 grid((a.n_tiles + wpb - 1) / wpb);
  if (edge)
    k_adj<T, K, true><<<grid, block, 0, st>>>(a);
  else
    k_adj<T, K, false><<<grid, block, 0, st>>>(a);
  return cudaGetLastError();
}

template <typename T>
__global__ void k_seeds(const double* __restrict__ gXr, const double* __restrict__ gXi, const T* __restrict__ tw,
                        int P, int nf, int n, T* __restrict__ seeds, int seed_len) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int p = blockIdx.y;
  if (t >= n || p >= P) return;
  double acc = 0.0;
  for (int f = 0; f < nf; ++f) {
    const double c = (double)tw[2 * ((int64_t)t * nf + f)];
    const double sn = (double)tw[2 * ((int64_t)t * nf + f) + 1];  // holds -sin
    acc += gXr[(int64_t)p * nf + f] * c + gXi[(int64_t)p * nf + f] * sn;
  }
  seeds[(int64_t)p * seed_len + t] = (T)acc;
}

// recF[slab][j][3][w] holds the state (E, H~, G) after j steps of the segment (j = 0..L);
// recA[slab][t][2][w] holds (mu, lJ) after step t. Rows start 4 cells before the window: window
// cell c sits at index c + 4, its left neighbour (needed for dH) at c + 3; w is a multiple of 4.
// Each thread sums four window cells over the segment. g[0] collects the source cell's
// d/d(da) (zero elsewhere), g[1..4] d/d(cb), d/d(dj), d/d(bq), d/d(cq).
template <typename T>
__global__ void k_grad(const T* __restrict__ recF, const T* __restrict__ recA, int n_slabs, int w, int nwin, int L,
                       int recF_len, GradSource src, double* __restrict__ g) {
  const int c0 = 4 * (blockIdx.x * blockDim.x + threadIdx.x);  // first of four window cells
  const int s = blockIdx.y;
  if (c0 >= nwin || s >= n_slabs) return;
  const int k = c0 + 4;
  // slot of the source cell among this thread's four, -1 if none
  const int64_t sc = src.cell[s] - src.w_lo - c0;
  const int qs = (sc >= 0 && sc < 4 && c0 + sc < nwin) ? (int)sc : -1;
  float fs[5][4] = {};
  double ds[5][4] = {};
  constexpr bool f64 = sizeof(T) == 8;
#pragma unroll 2
  for (int t = 0; t < L; ++t) {
    const T* F0 = recF + ((int64_t)s * recF_len + t) * 3 * w;
    const T* F1 = F0 + 3 * w;
    const T* A = recA + ((int64_t)s * L + t) * 2 * w;
    T mu[4], lj[4], En[4], Gn[4], H1[4], E1[4];
    ld4(A + k, mu);
    ld4(A + w + k, lj);
    ld4(F0 + k, En);
    ld4(F0 + 2 * w + k, Gn);
    ld4(F1 + w + k, H1);
    ld4(F1 + k, E1);
    const T hprev = F1[w + k - 1];
    // the source value this step added to E (and folded into G) at the source cell
    const T sv = qs >= 0 ? (T)pulse((double)(src.n0 + t + 1) * src.dt, src.t0, src.tau, src.amp) : T(0);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const T dH = H1[q] - (q ? H1[q - 1] : hprev);
      const T s_q = q == qs ? sv : T(0);
      const T E1p = E1[q] - s_q;  // E'^{n+1} before the source
      if (f64) {
        ds[0][q] -= (double)s_q * (double)lj[q];
        ds[1][q] -= (double)mu[q] * (double)dH;
        ds[2][q] += (double)lj[q] * (double)Gn[q];
        ds[3][q] += (double)lj[q] * (double)En[q];
        ds[4][q] += (double)lj[q] * (double)E1p;
      } else {
        fs[0][q] = fmaf(-(float)s_q, (float)lj[q], fs[0][q]);
        fs[1][q] = fmaf(-(float)mu[q], (float)dH, fs[1][q]);
        fs[2][q] = fmaf((float)lj[q], (float)Gn[q], fs[2][q]);
        fs[3][q] = fmaf((float)lj[q], (float)En[q], fs[3][q]);
        fs[4][q] = fmaf((float)lj[q], (float)E1p, fs[4][q]);
      }
    }
  }
  const int64_t stride = (int64_t)n_slabs * nwin;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    if (c0 + q >= nwin) break;
    const int64_t wi = (int64_t)s * nwin + c0 + q;
#pragma unroll
    for (int m = 0; m < 5; ++m) g[m * stride + wi] += f64 ? ds[m][q] : (double)fs[m][q];
  }
}

// phi1, phi2 and their x-derivatives: Horner sums of the Taylor series below x = 0.5 (degree
// 20, derivative by Horner on k c_k x^(k-1)); expm1 forms above.
__device__ void phis(double x, double& p1, double& p2, double& d1, double& d2) {
  if (x < 0.5) {
    double c1[21], c2[21];
    c1[0] = 1.0;
    c2[0] = 0.5;
    for (int k = 1; k <= 20; ++k) {
      c1[k] = -c1[k - 1] / (double)(k + 1);
      c2[k] = -c2[k - 1] / (double)(k + 2);
    }
    double r1 = c1[20], r2 = c2[20], q1 = 20.0 * c1[20], q2 = 20.0 * c2[20];
    for (int k = 19; k >= 0; --k) {
      r1 = fma(r1, x, c1[k]);
      r2 = fma(r2, x, c2[k]);
      if (k >= 1) {
        q1 = fma(q1, x, (double)k * c1[k]);
        q2 = fma(q2, x, (double)k * c2[k]);
      }
    }
    p1 = r1;
    p2 = r2;
    d1 = q1;
    d2 = q2;
  } else {
    const double em = expm1(-x);
    p1 = -em / x;
    p2 = (x + em) / (x * x);
    d1 = (1.0 + em - p1) / x;  // (a - phi1)/x
    d2 = (p1 - 2.0 * p2) / x;
  }
}

__global__ void k_chain(const double* __restrict__ g, const double* __restrict__ wp2, const double* __restrict__ nu,
                        const int64_t* __restrict__ off, int n_slabs, int64_t w_lo, int w, double dt, double S,
                        double* __restrict__ gw, double* __restrict__ gn) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int s = blockIdx.y;
  if (c >= w || s >= n_slabs) return;
  const int64_t cell = off[s] + w_lo + c;
  const double W = wp2[cell] * dt * dt, x = nu[cell] * dt;
  double p1, p2, d1, d2;
  phis(x, p1, p2, d1, d2);
  const double a = exp(-x);
  const double D = 1.0 + 0.5 * W * p2;
  const double cj = 0.5 * (1.0 + a) / D;
  // derivatives with respect to W (q = 0) and x (q = 1)
  const double dD[2] = {0.5 * p2, 0.5 * W * d2};
  const double dcj[2] = {-cj * dD[0] / D, -0.5 * a / D - cj * dD[1] / D};
  const double dP1[2] = {p1, W * d1};        // d(W phi1)
  const double dP2[2] = {p2, W * d2};        // d(W phi2)
  // The sums are over the folded coefficients: bq = cj bp + da a and cq = cj cc - da (bp, cc
  // as in Eq. 11), so d/d(da) gains a g_bq - g_cq and d/d(dj) gains da g_bq.
  const int64_t wi = (int64_t)s * w + c;
  const int64_t stride = (int64_t)n_slabs * w;
  const double da = -0.5 * W * p1 / D;
  const double g_da = g[wi] + a * g[3 * stride + wi] - g[4 * stride + wi];
  const double g_cb = g[stride + wi];
  const double g_dj = g[2 * stride + wi] + da * g[3 * stride + wi];
  const double g_bp = g[3 * stride + wi];  // coefficient of cj bp
  const double g_cc = g[4 * stride + wi];  // coefficient of cj cc
  double out[2];
  for (int q = 0; q < 2; ++q) {
    const double dda = -0.5 * dP1[q] / D + 0.5 * W * p1 * dD[q] / (D * D);
    const double dcb = -S * dD[q] / (D * D);
    const double ddj = q == 0 ? 0.0 : -a;
    const double dbp = dcj[q] * W * (p1 - p2) + cj * (dP1[q] - dP2[q]);  // d(cj bp)
    const double dcc = dcj[q] * W * p2 + cj * dP2[q];                    // d(cj cc)
    out[q] = g_da * dda + g_cb * dcb + g_dj * ddj + g_bp * dbp + g_cc * dcc;
  }
  gw[cell] = out[0] * dt * dt;  // dW/dwp2 = dt^2
  gn[cell] = out[1] * dt;       // dx/dnu = dt
}

template <typename T>
__global__ void k_rec_init(const T* __restrict__ E, const T* __restrict__ H, const T* __restrict__ J,
                           const int64_t* __restrict__ soff, const int64_t* __restrict__ nz, int n_slabs, int64_t c0,
                           int w, int rec_len, T* __restrict__ rec) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int s = blockIdx.y;
  if (c >= w || s >= n_slabs || c0 + c >= nz[s]) return;
  const int64_t i = soff[s] + c0 + c;
  T* r = rec + (int64_t)s * rec_len * 3 * w;
  r[c] = E[i];
  r[w + c] = H[i];
  r[2 * w + c] = J[i];
}

}  // namespace

template <>
cudaError_t launch_adj<float>(const AdjArgs<float>& a, int K, bool edge, int wpb, cudaStream_t st) {
  if (a.n_tiles <= 0) return cudaSuccess;
  switch (K) {
    case 4: return launch_a<float, 4>(a, edge, wpb, st);
    case 8: return launch_a<float, 8>(a, edge, wpb, st);
    case 16: return launch_a<float, 16>(a, edge, wpb, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_adj_pairs(const AdjArgs<float>& a, int K, int wpb, cudaStream_t st) {
  if (a.n_tiles <= 0) return cudaSuccess;
  const dim3 block(32 * wpb);
  const dim3 grid((a.n_tiles + wpb - 1) / wpb);
  switch (K) {
    case 8: k_adj2<8><<<grid, block, 0, st>>>(a); break;
    case 12: k_adj2<12><<<grid, block, 0, st>>>(a); break;
    case 16: k_adj2<16><<<grid, block, 0, st>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <>
cudaError_t launch_adj<double>(const AdjArgs<double>& a, int K, bool edge, int wpb, cudaStream_t st) {
  if (a.n_tiles <= 0) return cudaSuccess;
  switch (K) {
    case 4: return launch_a<double, 4>(a, edge, wpb, st);
    case 8: return launch_a<double, 8>(a, edge, wpb, st);
    default: return cudaErrorInvalidValue;
  }
}

template <typename T>
cudaError_t launch_seeds(const double* gXr, const double* gXi, const T* tw, int P, int nf, int n, T* seeds,
                         int seed_len, cudaStream_t st) {
  if (P <= 0 || n <= 0) return cudaSuccess;
  k_seeds<T><<<dim3((n + 127) / 128, P), 128, 0, st>>>(gXr, gXi, tw, P, nf, n, seeds, seed_len);
  return cudaGetLastError();
}
template cudaError_t launch_seeds<float>(const double*, const double*, const float*, int, int, int, float*, int,
                                         cudaStream_t);
template cudaError_t launch_seeds<double>(const double*, const double*, const double*, int, int, int, double*, int,
                                          cudaStream_t);

template <typename T>
cudaError_t launch_grad_accum(const T* recF, const T* recA, int n_slabs, int w, int nwin, int L, int recF_len,
                              const GradSource& src, double* g, cudaStream_t st) {
  const int threads = 64;
  const int per = 4 * threads;
  k_grad<T><<<dim3((nwin + per - 1) / per, n_slabs), threads, 0, st>>>(recF, recA, n_slabs, w, nwin, L, recF_len, src,
                                                                        g);
  return cudaGetLastError();
}
template cudaError_t launch_grad_accum<float>(const float*, const float*, int, int, int, int, int, const GradSource&,
                                              double*, cudaStream_t);
template cudaError_t launch_grad_accum<double>(const double*, const double*, int, int, int, int, int,
                                               const GradSource&, double*, cudaStream_t);

cudaError_t launch_grad_chain(const double* g, const double* wp2, const double* nu, const int64_t* off, int n_slabs,
                              int64_t w_lo, int w, double dt, double S, double* gw, double* gn, cudaStream_t st) {
  k_chain<<<dim3((w + 127) / 128, n_slabs), 128, 0, st>>>(g, wp2, nu, off, n_slabs, w_lo, w, dt, S, gw, gn);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_rec_init(const T* E, const T* H, const T* J, const int64_t* soff, const int64_t* nz, int n_slabs,
                            int64_t c0, int w, int rec_len, T* rec, cudaStream_t st) {
  k_rec_init<T><<<dim3((w + 127) / 128, n_slabs), 128, 0, st>>>(E, H, J, soff, nz, n_slabs, c0, w, rec_len, rec);
  return cudaGetLastError();
}
template cudaError_t launch_rec_init<float>(const float*, const float*, const float*, const int64_t*, const int64_t*,
                                            int, int64_t, int, int, float*, cudaStream_t);
template cudaError_t launch_rec_init<double>(const double*, const double*, const double*, const int64_t*,
                                             const int64_t*, int, int64_t, int, int, double*, cudaStream_t);

}  // namespace rketd
