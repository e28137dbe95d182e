// 2D RKETD-FDTD (fields uniform along z; the paper's stated generalisation, Sec. IV.B closing
// remarks and Sec. V), TMz (Ez, Hx, Hy) or TEz (Hz, Ex, Ey), in the normalised variables and with the
// folded current G = cj J~ - da E of the 1D step (rketd_internal.cuh), per-material coefficients.
//
// Arrays are [j][i] (x fastest). Yee positions: TMz Ez (i, j), Hx (i, j+1/2), Hy (i+1/2, j); TEz
// Hz (i+1/2, j+1/2), Ex (i+1/2, j), Ey (i, j+1/2). Every E component of cell (i, j) takes the
// material mat[j][i]. Boundaries: first-order Mur on the E components tangential to the y faces, and
// periodic x or first-order Mur on those tangential to the x faces. A soft line source on row src_j
// adds profile[i] s(t) to Ez (TMz) or Ex (TEz) after the E update (and folds it into G as the 1D step
// does); probes sample that component for the running DFT.
//
// The step is the paper's two-kernel structure (Sec. III): an H kernel, then an E+J kernel with the
// source and the Mur ends, one cell per thread, fields updated in place. Each Mur end cell is set by
// the thread of its interior neighbour (it holds that neighbour's old and new value); a TMz corner by
// the thread that also sets the x-Mur cell next to it.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/rketd.h"
#include "rketd_internal.cuh"
#include "tile_common.cuh"

namespace rketd {
namespace {

constexpr int kMat2 = 16;

template <typename T>
struct Mat2 {
  T cb[kMat2], dj[kMat2], bq[kMat2], cq[kMat2], da[kMat2];
};

template <typename T>
struct Args2 {
  T* F[5];  // TMz: Ez, Gz, Hx, Hy; TEz: Ex, Ey, Gx, Gy, Hz
  const uint8_t* mat;
  const T* profile;  // [nx] source weights
  Mat2<T> m;
  int nx, ny, per, src_j;
  T S, q;
  double t, t0, tau, amp;  // Eq. 15 pulse at t = (n+1) dt, evaluated in FP64 on the source row
};

// ---------------------------------------------------------------- TMz
template <typename T>
__global__ void __launch_bounds__(256) k2_tm_h(Args2<T> a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= a.nx || j >= a.ny) return;
  const int64_t c = (int64_t)j * a.nx + i;
  const T* Ez = a.F[0];
  T* Hx = a.F[2];
  T* Hy = a.F[3];
  const T e = Ez[c];
  if (j + 1 < a.ny) Hx[c] = fma(-a.S, Ez[c + a.nx] - e, Hx[c]);  // dHx/dt = -(1/mu0) dEz/dy
  const int ip = i + 1 < a.nx ? i + 1 : (a.per ? 0 : -1);
  if (ip >= 0) Hy[c] = fma(a.S, Ez[(int64_t)j * a.nx + ip] - e, Hy[c]);  // dHy/dt = (1/mu0) dEz/dx
}

template <typename T>
__global__ void __launch_bounds__(256) k2_tm_e(Args2<T> a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
  const int nx = a.nx, ny = a.ny;
  if (i >= nx || j < 1 || j > ny - 2) return;
  if (!a.per && (i == 0 || i == nx - 1)) return;
  const int64_t c = (int64_t)j * nx + i;
  T* Ez = a.F[0];
  T* G = a.F[1];
  const T* Hx = a.F[2];
  const T* Hy = a.F[3];
  const int im = i > 0 ? i - 1 : nx - 1;
  // eps0 dEz/dt = dHy/dx - dHx/dy - J: E' = E - (cb ((Hx_j - Hx_{j-1}) - (Hy_i - Hy_{i-1})) + G)
  const T curl = (Hx[c] - Hx[c - nx]) - (Hy[c] - Hy[(int64_t)j * nx + im]);
  const int m = a.mat[c];
  const T en = Ez[c];
  T enew = fold_e(en, a.m.cb[m], curl, G[c]);
  T gn = fold_g(G[c], a.m.dj[m], a.m.bq[m], a.m.cq[m], en, enew);
  if (j == a.src_j) {
    const T sv = (T)tile::pulse(a.t, a.t0, a.tau, a.amp) * a.profile[i];
    enew = enew + sv;
    gn = fma(-a.m.da[m], sv, gn);
  }
  G[c] = gn;
  // x-Mur (columns 0 and nx-1, set by columns 1 and nx-2), and the corners next to them
  if (!a.per && (i == 1 || i == nx - 2)) {
    const int ib = i == 1 ? 0 : nx - 1;
    const int64_t cb_ = (int64_t)j * nx + ib;
    const T e0o = Ez[cb_];
    const T ebn = fma(a.q, enew - e0o, en);
    Ez[cb_] = ebn;
    if (j == 1 || j == ny - 2) {  // corner (ib, 0) or (ib, ny-1) from (ib, 1) or (ib, ny-2)
      const int64_t cc = (int64_t)(j == 1 ? 0 : ny - 1) * nx + ib;
      Ez[cc] = fma(a.q, ebn - Ez[cc], e0o);
    }
  }
  // y-Mur (rows 0 and ny-1, set by rows 1 and ny-2)
  if (j == 1 || j == ny - 2) {
    const int64_t cc = (int64_t)(j == 1 ? 0 : ny - 1) * nx + i;
    Ez[cc] = fma(a.q, enew - Ez[cc], en);
  }
  Ez[c] = enew;
}

// ---------------------------------------------------------------- TEz
template <typename T>
__global__ void __launch_bounds__(256) k2_te_h(Args2<T> a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= a.nx || j >= a.ny - 1) return;
  const int ip = i + 1 < a.nx ? i + 1 : (a.per ? 0 : -1);
  if (ip < 0) return;
  const int64_t c = (int64_t)j * a.nx + i;
  const T* Ex = a.F[0];
  const T* Ey = a.F[1];
  T* Hz = a.F[4];
  // dHz/dt = (1/mu0) (dEx/dy - dEy/dx)
  Hz[c] = fma(a.S, (Ex[c + a.nx] - Ex[c]) - (Ey[(int64_t)j * a.nx + ip] - Ey[c]), Hz[c]);
}

template <typename T>
__global__ void __launch_bounds__(256) k2_te_e(Args2<T> a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
  const int nx = a.nx, ny = a.ny;
  if (i >= nx || j >= ny) return;
  const int64_t c = (int64_t)j * nx + i;
  T* Ex = a.F[0];
  T* Ey = a.F[1];
  T* Gx = a.F[2];
  T* Gy = a.F[3];
  const T* Hz = a.F[4];
  const int m = a.mat[c];
  // Ex (i+1/2, j): eps0 dEx/dt = dHz/dy - Jx, rows 1..ny-2 (i + 1/2 inside the grid)
  if (j >= 1 && j <= ny - 2 && (a.per || i <= nx - 2)) {
    const T curl = Hz[c - nx] - Hz[c];
    const T en = Ex[c];
    T enew = fold_e(en, a.m.cb[m], curl, Gx[c]);
    T gn = fold_g(Gx[c], a.m.dj[m], a.m.bq[m], a.m.cq[m], en, enew);
    if (j == a.src_j) {
      const T sv = (T)tile::pulse(a.t, a.t0, a.tau, a.amp) * a.profile[i];
      enew = enew + sv;
      gn = fma(-a.m.da[m], sv, gn);
    }
    Gx[c] = gn;
    if (j == 1 || j == ny - 2) {  // y-Mur on Ex
      const int64_t cc = (int64_t)(j == 1 ? 0 : ny - 1) * nx + i;
      Ex[cc] = fma(a.q, enew - Ex[cc], en);
    }
    Ex[c] = enew;
  }
  // Ey (i, j+1/2): eps0 dEy/dt = -dHz/dx - Jy, rows 0..ny-2
  if (j <= ny - 2 && (a.per || (i >= 1 && i <= nx - 2))) {
    const int im = i > 0 ? i - 1 : nx - 1;
    const T curl = Hz[c] - Hz[(int64_t)j * nx + im];
    const T en = Ey[c];
    const T enew = fold_e(en, a.m.cb[m], curl, Gy[c]);
    Gy[c] = fold_g(Gy[c], a.m.dj[m], a.m.bq[m], a.m.cq[m], en, enew);
    if (!a.per && (i == 1 || i == nx - 2)) {  // x-Mur on Ey
      const int64_t cc = (int64_t)j * nx + (i == 1 ? 0 : nx - 1);
      Ey[cc] = fma(a.q, enew - Ey[cc], en);
    }
    Ey[c] = enew;
  }
}

// ---------------------------------------------------------------- four cells per thread
// FP32 grids with nx a multiple of 4: each thread takes cells 4q .. 4q+3 of one row with 16-byte
// loads and stores (rows then start 16-byte aligned), and the one neighbour across the quad
// (i+1 after it, i-1 before it) with a scalar load. Same operations on the same values as the
// one-cell kernels above; a quad that holds a Mur end cell sets it from its interior neighbour
// in the same thread, and rows 1 and ny-2 set the y-Mur rows 0 and ny-1 (corners included, from
// the new values of the row, x-Mur cells among them).
template <typename T>
__device__ __forceinline__ void ld4(const T* p, T (&v)[4]) {
  if constexpr (sizeof(T) == 4) {
    const float4 q = *reinterpret_cast<const float4*>(p);
    v[0] = q.x;
    v[1] = q.y;
    v[2] = q.z;
    v[3] = q.w;
  } else {
    const double2 a = reinterpret_cast<const double2*>(p)[0], b = reinterpret_cast<const double2*>(p)[1];
    v[0] = a.x;
    v[1] = a.y;
    v[2] = b.x;
    v[3] = b.y;
  }
}

template <typename T>
__device__ __forceinline__ void st4(T* p, const T (&v)[4]) {
  if constexpr (sizeof(T) == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  } else {
    reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
    reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k2v_tm_h(Args2<T> a) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
  const int nx = a.nx, nq = nx >> 2;
  if (q >= nq || j >= a.ny) return;
  const int i0 = 4 * q;
  const int64_t c = (int64_t)j * nx + i0;
  T e[4], hx[4], hy[4];
  ld4(a.F[0] + c, e);
  if (j + 1 < a.ny) {
    T en[4];
    ld4(a.F[0] + c + nx, en);
    ld4(a.F[2] + c, hx);
#pragma unroll
    for (int k = 0; k < 4; ++k) hx[k] = fma(-a.S, en[k] - e[k], hx[k]);
    st4(a.F[2] + c, hx);
  }
  const int ip = i0 + 4 < nx ? i0 + 4 : (a.per ? 0 : -1);
  const T eR = ip >= 0 ? a.F[0][(int64_t)j * nx + ip] : T(0);
  ld4(a.F[3] + c, hy);
#pragma unroll
  for (int k = 0; k < 3; ++k) hy[k] = fma(a.S, e[k + 1] - e[k], hy[k]);
  if (ip >= 0) hy[3] = fma(a.S, eR - e[3], hy[3]);
  st4(a.F[3] + c, hy);
}

template <typename T>
__global__ void __launch_bounds__(256) k2v_tm_e(Args2<T> a) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
  const int nx = a.nx, ny = a.ny, nq = nx >> 2;
  if (q >= nq || j < 1 || j > ny - 2) return;
  const int i0 = 4 * q;
  const int64_t c = (int64_t)j * nx + i0;
  T* Ez = a.F[0];
  T* G = a.F[1];
  T hx[4], hxm[4], hy[4], e[4], g[4], en[4];
  ld4(a.F[2] + c, hx);
  ld4(a.F[2] + c - nx, hxm);
  ld4(a.F[3] + c, hy);
  ld4(Ez + c, e);
  ld4(G + c, g);
  const int im = i0 > 0 ? i0 - 1 : nx - 1;
  const T hyL = a.F[3][(int64_t)j * nx + im];
  const uchar4 mb = *reinterpret_cast<const uchar4*>(a.mat + c);
  const int mm[4] = {mb.x, mb.y, mb.z, mb.w};
  const T sv = j == a.src_j ? (T)tile::pulse(a.t, a.t0, a.tau, a.amp) : T(0);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int i = i0 + k;
    en[k] = e[k];
    if (!a.per && (i == 0 || i == nx - 1)) continue;
    const T curl = (hx[k] - hxm[k]) - (hy[k] - (k ? hy[k - 1] : hyL));
    const int m = mm[k];
    T enew = fold_e(e[k], a.m.cb[m], curl, g[k]);
    T gn = fold_g(g[k], a.m.dj[m], a.m.bq[m], a.m.cq[m], e[k], enew);
    if (j == a.src_j) {
      const T s_i = sv * a.profile[i];
      enew = enew + s_i;
      gn = fma(-a.m.da[m], s_i, gn);
    }
    g[k] = gn;
    en[k] = enew;
  }
  if (!a.per) {  // x-Mur: column 0 from column 1, column nx-1 from column nx-2 (old values in e)
    if (i0 == 0) en[0] = fma(a.q, en[1] - e[0], e[1]);
    if (i0 + 4 == nx) en[3] = fma(a.q, en[2] - e[3], e[2]);
  }
  if (j == 1 || j == ny - 2) {  // y-Mur: row 0 from row 1, row ny-1 from row ny-2
    const int64_t cc = (int64_t)(j == 1 ? 0 : ny - 1) * nx + i0;
    T eb[4];
    ld4(Ez + cc, eb);
#pragma unroll
    for (int k = 0; k < 4; ++k) eb[k] = fma(a.q, en[k] - eb[k], e[k]);
    st4(Ez + cc, eb);
  }
  st4(G + c, g);
  st4(Ez + c, en);
}

template <typename T>
__global__ void __launch_bounds__(256) k2v_te_h(Args2<T> a) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
  const int nx = a.nx, nq = nx >> 2;
  if (q >= nq || j >= a.ny - 1) return;
  const int i0 = 4 * q;
  const int64_t c = (int64_t)j * nx + i0;
  const int ip = i0 + 4 < nx ? i0 + 4 : (a.per ? 0 : -1);
  T ex[4], exn[4], ey[4], hz[4];
  ld4(a.F[0] + c, ex);
  ld4(a.F[0] + c + nx, exn);
  ld4(a.F[1] + c, ey);
  ld4(a.F[4] + c, hz);
  const T eyR = ip >= 0 ? a.F[1][(int64_t)j * nx + ip] : T(0);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    if (k == 3 && ip < 0) break;  // Hz (nx-1/2, j+1/2) is outside a Mur-bounded grid
    const T eyp = k < 3 ? ey[k + 1] : eyR;
    hz[k] = fma(a.S, (exn[k] - ex[k]) - (eyp - ey[k]), hz[k]);
  }
  st4(a.F[4] + c, hz);
}

template <typename T>
__global__ void __launch_bounds__(256) k2v_te_e(Args2<T> a) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
  const int nx = a.nx, ny = a.ny, nq = nx >> 2;
  if (q >= nq || j >= ny) return;
  const int i0 = 4 * q;
  const int64_t c = (int64_t)j * nx + i0;
  T* Ex = a.F[0];
  T* Ey = a.F[1];
  T* Gx = a.F[2];
  T* Gy = a.F[3];
  const T* Hz = a.F[4];
  const uchar4 mb = *reinterpret_cast<const uchar4*>(a.mat + c);
  const int mm[4] = {mb.x, mb.y, mb.z, mb.w};
  T hz[4];
  ld4(Hz + c, hz);
  // Ex (i+1/2, j), rows 1..ny-2: eps0 dEx/dt = dHz/dy - Jx
  if (j >= 1 && j <= ny - 2) {
    T hzm[4], e[4], g[4], en[4];
    ld4(Hz + c - nx, hzm);
    ld4(Ex + c, e);
    ld4(Gx + c, g);
    const T sv = j == a.src_j ? (T)tile::pulse(a.t, a.t0, a.tau, a.amp) : T(0);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int i = i0 + k;
      en[k] = e[k];
      if (!a.per && i == nx - 1) continue;  // no Ex at nx-1/2 on a Mur-bounded grid
      const int m = mm[k];
      T enew = fold_e(e[k], a.m.cb[m], hzm[k] - hz[k], g[k]);
      T gn = fold_g(g[k], a.m.dj[m], a.m.bq[m], a.m.cq[m], e[k], enew);
      if (j == a.src_j) {
        const T s_i = sv * a.profile[i];
        enew = enew + s_i;
        gn = fma(-a.m.da[m], s_i, gn);
      }
      g[k] = gn;
      en[k] = enew;
    }
    if (j == 1 || j == ny - 2) {  // y-Mur on Ex: row 0 from row 1, row ny-1 from row ny-2
      const int64_t cc = (int64_t)(j == 1 ? 0 : ny - 1) * nx + i0;
      T eb[4];
      ld4(Ex + cc, eb);
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if (a.per || i0 + k <= nx - 2) eb[k] = fma(a.q, en[k] - eb[k], e[k]);
      st4(Ex + cc, eb);
    }
    st4(Gx + c, g);
    st4(Ex + c, en);
  }
  // Ey (i, j+1/2), rows 0..ny-2: eps0 dEy/dt = -dHz/dx - Jy
  if (j <= ny - 2) {
    T e[4], g[4], en[4];
    ld4(Ey + c, e);
    ld4(Gy + c, g);
    const int im = i0 > 0 ? i0 - 1 : nx - 1;
    const T hzL = Hz[(int64_t)j * nx + im];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int i = i0 + k;
      en[k] = e[k];
      if (!a.per && (i == 0 || i == nx - 1)) continue;
      const int m = mm[k];
      const T enew = fold_e(e[k], a.m.cb[m], hz[k] - (k ? hz[k - 1] : hzL), g[k]);
      g[k] = fold_g(g[k], a.m.dj[m], a.m.bq[m], a.m.cq[m], e[k], enew);
      en[k] = enew;
    }
    if (!a.per) {  // x-Mur on Ey: column 0 from column 1, column nx-1 from column nx-2
      if (i0 == 0) en[0] = fma(a.q, en[1] - e[0], e[1]);
      if (i0 + 4 == nx) en[3] = fma(a.q, en[2] - e[3], e[2]);
    }
    st4(Gy + c, g);
    st4(Ey + c, en);
  }
}

template <typename T>
__global__ void k2_probe(const T* __restrict__ E, const int32_t* __restrict__ probes, int nx, int n,
                         T* __restrict__ series, int len, int pos) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < n) series[(int64_t)p * len + pos] = E[(int64_t)probes[2 * p + 1] * nx + probes[2 * p]];
}

// SI out: E as is, H = H~/eta0, J = (G + da E)/cj * eps0/dt with the cell's coefficients where the E
// component is advanced by Eq. 12 (comp 0: Ez or Ex, 1: Ey), 0 on the Mur end cells (no current)
template <typename T>
__global__ void k2_out(const T* __restrict__ X, const T* __restrict__ Ecomp, const uint8_t* __restrict__ mat,
                       const double* __restrict__ da, const double* __restrict__ cj, int nx, int ny, int kind, int pol,
                       int per, int comp, double hs, double js, double* __restrict__ out) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= (int64_t)nx * ny) return;
  if (kind == 0) {
    out[c] = (double)X[c];
  } else if (kind == 1) {
    out[c] = (double)X[c] * hs;
  } else {
    const int i = (int)(c % nx), j = (int)(c / nx);
    bool upd;
    if (comp == 1) upd = j <= ny - 2 && (per || (i >= 1 && i <= nx - 2));             // TEz Ey
    else if (pol == 1) upd = j >= 1 && j <= ny - 2 && (per || i <= nx - 2);           // TEz Ex
    else upd = j >= 1 && j <= ny - 2 && (per || (i >= 1 && i <= nx - 2));            // TMz Ez
    out[c] = upd ? ((double)X[c] + da[mat[c]] * (double)Ecomp[c]) / cj[mat[c]] * js : 0.0;
  }
}

// phi1, phi2 and psi = phi1 - (1 + e^{-x}) phi2 = (phi1 - 2 phi2) + x phi1 phi2 in FP64 (Taylor series
// below x = 0.5, summed from the smallest term; expm1 above).
void host_phi(double x, double& p1, double& p2, double& psi) {
  if (x < 0.5) {
    double t1 = 1.0, t2 = 0.5, t3 = -1.0 / 6.0;  // k-th terms of phi1, phi2, (phi1 - 2 phi2)/x
    double a1[24], a2[24], a3[24];
    for (int k = 0; k < 24; ++k) {
      a1[k] = t1;
      a2[k] = t2;
      a3[k] = t3;
      t1 *= -x / (k + 2);
      t2 *= -x / (k + 3);
      t3 *= -x * (k + 2) / ((double)(k + 1) * (k + 4));
    }
    double s1 = 0, s2 = 0, s3 = 0;
    for (int k = 23; k >= 0; --k) {
      s1 += a1[k];
      s2 += a2[k];
      s3 += a3[k];
    }
    p1 = s1;
    p2 = s2;
    psi = x * (s3 + s1 * s2);
  } else {
    const double em = std::expm1(-x);
    p1 = -em / x;
    p2 = (x + em) / (x * x);
    psi = p1 - (2.0 + em) * p2;
  }
}

}  // namespace
}  // namespace rketd

using namespace rketd;

struct rketd_ctx2d {
  rketd_grid2d g{};
  size_t esz = 4;
  int64_t N = 0;
  double S = 0, q = 0;
  cudaStream_t stream = nullptr;
  rketd_pulse pulse{};
  int n_mat = 0;
  double da[kMat2] = {}, cb[kMat2] = {}, cj[kMat2] = {}, dj[kMat2] = {}, bq[kMat2] = {}, cq[kMat2] = {};
  void* F[5] = {};
  uint8_t* mat = nullptr;
  void* profile = nullptr;
  double* da_d = nullptr;
  double* cj_d = nullptr;
  int n_probes = 0, n_freq = 0, B = 512;
  int32_t* probes_d = nullptr;
  double* freq_d = nullptr;
  void* series = nullptr;
  void* tw = nullptr;
  double* rot = nullptr;
  double *Xr = nullptr, *Xi = nullptr, *Xtmp = nullptr;
  int64_t step = 0, launches = 0;
  std::vector<void*> allocs;
  ~rketd_ctx2d() {
    for (void* p : allocs) cudaFree(p);
  }
  bool alloc(void** p, size_t bytes) {
    *p = nullptr;
    if (device_alloc(p, bytes ? bytes : 16) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    allocs.push_back(*p);
    return true;
  }
};

namespace {

rketd_status bad2(rketd_status st, const std::string& msg) {
  set_error_message(msg.c_str());
  return st;
}

template <typename T>
Args2<T> args2(rketd_ctx2d* c) {
  Args2<T> a{};
  for (int q = 0; q < 5; ++q) a.F[q] = (T*)c->F[q];
  a.mat = c->mat;
  a.profile = (const T*)c->profile;
  for (int m = 0; m < kMat2; ++m) {
    a.m.cb[m] = (T)c->cb[m];
    a.m.dj[m] = (T)c->dj[m];
    a.m.bq[m] = (T)c->bq[m];
    a.m.cq[m] = (T)c->cq[m];
    a.m.da[m] = (T)c->da[m];
  }
  a.nx = c->g.nx;
  a.ny = c->g.ny;
  a.per = c->g.periodic_x;
  a.src_j = c->g.src_j;
  a.S = (T)c->S;
  a.q = (T)c->q;
  return a;
}

template <typename T>
rketd_status fold2(rketd_ctx2d* c, int n, int64_t m0, double* Xr, double* Xi) {
  if (!c->n_probes || !n) return RKETD_OK;
  cudaError_t e = launch_dft_rotation(c->freq_d, c->n_freq, c->g.dt, m0, c->rot, c->stream);
  if (e == cudaSuccess)
    e = launch_dft<T>((const T*)c->series, c->B, n, (const T*)c->tw, c->n_probes, c->n_freq, Xr, Xi, c->stream,
                      c->rot);
  c->launches += 2;
  return e == cudaSuccess ? RKETD_OK : bad2(RKETD_ECUDA, std::string("2D DFT: ") + cudaGetErrorString(e));
}

template <typename T>
rketd_status step2(rketd_ctx2d* c, int64_t nsteps) {
  const dim3 block(32, 8);
  const dim3 grid((c->g.nx + 31) / 32, (c->g.ny + 7) / 8);
  // four FP32 cells per thread where every row starts 16-byte aligned (the FP64 step is bound by
  // the FP64 pipe, and runs faster one cell per thread)
  const bool quad = c->g.nx % 4 == 0 && c->esz == 4;
  const dim3 gridq((c->g.nx / 4 + 31) / 32, (c->g.ny + 7) / 8);
  Args2<T> a = args2<T>(c);
  a.t0 = c->pulse.t0;
  a.tau = c->pulse.tau;
  a.amp = c->pulse.amp;
  for (int64_t s = 0; s < nsteps; ++s) {
    a.t = (double)(c->step + 1) * c->g.dt;
    if (c->g.pol == RKETD_TMZ) {
      if (quad) {
        k2v_tm_h<T><<<gridq, block, 0, c->stream>>>(a);
        k2v_tm_e<T><<<gridq, block, 0, c->stream>>>(a);
      } else {
        k2_tm_h<T><<<grid, block, 0, c->stream>>>(a);
        k2_tm_e<T><<<grid, block, 0, c->stream>>>(a);
      }
    } else {
      if (quad) {
        k2v_te_h<T><<<gridq, block, 0, c->stream>>>(a);
        k2v_te_e<T><<<gridq, block, 0, c->stream>>>(a);
      } else {
        k2_te_h<T><<<grid, block, 0, c->stream>>>(a);
        k2_te_e<T><<<grid, block, 0, c->stream>>>(a);
      }
    }
    c->launches += 2;
    const int pos = (int)(c->step % c->B);
    if (c->n_probes) {
      k2_probe<T><<<(c->n_probes + 127) / 128, 128, 0, c->stream>>>((const T*)c->F[0], c->probes_d, c->g.nx,
                                                                   c->n_probes, (T*)c->series, c->B, pos);
      c->launches += 1;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return bad2(RKETD_ECUDA, std::string("2D step: ") + cudaGetErrorString(e));
    c->step += 1;
    if (c->step % c->B == 0) {
      rketd_status st = fold2<T>(c, c->B, c->step - c->B + 1, c->Xr, c->Xi);
      if (st) return st;
    }
  }
  return RKETD_OK;
}

rketd_status zero2(rketd_ctx2d* c) {
  const int nf = c->g.pol == RKETD_TMZ ? 4 : 5;
  for (int q = 0; q < nf; ++q)
    if (cudaMemsetAsync(c->F[q], 0, c->esz * c->N, c->stream) != cudaSuccess) return bad2(RKETD_ECUDA, "2D memset");
  if (c->n_probes) {
    const size_t xb = sizeof(double) * c->n_probes * c->n_freq;
    if (cudaMemsetAsync(c->Xr, 0, xb, c->stream) != cudaSuccess || cudaMemsetAsync(c->Xi, 0, xb, c->stream) != cudaSuccess)
      return bad2(RKETD_ECUDA, "2D memset");
  }
  c->step = 0;
  return RKETD_OK;
}

}  // namespace

extern "C" {

rketd_status rketd_create_2d(const rketd_grid2d* g, const uint8_t* mat, int32_t n_mat, const double* mat_wp2,
                             const double* mat_nu, const double* profile, const rketd_pulse* pulse, int32_t n_probes,
                             const int32_t* probes, const rketd_dft* dft, void* stream, rketd_ctx2d** out) {
  set_error_message("");
  if (!out) return bad2(RKETD_EINVAL, "out is NULL");
  *out = nullptr;
  if (!g || !mat || !mat_wp2 || !mat_nu || !profile || !pulse) return bad2(RKETD_EINVAL, "NULL argument");
  if (g->nx < 4 || g->ny < 4) return bad2(RKETD_EINVAL, "2D grid needs nx, ny >= 4");
  if (g->prec != RKETD_F32 && g->prec != RKETD_F64) return bad2(RKETD_EINVAL, "prec must be F32 or F64");
  if (g->pol != RKETD_TMZ && g->pol != RKETD_TEZ) return bad2(RKETD_EINVAL, "pol must be TMZ or TEZ");
  if (!(g->d > 0) || !(g->dt > 0) || !std::isfinite(g->d) || !std::isfinite(g->dt))
    return bad2(RKETD_EINVAL, "d and dt must be finite and > 0");
  const double S = g->dt / (g->d * std::sqrt(kMu0 * kEps0));
  if (!(S <= 1.0 / std::sqrt(2.0))) return bad2(RKETD_ECOURANT, "2D Courant number c dt/d exceeds 1/sqrt(2)");
  if (g->src_j < 1 || g->src_j > g->ny - 2) return bad2(RKETD_EINVAL, "source row outside 1..ny-2");
  if (n_mat < 1 || n_mat > kMat2) return bad2(RKETD_EINVAL, "n_mat must be 1..16");
  if (mat_wp2[0] != 0.0) return bad2(RKETD_EINVAL, "material 0 must be vacuum");
  for (int m = 0; m < n_mat; ++m)
    if (!(mat_wp2[m] >= 0) || !(mat_nu[m] >= 0) || !std::isfinite(mat_wp2[m]) || !std::isfinite(mat_nu[m]))
      return bad2(RKETD_EINVAL, "material parameters must be finite and >= 0");
  if (!(pulse->tau > 0) || !std::isfinite(pulse->t0) || !std::isfinite(pulse->amp))
    return bad2(RKETD_EINVAL, "pulse tau must be > 0, t0 and amp finite");
  const int64_t N = (int64_t)g->nx * g->ny;
  for (int64_t c2 = 0; c2 < N; ++c2)
    if (mat[c2] >= n_mat) return bad2(RKETD_EINVAL, "material index out of range");
  for (int i = 0; i < g->nx; ++i)
    if (!std::isfinite(profile[i])) return bad2(RKETD_EINVAL, "source profile must be finite");
  const int nf = (n_probes > 0 && dft) ? dft->n_freq : 0;
  if (n_probes < 0 || (n_probes > 0 && (!probes || !dft || nf < 1 || !dft->freq_hz)))
    return bad2(RKETD_EINVAL, "probes need n_freq >= 1, freq_hz and cells");
  for (int p = 0; p < n_probes; ++p)
    if (probes[2 * p] < 0 || probes[2 * p] >= g->nx || probes[2 * p + 1] < 0 || probes[2 * p + 1] >= g->ny)
      return bad2(RKETD_EINVAL, "probe outside the grid");
  rketd_ctx2d* c = new (std::nothrow) rketd_ctx2d();
  if (!c) return bad2(RKETD_ENOMEM, "host allocation");
  auto fail = [&](rketd_status st, const char* msg) {
    delete c;
    return bad2(st, msg);
  };
  c->g = *g;
  c->esz = g->prec == RKETD_F64 ? 8 : 4;
  c->N = N;
  c->S = S;
  c->q = (S - 1.0) / (S + 1.0);
  c->stream = (cudaStream_t)stream;
  c->pulse = *pulse;
  c->n_mat = n_mat;
  c->n_probes = n_probes;
  c->n_freq = nf;
  // per-material coefficients of the folded update (rketd_internal.cuh), FP64 on the host
  for (int m = 0; m < kMat2; ++m) {
    const double w = m < n_mat ? mat_wp2[m] * g->dt * g->dt : 0.0;
    const double x = m < n_mat ? mat_nu[m] * g->dt : 0.0;
    double p1, p2, psi;
    host_phi(x, p1, p2, psi);
    const double em = std::expm1(-x);
    const double D = 1.0 + 0.5 * w * p2;
    const double h = 0.5 * w / D;
    c->da[m] = -h * p1;
    c->cb[m] = S / D;
    c->cj[m] = 0.5 * (2.0 + em) / D;
    c->dj[m] = em;
    c->bq[m] = h * psi;
    c->cq[m] = h * (p1 + (2.0 + em) * p2);
  }
  const int nfields = g->pol == RKETD_TMZ ? 4 : 5;
  for (int q = 0; q < nfields; ++q)
    if (!c->alloc(&c->F[q], c->esz * N)) return fail(RKETD_ENOMEM, "2D fields");
  void* p;
  if (!c->alloc(&p, N)) return fail(RKETD_ENOMEM, "2D materials");
  c->mat = (uint8_t*)p;
  if (!c->alloc(&c->profile, c->esz * g->nx)) return fail(RKETD_ENOMEM, "2D profile");
  if (!c->alloc(&p, sizeof(double) * kMat2)) return fail(RKETD_ENOMEM, "2D table");
  c->da_d = (double*)p;
  if (!c->alloc(&p, sizeof(double) * kMat2)) return fail(RKETD_ENOMEM, "2D table");
  c->cj_d = (double*)p;
  std::vector<char> prof(c->esz * g->nx);
  for (int i = 0; i < g->nx; ++i) {
    if (c->esz == 8) ((double*)prof.data())[i] = profile[i];
    else ((float*)prof.data())[i] = (float)profile[i];
  }
  if (cudaMemcpy(c->mat, mat, N, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(c->profile, prof.data(), prof.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(c->da_d, c->da, sizeof(double) * kMat2, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(c->cj_d, c->cj, sizeof(double) * kMat2, cudaMemcpyHostToDevice) != cudaSuccess)
    return fail(RKETD_ECUDA, "2D upload");
  if (n_probes) {
    const int P = n_probes, B = c->B;
    if (!c->alloc(&p, sizeof(int32_t) * 2 * P)) return fail(RKETD_ENOMEM, "2D probes");
    c->probes_d = (int32_t*)p;
    if (!c->alloc(&p, sizeof(double) * nf)) return fail(RKETD_ENOMEM, "2D frequencies");
    c->freq_d = (double*)p;
    if (!c->alloc(&c->series, c->esz * (size_t)P * B) || !c->alloc(&c->tw, c->esz * 2 * (size_t)B * nf))
      return fail(RKETD_ENOMEM, "2D DFT buffers");
    if (!c->alloc(&p, sizeof(double) * 2 * nf)) return fail(RKETD_ENOMEM, "2D DFT rotation");
    c->rot = (double*)p;
    for (double** x : {&c->Xr, &c->Xi}) {
      if (!c->alloc(&p, sizeof(double) * (size_t)P * nf)) return fail(RKETD_ENOMEM, "2D spectra");
      *x = (double*)p;
    }
    if (!c->alloc(&p, sizeof(double) * 2 * (size_t)P * nf)) return fail(RKETD_ENOMEM, "2D spectra");
    c->Xtmp = (double*)p;
    if (cudaMemcpy(c->probes_d, probes, sizeof(int32_t) * 2 * P, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(c->freq_d, dft->freq_hz, sizeof(double) * nf, cudaMemcpyHostToDevice) != cudaSuccess)
      return fail(RKETD_ECUDA, "2D probe upload");
    cudaError_t e = c->esz == 8 ? launch_twiddles<double>(c->freq_d, nf, g->dt, 0, B, (double*)c->tw, c->stream)
                                : launch_twiddles<float>(c->freq_d, nf, g->dt, 0, B, (float*)c->tw, c->stream);
    if (e != cudaSuccess) return fail(RKETD_ECUDA, "2D twiddles");
    c->launches += 1;
  }
  rketd_status st = zero2(c);
  if (st) {
    delete c;
    return st;
  }
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return fail(RKETD_ECUDA, "2D create");
  *out = c;
  return RKETD_OK;
}

rketd_status rketd_reset_2d(rketd_ctx2d* c) {
  if (!c) return bad2(RKETD_EINVAL, "NULL context");
  return zero2(c);
}

rketd_status rketd_step_2d(rketd_ctx2d* c, int64_t nsteps) {
  if (!c) return bad2(RKETD_EINVAL, "NULL context");
  if (nsteps < 0) return bad2(RKETD_EINVAL, "nsteps < 0");
  return c->esz == 8 ? step2<double>(c, nsteps) : step2<float>(c, nsteps);
}

rketd_status rketd_sync_2d(rketd_ctx2d* c) {
  if (!c) return bad2(RKETD_EINVAL, "NULL context");
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e == cudaSuccess) e = cudaGetLastError();
  return e == cudaSuccess ? RKETD_OK : bad2(RKETD_ECUDA, cudaGetErrorString(e));
}

rketd_status rketd_get_field_2d(rketd_ctx2d* c, int32_t which, double* out) {
  if (!c || !out) return bad2(RKETD_EINVAL, "NULL argument");
  const bool tm = c->g.pol == RKETD_TMZ;
  // TMz: 0 Ez, 1 Hx, 2 Hy, 3 Jz; TEz: 0 Ex, 1 Ey, 2 Hz, 3 Jx, 4 Jy
  if (which < 0 || which >= (tm ? 4 : 5)) return bad2(RKETD_EINVAL, "field index out of range");
  int src, kind, ecomp = 0;
  if (tm) {
    const int map_src[4] = {0, 2, 3, 1}, map_kind[4] = {0, 1, 1, 2};
    src = map_src[which];
    kind = map_kind[which];
  } else {
    const int map_src[5] = {0, 1, 4, 2, 3}, map_kind[5] = {0, 0, 1, 2, 2};
    src = map_src[which];
    kind = map_kind[which];
    ecomp = which == 4 ? 1 : 0;
  }
  double* tmp = nullptr;
  cudaError_t e = device_alloc_async((void**)&tmp, sizeof(double) * c->N, c->stream);
  if (e != cudaSuccess) return bad2(RKETD_ENOMEM, "2D field staging");
  const unsigned blocks = (unsigned)((c->N + 255) / 256);
  const double hs = 1.0 / std::sqrt(kMu0 / kEps0), js = kEps0 / c->g.dt;
  const int nx = c->g.nx, ny = c->g.ny, pol = c->g.pol, per = c->g.periodic_x;
  if (c->esz == 8)
    k2_out<double><<<blocks, 256, 0, c->stream>>>((const double*)c->F[src], (const double*)c->F[ecomp], c->mat,
                                                  c->da_d, c->cj_d, nx, ny, kind, pol, per, ecomp, hs, js, tmp);
  else
    k2_out<float><<<blocks, 256, 0, c->stream>>>((const float*)c->F[src], (const float*)c->F[ecomp], c->mat, c->da_d,
                                                 c->cj_d, nx, ny, kind, pol, per, ecomp, hs, js, tmp);
  c->launches += 1;
  e = cudaMemcpyAsync(out, tmp, sizeof(double) * c->N, cudaMemcpyDeviceToHost, c->stream);
  cudaFreeAsync(tmp, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  return e == cudaSuccess ? RKETD_OK : bad2(RKETD_ECUDA, cudaGetErrorString(e));
}

rketd_status rketd_get_spectra_2d(rketd_ctx2d* c, double* re, double* im) {
  if (!c || !re || !im) return bad2(RKETD_EINVAL, "NULL argument");
  const size_t n = (size_t)c->n_probes * c->n_freq;
  if (!n) return RKETD_OK;
  if (cudaMemcpyAsync(c->Xtmp, c->Xr, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess ||
      cudaMemcpyAsync(c->Xtmp + n, c->Xi, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess)
    return bad2(RKETD_ECUDA, "2D spectra copy");
  const int pending = (int)(c->step % c->B);
  if (pending) {
    rketd_status st = c->esz == 8 ? fold2<double>(c, pending, c->step - pending + 1, c->Xtmp, c->Xtmp + n)
                                  : fold2<float>(c, pending, c->step - pending + 1, c->Xtmp, c->Xtmp + n);
    if (st) return st;
  }
  if (cudaMemcpyAsync(re, c->Xtmp, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
      cudaMemcpyAsync(im, c->Xtmp + n, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess)
    return bad2(RKETD_ECUDA, "2D spectra D2H");
  return RKETD_OK;
}

int64_t rketd_launch_count_2d(const rketd_ctx2d* c) { return c ? c->launches : -1; }

rketd_status rketd_check_finite_2d(rketd_ctx2d* c) {
  if (!c) return bad2(RKETD_EINVAL, "NULL context");
  int* flag = nullptr;
  if (device_alloc_async((void**)&flag, sizeof(int), c->stream) != cudaSuccess)
    return bad2(RKETD_ENOMEM, "finite scan");
  cudaError_t e = cudaMemsetAsync(flag, 0, sizeof(int), c->stream);
  const int nf = c->g.pol == RKETD_TMZ ? 4 : 5;
  for (int q = 0; q < nf && e == cudaSuccess; ++q) e = launch_finite_scan(c->esz == 8, c->F[q], c->N, flag, c->stream);
  const int64_t nx = (int64_t)c->n_probes * c->n_freq;
  if (e == cudaSuccess && nx) e = launch_finite_scan(true, c->Xr, nx, flag, c->stream);
  if (e == cudaSuccess && nx) e = launch_finite_scan(true, c->Xi, nx, flag, c->stream);
  int h = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
  cudaFreeAsync(flag, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return bad2(RKETD_ECUDA, std::string("finite scan: ") + cudaGetErrorString(e));
  if (h) return bad2(RKETD_ENUMERIC, "a field or spectrum holds NaN or Inf");
  return RKETD_OK;
}

rketd_status rketd_destroy_2d(rketd_ctx2d* c) {
  delete c;
  return RKETD_OK;
}

}  // extern "C"
