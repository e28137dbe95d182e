// 3D Yee RKETD-FDTD step (the paper's stated 2D/3D generalisation, Sec. IV.B and Sec. V):
// the three-component form of the 1D update, in the same normalised variables
// (E~ = E, H~ = eta0 H, carried current cj (dt/eps0) J) and with the same per-material
// coefficients (rketd_internal.cuh), plus CPML on every face backed by PEC walls (or
// periodic x and y), a total-field/scattered-field box fed by a 1D line, a soft sheet
// source and a running DFT of Ex at probe points.
//
// Streaming form: one H kernel and one E+J kernel per step. A thread owns an (i, j) column
// and marches along k, so the z-neighbours of each update stay in registers; x- and
// y-neighbours come from neighbouring threads through L1/L2. Arrays are [k][j][i].
// Yee positions: Ex (i+1/2, j, k), Ey (i, j+1/2, k), Ez (i, j, k+1/2),
//                Hx (i, j+1/2, k+1/2), Hy (i+1/2, j, k+1/2), Hz (i+1/2, j+1/2, k).
// Each E component takes the material at its own position: mat[c] packs the material
// indices of Ex, Ey, Ez of cell c in bits 0-1, 2-3, 4-5 (0 = vacuum).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/rketd.h"
#include "rketd_internal.cuh"

namespace rketd {
namespace {

constexpr int kMat = 4;
// derivative axis of each CPML memory (order Ex/y, Ex/z, Ey/z, Ey/x, Ez/x, Ez/y, Hx/y, Hx/z,
// Hy/z, Hy/x, Hz/x, Hz/y)
constexpr int kPsiAxis[12] = {1, 2, 2, 0, 0, 1, 1, 2, 2, 0, 0, 1};

template <typename T>
struct Mat3 {
  T da[kMat], cb[kMat], dj[kMat], bp[kMat], cc[kMat];
};

template <typename T>
struct Args3 {
  T *Ex, *Ey, *Ez, *Hx, *Hy, *Hz, *Jx, *Jy, *Jz;
  const uint8_t* mat;
  Mat3<T> m;
  int nx, ny, nz, per;
  T S, q;
  // CPML: tables [axis][E/H][b, c, kinv, flag][nmax]; memories in compact zones of width Z
  const T* tab;
  int nmax, np, Z;
  T* psi[12];  // Ex/y, Ex/z, Ey/z, Ey/x, Ez/x, Ez/y, Hx/y, Hx/z, Hy/z, Hy/x, Hz/x, Hz/y
  // TF/SF
  int tfsf, i0, i1, j0, j1, k0, k1;
  T* Ei;
  T* Hi;
  int inc_len, inc_off, inc_src;
  // sources and probes
  int sheet_k;
  double dt, tau, t0, amp;
  int64_t n0;
  const int* probes;  // [P][3]
  int n_probes;
  T* series;
  int series_len, series_pos;
};

__device__ __forceinline__ int64_t idx3(int i, int j, int k, int nx, int ny) {
  return ((int64_t)k * ny + j) * nx + i;
}

// compact CPML zone index of node n on an axis of N nodes (np layers): -1 outside
__device__ __forceinline__ int zone(int n, int N, int np) {
  if (np <= 0) return -1;
  if (n < np + 1) return n;
  if (n >= N - np - 1) return np + 1 + (n - (N - np - 1));
  return -1;
}

template <typename T>
__device__ __forceinline__ const T* tb(const Args3<T>& a, int ax, int h) {
  return a.tab + (int64_t)(ax * 2 + h) * 4 * a.nmax;
}

__device__ __forceinline__ double pulse3(double t, double t0, double tau, double amp) {
  const double u = (t - t0) / tau;
  return amp * u * exp(-0.5 * u * u);
}

// Stretched difference with CPML memory: psi = b psi + c dv; returns dv kinv + psi.
template <typename T>
__device__ __forceinline__ T stretch(const T* t, int nmax, int pos, T dv, T* psi) {
  if (t[3 * nmax + pos] == T(0)) return dv;
  const T p = fma(t[pos], *psi, t[nmax + pos] * dv);
  *psi = p;
  return fma(dv, t[2 * nmax + pos], p);
}

template <typename T>
__global__ void __launch_bounds__(256) k3_h(const Args3<T> a) {
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  if (blockIdx.z == 1) {  // the 1D incident line: H~ -= S (E_{m+1} - E_m)
    if (blockIdx.x != 0 || blockIdx.y != 0 || !a.tfsf) return;
    for (int m = threadIdx.y * blockDim.x + threadIdx.x; m < a.inc_len - 1; m += blockDim.x * blockDim.y)
      a.Hi[m] = fma(-a.S, a.Ei[m + 1] - a.Ei[m], a.Hi[m]);
    return;
  }
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= nx || j >= ny) return;
  const int ip = (i + 1 < nx) ? i + 1 : (a.per ? 0 : -1);
  const int jp = (j + 1 < ny) ? j + 1 : (a.per ? 0 : -1);
  const int64_t nxy = (int64_t)nx * ny;
  const T S = a.S;
  const T* tx = tb(a, 0, 1);
  const T* ty = tb(a, 1, 1);
  const T* tz = tb(a, 2, 1);
  const int zx = zone(i, nx, a.per ? 0 : a.np), zy = zone(j, ny, a.per ? 0 : a.np);
  const bool in_i = a.tfsf && i >= a.i0 && i <= a.i1 - 1;
  T ex = a.Ex[idx3(i, j, 0, nx, ny)], ey = a.Ey[idx3(i, j, 0, nx, ny)];
  for (int k = 0; k < nz; ++k) {
    const int64_t c = idx3(i, j, k, nx, ny);
    const bool kn = k + 1 < nz;
    const T exn = kn ? a.Ex[c + nxy] : T(0);
    const T eyn = kn ? a.Ey[c + nxy] : T(0);
    const T ez = a.Ez[c];
    const int zz = zone(k, nz, a.np);
    if (jp >= 0 && kn) {  // Hx
      T cy = a.Ez[idx3(i, jp, k, nx, ny)] - ez;
      T cz = eyn - ey;
      if (zy >= 0) cy = stretch(ty, a.nmax, j, cy, &a.psi[6][((int64_t)k * a.Z + zy) * nx + i]);
      if (zz >= 0) cz = stretch(tz, a.nmax, k, cz, &a.psi[7][((int64_t)zz * ny + j) * nx + i]);
      a.Hx[c] = fma(-S, cy - cz, a.Hx[c]);
    }
    if (ip >= 0 && kn) {  // Hy
      T cz = exn - ex;
      T cx = a.Ez[idx3(ip, j, k, nx, ny)] - ez;
      if (zz >= 0) cz = stretch(tz, a.nmax, k, cz, &a.psi[8][((int64_t)zz * ny + j) * nx + i]);
      if (zx >= 0) cx = stretch(tx, a.nmax, i, cx, &a.psi[9][((int64_t)k * ny + j) * a.Z + zx]);
      T h = fma(-S, cz - cx, a.Hy[c]);
      if (in_i && j >= a.j0 && j <= a.j1) {
        if (k == a.k0 - 1) h = fma(S, a.Ei[a.k0 + a.inc_off], h);
        if (k == a.k1) h = fma(-S, a.Ei[a.k1 + a.inc_off], h);
      }
      a.Hy[c] = h;
    }
    if (ip >= 0 && jp >= 0) {  // Hz
      T cx = a.Ey[idx3(ip, j, k, nx, ny)] - ey;
      T cy = a.Ex[idx3(i, jp, k, nx, ny)] - ex;
      if (zx >= 0) cx = stretch(tx, a.nmax, i, cx, &a.psi[10][((int64_t)k * ny + j) * a.Z + zx]);
      if (zy >= 0) cy = stretch(ty, a.nmax, j, cy, &a.psi[11][((int64_t)k * a.Z + zy) * nx + i]);
      T h = fma(-S, cx - cy, a.Hz[c]);
      if (in_i && k >= a.k0 && k <= a.k1) {
        if (j == a.j0 - 1) h = fma(-S, a.Ei[k + a.inc_off], h);
        if (j == a.j1) h = fma(S, a.Ei[k + a.inc_off], h);
      }
      a.Hz[c] = h;
    }
    ex = exn;
    ey = eyn;
  }
}

// E' = E + da E + cb curl - Jc,  Jc' = Jc + dj Jc + bp E + cc E'  (material m of the component)
template <typename T>
__device__ __forceinline__ T e_update(const Mat3<T>& M, int m, T e, T curl, T* J) {
  if (m == 0) return fma(M.cb[0], curl, e);
  const T jc = *J;
  T en = fma(M.da[m], e, e);
  en = fma(M.cb[m], curl, en);
  en = en - jc;
  T jn = fma(M.dj[m], jc, jc);
  jn = fma(M.bp[m], e, jn);
  jn = fma(M.cc[m], en, jn);
  *J = jn;
  return en;
}

template <typename T>
__global__ void __launch_bounds__(256) k3_e(const Args3<T> a) {
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const double t = (double)(a.n0 + 1) * a.dt;
  if (blockIdx.z == 1) {  // 1D incident line: E update, soft source, first-order Mur ends
    if (blockIdx.x != 0 || blockIdx.y != 0 || !a.tfsf) return;
    __shared__ T ends[4];
    const int tid = threadIdx.y * blockDim.x + threadIdx.x, nt = blockDim.x * blockDim.y, L = a.inc_len;
    if (tid == 0) {
      ends[0] = a.Ei[0];
      ends[1] = a.Ei[1];
      ends[2] = a.Ei[L - 2];
      ends[3] = a.Ei[L - 1];
    }
    __syncthreads();
    for (int m = 1 + tid; m < L - 1; m += nt) a.Ei[m] = fma(-a.S, a.Hi[m] - a.Hi[m - 1], a.Ei[m]);
    __syncthreads();
    if (tid == 0) {
      a.Ei[a.inc_src] = a.Ei[a.inc_src] + (T)pulse3(t, a.t0, a.tau, a.amp);
      a.Ei[0] = fma(a.q, a.Ei[1] - ends[0], ends[1]);
      a.Ei[L - 1] = fma(a.q, a.Ei[L - 2] - ends[3], ends[2]);
    }
    return;
  }
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= nx || j >= ny) return;
  const int im = (i > 0) ? i - 1 : (a.per ? nx - 1 : -1);
  const int jm = (j > 0) ? j - 1 : (a.per ? ny - 1 : -1);
  const bool xin = a.per || (i > 0 && i < nx - 1);
  const bool yin = a.per || (j > 0 && j < ny - 1);
  const bool ex_x = a.per || i < nx - 1;
  const bool ey_y = a.per || j < ny - 1;
  const T* tx = tb(a, 0, 0);
  const T* ty = tb(a, 1, 0);
  const T* tz = tb(a, 2, 0);
  const int zx = zone(i, nx, a.per ? 0 : a.np), zy = zone(j, ny, a.per ? 0 : a.np);
  const bool tf_ex = a.tfsf && i >= a.i0 && i <= a.i1 - 1 && j >= a.j0 && j <= a.j1;
  const bool tf_ez = a.tfsf && j >= a.j0 && j <= a.j1 && (i == a.i0 || i == a.i1);
  const T srcv = (T)pulse3(t, a.t0, a.tau, a.amp);
  // probes in this column
  int pk[4], ps[4], npc = 0;
  for (int p = 0; p < a.n_probes && npc < 4; ++p)
    if (a.probes[3 * p] == i && a.probes[3 * p + 1] == j) {
      pk[npc] = a.probes[3 * p + 2];
      ps[npc] = p;
      ++npc;
    }
  T hx_km = T(0), hy_km = T(0);
  for (int k = 0; k < nz; ++k) {
    const int64_t c = idx3(i, j, k, nx, ny);
    const bool zin = k > 0 && k < nz - 1;
    const T hx = a.Hx[c], hy = a.Hy[c], hz = a.Hz[c];
    const int mb = a.mat[c];
    const int zz = zone(k, nz, a.np);
    T ex_out = T(0);
    bool ex_written = false;
    if (ex_x && yin && zin) {  // Ex
      T cy = hz - a.Hz[idx3(i, jm, k, nx, ny)];
      T cz = hy - hy_km;
      if (zy >= 0) cy = stretch(ty, a.nmax, j, cy, &a.psi[0][((int64_t)k * a.Z + zy) * nx + i]);
      if (zz >= 0) cz = stretch(tz, a.nmax, k, cz, &a.psi[1][((int64_t)zz * ny + j) * nx + i]);
      T e = e_update(a.m, mb & 3, a.Ex[c], cy - cz, &a.Jx[c]);
      if (tf_ex) {
        if (k == a.k0) e = fma(a.S, a.Hi[a.k0 - 1 + a.inc_off], e);
        if (k == a.k1) e = fma(-a.S, a.Hi[a.k1 + a.inc_off], e);
      }
      if (k == a.sheet_k) e = e + srcv;
      a.Ex[c] = e;
      ex_out = e;
      ex_written = true;
    } else if (k == a.sheet_k) {  // the sheet covers the whole plane, walls included
      ex_out = a.Ex[c] + srcv;
      a.Ex[c] = ex_out;
      ex_written = true;
    }
    if (ey_y && xin && zin) {  // Ey
      T cz = hx - hx_km;
      T cx = hz - a.Hz[idx3(im, j, k, nx, ny)];
      if (zz >= 0) cz = stretch(tz, a.nmax, k, cz, &a.psi[2][((int64_t)zz * ny + j) * nx + i]);
      if (zx >= 0) cx = stretch(tx, a.nmax, i, cx, &a.psi[3][((int64_t)k * ny + j) * a.Z + zx]);
      a.Ey[c] = e_update(a.m, (mb >> 2) & 3, a.Ey[c], cz - cx, &a.Jy[c]);
    }
    if (k < nz - 1 && xin && yin) {  // Ez
      T cx = hy - a.Hy[idx3(im, j, k, nx, ny)];
      T cy = hx - a.Hx[idx3(i, jm, k, nx, ny)];
      if (zx >= 0) cx = stretch(tx, a.nmax, i, cx, &a.psi[4][((int64_t)k * ny + j) * a.Z + zx]);
      if (zy >= 0) cy = stretch(ty, a.nmax, j, cy, &a.psi[5][((int64_t)k * a.Z + zy) * nx + i]);
      T e = e_update(a.m, (mb >> 4) & 3, a.Ez[c], cx - cy, &a.Jz[c]);
      if (tf_ez && k >= a.k0 && k <= a.k1 - 1)
        e = fma(i == a.i0 ? -a.S : a.S, a.Hi[k + a.inc_off], e);
      a.Ez[c] = e;
    }
    for (int q = 0; q < npc; ++q)
      if (pk[q] == k)
        a.series[(int64_t)ps[q] * a.series_len + a.series_pos] = ex_written ? ex_out : a.Ex[c];
    hx_km = hx;
    hy_km = hy;
  }
}

// CPML tables: [axis][E (integer positions) / H (half positions)][b, c, 1/kappa, flag][nmax]
template <typename T>
__global__ void k3_tables(int nx, int ny, int nz, int np, int per, double dt, double m, double smax, double kmax,
                          double amax, int nmax, T* tab) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nmax) return;
  const int N[3] = {nx, ny, nz};
  for (int ax = 0; ax < 3; ++ax) {
    const int npa = (ax < 2 && per) ? 0 : np;
    for (int h = 0; h < 2; ++h) {
      T* t = tab + (int64_t)(ax * 2 + h) * 4 * nmax;
      const double x = h ? n + 0.5 : (double)n;
      const double inner = (double)(N[ax] - 1) - npa;
      double rho = 0.0;
      if (npa > 0 && n < N[ax]) {
        if (x < npa) rho = (npa - x) / npa;
        else if (x > inner) rho = (x - inner) / npa;
      }
      double b = 0, c = 0, ki = 1, flag = 0;
      if (rho > 0) {
        const double pm = pow(rho, m);
        const double sigma = smax * pm;
        const double kap = 1.0 + (kmax - 1.0) * pm;
        const double alpha = amax * (1.0 - rho);
        b = exp(-(sigma / kap + alpha) * dt / kEps0);
        const double den = sigma * kap + kap * kap * alpha;
        c = (sigma > 0.0 && den > 0.0) ? sigma * (b - 1.0) / den : 0.0;
        ki = 1.0 / kap;
        flag = 1;
      }
      t[n] = (T)b;
      t[nmax + n] = (T)c;
      t[2 * nmax + n] = (T)ki;
      t[3 * nmax + n] = (T)flag;
    }
  }
}

template <typename T>
__global__ void k3_gather(const T* src, int64_t n, double scale, const T* cj, const uint8_t* mat, int shift,
                          double* out) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= n) return;
  double v = (double)src[c] * scale;
  if (cj) v /= (double)cj[(mat[c] >> shift) & 3];
  out[c] = v;
}

}  // namespace
}  // namespace rketd

using namespace rketd;

struct rketd_ctx3d {
  rketd_grid3d g{};
  int prec = 0;
  size_t esz = 4;
  int64_t N = 0;
  double S = 0;
  cudaStream_t stream = nullptr;
  std::vector<void*> allocs;
  void* f[9] = {};
  uint8_t* mat = nullptr;
  void* tab = nullptr;
  int nmax = 0, Z = 0;
  void* psi[12] = {};
  size_t psi_bytes[12] = {};
  void* Ei = nullptr;
  void* Hi = nullptr;
  int* probes = nullptr;
  int n_probes = 0, n_freq = 0;
  double* freq = nullptr;
  void* series = nullptr;
  void* tw = nullptr;
  double *Xr = nullptr, *Xi = nullptr, *Xtmp = nullptr;
  int dft_block = 512;
  double coef[6][kMat] = {};  // da, cb, cj, dj, bp(cj-scaled), cc(cj-scaled) per material
  void* cj_d = nullptr;
  int n_mat = 1;
  rketd_pulse pulse{};
  int64_t step = 0;
  int64_t launches = 0;
  ~rketd_ctx3d() {
    for (void* p : allocs) cudaFree(p);
  }
  bool alloc(void** p, size_t bytes) {
    *p = nullptr;
    if (cudaMalloc(p, bytes ? bytes : 16) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    allocs.push_back(*p);
    return true;
  }
};

namespace {

rketd_status fail3(rketd_status st, const std::string& m) {
  set_error_message(m.c_str());
  return st;
}

#define CK3(call, what)                                                                      \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess)                                                                   \
      return fail3(e_ == cudaErrorMemoryAllocation ? RKETD_ENOMEM : RKETD_ECUDA,             \
                   std::string(what) + ": " + cudaGetErrorString(e_));                       \
  } while (0)

template <typename T>
Args3<T> args3(rketd_ctx3d* c) {
  Args3<T> a{};
  T** F[9] = {&a.Ex, &a.Ey, &a.Ez, &a.Hx, &a.Hy, &a.Hz, &a.Jx, &a.Jy, &a.Jz};
  for (int q = 0; q < 9; ++q) *F[q] = (T*)c->f[q];
  a.mat = c->mat;
  for (int m = 0; m < kMat; ++m) {
    a.m.da[m] = (T)c->coef[0][m];
    a.m.cb[m] = (T)c->coef[1][m];
    a.m.dj[m] = (T)c->coef[3][m];
    a.m.bp[m] = (T)c->coef[4][m];
    a.m.cc[m] = (T)c->coef[5][m];
  }
  a.nx = c->g.nx;
  a.ny = c->g.ny;
  a.nz = c->g.nz;
  a.per = c->g.periodic_xy;
  a.S = (T)c->S;
  a.q = (T)((c->S - 1.0) / (c->S + 1.0));
  a.tab = (const T*)c->tab;
  a.nmax = c->nmax;
  a.np = c->g.npml;
  a.Z = c->Z;
  for (int q = 0; q < 12; ++q) a.psi[q] = (T*)c->psi[q];
  a.tfsf = c->g.tfsf;
  a.i0 = c->g.box[0];
  a.i1 = c->g.box[1];
  a.j0 = c->g.box[2];
  a.j1 = c->g.box[3];
  a.k0 = c->g.box[4];
  a.k1 = c->g.box[5];
  a.Ei = (T*)c->Ei;
  a.Hi = (T*)c->Hi;
  a.inc_len = c->g.inc_len;
  a.inc_off = c->g.inc_off;
  a.inc_src = c->g.inc_src;
  a.sheet_k = c->g.sheet_k;
  a.dt = c->g.dt;
  a.tau = c->pulse.tau;
  a.t0 = c->pulse.t0;
  a.amp = c->pulse.amp;
  a.n0 = c->step;
  a.probes = c->probes;
  a.n_probes = c->n_probes;
  a.series = (T*)c->series;
  a.series_len = c->dft_block;
  a.series_pos = (int)(c->step % c->dft_block);
  return a;
}

template <typename T>
rketd_status fold3(rketd_ctx3d* c, int n, int64_t m0, double* Xr, double* Xi) {
  if (!c->n_probes || !n) return RKETD_OK;
  CK3(launch_twiddles<T>(c->freq, c->n_freq, c->g.dt, m0, n, (T*)c->tw, c->stream), "twiddles");
  CK3(launch_dft<T>((const T*)c->series, c->dft_block, n, (const T*)c->tw, c->n_probes, c->n_freq, Xr, Xi, c->stream),
      "dft");
  c->launches += 2;
  return RKETD_OK;
}

template <typename T>
rketd_status step3(rketd_ctx3d* c, int64_t nsteps) {
  const dim3 block(32, 8);
  const dim3 grid((c->g.nx + 31) / 32, (c->g.ny + 7) / 8, c->g.tfsf ? 2 : 1);
  for (int64_t s = 0; s < nsteps; ++s) {
    Args3<T> a = args3<T>(c);
    k3_h<T><<<grid, block, 0, c->stream>>>(a);
    k3_e<T><<<grid, block, 0, c->stream>>>(a);
    CK3(cudaGetLastError(), "3D step");
    c->launches += 2;
    c->step += 1;
    if (c->step % c->dft_block == 0) {
      rketd_status st = fold3<T>(c, c->dft_block, c->step - c->dft_block + 1, c->Xr, c->Xi);
      if (st) return st;
    }
  }
  return RKETD_OK;
}

}  // namespace

extern "C" {

rketd_status rketd_create_3d(const rketd_grid3d* g, const uint8_t* mat, int32_t n_mat, const double* mat_wp2,
                             const double* mat_nu, const rketd_pulse* pulse, int32_t n_probes, const int32_t* probes,
                             const rketd_dft* dft, void* stream, rketd_ctx3d** out) {
  set_error_message("");
  if (!out) return fail3(RKETD_EINVAL, "out is NULL");
  *out = nullptr;
  if (!g || !mat || !mat_wp2 || !mat_nu || !pulse) return fail3(RKETD_EINVAL, "NULL argument");
  if (g->nx < 4 || g->ny < 4 || g->nz < 4) return fail3(RKETD_EINVAL, "grid must be at least 4 cells per axis");
  if (!(g->d > 0) || !(g->dt > 0) || !std::isfinite(g->d) || !std::isfinite(g->dt))
    return fail3(RKETD_EINVAL, "d and dt must be finite and > 0");
  if (g->prec != RKETD_F32 && g->prec != RKETD_F64) return fail3(RKETD_EINVAL, "prec must be F32 or F64");
  const double S = g->dt / (g->d * std::sqrt(kMu0 * kEps0));
  if (!(S <= 1.0 / std::sqrt(3.0))) return fail3(RKETD_ECOURANT, "3D Courant number c dt/d exceeds 1/sqrt(3)");
  if (n_mat < 1 || n_mat > kMat) return fail3(RKETD_EINVAL, "n_mat must be 1..4 (entry 0 is vacuum)");
  for (int m = 0; m < n_mat; ++m)
    if (!(mat_wp2[m] >= 0) || !(mat_nu[m] >= 0) || !std::isfinite(mat_wp2[m]) || !std::isfinite(mat_nu[m]))
      return fail3(RKETD_EINVAL, "material wp2 and nu must be finite and >= 0");
  if (mat_wp2[0] != 0.0) return fail3(RKETD_EINVAL, "material 0 must be vacuum");
  const int np = g->npml;
  if (np < 1 || 2 * (np + 1) + 2 > g->nz || (!g->periodic_xy && (2 * (np + 1) + 2 > g->nx || 2 * (np + 1) + 2 > g->ny)))
    return fail3(RKETD_EINVAL, "npml must be >= 1 and fit the grid");
  if (g->tfsf) {
    const int* b = g->box;
    const int lx = g->periodic_xy ? 1 : np + 1, ly = lx;
    if (b[0] < lx || b[1] > g->nx - 1 - lx || b[0] >= b[1] || b[2] < ly || b[3] > g->ny - 1 - ly || b[2] >= b[3] ||
        b[4] < np + 2 || b[5] > g->nz - 2 - np || b[4] >= b[5])
      return fail3(RKETD_EINVAL, "TF/SF box must lie inside the grid, outside the CPML");
    if (g->inc_off < 2 || g->inc_len < g->nz + 2 * g->inc_off || g->inc_src < 1 || g->inc_src >= g->inc_off)
      return fail3(RKETD_EINVAL, "incident line must cover the grid with its source before it");
  }
  if (g->sheet_k >= 0 && (g->sheet_k < np + 1 || g->sheet_k > g->nz - 2 - np))
    return fail3(RKETD_EINVAL, "sheet source must lie outside the CPML");
  const int nf = dft ? dft->n_freq : 0;
  if (n_probes < 0 || (n_probes > 0 && (!probes || nf < 1 || !dft->freq_hz)))
    return fail3(RKETD_EINVAL, "probes need coordinates and frequencies");
  for (int p = 0; p < n_probes; ++p)
    if (probes[3 * p] < 0 || probes[3 * p] >= g->nx || probes[3 * p + 1] < 0 || probes[3 * p + 1] >= g->ny ||
        probes[3 * p + 2] < 0 || probes[3 * p + 2] >= g->nz)
      return fail3(RKETD_EINVAL, "probe outside the grid");
  rketd_ctx3d* c = new (std::nothrow) rketd_ctx3d();
  if (!c) return fail3(RKETD_ENOMEM, "host allocation");
  auto bad = [&](rketd_status s, const char* m) {
    delete c;
    return fail3(s, m);
  };
  c->g = *g;
  if (!(c->g.pml_sigma_max > 0)) c->g.pml_sigma_max = 0.8 * (g->pml_m + 1) / (std::sqrt(kMu0 / kEps0) * g->d);
  c->prec = g->prec;
  c->esz = g->prec == RKETD_F64 ? 8 : 4;
  c->N = (int64_t)g->nx * g->ny * g->nz;
  c->S = S;
  c->stream = (cudaStream_t)stream;
  c->pulse = *pulse;
  c->n_mat = n_mat;
  c->n_probes = n_probes;
  c->n_freq = n_probes ? nf : 0;
  // per-material coefficients (the 1D formulas, FP64 on the host for at most four entries,
  // then used as kernel arguments)
  for (int m = 0; m < kMat; ++m) {
    const double w = m < n_mat ? mat_wp2[m] * g->dt * g->dt : 0.0;
    const double x = m < n_mat ? mat_nu[m] * g->dt : 0.0;
    // phi1, phi2 by their Taylor series below 0.5, expm1 above
    double p1, p2;
    if (x < 0.5) {
      double t1 = 1.0, t2 = 0.5, s1 = 0, s2 = 0;
      double terms1[24], terms2[24];
      for (int q = 0; q < 24; ++q) {
        terms1[q] = t1;
        terms2[q] = t2;
        t1 *= -x / (q + 2);
        t2 *= -x / (q + 3);
      }
      for (int q = 23; q >= 0; --q) {
        s1 += terms1[q];
        s2 += terms2[q];
      }
      p1 = s1;
      p2 = s2;
    } else {
      const double em = std::expm1(-x);
      p1 = -em / x;
      p2 = (x + em) / (x * x);
    }
    const double em = std::expm1(-x);
    const double D = 1.0 + 0.5 * w * p2;
    const double cj = 0.5 * (2.0 + em) / D;
    c->coef[0][m] = -0.5 * w * p1 / D;
    c->coef[1][m] = S / D;
    c->coef[2][m] = cj;
    c->coef[3][m] = em;
    c->coef[4][m] = cj * (w * (p1 - p2));
    c->coef[5][m] = cj * (w * p2);
  }
  const size_t fb = c->esz * c->N;
  for (int q = 0; q < 9; ++q)
    if (!c->alloc(&c->f[q], fb)) return bad(RKETD_ENOMEM, "3D fields");
  if (!c->alloc((void**)&c->mat, c->N)) return bad(RKETD_ENOMEM, "3D materials");
  c->nmax = std::max(g->nx, std::max(g->ny, g->nz));
  c->Z = 2 * (np + 1);
  if (!c->alloc(&c->tab, c->esz * 24 * c->nmax)) return bad(RKETD_ENOMEM, "CPML tables");
  // compact zones: x-derivative memories [k][j][Z], y [k][Z][i], z [Z][j][i]
  const int64_t zsz[3] = {(int64_t)g->nz * g->ny * c->Z, (int64_t)g->nz * c->Z * g->nx,
                          (int64_t)c->Z * g->ny * g->nx};
  for (int q = 0; q < 12; ++q) {
    const int ax = kPsiAxis[q];
    c->psi_bytes[q] = (ax < 2 && g->periodic_xy) ? 16 : c->esz * zsz[ax];
    if (!c->alloc(&c->psi[q], c->psi_bytes[q])) return bad(RKETD_ENOMEM, "CPML memories");
  }
  if (!c->alloc(&c->Ei, c->esz * std::max(1, g->inc_len)) || !c->alloc(&c->Hi, c->esz * std::max(1, g->inc_len)))
    return bad(RKETD_ENOMEM, "incident line");
  if (!c->alloc(&c->cj_d, c->esz * kMat)) return bad(RKETD_ENOMEM, "coefficients");
  if (n_probes) {
    if (!c->alloc((void**)&c->probes, sizeof(int) * 3 * n_probes) || !c->alloc((void**)&c->freq, sizeof(double) * nf) ||
        !c->alloc(&c->series, c->esz * (size_t)n_probes * c->dft_block) ||
        !c->alloc(&c->tw, c->esz * 2 * (size_t)c->dft_block * nf) ||
        !c->alloc((void**)&c->Xr, sizeof(double) * n_probes * nf) || !c->alloc((void**)&c->Xi, sizeof(double) * n_probes * nf) ||
        !c->alloc((void**)&c->Xtmp, sizeof(double) * 2 * n_probes * nf))
      return bad(RKETD_ENOMEM, "probes");
    if (cudaMemcpy(c->probes, probes, sizeof(int) * 3 * n_probes, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(c->freq, dft->freq_hz, sizeof(double) * nf, cudaMemcpyHostToDevice) != cudaSuccess)
      return bad(RKETD_ECUDA, "probe upload");
  }
  if (cudaMemcpy(c->mat, mat, c->N, cudaMemcpyHostToDevice) != cudaSuccess) return bad(RKETD_ECUDA, "material upload");
  {
    std::vector<char> cj(c->esz * kMat);
    for (int m = 0; m < kMat; ++m) {
      if (c->prec == RKETD_F64) ((double*)cj.data())[m] = c->coef[2][m];
      else ((float*)cj.data())[m] = (float)c->coef[2][m];
    }
    if (cudaMemcpy(c->cj_d, cj.data(), cj.size(), cudaMemcpyHostToDevice) != cudaSuccess)
      return bad(RKETD_ECUDA, "coefficient upload");
  }
  const unsigned tb = (unsigned)((c->nmax + 127) / 128);
  if (c->prec == RKETD_F64)
    k3_tables<double><<<tb, 128, 0, c->stream>>>(g->nx, g->ny, g->nz, np, g->periodic_xy, g->dt, g->pml_m,
                                                 c->g.pml_sigma_max, g->pml_kappa_max, g->pml_alpha_max, c->nmax,
                                                 (double*)c->tab);
  else
    k3_tables<float><<<tb, 128, 0, c->stream>>>(g->nx, g->ny, g->nz, np, g->periodic_xy, g->dt, g->pml_m,
                                                c->g.pml_sigma_max, g->pml_kappa_max, g->pml_alpha_max, c->nmax,
                                                (float*)c->tab);
  c->launches += 1;
  rketd_status st = rketd_reset_3d(c);
  if (st) {
    delete c;
    return st;
  }
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return bad(RKETD_ECUDA, "create");
  *out = c;
  return RKETD_OK;
}

rketd_status rketd_reset_3d(rketd_ctx3d* c) {
  if (!c) return fail3(RKETD_EINVAL, "NULL context");
  const size_t fb = c->esz * c->N;
  for (int q = 0; q < 9; ++q) CK3(cudaMemsetAsync(c->f[q], 0, fb, c->stream), "reset");
  for (int q = 0; q < 12; ++q) CK3(cudaMemsetAsync(c->psi[q], 0, c->psi_bytes[q], c->stream), "reset");
  CK3(cudaMemsetAsync(c->Ei, 0, c->esz * std::max(1, c->g.inc_len), c->stream), "reset");
  CK3(cudaMemsetAsync(c->Hi, 0, c->esz * std::max(1, c->g.inc_len), c->stream), "reset");
  if (c->n_probes) {
    CK3(cudaMemsetAsync(c->Xr, 0, sizeof(double) * c->n_probes * c->n_freq, c->stream), "reset");
    CK3(cudaMemsetAsync(c->Xi, 0, sizeof(double) * c->n_probes * c->n_freq, c->stream), "reset");
  }
  c->step = 0;
  return RKETD_OK;
}

rketd_status rketd_step_3d(rketd_ctx3d* c, int64_t nsteps) {
  if (!c) return fail3(RKETD_EINVAL, "NULL context");
  if (nsteps < 0) return fail3(RKETD_EINVAL, "nsteps < 0");
  return c->prec == RKETD_F64 ? step3<double>(c, nsteps) : step3<float>(c, nsteps);
}

rketd_status rketd_get_field_3d(rketd_ctx3d* c, int32_t which, double* out) {
  if (!c || !out || which < 0 || which > 8) return fail3(RKETD_EINVAL, "invalid arguments");
  double* tmp;
  CK3(cudaMallocAsync((void**)&tmp, sizeof(double) * c->N, c->stream), "field staging");
  const double eta0 = std::sqrt(kMu0 / kEps0);
  const double scale = which < 3 ? 1.0 : (which < 6 ? 1.0 / eta0 : kEps0 / c->g.dt);
  const int shift = which >= 6 ? 2 * (which - 6) : 0;
  const unsigned blocks = (unsigned)((c->N + 255) / 256);
  if (c->prec == RKETD_F64)
    k3_gather<double><<<blocks, 256, 0, c->stream>>>((const double*)c->f[which], c->N, scale,
                                                     which >= 6 ? (const double*)c->cj_d : nullptr, c->mat, shift, tmp);
  else
    k3_gather<float><<<blocks, 256, 0, c->stream>>>((const float*)c->f[which], c->N, scale,
                                                    which >= 6 ? (const float*)c->cj_d : nullptr, c->mat, shift, tmp);
  cudaError_t e = cudaMemcpyAsync(out, tmp, sizeof(double) * c->N, cudaMemcpyDeviceToHost, c->stream);
  cudaFreeAsync(tmp, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  CK3(e, "get_field_3d");
  return RKETD_OK;
}

rketd_status rketd_get_spectra_3d(rketd_ctx3d* c, double* re, double* im) {
  if (!c || !re || !im) return fail3(RKETD_EINVAL, "NULL argument");
  const size_t n = (size_t)c->n_probes * c->n_freq;
  if (!n) return RKETD_OK;
  CK3(cudaMemcpyAsync(c->Xtmp, c->Xr, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream), "spectra");
  CK3(cudaMemcpyAsync(c->Xtmp + n, c->Xi, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream), "spectra");
  const int pending = (int)(c->step % c->dft_block);
  if (pending) {
    rketd_status st = c->prec == RKETD_F64 ? fold3<double>(c, pending, c->step - pending + 1, c->Xtmp, c->Xtmp + n)
                                           : fold3<float>(c, pending, c->step - pending + 1, c->Xtmp, c->Xtmp + n);
    if (st) return st;
  }
  CK3(cudaMemcpyAsync(re, c->Xtmp, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream), "spectra");
  CK3(cudaMemcpyAsync(im, c->Xtmp + n, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream), "spectra");
  CK3(cudaStreamSynchronize(c->stream), "spectra");
  return RKETD_OK;
}

int64_t rketd_launch_count_3d(const rketd_ctx3d* c) { return c ? c->launches : -1; }

rketd_status rketd_destroy_3d(rketd_ctx3d* c) {
  if (!c) return RKETD_OK;
  cudaStreamSynchronize(c->stream);
  delete c;
  return RKETD_OK;
}

}  // extern "C"
