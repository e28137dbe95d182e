// 3D Yee RKETD-FDTD step (the paper's stated 2D/3D generalisation, Sec. IV.B and Sec. V):
// the three-component form of the 1D update, in the same normalised variables
// (E~ = E, H~ = eta0 H, carried current cj (dt/eps0) J) and with the same per-material
// coefficients (rketd_internal.cuh), plus CPML on every face backed by PEC walls (or
// periodic x and y), a total-field/scattered-field box fed by a 1D line, a soft sheet
// source and a running DFT of Ex at probe points.
//
// Arrays are [k][j][i] (x fastest). Yee positions:
//   Ex (i+1/2, j, k), Ey (i, j+1/2, k), Ez (i, j, k+1/2),
//   Hx (i, j+1/2, k+1/2), Hy (i+1/2, j, k+1/2), Hz (i+1/2, j+1/2, k).
// Each E component takes the material at its own position: mat[c] packs the material
// indices of Ex, Ey, Ez of cell c in bits 0-1, 2-3, 4-5 (0 = vacuum).
//
// Three forms of one step, doing the same operations on the same values:
//  - plain: the paper's structure, an H kernel then an E+J kernel, fields updated in place;
//  - staged (default where it applies): the fused step below fed from shared memory, whole
//    planes of the step-n state brought in by the tensor memory accelerator (k3_staged);
//  - fused: one kernel per step reading the step-n state (E, H, the H-side CPML
//    memories, the incident line) and writing the step-n+1 state into a second set of
//    buffers. A warp owns 32 consecutive i of one j row and a chunk of k; the new H of its
//    own cells is stored and fed to the E update in registers: the i-1 neighbour comes from
//    the next lane down (lane 0 recomputes it), the k-1 neighbour from the previous k, and
//    the j-1 neighbour is recomputed from the step-n state (its owner may not have written
//    it yet). E and H are each read once and written once per step.
#include <cuda.h>
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
constexpr unsigned kFull = 0xffffffffu;

template <typename T>
struct Mat3 {
  T da[kMat], cb[kMat], dj[kMat], bp[kMat], cc[kMat];
};

template <typename T>
struct Args3 {
  // step-n state (read) and step-n+1 state (written); the plain kernels pass one set for both
  const T *Ex, *Ey, *Ez, *Hx, *Hy, *Hz;
  T *oEx, *oEy, *oEz, *oHx, *oHy, *oHz;
  T *Jx, *Jy, *Jz;  // carried currents, updated in place
  const uint8_t* mat;
  Mat3<T> m;
  int nx, ny, nz, per, kc;
  T S, q;
  // CPML: tables [axis][E/H][db = b - 1, c, 1/kappa, flag][nmax]; memories in compact face zones of
  // width Z: x-derivative [k][j][Z], y-derivative [k][Z][i], z-derivative [Z][j][i]
  const T* tab;
  int nmax, np, Z;
  T* psiE[6];        // Ex/y, Ex/z, Ey/z, Ey/x, Ez/x, Ez/y (in place)
  const T* psiH[6];  // Hx/y, Hx/z, Hy/z, Hy/x, Hz/x, Hz/y (read)
  T* opsiH[6];       // (written)
  // TF/SF box and its 1D line (index k + inc_off)
  int tfsf, i0, i1, j0, j1, k0, k1;
  const T* Ei;
  const T* Hi;
  T* oEi;
  T* oHi;
  int line_fresh;  // 1: Hi already holds H^{n+1/2} (plain form); 0: derive it from Ei, Hi
  int inc_len, inc_off, inc_src;
  // sources and probes
  int sheet_k;
  double dt, tau, t0, amp;
  int64_t n0;
  const int* probes;  // [P][3]
  int n_probes;
  T* series;
  int series_len, series_pos;
  int wait_limit;  // polls of the staged form's compute-path copy waits (a test hook may lower it)
  // staged form: facts of planes -1 .. nz of this step (PlaneS records, Stage3::pl_bytes apart),
  // written by k3_facts before the step's tile kernels
  unsigned char* ftab;
};

__device__ __forceinline__ int64_t idx3(int i, int j, int k, int nx, int ny) {
  return ((int64_t)k * ny + j) * nx + i;
}

// compact CPML zone of node n on an axis of N nodes with np layers (-1: outside)
__device__ __forceinline__ int zone(int n, int N, int np) {
  if (np <= 0) return -1;
  if (n < np + 1) return n;
  if (n >= N - np - 1) return np + 1 + (n - (N - np - 1));
  return -1;
}

template <typename T>
__device__ __forceinline__ int64_t zx_off(const Args3<T>& a, int j, int k, int z) {
  return ((int64_t)k * a.ny + j) * a.Z + z;
}
template <typename T>
__device__ __forceinline__ int64_t zy_off(const Args3<T>& a, int i, int k, int z) {
  return ((int64_t)k * a.Z + z) * a.nx + i;
}
template <typename T>
__device__ __forceinline__ int64_t zz_off(const Args3<T>& a, int i, int j, int z) {
  return ((int64_t)z * a.ny + j) * a.nx + i;
}

template <typename T>
__device__ __forceinline__ const T* tb(const Args3<T>& a, int ax, int h) {
  return a.tab + (int64_t)(ax * 2 + h) * 4 * a.nmax;
}

__device__ __forceinline__ double pulse3(double t, double t0, double tau, double amp) {
  const double u = (t - t0) / tau;
  return amp * u * exp(-0.5 * u * u);
}

// read of the step-n state: through the read-only cache when nothing in the kernel writes it
template <bool RO, typename T>
__device__ __forceinline__ T rd(const T* p) {
  if constexpr (RO) return __ldg(p);
  else return *p;
}

// CPML-stretched difference: psi' = psi + db psi + c dv (db = b - 1, kept as a deviation so that
// an FP32 copy is accurate where b is within 1e-5 of 1), result dv / kappa + psi'.
// pout = nullptr: the new memory is not stored (a neighbour's value recomputed).
template <bool RO, typename T>
__device__ __forceinline__ T stretch(const T* t, int nmax, int pos, T dv, const T* pin, T* pout) {
  if (t[3 * nmax + pos] == T(0)) return dv;
  const T po = rd<RO>(pin);
  const T p = fma(t[pos], po, fma(t[nmax + pos], dv, po));
  if (pout) *pout = p;
  return fma(dv, t[2 * nmax + pos], p);
}

// New H components at one cell (Eq. 14 per component, CPML, TF/SF corrections with the
// step-n incident E) from the values of the step-n E and H it depends on. Every form of the
// step calls these, so all forms do the same operations on the same values.
// own = false: the CPML memories are read but not stored (a neighbour's value recomputed).
template <bool RO, typename T>
__device__ __forceinline__ T hx_core(const Args3<T>& a, int i, int j, int k, T h, T ez_jp, T ez, T ey_kp, T ey,
                                     bool own) {
  const int jp = (j + 1 < a.ny) ? j + 1 : (a.per ? 0 : -1);
  if (jp < 0 || k + 1 >= a.nz) return h;
  T cy = ez_jp - ez;
  T cz = ey_kp - ey;
  const int zy = a.per ? -1 : zone(j, a.ny, a.np), zz = zone(k, a.nz, a.np);
  if (zy >= 0) {
    const int64_t o = zy_off(a, i, k, zy);
    cy = stretch<RO>(tb(a, 1, 1), a.nmax, j, cy, a.psiH[0] + o, own ? a.opsiH[0] + o : nullptr);
  }
  if (zz >= 0) {
    const int64_t o = zz_off(a, i, j, zz);
    cz = stretch<RO>(tb(a, 2, 1), a.nmax, k, cz, a.psiH[1] + o, own ? a.opsiH[1] + o : nullptr);
  }
  return fma(-a.S, cy - cz, h);
}

template <bool RO, typename T>
__device__ __forceinline__ T hy_core(const Args3<T>& a, int i, int j, int k, T h, T ex_kp, T ex, T ez_ip, T ez,
                                     bool own) {
  const int ip = (i + 1 < a.nx) ? i + 1 : (a.per ? 0 : -1);
  if (ip < 0 || k + 1 >= a.nz) return h;
  T cz = ex_kp - ex;
  T cx = ez_ip - ez;
  const int zz = zone(k, a.nz, a.np), zx = a.per ? -1 : zone(i, a.nx, a.np);
  if (zz >= 0) {
    const int64_t o = zz_off(a, i, j, zz);
    cz = stretch<RO>(tb(a, 2, 1), a.nmax, k, cz, a.psiH[2] + o, own ? a.opsiH[2] + o : nullptr);
  }
  if (zx >= 0) {
    const int64_t o = zx_off(a, j, k, zx);
    cx = stretch<RO>(tb(a, 0, 1), a.nmax, i, cx, a.psiH[3] + o, own ? a.opsiH[3] + o : nullptr);
  }
  T v = fma(-a.S, cz - cx, h);
  if (a.tfsf && i >= a.i0 && i <= a.i1 - 1 && j >= a.j0 && j <= a.j1) {
    if (k == a.k0 - 1) v = fma(a.S, rd<RO>(a.Ei + a.k0 + a.inc_off), v);
    if (k == a.k1) v = fma(-a.S, rd<RO>(a.Ei + a.k1 + a.inc_off), v);
  }
  return v;
}

template <bool RO, typename T>
__device__ __forceinline__ T hz_core(const Args3<T>& a, int i, int j, int k, T h, T ey_ip, T ey, T ex_jp, T ex,
                                     bool own) {
  const int ip = (i + 1 < a.nx) ? i + 1 : (a.per ? 0 : -1);
  const int jp = (j + 1 < a.ny) ? j + 1 : (a.per ? 0 : -1);
  if (ip < 0 || jp < 0) return h;
  T cx = ey_ip - ey;
  T cy = ex_jp - ex;
  const int zx = a.per ? -1 : zone(i, a.nx, a.np), zy = a.per ? -1 : zone(j, a.ny, a.np);
  if (zx >= 0) {
    const int64_t o = zx_off(a, j, k, zx);
    cx = stretch<RO>(tb(a, 0, 1), a.nmax, i, cx, a.psiH[4] + o, own ? a.opsiH[4] + o : nullptr);
  }
  if (zy >= 0) {
    const int64_t o = zy_off(a, i, k, zy);
    cy = stretch<RO>(tb(a, 1, 1), a.nmax, j, cy, a.psiH[5] + o, own ? a.opsiH[5] + o : nullptr);
  }
  T v = fma(-a.S, cx - cy, h);
  if (a.tfsf && i >= a.i0 && i <= a.i1 - 1 && k >= a.k0 && k <= a.k1) {
    if (j == a.j0 - 1) v = fma(-a.S, rd<RO>(a.Ei + k + a.inc_off), v);
    if (j == a.j1) v = fma(a.S, rd<RO>(a.Ei + k + a.inc_off), v);
  }
  return v;
}

// the same from global memory (neighbours loaded only where the update is defined)
template <bool RO, typename T>
__device__ __forceinline__ T hx_new(const Args3<T>& a, int i, int j, int k, bool own) {
  const int64_t c = idx3(i, j, k, a.nx, a.ny);
  const T h = rd<RO>(a.Hx + c);
  const int jp = (j + 1 < a.ny) ? j + 1 : (a.per ? 0 : -1);
  if (jp < 0 || k + 1 >= a.nz) return h;
  const int64_t nxy = (int64_t)a.nx * a.ny;
  return hx_core<RO>(a, i, j, k, h, rd<RO>(a.Ez + idx3(i, jp, k, a.nx, a.ny)), rd<RO>(a.Ez + c),
                     rd<RO>(a.Ey + c + nxy), rd<RO>(a.Ey + c), own);
}

template <bool RO, typename T>
__device__ __forceinline__ T hy_new(const Args3<T>& a, int i, int j, int k, bool own) {
  const int64_t c = idx3(i, j, k, a.nx, a.ny);
  const T h = rd<RO>(a.Hy + c);
  const int ip = (i + 1 < a.nx) ? i + 1 : (a.per ? 0 : -1);
  if (ip < 0 || k + 1 >= a.nz) return h;
  const int64_t nxy = (int64_t)a.nx * a.ny;
  return hy_core<RO>(a, i, j, k, h, rd<RO>(a.Ex + c + nxy), rd<RO>(a.Ex + c),
                     rd<RO>(a.Ez + idx3(ip, j, k, a.nx, a.ny)), rd<RO>(a.Ez + c), own);
}

template <bool RO, typename T>
__device__ __forceinline__ T hz_new(const Args3<T>& a, int i, int j, int k, bool own) {
  const int64_t c = idx3(i, j, k, a.nx, a.ny);
  const T h = rd<RO>(a.Hz + c);
  const int ip = (i + 1 < a.nx) ? i + 1 : (a.per ? 0 : -1);
  const int jp = (j + 1 < a.ny) ? j + 1 : (a.per ? 0 : -1);
  if (ip < 0 || jp < 0) return h;
  return hz_core<RO>(a, i, j, k, h, rd<RO>(a.Ey + idx3(ip, j, k, a.nx, a.ny)), rd<RO>(a.Ey + c),
                     rd<RO>(a.Ex + idx3(i, jp, k, a.nx, a.ny)), rd<RO>(a.Ex + c), own);
}

// incident H~ at line index m, time n+1/2
template <bool RO, typename T>
__device__ __forceinline__ T hinc(const Args3<T>& a, int m) {
  if (a.line_fresh) return a.Hi[m];
  return fma(-a.S, rd<RO>(a.Ei + m + 1) - rd<RO>(a.Ei + m), rd<RO>(a.Hi + m));
}

// E' = E + da E + cb curl - Jc,  Jc' = Jc + dj Jc + bp E + cc E'  (material m of the component)
template <typename T>
__device__ __forceinline__ T e_update(const Mat3<T>& M, int m, T e, T curl, T* J) {
  if (m == 0) return fma(M.cb[0], curl, e);
  const T jc = *J;
  // the small terms are summed before the carried E and J are added, so that da E and dj J
  // (a few ulp of E and J) are not rounded away on their own every step
  const T en = e + fma(M.cb[m], curl, fma(M.da[m], e, -jc));
  *J = jc + fma(M.cc[m], en, fma(M.bp[m], e, M.dj[m] * jc));
  return en;
}

// E and J update of one cell (Eqs. 12, 11, 13 per component) from the new H of the cell and
// of its i-1, j-1, k-1 neighbours; CPML, TF/SF corrections, sheet source. Returns the new Ex.
template <bool RO, typename T>
__device__ __forceinline__ T e_cell(const Args3<T>& a, int i, int j, int k, T ex, T ey, T ez, int mb, T hx, T hy,
                                    T hz, T hx_jm, T hz_jm, T hy_im, T hz_im, T hx_km, T hy_km, T srcv) {
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const int64_t c = idx3(i, j, k, nx, ny);
  const bool xin = a.per || (i > 0 && i < nx - 1);
  const bool yin = a.per || (j > 0 && j < ny - 1);
  const bool zin = k > 0 && k < nz - 1;
  const int zx = a.per ? -1 : zone(i, nx, a.np), zy = a.per ? -1 : zone(j, ny, a.np), zz = zone(k, nz, a.np);
  const T* tx = tb(a, 0, 0);
  const T* ty = tb(a, 1, 0);
  const T* tz = tb(a, 2, 0);
  if ((a.per || i < nx - 1) && yin && zin) {
    T cy = hz - hz_jm, cz = hy - hy_km;
    if (zy >= 0) {
      T* p = a.psiE[0] + zy_off(a, i, k, zy);
      cy = stretch<false>(ty, a.nmax, j, cy, p, p);
    }
    if (zz >= 0) {
      T* p = a.psiE[1] + zz_off(a, i, j, zz);
      cz = stretch<false>(tz, a.nmax, k, cz, p, p);
    }
    ex = e_update(a.m, mb & 3, ex, cy - cz, a.Jx + c);
    if (a.tfsf && i >= a.i0 && i <= a.i1 - 1 && j >= a.j0 && j <= a.j1) {
      if (k == a.k0) ex = fma(a.S, hinc<RO>(a, a.k0 - 1 + a.inc_off), ex);
      if (k == a.k1) ex = fma(-a.S, hinc<RO>(a, a.k1 + a.inc_off), ex);
    }
  }
  if (k == a.sheet_k) ex = ex + srcv;  // the sheet covers the whole plane, walls included
  a.oEx[c] = ex;
  if ((a.per || j < ny - 1) && xin && zin) {
    T cz = hx - hx_km, cx = hz - hz_im;
    if (zz >= 0) {
      T* p = a.psiE[2] + zz_off(a, i, j, zz);
      cz = stretch<false>(tz, a.nmax, k, cz, p, p);
    }
    if (zx >= 0) {
      T* p = a.psiE[3] + zx_off(a, j, k, zx);
      cx = stretch<false>(tx, a.nmax, i, cx, p, p);
    }
    ey = e_update(a.m, (mb >> 2) & 3, ey, cz - cx, a.Jy + c);
  }
  a.oEy[c] = ey;
  if (k < nz - 1 && xin && yin) {
    T cx = hy - hy_im, cy = hx - hx_jm;
    if (zx >= 0) {
      T* p = a.psiE[4] + zx_off(a, j, k, zx);
      cx = stretch<false>(tx, a.nmax, i, cx, p, p);
    }
    if (zy >= 0) {
      T* p = a.psiE[5] + zy_off(a, i, k, zy);
      cy = stretch<false>(ty, a.nmax, j, cy, p, p);
    }
    ez = e_update(a.m, (mb >> 4) & 3, ez, cx - cy, a.Jz + c);
    if (a.tfsf && j >= a.j0 && j <= a.j1 && (i == a.i0 || i == a.i1) && k >= a.k0 && k <= a.k1 - 1)
      ez = fma(i == a.i0 ? -a.S : a.S, hinc<RO>(a, k + a.inc_off), ez);
  }
  a.oEz[c] = ez;
  return ex;
}

// probes of one (i, j) column inside [k_lo, k_hi): up to 4, as (k, probe index)
template <typename T>
__device__ __forceinline__ int column_probes(const Args3<T>& a, int i, int j, int k_lo, int k_hi, int* pk, int* ps) {
  int n = 0;
  for (int p = 0; p < a.n_probes && n < 4; ++p)
    if (a.probes[3 * p] == i && a.probes[3 * p + 1] == j && a.probes[3 * p + 2] >= k_lo && a.probes[3 * p + 2] < k_hi) {
      pk[n] = a.probes[3 * p + 2];
      ps[n] = p;
      ++n;
    }
  return n;
}

// ---------------------------------------------------------------------------------------
// plain form: H kernel, then E+J kernel (in place); block z-slices cover k in chunks of a.kc
// and, with TF/SF, one extra slice advances the incident line.
template <typename T>
__global__ void __launch_bounds__(256) k3_h(const Args3<T> a) {
  const int nzc = (a.nz + a.kc - 1) / a.kc;
  if ((int)blockIdx.z >= nzc) {  // incident line: H~ -= S (E_{m+1} - E_m)
    if (blockIdx.x != 0 || blockIdx.y != 0) return;
    for (int m = threadIdx.y * blockDim.x + threadIdx.x; m < a.inc_len - 1; m += blockDim.x * blockDim.y)
      a.oHi[m] = fma(-a.S, a.Ei[m + 1] - a.Ei[m], a.Hi[m]);
    return;
  }
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= a.nx || j >= a.ny) return;
  const int kb = blockIdx.z * a.kc, ke = min(a.nz, kb + a.kc);
  for (int k = kb; k < ke; ++k) {
    const int64_t c = idx3(i, j, k, a.nx, a.ny);
    const T hx = hx_new<false>(a, i, j, k, true);
    const T hy = hy_new<false>(a, i, j, k, true);
    const T hz = hz_new<false>(a, i, j, k, true);
    a.oHx[c] = hx;
    a.oHy[c] = hy;
    a.oHz[c] = hz;
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k3_e(const Args3<T> a) {
  const int nx = a.nx, ny = a.ny;
  const double t = (double)(a.n0 + 1) * a.dt;
  const int nzc = (a.nz + a.kc - 1) / a.kc;
  if ((int)blockIdx.z >= nzc) {  // incident line: E update, soft source, first-order Mur ends
    if (blockIdx.x != 0 || blockIdx.y != 0) return;
    __shared__ T ends[4];
    const int tid = threadIdx.y * blockDim.x + threadIdx.x, nt = blockDim.x * blockDim.y, L = a.inc_len;
    if (tid == 0) {
      ends[0] = a.Ei[0];
      ends[1] = a.Ei[1];
      ends[2] = a.Ei[L - 2];
      ends[3] = a.Ei[L - 1];
    }
    __syncthreads();
    for (int m = 1 + tid; m < L - 1; m += nt) a.oEi[m] = fma(-a.S, a.Hi[m] - a.Hi[m - 1], a.Ei[m]);
    __syncthreads();
    if (tid == 0) {
      a.oEi[a.inc_src] = a.oEi[a.inc_src] + (T)pulse3(t, a.t0, a.tau, a.amp);
      a.oEi[0] = fma(a.q, a.oEi[1] - ends[0], ends[1]);
      a.oEi[L - 1] = fma(a.q, a.oEi[L - 2] - ends[3], ends[2]);
    }
    return;
  }
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= nx || j >= ny) return;
  const int im = (i > 0) ? i - 1 : (a.per ? nx - 1 : -1);
  const int jm = (j > 0) ? j - 1 : (a.per ? ny - 1 : -1);
  const int kb = blockIdx.z * a.kc, ke = min(a.nz, kb + a.kc);
  // the sheet source's value, only where this column range holds the sheet (FP64 is narrow here)
  const T srcv = (a.sheet_k >= kb && a.sheet_k < ke) ? (T)pulse3(t, a.t0, a.tau, a.amp) : T(0);
  int pk[4], ps[4];
  const int npc = column_probes(a, i, j, kb, ke, pk, ps);
  T hx_km = T(0), hy_km = T(0);
  if (kb > 0) {
    hx_km = a.Hx[idx3(i, j, kb - 1, nx, ny)];
    hy_km = a.Hy[idx3(i, j, kb - 1, nx, ny)];
  }
  for (int k = kb; k < ke; ++k) {
    const int64_t c = idx3(i, j, k, nx, ny);
    const T hx = a.Hx[c], hy = a.Hy[c], hz = a.Hz[c];
    T hx_jm = T(0), hz_jm = T(0), hy_im = T(0), hz_im = T(0);
    if (jm >= 0) {
      hx_jm = a.Hx[idx3(i, jm, k, nx, ny)];
      hz_jm = a.Hz[idx3(i, jm, k, nx, ny)];
    }
    if (im >= 0) {
      hy_im = a.Hy[idx3(im, j, k, nx, ny)];
      hz_im = a.Hz[idx3(im, j, k, nx, ny)];
    }
    const T ex = e_cell<false>(a, i, j, k, a.Ex[c], a.Ey[c], a.Ez[c], a.mat[c], hx, hy, hz, hx_jm, hz_jm, hy_im,
                               hz_im, hx_km, hy_km, srcv);
    for (int q = 0; q < npc; ++q)
      if (pk[q] == k) a.series[(int64_t)ps[q] * a.series_len + a.series_pos] = ex;
    hx_km = hx;
    hy_km = hy;
  }
}

// ---------------------------------------------------------------------------------------
// fused form: one kernel per step, step-n state in, step-n+1 state out. blockDim.x = 32.
template <typename T>
__global__ void __launch_bounds__(256) k3_fused(const Args3<T> a) {
  const int nx = a.nx, ny = a.ny;
  const double t = (double)(a.n0 + 1) * a.dt;
  const int nzc = (a.nz + a.kc - 1) / a.kc;
  if ((int)blockIdx.z >= nzc) {  // incident line, step n -> n+1 (H, then E, source, Mur ends)
    if (blockIdx.x != 0 || blockIdx.y != 0) return;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x, nt = blockDim.x * blockDim.y, L = a.inc_len;
    for (int m = tid; m < L - 1; m += nt) a.oHi[m] = fma(-a.S, a.Ei[m + 1] - a.Ei[m], a.Hi[m]);
    if (tid == 0) a.oHi[L - 1] = a.Hi[L - 1];
    __syncthreads();
    for (int m = 1 + tid; m < L - 1; m += nt) a.oEi[m] = fma(-a.S, a.oHi[m] - a.oHi[m - 1], a.Ei[m]);
    __syncthreads();
    if (tid == 0) {
      a.oEi[a.inc_src] = a.oEi[a.inc_src] + (T)pulse3(t, a.t0, a.tau, a.amp);
      a.oEi[0] = fma(a.q, a.oEi[1] - a.Ei[0], a.Ei[1]);
      a.oEi[L - 1] = fma(a.q, a.oEi[L - 2] - a.Ei[L - 1], a.Ei[L - 2]);
    }
    return;
  }
  const int lane = threadIdx.x;
  const int i = blockIdx.x * 32 + lane;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (j >= ny) return;  // whole warp
  const bool act = i < nx;
  const int im = (i > 0) ? i - 1 : (a.per ? nx - 1 : -1);
  const int jm = (j > 0) ? j - 1 : (a.per ? ny - 1 : -1);
  const int kb = blockIdx.z * a.kc, ke = min(a.nz, kb + a.kc);
  // the sheet source's value, only where this column range holds the sheet (FP64 is narrow here)
  const T srcv = (a.sheet_k >= kb && a.sheet_k < ke) ? (T)pulse3(t, a.t0, a.tau, a.amp) : T(0);
  int pk[4], ps[4];
  const int npc = act ? column_probes(a, i, j, kb, ke, pk, ps) : 0;
  T hx_km = T(0), hy_km = T(0);
  if (act && kb > 0) {
    hx_km = hx_new<true>(a, i, j, kb - 1, false);
    hy_km = hy_new<true>(a, i, j, kb - 1, false);
  }
  for (int k = kb; k < ke; ++k) {
    T hx = T(0), hy = T(0), hz = T(0);
    if (act) {
      const int64_t c = idx3(i, j, k, nx, ny);
      hx = hx_new<true>(a, i, j, k, true);
      hy = hy_new<true>(a, i, j, k, true);
      hz = hz_new<true>(a, i, j, k, true);
      a.oHx[c] = hx;
      a.oHy[c] = hy;
      a.oHz[c] = hz;
    }
    T hy_im = __shfl_up_sync(kFull, hy, 1);
    T hz_im = __shfl_up_sync(kFull, hz, 1);
    if (!act) continue;
    if (lane == 0 && im >= 0) {
      hy_im = hy_new<true>(a, im, j, k, false);
      hz_im = hz_new<true>(a, im, j, k, false);
    }
    T hx_jm = T(0), hz_jm = T(0);
    if (jm >= 0) {
      hx_jm = hx_new<true>(a, i, jm, k, false);
      hz_jm = hz_new<true>(a, i, jm, k, false);
    }
    const int64_t c = idx3(i, j, k, nx, ny);
    const T ex = e_cell<true>(a, i, j, k, __ldg(a.Ex + c), __ldg(a.Ey + c), __ldg(a.Ez + c), __ldg(a.mat + c), hx, hy,
                              hz, hx_jm, hz_jm, hy_im, hz_im, hx_km, hy_km, srcv);
    for (int q = 0; q < npc; ++q)
      if (pk[q] == k) a.series[(int64_t)ps[q] * a.series_len + a.series_pos] = ex;
    hx_km = hx;
    hy_km = hy;
  }
}

// ---------------------------------------------------------------------------------------
// staged form: the fused step with the step-n E, H and material planes brought into shared
// memory by the tensor memory accelerator, kStages planes ahead, one mbarrier per stage.
// Block = kTY compute warps (warp w owns row j0 + w, lane l owns column i0 + l) plus one
// halo warp that issues the copies and computes the new H of the j0-1 row (Hx, Hz) and of
// the i0-1 column (Hy, Hz) that the E update needs. Box of each E/H plane: x in
// [i0-4, i0+36) (16-byte aligned start), y in [j0-1, j0+kTY+1); out-of-grid parts read 0.
// Non-periodic grids with nx a multiple of 16.
#ifndef RKETD_3D_TY
#define RKETD_3D_TY 8
#endif
#ifndef RKETD_3D_STAGES
#define RKETD_3D_STAGES 4
#endif
#ifndef RKETD_3D_L2PROMO
#define RKETD_3D_L2PROMO 2  // L2 promotion of the staged copies: 0 none, 1 64 B, 2 128 B, 3 256 B
#endif
#ifndef RKETD_3D_KC_GEN
#define RKETD_3D_KC_GEN 0  // planes per boundary-tile item; 0: the context's k chunk
#endif
#ifndef RKETD_3D_MINB
#define RKETD_3D_MINB 0  // 0: resident blocks per SM that the shared memory allows (4 FP32, 2 FP64)
#endif

constexpr int kTY = RKETD_3D_TY;         // compute warps (rows) per block
constexpr int kStages = RKETD_3D_STAGES;  // planes in the copy ring (>= 3)
static_assert(kTY >= 1 && kTY <= 32 && kStages >= 3, "staged form shape");
constexpr int kBW = 40;
constexpr int kBH = kTY + 2;
constexpr int kHW = 33;  // new-H tile row: i0-1 .. i0+31
constexpr int kHH = kTY + 1;
constexpr int kWaitLimit = 1 << 20;

// Facts of one z plane for the staged form, written next to its stage by the thread that
// issues the plane's copies and read by all threads once the stage's mbarrier completes.
template <typename T>
struct PlaneS {
  T zb[2], zc[2], zk[2];  // z CPML coefficients (db, c, 1/kappa) at this plane: [0] H position z+1/2, [1] E position z
  T ei_hy, ei_hz;         // step-n incident E for the Hy and Hz corrections
  T hi_ex, hi_ez;         // step-n+1/2 incident H for the Ex and Ez corrections
  int zz;                 // compact z zone
  unsigned f;             // kP* flags
};
enum : unsigned {
  kPVk = 1u, kPZin = 2u, kPZlast = 4u, kPFzH = 8u, kPFzE = 16u, kPTfHz = 32u, kPTfEz = 64u, kPSheet = 128u,
  kPHyP = 256u, kPHyM = 512u, kPExP = 1024u, kPExM = 2048u, kPLean = 4096u
};
constexpr int kXN = 34;  // x coefficient entries of a tile: i0-1 .. i0+32
// work kinds of the staged form: general (boundary tiles), interior tiles in the middle z range
// (no CPML memory at all), interior tiles in the two z CPML slabs
enum { kModeGen = 0, kModeMid = 1, kModeZc = 2, kModeGenX = 3, kModeGenY = 4, kModeGenF = 5 };
// what each kind of work item can meet: the x / y CPML with the x / y domain edges, the z CPML,
// and the TF/SF x/y faces (kModeGen*: boundary tiles split by the CPML axes they reach; kModeGenF
// tiles reach only TF/SF x/y faces)
template <int MODE>
struct Kind3 {
  static constexpr bool interior = MODE == kModeMid || MODE == kModeZc;
  static constexpr bool xc = MODE == kModeGen || MODE == kModeGenX;
  static constexpr bool yc = MODE == kModeGen || MODE == kModeGenY;
  static constexpr bool zc = MODE != kModeMid;
};

template <typename T>
struct Stage3 {
  static constexpr int box = ((kBW * kBH * (int)sizeof(T) + 127) / 128) * 128 / (int)sizeof(T);  // padded to 128 B
  static constexpr int mat_bytes = 32 * kTY;
  static constexpr int bytes = 6 * box * (int)sizeof(T) + mat_bytes;  // one plane of Ex..Hz + material
  static constexpr int tx = 6 * kBW * kBH * (int)sizeof(T) + mat_bytes;  // bytes the copies deliver
  static constexpr int hn = ((kHW * kHH + 31) / 32) * 32;
  static constexpr int off_hn = kStages * bytes;
  static constexpr int off_bar = off_hn + 2 * 3 * hn * (int)sizeof(T);
  static constexpr int off_pl = ((off_bar + kStages * 8 + 15) / 16) * 16;
  static constexpr int pl_bytes = ((int)sizeof(PlaneS<T>) + 15) / 16 * 16;
  static constexpr int off_xy = off_pl + kStages * pl_bytes;
  // per-tile CPML coefficients, 8 values per x (kXN) and y (kTY+1) position:
  // H: db, c, 1/kappa, flag; E: db, c, 1/kappa, flag
  static constexpr int smem = off_xy + (kXN + kTY + 1) * 8 * (int)sizeof(T);
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// bounded wait for the phase with the given parity, at most `limit` polls; false if it did not
// complete
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int limit = kWaitLimit) {
  const uint32_t addr = smem_u32(bar);
  for (int it = 0; it < limit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void tma_load3(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
          smem_u32(dst)),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

// untiled bulk copy of `bytes` (a multiple of 16; both addresses 16-byte aligned) from global
// to shared memory, completing on the mbarrier
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"((uint64_t)src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

template <typename T>
struct Maps3 {
  CUtensorMap f[6];  // Ex, Ey, Ez, Hx, Hy, Hz of the step-n set
  CUtensorMap mat;
};

// Per-cell facts of the staged form that depend on (i, j) only, worked out once per thread.
struct Col3 {
  bool vi, vj;               // i+1 < nx, j+1 < ny
  bool fxH, fyH, fxE, fyE;   // x / y CPML memory active (H positions i+1/2, j+1/2; E positions i, j)
  bool ex_xy, ey_xy, ez_xy;  // E component updated, as far as x and y decide
  bool tf_xy;                // i in [i0, i1-1] and j in [j0, j1] (TF/SF Hy and Ex faces)
  bool tf_hz_i;              // i in [i0, i1-1]
  int sg_hz;                 // -1 at j = j0-1, +1 at j = j1, else 0 (Hz faces)
  int sg_ez;                 // -1 at i = i0, +1 at i = i1 when j in [j0, j1], else 0 (Ez faces)
  int zx, zy;                // compact zone indices
  // 32-bit offsets of the cell's CPML memories in plane 0 (x-derivative [k][j][Z], y-derivative
  // [k][Z][i]) and in zone 0 (z-derivative [Z][j][i]); a plane or zone adds a fixed stride. The
  // staged form is used only where every memory array has fewer than 2^31 entries.
  int xo, yo, zo;
};

template <typename T>
__device__ __forceinline__ Col3 col3(const Args3<T>& a, int i, int j) {
  Col3 c;
  const int nx = a.nx, ny = a.ny;
  c.vi = i + 1 < nx;
  c.vj = j + 1 < ny;
  c.zx = zone(i, nx, a.np);
  c.zy = zone(j, ny, a.np);
  c.fxH = c.zx >= 0 && tb(a, 0, 1)[3 * a.nmax + i] != T(0);
  c.fyH = c.zy >= 0 && tb(a, 1, 1)[3 * a.nmax + j] != T(0);
  c.fxE = c.zx >= 0 && tb(a, 0, 0)[3 * a.nmax + i] != T(0);
  c.fyE = c.zy >= 0 && tb(a, 1, 0)[3 * a.nmax + j] != T(0);
  const bool xin = i > 0 && i < nx - 1, yin = j > 0 && j < ny - 1;
  c.ex_xy = i < nx - 1 && yin;
  c.ey_xy = j < ny - 1 && xin;
  c.ez_xy = xin && yin;
  const bool ti = a.tfsf && i >= a.i0 && i <= a.i1 - 1;
  c.tf_xy = ti && j >= a.j0 && j <= a.j1;
  c.tf_hz_i = ti;
  c.sg_hz = (j == a.j0 - 1) ? -1 : (j == a.j1 ? 1 : 0);
  c.sg_ez = (a.tfsf && j >= a.j0 && j <= a.j1) ? (i == a.i0 ? -1 : (i == a.i1 ? 1 : 0)) : 0;
  c.xo = j * a.Z + c.zx;
  c.yo = c.zy * nx + i;
  c.zo = j * nx + i;
  return c;
}

template <typename T>
__device__ __forceinline__ void plane_facts(const Args3<T>& a, int z, PlaneS<T>* p) {
  unsigned f = 0;
  p->zz = -1;
  for (int h = 0; h < 2; ++h) p->zb[h] = p->zc[h] = p->zk[h] = T(0);
  p->ei_hy = p->ei_hz = p->hi_ex = p->hi_ez = T(0);
  if (z < 0 || z >= a.nz) {
    p->f = 0;
    return;
  }
  const int nz = a.nz, np = a.np;
  if (z + 1 < nz) f |= kPVk;
  if (z > 0 && z < nz - 1) f |= kPZin;
  if (z < nz - 1) f |= kPZlast;
  const int zz = zone(z, nz, np);
  p->zz = zz;
  if (zz >= 0)
    for (int h = 0; h < 2; ++h) {
      const T* t = tb(a, 2, h == 0 ? 1 : 0);
      if (t[3 * a.nmax + z] != T(0)) {
        f |= h == 0 ? kPFzH : kPFzE;
        p->zb[h] = t[z];
        p->zc[h] = t[a.nmax + z];
        p->zk[h] = t[2 * a.nmax + z];
      }
    }
  if (a.tfsf) {
    if (z == a.k0 - 1) {
      f |= kPHyP;
      p->ei_hy = a.Ei[a.k0 + a.inc_off];
    } else if (z == a.k1) {
      f |= kPHyM;
      p->ei_hy = a.Ei[a.k1 + a.inc_off];
    }
    if (z >= a.k0 && z <= a.k1) {
      f |= kPTfHz;
      p->ei_hz = a.Ei[z + a.inc_off];
    }
    if (z == a.k0) {
      f |= kPExP;
      p->hi_ex = hinc<true>(a, a.k0 - 1 + a.inc_off);
    } else if (z == a.k1) {
      f |= kPExM;
      p->hi_ex = hinc<true>(a, a.k1 + a.inc_off);
    }
    if (z >= a.k0 && z <= a.k1 - 1) {
      f |= kPTfEz;
      p->hi_ez = hinc<true>(a, z + a.inc_off);
    }
  }
  if (z == a.sheet_k) f |= kPSheet;
  if (!(f & (kPFzH | kPFzE)) && (f & kPVk) && (f & kPZin) && z != a.sheet_k &&
      !(a.tfsf && (z == a.k0 - 1 || z == a.k0 || z == a.k1)))
    f |= kPLean;
  p->f = f;
}

// A plane's facts as the update functions see them: the flags in a register (tested many times
// per cell), the rest read from the plane's shared-memory record where a flag asks for it.
template <typename T>
struct PlaneR {
  unsigned f;
  const PlaneS<T>* s;
};

// CPML stretch with the coefficients (db = b - 1, c, 1/kappa) and the old memory value given
// (stretch() once its flag is known to be set)
template <typename T>
__device__ __forceinline__ T stretch_c(T db, T cc, T ki, T dv, T psi, T* pout) {
  const T p = fma(db, psi, fma(cc, dv, psi));
  if (pout) *pout = p;
  return fma(dv, ki, p);
}

// The CPML memories one cell reads in one plane, loaded at the top of the plane's iteration so
// that their latency overlaps the copy wait and the H phase: H side in the order of psiH, E side
// in the order of psiE (slots that the cell does not use are left alone).
template <typename T>
struct Pre3 {
  T h[6], e[6];
  int ox, oy, oz;  // the cell's offsets into the x-, y- and z-derivative memories in this plane
};

template <bool XC, bool YC, bool HSIDE, bool ESIDE, typename T>
__device__ __forceinline__ void prefetch3(const Args3<T>& a, const Col3& c, int z, int zz, unsigned hmask, Pre3<T>& v) {
  v.oz = zz * (a.nx * a.ny) + c.zo;
  if constexpr (XC) v.ox = z * (a.ny * a.Z) + c.xo;
  if constexpr (YC) v.oy = z * (a.Z * a.nx) + c.yo;
  if (zz >= 0) {
    const int o = v.oz;
    if (HSIDE && (hmask & 2u)) v.h[1] = __ldg(a.psiH[1] + o);
    if (HSIDE && (hmask & 4u)) v.h[2] = __ldg(a.psiH[2] + o);
    if constexpr (ESIDE) {
      if (hmask & 64u) {
        v.e[1] = a.psiE[1][o];
        v.e[2] = a.psiE[2][o];
      }
    }
  }
  if constexpr (XC) {
    if (c.zx >= 0) {
      const int o = v.ox;
      if (HSIDE && (hmask & 8u)) v.h[3] = __ldg(a.psiH[3] + o);
      if (HSIDE && (hmask & 16u)) v.h[4] = __ldg(a.psiH[4] + o);
      if constexpr (ESIDE) {
        v.e[3] = a.psiE[3][o];
        v.e[4] = a.psiE[4][o];
      }
    }
  }
  if constexpr (YC) {
    if (c.zy >= 0) {
      const int o = v.oy;
      if (HSIDE && (hmask & 1u)) v.h[0] = __ldg(a.psiH[0] + o);
      if (HSIDE && (hmask & 32u)) v.h[5] = __ldg(a.psiH[5] + o);
      if constexpr (ESIDE) {
        v.e[0] = a.psiE[0][o];
        v.e[5] = a.psiE[5][o];
      }
    }
  }
}

#ifndef RKETD_3D_PSI_AHEAD
#define RKETD_3D_PSI_AHEAD 1
#endif
// L2 prefetch of the CPML memories (E side and the step-n H side) of a compute thread's own cell
// in plane z, issued RKETD_3D_PSI_AHEAD planes before their loads: the loads then find them in
// L2, without holding registers or shared memory meanwhile.
template <bool XC, bool YC, typename T>
__device__ __forceinline__ void l2_prefetch_psi(const Args3<T>& a, const Col3& c, int z) {
  const int zz = zone(z, a.nz, a.np);
  if (zz >= 0) {
    const int oz = zz * (a.nx * a.ny) + c.zo;
    asm volatile("prefetch.global.L2 [%0];" ::"l"(a.psiE[1] + oz));
    asm volatile("prefetch.global.L2 [%0];" ::"l"(a.psiE[2] + oz));
    asm volatile("prefetch.global.L2 [%0];" ::"l"(a.psiH[1] + oz));
    asm volatile("prefetch.global.L2 [%0];" ::"l"(a.psiH[2] + oz));
  }
  if constexpr (XC) {
    if (c.zx >= 0) {
      const int ox = z * (a.ny * a.Z) + c.xo;
      asm volatile("prefetch.global.L2 [%0];" ::"l"(a.psiE[3] + ox));
      asm volatile("prefetch.global.L2 [%0];" ::"l"(a.psiE[4] + ox));
      asm volatile("prefetch.global.L2 [%0];" ::"l"(a.psiH[3] + ox));
      asm volatile("prefetch.global.L2 [%0];" ::"l"(a.psiH[4] + ox));
    }
  }
  if constexpr (YC) {
    if (c.zy >= 0) {
      const int oy = z * (a.Z * a.nx) + c.yo;
      asm volatile("prefetch.global.L2 [%0];" ::"l"(a.psiE[0] + oy));
      asm volatile("prefetch.global.L2 [%0];" ::"l"(a.psiE[5] + oy));
      asm volatile("prefetch.global.L2 [%0];" ::"l"(a.psiH[0] + oy));
      asm volatile("prefetch.global.L2 [%0];" ::"l"(a.psiH[5] + oy));
    }
  }
}

// L2 prefetch of the step-n H-side CPML memories of a halo cell in plane z (mask bits as prefetch3)
template <bool XC, bool YC, typename T>
__device__ __forceinline__ void l2_prefetch_halo(const Args3<T>& a, const Col3& c, int z, unsigned hmask) {
  const int zz = zone(z, a.nz, a.np);
  if (zz >= 0) {
    const int oz = zz * (a.nx * a.ny) + c.zo;
    if (hmask & 2u) asm volatile("prefetch.global.L2 [%0];" ::"l"(a.psiH[1] + oz));
    if (hmask & 4u) asm volatile("prefetch.global.L2 [%0];" ::"l"(a.psiH[2] + oz));
  }
  if constexpr (XC) {
    if (c.zx >= 0) {
      const int ox = z * (a.ny * a.Z) + c.xo;
      if (hmask & 8u) asm volatile("prefetch.global.L2 [%0];" ::"l"(a.psiH[3] + ox));
      if (hmask & 16u) asm volatile("prefetch.global.L2 [%0];" ::"l"(a.psiH[4] + ox));
    }
  }
  if constexpr (YC) {
    if (c.zy >= 0) {
      const int oy = z * (a.Z * a.nx) + c.yo;
      if (hmask & 1u) asm volatile("prefetch.global.L2 [%0];" ::"l"(a.psiH[0] + oy));
      if (hmask & 32u) asm volatile("prefetch.global.L2 [%0];" ::"l"(a.psiH[5] + oy));
    }
  }
}

// The staged form's updates of one cell: the operations of hx_core .. e_cell for non-periodic
// grids, with the per-cell facts (c), the x and y coefficient rows of the tile (X, Y: H b, c,
// 1/kappa, flag, then E) and the plane's facts (p). The kind of work item (Kind3) leaves out at
// compile time the terms its cells cannot meet: the x or y CPML with the x or y domain edges, the
// z CPML, the TF/SF x/y faces.
template <int MODE, typename T>
__device__ __forceinline__ T hx_s(const Args3<T>& a, const Col3& c, const T* Y, const PlaneR<T> p, const Pre3<T>& v,
                                  int i, int j, int k, T h, T ez_jp, T ez, T ey_kp, T ey, bool own) {
  using K = Kind3<MODE>;
  if (!(p.f & kPVk)) return h;
  if constexpr (K::yc)
    if (!c.vj) return h;
  T cy = ez_jp - ez;
  T cz = ey_kp - ey;
  if constexpr (K::yc)
    if (c.fyH) {
      const int o = v.oy;
      cy = stretch_c(Y[0], Y[1], Y[2], cy, v.h[0], own ? a.opsiH[0] + o : nullptr);
    }
  if (K::zc && (p.f & kPFzH)) {
    const int o = v.oz;
    cz = stretch_c(p.s->zb[0], p.s->zc[0], p.s->zk[0], cz, v.h[1], own ? a.opsiH[1] + o : nullptr);
  }
  return fma(-a.S, cy - cz, h);
}

template <int MODE, typename T>
__device__ __forceinline__ T hy_s(const Args3<T>& a, const Col3& c, const T* X, const PlaneR<T> p, const Pre3<T>& v,
                                  int i, int j, int k, T h, T ex_kp, T ex, T ez_ip, T ez, bool own) {
  using K = Kind3<MODE>;
  if (!(p.f & kPVk)) return h;
  if constexpr (K::xc)
    if (!c.vi) return h;
  T cz = ex_kp - ex;
  T cx = ez_ip - ez;
  if (K::zc && (p.f & kPFzH)) {
    const int o = v.oz;
    cz = stretch_c(p.s->zb[0], p.s->zc[0], p.s->zk[0], cz, v.h[2], own ? a.opsiH[2] + o : nullptr);
  }
  if constexpr (K::xc)
    if (c.fxH) {
      const int o = v.ox;
      cx = stretch_c(X[0], X[1], X[2], cx, v.h[3], own ? a.opsiH[3] + o : nullptr);
    }
  T r = fma(-a.S, cz - cx, h);
  if (c.tf_xy && (p.f & (kPHyP | kPHyM))) r = fma((p.f & kPHyP) ? a.S : -a.S, p.s->ei_hy, r);
  return r;
}

template <int MODE, typename T>
__device__ __forceinline__ T hz_s(const Args3<T>& a, const Col3& c, const T* X, const T* Y, const PlaneR<T> p,
                                  const Pre3<T>& v, int i, int j, int k, T h, T ey_ip, T ey, T ex_jp, T ex, bool own) {
  using K = Kind3<MODE>;
  if constexpr (K::interior) {
    return fma(-a.S, (ey_ip - ey) - (ex_jp - ex), h);
  } else {
    if constexpr (K::xc)
      if (!c.vi) return h;
    if constexpr (K::yc)
      if (!c.vj) return h;
    T cx = ey_ip - ey;
    T cy = ex_jp - ex;
    if constexpr (K::xc)
      if (c.fxH) {
        const int o = v.ox;
        cx = stretch_c(X[0], X[1], X[2], cx, v.h[4], own ? a.opsiH[4] + o : nullptr);
      }
    if constexpr (K::yc)
      if (c.fyH) {
        const int o = v.oy;
        cy = stretch_c(Y[0], Y[1], Y[2], cy, v.h[5], own ? a.opsiH[5] + o : nullptr);
      }
    T r = fma(-a.S, cx - cy, h);
    if (c.tf_hz_i && c.sg_hz && (p.f & kPTfHz)) r = fma(c.sg_hz > 0 ? a.S : -a.S, p.s->ei_hz, r);
    return r;
  }
}

// E and J of one cell; returns the new Ex. The CPML memories of E are updated in place.
template <int MODE, typename T>
__device__ __forceinline__ T e_s(const Args3<T>& a, const Col3& c, const T* X, const T* Y, const PlaneR<T> p,
                                 const Pre3<T>& v, int i, int j, int k, int64_t ci, T ex, T ey, T ez, int mb, T hx, T hy,
                                 T hz, T hx_jm, T hz_jm, T hy_im, T hz_im, T hx_km, T hy_km, T srcv) {
  using K = Kind3<MODE>;
  const bool zin = p.f & kPZin;
  constexpr bool edges = K::xc || K::yc;  // only then can x or y decide that a component is not updated
  if (zin && (!edges || c.ex_xy)) {
    T cy = hz - hz_jm, cz = hy - hy_km;
    if constexpr (K::yc)
      if (c.fyE) {
        T* q = a.psiE[0] + v.oy;
        cy = stretch_c<T>(Y[4], Y[5], Y[6], cy, v.e[0], q);
      }
    if (K::zc && (p.f & kPFzE)) {
      T* q = a.psiE[1] + v.oz;
      cz = stretch_c<T>(p.s->zb[1], p.s->zc[1], p.s->zk[1], cz, v.e[1], q);
    }
    ex = e_update(a.m, mb & 3, ex, cy - cz, a.Jx + ci);
    if (c.tf_xy && (p.f & (kPExP | kPExM))) ex = fma((p.f & kPExP) ? a.S : -a.S, p.s->hi_ex, ex);
  }
  if (p.f & kPSheet) ex = ex + srcv;
  a.oEx[ci] = ex;
  if (zin && (!edges || c.ey_xy)) {
    T cz = hx - hx_km, cx = hz - hz_im;
    if (K::zc && (p.f & kPFzE)) {
      T* q = a.psiE[2] + v.oz;
      cz = stretch_c<T>(p.s->zb[1], p.s->zc[1], p.s->zk[1], cz, v.e[2], q);
    }
    if constexpr (K::xc)
      if (c.fxE) {
        T* q = a.psiE[3] + v.ox;
        cx = stretch_c<T>(X[4], X[5], X[6], cx, v.e[3], q);
      }
    ey = e_update(a.m, (mb >> 2) & 3, ey, cz - cx, a.Jy + ci);
  }
  a.oEy[ci] = ey;
  if ((p.f & kPZlast) && (!edges || c.ez_xy)) {
    T cx = hy - hy_im, cy = hx - hx_jm;
    if constexpr (K::xc)
      if (c.fxE) {
        T* q = a.psiE[4] + v.ox;
        cx = stretch_c<T>(X[4], X[5], X[6], cx, v.e[4], q);
      }
    if constexpr (K::yc)
      if (c.fyE) {
        T* q = a.psiE[5] + v.oy;
        cy = stretch_c<T>(Y[4], Y[5], Y[6], cy, v.e[5], q);
      }
    ez = e_update(a.m, (mb >> 4) & 3, ez, cx - cy, a.Jz + ci);
    if constexpr (!K::interior)
      if (c.sg_ez && (p.f & kPTfEz)) ez = fma(c.sg_ez < 0 ? -a.S : a.S, p.s->hi_ez, ez);
  }
  a.oEz[ci] = ez;
  return ex;
}

// Interior-column tile: the tile with its i0-1 / j0-1 halo clear of the x/y CPML and of the
// TF/SF x and y faces (the host sorts tiles with the same test).
__host__ __device__ __forceinline__ bool interior_tile(int i0, int j0, int nx, int ny, int np, int tfsf, const int* box) {
  if (!(i0 - 1 >= np + 1 && i0 + 31 <= nx - np - 2 && j0 - 1 >= np + 1 && j0 + kTY - 1 <= ny - np - 2)) return false;
  if (tfsf) {
    const int jl = j0 - 1, jh = j0 + kTY - 1;
    if ((box[2] - 1 >= jl && box[2] - 1 <= jh) || (box[3] >= jl && box[3] <= jh)) return false;
    if ((box[0] >= i0 && box[0] <= i0 + 31) || (box[1] >= i0 && box[1] <= i0 + 31)) return false;
  }
  return true;
}

// One launch handles the work items of one kind: an item is a tile origin (i0, j0) and a range
// of planes [kb, ke). kModeGen, kModeGenX, kModeGenY, kModeGenF: boundary tiles (reaching the x
// and y CPML, the x CPML only, the y CPML only, only TF/SF x/y faces), general path. kModeMid:
// interior tiles in the middle z range, bare updates. kModeZc: interior tiles in the z CPML slabs
// and at the TF/SF z faces and the sheet. With TF/SF the kModeGen launch carries one more block
// (blockIdx.x == n_items) that advances the incident line.
// Resident blocks per SM the register budget is set for: the shared memory allows 4 (FP32) or
// 2 (FP64). Every FP32 kind is held to 4, although the boundary kinds then spill a few bytes:
// they are latency-bound, and the fourth block gains more than the spills cost (76.7 -> 78.5
// Gcell/s on the 512^3 sphere). The x-and-y kind, whose few items cannot fill the GPU anyway
// and which would spill most, keeps 3.
template <typename T, int MODE>
constexpr int staged_min_blocks() {
  return RKETD_3D_MINB ? RKETD_3D_MINB : (sizeof(T) == 4 ? (MODE == kModeGen ? 3 : 4) : 2);
}

template <typename T, int MODE>
__global__ void __launch_bounds__(32 * (kTY + 1), (staged_min_blocks<T, MODE>()))
    k3_staged(const Args3<T> a, const __grid_constant__ Maps3<T> mp, const int4* __restrict__ items, int n_items,
              int* err) {
  using K = Kind3<MODE>;
  constexpr bool INTERIOR = K::interior;
  using St = Stage3<T>;
  extern __shared__ __align__(128) unsigned char sm[];
  const int nx = a.nx, ny = a.ny;
  const int lane = threadIdx.x, w = threadIdx.y;
  const int tid = w * 32 + lane, nt = 32 * (kTY + 1);
  const double t = (double)(a.n0 + 1) * a.dt;
  if ((int)blockIdx.x >= n_items) {  // incident line, step n -> n+1 (as the fused form)
    const int L = a.inc_len;
    for (int m = tid; m < L - 1; m += nt) a.oHi[m] = fma(-a.S, a.Ei[m + 1] - a.Ei[m], a.Hi[m]);
    if (tid == 0) a.oHi[L - 1] = a.Hi[L - 1];
    __syncthreads();
    for (int m = 1 + tid; m < L - 1; m += nt) a.oEi[m] = fma(-a.S, a.oHi[m] - a.oHi[m - 1], a.Ei[m]);
    __syncthreads();
    if (tid == 0) {
      a.oEi[a.inc_src] = a.oEi[a.inc_src] + (T)pulse3(t, a.t0, a.tau, a.amp);
      a.oEi[0] = fma(a.q, a.oEi[1] - a.Ei[0], a.Ei[1]);
      a.oEi[L - 1] = fma(a.q, a.oEi[L - 2] - a.Ei[L - 1], a.Ei[L - 2]);
    }
    return;
  }
  const int4 item = items[blockIdx.x];
  const int i0 = item.x, j0 = item.y;
  const int kb = item.z, ke = item.w;
  const int NP = ke - kb + 2;  // planes kb-1 .. ke
  T* hn = (T*)(sm + St::off_hn);
  uint64_t* bar = (uint64_t*)(sm + St::off_bar);
  auto facts = [&](int q) -> PlaneS<T>* { return (PlaneS<T>*)(sm + St::off_pl + (q % kStages) * St::pl_bytes); };
  T* xs = (T*)(sm + St::off_xy);  // [kXN][8]
  T* ys = xs + kXN * 8;           // [kTY+1][8]
  auto plane = [&](int q) { return (const T*)(sm + (q % kStages) * St::bytes); };
  const bool producer = (w == kTY && lane == 0);
  auto issue = [&](int q) {
    const int s = q % kStages;
    unsigned char* dst = sm + s * St::bytes;
    const int z = kb - 1 + q;
    // the plane's facts (computed for this step by k3_facts) arrive with its copies
    mbar_expect_tx(&bar[s], St::tx + (MODE != kModeMid ? St::pl_bytes : 0));
    if constexpr (MODE != kModeMid) bulk_load(facts(q), a.ftab + (size_t)(z + 1) * St::pl_bytes, St::pl_bytes, &bar[s]);
    for (int f = 0; f < 6; ++f) tma_load3(dst + f * St::box * sizeof(T), &mp.f[f], i0 - 4, j0 - 1, z, &bar[s]);
    tma_load3(dst + 6 * St::box * sizeof(T), &mp.mat, i0, j0, z, &bar[s]);
  };
  if (producer) {
    for (int s = 0; s < kStages; ++s) mbar_init(&bar[s], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if constexpr (!INTERIOR) {
    // x coefficient rows for i0-1 .. i0+32 and y rows for j0-1 .. j0+kTY-1
    for (int e = tid; e < kXN + kTY + 1; e += nt) {
      const bool isx = e < kXN;
      const int ax = isx ? 0 : 1;
      const int n = isx ? i0 - 1 + e : j0 - 1 + (e - kXN);
      const int N = isx ? nx : ny;
      T* row = isx ? xs + 8 * e : ys + 8 * (e - kXN);
      for (int h = 0; h < 2; ++h) {
        const T* tt = tb(a, ax, h == 0 ? 1 : 0);
        const bool in = n >= 0 && n < N;
        row[4 * h + 0] = in ? tt[n] : T(0);
        row[4 * h + 1] = in ? tt[a.nmax + n] : T(0);
        row[4 * h + 2] = in ? tt[2 * a.nmax + n] : T(1);
        row[4 * h + 3] = in ? tt[3 * a.nmax + n] : T(0);
      }
    }
  }
  __syncthreads();
  int issued = 0;  // planes whose copies the producer has issued
  if (producer)
    for (; issued < kStages && issued < NP; ++issued) issue(issued);
  const int i = i0 + lane, j = j0 + w;
  const bool act = w < kTY && i < nx && j < ny;
  // the sheet source's value, only in items that hold the sheet plane (block-uniform): one FP64
  // evaluation per warp, broadcast from lane 0 (the FP64 pipe is narrow on this part)
  T srcv = T(0);
  if (a.sheet_k >= kb && a.sheet_k < ke) {
    double v = 0.0;
    if (lane == 0) v = pulse3(t, a.t0, a.tau, a.amp);
    srcv = (T)__shfl_sync(0xffffffffu, v, 0);
  }
  int pk[4], ps[4];
  const int npc = act ? column_probes(a, i, j, kb, ke, pk, ps) : 0;
  constexpr int EX = 0, EY = St::box, EZ = 2 * St::box, HX = 3 * St::box, HY = 4 * St::box, HZ = 5 * St::box;
  const int64_t nxy = (int64_t)nx * ny;
  const int64_t c0 = (int64_t)j * nx + i;
  // per-cell facts: own cell (compute warps) or j0-1 row cell (halo warp); i0-1 column cell
  const Col3 cc = col3(a, w < kTY ? min(i, nx - 1) : min(i0 + lane, nx - 1), w < kTY ? min(j, ny - 1) : max(j0 - 1, 0));
  const Col3 cc2 = col3(a, max(i0 - 1, 0), min(j0 + (lane < kTY ? lane : 0), ny - 1));
  // coefficient rows: own cell (x lane+1, y w+1); halo row cell (x lane+1, y 0); column cell (x 0, y lane+1)
  const T* Xo = xs + 8 * (lane + 1);
  const T* Yo = ys + 8 * (w < kTY ? w + 1 : 0);
  const T* Xc = xs;
  const T* Yc = ys + 8 * (lane < kTY ? lane + 1 : 0);
  T hx_km = T(0), hy_km = T(0);
  bool fail = false, bad = false;  // fail: this thread's wait gave up; bad: some thread's did
  for (int q = 0; q + 1 < NP; ++q) {
    const int z = kb - 1 + q;
    // CPML memories of this plane (kinds other than the middle one), loaded before the copy wait:
    // own cell (compute warps), or the halo-row (pv) and halo-column (pc) cells (halo warp).
    // Loading them a plane ahead held more registers live and measured slower.
    Pre3<T> pv, pc;
    if constexpr (MODE != kModeMid) {
      const int zz = z >= 0 ? zone(z, a.nz, a.np) : -1;
      if (z >= 0) {
        if (act) {
          prefetch3<K::xc, K::yc, true, true>(a, cc, z, zz, 0x7fu, pv);
          if (RKETD_3D_PSI_AHEAD > 0 && z + RKETD_3D_PSI_AHEAD < ke)
            l2_prefetch_psi<K::xc, K::yc>(a, cc, z + RKETD_3D_PSI_AHEAD);
        }
        else if (w == kTY && q > 0) {
          const bool nxt = RKETD_3D_PSI_AHEAD > 0 && z + RKETD_3D_PSI_AHEAD < ke;
          if (j0 - 1 >= 0 && i0 + lane < nx) {
            prefetch3<K::xc, K::yc, true, false>(a, cc, z, zz, 0x33u, pv);
            if (nxt) l2_prefetch_halo<K::xc, K::yc>(a, cc, z + RKETD_3D_PSI_AHEAD, 0x33u);
          }
          if (lane < kTY && i0 > 0 && j0 + lane < ny) {
            prefetch3<K::xc, K::yc, true, false>(a, cc2, z, zz, 0x3cu, pc);
            if (nxt) l2_prefetch_halo<K::xc, K::yc>(a, cc2, z + RKETD_3D_PSI_AHEAD, 0x3cu);
          }
        }
      }
    }
    if (q == 0) fail |= !mbar_wait(&bar[0], 0, a.wait_limit);
    fail |= !mbar_wait(&bar[(q + 1) % kStages], ((q + 1) / kStages) & 1, a.wait_limit);
    const T* P0 = plane(q);
    const T* P1 = plane(q + 1);
    const PlaneR<T> pf{facts(q)->f, facts(q)};
    T* H0 = hn + (q & 1) * 3 * St::hn;  // new Hx, Hy, Hz of plane z on the [i0-1, i0+32) x [j0-1, j0+kTY) tile
    T hx = T(0), hy = T(0), hz = T(0);
    // lean plane: interior-column tile and z clear of the z CPML, the TF/SF z faces and the
    // sheet: the bare Eq. 14 / Eq. 13 / Eq. 11 arithmetic (decided uniformly per block)
    constexpr bool lean = MODE == kModeMid;  // every plane of a middle item is a bare update
    const bool own = q > 0;
    if (z >= 0 && !fail) {
      if (act) {
        const int o = (w + 1) * kBW + lane + 4;
        if (lean) {
          hx = fma(-a.S, (P0[EZ + o + kBW] - P0[EZ + o]) - (P1[EY + o] - P0[EY + o]), P0[HX + o]);
          hy = fma(-a.S, (P1[EX + o] - P0[EX + o]) - (P0[EZ + o + 1] - P0[EZ + o]), P0[HY + o]);
        } else {
          hx = hx_s<MODE>(a, cc, Yo, pf, pv, i, j, z, P0[HX + o], P0[EZ + o + kBW], P0[EZ + o], P1[EY + o],
                              P0[EY + o], own);
          hy = hy_s<MODE>(a, cc, Xo, pf, pv, i, j, z, P0[HY + o], P1[EX + o], P0[EX + o], P0[EZ + o + 1],
                              P0[EZ + o], own);
        }
        hz = hz_s<MODE>(a, cc, Xo, Yo, pf, pv, i, j, z, P0[HZ + o], P0[EY + o + 1], P0[EY + o], P0[EX + o + kBW],
                            P0[EX + o], own);
        if (own) {
          const int64_t c = c0 + (int64_t)z * nxy;
          a.oHx[c] = hx;
          a.oHy[c] = hy;
          a.oHz[c] = hz;
          const int h = (w + 1) * kHW + lane + 1;
          H0[h] = hx;
          H0[St::hn + h] = hy;
          H0[2 * St::hn + h] = hz;
        }
      } else if (w == kTY && own) {
        const int ih = i0 + lane, jh = j0 - 1;  // row j0-1: Hx, Hz
        const int jc = j0 + lane;               // column i0-1 (lanes < kTY): Hy, Hz
        const int o = lane + 4, oc = (lane + 1) * kBW + 3, hc = (lane + 1) * kHW;
        if (jh >= 0 && ih < nx) {
          H0[lane + 1] = lean ? fma(-a.S, (P0[EZ + o + kBW] - P0[EZ + o]) - (P1[EY + o] - P0[EY + o]), P0[HX + o])
                              : hx_s<MODE>(a, cc, ys, pf, pv, ih, jh, z, P0[HX + o], P0[EZ + o + kBW], P0[EZ + o],
                                               P1[EY + o], P0[EY + o], false);
          H0[2 * St::hn + lane + 1] = hz_s<MODE>(a, cc, Xo, ys, pf, pv, ih, jh, z, P0[HZ + o], P0[EY + o + 1],
                                                     P0[EY + o], P0[EX + o + kBW], P0[EX + o], false);
        }
        if (lane < kTY && i0 > 0 && jc < ny) {
          H0[St::hn + hc] = lean ? fma(-a.S, (P1[EX + oc] - P0[EX + oc]) - (P0[EZ + oc + 1] - P0[EZ + oc]),
                                       P0[HY + oc])
                                 : hy_s<MODE>(a, cc2, Xc, pf, pc, i0 - 1, jc, z, P0[HY + oc], P1[EX + oc],
                                                  P0[EX + oc], P0[EZ + oc + 1], P0[EZ + oc], false);
          H0[2 * St::hn + hc] = hz_s<MODE>(a, cc2, Xc, Yc, pf, pc, i0 - 1, jc, z, P0[HZ + oc], P0[EY + oc + 1],
                                               P0[EY + oc], P0[EX + oc + kBW], P0[EX + oc], false);
        }
      }
    }
    if (__syncthreads_or(fail)) {
      bad = true;
      break;
    }
    // every thread is past plane q-1: its stage takes plane q-1+kStages
    if (producer && q >= 1 && issued < NP) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(issued);
      ++issued;
    }
    if (act && z >= 0 && own) {
      const int o = (w + 1) * kBW + lane + 4;
      const int h = (w + 1) * kHW + lane + 1;
      const unsigned char* mt = sm + (q % kStages) * St::bytes + 6 * St::box * sizeof(T);
      const int mb = mt[w * 32 + lane];
      const int64_t c = c0 + (int64_t)z * nxy;
      const T hx_jm = H0[h - kHW], hz_jm = H0[2 * St::hn + h - kHW];
      const T hy_im = H0[St::hn + h - 1], hz_im = H0[2 * St::hn + h - 1];
      T ex;
      if (lean) {
        ex = e_update(a.m, mb & 3, P0[EX + o], (hz - hz_jm) - (hy - hy_km), a.Jx + c);
        a.oEx[c] = ex;
        a.oEy[c] = e_update(a.m, (mb >> 2) & 3, P0[EY + o], (hx - hx_km) - (hz - hz_im), a.Jy + c);
        a.oEz[c] = e_update(a.m, (mb >> 4) & 3, P0[EZ + o], (hy - hy_im) - (hx - hx_jm), a.Jz + c);
      } else {
        ex = e_s<MODE>(a, cc, Xo, Yo, pf, pv, i, j, z, c, P0[EX + o], P0[EY + o], P0[EZ + o], mb, hx, hy, hz, hx_jm,
                           hz_jm, hy_im, hz_im, hx_km, hy_km, srcv);
      }
      for (int r = 0; r < npc; ++r)
        if (pk[r] == z) a.series[(int64_t)ps[r] * a.series_len + a.series_pos] = ex;
    }
    hx_km = hx;
    hy_km = hy;
  }
  if (bad && producer) {
    // report, and let the copies still in flight land before the block's memory is released
    // (these drain waits keep the full limit whatever the compute-path limit is)
    atomicExch(err, 1);
    for (int q = issued > kStages ? issued - kStages : 0; q < issued; ++q)
      mbar_wait(&bar[q % kStages], (q / kStages) & 1, kWaitLimit);
  }
}

// The staged form's plane facts of one step (planes -1 .. nz, one thread each): computed once per
// step here instead of by each tile's copy-issuing thread, whose table and incident-line loads
// held up the halo warp of every boundary tile on every plane.
template <typename T>
__global__ void k3_facts(const Args3<T> a) {
  const int z = (int)(blockIdx.x * blockDim.x + threadIdx.x) - 1;
  if (z > a.nz) return;
  plane_facts(a, z, (PlaneS<T>*)(a.ftab + (size_t)(z + 1) * Stage3<T>::pl_bytes));
}

// CPML tables: [axis][E (integer positions) / H (half positions)][db = b - 1, c, 1/kappa, flag][nmax]
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
        b = expm1(-(sigma / kap + alpha) * dt / kEps0);  // stored as the deviation db = b - 1
        const double den = sigma * kap + kap * kap * alpha;
        c = (sigma > 0.0 && den > 0.0) ? sigma * b / den : 0.0;
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

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

struct rketd_ctx3d {
  rketd_grid3d g{};
  int prec = 0, fused = 1, staged = 0, cur = 0, kc = 64;
  Maps3<float> maps32[2];
  Maps3<double> maps64[2];
  int* err = nullptr;
  int4* items = nullptr;  // staged form work items (tile origin, plane range), by kind
  unsigned char* ftab = nullptr;  // staged form: plane facts of the current step (planes -1 .. nz)
  int n_mid = 0, n_zc = 0, n_gen[4] = {};  // general kinds: x and y, x only, y only, faces only
  // the boundary-tile launch runs on a high-priority side stream, overlapping the interior one
  cudaStream_t side = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
  size_t esz = 4;
  int64_t N = 0;
  double S = 0;
  cudaStream_t stream = nullptr;
  std::vector<void*> allocs;
  std::vector<std::pair<void*, size_t>> zeroed;  // every state buffer, cleared by reset
  void* E[2][3] = {};
  void* H[2][3] = {};
  void* J[3] = {};
  uint8_t* mat = nullptr;
  void* tab = nullptr;
  int nmax = 0, Z = 0;
  void* psiE[6] = {};
  void* psiH[2][6] = {};
  void* Ei[2] = {};
  void* Hi[2] = {};
  int* probes = nullptr;
  int n_probes = 0, n_freq = 0;
  double* freq = nullptr;
  void* series = nullptr;
  void* tw = nullptr;
  double *Xr = nullptr, *Xi = nullptr, *Xtmp = nullptr;
  int dft_block = 512;
  double coef[6][kMat] = {};  // da, cb, cj, dj, bp (cj-scaled), cc (cj-scaled) per material
  void* cj_d = nullptr;
  int n_mat = 1;
  rketd_pulse pulse{};
  int64_t step = 0;
  int64_t launches = 0;
  int wait_limit = kWaitLimit;
  int64_t tile_planes[6] = {};  // staged form: planes of 32 x kTY tiles per work kind (kModeGen .. kModeGenF)
  ~rketd_ctx3d() {
    for (void* p : allocs) cudaFree(p);
    if (fork) cudaEventDestroy(fork);
    if (join) cudaEventDestroy(join);
    if (side) cudaStreamDestroy(side);
  }
  bool alloc(void** p, size_t bytes, bool state = false) {
    *p = nullptr;
    if (!bytes) bytes = 16;
    if (device_alloc(p, bytes) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    allocs.push_back(*p);
    if (state) zeroed.push_back({*p, bytes});
    return true;
  }
};

namespace {

// derivative axis of each CPML memory, E side then H side (Ex/y, Ex/z, Ey/z, Ey/x, Ez/x, Ez/y;
// Hx/y, Hx/z, Hy/z, Hy/x, Hz/x, Hz/y)
constexpr int kPsiAxis[6] = {1, 2, 2, 0, 0, 1};

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
  a.wait_limit = c->wait_limit;
  const int in = c->cur, out = c->fused ? 1 - c->cur : c->cur;
  a.Ex = (const T*)c->E[in][0];
  a.Ey = (const T*)c->E[in][1];
  a.Ez = (const T*)c->E[in][2];
  a.Hx = (const T*)c->H[in][0];
  a.Hy = (const T*)c->H[in][1];
  a.Hz = (const T*)c->H[in][2];
  a.oEx = (T*)c->E[out][0];
  a.oEy = (T*)c->E[out][1];
  a.oEz = (T*)c->E[out][2];
  a.oHx = (T*)c->H[out][0];
  a.oHy = (T*)c->H[out][1];
  a.oHz = (T*)c->H[out][2];
  a.Jx = (T*)c->J[0];
  a.Jy = (T*)c->J[1];
  a.Jz = (T*)c->J[2];
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
  a.kc = c->kc;
  a.S = (T)c->S;
  a.q = (T)((c->S - 1.0) / (c->S + 1.0));
  a.tab = (const T*)c->tab;
  a.nmax = c->nmax;
  a.np = c->g.npml;
  a.Z = c->Z;
  for (int q = 0; q < 6; ++q) {
    a.psiE[q] = (T*)c->psiE[q];
    a.psiH[q] = (const T*)c->psiH[in][q];
    a.opsiH[q] = (T*)c->psiH[out][q];
  }
  a.tfsf = c->g.tfsf;
  a.i0 = c->g.box[0];
  a.i1 = c->g.box[1];
  a.j0 = c->g.box[2];
  a.j1 = c->g.box[3];
  a.k0 = c->g.box[4];
  a.k1 = c->g.box[5];
  a.Ei = (const T*)c->Ei[in];
  a.Hi = (const T*)c->Hi[in];
  a.oEi = (T*)c->Ei[out];
  a.oHi = (T*)c->Hi[out];
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
  a.ftab = c->ftab;
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
const Maps3<T>& maps(const rketd_ctx3d* c, int set);
template <>
const Maps3<float>& maps<float>(const rketd_ctx3d* c, int set) {
  return c->maps32[set];
}
template <>
const Maps3<double>& maps<double>(const rketd_ctx3d* c, int set) {
  return c->maps64[set];
}

// Work items of the staged form for the current k chunk. Interior-column tiles split their z
// range into the two z CPML slabs [0, np+1) and [nz-np-1, nz) plus one-plane items at the TF/SF
// z faces and the sheet (kModeZc), and the rest of the middle, cut into chunks of kc planes
// (kModeMid: every plane there is a bare update); the other tiles cover all planes in chunks of
// kc (kModeGen).
rketd_status plan_items3(rketd_ctx3d* c) {
  const rketd_grid3d& g = c->g;
  const int np = g.npml, nz = g.nz, kc = c->kc;
  // chunk-major order: the tiles of one plane range are neighbours in the launch, so the halo
  // rows that adjacent tiles share are read while still in L2
  std::vector<int2> inner, outer[4];
  const auto touches = [&](int lo, int hi, int N) { return lo <= np || hi >= N - np - 1; };  // CPML zone or edge
  for (int j0 = 0; j0 < g.ny; j0 += kTY)
    for (int i0 = 0; i0 < g.nx; i0 += 32) {
      if (interior_tile(i0, j0, g.nx, g.ny, np, g.tfsf, g.box)) {
        inner.push_back(make_int2(i0, j0));
      } else {
        const bool xc = touches(i0 - 1, i0 + 31, g.nx), yc = touches(j0 - 1, j0 + kTY - 1, g.ny);
        outer[xc && yc ? 0 : (xc ? 1 : (yc ? 2 : 3))].push_back(make_int2(i0, j0));
      }
    }
  std::vector<int4> mid, zc, gen[4];
  // Planes of the middle range that need more than the bare update go to z-general items: the
  // TF/SF z faces (Hy at k0-1 and k1, Ex at k0 and k1), the sheet, and the plane after each Hy
  // face, because a middle item starting there would compute its first plane's k-1 neighbour
  // (the corrected Hy of the face plane) without the correction. Consecutive ones form one item;
  // a run that starts within kSlabReach planes of a z CPML slab joins that slab's item (the
  // planes between them are bare updates, which the z-general kind also does), so that the usual
  // TF/SF faces a few cells inside the CPML do not make items of one or two planes per tile.
  constexpr int kSlabReach = 16;
  int lo_all = np + 1, hi_all = nz - np - 1;
  std::vector<int> special;
  if (g.tfsf) special.insert(special.end(), {g.box[4] - 1, g.box[4], g.box[5], g.box[5] + 1});
  if (g.sheet_k >= 0) special.push_back(g.sheet_k);
  std::sort(special.begin(), special.end());
  special.erase(std::unique(special.begin(), special.end()), special.end());
  special.erase(std::remove_if(special.begin(), special.end(), [&](int z) { return z < lo_all || z >= hi_all; }),
                special.end());
  std::vector<std::pair<int, int>> runs;  // [start, end) of consecutive special planes
  for (const int z : special) {
    if (!runs.empty() && runs.back().second == z) runs.back().second = z + 1;
    else runs.push_back({z, z + 1});
  }
  while (!runs.empty() && runs.front().first - lo_all <= kSlabReach && runs.front().second < hi_all) {
    lo_all = runs.front().second;
    runs.erase(runs.begin());
  }
  while (!runs.empty() && hi_all - runs.back().second <= kSlabReach && runs.back().first > lo_all) {
    hi_all = runs.back().first;
    runs.pop_back();
  }
  for (const int2 t : inner) zc.push_back(make_int4(t.x, t.y, 0, lo_all));
  for (const int2 t : inner) zc.push_back(make_int4(t.x, t.y, hi_all, nz));
  for (const auto& r : runs)
    for (const int2 t : inner) zc.push_back(make_int4(t.x, t.y, r.first, r.second));
  int lo = lo_all;
  for (size_t ridx = 0; ridx <= runs.size(); ++ridx) {
    const int hi = ridx < runs.size() ? runs[ridx].first : hi_all;
    for (int kb = lo; kb < hi; kb += kc)
      for (const int2 t : inner) mid.push_back(make_int4(t.x, t.y, kb, std::min(kb + kc, hi)));
    if (ridx < runs.size()) lo = runs[ridx].second;
  }
  const int kcg = RKETD_3D_KC_GEN > 0 ? RKETD_3D_KC_GEN : kc;
  for (int kind = 0; kind < 4; ++kind)
    for (int kb = 0; kb < nz; kb += kcg)
      for (const int2 t : outer[kind]) gen[kind].push_back(make_int4(t.x, t.y, kb, std::min(kb + kcg, nz)));
  c->n_mid = (int)mid.size();
  c->n_zc = (int)zc.size();
  auto planes = [](const std::vector<int4>& v) {
    int64_t n = 0;
    for (const int4& t : v) n += t.w - t.z;
    return n;
  };
  c->tile_planes[kModeMid] = planes(mid);
  c->tile_planes[kModeZc] = planes(zc);
  c->tile_planes[kModeGen] = planes(gen[0]);
  c->tile_planes[kModeGenX] = planes(gen[1]);
  c->tile_planes[kModeGenY] = planes(gen[2]);
  c->tile_planes[kModeGenF] = planes(gen[3]);
  std::vector<int4> all(mid);
  all.insert(all.end(), zc.begin(), zc.end());
  for (int kind = 0; kind < 4; ++kind) {
    c->n_gen[kind] = (int)gen[kind].size();
    all.insert(all.end(), gen[kind].begin(), gen[kind].end());
  }
  if (c->items) {
    cudaFree(c->items);
    c->allocs.erase(std::remove(c->allocs.begin(), c->allocs.end(), (void*)c->items), c->allocs.end());
    c->items = nullptr;
  }
  if (!c->alloc((void**)&c->items, sizeof(int4) * std::max<size_t>(all.size(), 1)))
    return fail3(RKETD_ENOMEM, "work items");
  CK3(cudaMemcpy(c->items, all.data(), sizeof(int4) * all.size(), cudaMemcpyHostToDevice), "work items");
  return RKETD_OK;
}

// tensor maps of the staged form: a 3D box of kBW x kBH x 1 values of each field array and
// 32 x kTY x 1 bytes of the material array, zero fill outside the grid
template <typename T>
rketd_status make_maps(rketd_ctx3d* c) {
  static EncodeTiledFn encode = nullptr;
  if (!encode) {
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
      return fail3(RKETD_ECUDA, "cuTensorMapEncodeTiled is not available");
    encode = (EncodeTiledFn)fn;
  }
  const rketd_grid3d& g = c->g;
  const cuuint64_t dims[3] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz};
  const cuuint64_t fstr[2] = {(cuuint64_t)g.nx * sizeof(T), (cuuint64_t)g.nx * g.ny * sizeof(T)};
  const cuuint64_t mstr[2] = {(cuuint64_t)g.nx, (cuuint64_t)g.nx * g.ny};
  const cuuint32_t fbox[3] = {kBW, kBH, 1}, mbox[3] = {32, kTY, 1}, es[3] = {1, 1, 1};
  const CUtensorMapDataType dt = sizeof(T) == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  for (int set = 0; set < 2; ++set) {
    Maps3<T>& m = const_cast<Maps3<T>&>(maps<T>(c, set));
    void* arrs[6] = {c->E[set][0], c->E[set][1], c->E[set][2], c->H[set][0], c->H[set][1], c->H[set][2]};
    for (int f = 0; f < 6; ++f)
      if (encode(&m.f[f], dt, 3, arrs[f], dims, fstr, fbox, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                 CU_TENSOR_MAP_SWIZZLE_NONE, (CUtensorMapL2promotion)RKETD_3D_L2PROMO,
                 CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return fail3(RKETD_ECUDA, "field tensor map");
    if (encode(&m.mat, CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, c->mat, dims, mstr, mbox, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, (CUtensorMapL2promotion)RKETD_3D_L2PROMO,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return fail3(RKETD_ECUDA, "material tensor map");
  }
  CK3(cudaFuncSetAttribute(k3_staged<T, kModeGen>, cudaFuncAttributeMaxDynamicSharedMemorySize, Stage3<T>::smem),
      "staged kernel shared memory");
  CK3(cudaFuncSetAttribute(k3_staged<T, kModeMid>, cudaFuncAttributeMaxDynamicSharedMemorySize, Stage3<T>::smem),
      "staged kernel shared memory");
  CK3(cudaFuncSetAttribute(k3_staged<T, kModeZc>, cudaFuncAttributeMaxDynamicSharedMemorySize, Stage3<T>::smem),
      "staged kernel shared memory");
  CK3(cudaFuncSetAttribute(k3_staged<T, kModeGenX>, cudaFuncAttributeMaxDynamicSharedMemorySize, Stage3<T>::smem),
      "staged kernel shared memory");
  CK3(cudaFuncSetAttribute(k3_staged<T, kModeGenY>, cudaFuncAttributeMaxDynamicSharedMemorySize, Stage3<T>::smem),
      "staged kernel shared memory");
  CK3(cudaFuncSetAttribute(k3_staged<T, kModeGenF>, cudaFuncAttributeMaxDynamicSharedMemorySize, Stage3<T>::smem),
      "staged kernel shared memory");
  if (!c->alloc((void**)&c->ftab, (size_t)(g.nz + 2) * Stage3<T>::pl_bytes)) return fail3(RKETD_ENOMEM, "plane facts");
  rketd_status st = plan_items3(c);
  if (st) return st;
  int prio_lo = 0, prio_hi = 0;
  CK3(cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi), "stream priorities");
  CK3(cudaStreamCreateWithPriority(&c->side, cudaStreamNonBlocking, prio_hi), "side stream");
  CK3(cudaEventCreateWithFlags(&c->fork, cudaEventDisableTiming), "fork event");
  CK3(cudaEventCreateWithFlags(&c->join, cudaEventDisableTiming), "join event");
  return RKETD_OK;
}

// device-side status of the staged form (a bounded wait that gave up); synchronises
rketd_status check3(rketd_ctx3d* c) {
  CK3(cudaStreamSynchronize(c->stream), "3D step");
  int e = 0;
  CK3(cudaMemcpy(&e, c->err, sizeof(int), cudaMemcpyDeviceToHost), "3D status");
  if (e) return fail3(RKETD_ETIMEOUT, "a staged-copy wait gave up; fields are not valid");
  return RKETD_OK;
}

template <typename T>
rketd_status step3(rketd_ctx3d* c, int64_t nsteps) {
  const int ty = 8;
  const unsigned nzc = (unsigned)((c->g.nz + c->kc - 1) / c->kc);
  const dim3 block(32, ty);
  const dim3 grid((c->g.nx + 31) / 32, (c->g.ny + ty - 1) / ty, nzc + (c->g.tfsf ? 1 : 0));
  const dim3 sblock(32, kTY + 1);
  const int line = c->g.tfsf ? 1 : 0;
  for (int64_t s = 0; s < nsteps; ++s) {
    Args3<T> a = args3<T>(c);
    if (c->staged) {
      // boundary tiles (CPML, faces: more work per cell) first, on the high-priority side
      // stream, so that they run alongside the interior tiles; joined back afterwards
      const int n_gen_all = c->n_gen[0] + c->n_gen[1] + c->n_gen[2] + c->n_gen[3];
      if (n_gen_all + c->n_zc) {
        k3_facts<T><<<(unsigned)((c->g.nz + 2 + 127) / 128), 128, 0, c->stream>>>(a);
        c->launches += 1;
      }
      const bool forked = (c->n_mid + c->n_zc) && (n_gen_all + line);
      if (forked) {
        CK3(cudaEventRecord(c->fork, c->stream), "fork");
        CK3(cudaStreamWaitEvent(c->side, c->fork, 0), "fork");
      }
      const Maps3<T>& mp = maps<T>(c, c->cur);
      cudaStream_t gs = forked ? c->side : c->stream;
      const int4* gi = c->items + c->n_mid + c->n_zc;
      if (c->n_gen[0] + line) {  // the incident line rides with this launch
        k3_staged<T, kModeGen><<<c->n_gen[0] + line, sblock, Stage3<T>::smem, gs>>>(a, mp, gi, c->n_gen[0], c->err);
        c->launches += 1;
      }
      gi += c->n_gen[0];
      if (c->n_gen[1]) {
        k3_staged<T, kModeGenX><<<c->n_gen[1], sblock, Stage3<T>::smem, gs>>>(a, mp, gi, c->n_gen[1], c->err);
        c->launches += 1;
      }
      gi += c->n_gen[1];
      if (c->n_gen[2]) {
        k3_staged<T, kModeGenY><<<c->n_gen[2], sblock, Stage3<T>::smem, gs>>>(a, mp, gi, c->n_gen[2], c->err);
        c->launches += 1;
      }
      gi += c->n_gen[2];
      if (c->n_gen[3]) {
        k3_staged<T, kModeGenF><<<c->n_gen[3], sblock, Stage3<T>::smem, gs>>>(a, mp, gi, c->n_gen[3], c->err);
        c->launches += 1;
      }
      // main stream: the middle items, which share the GPU with the side stream's boundary kinds
      // from the start. The z-CPML slab items of the interior tiles follow the boundary kinds on
      // the side stream, so that they run beside the end of the middle launch rather than after it
      // (1.2% faster on the 512^3 sphere than after the middle items on the main stream).
      if (c->n_mid) {
        k3_staged<T, kModeMid><<<c->n_mid, sblock, Stage3<T>::smem, c->stream>>>(a, mp, c->items, c->n_mid, c->err);
        c->launches += 1;
      }
      if (c->n_zc) {
        k3_staged<T, kModeZc><<<c->n_zc, sblock, Stage3<T>::smem, gs>>>(a, mp, c->items + c->n_mid, c->n_zc, c->err);
        c->launches += 1;
      }
      if (forked) {
        CK3(cudaEventRecord(c->join, c->side), "join");
        CK3(cudaStreamWaitEvent(c->stream, c->join, 0), "join");
      }
      c->cur = 1 - c->cur;
    } else if (c->fused) {
      k3_fused<T><<<grid, block, 0, c->stream>>>(a);
      c->launches += 1;
      c->cur = 1 - c->cur;
    } else {
      a.line_fresh = 1;
      k3_h<T><<<grid, block, 0, c->stream>>>(a);
      k3_e<T><<<grid, block, 0, c->stream>>>(a);
      c->launches += 2;
    }
    CK3(cudaGetLastError(), "3D step");
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
  if ((int64_t)g->nx * g->ny > (int64_t)1 << 31) return fail3(RKETD_EINVAL, "nx * ny must fit in 32 bits");
  if (!(g->d > 0) || !(g->dt > 0) || !std::isfinite(g->d) || !std::isfinite(g->dt))
    return fail3(RKETD_EINVAL, "d and dt must be finite and > 0");
  if (g->prec != RKETD_F32 && g->prec != RKETD_F64) return fail3(RKETD_EINVAL, "prec must be F32 or F64");
  if (g->variant < 0 || g->variant > 3)
    return fail3(RKETD_EINVAL, "variant must be 0 (auto), 1 (plain), 2 (fused) or 3 (staged)");
  // staged form: CPML on every face, 16-byte aligned rows, CPML memory offsets within 32 bits
  const int64_t zw = 2 * ((int64_t)std::max(g->npml, 0) + 1), lim = int64_t(1) << 31;
  const bool can_stage = !g->periodic_xy && g->nx % 16 == 0 && (int64_t)g->nz * g->ny * zw < lim &&
                         (int64_t)g->nz * zw * g->nx < lim && zw * g->ny * g->nx < lim;
  if (g->variant == 3 && !can_stage)
    return fail3(RKETD_EUNSUPPORTED,
                 "the staged form needs CPML on every face, nx a multiple of 16 and CPML memories of < 2^31 entries");
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
  // at most 4 probes per (i, j) column are sampled by one thread
  for (int p = 0; p < n_probes; ++p) {
    int same = 0;
    for (int q = 0; q < n_probes; ++q) same += probes[3 * q] == probes[3 * p] && probes[3 * q + 1] == probes[3 * p + 1];
    if (same > 4) return fail3(RKETD_EINVAL, "at most 4 probes may share an (i, j) column");
  }
  rketd_ctx3d* c = new (std::nothrow) rketd_ctx3d();
  if (!c) return fail3(RKETD_ENOMEM, "host allocation");
  auto bad = [&](rketd_status s, const char* m) {
    delete c;
    return fail3(s, m);
  };
  c->g = *g;
  if (!(c->g.pml_sigma_max > 0)) c->g.pml_sigma_max = 0.8 * (g->pml_m + 1) / (std::sqrt(kMu0 / kEps0) * g->d);
  c->prec = g->prec;
  c->fused = g->variant != 1;
  c->staged = g->variant == 3 || (g->variant == 0 && can_stage);
  c->esz = g->prec == RKETD_F64 ? 8 : 4;
  c->N = (int64_t)g->nx * g->ny * g->nz;
  c->S = S;
  c->stream = (cudaStream_t)stream;
  c->pulse = *pulse;
  c->n_mat = n_mat;
  c->n_probes = n_probes;
  c->n_freq = n_probes ? nf : 0;
  // per-material coefficients of the update (FP64 on the host for at most four materials,
  // passed to the kernels as arguments)
  for (int m = 0; m < kMat; ++m) {
    const double w = m < n_mat ? mat_wp2[m] * g->dt * g->dt : 0.0;
    const double x = m < n_mat ? mat_nu[m] * g->dt : 0.0;
    // phi1 = (1 - e^-x)/x and phi2 = (e^-x - 1 + x)/x^2: Taylor series below 0.5 (summed
    // smallest term first), expm1 above
    double p1, p2;
    if (x < 0.5) {
      double t1 = 1.0, t2 = 0.5;
      double terms1[24], terms2[24];
      for (int q = 0; q < 24; ++q) {
        terms1[q] = t1;
        terms2[q] = t2;
        t1 *= -x / (q + 2);
        t2 *= -x / (q + 3);
      }
      double s1 = 0, s2 = 0;
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
  const int sets = c->fused ? 2 : 1;
  for (int s = 0; s < sets; ++s)
    for (int q = 0; q < 3; ++q)
      if (!c->alloc(&c->E[s][q], fb, true) || !c->alloc(&c->H[s][q], fb, true)) return bad(RKETD_ENOMEM, "3D fields");
  if (!c->fused)
    for (int q = 0; q < 3; ++q) {
      c->E[1][q] = c->E[0][q];
      c->H[1][q] = c->H[0][q];
    }
  for (int q = 0; q < 3; ++q)
    if (!c->alloc(&c->J[q], fb, true)) return bad(RKETD_ENOMEM, "3D currents");
  if (!c->alloc((void**)&c->mat, c->N)) return bad(RKETD_ENOMEM, "3D materials");
  c->nmax = std::max(g->nx, std::max(g->ny, g->nz));
  c->Z = 2 * (np + 1);
  if (!c->alloc(&c->tab, c->esz * 24 * c->nmax)) return bad(RKETD_ENOMEM, "CPML tables");
  const int64_t zsz[3] = {(int64_t)g->nz * g->ny * c->Z, (int64_t)g->nz * c->Z * g->nx,
                          (int64_t)c->Z * g->ny * g->nx};
  for (int q = 0; q < 6; ++q) {
    const int ax = kPsiAxis[q];
    const size_t bytes = (ax < 2 && g->periodic_xy) ? 16 : c->esz * zsz[ax];
    if (!c->alloc(&c->psiE[q], bytes, true)) return bad(RKETD_ENOMEM, "CPML memories");
    // H side: Hx/y, Hx/z, Hy/z, Hy/x, Hz/x, Hz/y have the axes of Ex/y, Ex/z, Ey/z, Ey/x, Ez/x, Ez/y
    for (int s = 0; s < sets; ++s)
      if (!c->alloc(&c->psiH[s][q], bytes, true)) return bad(RKETD_ENOMEM, "CPML memories");
    if (!c->fused) c->psiH[1][q] = c->psiH[0][q];
  }
  const size_t lb = c->esz * std::max(1, g->inc_len);
  for (int s = 0; s < sets; ++s)
    if (!c->alloc(&c->Ei[s], lb, true) || !c->alloc(&c->Hi[s], lb, true)) return bad(RKETD_ENOMEM, "incident line");
  if (!c->fused) {
    c->Ei[1] = c->Ei[0];
    c->Hi[1] = c->Hi[0];
  }
  if (!c->alloc(&c->cj_d, c->esz * kMat)) return bad(RKETD_ENOMEM, "coefficients");
  if (!c->alloc((void**)&c->err, sizeof(int), true)) return bad(RKETD_ENOMEM, "status word");
  if (n_probes) {
    if (!c->alloc((void**)&c->probes, sizeof(int) * 3 * n_probes) || !c->alloc((void**)&c->freq, sizeof(double) * nf) ||
        !c->alloc(&c->series, c->esz * (size_t)n_probes * c->dft_block) ||
        !c->alloc(&c->tw, c->esz * 2 * (size_t)c->dft_block * nf) ||
        !c->alloc((void**)&c->Xr, sizeof(double) * n_probes * nf, true) ||
        !c->alloc((void**)&c->Xi, sizeof(double) * n_probes * nf, true) ||
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
  const unsigned tbk = (unsigned)((c->nmax + 127) / 128);
  if (c->prec == RKETD_F64)
    k3_tables<double><<<tbk, 128, 0, c->stream>>>(g->nx, g->ny, g->nz, np, g->periodic_xy, g->dt, g->pml_m,
                                                  c->g.pml_sigma_max, g->pml_kappa_max, g->pml_alpha_max, c->nmax,
                                                  (double*)c->tab);
  else
    k3_tables<float><<<tbk, 128, 0, c->stream>>>(g->nx, g->ny, g->nz, np, g->periodic_xy, g->dt, g->pml_m,
                                                 c->g.pml_sigma_max, g->pml_kappa_max, g->pml_alpha_max, c->nmax,
                                                 (float*)c->tab);
  c->launches += 1;
  if (c->staged) {
    rketd_status sm = c->prec == RKETD_F64 ? make_maps<double>(c) : make_maps<float>(c);
    if (sm) {
      delete c;
      return sm;
    }
  }
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
  for (auto& z : c->zeroed) CK3(cudaMemsetAsync(z.first, 0, z.second, c->stream), "reset");
  c->step = 0;
  c->cur = 0;
  return RKETD_OK;
}

rketd_status rketd_step_3d(rketd_ctx3d* c, int64_t nsteps) {
  if (!c) return fail3(RKETD_EINVAL, "NULL context");
  if (nsteps < 0) return fail3(RKETD_EINVAL, "nsteps < 0");
  return c->prec == RKETD_F64 ? step3<double>(c, nsteps) : step3<float>(c, nsteps);
}

rketd_status rketd_get_field_3d(rketd_ctx3d* c, int32_t which, double* out) {
  if (!c || !out || which < 0 || which > 8) return fail3(RKETD_EINVAL, "invalid arguments");
  const void* src = which < 3 ? c->E[c->cur][which] : (which < 6 ? c->H[c->cur][which - 3] : c->J[which - 6]);
  double* tmp;
  CK3(device_alloc_async((void**)&tmp, sizeof(double) * c->N, c->stream), "field staging");
  const double eta0 = std::sqrt(kMu0 / kEps0);
  const double scale = which < 3 ? 1.0 : (which < 6 ? 1.0 / eta0 : kEps0 / c->g.dt);
  const int shift = which >= 6 ? 2 * (which - 6) : 0;
  const unsigned blocks = (unsigned)((c->N + 255) / 256);
  if (c->prec == RKETD_F64)
    k3_gather<double><<<blocks, 256, 0, c->stream>>>((const double*)src, c->N, scale,
                                                     which >= 6 ? (const double*)c->cj_d : nullptr, c->mat, shift, tmp);
  else
    k3_gather<float><<<blocks, 256, 0, c->stream>>>((const float*)src, c->N, scale,
                                                    which >= 6 ? (const float*)c->cj_d : nullptr, c->mat, shift, tmp);
  cudaError_t e = cudaMemcpyAsync(out, tmp, sizeof(double) * c->N, cudaMemcpyDeviceToHost, c->stream);
  cudaFreeAsync(tmp, c->stream);
  CK3(e, "get_field_3d");
  return check3(c);
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
  return check3(c);
}

rketd_status rketd_work_3d(const rketd_ctx3d* c, int64_t tile_planes[6]) {
  if (!c || !tile_planes) return fail3(RKETD_EINVAL, "NULL argument");
  for (int k = 0; k < 6; ++k) tile_planes[k] = c->tile_planes[k];
  return RKETD_OK;
}

rketd_status rketd_set_wait_limit_3d(rketd_ctx3d* c, int32_t polls) {
  if (!c) return fail3(RKETD_EINVAL, "NULL context");
  c->wait_limit = polls < 0 ? kWaitLimit : std::min<int32_t>(polls, kWaitLimit);
  return RKETD_OK;
}

rketd_status rketd_check_finite_3d(rketd_ctx3d* c) {
  if (!c) return fail3(RKETD_EINVAL, "NULL context");
  int* flag = nullptr;
  CK3(device_alloc_async((void**)&flag, sizeof(int), c->stream), "finite scan");
  cudaError_t e = cudaMemsetAsync(flag, 0, sizeof(int), c->stream);
  const bool f64 = c->prec == RKETD_F64;
  for (int q = 0; q < 3 && e == cudaSuccess; ++q) {
    e = launch_finite_scan(f64, c->E[c->cur][q], c->N, flag, c->stream);
    if (e == cudaSuccess) e = launch_finite_scan(f64, c->H[c->cur][q], c->N, flag, c->stream);
    if (e == cudaSuccess) e = launch_finite_scan(f64, c->J[q], c->N, flag, c->stream);
  }
  const int64_t nx = (int64_t)c->n_probes * c->n_freq;
  if (e == cudaSuccess && nx) e = launch_finite_scan(true, c->Xr, nx, flag, c->stream);
  if (e == cudaSuccess && nx) e = launch_finite_scan(true, c->Xi, nx, flag, c->stream);
  int h = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
  cudaFreeAsync(flag, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return fail3(RKETD_ECUDA, std::string("finite scan: ") + cudaGetErrorString(e));
  if (h) return fail3(RKETD_ENUMERIC, "a field or spectrum holds NaN or Inf");
  return RKETD_OK;
}

rketd_status rketd_sync_3d(rketd_ctx3d* c) {
  if (!c) return fail3(RKETD_EINVAL, "NULL context");
  return check3(c);
}

rketd_status rketd_kernel_chunk_3d(rketd_ctx3d* c, int32_t k_chunk) {
  if (!c || k_chunk < 1 || k_chunk > 4096) return fail3(RKETD_EINVAL, "k_chunk must be 1..4096");
  c->kc = k_chunk;
  if (c->staged) {
    CK3(cudaStreamSynchronize(c->stream), "k chunk");
    return plan_items3(c);
  }
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
