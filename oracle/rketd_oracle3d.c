/*
 * rketd_oracle3d.c -- TEST INFRASTRUCTURE, not part of the product.
 *
 * Plain serial FP64 3D Yee RKETD-FDTD in SI units: the three-component form of Eqs. 1-3
 * (the paper's Sec. II before its 1D reduction, Eqs. 4-6), discretised component by component
 * exactly as the 1D oracle discretises Eqs. 12, 11 and 14, with the paper's own 2D/3D
 * generalisation as the stated next step (Sec. IV.B, Sec. V). Arrays are [k][j][i] (x fastest).
 * Yee positions: Ex (i+1/2, j, k), Ey (i, j+1/2, k), Ez (i, j, k+1/2),
 *                Hx (i, j+1/2, k+1/2), Hy (i+1/2, j, k+1/2), Hz (i+1/2, j+1/2, k).
 * Boundaries: CPML (as in the 1D oracle, per axis) backed by PEC walls on every face, or
 * periodic in x and y with CPML only along z. Sources: a total-field/scattered-field box fed
 * by an auxiliary 1D line (Ex-polarised plane wave along +z; the 1D line obeys the same
 * discrete equations, so the box leaks nothing in vacuum), and/or a soft sheet source on Ex
 * at one z plane. Plasma: each E component takes the material at its own Yee position; the
 * byte mat[i,j,k] packs the indices of Ex, Ey, Ez of that cell in bits 0-1, 2-3, 4-5.
 * One step: H update (+ TF/SF H corrections), 1D incident H, E and J update (+ TF/SF E
 * corrections, sheet source), 1D incident E, running DFT of Ex at the probes.
 * Only tests/ and bench.py's CPU legs load this file; it shares no code with the CUDA path.
 *
 * Pins (tests/test_oracle3d_pins.py): reduction to the 1D oracle along z for both polarisations,
 * the exact lattice recurrence of a transverse Fourier mode (every x/y difference term), a cyclic
 * rotation of the cube mapping the x/y-face CPML onto the z-face CPML bit for bit, the x/y-face
 * CPML reflection against a domain with unreachable faces, and the TF/SF box in vacuum.
 * OR_MUTANT 5-8 plant one mistake each (tests only) for the check that the pins reject them.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define O3_EPS0 8.8541878128e-12
#define O3_MU0 1.25663706212e-6
#define O3_PI 3.14159265358979323846

double or_phi1(double x);
double or_phi2(double x);

typedef struct {
  int32_t nx, ny, nz;
  double d, dt;
  int32_t periodic_xy;  /* 1: periodic x and y, CPML along z only; 0: CPML on all faces */
  int32_t npml;
  double pml_m, pml_sigma_max, pml_kappa_max, pml_alpha_max;
  int32_t tfsf;          /* 1: TF/SF box [i0,i1] x [j0,j1] x [k0,k1] */
  int32_t box[6];
  int32_t sheet_k;       /* >= 0: soft sheet source on Ex at this k */
  double src_tau, src_t0, src_amp;
  int32_t n_probes, n_freq;
  int32_t inc_off;       /* 1D line index = k + inc_off */
  int32_t inc_len;       /* 1D line length (>= nz + 2 inc_off) */
  int32_t inc_src;       /* 1D soft-source index */
} or_grid3d;

static double o3_pulse(const or_grid3d* g, double t) {
  double u = (t - g->src_t0) / g->src_tau;
  return g->src_amp * u * exp(-0.5 * u * u);
}

/* CPML grading at relative depth rho (as the 1D oracle). */
static void o3_cpml_point(const or_grid3d* g, double rho, double* b, double* c, double* kinv) {
  double pm = pow(rho, g->pml_m);
  double sigma = g->pml_sigma_max * pm;
  double kap = 1.0 + (g->pml_kappa_max - 1.0) * pm;
  double alpha = g->pml_alpha_max * (1.0 - rho);
  double bb = exp(-(sigma / kap + alpha) * g->dt / O3_EPS0);
  double den = sigma * kap + kap * kap * alpha;
  *b = bb;
  *c = (sigma == 0.0 || den == 0.0) ? 0.0 : sigma * (bb - 1.0) / den;
  *kinv = 1.0 / kap;
}

/* Relative depth of position x (in cells) along an axis of n nodes with np-cell layers. */
static double o3_rho(int np, int n, double x) {
  double inner_r = (double)(n - 1) - np;
  if (np <= 0) return 0.0;
  if (x < np) return (np - x) / np;
  if (x > inner_r) return (x - inner_r) / np;
  return 0.0;
}

#define IDX(i, j, k) ((((int64_t)(k)) * ny + (j)) * nx + (i))

/*
 * Advances n_steps steps from step n_start. fields: [9][nx*ny*nz] = Ex, Ey, Ez, Hx, Hy, Hz,
 * Jx, Jy, Jz (in/out, SI). psi: [12][nx*ny*nz] CPML memories (in/out), order
 * Ex/y, Ex/z, Ey/z, Ey/x, Ez/x, Ez/y, Hx/y, Hx/z, Hy/z, Hy/x, Hz/x, Hz/y. inc: [2][inc_len]
 * incident Ex, Hy of the 1D line (in/out). mat[nx*ny*nz]: packed material indices of Ex, Ey, Ez
 * (2 bits each, 0 = vacuum);
 * mat_wp2/mat_nu [n_mat]. probes [n_probes*3] (i, j, k) of Ex samples. X_re/X_im
 * [n_probes*n_freq] accumulated; series [n_probes*n_steps] optional.
 */
int or_run3d(const or_grid3d* g, const uint8_t* mat, const double* mat_wp2, const double* mat_nu, int32_t n_mat,
             const int32_t* probes, const double* freq_hz, int64_t n_start, int64_t n_steps, double* fields,
             double* psi, double* inc, double* X_re, double* X_im, double* series) {
  const int nx = g->nx, ny = g->ny, nz = g->nz;
  const int64_t N = (int64_t)nx * ny * nz;
  const double dt = g->dt, d = g->d;
  const int per = g->periodic_xy;
  if (nx < 4 || ny < 4 || nz < 4) return -1;
  double *Ex = fields, *Ey = fields + N, *Ez = fields + 2 * N;
  double *Hx = fields + 3 * N, *Hy = fields + 4 * N, *Hz = fields + 5 * N;
  double *Jx = fields + 6 * N, *Jy = fields + 7 * N, *Jz = fields + 8 * N;
  double* P[12];
  for (int q = 0; q < 12; ++q) P[q] = psi + q * N;
  /* material constants of Eqs. 11 and 13 (as in the 1D oracle) */
  double* ma = (double*)malloc(sizeof(double) * n_mat);
  double* mb1 = (double*)malloc(sizeof(double) * n_mat);
  double* mb2 = (double*)malloc(sizeof(double) * n_mat);
  double* mEE = (double*)malloc(sizeof(double) * n_mat);
  double* mEH = (double*)malloc(sizeof(double) * n_mat);
  double* mEJ = (double*)malloc(sizeof(double) * n_mat);
  for (int m = 0; m < n_mat; ++m) {
    double x = mat_nu[m] * dt;
    ma[m] = exp(-x);
    mb1[m] = O3_EPS0 * mat_wp2[m] * dt * or_phi1(x);
    mb2[m] = O3_EPS0 * mat_wp2[m] * dt * or_phi2(x);
    double D = 1.0 + dt / (2.0 * O3_EPS0) * mb2[m];
    mEE[m] = (1.0 - dt / (2.0 * O3_EPS0) * (mb1[m] - mb2[m])) / D;
    mEH[m] = (dt / O3_EPS0) / D;
    mEJ[m] = (dt / (2.0 * O3_EPS0)) * (1.0 + ma[m]) / D;
  }
  /* CPML tables per axis: [axis][E or H][pos] -> (b, c, 1/kappa, flag) */
  int nn[3] = {nx, ny, nz};
  int npax[3] = {per ? 0 : g->npml, per ? 0 : g->npml, g->npml};
  double* tab[3][2];
  for (int ax = 0; ax < 3; ++ax)
    for (int h = 0; h < 2; ++h) {
      tab[ax][h] = (double*)calloc((size_t)4 * nn[ax], sizeof(double));
      for (int n = 0; n < nn[ax]; ++n) {
        double x = h ? n + 0.5 : (double)n;
        double rho = o3_rho(npax[ax], nn[ax], x);
        double* t = tab[ax][h] + 4 * n;
        t[2] = 1.0;
        if (rho > 0.0) {
          o3_cpml_point(g, rho, &t[0], &t[1], &t[2]);
          t[3] = 1.0;
        }
      }
    }
#define TB(ax, h, n) (tab[ax][h] + 4 * (n))
  const double cH = dt / O3_MU0;
  double* Ei = inc;
  double* Hi = inc + g->inc_len;
  const int L1 = g->inc_len, off = g->inc_off;
  const double S1 = dt / (sqrt(O3_MU0 * O3_EPS0) * d);
  const double q1 = (S1 - 1.0) / (S1 + 1.0);
  const int i0 = g->box[0], i1 = g->box[1], j0 = g->box[2], j1 = g->box[3], k0 = g->box[4], k1 = g->box[5];

  for (int64_t step = 0; step < n_steps; ++step) {
    const int64_t n = n_start + step;
    /* ---- H ---- */
    for (int k = 0; k < nz; ++k)
      for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
          const int64_t c = IDX(i, j, k);
          const int ip = (i + 1 < nx) ? i + 1 : (per ? 0 : -1);
          const int jp = (j + 1 < ny) ? j + 1 : (per ? 0 : -1);
          const int kp = (k + 1 < nz) ? k + 1 : -1;
          /* Hx (i, j+1/2, k+1/2) */
          if (jp >= 0 && kp >= 0) {
#if defined(OR_MUTANT) && OR_MUTANT == 6
            /* planted mistake: Hx's y difference taken along x */
            double dEz = Ez[IDX(ip >= 0 ? ip : i, j, k)] - Ez[c];
#else
            double dEz = Ez[IDX(i, jp, k)] - Ez[c];
#endif
            double dEy = Ey[IDX(i, j, kp)] - Ey[c];
            const double* ty = TB(1, 1, j);
            const double* tz = TB(2, 1, k);
            double cy = dEz / d, cz = dEy / d;
            if (ty[3] != 0.0) { P[6][c] = ty[0] * P[6][c] + ty[1] * cy; cy = dEz * ty[2] / d + P[6][c]; }
            if (tz[3] != 0.0) { P[7][c] = tz[0] * P[7][c] + tz[1] * cz; cz = dEy * tz[2] / d + P[7][c]; }
            Hx[c] = Hx[c] - cH * (cy - cz);
          }
          /* Hy (i+1/2, j, k+1/2) */
          if (ip >= 0 && kp >= 0) {
            double dEx = Ex[IDX(i, j, kp)] - Ex[c];
            double dEz = Ez[IDX(ip, j, k)] - Ez[c];
            const double* tz = TB(2, 1, k);
#if defined(OR_MUTANT) && OR_MUTANT == 7
            /* planted mistake: Hy's x-face CPML graded at the E nodes */
            const double* tx = TB(0, 0, i);
#else
            const double* tx = TB(0, 1, i);
#endif
            double cz = dEx / d, cx = dEz / d;
            if (tz[3] != 0.0) { P[8][c] = tz[0] * P[8][c] + tz[1] * cz; cz = dEx * tz[2] / d + P[8][c]; }
            if (tx[3] != 0.0) { P[9][c] = tx[0] * P[9][c] + tx[1] * cx; cx = dEz * tx[2] / d + P[9][c]; }
            Hy[c] = Hy[c] - cH * (cz - cx);
          }
          /* Hz (i+1/2, j+1/2, k) */
          if (ip >= 0 && jp >= 0) {
            double dEy = Ey[IDX(ip, j, k)] - Ey[c];
            double dEx = Ex[IDX(i, jp, k)] - Ex[c];
            const double* tx = TB(0, 1, i);
            const double* ty = TB(1, 1, j);
            double cx = dEy / d, cy = dEx / d;
            if (tx[3] != 0.0) { P[10][c] = tx[0] * P[10][c] + tx[1] * cx; cx = dEy * tx[2] / d + P[10][c]; }
            if (ty[3] != 0.0) { P[11][c] = ty[0] * P[11][c] + ty[1] * cy; cy = dEx * ty[2] / d + P[11][c]; }
            Hz[c] = Hz[c] - cH * (cx - cy);
          }
        }
    /* TF/SF corrections of H: incident Ex at time n */
    if (g->tfsf) {
      const double f = dt / (O3_MU0 * d);
      for (int j = j0; j <= j1; ++j)
        for (int i = i0; i <= i1 - 1; ++i) {
          Hy[IDX(i, j, k0 - 1)] += f * Ei[k0 + off];
          Hy[IDX(i, j, k1)] -= f * Ei[k1 + off];
        }
      for (int k = k0; k <= k1; ++k)
        for (int i = i0; i <= i1 - 1; ++i) {
          Hz[IDX(i, j0 - 1, k)] -= f * Ei[k + off];
          Hz[IDX(i, j1, k)] += f * Ei[k + off];
        }
      /* 1D incident H */
      for (int m = 0; m < L1 - 1; ++m) Hi[m] = Hi[m] - dt / O3_MU0 * ((Ei[m + 1] - Ei[m]) / d);
    }
    /* ---- E and J ---- */
    for (int k = 0; k < nz; ++k)
      for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
          const int64_t c = IDX(i, j, k);
          const int im = (i > 0) ? i - 1 : (per ? nx - 1 : -1);
          const int jm = (j > 0) ? j - 1 : (per ? ny - 1 : -1);
          const int km = (k > 0) ? k - 1 : -1;
          const int mx = mat[c] & 3, my = (mat[c] >> 2) & 3, mz = (mat[c] >> 4) & 3;
          const int xin = per || (i > 0 && i < nx - 1), yin = per || (j > 0 && j < ny - 1), zin = k > 0 && k < nz - 1;
          /* Ex (i+1/2, j, k): tangential to y and z walls */
          if ((per || i < nx - 1) && yin && zin) {
            double dHz = Hz[c] - Hz[IDX(i, jm, k)];
            double dHy = Hy[c] - Hy[IDX(i, j, km)];
            const double* ty = TB(1, 0, j);
            const double* tz = TB(2, 0, k);
            double cy = dHz / d, cz = dHy / d;
#if defined(OR_MUTANT) && OR_MUTANT == 8
            /* planted mistake: Ex's y-face CPML memory driven with the wrong sign */
            if (ty[3] != 0.0) { P[0][c] = ty[0] * P[0][c] - ty[1] * cy; cy = dHz * ty[2] / d + P[0][c]; }
#else
            if (ty[3] != 0.0) { P[0][c] = ty[0] * P[0][c] + ty[1] * cy; cy = dHz * ty[2] / d + P[0][c]; }
#endif
            if (tz[3] != 0.0) { P[1][c] = tz[0] * P[1][c] + tz[1] * cz; cz = dHy * tz[2] / d + P[1][c]; }
            double curl = cy - cz;
            double En = Ex[c];
            double Enew = mEE[mx] * En + mEH[mx] * curl - mEJ[mx] * Jx[c];
            Jx[c] = ma[mx] * Jx[c] + mb1[mx] * En + mb2[mx] * (Enew - En);
            Ex[c] = Enew;
          }
          /* Ey (i, j+1/2, k) */
          if ((per || j < ny - 1) && xin && zin) {
            double dHx = Hx[c] - Hx[IDX(i, j, km)];
            double dHz = Hz[c] - Hz[IDX(im, j, k)];
            const double* tz = TB(2, 0, k);
            const double* tx = TB(0, 0, i);
            double cz = dHx / d, cx = dHz / d;
            if (tz[3] != 0.0) { P[2][c] = tz[0] * P[2][c] + tz[1] * cz; cz = dHx * tz[2] / d + P[2][c]; }
            if (tx[3] != 0.0) { P[3][c] = tx[0] * P[3][c] + tx[1] * cx; cx = dHz * tx[2] / d + P[3][c]; }
#if defined(OR_MUTANT) && OR_MUTANT == 5
            /* planted mistake: Ey's x term with the wrong sign */
            double curl = cz + cx;
#else
            double curl = cz - cx;
#endif
            double En = Ey[c];
            double Enew = mEE[my] * En + mEH[my] * curl - mEJ[my] * Jy[c];
            Jy[c] = ma[my] * Jy[c] + mb1[my] * En + mb2[my] * (Enew - En);
            Ey[c] = Enew;
          }
          /* Ez (i, j, k+1/2) */
          if (k < nz - 1 && xin && yin) {
            double dHy = Hy[c] - Hy[IDX(im, j, k)];
            double dHx = Hx[c] - Hx[IDX(i, jm, k)];
            const double* tx = TB(0, 0, i);
            const double* ty = TB(1, 0, j);
            double cx = dHy / d, cy = dHx / d;
            if (tx[3] != 0.0) { P[4][c] = tx[0] * P[4][c] + tx[1] * cx; cx = dHy * tx[2] / d + P[4][c]; }
            if (ty[3] != 0.0) { P[5][c] = ty[0] * P[5][c] + ty[1] * cy; cy = dHx * ty[2] / d + P[5][c]; }
            double curl = cx - cy;
            double En = Ez[c];
            double Enew = mEE[mz] * En + mEH[mz] * curl - mEJ[mz] * Jz[c];
            Jz[c] = ma[mz] * Jz[c] + mb1[mz] * En + mb2[mz] * (Enew - En);
            Ez[c] = Enew;
          }
        }
    const double t = (double)(n + 1) * dt;
    if (g->tfsf) {
      /* TF/SF corrections of E: incident Hy at time n+1/2 (vacuum at the box faces) */
      const double f = dt / (O3_EPS0 * d);
      for (int j = j0; j <= j1; ++j)
        for (int i = i0; i <= i1 - 1; ++i) {
          Ex[IDX(i, j, k0)] += f * Hi[k0 - 1 + off];
          Ex[IDX(i, j, k1)] -= f * Hi[k1 + off];
        }
      for (int k = k0; k <= k1 - 1; ++k)
        for (int j = j0; j <= j1; ++j) {
          Ez[IDX(i0, j, k)] -= f * Hi[k + off];
          Ez[IDX(i1, j, k)] += f * Hi[k + off];
        }
      /* 1D incident E, soft source, Mur ends */
      const double e1 = Ei[1], e0 = Ei[0], eN2 = Ei[L1 - 2], eN1 = Ei[L1 - 1];
      for (int mm = 1; mm < L1 - 1; ++mm) Ei[mm] = Ei[mm] - dt / O3_EPS0 * ((Hi[mm] - Hi[mm - 1]) / d);
      Ei[g->inc_src] = Ei[g->inc_src] + o3_pulse(g, t);
      Ei[0] = e1 + q1 * (Ei[1] - e0);
      Ei[L1 - 1] = eN2 + q1 * (Ei[L1 - 2] - eN1);
    }
    if (g->sheet_k >= 0)
      for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) Ex[IDX(i, j, g->sheet_k)] = Ex[IDX(i, j, g->sheet_k)] + o3_pulse(g, t);
    for (int p = 0; p < g->n_probes; ++p) {
      const double e = Ex[IDX(probes[3 * p], probes[3 * p + 1], probes[3 * p + 2])];
      if (series) series[(int64_t)p * n_steps + step] = e;
      for (int f = 0; f < g->n_freq; ++f) {
        const double ph = 2.0 * O3_PI * freq_hz[f] * t;
        X_re[p * g->n_freq + f] += e * cos(ph);
        X_im[p * g->n_freq + f] -= e * sin(ph);
      }
    }
  }
  for (int ax = 0; ax < 3; ++ax)
    for (int h = 0; h < 2; ++h) free(tab[ax][h]);
  free(ma); free(mb1); free(mb2); free(mEE); free(mEH); free(mEJ);
  return 0;
}
