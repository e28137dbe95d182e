/*
 * rketd_oracle2d.c -- TEST INFRASTRUCTURE, not part of the product.
 *
 * Plain serial FP64 2D Yee RKETD-FDTD in SI units: Eqs. 1-3 with fields uniform along z (the
 * paper's stated 2D generalisation, Sec. IV.B closing remarks and Sec. V), discretised component by
 * component exactly as the 1D oracle discretises Eqs. 12, 11 and 14. Two polarisations:
 *   TMz: Ez (i, j), Hx (i, j+1/2), Hy (i+1/2, j), current Jz with Ez;
 *   TEz: Hz (i+1/2, j+1/2), Ex (i+1/2, j), Ey (i, j+1/2), currents Jx, Jy with Ex, Ey.
 * Arrays are [j][i] (x fastest), nx x ny entries each. Every E component of cell (i, j) takes the
 * Drude material of that cell: mat[j][i] indexes mat_wp2 / mat_nu (0 = vacuum).
 * Boundaries: first-order Mur on the E components tangential to the y faces (rows j = 0 and
 * j = ny-1); in x either periodic, or first-order Mur on the E components tangential to the x faces
 * (columns i = 0 and i = nx-1; TMz Ez, TEz Ey). Source: a soft line source on row src_j adding
 * profile[i] s(t) to Ez (TMz) or Ex (TEz) after the E update, s the Eq. 15 pulse, on the nodes that
 * exist (with Mur x ends TEz has no Ex at i = nx-1, position nx-1/2, so that node stays 0). Probes
 * sample Ez (TMz) or Ex (TEz); running DFT as the 1D oracle.
 * One step: H (Eq. 14 in curl form), then E with J (Eq. 12 with Eq. 11 substituted, solved for
 * E^{n+1}, and Eq. 11), the source, the Mur ends, the probes.
 * Only tests/ and bench.py's CPU legs load this file; it shares no code with the CUDA path.
 * Pins: tests/test_oracle2d_pins.py (reduction to the 1D oracle at normal incidence, the lattice
 * recurrence of a single 2D Fourier mode, the oblique response of a layer against the lattice model).
 * OR_MUTANT 11-13 plant one mistake each (tests only).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

#define O2_EPS0 8.8541878128e-12
#define O2_MU0 1.25663706212e-6
#define O2_PI 3.14159265358979323846

double or_phi1(double x);
double or_phi2(double x);

typedef struct {
  int32_t nx, ny;
  double d, dt;          /* cell size (m), time step (s) */
  int32_t pol;           /* 0: TMz (Ez, Hx, Hy); 1: TEz (Hz, Ex, Ey) */
  int32_t periodic_x;    /* 1: periodic in x; 0: first-order Mur at the x faces */
  int32_t src_j;         /* soft line source row */
  double src_tau, src_t0, src_amp;
  int32_t n_probes, n_freq;
} or_grid2d;

static double o2_pulse(const or_grid2d* g, double t) {
  double u = (t - g->src_t0) / g->src_tau;
  return g->src_amp * u * exp(-0.5 * u * u);
}

#define I2(i, j) ((int64_t)(j) * nx + (i))

/*
 * Advances n_steps steps from step n_start. fields [6][nx*ny]: TMz (Ez, Hx, Hy, Jz, -, -), TEz
 * (Ex, Ey, Hz, Jx, Jy, -), SI, in/out. profile[nx]: source weight per column. probes [n_probes*2]
 * (i, j). X_re/X_im [n_probes*n_freq] accumulated; series [n_probes*n_steps] optional.
 * Returns 0 or a negative code.
 */
int or_run2d(const or_grid2d* g, const uint8_t* mat, const double* mat_wp2, const double* mat_nu, int32_t n_mat,
             const double* profile, const int32_t* probes, const double* freq_hz, int64_t n_start, int64_t n_steps,
             double* fields, double* X_re, double* X_im, double* series) {
  const int nx = g->nx, ny = g->ny;
  const int64_t N = (int64_t)nx * ny;
  const double dt = g->dt, d = g->d;
  const int per = g->periodic_x;
  if (nx < 4 || ny < 4 || g->src_j < 1 || g->src_j > ny - 2 || n_mat < 1) return -1;
  for (int64_t c = 0; c < N; ++c)
    if (mat[c] >= n_mat) return -2;
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
    mb1[m] = O2_EPS0 * mat_wp2[m] * dt * or_phi1(x);
    mb2[m] = O2_EPS0 * mat_wp2[m] * dt * or_phi2(x);
    double D = 1.0 + dt / (2.0 * O2_EPS0) * mb2[m];
    mEE[m] = (1.0 - dt / (2.0 * O2_EPS0) * (mb1[m] - mb2[m])) / D;
    mEH[m] = (dt / O2_EPS0) / D;
    mEJ[m] = (dt / (2.0 * O2_EPS0)) * (1.0 + ma[m]) / D;
  }
  const double cH = dt / O2_MU0;
  const double S = dt / (sqrt(O2_MU0 * O2_EPS0) * d);
  const double q = (S - 1.0) / (S + 1.0);
  double* oldc = (double*)malloc(sizeof(double) * 4 * (nx > ny ? nx : ny));
  double* F0 = fields;
  double* F1 = fields + N;
  double* F2 = fields + 2 * N;
  double* F3 = fields + 3 * N;
  double* F4 = fields + 4 * N;

  for (int64_t step = 0; step < n_steps; ++step) {
    const int64_t n = n_start + step;
    const double t = (double)(n + 1) * dt;
    if (g->pol == 0) {
      double *Ez = F0, *Hx = F1, *Hy = F2, *Jz = F3;
      /* ---- H: dHx/dt = -(1/mu0) dEz/dy, dHy/dt = (1/mu0) dEz/dx ---- */
      for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
          const int64_t c = I2(i, j);
          if (j + 1 < ny) Hx[c] = Hx[c] - cH * ((Ez[I2(i, j + 1)] - Ez[c]) / d);
          const int ip = i + 1 < nx ? i + 1 : (per ? 0 : -1);
#if defined(OR_MUTANT) && OR_MUTANT == 11
          /* planted mistake: Hy's x term with the wrong sign */
          if (ip >= 0) Hy[c] = Hy[c] - cH * ((Ez[I2(ip, j)] - Ez[c]) / d);
#else
          if (ip >= 0) Hy[c] = Hy[c] + cH * ((Ez[I2(ip, j)] - Ez[c]) / d);
#endif
        }
      /* old boundary values for Mur: rows 0, 1, ny-2, ny-1 (and columns 0, 1, nx-2, nx-1) */
      double* oy = oldc;  /* [4][nx] */
      for (int i = 0; i < nx; ++i) {
        oy[i] = Ez[I2(i, 0)];
        oy[nx + i] = Ez[I2(i, 1)];
        oy[2 * nx + i] = Ez[I2(i, ny - 2)];
        oy[3 * nx + i] = Ez[I2(i, ny - 1)];
      }
      double* ox = (double*)malloc(sizeof(double) * 4 * ny);
      for (int j = 0; j < ny; ++j) {
        ox[j] = Ez[I2(0, j)];
        ox[ny + j] = Ez[I2(1, j)];
        ox[2 * ny + j] = Ez[I2(nx - 2, j)];
        ox[3 * ny + j] = Ez[I2(nx - 1, j)];
      }
      /* ---- Ez and Jz: eps0 dEz/dt = dHy/dx - dHx/dy - Jz ---- */
      for (int j = 1; j < ny - 1; ++j)
        for (int i = 0; i < nx; ++i) {
          if (!per && (i == 0 || i == nx - 1)) continue;
          const int64_t c = I2(i, j);
          const int im = i > 0 ? i - 1 : nx - 1;
          const double curl = (Hy[c] - Hy[I2(im, j)]) / d - (Hx[c] - Hx[I2(i, j - 1)]) / d;
          const int m = mat[c];
          const double En = Ez[c];
          const double Enew = mEE[m] * En + mEH[m] * curl - mEJ[m] * Jz[c];
          Jz[c] = ma[m] * Jz[c] + mb1[m] * En + mb2[m] * (Enew - En);
          Ez[c] = Enew;
        }
      for (int i = 0; i < nx; ++i) Ez[I2(i, g->src_j)] = Ez[I2(i, g->src_j)] + profile[i] * o2_pulse(g, t);
      if (!per)
        for (int j = 1; j < ny - 1; ++j) {
          Ez[I2(0, j)] = ox[ny + j] + q * (Ez[I2(1, j)] - ox[j]);
          Ez[I2(nx - 1, j)] = ox[2 * ny + j] + q * (Ez[I2(nx - 2, j)] - ox[3 * ny + j]);
        }
      for (int i = 0; i < nx; ++i) {
        Ez[I2(i, 0)] = oy[nx + i] + q * (Ez[I2(i, 1)] - oy[i]);
        Ez[I2(i, ny - 1)] = oy[2 * nx + i] + q * (Ez[I2(i, ny - 2)] - oy[3 * nx + i]);
      }
      free(ox);
    } else {
      double *Ex = F0, *Ey = F1, *Hz = F2, *Jx = F3, *Jy = F4;
      /* ---- Hz: dHz/dt = (1/mu0) (dEx/dy - dEy/dx) at (i+1/2, j+1/2) ---- */
      for (int j = 0; j < ny - 1; ++j)
        for (int i = 0; i < nx; ++i) {
          const int ip = i + 1 < nx ? i + 1 : (per ? 0 : -1);
          if (ip < 0) continue;
          const int64_t c = I2(i, j);
#if defined(OR_MUTANT) && OR_MUTANT == 13
          /* planted mistake: Hz's x difference taken at the wrong Ey pair */
          Hz[c] = Hz[c] + cH * ((Ex[I2(i, j + 1)] - Ex[c]) / d - (Ey[c] - Ey[I2(i > 0 ? i - 1 : nx - 1, j)]) / d);
#else
          Hz[c] = Hz[c] + cH * ((Ex[I2(i, j + 1)] - Ex[c]) / d - (Ey[I2(ip, j)] - Ey[c]) / d);
#endif
        }
      double* oy = oldc;  /* Ex rows 0, 1, ny-2, ny-1 */
      for (int i = 0; i < nx; ++i) {
        oy[i] = Ex[I2(i, 0)];
        oy[nx + i] = Ex[I2(i, 1)];
        oy[2 * nx + i] = Ex[I2(i, ny - 2)];
        oy[3 * nx + i] = Ex[I2(i, ny - 1)];
      }
      double* ox = (double*)malloc(sizeof(double) * 4 * ny); /* Ey columns 0, 1, nx-2, nx-1 */
      for (int j = 0; j < ny; ++j) {
        ox[j] = Ey[I2(0, j)];
        ox[ny + j] = Ey[I2(1, j)];
        ox[2 * ny + j] = Ey[I2(nx - 2, j)];
        ox[3 * ny + j] = Ey[I2(nx - 1, j)];
      }
      /* ---- Ex (i+1/2, j): eps0 dEx/dt = dHz/dy - Jx, interior rows ---- */
      for (int j = 1; j < ny - 1; ++j)
        for (int i = 0; i < nx; ++i) {
          if (!per && i == nx - 1) continue;  /* Ex exists for i + 1/2 < nx - 1 */
          const int64_t c = I2(i, j);
          const double curl = (Hz[c] - Hz[I2(i, j - 1)]) / d;
          const int m = mat[c];
          const double En = Ex[c];
          const double Enew = mEE[m] * En + mEH[m] * curl - mEJ[m] * Jx[c];
          Jx[c] = ma[m] * Jx[c] + mb1[m] * En + mb2[m] * (Enew - En);
          Ex[c] = Enew;
        }
      /* ---- Ey (i, j+1/2): eps0 dEy/dt = -dHz/dx - Jy ---- */
      for (int j = 0; j < ny - 1; ++j)
        for (int i = 0; i < nx; ++i) {
          if (!per && (i == 0 || i == nx - 1)) continue;
          const int64_t c = I2(i, j);
          const int im = i > 0 ? i - 1 : nx - 1;
          const double curl = -((Hz[c] - Hz[I2(im, j)]) / d);
#if defined(OR_MUTANT) && OR_MUTANT == 12
          /* planted mistake: Ey (i, j+1/2) takes the material of row j + 1 */
          const int m = mat[I2(i, j + 1)];
#else
          const int m = mat[c];
#endif
          const double En = Ey[c];
          const double Enew = mEE[m] * En + mEH[m] * curl - mEJ[m] * Jy[c];
          Jy[c] = ma[m] * Jy[c] + mb1[m] * En + mb2[m] * (Enew - En);
          Ey[c] = Enew;
        }
      /* the source drives only Ex nodes that exist: with Mur x ends, Ex (nx-1/2, j) is outside */
      for (int i = 0; i < (per ? nx : nx - 1); ++i)
        Ex[I2(i, g->src_j)] = Ex[I2(i, g->src_j)] + profile[i] * o2_pulse(g, t);
      if (!per)
        for (int j = 0; j < ny - 1; ++j) {
          Ey[I2(0, j)] = ox[ny + j] + q * (Ey[I2(1, j)] - ox[j]);
          Ey[I2(nx - 1, j)] = ox[2 * ny + j] + q * (Ey[I2(nx - 2, j)] - ox[3 * ny + j]);
        }
      for (int i = 0; i < nx; ++i) {
        Ex[I2(i, 0)] = oy[nx + i] + q * (Ex[I2(i, 1)] - oy[i]);
        Ex[I2(i, ny - 1)] = oy[2 * nx + i] + q * (Ex[I2(i, ny - 2)] - oy[3 * nx + i]);
      }
      free(ox);
    }
    for (int p = 0; p < g->n_probes; ++p) {
      const double e = F0[I2(probes[2 * p], probes[2 * p + 1])];
      if (series) series[(int64_t)p * n_steps + step] = e;
      for (int f = 0; f < g->n_freq; ++f) {
        const double ph = 2.0 * O2_PI * freq_hz[f] * t;
        X_re[p * g->n_freq + f] += e * cos(ph);
        X_im[p * g->n_freq + f] -= e * sin(ph);
      }
    }
  }
  free(oldc);
  free(ma); free(mb1); free(mb2); free(mEE); free(mEH); free(mEJ);
  return 0;
}
