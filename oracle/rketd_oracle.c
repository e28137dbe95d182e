/*
 * rketd_oracle.c -- TEST INFRASTRUCTURE, not part of the product.
 *
 * A plain, serial, FP64 CPU implementation of the RKETD-FDTD scheme for an
 * unmagnetized (Drude) plasma, written directly from the paper's equations in
 * SI units with no normalisation, no blocking and no fusion. It is the oracle
 * that the CUDA library is checked against. Only tests/, the smoke() entry of
 * __graft_entry__ and the cpu_baseline leg of bench.py load this file; the
 * CUDA library never includes, links or calls it, and the two share no code.
 *
 * Compiled with -ffp-contract=off so that every multiply and add rounds on its
 * own. The OpenMP build (-fopenmp) parallelises only the independent per-cell
 * loops, so its fields are bitwise equal to the serial build.
 *
 * Model (paper Sec. II): Eqs. 4-6, the 1D curl equations with the Drude current
 *   -dHy/dz = eps0 dEx/dt + Jx,  dEx/dz = -mu0 dHy/dt,  dJx/dt + nu Jx = eps0 wp^2 Ex.
 * One time step n -> n+1, in the order the paper derives it:
 *   1. H^{n+1/2} from H^{n-1/2} and E^n by Eq. 14 (the printed "dx" read as dz);
 *   2. E^{n+1} from Eq. 12 with J^{n+1} taken from Eq. 11 and solved for E^{n+1}
 *      (the corrected Eq. 13: every term on the right is divided by the
 *      denominator D of the printed E^n coefficient);
 *   3. J^{n+1} from Eq. 11 with E^n and E^{n+1};
 *   4. soft source of Eq. 15 added to E^{n+1} at the source cell;
 *   5. end cells: first-order Mur, or PEC walls behind a CPML or behind the paper's
 *      split-field PML (which replaces steps 1-3 in its layers);
 *   6. running DFT of E^{n+1} at the probe cells.
 * Eq. 11 is used rather than Eq. 10: integrating the linear interpolant of F
 * between t_n and t_{n+1} against e^{nu tau} in Eq. 7 gives Eq. 11's terms.
 * The grid's `scheme` also selects the paper's two other recursions for J (for the
 * accuracy-order comparison): the first-order ETD of Eq. 9 and Eq. 10 read literally
 * (F extrapolated from F_{n-1} and F_n, an explicit second-order ETD); both are explicit
 * in J, and E^{n+1} then follows from Eq. 12 directly.
 *
 * Parity pins: see tests/test_oracle_pins.py (discrete transfer matrix,
 * continuous slab, wp = 0 reduction, nu = 0 energy balance, Courant limit,
 * per-step algebra of Eqs. 11 and 12, CPML reflection).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_EPS0 8.8541878128e-12
#define OR_MU0 1.25663706212e-6
#define OR_PI 3.14159265358979323846

typedef struct {
  int64_t nz;          /* E nodes 0..nz-1; H nodes k+1/2 for k = 0..nz-2 */
  double dz, dt;       /* m, s */
  int32_t bc;          /* 0: first-order Mur at both ends; 1: CPML with PEC outer walls;
                          2: the paper's split-field PML (Sec. III, Sec. IV.B) with PEC outer walls */
  int32_t cpml_cells;  /* CPML / PML thickness in cells (bc == 1, 2) */
  double cpml_m, cpml_sigma_max, cpml_kappa_max, cpml_alpha_max;
  int64_t src_cell;    /* soft source cell */
  double src_tau, src_t0, src_amp;
  int32_t n_probes, n_freq;
  int32_t scheme;      /* current recursion: 0 = Eq. 11 (RKETD), 1 = Eq. 9 (first-order ETD),
                          2 = Eq. 10 read literally (explicit second-order ETD) */
} or_grid1d;

/* phi1(x) = (1 - e^{-x})/x and phi2(x) = (e^{-x} - 1 + x)/x^2 with x = nu*dt: the two
 * integrals that turn Eq. 7 into Eq. 11 ((1 - e^{-nu dt})/nu = dt*phi1 and
 * (e^{-nu dt} - 1 + nu dt)/(nu^2 dt) = dt*phi2). Their limits at x = 0 are 1 and 1/2.
 * For x < 1 the Taylor series sum_k (-x)^k/(k+1)! and sum_k (-x)^k/(k+2)! are summed
 * in nested form (40 terms, truncation below 1e-47); otherwise expm1 avoids the
 * cancellation in 1 - e^{-x}. */
double or_phi1(double x) {
  if (x < 1.0) {
    double s = 1.0;
    for (int j = 41; j >= 2; --j) s = 1.0 + (-x) / (double)j * s;
    return s;
  }
  return -expm1(-x) / x;
}

double or_phi2(double x) {
  if (x < 1.0) {
    double s = 1.0;
    for (int j = 42; j >= 3; --j) s = 1.0 + (-x) / (double)j * s;
    return 0.5 * s;
  }
  return (expm1(-x) + x) / (x * x);
}

/* Eq. 15 soft-source pulse, normalised by tau: amp*((t-t0)/tau)*exp(-(t-t0)^2/(2 tau^2)). */
double or_source(const or_grid1d* g, double t) {
  double u = (t - g->src_t0) / g->src_tau;
  return g->src_amp * u * exp(-0.5 * u * u);
}

/* CPML grading at relative depth rho in (0, 1] (Roden-Gedney convolutional PML):
 * sigma = sigma_max rho^m, kappa = 1 + (kappa_max-1) rho^m, alpha = alpha_max (1-rho),
 * b = exp(-(sigma/kappa + alpha) dt/eps0), c = sigma (b-1) / (sigma kappa + kappa^2 alpha). */
static void or_cpml_point(const or_grid1d* g, double rho, double* b, double* c, double* kappa) {
  double pm = pow(rho, g->cpml_m);
  double sigma = g->cpml_sigma_max * pm;
  double kap = 1.0 + (g->cpml_kappa_max - 1.0) * pm;
  double alpha = g->cpml_alpha_max * (1.0 - rho);
  double bb = exp(-(sigma / kap + alpha) * g->dt / OR_EPS0);
  double den = sigma * kap + kap * kap * alpha;
  *b = bb;
  *c = (sigma == 0.0 || den == 0.0) ? 0.0 : sigma * (bb - 1.0) / den;
  *kappa = kap;
}

/* Relative CPML depth of a node at position x (in cells): 0 outside the layers. */
static double or_cpml_rho(const or_grid1d* g, double x) {
  double n = (double)g->cpml_cells;
  double right_inner = (double)(g->nz - 1) - n;
  if (g->bc != 1 || g->cpml_cells <= 0) return 0.0;
  if (x < n) return (n - x) / n;
  if (x > right_inner) return (x - right_inner) / n;
  return 0.0;
}

/* Relative depth of a node in the split-field PML layers (bc == 2), graded as the CPML. */
static double or_pml_rho(const or_grid1d* g, double x) {
  double n = (double)g->cpml_cells;
  double right_inner = (double)(g->nz - 1) - n;
  if (g->bc != 2 || g->cpml_cells <= 0) return 0.0;
  if (x < n) return (n - x) / n;
  if (x > right_inner) return (x - right_inner) / n;
  return 0.0;
}

/* Validates the problem; returns 0 or a negative code. */
static int or_check(const or_grid1d* g, const int64_t* probe_cells) {
  if (g->nz < 4 || g->dz <= 0 || g->dt <= 0) return -1;
  if (g->src_cell < 1 || g->src_cell > g->nz - 2) return -2;
  for (int p = 0; p < g->n_probes; ++p)
    if (probe_cells[p] < 0 || probe_cells[p] >= g->nz) return -3;
  if ((g->bc == 1 || g->bc == 2) && (g->cpml_cells < 1 || 2 * g->cpml_cells + 2 > g->nz)) return -4;
  if (g->bc < 0 || g->bc > 2) return -4;
  if (g->scheme < 0 || g->scheme > 2) return -6;
  return 0;
}

/*
 * Advances the state (E^n, H^{n-1/2}, J^n, CPML psi) by n_steps steps starting at step
 * index n_start, accumulating the running DFT X_p(f) += E_p^{m} exp(-j 2 pi f m dt) for
 * every new step index m = n_start+1 .. n_start+n_steps. All arrays are SI, caller-owned:
 *   wp2[nz], nu[nz]   plasma frequency squared (rad^2/s^2) and collision frequency (1/s)
 *   E[nz], J[nz], psiE[nz]; H[nz-1], psiH[nz-1]      (in/out)
 *   X_re/X_im[n_probes*n_freq]                        (in/out, accumulated)
 *   series[n_probes*n_steps] (may be NULL): E at each probe after each step.
 *   Eprev[nz] (scheme 2 only, in/out): E^{n-1}, which Eq. 10's F_{n-1} needs; zero at rest.
 * Returns 0, or a negative code for invalid input (nothing is modified then).
 *
 * Schemes 1 and 2 (Eqs. 9 and 10) give J^{n+1} from values at steps n and n-1 only, so the step
 * computes J^{n+1} first and then E^{n+1} from Eq. 12 as printed (no solve is needed):
 *   Eq. 9:  J^{n+1} = e^{-nu dt} J^n + (1 - e^{-nu dt})/nu F_n,  F = eps0 wp^2 E;
 *   Eq. 10: F taken as F_n + (tau/dt)(F_n - F_{n-1}) over the step in Eq. 7, which adds
 *           (e^{-nu dt} - 1 + nu dt)/(nu^2 dt) (F_n - F_{n-1}) to the Eq. 9 value.
 */
int or_run1d(const or_grid1d* g, const double* wp2, const double* nu, const int64_t* probe_cells,
             const double* freq_hz, int64_t n_start, int64_t n_steps, double* E, double* H, double* J,
             double* psiE, double* psiH, double* X_re, double* X_im, double* series, double* Eprev) {
  int rc = or_check(g, probe_cells);
  if (rc) return rc;
  if (g->scheme == 2 && !Eprev) return -7;
  const int64_t nz = g->nz;
  const double dt = g->dt, dz = g->dz;
  /* Per-cell constants of Eqs. 11 and 13, evaluated once. */
  double* a = (double*)malloc(sizeof(double) * nz);
  double* b1 = (double*)malloc(sizeof(double) * nz);
  double* b2 = (double*)malloc(sizeof(double) * nz);
  double* cEE = (double*)malloc(sizeof(double) * nz);
  double* cEH = (double*)malloc(sizeof(double) * nz);
  double* cEJ = (double*)malloc(sizeof(double) * nz);
  double* pbE = (double*)calloc(nz, sizeof(double));
  double* pcE = (double*)calloc(nz, sizeof(double));
  double* pkE = (double*)malloc(sizeof(double) * nz);
  double* pbH = (double*)calloc(nz, sizeof(double));
  double* pcH = (double*)calloc(nz, sizeof(double));
  double* pkH = (double*)malloc(sizeof(double) * nz);
  char* inE = (char*)calloc(nz, 1);
  char* inH = (char*)calloc(nz, 1);
  /* Split-field PML (bc == 2, the paper's boundary, Berenger's PML). In 1D only the z-split field
     exists, so the layer is one graded conductivity sigma on E with the matched magnetic
     conductivity sigma* = sigma mu0/eps0 on H, advanced by exponential differencing:
       E^{n+1} = e^{-sigma dt/eps0} E^n - (1 - e^{-sigma dt/eps0})/(sigma dz) (H_{k+1/2} - H_{k-1/2}),
       H^{n+1/2} = e^{-sigma* dt/mu0} H^{n-1/2} - (1 - e^{-sigma* dt/mu0})/(sigma* dz) (E_{k+1} - E_k),
     sigma = sigma_max rho^m at the node's relative depth rho, as the CPML (sigma* dt/mu0 = sigma dt/eps0).
     The layer is vacuum: no current. */
  double* paE = (double*)calloc(nz, sizeof(double));
  double* pfE = (double*)calloc(nz, sizeof(double));
  double* paH = (double*)calloc(nz, sizeof(double));
  double* pfH = (double*)calloc(nz, sizeof(double));
  char* inPE = (char*)calloc(nz, 1);
  char* inPH = (char*)calloc(nz, 1);
  for (int64_t k = 0; k < nz; ++k) {
    for (int h = 0; h < 2; ++h) {
      if (h == 1 && k == nz - 1) continue;
      double rho = or_pml_rho(g, (double)k + 0.5 * h);
      if (rho <= 0.0) continue;
      double sigma = g->cpml_sigma_max * pow(rho, g->cpml_m);
      double xs = sigma * dt / OR_EPS0;
      /* (1 - e^{-x})/(sigma dz) = dt/(eps0 dz) phi1(x); for H with sigma*: dt/(mu0 dz) phi1(x) */
      if (h == 0) {
        inPE[k] = 1;
        paE[k] = exp(-xs);
        pfE[k] = dt / (OR_EPS0 * dz) * or_phi1(xs);
      } else {
        inPH[k] = 1;
        paH[k] = exp(-xs);
        pfH[k] = dt / (OR_MU0 * dz) * or_phi1(xs);
#if defined(OR_MUTANT) && OR_MUTANT == 10
        /* planted mistake: no magnetic conductivity (sigma* = 0), an unmatched layer */
        paH[k] = 1.0;
        pfH[k] = dt / (OR_MU0 * dz);
#endif
      }
    }
    if (inPE[k] && wp2[k] != 0.0) {
      free(a); free(b1); free(b2); free(cEE); free(cEH); free(cEJ);
      free(pbE); free(pcE); free(pkE); free(pbH); free(pcH); free(pkH); free(inE); free(inH);
      free(paE); free(pfE); free(paH); free(pfH); free(inPE); free(inPH);
      return -8;  /* the split-field PML layers are vacuum */
    }
  }
  for (int64_t k = 0; k < nz; ++k) {
    double x = nu[k] * dt;
    /* Eq. 11: J^{n+1} = a J^n + beta1 E^n + beta2 (E^{n+1} - E^n) with
       a = e^{-nu dt}, beta1 = eps0 wp^2 (1 - a)/nu, beta2 = eps0 wp^2 (a - 1 + nu dt)/(nu^2 dt). */
    a[k] = exp(-x);
    b1[k] = OR_EPS0 * wp2[k] * dt * or_phi1(x);
    b2[k] = OR_EPS0 * wp2[k] * dt * or_phi2(x);
    /* Eq. 12 with Eq. 11 substituted and solved for E^{n+1} (Eq. 13 with the /D on every term):
       D E^{n+1} = (1 - dt/(2 eps0) (beta1 - beta2)) E^n - dt/eps0 curlH - dt/(2 eps0) (1 + a) J^n,
       D = 1 + dt/(2 eps0) beta2. */
    double D = 1.0 + dt / (2.0 * OR_EPS0) * b2[k];
    cEE[k] = (1.0 - dt / (2.0 * OR_EPS0) * (b1[k] - b2[k])) / D;
    cEH[k] = (dt / OR_EPS0) / D;
    cEJ[k] = (dt / (2.0 * OR_EPS0)) * (1.0 + a[k]) / D;
    pkE[k] = 1.0;
    pkH[k] = 1.0;
    double rE = or_cpml_rho(g, (double)k);
    if (rE > 0.0) {
      inE[k] = 1;
      or_cpml_point(g, rE, &pbE[k], &pcE[k], &pkE[k]);
    }
    if (k < nz - 1) {
      double rH = or_cpml_rho(g, (double)k + 0.5);
      if (rH > 0.0) {
        inH[k] = 1;
        or_cpml_point(g, rH, &pbH[k], &pcH[k], &pkH[k]);
      }
    }
  }
  /* Mur coefficient (S-1)/(S+1), S = c dt/dz with c = 1/sqrt(mu0 eps0). */
  const double S = dt / (sqrt(OR_MU0 * OR_EPS0) * dz);
  const double q = (S - 1.0) / (S + 1.0);
#if defined(OR_MUTANT) && OR_MUTANT == 4
  /* planted mistake: Mur coefficient with the wrong sign */
  const double qq = -q;
#define q qq
#endif

  for (int64_t step = 0; step < n_steps; ++step) {
    const int64_t n = n_start + step; /* advancing E^n -> E^{n+1} */
    /* 1. Eq. 14: H^{n+1/2}_{k+1/2} = H^{n-1/2}_{k+1/2} - dt/(mu0 dz) (E^n_{k+1} - E^n_k). */
#ifdef _OPENMP
#pragma omp parallel for schedule(static) if (nz > 8192)
#endif
    for (int64_t k = 0; k < nz - 1; ++k) {
      double dE = E[k + 1] - E[k];
      if (inPH[k]) { /* split-field PML */
        H[k] = paH[k] * H[k] - pfH[k] * dE;
        continue;
      }
      double curl;
      if (inH[k]) {
        psiH[k] = pbH[k] * psiH[k] + pcH[k] * (dE / dz);
        curl = dE / (pkH[k] * dz) + psiH[k];
      } else {
        curl = dE / dz;
      }
      H[k] = H[k] - dt / OR_MU0 * curl;
    }
    const double E0_old = E[0], E1_old = E[1];
    const double ENm1_old = E[nz - 1], ENm2_old = E[nz - 2];
    /* 2-3. Eq. 13 (corrected) for E^{n+1}, then Eq. 11 for J^{n+1}. */
#ifdef _OPENMP
#pragma omp parallel for schedule(static) if (nz > 8192)
#endif
    for (int64_t k = 1; k < nz - 1; ++k) {
      double dH = H[k] - H[k - 1];
      if (inPE[k]) { /* split-field PML */
        E[k] = paE[k] * E[k] - pfE[k] * dH;
        continue;
      }
      double curl;
      if (inE[k]) {
        psiE[k] = pbE[k] * psiE[k] + pcE[k] * (dH / dz);
        curl = dH / (pkE[k] * dz) + psiE[k];
      } else {
        curl = dH / dz;
      }
      double En = E[k];
      if (g->scheme == 0) {
      double Enew = cEE[k] * En - cEH[k] * curl - cEJ[k] * J[k];
#if defined(OR_MUTANT) && OR_MUTANT == 1
      /* planted mistake: Eq. 13 as printed (no 1/D on the curl and J terms) */
      Enew = cEE[k] * En - (dt / OR_EPS0) * curl - (dt / (2.0 * OR_EPS0)) * (1.0 + a[k]) * J[k];
#endif
#if defined(OR_MUTANT) && OR_MUTANT == 2
      /* planted mistake: E^n and E^{n+1} swapped in the last term of Eq. 11 */
      J[k] = a[k] * J[k] + b1[k] * En + b2[k] * (En - Enew);
#else
      J[k] = a[k] * J[k] + b1[k] * En + b2[k] * (Enew - En);
#endif
      E[k] = Enew;
      } else {
        /* Eq. 9 (b1 = eps0 wp^2 dt phi1 = eps0 wp^2 (1 - a)/nu), then Eq. 10's extra term */
        double Jnew = a[k] * J[k] + b1[k] * En;
        if (g->scheme == 2) {
#if defined(OR_MUTANT) && OR_MUTANT == 9
          /* planted mistake: F_{n-1} - F_n in place of F_n - F_{n-1} in Eq. 10 */
          Jnew = Jnew + b2[k] * (Eprev[k] - En);
#else
          Jnew = Jnew + b2[k] * (En - Eprev[k]);
#endif
          Eprev[k] = En;
        }
        /* Eq. 12 with J^{n+1} and J^n */
        E[k] = En - dt / OR_EPS0 * curl - dt / (2.0 * OR_EPS0) * (Jnew + J[k]);
        J[k] = Jnew;
      }
    }
    /* 4. Eq. 15 soft source at t = (n+1) dt. */
    E[g->src_cell] = E[g->src_cell] + or_source(g, (double)(n + 1) * dt);
    /* 5. End cells. */
    if (g->bc == 1 || g->bc == 2) {
      E[0] = 0.0;
      E[nz - 1] = 0.0;
    } else {
      E[0] = E1_old + q * (E[1] - E0_old);
      E[nz - 1] = ENm2_old + q * (E[nz - 2] - ENm1_old);
    }
    /* 6. Running DFT at the probes. */
    const double t = (double)(n + 1) * dt;
    for (int p = 0; p < g->n_probes; ++p) {
      const double e = E[probe_cells[p]];
      if (series) series[(int64_t)p * n_steps + step] = e;
      for (int f = 0; f < g->n_freq; ++f) {
        const double ph = 2.0 * OR_PI * freq_hz[f] * t;
        X_re[p * g->n_freq + f] += e * cos(ph);
#if defined(OR_MUTANT) && OR_MUTANT == 3
        /* planted mistake: DFT kernel e^{+j w t} */
        X_im[p * g->n_freq + f] += e * sin(ph);
#else
        X_im[p * g->n_freq + f] -= e * sin(ph);
#endif
      }
    }
  }
  free(a); free(b1); free(b2); free(cEE); free(cEH); free(cEJ);
  free(pbE); free(pcE); free(pkE); free(pbH); free(pcH); free(pkH); free(inE); free(inH);
  free(paE); free(pfE); free(paH); free(pfH); free(inPE); free(inPH);
  return 0;
}


/* ------------------------------------------------------------------------------------------
 * Adjoint (reverse mode) of the Mur-terminated scheme, for gradients of a loss that depends on
 * the running DFT at the probes. Plain form: the forward trajectory is stored whole (state
 * before every step) and the steps are transposed one at a time in reverse order.
 * ------------------------------------------------------------------------------------------ */

/* d phi1/dx and d phi2/dx. For x < 1 the term-by-term derivatives of the Taylor series of
 * or_phi1/or_phi2, sum_j (j+1)(-1)^(j+1) x^j/(j+2)! and sum_j (j+1)(-1)^(j+1) x^j/(j+3)!, are
 * summed from the smallest term (40 terms); otherwise (a - phi1)/x and (phi1 - 2 phi2)/x. */
double or_dphi1(double x) {
  if (x < 1.0) {
    double terms[40];
    double fact = 2.0; /* (j+2)! */
    double xp = 1.0;   /* x^j */
    for (int j = 0; j < 40; ++j) {
      terms[j] = (double)(j + 1) * xp / fact * ((j % 2 == 0) ? -1.0 : 1.0);
      xp *= x;
      fact *= (double)(j + 3);
    }
    double s = 0.0;
    for (int j = 39; j >= 0; --j) s += terms[j];
    return s;
  }
  return (exp(-x) - or_phi1(x)) / x;
}

double or_dphi2(double x) {
  if (x < 1.0) {
    double terms[40];
    double fact = 6.0; /* (j+3)! */
    double xp = 1.0;
    for (int j = 0; j < 40; ++j) {
      terms[j] = (double)(j + 1) * xp / fact * ((j % 2 == 0) ? -1.0 : 1.0);
      xp *= x;
      fact *= (double)(j + 4);
    }
    double s = 0.0;
    for (int j = 39; j >= 0; --j) s += terms[j];
    return s;
  }
  return (or_phi1(x) - 2.0 * or_phi2(x)) / x;
}

/* Per-cell constants of Eqs. 11 and 13 (as in or_run1d) and their derivatives with respect to
 * wp2 (index 0) and nu (index 1):
 *   a = e^{-nu dt}, b1 = eps0 wp2 dt phi1, b2 = eps0 wp2 dt phi2, D = 1 + h b2 (h = dt/(2 eps0)),
 *   cEE = (1 - h (b1 - b2))/D, cEH = (dt/eps0)/D, cEJ = h (1 + a)/D. */
typedef struct {
  double a, b1, b2, cEE, cEH, cEJ;
  double da[2], db1[2], db2[2], dcEE[2], dcEH[2], dcEJ[2];
} or_cell;

static void or_cell_consts(double wp2, double nu, double dt, or_cell* c) {
  const double x = nu * dt;
  const double h = dt / (2.0 * OR_EPS0);
  const double p1 = or_phi1(x), p2 = or_phi2(x);
  c->a = exp(-x);
  c->b1 = OR_EPS0 * wp2 * dt * p1;
  c->b2 = OR_EPS0 * wp2 * dt * p2;
  const double D = 1.0 + dt / (2.0 * OR_EPS0) * c->b2;
  c->cEE = (1.0 - dt / (2.0 * OR_EPS0) * (c->b1 - c->b2)) / D;
  c->cEH = (dt / OR_EPS0) / D;
  c->cEJ = (dt / (2.0 * OR_EPS0)) * (1.0 + c->a) / D;
  c->da[0] = 0.0;
  c->da[1] = -dt * c->a;
  c->db1[0] = OR_EPS0 * dt * p1;
  c->db1[1] = OR_EPS0 * wp2 * dt * dt * or_dphi1(x);
  c->db2[0] = OR_EPS0 * dt * p2;
  c->db2[1] = OR_EPS0 * wp2 * dt * dt * or_dphi2(x);
  for (int q = 0; q < 2; ++q) {
    const double dD = h * c->db2[q];
    c->dcEE[q] = (-h * (c->db1[q] - c->db2[q]) - c->cEE * dD) / D;
    c->dcEH[q] = -c->cEH * dD / D;
    c->dcEJ[q] = (h * c->da[q] - c->cEJ * dD) / D;
  }
}

/* One transposed step. On entry (lE, lH, lJ) is the adjoint of the state after step n
 * (E^{n+1}, H^{n+1/2}, J^{n+1}); on exit the adjoint of the state before it. If the forward
 * values (E^n, J^n, H^{n+1/2}, E^{n+1} before the source) are given, gW/gN accumulate
 * lambda^{n+1} . d(step)/d(wp2_k) and d/d(nu_k) for every interior cell. Scratch: tmp[3 nz]. */
static void or_adjoint_step_impl(const or_grid1d* g, const or_cell* cell, double* lE, double* lH, double* lJ,
                                 const double* En, const double* Jn, const double* Hh, const double* Enew,
                                 double* gW, double* gN, double* tmp) {
  const int64_t nz = g->nz;
  const double dt = g->dt, dz = g->dz;
  const double S = dt / (sqrt(OR_MU0 * OR_EPS0) * dz);
  const double q = (S - 1.0) / (S + 1.0);
  double* lEpre = tmp;       /* adjoint of E^n */
  double* lHpost = tmp + nz; /* adjoint of H^{n+1/2} (after the H update) */
  for (int64_t k = 0; k < nz; ++k) lEpre[k] = 0.0;
  for (int64_t k = 0; k < nz - 1; ++k) lHpost[k] = lH[k];
  /* 5. Mur ends: E_0' = E_1 + q (E_1' - E_0), E_{N-1}' = E_{N-2} + q (E_{N-2}' - E_{N-1}). */
  lE[1] += q * lE[0];
  lEpre[1] += lE[0];
  lEpre[0] += -q * lE[0];
  lE[0] = 0.0;
  lE[nz - 2] += q * lE[nz - 1];
  lEpre[nz - 2] += lE[nz - 1];
  lEpre[nz - 1] += -q * lE[nz - 1];
  lE[nz - 1] = 0.0;
  /* 4. the source is additive: nothing to transpose. */
  /* 2-3. interior E (Eq. 13) and J (Eq. 11). */
  for (int64_t k = 1; k < nz - 1; ++k) {
    const or_cell* c = &cell[k];
    const double lJp = lJ[k];
    const double mu = lE[k] + c->b2 * lJp; /* adjoint of E^{n+1}_k through both outputs */
    if (gW && En) {
      const double dH = Hh[k] - Hh[k - 1];
      for (int qq = 0; qq < 2; ++qq) {
        const double dEn = c->dcEE[qq] * En[k] - c->dcEH[qq] * (dH / dz) - c->dcEJ[qq] * Jn[k];
        const double dJn = c->da[qq] * Jn[k] + c->db1[qq] * En[k] + c->db2[qq] * (Enew[k] - En[k]);
        const double gval = mu * dEn + lJp * dJn;
        if (qq == 0) gW[k] += gval; else gN[k] += gval;
      }
    }
    lEpre[k] += c->cEE * mu + (c->b1 - c->b2) * lJp;
    lJ[k] = -c->cEJ * mu + c->a * lJp;
    lHpost[k] += -c->cEH / dz * mu;
    lHpost[k - 1] += c->cEH / dz * mu;
  }
  /* J at the two end cells is not updated: its adjoint passes through. */
  /* 1. Eq. 14: H' = H - dt/(mu0 dz) (E_{k+1} - E_k). */
  const double cH = dt / (OR_MU0 * dz);
  for (int64_t k = 0; k < nz - 1; ++k) {
    lEpre[k + 1] += -cH * lHpost[k];
    lEpre[k] += cH * lHpost[k];
    lH[k] = lHpost[k];
  }
  for (int64_t k = 0; k < nz; ++k) lE[k] = lEpre[k];
}

/* Transposed single step without gradients (for dot-product tests): (lE, lH, lJ) in place. */
int or_adjoint_step(const or_grid1d* g, const double* wp2, const double* nu, double* lE, double* lH, double* lJ) {
  if (g->bc != 0 || g->scheme != 0 || g->nz < 4) return -1;
  or_cell* cell = (or_cell*)malloc(sizeof(or_cell) * g->nz);
  double* tmp = (double*)malloc(sizeof(double) * 3 * g->nz);
  for (int64_t k = 0; k < g->nz; ++k) or_cell_consts(wp2[k], nu[k], g->dt, &cell[k]);
  or_adjoint_step_impl(g, cell, lE, lH, lJ, NULL, NULL, NULL, NULL, NULL, NULL, tmp);
  free(cell);
  free(tmp);
  return 0;
}

/*
 * Gradient of a loss L(X) of the probe spectra after n_steps steps from rest, with respect to
 * wp2 and nu of every cell. gXr/gXi [n_probes*n_freq] are dL/dRe X and dL/dIm X. The forward
 * run is or_run1d one step at a time (states stored); the seed of sample m at probe p is
 * dL/dE_p^m = sum_f (gXr cos(2 pi f m dt) - gXi sin(2 pi f m dt)). Mur ends only.
 * Outputs grad_wp2[nz], grad_nu[nz] (overwritten). Returns 0 or a negative code.
 */
int or_adjoint1d(const or_grid1d* g, const double* wp2, const double* nu, const int64_t* probe_cells,
                 const double* freq_hz, int64_t n_steps, const double* gXr, const double* gXi, double* grad_wp2,
                 double* grad_nu) {
  int rc = or_check(g, probe_cells);
  if (rc) return rc;
  if (g->bc != 0 || g->scheme != 0) return -5;
  const int64_t nz = g->nz;
  const int64_t N = n_steps;
  double* Et = (double*)calloc((size_t)(N + 1) * nz, sizeof(double));
  double* Ht = (double*)calloc((size_t)(N + 1) * (nz - 1), sizeof(double));
  double* Jt = (double*)calloc((size_t)(N + 1) * nz, sizeof(double));
  double* psiE = (double*)calloc(nz, sizeof(double));
  double* psiH = (double*)calloc(nz, sizeof(double));
  double* xr = (double*)calloc((size_t)g->n_probes * g->n_freq + 1, sizeof(double));
  double* xi = (double*)calloc((size_t)g->n_probes * g->n_freq + 1, sizeof(double));
  double* E = (double*)calloc(nz, sizeof(double));
  double* H = (double*)calloc(nz, sizeof(double));
  double* J = (double*)calloc(nz, sizeof(double));
  /* forward: state n stored before step n */
  for (int64_t n = 0; n < N; ++n) {
    memcpy(Et + n * nz, E, sizeof(double) * nz);
    memcpy(Ht + n * (nz - 1), H, sizeof(double) * (nz - 1));
    memcpy(Jt + n * nz, J, sizeof(double) * nz);
    or_run1d(g, wp2, nu, probe_cells, freq_hz, n, 1, E, H, J, psiE, psiH, xr, xi, NULL, NULL);
  }
  memcpy(Et + N * nz, E, sizeof(double) * nz);
  memcpy(Ht + N * (nz - 1), H, sizeof(double) * (nz - 1));
  memcpy(Jt + N * nz, J, sizeof(double) * nz);
  /* reverse */
  or_cell* cell = (or_cell*)malloc(sizeof(or_cell) * nz);
  for (int64_t k = 0; k < nz; ++k) or_cell_consts(wp2[k], nu[k], g->dt, &cell[k]);
  double* lE = (double*)calloc(nz, sizeof(double));
  double* lH = (double*)calloc(nz, sizeof(double));
  double* lJ = (double*)calloc(nz, sizeof(double));
  double* tmp = (double*)malloc(sizeof(double) * 3 * nz);
  double* Enew = (double*)malloc(sizeof(double) * nz);
  for (int64_t k = 0; k < nz; ++k) grad_wp2[k] = grad_nu[k] = 0.0;
  for (int64_t n = N - 1; n >= 0; --n) {
    const int64_t m = n + 1;
    const double t = (double)m * g->dt;
    for (int p = 0; p < g->n_probes; ++p) {
      double seed = 0.0;
      for (int f = 0; f < g->n_freq; ++f) {
        const double ph = 2.0 * OR_PI * freq_hz[f] * t;
        seed += gXr[p * g->n_freq + f] * cos(ph) - gXi[p * g->n_freq + f] * sin(ph);
      }
      lE[probe_cells[p]] += seed;
    }
    /* E^{n+1} before the source was added */
    memcpy(Enew, Et + m * nz, sizeof(double) * nz);
    Enew[g->src_cell] -= or_source(g, t);
    or_adjoint_step_impl(g, cell, lE, lH, lJ, Et + n * nz, Jt + n * nz, Ht + m * (nz - 1), Enew, grad_wp2, grad_nu,
                         tmp);
  }
  free(Et); free(Ht); free(Jt); free(psiE); free(psiH); free(xr); free(xi); free(E); free(H); free(J);
  free(cell); free(lE); free(lH); free(lJ); free(tmp); free(Enew);
  return 0;
}

/* Number of OpenMP threads this build uses (1 for the serial build). */
int or_threads(void) {
#ifdef _OPENMP
  int n = 1;
#pragma omp parallel
  {
#pragma omp single
    n = omp_get_num_threads();
  }
  return n;
#else
  return 1;
#endif
}
