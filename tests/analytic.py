"""Closed forms that pin the FP64 oracle (test infrastructure).

Nothing here calls the oracle or the CUDA library; every formula is derived
from the paper's equations or from textbook electromagnetics:

* `lattice_eps`   -- permittivity of the *discrete* RKETD-Yee scheme at one
  frequency: substituting E^n_k = E_k z^n, H at z^{n+1/2}, z = e^{j w dt} into
  Eqs. 11, 12 and 14 gives E_{k+1} - 2 E_k + E_{k-1} = -q_k E_k with
  q_k = (2 sin(theta/2)/S)^2 eps_k and
  eps_k = 1 + w_k cos(theta/2) (phi1 - phi2 + phi2 z) / (2j sin(theta/2) (z - a_k)),
  w_k = wp_k^2 dt^2, a_k = e^{-nu_k dt}.
* `slab_rt_lattice` -- reflection/transmission of the slab on the infinite
  lattice (transfer recursion through the slab, fit of incident/reflected
  waves in vacuum).
* `domain_response` -- exact steady-state response of the whole finite lattice,
  including the first-order Mur end rows and the soft source; R and T from two
  such solves (plasma and vacuum) are what the running DFT converges to as the
  window grows.
* `fresnel_slab` -- continuous (Airy) slab with eps_r = 1 - wp^2/(w (w - j nu)).
* `domain_response_pml` -- the same steady-state response for a lattice terminated by the paper's
  split-field PML (graded matched conductivities, exponential differencing) and PEC walls.
* `current_response` -- the z-domain current of each recursion (Eq. 11, Eq. 9, Eq. 10).
"""
from __future__ import annotations

import math

import mpmath as mp
import numpy as np
from scipy.linalg import solve_banded

EPS0 = 8.8541878128e-12
MU0 = 1.25663706212e-6


def courant(dz: float, dt: float) -> float:
    return dt / (math.sqrt(MU0 * EPS0) * dz)


def phi_mp(x: float):
    """phi1 = (1 - e^{-x})/x, phi2 = (e^{-x} - 1 + x)/x^2 to 40 digits (limits 1, 1/2 at x = 0)."""
    with mp.workdps(40):
        X = mp.mpf(x)
        if X == 0:
            return 1.0, 0.5
        e = mp.exp(-X)
        return float((1 - e) / X), float((e - 1 + X) / X ** 2)


def _material_cache(wp2: np.ndarray, nu: np.ndarray, dt: float):
    """Unique (wp2, nu) pairs with their e^{-nu dt}, phi1, phi2."""
    pairs = {}
    for w, n in zip(wp2.tolist(), nu.tolist()):
        if (w, n) not in pairs:
            p1, p2 = phi_mp(n * dt)
            pairs[(w, n)] = (w * dt * dt, math.exp(-n * dt), p1, p2)
    return pairs


def current_response(z: np.ndarray, w: float, p1: float, p2: float, scheme: int = 0) -> np.ndarray:
    """beta0 z + beta1 + beta2/z of a current recursion written (normalised, J~ = dt J/eps0) as
    J~^{n+1} = a J~^n + beta0 E^{n+1} + beta1 E^n + beta2 E^{n-1}:
      scheme 0, Eq. 11 (RKETD):          beta0 = w phi2, beta1 = w (phi1 - phi2), beta2 = 0;
      scheme 1, Eq. 9 (first-order ETD): beta0 = 0,      beta1 = w phi1,          beta2 = 0;
      scheme 2, Eq. 10 (explicit ETD2):  beta0 = 0,      beta1 = w (phi1 + phi2), beta2 = -w phi2."""
    if scheme == 0:
        return w * (p2 * z + (p1 - p2))
    if scheme == 1:
        return w * p1 + 0.0 * z
    return w * (p1 + p2) - w * p2 / z


def lattice_eps(theta: np.ndarray, w: float, a: float, p1: float, p2: float, scheme: int = 0) -> np.ndarray:
    """Discrete permittivity of one cell at normalised frequencies theta = w dt.

    With J~ = chi(z) E, chi = current_response/(z - a), Eq. 12's average (J~^{n+1} + J~^n)/2 adds
    (z + 1) chi / 2 to (z - 1), so eps = 1 + cos(theta/2) chi / (2j sin(theta/2))."""
    z = np.exp(1j * theta)
    s = np.sin(theta / 2)
    c = np.cos(theta / 2)
    return 1.0 + c * current_response(z, w, p1, p2, scheme) / (2j * s * (z - a))


def lattice_q(theta: np.ndarray, S: float, wp2: np.ndarray, nu: np.ndarray, dt: float, scheme: int = 0) -> np.ndarray:
    """q_k(theta) for every cell: shape [len(theta), nz]."""
    cache = _material_cache(wp2, nu, dt)
    s = np.sin(theta / 2)
    out = np.empty((len(theta), len(wp2)), dtype=np.complex128)
    keys = list(zip(wp2.tolist(), nu.tolist()))
    epsd = {k: lattice_eps(theta, *v, scheme=scheme) for k, v in cache.items()}
    for i, k in enumerate(keys):
        out[:, i] = (2 * s / S) ** 2 * epsd[k]
    return out


def vacuum_K(theta: np.ndarray, S: float) -> np.ndarray:
    """Numerical wavenumber per cell: cos K = 1 - 2 sin^2(theta/2)/S^2 (Yee dispersion)."""
    return np.arccos(1 - 2 * np.sin(theta / 2) ** 2 / S ** 2)


def slab_rt_lattice(wp2, nu, dz, dt, freqs, p_r, p_t, scheme: int = 0):
    """R, T of the plasma region on the infinite lattice, referred to the probe cells.

    Start right of the slab with a purely transmitted wave e^{-jKk}, iterate
    E_{k-1} = (2 - q_k) E_k - E_{k+1} to the left vacuum, fit A e^{-jKk} + B e^{jKk}.
    R = (B/A) e^{2jK p_r} (what (X_tot - X_inc)/X_inc measures at p_r), T = 1/A.
    """
    wp2 = np.asarray(wp2, float)
    nu = np.asarray(nu, float)
    S = courant(dz, dt)
    theta = 2 * np.pi * np.asarray(freqs) * dt
    idx = np.nonzero(wp2)[0]
    lo, hi = int(idx[0]), int(idx[-1])
    assert lo - 2 > p_r and hi + 2 < p_t
    K = vacuum_K(theta, S)
    sub = slice(lo - 2, hi + 3)
    q = lattice_q(theta, S, wp2[sub], nu[sub], dt, scheme)  # cells lo-2 .. hi+2
    n = hi - lo + 5
    Ek1 = np.exp(-1j * K * (hi + 2))  # E_{k+1}
    Ek = np.exp(-1j * K * (hi + 1))  # E_k
    for j in range(n - 2, 0, -1):  # local j = cell - (lo-2); k from hi+1 down to lo-1
        Em1 = (2 - q[:, j]) * Ek - Ek1
        Ek1, Ek = Ek, Em1
    # Ek = E at cell lo-2, Ek1 = E at cell lo-1 (both vacuum)
    k0 = lo - 2
    e0, e1 = Ek, Ek1
    # e0 = A e^{-jK k0} + B e^{jK k0}; e1 = A e^{-jK(k0+1)} + B e^{jK(k0+1)}
    m00 = np.exp(-1j * K * k0)
    m01 = np.exp(1j * K * k0)
    m10 = np.exp(-1j * K * (k0 + 1))
    m11 = np.exp(1j * K * (k0 + 1))
    det = m00 * m11 - m01 * m10
    A = (e0 * m11 - m01 * e1) / det
    B = (m00 * e1 - e0 * m10) / det
    R = (B / A) * np.exp(2j * K * p_r)
    T = 1.0 / A
    return R, T


def domain_response(wp2, nu, dz, dt, freqs, src_cell, cells, scheme: int = 0):
    """Steady-state phasors at `cells` of the finite lattice driven by a unit soft source.

    Rows: interior E_{k-1} + (q_k - 2) E_k + E_{k+1} = delta_{k, src}; first-order Mur at
    both ends, E_0 (z + q) - E_1 (1 + q z) = 0 with q = (S-1)/(S+1) and the mirror row.
    The source scale is common to the plasma and vacuum solves and cancels in R and T.
    """
    wp2 = np.asarray(wp2, float)
    nu = np.asarray(nu, float)
    nz = len(wp2)
    S = courant(dz, dt)
    qm = (S - 1) / (S + 1)
    theta = 2 * np.pi * np.asarray(freqs) * dt
    qq = lattice_q(theta, S, wp2, nu, dt, scheme)
    out = np.empty((len(theta), len(cells)), dtype=np.complex128)
    for i, th in enumerate(theta):
        z = np.exp(1j * th)
        ab = np.zeros((3, nz), dtype=np.complex128)  # banded: upper, diag, lower
        ab[0, 1:] = 1.0
        ab[1, :] = qq[i] - 2.0
        ab[2, :-1] = 1.0
        # Mur rows
        ab[1, 0] = z + qm
        ab[0, 1] = -(1 + qm * z)
        ab[1, nz - 1] = z + qm
        ab[2, nz - 2] = -(1 + qm * z)
        rhs = np.zeros(nz, dtype=np.complex128)
        rhs[src_cell] = 1.0
        sol = solve_banded((1, 1), ab, rhs)
        out[i] = sol[list(cells)]
    return out


def domain_rt(slab):
    """R and T the running DFT converges to for a Mur-terminated slab problem."""
    cells = slab.probes
    tot = domain_response(slab.wp2, slab.nu, slab.dz, slab.dt, slab.freq_hz, slab.src_cell, cells,
                          getattr(slab, "scheme", 0))
    inc = domain_response(np.zeros(slab.nz), np.zeros(slab.nz), slab.dz, slab.dt, slab.freq_hz,
                          slab.src_cell, cells)
    R = (tot[:, 0] - inc[:, 0]) / inc[:, 0]
    T = tot[:, 1] / inc[:, 1]
    return R, T


def fresnel_slab(freqs, wp2: float, nu: float, d: float):
    """Continuous slab of thickness d in vacuum, e^{+jwt} convention.

    eps_r = 1 - wp^2/(w (w - j nu)), n = sqrt(eps_r) with Im n <= 0, r = (1-n)/(1+n),
    delta = n k0 d, R = r (1 - e^{-2j delta})/(1 - r^2 e^{-2j delta}),
    T e^{-j k0 d} = (1 - r^2) e^{-j delta}/(1 - r^2 e^{-2j delta}).
    Returns (|R|, |T|).
    """
    c = 1.0 / math.sqrt(MU0 * EPS0)
    w = 2 * np.pi * np.asarray(freqs, float)
    eps = 1 - wp2 / (w * (w - 1j * nu))
    n = np.sqrt(eps.astype(np.complex128))
    n = np.where(n.imag > 0, -n, n)
    r = (1 - n) / (1 + n)
    k0 = w / c
    ph = np.exp(-2j * n * k0 * d)
    R = r * (1 - ph) / (1 - r * r * ph)
    T = (1 - r * r) * np.exp(-1j * n * k0 * d) / (1 - r * r * ph)
    return np.abs(R), np.abs(T)


def plain_yee_vacuum(nz, dz, dt, steps, src_cell, src, probes):
    """Textbook 1D Yee leapfrog in SI (Eqs. 12 and 14 with J = 0), first-order Mur ends.

    `src(t)` is added to E at src_cell after each E update. Returns (E, H, series).
    """
    S = courant(dz, dt)
    qm = (S - 1) / (S + 1)
    E = np.zeros(nz)
    H = np.zeros(nz - 1)
    ser = np.zeros((len(probes), steps))
    for n in range(steps):
        H = H - dt / MU0 * ((E[1:] - E[:-1]) / dz)
        e0, e1, em1, em2 = E[0], E[1], E[-1], E[-2]
        E[1:-1] = E[1:-1] - (dt / EPS0) * ((H[1:] - H[:-1]) / dz)
        E[src_cell] = E[src_cell] + src((n + 1) * dt)
        E[0] = e1 + qm * (E[1] - e0)
        E[-1] = em2 + qm * (E[-2] - em1)
        ser[:, n] = E[probes]
    return E, H, ser


def normalized_run(slab, steps):
    """Independent NumPy restatement of the scheme in normalised variables (mur ends).

    E~ = E, H~ = eta0 H, J~ = (dt/eps0) J, S = c dt/dz. Per step:
    H~ -= S (E_{k+1} - E_k)                                        (Eq. 14)
    E' = [(1 - w(phi1 - phi2)/2) E - S (H~_{k+1/2} - H~_{k-1/2}) - (1 + a)/2 J~]/(1 + w phi2/2)
                                                                   (Eqs. 11 + 12 solved)
    J~' = a J~ + w phi1 E + w phi2 (E' - E)                         (Eq. 11)
    then the Eq. 15 soft source and first-order Mur ends. Returns (E, H (SI), J (SI), X).
    """
    nz = slab.nz
    dt, dz = slab.dt, slab.dz
    S = courant(dz, dt)
    qm = (S - 1) / (S + 1)
    eta0 = math.sqrt(MU0 / EPS0)
    cache = _material_cache(np.asarray(slab.wp2, float), np.asarray(slab.nu, float), dt)
    keys = list(zip(np.asarray(slab.wp2, float).tolist(), np.asarray(slab.nu, float).tolist()))
    w = np.array([cache[k][0] for k in keys])
    a = np.array([cache[k][1] for k in keys])
    p1 = np.array([cache[k][2] for k in keys])
    p2 = np.array([cache[k][3] for k in keys])
    D = 1 + w * p2 / 2
    E = np.zeros(nz)
    Ht = np.zeros(nz - 1)
    Jt = np.zeros(nz)
    P = len(slab.probes)
    X = np.zeros((P, len(slab.freq_hz)), dtype=np.complex128)
    f = np.asarray(slab.freq_hz)
    for n in range(steps):
        Ht = Ht - S * (E[1:] - E[:-1])
        e0, e1, em1, em2 = E[0], E[1], E[-1], E[-2]
        En = E[1:-1].copy()
        i = slice(1, -1)
        Enew = ((1 - w[i] * (p1[i] - p2[i]) / 2) * En - S * (Ht[1:] - Ht[:-1]) - (1 + a[i]) / 2 * Jt[i]) / D[i]
        Jt[i] = a[i] * Jt[i] + w[i] * p1[i] * En + w[i] * p2[i] * (Enew - En)
        E[i] = Enew
        t = (n + 1) * dt
        u = (t - slab.src_t0) / slab.src_tau
        E[slab.src_cell] += slab.src_amp * u * math.exp(-0.5 * u * u)
        E[0] = e1 + qm * (E[1] - e0)
        E[-1] = em2 + qm * (E[-2] - em1)
        X += E[slab.probes][:, None] * np.exp(-2j * np.pi * f[None, :] * t)
    return E, Ht / eta0, Jt * EPS0 / dt, X


def split_pml_profile(nz: int, n: int, m: float, sigma_max: float, dt: float, dz: float):
    """Per-node coefficients of the split-field PML (normalised fields, S = c dt/dz):
    E' = aE E - S fE (H~_{k+1/2} - H~_{k-1/2}),  H~' = aH H~ - S fH (E_{k+1} - E_k),
    a = e^{-x}, f = (1 - e^{-x})/x, x = sigma dt/eps0 (sigma* dt/mu0 for H with the matched sigma*),
    sigma = sigma_max rho^m at relative depth rho = (n - d)/n from the inner interface (d the node's
    distance from the outer wall in cells). Outside the layers a = f = 1. Returns (aE, fE, inE) for E
    nodes 0..nz-1 and (aH, fH) for H nodes k+1/2, k = 0..nz-2."""
    def coef(pos):
        right_inner = nz - 1 - n
        rho = (n - pos) / n if pos < n else ((pos - right_inner) / n if pos > right_inner else 0.0)
        if rho <= 0.0:
            return 1.0, 1.0, False
        x = sigma_max * rho ** m * dt / EPS0
        with mp.workdps(40):
            X = mp.mpf(x)
            return float(mp.exp(-X)), float((1 - mp.exp(-X)) / X), True
    E = [coef(k) for k in range(nz)]
    H = [coef(k + 0.5) for k in range(nz - 1)]
    aE = np.array([c[0] for c in E]); fE = np.array([c[1] for c in E]); inE = np.array([c[2] for c in E])
    aH = np.array([c[0] for c in H]); fH = np.array([c[1] for c in H])
    return aE, fE, inE, aH, fH


def domain_response_pml(wp2, nu, dz, dt, freqs, src_cell, cells, n, m, sigma_max, scheme: int = 0):
    """Steady-state phasors at `cells` of a finite lattice with the split-field PML of n cells at both
    ends and PEC walls (E_0 = E_{nz-1} = 0), driven by a soft source (the same scale in every solve).

    E^n = E z^n, H~^{n+1/2} = H z^{n+1/2}. With w_{k+1/2} = S fH_{k+1/2}/(z - aH_{k+1/2}) (S/(z-1)
    outside the layers), each E row reads
      (z - aE_k) eps_k E_k = S fE_k z [w_{k+1/2}(E_{k+1} - E_k) - w_{k-1/2}(E_k - E_{k-1})] + z s delta_{k,src},
    eps_k the lattice permittivity of the cell (1 in the vacuum layers)."""
    wp2 = np.asarray(wp2, float)
    nu = np.asarray(nu, float)
    nz = len(wp2)
    S = courant(dz, dt)
    aE, fE, inE, aH, fH = split_pml_profile(nz, n, m, sigma_max, dt, dz)
    cache = _material_cache(wp2, nu, dt)
    keys = list(zip(wp2.tolist(), nu.tolist()))
    theta = 2 * np.pi * np.asarray(freqs) * dt
    epsd = {k: lattice_eps(theta, *v, scheme=scheme) for k, v in cache.items()}
    out = np.empty((len(theta), len(cells)), dtype=np.complex128)
    for i, th in enumerate(theta):
        z = np.exp(1j * th)
        w = S * fH / (z - aH)  # [nz-1]
        eps = np.array([epsd[k][i] for k in keys])
        ab = np.zeros((3, nz), dtype=np.complex128)  # banded: upper, diag, lower
        C = S * fE[1:-1] * z * w[1:]  # coefficient of E_{k+1} in row k = 1..nz-2
        A = S * fE[1:-1] * z * w[:-1]  # coefficient of E_{k-1}
        ab[1, 1:-1] = -(z - aE[1:-1]) * eps[1:-1] - C - A
        ab[0, 2:] = C
        ab[2, :-2] = A
        ab[1, 0] = ab[1, -1] = 1.0  # PEC rows
        rhs = np.zeros(nz, dtype=np.complex128)
        rhs[src_cell] = -z
        sol = solve_banded((1, 1), ab, rhs)
        out[i] = sol[list(cells)]
    return out


def domain_response_2d_mode(wp2_rows, nu_rows, d, dt, freqs, src_row, rows, mu_x, pol, scheme: int = 0):
    """Steady-state phasors at `rows` of one transverse Fourier mode of the 2D lattice (periodic in x,
    layered in y, first-order Mur rows at j = 0 and ny-1), driven by the line source on src_row.

    mu_x = 4 sin^2(kx d/2) is the mode's x second-difference eigenvalue. With E^n = E z^n and the
    layer's lattice permittivity eps_j (row j's material):
      TMz (Ez): E_{j+1} - 2 E_j + E_{j-1} = -(q_j - mu_x) E_j, q_j = (2 sin(theta/2)/S)^2 eps_j;
      TEz (Ex at rows j, Ey at rows j + 1/2 with row j's material, Hz at rows j + 1/2): eliminating Ey
      and Hz from the three updates gives
        g_j (X_{j+1} - X_j) - g_{j-1} (X_j - X_{j-1}) = (z - 1) eps_j X_j / S^2,
        g_j = z / ((z - 1) + S^2 mu_x z / ((z - 1) eps_j)),
      which is the TMz row for mu_x = 0.
    The source adds to the row of src_row; Mur rows as the 1D lattice."""
    wp2_rows = np.asarray(wp2_rows, float)
    nu_rows = np.asarray(nu_rows, float)
    ny = len(wp2_rows)
    S = courant(d, dt)
    qm = (S - 1) / (S + 1)
    theta = 2 * np.pi * np.asarray(freqs) * dt
    cache = _material_cache(wp2_rows, nu_rows, dt)
    keys = list(zip(wp2_rows.tolist(), nu_rows.tolist()))
    epsd = {k: lattice_eps(theta, *v, scheme=scheme) for k, v in cache.items()}
    out = np.empty((len(theta), len(rows)), dtype=np.complex128)
    for i, th in enumerate(theta):
        z = np.exp(1j * th)
        eps = np.array([epsd[k][i] for k in keys])
        ab = np.zeros((3, ny), dtype=np.complex128)
        if pol == "tm":
            q = (2 * np.sin(th / 2) / S) ** 2 * eps - mu_x
            ab[0, 2:] = 1.0
            ab[1, 1:-1] = q[1:-1] - 2.0
            ab[2, :-2] = 1.0
            rhs_val = 1.0
        else:
            g = z / ((z - 1) + S * S * mu_x * z / ((z - 1) * eps[:-1]))  # j = 0 .. ny-2
            ab[0, 2:] = g[1:]
            ab[1, 1:-1] = -g[1:] - g[:-1] - (z - 1) * eps[1:-1] / (S * S)
            ab[2, :-2] = g[:-1]
            rhs_val = -z / (S * S)
        ab[1, 0] = z + qm
        ab[0, 1] = -(1 + qm * z)
        ab[1, ny - 1] = z + qm
        ab[2, ny - 2] = -(1 + qm * z)
        rhs = np.zeros(ny, dtype=np.complex128)
        rhs[src_row] = rhs_val
        out[i] = solve_banded((1, 1), ab, rhs)[list(rows)]
    return out
