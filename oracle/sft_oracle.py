"""Plain FP64 restatement of the HipFT surface-flux-transport step (numpy).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  Nothing here is
blocked, fused or reordered beyond what the paper states: each operator is
written as the formula it restates, over whole numpy arrays, in FP64.

Storage convention shared with the maps the paper reads and writes:
``B[j, k]``, j = 0 .. nt-1 over colatitude theta in [0, pi] with BOTH poles
included (rows 0 and nt-1 hold the pole value replicated over k), k = 0 ..
np-1 over the np unique longitudes (the paper's one/two-point phi overlap is
realised by periodic indexing).  Units are the paper's code units
(Sec. 3.3): lengths in solar radii, time in hours, B in Gauss.

Readings of points where the paper is silent or garbled are marked
"Reading:" in the docstrings.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# --------------------------------------------------------------------------
# Sec. 3.3 (Units).  R_sun = 6.96e8 m is the value that reproduces both
# printed conversion constants (the 6.69e8 in Sec. 2.1 is a typo).
# --------------------------------------------------------------------------
R_SUN_M = 6.96e8
R_SUN_CM = 6.96e10
M_S_TO_RS_HR = 3600.0 / R_SUN_M                 # m/s   -> R_sun/hr
KM2_S_TO_RS2_HR = 3600.0 * 1.0e6 / R_SUN_M**2   # km^2/s -> R_sun^2/hr


# --------------------------------------------------------------------------
# Sec. 3.2 (Grid)
# --------------------------------------------------------------------------
class Grid:
    """Uniform logically-rectangular grid of Sec. 3.2.

    Reading: ``nt`` counts theta points including both poles
    (theta_j = j*pi/(nt-1)); ``np_`` counts unique longitudes
    (phi_k = k*2*pi/np_).  Velocities in theta live on the theta half grid
    theta_{j+1/2}; the polar caps extend to theta = dtheta/2 (App. A).
    """

    def __init__(self, nt: int, np_: int):
        if nt < 4 or np_ < 4:
            raise ValueError("grid too small")
        self.nt, self.np = nt, np_
        self.dth = math.pi / (nt - 1)
        self.dph = 2.0 * math.pi / np_
        self.theta = np.arange(nt) * self.dth
        self.theta[-1] = math.pi
        self.theta_h = (np.arange(nt - 1) + 0.5) * self.dth   # theta_{f+1/2}
        self.phi = np.arange(np_) * self.dph
        self.sin_t = np.sin(self.theta)
        self.sin_t[0] = 0.0
        self.sin_t[-1] = 0.0
        self.sin_th = np.sin(self.theta_h)
        self.lat = 0.5 * math.pi - self.theta
        # App. A: area of one polar cap out to theta = dtheta/2 (exact form).
        self.cap_area = 2.0 * math.pi * (1.0 - math.cos(0.5 * self.dth))
        # Area weight of every stored entry: sin(theta_j) dtheta dphi in the
        # interior; a pole row carries its cap area spread over its np copies.
        self.area = np.empty((nt, np_))
        self.area[1:-1, :] = (self.sin_t[1:-1] * self.dth * self.dph)[:, None]
        self.area[0, :] = self.cap_area / np_
        self.area[-1, :] = self.cap_area / np_


# --------------------------------------------------------------------------
# Sec. 2.1.1: analytic differential rotation and meridional flow
# --------------------------------------------------------------------------
def flow_profiles(g: Grid, d0, d2, d4, m1, m3, m5):
    """Eq. (dr) and Eq. (mf), converted to code units (R_sun/hr).

    Returns (vt, vp): vt[f] = v_theta at theta_{f+1/2}, f = 0..nt-2;
    vp[j] = v_phi at theta_j (the same on every phi half-grid point of row j).
    """
    c = np.cos(g.theta)
    vp = (d0 + d2 * c**2 + d4 * c**4) * g.sin_t * M_S_TO_RS_HR
    ch = np.cos(g.theta_h)
    vt = -(m1 * ch + m3 * ch**3 + m5 * ch**5) * g.sin_th * M_S_TO_RS_HR
    return vt, vp


def advection_dt_limit(g: Grid, vt, vp, time_scheme="ssprk43", safety=0.9):
    """Stable advection step: Eq. (advection_timestep) for FE / SSPRK(3,3),
    Eq. (ssprk43_dt) (twice as large) for SSPRK(4,3), times the safety
    factor of Sec. 3.6.2.  Velocities are the larger of the two flanking
    staggered values; pole rows (sin theta = 0) are excluded."""
    j = np.arange(1, g.nt - 1)
    vth = np.maximum(np.abs(vt[j - 1]), np.abs(vt[j]))
    rate = vth / g.dth + np.abs(vp[j]) / (g.sin_t[j] * g.dph)
    rmax = rate.max()
    if rmax <= 0.0:
        return math.inf
    lim = 1.0 / rmax
    if time_scheme in ("fe", "ssprk33"):
        lim *= 0.5
    return safety * lim


# --------------------------------------------------------------------------
# Sec. 3.6.1 and App. B: face fluxes
# --------------------------------------------------------------------------
def upwind_face_flux(v, B_lo, B_hi, alpha_uw=1.0):
    """UW/CD flux at face i-1/2 (Sec. 3.6.1): B_lo = B_{i-1}, B_hi = B_i.
    sign(0) is taken as +1."""
    uw = alpha_uw * np.where(v >= 0.0, 1.0, -1.0)
    return v * 0.5 * ((1.0 - uw) * B_hi + (1.0 + uw) * B_lo)


def weno3_face_flux(LMm2, LMm1, LM0, LPm1, LP0, LPp1, eps_w):
    """WENO3-CS(h) flux F_{i-1/2} = u+ + u- of App. B on a uniform grid.

    Arguments are LM_{i-2}, LM_{i-1}, LM_i and LP_{i-1}, LP_i, LP_{i+1}.
    On a uniform grid every D factor of App. B is 1/2 (c/cp, c/cm),
    1/3 (p/t, m/t) or 2/3 (cp/t, cm/t).
    Reading: the appendix's mixed D indices are garbled; the uniform-grid
    values make them irrelevant.
    """
    Dc = 0.5
    Dp_t = Dm_t = 1.0 / 3.0
    Dcm_t = Dcp_t = 2.0 / 3.0
    # reconstruction polynomials
    p0m = (1.0 + Dc) * LMm1 - Dc * LMm2
    p1m = Dc * LMm1 + Dc * LM0
    p0p = (1.0 + Dc) * LP0 - Dc * LPp1
    p1p = Dc * LP0 + Dc * LPm1
    # smoothness indicators
    b0m = 4.0 * (Dc * (LMm1 - LMm2)) ** 2
    b1m = 4.0 * (Dc * (LM0 - LMm1)) ** 2
    b0p = 4.0 * (Dc * (LPp1 - LP0)) ** 2
    b1p = 4.0 * (Dc * (LP0 - LPm1)) ** 2
    # nonlinear weights
    w0m = Dp_t / (eps_w + b0m) ** 2
    w1m = Dcm_t / (eps_w + b1m) ** 2
    w0p = Dm_t / (eps_w + b0p) ** 2
    w1p = Dcp_t / (eps_w + b1p) ** 2
    um = (w0m * p0m + w1m * p1m) / (w0m + w1m)
    up = (w0p * p0p + w1p * p1p) / (w0p + w1p)
    return up + um


def llf_split(B, v_minus, v_plus, alpha, a=None):
    """Local Lax-Friedrichs splitting of App. B:
    LP_i = B_i (v_{i+1/2} - alpha_i)/2, LM_i = B_i (v_{i-1/2} + alpha_i)/2.
    With flow attenuation (Eq. flow_attenuation) the advective part carries
    the cell's factor a_i: LP_i = (v_{i+1/2} a_i B_i - alpha_i B_i)/2,
    LM_i = (v_{i-1/2} a_i B_i + alpha_i B_i)/2."""
    if a is None:
        LP = 0.5 * B * (v_plus - alpha)
        LM = 0.5 * B * (v_minus + alpha)
    else:
        LP = 0.5 * (v_plus * a * B - alpha * B)
        LM = 0.5 * (v_minus * a * B + alpha * B)
    return LP, LM


def attenuation_factor(B, b0):
    """Eq. (flow_attenuation): the flow is scaled by 1 - tanh(|B_r| / B_0).
    Reading: the factor is taken where the flow meets the field, i.e. every
    flux term v B_i of cell i becomes v a_i B_i (the flux function
    f(B) = v (1 - tanh(|B|/B_0)) B); b0 = None or 0 switches it off."""
    if not b0:
        return None
    return 1.0 - np.tanh(np.abs(B) / b0)


def _theta_face_is_upwind(nt):
    """Reading: the pole-cap faces (App. A) and the other face of each
    pole-adjacent cell use upwinding (Sec. 3.6.1, boundary conditions), so
    that each face has ONE flux (conservative) and no WENO stencil reaches
    a pole row.  Faces f (between rows f and f+1), f = 0..nt-2."""
    up = np.zeros(nt - 1, dtype=bool)
    up[[0, 1, nt - 3, nt - 2]] = True
    return up


def theta_face_fluxes(g: Grid, B, vt, space="weno3", eps_w="h", alpha_uw=1.0, a=None):
    """F_theta at every theta face f+1/2 (shape (nt-1, np)); a = the flow
    attenuation factor per cell (None: off)."""
    nt = g.nt
    Ft = np.empty((nt - 1, g.np))
    f = np.arange(nt - 1)
    aB = B if a is None else a * B
    uw_flux = upwind_face_flux(vt[:, None], aB[:-1, :], aB[1:, :], alpha_uw)
    if space == "upwind":
        return uw_flux
    eps = g.dth if eps_w == "h" else float(eps_w)
    # LLF split on interior rows i = 1..nt-2; alpha_i is the max |v| over
    # faces i-5/2 .. i+5/2 (f = i-3 .. i+2), clipped to the faces that exist.
    i = np.arange(1, nt - 1)
    av = np.abs(vt)
    alpha = np.array([av[max(ii - 3, 0):min(ii + 2, nt - 2) + 1].max() for ii in i])
    LP = np.zeros_like(B)
    LM = np.zeros_like(B)
    LP[i], LM[i] = llf_split(B[i], vt[i - 1][:, None], vt[i][:, None], alpha[:, None],
                             None if a is None else a[i])
    Ft[:] = uw_flux
    fw = f[~_theta_face_is_upwind(nt)]
    iw = fw + 1   # face f is F_{i-1/2} with i = f + 1
    Ft[fw] = weno3_face_flux(LM[iw - 2], LM[iw - 1], LM[iw],
                             LP[iw - 1], LP[iw], LP[iw + 1], eps)
    return Ft


def phi_face_fluxes(g: Grid, B, vp, space="weno3", eps_w="h", alpha_uw=1.0, a=None):
    """F_phi at faces k-1/2 of every row (shape (nt, np)); periodic in phi.
    v_phi is uniform along a row for the analytic flows, so alpha_i = |v|."""
    v = vp[:, None] * np.ones((1, g.np))
    if space == "upwind":
        aB = B if a is None else a * B
        return upwind_face_flux(v, np.roll(aB, 1, axis=1), aB, alpha_uw)
    eps = g.dph if eps_w == "h" else float(eps_w)
    alpha = np.abs(v)
    LP, LM = llf_split(B, v, v, alpha, a)

    def sh(a, s):   # a_{k+s}
        return np.roll(a, -s, axis=1)

    return weno3_face_flux(sh(LM, -2), sh(LM, -1), LM,
                           sh(LP, -1), LP, sh(LP, 1), eps)


def advection_operator(g: Grid, B, vt, vp, space="weno3", eps_w="h", alpha_uw=1.0, b0=None):
    """F_A(B) = div_s(B v) by the conservative finite difference of
    Sec. 3.6.1 with the polar finite-volume caps of App. A; b0 > 0 attenuates
    the flow by Eq. (flow_attenuation) (the LLF bound alpha = max |v| and the
    time-step limit keep the unattenuated flow: attenuation only slows it,
    and |d f/d B| <= |v| for the attenuated flux)."""
    a = attenuation_factor(B, b0)
    Ft = theta_face_fluxes(g, B, vt, space, eps_w, alpha_uw, a)
    Fp = phi_face_fluxes(g, B, vp, space, eps_w, alpha_uw, a)
    out = np.zeros_like(B)
    j = np.arange(1, g.nt - 1)
    st = g.sin_t[j][:, None]
    # sin(theta_{j+1/2}) F_{j+1/2} - sin(theta_{j-1/2}) F_{j-1/2}
    dtheta = (g.sin_th[j][:, None] * Ft[j] - g.sin_th[j - 1][:, None] * Ft[j - 1]) / (st * g.dth)
    Fp_in = Fp[j]                       # F_{k-1/2}
    Fp_out = np.roll(Fp_in, -1, axis=1)  # F_{k+1/2}
    dphi = (Fp_out - Fp_in) / (st * g.dph)
    out[j] = dtheta + dphi
    # App. A: the cap's divergence is its boundary flux over its area.
    line = math.sin(0.5 * g.dth) * g.dph
    out[0, :] = line * Ft[0].sum() / g.cap_area
    out[-1, :] = -line * Ft[-1].sum() / g.cap_area
    return out


# --------------------------------------------------------------------------
# Sec. 3.6.2: advection time schemes (generic in the operator F_A)
# --------------------------------------------------------------------------
def fe_advance(f, dt, FA):
    """Eq. (adv_euler)."""
    return f - dt * FA(f)


def ssprk33_advance(f, dt, FA):
    """SSPRK(3,3), Sec. 3.6.2."""
    f1 = f - dt * FA(f)
    f2 = 0.75 * f + 0.25 * f1 - 0.25 * dt * FA(f1)
    return f / 3.0 + 2.0 / 3.0 * f2 - 2.0 / 3.0 * dt * FA(f2)


def ssprk43_advance(f, dt, FA):
    """SSPRK(4,3), Sec. 3.6.2."""
    f1 = f - 0.5 * dt * FA(f)
    f2 = f1 - 0.5 * dt * FA(f1)
    f3 = 2.0 / 3.0 * f + f2 / 3.0 - dt / 6.0 * FA(f2)
    return f3 - 0.5 * dt * FA(f3)


ADV_TIME = {"fe": fe_advance, "ssprk33": ssprk33_advance, "ssprk43": ssprk43_advance}


# --------------------------------------------------------------------------
# Sec. 3.7.1: diffusion operator, its matrix, and App. A polar caps
# --------------------------------------------------------------------------
def constant_nu(g: Grid, nu_rs2_hr: float):
    """nu on the half-half grid (theta_{f+1/2}, phi_{k+1/2}), shape (nt-1, np);
    entry [f, k] is nu_{f+1/2, k+1/2}."""
    return np.full((g.nt - 1, g.np), float(nu_rs2_hr))


def grid_nu(g: Grid, alpha_nu: float):
    """Eq. (diffgrid): nu_g = alpha_nu [(dtheta)^2 + (dphi sin theta)^2], on
    the half-half grid of the operator, shape (nt-1, np).  Reading: nu lives
    where the operator takes it, at theta_{f+1/2} (uniform in phi); alpha_nu
    is in 1/hour (the time unit), so nu_g is in R_sun^2/hour."""
    nu = alpha_nu * (g.dth ** 2 + (g.dph * g.sin_th) ** 2)   # sin_th[f] = sin(theta_{f+1/2})
    return np.repeat(nu[:, None], g.np, axis=1)


def diffusion_operator(g: Grid, B, nu_hh):
    """Eq. (diffusion_op) on interior rows, App. A on the poles.
    nu_hh[f, k] = nu_{f+1/2, k+1/2}."""
    out = np.zeros_like(B)
    j = np.arange(1, g.nt - 1)
    st = g.sin_t[j][:, None]
    nu_up = nu_hh[j]              # nu_{j+1/2, k+1/2}
    nu_dn = nu_hh[j - 1]          # nu_{j-1/2, k+1/2}
    nu_up_m = np.roll(nu_up, 1, axis=1)   # nu_{j+1/2, k-1/2}
    nu_dn_m = np.roll(nu_dn, 1, axis=1)   # nu_{j-1/2, k-1/2}
    Bj = B[j]
    Bn = B[j + 1]
    Bs = B[j - 1]
    Bk_p = np.roll(Bj, -1, axis=1)
    Bk_m = np.roll(Bj, 1, axis=1)
    theta_part = (0.5 * (nu_up + nu_up_m) * g.sin_th[j][:, None] * (Bn - Bj) / g.dth
                  - 0.5 * (nu_dn + nu_dn_m) * g.sin_th[j - 1][:, None] * (Bj - Bs) / g.dth
                  ) / (st * g.dth)
    phi_part = (0.5 * (nu_up + nu_dn) * (Bk_p - Bj) / g.dph
                - 0.5 * (nu_up_m + nu_dn_m) * (Bj - Bk_m) / g.dph
                ) / (st**2 * g.dph)
    out[j] = theta_part + phi_part
    # App. A: cap flux through theta = dtheta/2, central difference in theta.
    line = math.sin(0.5 * g.dth) * g.dph
    nu_n = 0.5 * (nu_hh[0] + np.roll(nu_hh[0], 1))      # nu at (1/2, k)
    nu_s = 0.5 * (nu_hh[-1] + np.roll(nu_hh[-1], 1))
    Fn = nu_n * (B[1] - B[0, 0]) / g.dth
    Fs = nu_s * (B[-1, 0] - B[-2]) / g.dth
    out[0, :] = line * Fn.sum() / g.cap_area
    out[-1, :] = -line * Fs.sum() / g.cap_area
    return out


def diffusion_matrix(g: Grid, nu_hh):
    """Eq. (diffusion_matrix): the operator as a sparse matrix acting on the
    unique unknowns [B_north, B[1,0..np-1], ..., B[nt-2, ...], B_south],
    with the App. A cap rows added.  Returned as scipy CSR."""
    import scipy.sparse as sp
    nt, np_ = g.nt, g.np
    n = 2 + (nt - 2) * np_
    rows, cols, vals = [], [], []

    def idx(j, k):
        if j == 0:
            return 0
        if j == nt - 1:
            return n - 1
        return 1 + (j - 1) * np_ + (k % np_)

    for j in range(1, nt - 1):
        for k in range(np_):
            nu_pp = nu_hh[j, k]
            nu_pm = nu_hh[j, (k - 1) % np_]
            nu_mp = nu_hh[j - 1, k]
            nu_mm = nu_hh[j - 1, (k - 1) % np_]
            a_km = (nu_pm + nu_mm) / (2 * g.dph * g.dph * g.sin_t[j] ** 2)
            a_kp = (nu_pp + nu_mp) / (2 * g.dph * g.dph * g.sin_t[j] ** 2)
            a_jm = (nu_mp + nu_mm) * g.sin_th[j - 1] / (2 * g.dth * g.dth * g.sin_t[j])
            a_jp = (nu_pp + nu_pm) * g.sin_th[j] / (2 * g.dth * g.dth * g.sin_t[j])
            a_jj = -(a_jm + a_jp + a_km + a_kp)
            i = idx(j, k)
            for jj, kk, a in ((j, k - 1, a_km), (j - 1, k, a_jm), (j, k, a_jj),
                              (j + 1, k, a_jp), (j, k + 1, a_kp)):
                rows.append(i)
                cols.append(idx(jj, kk))
                vals.append(a)
    line = math.sin(0.5 * g.dth) * g.dph
    for pole, jn in ((0, 1), (n - 1, nt - 2)):
        f = 0 if pole == 0 else nt - 2
        diag = 0.0
        for k in range(np_):
            nu_face = 0.5 * (nu_hh[f, k] + nu_hh[f, (k - 1) % np_])
            c = line * nu_face / (g.dth * g.cap_area)
            rows.append(pole)
            cols.append(idx(jn, k))
            vals.append(c)
            diag -= c
        rows.append(pole)
        cols.append(pole)
        vals.append(diag)
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, n))


def unique_unknowns(B):
    """[B_north, interior rows flattened, B_south] (the matrix ordering)."""
    return np.concatenate([[B[0, 0]], B[1:-1].ravel(), [B[-1, 0]]])


def euler_dt_limit(g: Grid, nu_hh):
    """Stable explicit-Euler diffusion step, Sec. 3.7.2.
    Reading: Gershgorin bound 1/max|a_ii| over all rows of the matrix
    (the paper says only that the DIA form makes it easy to compute)."""
    M = diffusion_matrix(g, nu_hh)
    amax = np.abs(M.diagonal()).max()
    return math.inf if amax == 0.0 else 1.0 / amax


# --------------------------------------------------------------------------
# Sec. 3.7.2: RKL2 super time stepping (Meyer, Balsara & Aslam 2014)
# --------------------------------------------------------------------------
def rkl2_stage_count(dt, dt_euler):
    """Smallest s >= 2 with dt <= dt_euler (s^2 + s - 2)/4."""
    if not math.isfinite(dt_euler):
        return 2
    s = math.ceil(0.5 * (-1.0 + math.sqrt(9.0 + 16.0 * dt / dt_euler)))
    while (s * s + s - 2) * dt_euler < 4.0 * dt:
        s += 1
    return max(s, 2)


def rkl2_coefficients(s):
    """RKL2 coefficients (Meyer, Balsara & Aslam 2014, the scheme the paper
    cites for Sec. 3.7.2).  Arrays indexed by stage j = 0..s:
    mu, nu, mut (mu-tilde), gt (gamma-tilde); entries j < 2 unused except
    mut[1]."""
    w1 = 4.0 / (s * s + s - 2)
    b = np.empty(s + 1)
    b[:3] = 1.0 / 3.0
    for j in range(3, s + 1):
        b[j] = (j * j + j - 2) / (2.0 * j * (j + 1))
    a = 1.0 - b
    mu = np.zeros(s + 1)
    nu = np.zeros(s + 1)
    mut = np.zeros(s + 1)
    gt = np.zeros(s + 1)
    mut[1] = b[1] * w1
    for j in range(2, s + 1):
        mu[j] = (2.0 * j - 1.0) / j * b[j] / b[j - 1]
        nu[j] = -(j - 1.0) / j * b[j] / b[j - 2]
        mut[j] = mu[j] * w1
        gt[j] = -a[j - 1] * mut[j]
    return mu, nu, mut, gt


def rkl2_advance(Y0, dt, L, s):
    """One RKL2 super-step of s stages for dY/dt = L(Y)."""
    mu, nu, mut, gt = rkl2_coefficients(s)
    LY0 = L(Y0)
    Ym2 = Y0
    Ym1 = Y0 + mut[1] * dt * LY0
    for j in range(2, s + 1):
        Y = (mu[j] * Ym1 + nu[j] * Ym2 + (1.0 - mu[j] - nu[j]) * Y0
             + mut[j] * dt * L(Ym1) + gt[j] * dt * LY0)
        Ym2, Ym1 = Ym1, Y
    return Ym1


# --------------------------------------------------------------------------
# Sec. 3.7.2: RKG2(3/2) super time stepping (the paper's default; its
# coefficients are only cited).  Reading: the second-order scheme built like
# RKL2 on the Gegenbauer polynomials C_j = C_j^(3/2) instead of the Legendre
# polynomials: R_j(z) = a_j + b_j C_j(1 + w1 z), with w1 and b_j fixed by
# R_s(0) = R_s'(0) = R_s''(0) = 1 (second order), the three-term Gegenbauer
# recurrence j C_j(x) = (2j+1) x C_{j-1}(x) - (j+1) C_{j-2}(x) giving the
# stages, and b_0 = b_1 = b_2 as RKL2 takes them.  From C_j(1) =
# (j+1)(j+2)/2, C_j'(1) = j(j+1)(j+2)(j+3)/8 and C_j''(1) =
# (j-1)j(j+1)(j+2)(j+3)(j+4)/48:  w1 = 6/((s-1)(s+4)),
# b_j = 4(j-1)(j+4)/(3j(j+1)(j+2)(j+3)), a_j = 1 - b_j C_j(1), stable for
# z in [-(s-1)(s+4)/3, 0], i.e. dt <= dt_E (s^2+3s-4)/6.
# --------------------------------------------------------------------------
def rkg2_stage_count(dt, dt_euler):
    """Smallest s >= 2 with dt <= dt_euler (s^2 + 3s - 4)/6."""
    if not math.isfinite(dt_euler):
        return 2
    s = max(2, math.ceil(0.5 * (-3.0 + math.sqrt(25.0 + 24.0 * dt / dt_euler))))
    while (s * s + 3 * s - 4) * dt_euler < 6.0 * dt:
        s += 1
    while s > 2 and ((s - 1) ** 2 + 3 * (s - 1) - 4) * dt_euler >= 6.0 * dt:
        s -= 1
    return s


def rkg2_coefficients(s):
    """RKG2(3/2) coefficients for s stages, arrays indexed by stage j = 0..s:
    mu, nu, mut (mu-tilde), gt (gamma-tilde), as rkl2_coefficients."""
    w1 = 6.0 / ((s - 1.0) * (s + 4.0))
    b = np.empty(s + 1)
    for j in range(2, s + 1):
        b[j] = 4.0 * (j - 1.0) * (j + 4.0) / (3.0 * j * (j + 1.0) * (j + 2.0) * (j + 3.0))
    b[0] = b[1] = b[2]
    cj1 = np.array([(j + 1.0) * (j + 2.0) / 2.0 for j in range(s + 1)])   # C_j(1)
    a = 1.0 - b * cj1
    mu = np.zeros(s + 1)
    nu = np.zeros(s + 1)
    mut = np.zeros(s + 1)
    gt = np.zeros(s + 1)
    mut[1] = 3.0 * b[1] * w1          # C_1'(1) b_1 w1
    for j in range(2, s + 1):
        mu[j] = (2.0 * j + 1.0) / j * b[j] / b[j - 1]
        nu[j] = -(j + 1.0) / j * b[j] / b[j - 2]
        mut[j] = mu[j] * w1
        gt[j] = -a[j - 1] * mut[j]
    return mu, nu, mut, gt


def rkg2_advance(Y0, dt, L, s):
    """One RKG2(3/2) super-step of s stages for dY/dt = L(Y): the stage
    recurrence of rkl2_advance with the RKG2 coefficients."""
    mu, nu, mut, gt = rkg2_coefficients(s)
    LY0 = L(Y0)
    Ym2 = Y0
    Ym1 = Y0 + mut[1] * dt * LY0
    for j in range(2, s + 1):
        Y = (mu[j] * Ym1 + nu[j] * Ym2 + (1.0 - mu[j] - nu[j]) * Y0
             + mut[j] * dt * L(Ym1) + gt[j] * dt * LY0)
        Ym2, Ym1 = Ym1, Y
    return Ym1


def fe_diffusion_advance(B, dt, L, dt_euler):
    """Explicit forward Euler diffusion (Sec. 3.7.2, reference/testing),
    sub-cycled at the Euler limit."""
    n = max(1, math.ceil(dt / dt_euler))
    h = dt / n
    for _ in range(n):
        B = B + h * L(B)
    return B


# --------------------------------------------------------------------------
# Sec. 2.3: data assimilation
# --------------------------------------------------------------------------
def assimilation_weight(mu, lat, alpha_mu, mu_lim, lat_lim):
    """Eq. (data_assim_f): F = mu^alpha_mu where mu > mu_lim and
    |latitude| < lat_lim, else 0 (strict inequalities, as printed)."""
    mu = np.asarray(mu, dtype=np.float64)
    ok = (mu > mu_lim) & (np.abs(lat) < lat_lim)
    return np.where(ok, np.power(np.maximum(mu, 0.0), alpha_mu), 0.0)


def flux_balance_factors(g: Grid, X):
    """Eq. (fluxbal): positive/negative total fluxes of X and the two
    multiplicative factors.  Returns (phi_p, phi_m, fac_pos, fac_neg);
    factors are 1 when either flux is zero (nothing to balance against).
    Reading: ratio r = |phi_+ / phi_-|; X > 0 is divided by sqrt(r),
    X <= 0 is multiplied by sqrt(r)."""
    A = g.area
    phi_p = float((A * np.where(X > 0.0, X, 0.0)).sum())
    phi_m = float((A * np.where(X < 0.0, X, 0.0)).sum())
    if phi_p == 0.0 or phi_m == 0.0:
        return phi_p, phi_m, 1.0, 1.0
    r = abs(phi_p / phi_m)
    return phi_p, phi_m, 1.0 / math.sqrt(r), math.sqrt(r)


def assimilate(g: Grid, B, Bd, F, balance=True):
    """Eq. (data_assim) as rewritten in Eq. (data_assim_deltab), with the
    optional multiplicative flux balance of Eq. (fluxbal) on Delta B."""
    dB = F * (Bd - B)
    if balance:
        _, _, fp, fm = flux_balance_factors(g, dB)
        dB = np.where(dB > 0.0, dB * fp, dB * fm)
    return B + dB


def flux_balance_map(g: Grid, B):
    """Multiplicative flux balance of a whole map (Sec. 5.1 input option),
    the Eq. (fluxbal) factors applied to B itself."""
    _, _, fp, fm = flux_balance_factors(g, B)
    return np.where(B > 0.0, B * fp, B * fm)


# --------------------------------------------------------------------------
# Sec. 2.6: analysis quantities
# --------------------------------------------------------------------------
@dataclass
class Diagnostics:
    flux_signed: float
    flux_pos: float
    flux_neg: float
    flux_pole_n: float
    flux_pole_s: float
    area_pole_n: float
    area_pole_s: float
    brmin: float
    brmax: float
    absmin: float
    dipole_axial: float
    h1: float
    h2: float

    @property
    def dipole_equatorial(self):
        return math.hypot(self.h1, self.h2)


def diagnostics(g: Grid, B, lat_cut_deg=60.0):
    """Sec. 2.6.  Fluxes in Mx (area in code units times R_sun^2 in cm^2),
    polar areas in cm^2, dipoles D, h1, h2 (Eq. eqdipole1) in Gauss.
    Polar regions are the cells with |latitude| >= lat_cut_deg."""
    A = g.area
    Mx = R_SUN_CM**2
    cut = math.radians(lat_cut_deg)
    north = (g.lat >= cut - 1e-12)[:, None] * np.ones((1, g.np), dtype=bool)
    south = (g.lat <= -cut + 1e-12)[:, None] * np.ones((1, g.np), dtype=bool)
    c = np.cos(g.theta)[:, None]
    s = g.sin_t[:, None]
    cp = np.cos(g.phi)[None, :]
    sp_ = np.sin(g.phi)[None, :]
    k3 = 3.0 / (4.0 * math.pi)
    return Diagnostics(
        flux_signed=float((A * B).sum() * Mx),
        flux_pos=float((A * np.where(B > 0, B, 0.0)).sum() * Mx),
        flux_neg=float((A * np.where(B < 0, B, 0.0)).sum() * Mx),
        flux_pole_n=float((A * B)[north].sum() * Mx),
        flux_pole_s=float((A * B)[south].sum() * Mx),
        area_pole_n=float(A[north].sum() * Mx),
        area_pole_s=float(A[south].sum() * Mx),
        brmin=float(B.min()),
        brmax=float(B.max()),
        absmin=float(np.abs(B).min()),
        dipole_axial=float(k3 * (A * B * c).sum()),
        h1=float(k3 * (A * B * s * cp).sum()),
        h2=float(k3 * (A * B * s * sp_).sum()),
    )


def total_flux(g: Grid, B):
    """Signed surface integral of B in code units (sum of area * B)."""
    return float((g.area * B).sum())


def hh_metric(X, Y):
    """Eq. (hh), the absolute-value Hanna-Heinold metric."""
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    return math.sqrt(float((np.abs(X - Y) ** 2).sum() / (np.abs(X) * np.abs(Y)).sum()))


# --------------------------------------------------------------------------
# Sec. 2.4: random flux emergence (RFE)
# --------------------------------------------------------------------------
SPLITMIX_GAMMA = 0x9E3779B97F4A7C15


def splitmix64_output(z):
    """The SplitMix64 output function (Steele, Lea & Flood 2014) on uint64
    array z (arithmetic mod 2^64)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def rfe_normals(g: Grid, seed, k):
    """Standard normal draws Y of RFE map k (the N(0, 1) samples of Sec. 2.4),
    one per unique cell (each pole cap is one cell; its row repeats it).
    Counter-based: cell c of map k takes the SplitMix64 outputs of the states
    seed + (2n+1) gamma and seed + (2n+2) gamma with n = k N_cells + c, as
    uniforms u = (top 53 bits + 1/2) / 2^53, and Box-Muller
    Y = sqrt(-2 ln u1) cos(2 pi u2)."""
    nt, np_ = g.nt, g.np
    ncell = (nt - 2) * np_ + 2
    cid = np.empty((nt, np_), dtype=np.uint64)
    cid[0, :] = 0
    cid[1:-1, :] = 1 + np.arange((nt - 2) * np_, dtype=np.uint64).reshape(nt - 2, np_)
    cid[-1, :] = ncell - 1
    n = np.uint64(k) * np.uint64(ncell) + cid
    gam = np.uint64(SPLITMIX_GAMMA)
    with np.errstate(over="ignore"):
        z1 = splitmix64_output(np.uint64(seed) + (np.uint64(2) * n + np.uint64(1)) * gam)
        z2 = splitmix64_output(np.uint64(seed) + (np.uint64(2) * n + np.uint64(2)) * gam)
    u1 = ((z1 >> np.uint64(11)).astype(np.float64) + 0.5) * 2.0 ** -53
    u2 = ((z2 >> np.uint64(11)).astype(np.float64) + 0.5) * 2.0 ** -53
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


def rfe_map(g: Grid, method, rate_mx_hr, seed, k):
    """RFE source map k in G/hour: Eq. (rfe_m1) (method 1: uniform unsigned
    flux per cell, divided by the cell's area) or Eq. (rfe_m2) (method 2:
    uniform unsigned flux per unit area), flux balanced as Eq. (fluxbal)."""
    Y = rfe_normals(g, seed, k)
    r2 = R_SUN_CM ** 2
    if method == 1:
        ncell = (g.nt - 2) * g.np + 2
        cell_area = g.area * r2                      # interior cells
        cell_area[0, :] = g.cap_area * r2            # each cap is one cell
        cell_area[-1, :] = g.cap_area * r2
        S = rate_mx_hr / (cell_area * ncell) * math.sqrt(0.5 * math.pi) * Y
    else:
        S = rate_mx_hr / (4.0 * math.pi * r2) * math.sqrt(0.5 * math.pi) * Y
    _, _, fp, fm = flux_balance_factors(g, S)
    return np.where(S > 0.0, S * fp, S * fm)


def rfe_weights(t0, tau, a, b):
    """Maps and weights of the exact integral over [a, b] of Eq. (rfe_s),
    S(t) = (1 - alpha) S_k + alpha S_{k+1}, alpha = (t - t_k) / tau on
    t_k = t0 + k tau <= t <= t_{k+1} (tau = inf: S = S_0).  Returns
    {k: weight (hours)}; the integral is sum_k weight_k S_k (linear in t:
    each piece integrates exactly at its midpoint)."""
    w = {}
    if not math.isfinite(tau):
        w[0] = b - a
        return w
    t = a
    while t < b:
        k = math.floor((t - t0) / tau + 1e-12)
        end = min(b, t0 + (k + 1) * tau)
        al = (0.5 * (t + end) - (t0 + k * tau)) / tau
        w[k] = w.get(k, 0.0) + (end - t) * (1.0 - al)
        w[k + 1] = w.get(k + 1, 0.0) + (end - t) * al
        t = end
    return w


# --------------------------------------------------------------------------
# Sec. 3.4 / 3.5: one realization's run (dt controller + Lie splitting)
# --------------------------------------------------------------------------
@dataclass
class Params:
    """Per-realization model and method choices (Sec. 2.1, 2.2, 3.6, 3.7).
    Flow coefficients in m/s (Eq. dr, Eq. mf), nu in km^2/s."""
    d0: float = 46.0
    d2: float = -262.0
    d4: float = -379.0
    m1: float = 22.0
    m3: float = 11.0
    m5: float = -28.0
    nu: float = 500.0
    adv_space: str = "weno3"     # "weno3" | "upwind"
    adv_time: str = "ssprk43"    # "ssprk43" | "ssprk33" | "fe"
    diffusion: str = "rkl2"      # "rkl2" | "rkg2" | "fe" | "off"
    advection: bool = True
    alpha_uw: float = 1.0
    safety: float = 0.9
    eps_w: object = "h"
    atten_b0: float = 0.0        # Eq. (flow_attenuation) saturation field (G); 0 = off
    splitting: str = "lie"       # "lie" (Eq. num_opsplit_nostrang) | "strang" (Eq. num_opsplit_strang)
    nu_grid_alpha: float = 0.0   # > 0: grid-based nu of Eq. (diffgrid) (1/hour) instead of nu
    rfe_method: int = 0          # random flux emergence (Sec. 2.4): 0 off, 1 Eq. (rfe_m1), 2 Eq. (rfe_m2)
    rfe_rate: float = 0.0        # total unsigned flux per hour, Mx/hour
    rfe_lifetime: float = math.inf   # hours between source maps (tau of Eq. rfe_s)
    rfe_seed: int = 0
    rfe_t0: float = 0.0          # time of source map 0


@dataclass
class Realization:
    g: Grid
    p: Params
    B: np.ndarray
    t: float = 0.0
    steps: int = 0
    vt: np.ndarray = field(init=False)
    vp: np.ndarray = field(init=False)
    nu_hh: np.ndarray = field(init=False)
    dt_adv: float = field(init=False)
    dt_euler: float = field(init=False)

    def __post_init__(self):
        p, g = self.p, self.g
        self.vt, self.vp = flow_profiles(g, p.d0, p.d2, p.d4, p.m1, p.m3, p.m5)
        self.nu_hh = (grid_nu(g, p.nu_grid_alpha) if p.nu_grid_alpha > 0.0
                      else constant_nu(g, p.nu * KM2_S_TO_RS2_HR))
        self.dt_adv = (advection_dt_limit(g, self.vt, self.vp, p.adv_time, p.safety)
                       if p.advection else math.inf)
        self.dt_euler = euler_dt_limit(g, self.nu_hh) if p.diffusion != "off" else math.inf
        self.B = np.array(self.B, dtype=np.float64, copy=True)

    def FA(self, B):
        p = self.p
        return advection_operator(self.g, B, self.vt, self.vp, p.adv_space, p.eps_w, p.alpha_uw, p.atten_b0)

    def L(self, B):
        return diffusion_operator(self.g, B, self.nu_hh)

    def _A(self, B, dt):
        return ADV_TIME[self.p.adv_time](B, dt, self.FA) if self.p.advection else B

    def _D(self, B, dt):
        if self.p.diffusion == "rkl2":
            return rkl2_advance(B, dt, self.L, rkl2_stage_count(dt, self.dt_euler))
        if self.p.diffusion == "rkg2":
            return rkg2_advance(B, dt, self.L, rkg2_stage_count(dt, self.dt_euler))
        if self.p.diffusion == "fe":
            return fe_diffusion_advance(B, dt, self.L, self.dt_euler)
        return B

    def _S(self, B, a, b):
        """The RFE source integrated over [a, b] (exactly, Eq. rfe_s)."""
        p = self.p
        if p.rfe_method == 0 or p.rfe_rate == 0.0:
            return B
        out = B.copy()
        for k, w in sorted(rfe_weights(p.rfe_t0, p.rfe_lifetime, a, b).items()):
            if w != 0.0:
                out = out + w * rfe_map(self.g, p.rfe_method, p.rfe_rate, p.rfe_seed, k)
        return out

    def lie_step(self, dt):
        """One time step (Sec. 3.5).  Eq. (num_opsplit_nostrang):
        B* = A(B^n, dt), B** = D(B*, dt), B^{n+1} = S(B**) with S the random
        flux emergence source integrated over the step.  Eq.
        (num_opsplit_strang): S over the first half step, A(dt/2), D(dt),
        A(dt/2), S over the second half.  (Assimilation follows the advance.)"""
        t = self.t
        if self.p.splitting == "strang":
            B = self._S(self.B, t, t + 0.5 * dt)
            B = self._A(self._D(self._A(B, 0.5 * dt), dt), 0.5 * dt)
            self.B = self._S(B, t + 0.5 * dt, t + dt)
        else:
            self.B = self._S(self._D(self._A(self.B, dt), dt), t, t + dt)

    def flow_dt_limit(self):
        """The step the flow allows: its CFL limit, twice that with Strang
        splitting (each advection advance is dt/2, Sec. 3.5)."""
        return 2.0 * self.dt_adv if self.p.splitting == "strang" else self.dt_adv

    def next_dt(self, t_target):
        """Sec. 3.4: start from the time remaining to the target (the next
        output / assimilation time) and reduce it to the stable flow step
        (and, with RFE, to the source lifetime, so that a step spans at most
        two source segments)."""
        remaining = t_target - self.t
        lim = self.flow_dt_limit()
        if self.p.rfe_method != 0 and self.p.rfe_rate != 0.0:
            lim = min(lim, self.p.rfe_lifetime)
        return remaining if remaining <= lim else lim

    def advance(self, t_target, max_steps=None):
        n = 0
        while self.t < t_target and (max_steps is None or n < max_steps):
            dt = self.next_dt(t_target)
            last = dt == t_target - self.t
            self.lie_step(dt)
            self.t = t_target if last else self.t + dt
            self.steps += 1
            n += 1
        return n
