"""Seeded synthetic workloads shaped like the paper's runs.

The paper's own inputs (HMI / MagMAP maps, ConFlow flows) are not available,
so these closed-form fields stand in for them:

* ``dipole`` + ``bipolar_pairs``: a 10 G axial dipole plus tilted bipolar
  active-region pairs (peak 300-1000 G, sigma 2-4 deg, Joy tilt 0.5*lat,
  leading polarity equatorward, Hale sign flipped between hemispheres).
* ``draw_realization_params``: per-realization flow/diffusion parameters
  (rotation coefficients +-10 %, meridional amplitude U[10,20] m/s,
  eta U[250,750] km^2/s).
* ``ObservationStream``: an analytic "hidden truth" (regions that emerge
  once a day at |lat| 5-35 deg, drift with the rotation rate of their
  latitude, and decay) and an observer mu map of the Earth-facing hemisphere.
* ``soccer_ball`` / ``gaussian_pair``: the paper's two validation fields
  (Sec. 3.1) with their closed-form time dependence.

All randomness comes from SplitMix64 (Steele, Lea & Flood 2014) so the same
seed gives the same numbers on every machine.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

MASK64 = (1 << 64) - 1
CARRINGTON_SYNODIC_DAYS = 27.2753


class SplitMix64:
    """SplitMix64 counter-based generator (Steele, Lea & Flood 2014)."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform(self, lo=0.0, hi=1.0) -> float:
        return lo + (hi - lo) * ((self.next_u64() >> 11) * (1.0 / (1 << 53)))

    def normal(self) -> float:
        u1 = max(self.uniform(), 1e-300)
        u2 = self.uniform()
        return math.sqrt(-2.0 * math.log(u1)) * math.cos(2.0 * math.pi * u2)


def coords(nt: int, np_: int):
    """Colatitude (poles included) and unique-longitude coordinates."""
    theta = np.arange(nt) * (math.pi / (nt - 1))
    theta[-1] = math.pi
    phi = np.arange(np_) * (2.0 * math.pi / np_)
    return theta, phi


def dipole(nt: int, np_: int, b0=10.0):
    """Axial dipole b0*cos(theta) (G)."""
    theta, _ = coords(nt, np_)
    return np.repeat((b0 * np.cos(theta))[:, None], np_, axis=1)


@dataclass
class BipolarPair:
    lat: float      # deg, pair centre
    lon: float      # deg
    peak: float     # G, leading-polarity sign included
    sigma: float    # deg
    sep: float      # deg, centre-to-centre separation
    tilt: float     # deg (Joy)


def draw_pairs(rng: SplitMix64, n, lat_lo=5.0, lat_hi=35.0, peak=(300.0, 1000.0),
               sigma=(2.0, 4.0), joy=0.5, sep_sigmas=3.0, cycle_sign=1.0):
    """Random active-region pairs.  Leading (westward, +phi) polarity is
    -cycle_sign in the north and +cycle_sign in the south (Hale)."""
    out = []
    for _ in range(n):
        hemi = 1.0 if rng.uniform() < 0.5 else -1.0
        lat = hemi * rng.uniform(lat_lo, lat_hi)
        lon = rng.uniform(0.0, 360.0)
        amp = rng.uniform(*peak)
        sig = rng.uniform(*sigma)
        lead_sign = -cycle_sign * hemi
        out.append(BipolarPair(lat, lon, lead_sign * amp, sig, sep_sigmas * sig, joy * abs(lat)))
    return out


def _gauss_on_sphere(theta, phi, lat_c, lon_c, sigma_rad):
    lat = 0.5 * math.pi - theta[:, None]
    cosd = (np.sin(lat) * math.sin(lat_c)
            + np.cos(lat) * math.cos(lat_c) * np.cos(phi[None, :] - lon_c))
    d = np.arccos(np.clip(cosd, -1.0, 1.0))
    return np.exp(-0.5 * (d / sigma_rad) ** 2)


def render_pairs(nt, np_, pairs, amp_scale=1.0, sigma_scale=1.0, lon_shift_deg=None):
    """Sum of the pairs' two Gaussian lobes on the grid (G).  The leading
    lobe sits half a separation ahead in longitude and tilted equatorward."""
    theta, phi = coords(nt, np_)
    B = np.zeros((nt, np_))
    for i, p in enumerate(pairs):
        half = 0.5 * math.radians(p.sep)
        tilt = math.radians(p.tilt)
        latc = math.radians(p.lat)
        lonc = math.radians(p.lon + (0.0 if lon_shift_deg is None else lon_shift_deg[i]))
        dlat = half * math.sin(tilt) * (-1.0 if p.lat > 0 else 1.0)
        dlon = half * math.cos(tilt) / max(math.cos(latc), 1e-3)
        sig = math.radians(p.sigma) * sigma_scale
        a = p.peak * amp_scale
        B += a * _gauss_on_sphere(theta, phi, latc + dlat, lonc + dlon, sig)
        B -= a * _gauss_on_sphere(theta, phi, latc - dlat, lonc - dlon, sig)
    # a pole row is one point: keep its k = 0 value everywhere
    B[0, :] = B[0, 0]
    B[-1, :] = B[-1, 0]
    return B


def initial_map(nt, np_, seed=1, n_pairs=12, dipole_g=10.0):
    """Dipole plus seeded bipolar pairs (net flux is balanced afterwards by
    the solver's own map flux-balance option)."""
    rng = SplitMix64(seed)
    return dipole(nt, np_, dipole_g) + render_pairs(nt, np_, draw_pairs(rng, n_pairs))


# --------------------------------------------------------------------------
# flow parameters
# --------------------------------------------------------------------------
def omega_to_dr_coeffs(o0, o2, o4, frame_deg_day=360.0 / CARRINGTON_SYNODIC_DAYS,
                       r_sun_m=6.96e8):
    """Rotation rate Omega(lat) = o0 + o2 sin^2(lat) + o4 sin^4(lat) (deg/day)
    relative to a frame rotating at frame_deg_day, expressed as the (d0, d2,
    d4) m/s coefficients of v_phi = (d0 + d2 cos^2 th + d4 cos^4 th) sin th."""
    k = math.radians(1.0) / 86400.0 * r_sun_m
    return (o0 - frame_deg_day) * k, o2 * k, o4 * k


def meridional_sin2lat(u_ms):
    """Poleward flow u*sin(2 lat) as the (m1, m3, m5) m/s coefficients of
    v_theta = -(m1 cos th + m3 cos^3 th + m5 cos^5 th) sin th."""
    return 2.0 * u_ms, 0.0, 0.0


DEFAULT_OMEGA = (13.38, -2.30, -1.62)


def draw_realization_params(n, seed=3, spread=0.10, u_range=(10.0, 20.0),
                            eta_range=(250.0, 750.0)):
    """Per-realization (d0, d2, d4, m1, m3, m5, nu) tuples."""
    rng = SplitMix64(seed)
    out = []
    for _ in range(n):
        o = [c * rng.uniform(1.0 - spread, 1.0 + spread) for c in DEFAULT_OMEGA]
        d = omega_to_dr_coeffs(*o)
        m = meridional_sin2lat(rng.uniform(*u_range))
        eta = rng.uniform(*eta_range)
        out.append(tuple(d) + tuple(m) + (eta,))
    return out


# --------------------------------------------------------------------------
# observations (hidden truth + observer geometry)
# --------------------------------------------------------------------------
class ObservationStream:
    """Analytic stand-in for hourly magnetogram-derived maps.

    Truth(t) = dipole + regions; region i emerges at day i (one per day),
    rotates at Omega(lat) relative to the Carrington frame, decays with an
    e-folding time of 10 days and spreads as sigma*sqrt(1 + age/5 d).
    Observer: sub-Earth Carrington longitude phi_E(t) = phi_E0 - 2 pi t / P_syn,
    disk-centre latitude 0, mu = max(0, sin th cos(phi - phi_E)).
    """

    def __init__(self, nt, np_, seed=2, days=365, phi_e0_deg=180.0):
        self.nt, self.np = nt, np_
        rng = SplitMix64(seed)
        self.pairs = draw_pairs(rng, days)
        self.phi_e0 = math.radians(phi_e0_deg)
        self.theta, self.phi = coords(nt, np_)

    def truth(self, t_hours):
        day = t_hours / 24.0
        B = dipole(self.nt, self.np)
        live, amp, sig, shift = [], [], [], []
        for i, p in enumerate(self.pairs):
            age = day - i
            if age < 0:
                break
            s2 = math.sin(math.radians(p.lat)) ** 2
            rate = DEFAULT_OMEGA[0] + DEFAULT_OMEGA[1] * s2 + DEFAULT_OMEGA[2] * s2 * s2
            live.append(p)
            amp.append(math.exp(-age / 10.0))
            sig.append(math.sqrt(1.0 + age / 5.0))
            shift.append((rate - 360.0 / CARRINGTON_SYNODIC_DAYS) * age)
        for p, a, s, sh in zip(live, amp, sig, shift):
            B += render_pairs(self.nt, self.np, [p], amp_scale=a / s**2,
                              sigma_scale=s, lon_shift_deg=[sh])
        return B

    def truth_torch(self, t_hours, device="cuda", chunk=32):
        """truth(t_hours) evaluated with torch (FP64) on `device`: the same
        dipole and pair lobes, all live regions of a chunk at once.  For
        year-long hourly streams, where the host version is too slow."""
        import torch
        day = t_hours / 24.0
        th = torch.as_tensor(self.theta, dtype=torch.float64, device=device)
        ph = torch.as_tensor(self.phi, dtype=torch.float64, device=device)
        lat = (0.5 * math.pi - th)[None, :, None]
        sl, cl = torch.sin(lat), torch.cos(lat)
        B = (10.0 * torch.cos(th))[:, None].expand(self.nt, self.np).clone()
        lobes = []  # (amplitude, lat, lon, sigma) of every live lobe
        for i, p in enumerate(self.pairs):
            age = day - i
            if age < 0:
                break
            s2 = math.sin(math.radians(p.lat)) ** 2
            rate = DEFAULT_OMEGA[0] + DEFAULT_OMEGA[1] * s2 + DEFAULT_OMEGA[2] * s2 * s2
            a = math.exp(-age / 10.0)
            sg = math.sqrt(1.0 + age / 5.0)
            sh = (rate - 360.0 / CARRINGTON_SYNODIC_DAYS) * age
            half = 0.5 * math.radians(p.sep)
            tilt = math.radians(p.tilt)
            latc = math.radians(p.lat)
            lonc = math.radians(p.lon + sh)
            dlat = half * math.sin(tilt) * (-1.0 if p.lat > 0 else 1.0)
            dlon = half * math.cos(tilt) / max(math.cos(latc), 1e-3)
            amp = p.peak * a / sg ** 2
            sig = math.radians(p.sigma) * sg
            lobes.append((amp, latc + dlat, lonc + dlon, sig))
            lobes.append((-amp, latc - dlat, lonc - dlon, sig))
        for c0 in range(0, len(lobes), chunk):
            L = torch.tensor(lobes[c0:c0 + chunk], dtype=torch.float64, device=device)
            a, la, lo, sg = (L[:, q][:, None, None] for q in range(4))
            cosd = sl * torch.sin(la) + cl * torch.cos(la) * torch.cos(ph[None, None, :] - lo)
            d = torch.arccos(torch.clamp(cosd, -1.0, 1.0))
            B += (a * torch.exp(-0.5 * (d / sg) ** 2)).sum(0)
        B[0, :] = B[0, 0].clone()
        B[-1, :] = B[-1, 0].clone()
        return B

    def mu_torch(self, t_hours, device="cuda"):
        """mu(t_hours) evaluated with torch (FP64) on `device`."""
        import torch
        phi_e = self.phi_e0 - 2.0 * math.pi * t_hours / (CARRINGTON_SYNODIC_DAYS * 24.0)
        th = torch.as_tensor(self.theta, dtype=torch.float64, device=device)
        ph = torch.as_tensor(self.phi, dtype=torch.float64, device=device)
        m = torch.clamp(torch.sin(th)[:, None] * torch.cos(ph[None, :] - phi_e), min=0.0)
        m[0, :] = 0.0
        m[-1, :] = 0.0
        return m

    def mu(self, t_hours):
        phi_e = self.phi_e0 - 2.0 * math.pi * t_hours / (CARRINGTON_SYNODIC_DAYS * 24.0)
        m = np.sin(self.theta)[:, None] * np.cos(self.phi[None, :] - phi_e)
        m = np.maximum(m, 0.0)
        m[0, :] = 0.0
        m[-1, :] = 0.0
        return m


# --------------------------------------------------------------------------
# the paper's validation fields (Sec. 3.1)
# --------------------------------------------------------------------------
def _sph_y6(theta, phi):
    """Real fully normalised Y_6^0 and Y_6^5 (explicit Legendre forms)."""
    x = np.cos(theta)[:, None]
    s = np.sin(theta)[:, None]
    p60 = (231 * x**6 - 315 * x**4 + 105 * x**2 - 5) / 16.0
    p65 = 10395.0 * x * s**5
    n60 = math.sqrt(13.0 / (4.0 * math.pi))
    n65 = math.sqrt(2.0 * 13.0 / (4.0 * math.pi) * math.factorial(1) / math.factorial(11))
    return n60 * p60 * np.ones((1, phi.size)), n65 * p65 * np.cos(5.0 * phi)[None, :]


def soccer_ball(nt, np_, nu_rs2_hr=0.0, t_hours=0.0, omega_rad_hr=0.0):
    """Eq. (soccerball): exp(-42 nu t)(Y_6^0 + sqrt(14/11) Y_6^5), optionally
    rigidly rotated by omega*t in phi."""
    theta, phi = coords(nt, np_)
    y0, y5 = _sph_y6(theta, phi - omega_rad_hr * t_hours)
    return math.exp(-42.0 * nu_rs2_hr * t_hours) * (y0 + math.sqrt(14.0 / 11.0) * y5)


def gaussian_pair(nt, np_, vtheta_rad_hr=0.0, vphi_rad_hr=0.0, t_hours=0.0, sigma=0.03):
    """Eq. (testblob): two opposite-polarity Gaussians times 1/sin(theta),
    exact under constant v_theta (App. C) and rigid rotation in phi.  The pole
    rows (where 1/sin(theta) is singular and the lobes cancel) are set to 0."""
    theta, phi = coords(nt, np_)
    th = theta[:, None]
    ph = phi[None, :]
    shift_t = th - math.pi / 4 - vtheta_rad_hr * t_hours

    def wrap(a):
        return (a + math.pi) % (2.0 * math.pi) - math.pi

    g1 = np.exp(-shift_t**2 / sigma - wrap(ph - math.pi / 2 - vphi_rad_hr * t_hours) ** 2 / sigma)
    g2 = np.exp(-shift_t**2 / sigma - wrap(ph - 3 * math.pi / 2 - vphi_rad_hr * t_hours) ** 2 / sigma)
    with np.errstate(divide="ignore", invalid="ignore"):
        B = (g2 - g1) / np.sin(th)
    B[0, :] = 0.0
    B[-1, :] = 0.0
    return B
