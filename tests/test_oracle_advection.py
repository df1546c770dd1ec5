"""Pins for the oracle's advection (Sec. 3.6, App. A, App. B, App. C).

Each test checks the oracle against something the paper or mathematics
fixes: exact conservation, an exact discrete shift, closed-form amplification
polynomials, exactness on linear data, the ENO property, and the
convergence orders the paper reports.
"""
import math

import numpy as np
import pytest

import oracle as O
import sft_inputs as I

OMEGA_ROT = 2.0 * math.pi / 672.0   # rad/hr: one rotation in 672 hr (Sec. 3.1)


def _rigid(g, omega=OMEGA_ROT):
    vt = np.zeros(g.nt - 1)
    vp = omega * g.sin_t
    return vt, vp


def test_units_constants(paper_values):
    assert O.M_S_TO_RS_HR == pytest.approx(paper_values["m_s_to_rs_hr"]["value"], rel=1e-15)
    assert O.KM2_S_TO_RS2_HR == pytest.approx(paper_values["km2_s_to_rs2_hr"]["value"], rel=1e-13)
    v = paper_values["rigid_rotation_km_s"]
    # 1.80766 km/s at the equator is one rotation per 672 hr
    assert v["value"] * 1e3 * O.M_S_TO_RS_HR == pytest.approx(2 * math.pi / v["period_hours"], rel=1e-5)


@pytest.mark.parametrize("space", ["weno3", "upwind"])
def test_advection_operator_conserves_total_flux(space):
    g = O.Grid(40, 96)
    B = I.initial_map(40, 96, seed=7)
    vt, vp = O.flow_profiles(g, 46.0, -262.0, -379.0, 22.0, 11.0, -28.0)
    FA = O.advection_operator(g, B, vt, vp, space)
    scale = (g.area * np.abs(FA)).sum()
    assert abs((g.area * FA).sum()) <= 1e-14 * scale
    # and through a whole SSPRK(4,3) step
    dt = O.advection_dt_limit(g, vt, vp)
    B1 = O.ssprk43_advance(B, dt, lambda f: O.advection_operator(g, f, vt, vp, space))
    tot = (g.area * np.abs(B)).sum()
    assert abs(O.total_flux(g, B1) - O.total_flux(g, B)) <= 1e-14 * tot


def test_fe_upwind_courant_one_is_exact_shift():
    """Rigid rotation, v_theta = 0, Courant number exactly 1 in phi:
    forward Euler + upwind moves every row by one cell per step."""
    g = O.Grid(20, 48)
    B0 = I.initial_map(20, 48, seed=3)
    vt, vp = _rigid(g)
    dt = g.dph / OMEGA_ROT
    B = B0.copy()
    for n in range(1, 6):
        B = O.fe_advance(B, dt, lambda f: O.advection_operator(g, f, vt, vp, "upwind"))
        ref = np.roll(B0, n, axis=1)
        ref[0] = B0[0]
        ref[-1] = B0[-1]
        assert np.abs(B - ref).max() <= 1e-12 * np.abs(B0).max()


def test_constant_field_is_steady_under_rotation_only():
    g = O.Grid(33, 64)
    vt = np.zeros(g.nt - 1)
    _, vp = O.flow_profiles(g, 46.0, -262.0, -379.0, 0, 0, 0)
    B = np.full((g.nt, g.np), 3.7)
    for space in ("weno3", "upwind"):
        assert np.abs(O.advection_operator(g, B, vt, vp, space)).max() <= 1e-13


def test_weno_exact_on_linear_data():
    """Both WENO3 polynomials reproduce linear data at the face, so the flux
    is exact whatever the weights (App. B)."""
    rng = np.random.default_rng(0)
    for _ in range(20):
        a, b = rng.normal(size=2)
        LM = a + b * np.arange(-2, 1)   # values at i-2, i-1, i
        face = a + b * (-0.5)           # value at i-1/2
        F = O.weno3_face_flux(LM[0], LM[1], LM[2], 0.0, 0.0, 0.0, 1e-3)
        assert F == pytest.approx(face, abs=1e-13)
        LP = a + b * np.arange(-1, 2)   # values at i-1, i, i+1
        F = O.weno3_face_flux(0.0, 0.0, 0.0, LP[0], LP[1], LP[2], 1e-3)
        assert F == pytest.approx(face, abs=1e-13)


def test_weno_linear_weights_give_third_order_stencil():
    """Smooth data (beta -> 0 relative to eps): u- -> -1/6 u_{i-2} + 5/6 u_{i-1}
    + 1/3 u_i, the third-order upwind-biased face value."""
    x = np.array([-2.0, -1.0, 0.0])
    u = np.array([0.3, 0.7, -0.2]) * 1e-6   # tiny differences: weights linear
    F = O.weno3_face_flux(u[0], u[1], u[2], 0.0, 0.0, 0.0, 1.0)
    assert F == pytest.approx(-u[0] / 6 + 5 * u[1] / 6 + u[2] / 3, rel=1e-9)
    del x


def test_weno_picks_smooth_stencil_at_a_jump():
    F = O.weno3_face_flux(0.0, 0.0, 1.0, 0.0, 0.0, 0.0, 1e-3)   # jump between i-1 and i
    assert abs(F) < 1e-5
    F = O.weno3_face_flux(0.0, 0.0, 0.0, 1.0, 0.0, 0.0, 1e-3)   # jump between i-1 and i (left-moving)
    assert abs(F) < 1e-5


def test_upwind_flux_forms():
    assert O.upwind_face_flux(2.0, 3.0, 5.0, 1.0) == pytest.approx(6.0)      # v > 0: B_{i-1}
    assert O.upwind_face_flux(-2.0, 3.0, 5.0, 1.0) == pytest.approx(-10.0)   # v < 0: B_i
    assert O.upwind_face_flux(0.0, 3.0, 5.0, 1.0) == 0.0
    # Reading: with the printed flux formula the central average is alpha_uw = 0
    # (the text's "alpha_uw = 0.5 is central" contradicts the formula).
    assert O.upwind_face_flux(2.0, 3.0, 5.0, 0.0) == pytest.approx(8.0)
    assert O.upwind_face_flux(2.0, 3.0, 5.0, 0.5) == pytest.approx(7.0)


@pytest.mark.parametrize("z", [-0.3, -1.7 + 0.4j, -2.5, 0.2 - 1.1j, -3.9])
def test_ssp_rk_amplification_polynomials(z):
    one = np.array([1.0 + 0j])
    lin = lambda f: -z * f   # F_A(f) = -z f, dt = 1
    assert O.fe_advance(one, 1.0, lin)[0] == pytest.approx(1 + z)
    assert O.ssprk33_advance(one, 1.0, lin)[0] == pytest.approx(1 + z + z**2 / 2 + z**3 / 6)
    assert O.ssprk43_advance(one, 1.0, lin)[0] == pytest.approx(1 + z + z**2 / 2 + z**3 / 6 + z**4 / 48)


def test_cfl_limits_closed_form():
    g = O.Grid(65, 128)
    vt, vp = _rigid(g)
    assert O.advection_dt_limit(g, vt, vp, "ssprk43", 0.9) == pytest.approx(0.9 * g.dph / OMEGA_ROT, rel=1e-12)
    assert O.advection_dt_limit(g, vt, vp, "fe", 0.9) == pytest.approx(0.45 * g.dph / OMEGA_ROT, rel=1e-12)
    vt = np.full(g.nt - 1, 0.01)
    vp = np.zeros(g.nt)
    assert O.advection_dt_limit(g, vt, vp, "ssprk43", 1.0) == pytest.approx(g.dth / 0.01, rel=1e-12)


def _phi_error(np_, space, eps):
    nt = 16
    g = O.Grid(nt, np_)
    p = O.Params(d0=OMEGA_ROT / O.M_S_TO_RS_HR, d2=0, d4=0, m1=0, m3=0, m5=0,
                 diffusion="off", adv_space=space, eps_w=eps)
    r = O.Realization(g, p, I.gaussian_pair(nt, np_))
    r.advance(672.0)
    return O.hh_metric(r.B, I.gaussian_pair(nt, np_, vphi_rad_hr=OMEGA_ROT, t_hours=672.0))


def _theta_error(nt, space, eps):
    np_ = 16
    vth = (math.pi / 2) / 672.0
    g = O.Grid(nt, np_)
    p = O.Params(d0=0, d2=0, d4=0, m1=0, m3=0, m5=0, diffusion="off", adv_space=space, eps_w=eps)
    r = O.Realization(g, p, I.gaussian_pair(nt, np_))
    r.vt = np.full(nt - 1, vth)
    r.vp = np.zeros(nt)
    r.dt_adv = O.advection_dt_limit(g, r.vt, r.vp)
    r.advance(672.0)
    return O.hh_metric(r.B, I.gaussian_pair(nt, np_, vtheta_rad_hr=vth, t_hours=672.0))


@pytest.mark.parametrize("space,eps,lo,hi", [
    ("weno3", "h", 2.7, 3.4),        # WENO3-CS(h): third order (App. B, Sec. 3.8)
    ("weno3", 1e-12, 1.3, 2.1),      # WENO3 with eps_w = 1e-12: (towards) second order
    ("upwind", "h", 0.5, 1.1),       # upwind: first order (Sec. 3.6.1)
])
def test_theta_advection_order_app_c(space, eps, lo, hi):
    """Gaussians times 1/sin(theta) under constant v_theta are exact (App. C);
    they travel pi/2 in 672 hr (Sec. 3.1)."""
    e1, e2 = _theta_error(256, space, eps), _theta_error(512, space, eps)
    order = math.log2(e1 / e2)
    assert lo <= order <= hi, order


@pytest.mark.parametrize("space,eps,lo,hi", [
    ("weno3", "h", 2.4, 3.4),
    ("weno3", 1e-12, 1.2, 2.0),
    ("upwind", "h", 0.3, 1.1),
])
def test_phi_advection_order_rigid_rotation(space, eps, lo, hi):
    e1, e2 = _phi_error(256, space, eps), _phi_error(512, space, eps)
    order = math.log2(e1 / e2)
    assert lo <= order <= hi, order
    if space == "weno3" and eps == "h":
        assert e2 < _phi_error(512, "weno3", 1e-12)


def test_flow_profiles_closed_forms():
    """Eq. (dr) with d_i from a rotation rate Omega(lat) = o0 + o2 sin^2 + o4 sin^4
    (deg/day, relative to a frame) is v_phi = (Omega - frame) * pi/180/24 * sin(theta)
    in R_sun/hr; Eq. (mf) with m1 = 2U, m3 = m5 = 0 is -U sin(2 theta) (m/s)."""
    g = O.Grid(37, 72)
    o = (13.38, -2.30, -1.62)
    frame = 360.0 / 27.2753
    d = I.omega_to_dr_coeffs(*o, frame_deg_day=frame)
    vt, vp = O.flow_profiles(g, d[0], d[1], d[2], 30.0, 0.0, 0.0)
    lat = g.lat
    omega = o[0] + o[1] * np.sin(lat) ** 2 + o[2] * np.sin(lat) ** 4 - frame
    np.testing.assert_allclose(vp, omega * math.pi / 180 / 24 * g.sin_t, rtol=1e-12, atol=1e-18)
    np.testing.assert_allclose(vt, -15.0 * np.sin(2 * g.theta_h) * O.M_S_TO_RS_HR, rtol=1e-12, atol=1e-20)
    # poleward: negative (toward theta = 0) in the north, positive in the south
    assert vt[: (g.nt - 1) // 2].max() < 0 < vt[(g.nt - 1) // 2:].min()


# --------------------------------------------------------------------------
# Eq. (flow_attenuation): v -> v [1 - tanh(|B_r| / B_0)]
# --------------------------------------------------------------------------
@pytest.mark.parametrize("space", ["weno3", "upwind"])
def test_attenuation_off_in_the_weak_field_limit(space):
    """B_0 -> infinity: the factor is 1 and the operator is the plain one."""
    g = O.Grid(33, 64)
    B = I.initial_map(33, 64, seed=3)
    vt, vp = O.flow_profiles(g, 46.0, -262.0, -379.0, 22.0, 11.0, -28.0)
    plain = O.advection_operator(g, B, vt, vp, space)
    att = O.advection_operator(g, B, vt, vp, space, b0=1e300)
    assert np.abs(att - plain).max() <= 1e-14 * np.abs(plain).max()


@pytest.mark.parametrize("space", ["weno3", "upwind"])
def test_attenuated_operator_conserves_total_flux(space):
    g = O.Grid(40, 96)
    B = I.initial_map(40, 96, seed=7)
    vt, vp = O.flow_profiles(g, 46.0, -262.0, -379.0, 22.0, 11.0, -28.0)
    FA = O.advection_operator(g, B, vt, vp, space, b0=200.0)
    assert abs((g.area * FA).sum()) <= 1e-14 * (g.area * np.abs(FA)).sum()
    assert np.abs(FA - O.advection_operator(g, B, vt, vp, space)).max() > 1e-3 * np.abs(FA).max()


def test_attenuation_of_a_uniform_magnitude_field_scales_the_flow():
    """With |B| = c everywhere the factor is the constant 1 - tanh(c/B_0): the
    upwind operator equals the plain one with the flow scaled by it."""
    g = O.Grid(33, 64)
    rng = np.random.default_rng(5)
    B = np.where(rng.random((33, 64)) < 0.5, -1.0, 1.0) * 700.0
    B[0, :] = 700.0
    B[-1, :] = -700.0
    vt, vp = O.flow_profiles(g, 46.0, -262.0, -379.0, 22.0, 11.0, -28.0)
    a = 1.0 - math.tanh(700.0 / 500.0)
    att = O.advection_operator(g, B, vt, vp, "upwind", b0=500.0)
    scaled = O.advection_operator(g, B, a * vt, a * vp, "upwind")
    assert np.abs(att - scaled).max() <= 1e-13 * np.abs(scaled).max()


def test_saturated_field_is_frozen_under_upwind():
    """|B| >= 20 B_0 gives tanh = 1 in FP64: the attenuated flow is zero and
    the upwind flux vanishes identically (an active region that does not move)."""
    g = O.Grid(33, 64)
    B = 1e4 * (1.0 + I.initial_map(33, 64, seed=9) ** 2 / 1e6)
    B[0, :] = B[0, 0]
    B[-1, :] = B[-1, 0]
    vt, vp = O.flow_profiles(g, 46.0, -262.0, -379.0, 22.0, 11.0, -28.0)
    assert np.all(O.advection_operator(g, B, vt, vp, "upwind", b0=500.0) == 0.0)
