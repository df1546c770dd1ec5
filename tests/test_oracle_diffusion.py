"""Pins for the oracle's diffusion (Sec. 3.7, App. A) and RKL2 (Sec. 3.7.2)."""
import math

import numpy as np
import pytest

import oracle as O
import sft_inputs as I

NU500 = 500.0 * O.KM2_S_TO_RS2_HR


def test_stencil_equals_assembled_matrix_with_variable_nu():
    """Eq. (diffusion_op) applied directly == the Eq. (diffusion_matrix)
    coefficients assembled entry by entry (brute force, 8 x 16, random nu)."""
    rng = np.random.default_rng(1)
    g = O.Grid(8, 16)
    nu = rng.uniform(0.5, 2.0, size=(g.nt - 1, g.np))
    B = rng.normal(size=(g.nt, g.np))
    B[0] = B[0, 0]
    B[-1] = B[-1, 0]
    L = O.diffusion_operator(g, B, nu)
    M = O.diffusion_matrix(g, nu)
    got = M @ O.unique_unknowns(B)
    np.testing.assert_allclose(got, O.unique_unknowns(L), rtol=1e-12, atol=1e-12 * np.abs(L).max())


def test_matrix_is_self_adjoint_and_annihilates_constants():
    rng = np.random.default_rng(2)
    g = O.Grid(10, 12)
    nu = rng.uniform(0.5, 2.0, size=(g.nt - 1, g.np))
    M = O.diffusion_matrix(g, nu).toarray()
    w = O.unique_unknowns(g.area)
    w[0] = w[-1] = g.cap_area
    WM = w[:, None] * M
    assert np.abs(WM - WM.T).max() <= 1e-13 * np.abs(WM).max()
    assert np.abs(M.sum(axis=1)).max() <= 1e-12 * np.abs(M).max()


def test_diffusion_conserves_total_flux():
    g = O.Grid(24, 48)
    B = I.initial_map(24, 48, seed=11)
    L = O.diffusion_operator(g, B, O.constant_nu(g, NU500))
    assert abs((g.area * L).sum()) <= 1e-14 * (g.area * np.abs(L)).sum()


def test_euler_limit_bounds_the_spectrum():
    g = O.Grid(9, 12)
    nu = O.constant_nu(g, 1.0)
    M = O.diffusion_matrix(g, nu).toarray()
    lam = np.linalg.eigvals(M)
    assert np.abs(lam.imag).max() < 1e-9 * np.abs(lam).max()
    dte = O.euler_dt_limit(g, nu)
    true_limit = 2.0 / np.abs(lam.real).max()
    assert dte <= true_limit * (1 + 1e-12)
    assert dte >= 0.5 * true_limit


def test_euler_limit_matches_paper_512x1024(paper_values):
    v = paper_values["euler_dt_512x1024_nu500_hours"]
    g = O.Grid(512, 1024)
    dte = O.euler_dt_limit(g, O.constant_nu(g, NU500))
    assert dte == pytest.approx(v["value"], rel=v["rel_tol"])


def _rkl2_scalar(s, z):
    z = np.asarray(z, dtype=np.complex128)
    return O.rkl2_advance(np.ones_like(z), 1.0, lambda y: z * y, s)


@pytest.mark.parametrize("s", [2, 3, 4, 7, 16, 50, 145, 600])
def test_rkl2_stable_on_its_interval(s):
    """|R_s(z)| <= 1 for z in [-(s^2+s-2)/2, 0] (Meyer, Balsara & Aslam 2014)."""
    z = np.linspace(-(s * s + s - 2) / 2.0, 0.0, 40001)
    assert np.abs(_rkl2_scalar(s, z)).max() <= 1.0 + 1e-9


@pytest.mark.parametrize("s", [2, 5, 40])
def test_rkl2_is_second_order(s):
    for z in (1e-2, 2e-3):
        err = abs(_rkl2_scalar(s, [-z])[0] - (1 - z + z * z / 2))
        assert err < 0.5 * z**3


def test_rkl2_stage_count_is_minimal():
    for ratio in (0.3, 1.0, 1.01, 7.9, 20888.0, 1.4e7):
        s = O.rkl2_stage_count(ratio, 1.0)
        assert (s * s + s - 2) / 4.0 >= ratio
        assert s == 2 or ((s - 1) ** 2 + (s - 1) - 2) / 4.0 < ratio


def test_soccer_ball_second_order_in_space(paper_values):
    """Eq. (soccerball) decays as exp(-42 nu t); the discrete solution
    converges at second order (Sec. 3.8)."""
    errs = []
    for nt, np_ in ((32, 64), (64, 128), (128, 256)):
        g = O.Grid(nt, np_)
        r = O.Realization(g, O.Params(advection=False, nu=500.0), I.soccer_ball(nt, np_))
        r.dt_adv = 8.0
        r.advance(672.0)
        errs.append(O.hh_metric(r.B, I.soccer_ball(nt, np_, NU500, 672.0)))
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(1.8 <= o <= 2.2 for o in orders), orders


def test_axial_dipole_decay_and_pole_cap():
    """l = 1: cos(theta) decays as exp(-2 nu t); the pole cap value follows it
    and the measured axial dipole converges at second order."""
    dec = math.exp(-2.0 * NU500 * 672.0)
    errD = []
    for nt, np_ in ((32, 64), (64, 128)):
        g = O.Grid(nt, np_)
        r = O.Realization(g, O.Params(advection=False, nu=500.0), I.dipole(nt, np_, 1.0))
        r.dt_adv = 24.0
        r.advance(672.0)
        assert r.B[0, 0] == pytest.approx(dec, rel=2e-5)
        assert r.B[-1, 0] == pytest.approx(-dec, rel=2e-5)
        errD.append(abs(O.diagnostics(g, r.B).dipole_axial / dec - 1))
    assert 1.8 <= math.log2(errD[0] / errD[1]) <= 2.2


def test_soccer_ball_one_rkl2_step_matches_paper(paper_values):
    """Sec. 3.7.2: one 672 hr RKL2 step of the diffusion-only soccer ball at
    512x1024 ends with HH = 8.0e-5.  The oracle's matrix form (pinned equal
    to its stencil above) is used for speed."""
    v = paper_values["soccer_ball_rkl2_one_step_hh"]
    nu = v["nu_km2_s"] * O.KM2_S_TO_RS2_HR
    g = O.Grid(v["nt"], v["np"])
    M = O.diffusion_matrix(g, O.constant_nu(g, nu))
    dte = 1.0 / np.abs(M.diagonal()).max()
    s = O.rkl2_stage_count(v["t_hours"], dte)
    u0 = O.unique_unknowns(I.soccer_ball(g.nt, g.np))
    u = O.rkl2_advance(u0, v["t_hours"], lambda y: M @ y, s)
    ex = O.unique_unknowns(I.soccer_ball(g.nt, g.np, nu, v["t_hours"]))
    assert O.hh_metric(u, ex) == pytest.approx(v["value"], rel=v["rel_tol"])


# --------------------------------------------------------------------------
# Eq. (diffgrid): grid-based diffusivity (the flux-preserving smoother)
# --------------------------------------------------------------------------
def test_grid_nu_closed_form_and_conservation():
    g = O.Grid(65, 128)
    nu = O.grid_nu(g, 0.5)
    th0 = 0.5 * g.dth   # theta_{1/2}
    assert nu[0, 0] == pytest.approx(0.5 * (g.dth ** 2 + (g.dph * math.sin(th0)) ** 2), rel=1e-15)
    assert np.all(nu[:, 1:] == nu[:, :1])             # uniform in phi
    assert nu[(g.nt - 1) // 2 - 1].max() <= 0.5 * (g.dth ** 2 + g.dph ** 2)
    B = I.initial_map(65, 128, seed=11)
    L = O.diffusion_operator(g, B, nu)
    assert abs((g.area * L).sum()) <= 1e-13 * (g.area * np.abs(L)).sum()
    # the operator equals the entry-by-entry Eq. (diffusion_matrix) assembly
    M = O.diffusion_matrix(g, nu)
    u = O.unique_unknowns(B)
    assert np.abs(M @ u - O.unique_unknowns(L)).max() <= 1e-12 * np.abs(L).max()


def test_grid_nu_smoother_flattens_a_blob_and_keeps_flux():
    """One smoothing hour with alpha = 0.5 on a narrow Gaussian (sigma = 2
    cells): the peak drops, the blob widens, the total flux is unchanged.
    (A single-cell spike rings under one large RKL2 step: the paper's PTL
    limit, which it only cites, is what keeps such runs oscillation-free.)"""
    g = O.Grid(65, 128)
    th, ph = np.meshgrid(g.theta, g.phi, indexing="ij")
    d2 = ((th - g.theta[20]) / g.dth) ** 2 + ((ph - g.phi[40]) * np.sin(g.theta[20]) / g.dth) ** 2
    B = 1000.0 * np.exp(-d2 / 8.0)
    r = O.Realization(g, O.Params(advection=False, nu_grid_alpha=0.5), B)
    r.advance(1.0)
    assert r.B.max() < 0.95 * B.max()
    assert r.B[26, 40] > B[26, 40] and r.B.min() > -1e-3 * B.max()   # the tail (3 sigma) grows
    assert O.total_flux(g, r.B) == pytest.approx(O.total_flux(g, B), rel=1e-13)


def test_grid_nu_euler_limit_scales_inversely_with_alpha():
    g = O.Grid(65, 128)
    assert O.euler_dt_limit(g, O.grid_nu(g, 0.5)) == pytest.approx(
        2.0 * O.euler_dt_limit(g, O.grid_nu(g, 1.0)), rel=1e-14)


# --------------------------------------------------------------------------
# Sec. 3.7.2: explicit forward-Euler diffusion (the paper's reference and
# testing stepper), sub-cycled at the Euler limit
# --------------------------------------------------------------------------
def _fewest_substeps(dt, dte):
    """Brute force: the smallest n with dt / n <= dte."""
    n = 1
    while dt / n > dte:
        n += 1
    return n


@pytest.mark.parametrize("dt,dte", [(1.0, 1.0), (1.0, 0.3), (2.5, 0.25), (7.0, 0.07 * 1.0000001),
                                    (0.01, 5.0)])
def test_fe_diffusion_scalar_is_the_euler_power(dt, dte):
    """On the scalar test dY/dt = z Y the sub-cycled stepper is exactly
    (1 + z dt/n)^n with n the fewest sub-steps that respect the limit."""
    n = _fewest_substeps(dt, dte)
    z = np.array([-0.3, -1.7 + 0.4j, 0.2j, -3.0 / dte])
    got = O.fe_diffusion_advance(np.ones_like(z), dt, lambda y: z * y, dte)
    want = (1.0 + z * (dt / n)) ** n
    np.testing.assert_allclose(got, want, rtol=1e-13, atol=0)


def test_fe_diffusion_is_first_order_in_the_substep():
    """Against exp(dt M) u0 of the assembled Eq. (diffusion_matrix) (the
    exact semi-discrete solution, independent of any stepper), the error
    halves with the sub-step: first order."""
    from scipy.sparse.linalg import expm_multiply
    g = O.Grid(17, 32)
    nu = O.constant_nu(g, 0.02)
    M = O.diffusion_matrix(g, nu)
    u0 = O.unique_unknowns(I.initial_map(17, 32, seed=5))
    T = 3.0
    exact = expm_multiply(T * M, u0)
    dte = O.euler_dt_limit(g, nu)
    errs = []
    for k in range(3):
        u = O.fe_diffusion_advance(u0, T, lambda y: M @ y, dte / 2 ** k)
        errs.append(np.abs(u - exact).max())
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(0.9 <= o <= 1.1 for o in orders), orders


def test_fe_diffusion_axial_dipole_decays_as_exp_minus_2nut():
    """l = 1: the pole cap of cos(theta) follows exp(-2 nu t) (App. A cap,
    Sec. 3.7.2 explicit Euler)."""
    g = O.Grid(32, 64)
    nu = O.constant_nu(g, NU500)
    dte = O.euler_dt_limit(g, nu)
    B = I.dipole(32, 64, 1.0)
    out = O.fe_diffusion_advance(B, 672.0, lambda y: O.diffusion_operator(g, y, nu), dte)
    assert out[0, 0] == pytest.approx(math.exp(-2.0 * NU500 * 672.0), rel=2e-4)


def test_fe_diffusion_stable_at_the_limit_and_unstable_beyond():
    """With sub-steps at the Gershgorin limit the stiffest mode never grows;
    with sub-steps 5 % beyond 2/|lambda_max| (the true explicit-Euler limit)
    it grows without bound."""
    g = O.Grid(9, 12)
    nu = O.constant_nu(g, 1.0)
    M = O.diffusion_matrix(g, nu).toarray()
    lam, V = np.linalg.eig(M)
    i = np.argmax(np.abs(lam.real))
    v = np.real(V[:, i])
    dte = O.euler_dt_limit(g, nu)
    stable = O.fe_diffusion_advance(v, 200 * dte, lambda y: M @ y, dte)
    assert np.abs(stable).max() <= np.abs(v).max() * (1 + 1e-9)
    h = 1.05 * 2.0 / abs(lam[i].real)
    grown = O.fe_diffusion_advance(v, 200 * h, lambda y: M @ y, h)
    assert np.abs(grown).max() > 1e3 * np.abs(v).max()


# --------------------------------------------------------------------------
# Sec. 3.7.2: RKG2(3/2), the paper's default super time stepper
# --------------------------------------------------------------------------
def _rkg2_scalar(s, z, record=None):
    z = np.asarray(z, dtype=np.complex128)

    def L(y):
        if record is not None:
            record.append(np.array(y))
        return z * y
    return O.rkg2_advance(np.ones_like(z), 1.0, L, s)


@pytest.mark.parametrize("s", [2, 3, 5, 16, 81, 400])
def test_rkg2_is_the_shifted_gegenbauer_polynomial(s):
    """The s-stage recurrence equals a + b C_s(1 + w1 z), C_s the Gegenbauer
    polynomial with parameter 3/2 (scipy), with w1 = C_s'(1)/C_s''(1),
    b = C_s''(1)/C_s'(1)^2, a = 1 - b C_s(1): the derivatives from
    d/dx C_n^(l) = 2 l C_{n-1}^(l+1) evaluated by scipy at x = 1."""
    from scipy.special import eval_gegenbauer as C
    c1 = 3.0 * C(s - 1, 2.5, 1.0)
    c2 = 15.0 * C(s - 2, 3.5, 1.0) if s >= 2 else 0.0
    w1, b = c1 / c2, c2 / c1 ** 2
    a = 1.0 - b * C(s, 1.5, 1.0)
    z = np.linspace(-2.0 / w1, 0.0, 997)
    want = a + b * C(s, 1.5, 1.0 + w1 * z)
    got = _rkg2_scalar(s, z).real
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-11)


@pytest.mark.parametrize("s", [2, 3, 4, 7, 16, 50, 145, 600])
def test_rkg2_stable_on_its_interval_with_bounded_stages(s):
    """|R_s(z)| <= 1 on [-(s-1)(s+4)/3, 0], and so is every internal stage
    (internal stability)."""
    z = np.linspace(-(s - 1.0) * (s + 4.0) / 3.0, 0.0, 4001)
    stages = []
    out = _rkg2_scalar(s, z, stages)
    assert np.abs(out).max() <= 1.0 + 1e-9
    assert max(np.abs(y).max() for y in stages) <= 1.0 + 1e-9
    # and it is not stable much beyond the interval (odd s ends at R = -1 + 2a_s... > -1)
    zz = np.array([-(s - 1.0) * (s + 4.0) / 3.0 * 1.3])
    assert abs(_rkg2_scalar(s, zz)[0]) > 1.0


@pytest.mark.parametrize("s", [2, 5, 40])
def test_rkg2_is_second_order(s):
    for z in (1e-2, 2e-3):
        err = abs(_rkg2_scalar(s, [-z])[0] - (1 - z + z * z / 2))
        assert err < 0.5 * z ** 3


def test_rkg2_stage_count_is_minimal():
    for ratio in (0.3, 1.0, 1.01, 7.9, 20888.0, 1.4e7):
        s = O.rkg2_stage_count(ratio, 1.0)
        assert (s * s + 3 * s - 4) / 6.0 >= ratio
        assert s == 2 or ((s - 1) ** 2 + 3 * (s - 1) - 4) / 6.0 < ratio


def test_soccer_ball_one_rkg2_step_matches_paper(paper_values):
    """Sec. 3.7.2: one 672 hr RKG2(3/2) step of the diffusion-only soccer ball
    at 512x1024 ends with HH = 6.3e-5 (RKL2: 8.0e-5), and takes more stages
    than RKL2 in the ratio of the printed run times (0.55 s / 0.45 s)."""
    v = paper_values["soccer_ball_rkg2_one_step_hh"]
    nu = v["nu_km2_s"] * O.KM2_S_TO_RS2_HR
    g = O.Grid(v["nt"], v["np"])
    M = O.diffusion_matrix(g, O.constant_nu(g, nu))
    dte = 1.0 / np.abs(M.diagonal()).max()
    s = O.rkg2_stage_count(v["t_hours"], dte)
    u0 = O.unique_unknowns(I.soccer_ball(g.nt, g.np))
    u = O.rkg2_advance(u0, v["t_hours"], lambda y: M @ y, s)
    ex = O.unique_unknowns(I.soccer_ball(g.nt, g.np, nu, v["t_hours"]))
    assert O.hh_metric(u, ex) == pytest.approx(v["value"], rel=v["rel_tol"])
    r = paper_values["rkg2_over_rkl2_time"]
    assert s / O.rkl2_stage_count(v["t_hours"], dte) == pytest.approx(r["value"], rel=r["rel_tol"])
