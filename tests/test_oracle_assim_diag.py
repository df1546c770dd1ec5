"""Pins for the oracle's assimilation (Sec. 2.3), analysis quantities
(Sec. 2.6), HH metric (Eq. hh) and step driver (Sec. 3.4, 3.5)."""
import math

import numpy as np
import pytest

import oracle as O
import sft_inputs as I


def test_weight_function_strict_limits():
    mu = np.array([0.05, 0.1, 0.1000001, 0.5, 1.0, 0.9])
    lat = np.radians([0.0, 0.0, 0.0, 10.0, 0.0, 60.0])
    F = O.assimilation_weight(mu, lat, 2.0, 0.1, math.radians(60.0))
    np.testing.assert_allclose(F, [0.0, 0.0, 0.1000001**2, 0.25, 1.0, 0.0])


def test_assimilation_limits():
    g = O.Grid(16, 32)
    B = I.initial_map(16, 32, seed=4)
    Bd = I.initial_map(16, 32, seed=5)
    np.testing.assert_allclose(O.assimilate(g, B, Bd, np.ones_like(B), balance=False), Bd,
                               rtol=0, atol=1e-13 * np.abs(Bd).max())
    np.testing.assert_array_equal(O.assimilate(g, B, Bd, np.zeros_like(B), balance=True), B)


def test_balanced_increment_fluxes_are_geometric_mean():
    g = O.Grid(20, 40)
    B = I.initial_map(20, 40, seed=4)
    Bd = 1.7 * I.initial_map(20, 40, seed=5) + 3.0
    F = np.linspace(0, 1, B.size).reshape(B.shape)
    Bn = O.assimilate(g, B, Bd, F, balance=True)
    dB = Bn - B
    pp = (g.area * np.where(dB > 0, dB, 0)).sum()
    pm = (g.area * np.where(dB < 0, dB, 0)).sum()
    raw = F * (Bd - B)
    rp = (g.area * np.where(raw > 0, raw, 0)).sum()
    rm = (g.area * np.where(raw < 0, raw, 0)).sum()
    assert pp == pytest.approx(-pm, rel=1e-12)
    assert pp == pytest.approx(math.sqrt(rp * -rm), rel=1e-12)


def test_map_flux_balance_zeroes_net_flux():
    g = O.Grid(30, 60)
    B = O.flux_balance_map(g, I.initial_map(30, 60, seed=1) + 0.5)
    assert abs(O.total_flux(g, B)) <= 1e-14 * (g.area * np.abs(B)).sum()


def test_dipole_moments_closed_form():
    """D of B = 10 cos(theta) is 10 G; h1 of sin(theta)cos(phi) is 1, h2 0."""
    errs = []
    for nt, np_ in ((64, 128), (128, 256)):
        g = O.Grid(nt, np_)
        d = O.diagnostics(g, I.dipole(nt, np_, 10.0))
        errs.append(abs(d.dipole_axial - 10.0))
        assert abs(d.h1) < 1e-12 and abs(d.h2) < 1e-12
        assert abs(d.flux_signed) <= 1e-12 * d.flux_pos
        th, ph = I.coords(nt, np_)
        E = np.sin(th)[:, None] * np.cos(ph)[None, :]
        e = O.diagnostics(g, E)
        assert e.h1 == pytest.approx(1.0, rel=2e-3)
        assert abs(e.h2) < 1e-12 and abs(e.dipole_axial) < 1e-12
        assert e.dipole_equatorial == pytest.approx(e.h1)
    assert errs[1] < 0.3 * errs[0]   # second-order quadrature error
    assert errs[0] < 1e-2


def test_fluxes_and_polar_regions():
    nt, np_ = 91, 180
    g = O.Grid(nt, np_)
    B = I.initial_map(nt, np_, seed=9)
    d = O.diagnostics(g, B, lat_cut_deg=60.0)
    assert d.flux_pos + d.flux_neg == pytest.approx(d.flux_signed, rel=1e-12, abs=1e-12 * d.flux_pos)
    # rows at latitude >= 60 deg cover the cap down to 60 deg - dtheta/2:
    # 2 pi R^2 (1 - sin 59 deg) for dtheta = 2 deg (midpoint quadrature)
    cap = 2 * math.pi * (1 - math.sin(math.radians(59.0))) * O.R_SUN_CM**2
    assert d.area_pole_n == pytest.approx(cap, rel=2e-3)
    assert d.area_pole_n == pytest.approx(d.area_pole_s, rel=1e-12)
    assert d.brmin == B.min() and d.brmax == B.max() and d.absmin == np.abs(B).min()


def test_hh_metric_values():
    X = I.initial_map(16, 32, seed=2)
    assert O.hh_metric(X, X) == 0.0
    assert O.hh_metric(X, 2 * X) == pytest.approx(1 / math.sqrt(2), rel=1e-14)


def test_dt_controller_lands_on_target():
    """Sec. 3.4: dt starts as the time remaining and is cut to the flow limit,
    so the run hits the target time exactly with ceil(T/dt_adv) steps."""
    g = O.Grid(17, 32)
    p = O.Params(nu=300.0)
    r = O.Realization(g, p, I.dipole(17, 32))
    T = 5.3 * r.dt_adv
    r.advance(T)
    assert r.t == T
    assert r.steps == 6
    r2 = O.Realization(g, p, I.dipole(17, 32))
    assert r2.advance(T, max_steps=2) == 2 and r2.t == pytest.approx(2 * r2.dt_adv)
