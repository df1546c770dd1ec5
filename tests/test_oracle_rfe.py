"""Pins for the random flux emergence of Sec. 2.4 (oracle).

The normal draws are checked against the normal law (moments, the one-sigma
fraction, independence of maps); the source maps against Eq. (mean) (the
requested unsigned flux per hour is what a map carries) and Eq. (fluxbal)
(zero net flux); the time weights against the exact integral of the linear
interpolation of Eq. (rfe_s); and a whole run against the paper's own RFE
check: with an infinite lifetime the total unsigned flux grows at the
requested rate, with a short lifetime far more slowly, and the net flux
stays zero.
"""
import math

import numpy as np
import pytest

import oracle as O

RATE = 1e23   # Mx / hour


def test_normals_follow_the_normal_law():
    g = O.Grid(257, 512)
    Y = O.rfe_normals(g, seed=11, k=0)[1:-1].ravel()   # interior cells, one draw each
    n = Y.size
    assert abs(Y.mean()) <= 4.0 / math.sqrt(n)
    assert abs(Y.std() - 1.0) <= 4.0 * math.sqrt(0.5 / n)
    frac = np.mean(np.abs(Y) < 1.0)
    assert abs(frac - math.erf(1.0 / math.sqrt(2.0))) <= 4.0 * math.sqrt(0.25 / n)
    Y1 = O.rfe_normals(g, seed=11, k=1)[1:-1].ravel()
    assert abs(np.corrcoef(Y, Y1)[0, 1]) <= 4.0 / math.sqrt(n)
    assert np.array_equal(Y, O.rfe_normals(g, seed=11, k=0)[1:-1].ravel())


@pytest.mark.parametrize("method", [1, 2])
def test_map_carries_the_requested_flux_and_is_balanced(method):
    g = O.Grid(257, 512)
    S = O.rfe_map(g, method, RATE, seed=5, k=3)
    A = g.area * O.R_SUN_CM ** 2
    unsigned = float((A * np.abs(S)).sum())
    assert unsigned == pytest.approx(RATE, rel=0.02)        # Eq. (mean): <|X|> = sqrt(2/pi) sigma
    assert abs(float((A * S).sum())) <= 1e-12 * unsigned     # Eq. (fluxbal)
    assert np.all(S[0] == S[0, 0]) and np.all(S[-1] == S[-1, 0])


def test_method_1_is_larger_where_cells_are_smaller():
    g = O.Grid(257, 512)
    S = np.abs(O.rfe_map(g, 1, RATE, seed=9, k=0))
    polar = (S[5:15] * g.sin_t[5:15, None]).mean()
    equator = (S[123:133] * g.sin_t[123:133, None]).mean()
    assert polar == pytest.approx(equator, rel=0.1)         # |S| ~ 1 / cell area ~ 1 / sin(theta)
    assert S[5:15].mean() > 5.0 * S[123:133].mean()


def test_time_weights_integrate_the_interpolation_exactly():
    tau, t0 = 0.3, 0.05
    f = {k: float(k * k + 1) for k in range(10)}             # a scalar "map" per index

    def S(t):
        k = math.floor((t - t0) / tau)
        al = (t - t0 - k * tau) / tau
        return (1.0 - al) * f[k] + al * f[k + 1]

    for a, b in ((0.1, 0.3), (0.1, 0.5), (0.35, 0.65), (0.05, 0.35)):
        w = O.rfe_weights(t0, tau, a, b)
        assert sum(w.values()) == pytest.approx(b - a, rel=1e-14)
        ts = np.linspace(a, b, 200001)
        ref = np.trapezoid([S(t) for t in ts], ts)
        assert sum(wk * f[k] for k, wk in w.items()) == pytest.approx(ref, rel=1e-8)
    assert O.rfe_weights(t0, math.inf, 2.0, 3.5) == {0: 1.5}


def _rfe_only(lifetime, hours):
    g = O.Grid(65, 128)
    p = O.Params(advection=False, diffusion="off", rfe_method=2, rfe_rate=RATE, rfe_lifetime=lifetime,
                 rfe_seed=3)
    r = O.Realization(g, p, np.zeros((65, 128)))
    r.advance(hours)
    A = g.area * O.R_SUN_CM ** 2
    return float((A * np.abs(r.B)).sum()), float((A * r.B).sum())


def test_rfe_run_realizes_the_rate_with_infinite_lifetime():
    """The paper's RFE check (no flows, no diffusion, from a zero map)."""
    unsigned, net = _rfe_only(math.inf, 10.0)
    assert unsigned == pytest.approx(10.0 * RATE, rel=0.02)
    assert abs(net) <= 1e-12 * unsigned
    short, net_s = _rfe_only(0.3, 10.0)
    assert short < 0.3 * unsigned                              # cancellation between samples
    assert abs(net_s) <= 1e-12 * short


def test_splitmix64_reproduces_the_published_sequence():
    """The output function on the states k * gamma (k = 1, 2, 3) is the
    generator of Steele, Lea & Flood (2014) seeded with 0, whose first three
    outputs are published with its reference implementation."""
    gam = np.uint64(O.SPLITMIX_GAMMA)
    with np.errstate(over="ignore"):
        got = [int(O.splitmix64_output(np.uint64(k) * gam)) for k in (1, 2, 3)]
    assert got == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
