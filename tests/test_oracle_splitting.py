"""Pins for the operator splitting of Sec. 3.5 (oracle): Lie (Eq.
num_opsplit_nostrang) and Strang (Eq. num_opsplit_strang).

The splitting errors are measured against the combined semi-discrete
system dB/dt = -F_A(B) + L(B) integrated by classical RK4 with a step far
below every limit (a reference that shares no splitting with the schemes):
Lie converges at first order, Strang at second (differential rotation and
meridional flow do not commute with diffusion).  Upwind advection keeps
the operators linear.
"""
import math

import numpy as np
import pytest

import oracle as O
import sft_inputs as I

T = 48.0


@pytest.fixture(scope="module")
def case():
    g = O.Grid(17, 32)
    B0 = I.initial_map(17, 32, seed=4)
    r = O.Realization(g, O.Params(adv_space="upwind", nu=500.0), B0)
    f = lambda B: -r.FA(B) + r.L(B)
    n = 4000
    h = T / n
    B = B0.copy()
    for _ in range(n):
        k1 = f(B)
        k2 = f(B + 0.5 * h * k1)
        k3 = f(B + 0.5 * h * k2)
        k4 = f(B + h * k3)
        B = B + h / 6.0 * (k1 + 2.0 * k2 + 2.0 * k3 + k4)
    return g, B0, B


def _split(g, B0, split, n, **kw):
    r = O.Realization(g, O.Params(adv_space="upwind", splitting=split, nu=500.0, **kw), B0)
    for _ in range(n):
        r.lie_step(T / n)
    return r.B


@pytest.mark.parametrize("split,lo,hi", [("lie", 0.9, 1.1), ("strang", 1.85, 2.1)])
def test_splitting_order(case, split, lo, hi):
    g, B0, ref = case
    errs = [np.abs(_split(g, B0, split, n) - ref).max() for n in (4, 8, 16)]
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(lo <= o <= hi for o in orders), orders


def test_strang_without_advection_is_lie():
    g = O.Grid(17, 32)
    B0 = I.initial_map(17, 32, seed=6)
    a = _split(g, B0, "lie", 3, advection=False)
    b = _split(g, B0, "strang", 3, advection=False)
    assert np.array_equal(a, b)


def test_strang_without_diffusion_is_two_half_advection_steps():
    g = O.Grid(17, 32)
    B0 = I.initial_map(17, 32, seed=8)
    a = _split(g, B0, "strang", 2, diffusion="off")
    r = O.Realization(g, O.Params(adv_space="upwind", diffusion="off"), B0)
    for _ in range(4):
        r.lie_step(T / 4)
    assert np.array_equal(a, r.B)


def test_strang_doubles_the_flow_step():
    g = O.Grid(33, 64)
    B0 = I.initial_map(33, 64, seed=2)
    lie = O.Realization(g, O.Params(), B0)
    strang = O.Realization(g, O.Params(splitting="strang"), B0)
    assert strang.next_dt(1e9) == 2.0 * lie.next_dt(1e9) == 2.0 * lie.dt_adv
