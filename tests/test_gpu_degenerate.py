"""Degenerate cases of the step on the GPU.

The smallest grid the library accepts (5 x 8: three interior rows between
the caps, every theta face upwind) against the oracle; a zero-length step; a
realization without flow and with zero diffusivity riding in a batch with
others (bitwise unchanged);
a uniform field under rotation-only flow and diffusion (a steady state of
both operators: WENO of a constant is exact, the Laplacian of a constant is
zero).
"""
import numpy as np
import pytest

import sft_inputs as I
from paper_2501_06377_gb300 import build as B
from paper_2501_06377_gb300.sft import FlowParams, Grid
from tests.sft_testlib import oracle_run, params_from_draw, rel_linf

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5}


@pytest.fixture(scope="module", autouse=True)
def _built():
    B.build()
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_smallest_grid_matches_oracle(prec):
    shape = (5, 8)
    fp = params_from_draw(I.draw_realization_params(1, seed=9)[0])
    B0 = I.initial_map(*shape, seed=3)
    g = Grid([shape], prec)
    g.set_state(0, B0)
    g.set_flows([fp])
    g.step(20.0)
    ref = oracle_run(shape, fp, B0.astype(g.dtype).astype(np.float64), 20.0)
    assert g.diagnostics()[0]["steps"] == ref.steps
    assert rel_linf(g.get_state(0), ref.B) <= TOL[prec]


def test_zero_length_step_leaves_the_state_alone():
    shape = (37, 64)
    g = Grid([shape], "fp32")
    B0 = I.initial_map(*shape, seed=4).astype(np.float32)
    g.set_state(0, B0)
    g.set_flows([FlowParams()])
    g.set_time(5.0)
    before = g.get_state(0)
    assert g.step(5.0) == 0
    assert np.array_equal(g.get_state(0), before)
    assert g.get_time()[0] == 5.0


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_switched_off_member_is_untouched_in_a_batch(prec):
    shapes = [(37, 64), (37, 64), (41, 96)]
    draws = I.draw_realization_params(3, seed=5)
    params = [params_from_draw(d) for d in draws]
    params[1] = FlowParams(advection=False, nu=0.0)   # no flow, zero diffusivity: every increment is 0
    g = Grid(shapes, prec)
    maps = [I.initial_map(*s, seed=20 + r).astype(g.dtype) for r, s in enumerate(shapes)]
    for r, m in enumerate(maps):
        g.set_state(r, m)
    g.set_flows(params)
    g.step(6.0)
    assert np.array_equal(g.get_state(1), maps[1])
    for r in (0, 2):
        ref = oracle_run(shapes[r], params[r], maps[r].astype(np.float64), 6.0)
        assert rel_linf(g.get_state(r), ref.B) <= TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_uniform_field_is_steady_under_rotation_and_diffusion(prec):
    shape = (65, 128)
    fp = FlowParams(m1=0.0, m3=0.0, m5=0.0, nu=600.0)   # differential rotation only, plus diffusion
    g = Grid([shape], prec)
    B0 = np.full(shape, 7.5, dtype=g.dtype)
    g.set_state(0, B0)
    g.set_flows([fp])
    g.step(48.0)
    tol = 1e-13 if prec == "fp64" else 2e-6
    assert np.abs(g.get_state(0) - 7.5).max() <= tol * 7.5
