"""The debug build and host fault injection on the GPU.

Debug build: libsft_debug.so (kernels compiled with -DSFT_DEBUG check every
index they derive from their tiles and descriptors, record a failure on the
device and keep the access in bounds).  A child process runs a case per
kernel family on grids with ragged phi tails -- FP64 single-stage RKL2,
FP32 fused RKL2 on float4 and scalar rows, Strang splitting with flow
attenuation and random flux emergence, grid-based nu with upwind
advection, assimilation, diagnostics -- against the FP64 oracle: the
results meet the parity bar and no check fails.  The record path is tested
with probes that make no memory access.

Fault injection: allocation failures injected on the host, one allocation
at a time, through every allocation that creating a grid, setting its
flows (with a grid-based-nu geometry block), random flux emergence,
assimilation and the first steps make.  Each failing call returns
SFT_ERR_OOM; repeating it completes the run with the same bits as a run
without failures, and no device memory stays allocated.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import sft_inputs as I
from paper_2501_06377_gb300 import build as B
from paper_2501_06377_gb300.sft import AssimParams, Grid, RfeParams, SFTError, SFT_ERR_OOM, load
from tests.sft_testlib import params_from_draw

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TOL = {"fp64": 1e-12, "fp32": 1e-5}


@pytest.fixture(scope="module", autouse=True)
def _built():
    B.build()
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def test_debug_build_runs_every_kernel_family_without_a_failed_check():
    B.build(debug=True)
    p = subprocess.run([sys.executable, "-m", "tests.sft_debug_child"], cwd=ROOT, capture_output=True,
                       text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-3000:]
    out = json.loads(p.stdout.strip().splitlines()[-1])
    assert out["fusion"] > 1                       # the FP32 cases ran the fused kernel
    for name, err in out["errors"].items():
        assert err <= TOL[name[:4]], (name, err)
    assert out["checks_status"] == 0
    assert out["count"] == 0 and out["first"] == 0, hex(out["first"])
    mask = (1 << 48) - 1
    first = (9 << 48) | (-3 & mask)
    assert out["probes"] == [[0, 0], [first, 1], [first, 2], [0, 0]]


# big enough that a leaked state or work array shows in the device's free memory
SHAPES = [(513, 1024), (129, 520), (513, 1024)]
T_END = 2.0


def _run(fail_at=0):
    """The whole sequence; with fail_at = n the n-th allocation fails once and
    the failing call is repeated.  Returns (states, failed call or None)."""
    lib = load()
    draws = I.draw_realization_params(len(SHAPES), seed=23)
    params = [params_from_draw(d) for d in draws]
    params[1].nu_grid_alpha = 0.5                  # a geometry block of its own
    rfe = [RfeParams(method=2, rate_mx_per_hour=1e23, lifetime_hours=0.5, seed=4, origin_hours=0.0),
           None, None]
    streams = [I.ObservationStream(*s, seed=3) for s in (SHAPES[0], SHAPES[1])]   # one map per shape
    obs = np.concatenate([s.truth(10.0).astype(np.float32).ravel() for s in streams])
    mu = np.concatenate([s.mu(10.0).astype(np.float32).ravel() for s in streams])
    ap = AssimParams(alpha_mu=2.0, mu_lim=0.1, lat_lim_deg=60.0, flux_balance=True)
    state = {}

    def create():
        state["g"] = Grid(SHAPES, "fp32")
        for r, s in enumerate(SHAPES):
            state["g"].set_state(r, I.initial_map(*s, seed=60 + r))

    calls = [("create", create),
             ("set_flows", lambda: state["g"].set_flows(params)),
             ("set_rfe", lambda: state["g"].set_rfe(rfe)),
             ("step1", lambda: state["g"].step(1.0)),
             ("assimilate", lambda: state["g"].assimilate(obs, mu, 2, ap)),
             ("step2", lambda: state["g"].step(T_END)),
             ("diagnostics", lambda: state["g"].diagnostics())]
    failed = None
    lib.sft_debug_fail_alloc(fail_at)
    try:
        for name, fn in calls:
            try:
                fn()
            except SFTError as e:
                assert failed is None, (failed, name, str(e))   # the injector fires once
                assert e.status == SFT_ERR_OOM, str(e)
                failed = name
                if name == "create":
                    return None, failed
                fn()                                          # the same call again succeeds
        g = state["g"]
        return [g.get_state(r) for r in range(len(SHAPES))], failed
    finally:
        lib.sft_debug_fail_alloc(0)
        if "g" in state:
            state["g"].close()


def test_injected_allocation_failures_are_reported_and_recovered():
    import torch
    ref, failed = _run(0)
    assert failed is None
    assert np.array_equal(_run(0)[0][1], ref[1])   # repeatable; modules loaded before the baseline
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    seen = set()
    n = 1
    while True:
        got, failed = _run(n)
        if failed is None:
            break
        seen.add(failed)
        if got is not None:
            for a, b in zip(got, ref):
                assert np.array_equal(a, b), (n, failed)
        n += 1
        assert n < 400
    # every call that allocates was hit at least once
    assert {"create", "set_flows", "set_rfe", "step1", "assimilate"} <= seen, seen
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert free0 - free1 <= 3 << 20, (free0 - free1) / 2 ** 20   # no state or work array left behind
