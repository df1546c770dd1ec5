"""The ensemble configurations end to end on the GPU against the FP64 oracle.

* 512x1024 FP32, the model started from the dipole only, hourly weighted
  and flux-balanced assimilation of a synthetic hidden truth (first hours).
* An uneven batch of three grid shapes with per-shape observation streams
  (reduced sizes so the oracle can follow every realization), and the
  full-size 256-realization uneven batch (199.8 M cells) checked on a
  sampled realization against the oracle and on invariants, also under an
  HBM budget that forces several waves.
* One full-size step of the 64 x 1024x2048 ensemble, sampled.
FP32 bar: relative L-inf <= 1e-5 of max|Br|.
"""
import math

import numpy as np
import pytest

import oracle as O
import sft_inputs as I
from paper_2501_06377_gb300 import build as B
from paper_2501_06377_gb300.sft import AssimParams, FlowParams, Grid
from tests.sft_testlib import oracle_params, params_from_draw, rel_linf

pytestmark = pytest.mark.gpu

AP = AssimParams(alpha_mu=4.0, mu_lim=0.1, lat_lim_deg=90.0, flux_balance=True)


@pytest.fixture(scope="module", autouse=True)
def _built():
    B.build()
    import torch
    assert torch.cuda.is_available()


def _c2_flow():
    d = I.omega_to_dr_coeffs(*I.DEFAULT_OMEGA)
    return FlowParams(d0=d[0], d2=d[1], d4=d[2], m1=30.0, m3=0.0, m5=0.0, nu=500.0)


def _oracle_assim(g, B, obs, mu):
    F = O.assimilation_weight(mu, g.lat[:, None], AP.alpha_mu, AP.mu_lim, math.radians(AP.lat_lim_deg))
    return O.assimilate(g, B, obs, F, AP.flux_balance)


def test_c2_hourly_assimilation_512x1024(record_precision):
    shape = (512, 1024)
    fp = _c2_flow()
    st = I.ObservationStream(*shape, seed=2)
    B0 = I.dipole(*shape).astype(np.float32)
    g = Grid([shape], "fp32")
    g.set_state(0, B0)
    g.set_flows([fp])
    ref = O.Realization(O.Grid(*shape), oracle_params(fp), B0.astype(np.float64))
    for hour in (1, 2, 3):
        g.step(float(hour))
        ref.advance(float(hour))
        obs = st.truth(float(hour)).astype(np.float32)
        mu = st.mu(float(hour)).astype(np.float32)
        g.assimilate(obs, mu, False, AP)
        ref.B = _oracle_assim(ref.g, ref.B, obs.astype(np.float64), mu.astype(np.float64))
    got = g.get_state(0)
    record_precision("C2 512x1024 FP32, 3 h with hourly assimilation", rel_linf(got, ref.B), 1e-5)
    assert rel_linf(got, ref.B) <= 1e-5, rel_linf(got, ref.B)
    assert np.abs(got - B0).max() > 1.0   # the observations did enter


def _uneven(shapes_counts, seed=3):
    shapes = [s for s, n in shapes_counts for _ in range(n)]
    draws = I.draw_realization_params(len(shapes), seed=seed)
    return shapes, [params_from_draw(d) for d in draws]


def test_c4_uneven_batch_per_shape_observations(record_precision):
    shapes, params = _uneven([((64, 128), 4), ((128, 256), 3), ((90, 180), 2)])
    distinct = [(64, 128), (128, 256), (90, 180)]
    streams = {s: I.ObservationStream(*s, seed=2) for s in distinct}
    g = Grid(shapes, "fp32")
    refs = []
    for r, s in enumerate(shapes):
        B0 = I.dipole(*s).astype(np.float32)
        g.set_state(r, B0)
        refs.append(O.Realization(O.Grid(*s), oracle_params(params[r]), B0.astype(np.float64)))
    g.set_flows(params)
    for hour in (1, 2, 3):
        g.step(float(hour))
        obs = {s: streams[s].truth(float(hour)).astype(np.float32) for s in distinct}
        mu = {s: streams[s].mu(float(hour)).astype(np.float32) for s in distinct}
        g.assimilate(np.concatenate([obs[s].ravel() for s in distinct]),
                     np.concatenate([mu[s].ravel() for s in distinct]), 2, AP)
        for r, s in enumerate(shapes):
            refs[r].advance(float(hour))
            refs[r].B = _oracle_assim(refs[r].g, refs[r].B, obs[s].astype(np.float64), mu[s].astype(np.float64))
    errs = [rel_linf(g.get_state(r), refs[r].B) for r in range(len(shapes))]
    record_precision("C4 reduced: 9 realizations, 3 shapes, FP32, 3 h with per-shape assimilation", max(errs), 1e-5)
    for r in range(len(shapes)):
        assert errs[r] <= 1e-5, (r, errs[r])


FULL_C4 = [((256, 512), 128), ((512, 1024), 96), ((1440, 2880), 32)]


def _run_full_c4(budget=0):
    shapes, params = _uneven(FULL_C4, seed=3)
    distinct = [s for s, _ in FULL_C4]
    dip = {s: I.dipole(*s).astype(np.float32) for s in distinct}
    g = Grid(shapes, "fp32", hbm_budget=budget)
    for r, s in enumerate(shapes):
        g.set_state(r, dip[s])
    g.set_flows(params)
    d0 = g.diagnostics()
    n = g.step(1.0)
    d1 = g.diagnostics()
    return g, shapes, params, d0, d1, n


def test_c4_full_size_uneven_batch(record_precision):
    """256 realizations, 199.8 M cells, one hour: each realization takes
    ceil(1 h / its CFL step) steps; total flux is conserved; a sampled 256x512 realization
    matches the oracle; an HBM budget for about a third of the work arrays
    (several waves) gives the same bits."""
    g, shapes, params, d0, d1, n = _run_full_c4()
    # Sec. 3.4 controller: ceil(1 h / dt_CFL) steps per realization
    want = [math.ceil(1.0 / min(1.0, g.step_plan(r, 1.0)[0]) - 1e-12) for r in range(len(shapes))]
    assert [d["steps"] for d in d1] == want
    assert n == max(want) and max(want) >= 2
    for a, b in zip(d0, d1):
        assert b["nonfinite"] == 0
        assert abs(b["flux_signed"] - a["flux_signed"]) <= 1e-5 * a["flux_pos"]
    ref = O.Realization(O.Grid(256, 512), oracle_params(params[0]), I.dipole(256, 512).astype(np.float32).astype(np.float64))
    ref.advance(1.0)
    drift = max(abs(b["flux_signed"] - a["flux_signed"]) / a["flux_pos"] for a, b in zip(d0, d1))
    record_precision("C4 full size: 256 realizations, 199.8 M cells, FP32, 1 h (256x512 sampled)",
                     rel_linf(g.get_state(0), ref.B), 1e-5, drift)
    assert rel_linf(g.get_state(0), ref.B) <= 1e-5
    sample = [0, 127, 128, 223, 224, 255]
    full = {r: g.get_state(r) for r in sample}
    g.close()
    cells = sum(a * ((b + 31) // 32 * 32) for (a, b), k in FULL_C4 for _ in range(k))
    budget = cells * 4 + (64 << 20) + 5 * 4 * cells // 3
    gw, *_ = _run_full_c4(budget)
    assert gw.wave_size() < len(shapes)
    for r in sample:
        np.testing.assert_array_equal(gw.get_state(r), full[r])


def test_c3_full_size_step_sampled(record_precision):
    """One step of 64 x 1024x2048 (the benchmarked ensemble); realization 0
    against the oracle (one CFL step, ~580 RKL2 stages at 2 M cells)."""
    nt, np_ = 1024, 2048
    draws = I.draw_realization_params(64, seed=3)
    params = [params_from_draw(d) for d in draws]
    maps = [I.initial_map(nt, np_, seed=1 + i).astype(np.float32) for i in range(2)]
    g = Grid([(nt, np_)] * 64, "fp32")
    for r in range(64):
        g.set_state(r, maps[r % 2])
    g.set_flows(params)
    d0 = g.diagnostics()
    assert g.step(27 * 24.0, max_steps=1) == 1
    d1 = g.diagnostics()
    for a, b in zip(d0, d1):
        assert b["nonfinite"] == 0
        assert abs(b["flux_signed"] - a["flux_signed"]) <= 1e-5 * a["flux_pos"]
    ref = O.Realization(O.Grid(nt, np_), oracle_params(params[0]), maps[0].astype(np.float64))
    ref.advance(27 * 24.0, max_steps=1)
    drift = max(abs(b["flux_signed"] - a["flux_signed"]) / a["flux_pos"] for a, b in zip(d0, d1))
    record_precision("C3 64x1024x2048 FP32, one CFL step (realization 0 sampled)",
                     rel_linf(g.get_state(0), ref.B), 1e-5, drift)
    assert rel_linf(g.get_state(0), ref.B) <= 1e-5, rel_linf(g.get_state(0), ref.B)
