"""Child process of the debug-build GPU test: loads libsft_debug.so (the
kernels check every index they derive from their tiles and descriptors),
runs a case per kernel family against the FP64 oracle and prints one JSON
line with the errors and the device record of failed checks.

Run as `python -m tests.sft_debug_child` from the repository root.  A child
process because the binding loads one library per process.
"""
import json
import math
import sys

import numpy as np

import oracle as O
import sft_inputs as I
from paper_2501_06377_gb300 import build as B
from paper_2501_06377_gb300 import sft
from paper_2501_06377_gb300.sft import AssimParams, Grid, RfeParams
from tests.sft_testlib import oracle_params, params_from_draw, rel_linf


def _grid(shapes, prec, seed, **kw):
    draws = I.draw_realization_params(len(shapes), seed=seed)
    params = [params_from_draw(d, **kw) for d in draws]
    g = Grid(shapes, prec)
    maps = [I.initial_map(*s, seed=40 + r) for r, s in enumerate(shapes)]
    for r, m in enumerate(maps):
        g.set_state(r, m)
    return g, params, maps


def _oracle(shape, fp, B0, t_end, rp=None):
    p = oracle_params(fp)
    if rp is not None:
        p.rfe_method, p.rfe_rate, p.rfe_seed = rp.method, rp.rate_mx_per_hour, rp.seed
        p.rfe_lifetime = rp.lifetime_hours
    r = O.Realization(O.Grid(*shape), p, np.asarray(B0, dtype=np.float64))
    r.advance(t_end)
    return r.B


def case_steps(prec, shapes, seed, t_end, rfe=False, **kw):
    """Advection + RKL2 (fused in FP32 where the shape allows), poles,
    optionally random flux emergence; worst relative L-inf over realizations."""
    g, params, maps = _grid(shapes, prec, seed, **kw)
    g.set_flows(params)
    rps = None
    if rfe:
        rps = [RfeParams(method=1 + r % 2, rate_mx_per_hour=1e23, lifetime_hours=0.3, seed=3 + r)
               for r in range(len(shapes))]
        g.set_rfe(rps)
    g.step(t_end)
    g.diagnostics()
    err = 0.0
    for r, s in enumerate(shapes):
        ref = _oracle(s, params[r], maps[r], t_end, rps[r] if rps else None)
        err = max(err, rel_linf(g.get_state(r), ref))
    return err, g.get_fusion()


def case_assim(prec):
    shapes = [(40, 96), (33, 70)]
    g, params, maps = _grid(shapes, prec, 6)
    obs, mus = [], []
    for s in shapes:
        st = I.ObservationStream(*s, seed=2)
        obs.append(st.truth(30.0).astype(g.dtype))
        mus.append(st.mu(30.0).astype(g.dtype))
    ap = AssimParams(alpha_mu=2.0, mu_lim=0.1, lat_lim_deg=60.0, flux_balance=True)
    g.assimilate(np.concatenate([o.ravel() for o in obs]), np.concatenate([m.ravel() for m in mus]), True, ap)
    err = 0.0
    for r, s in enumerate(shapes):
        gr = O.Grid(*s)
        F = O.assimilation_weight(mus[r].astype(np.float64), gr.lat[:, None], 2.0, 0.1, math.radians(60.0))
        ref = O.assimilate(gr, maps[r].astype(g.dtype).astype(np.float64), obs[r].astype(np.float64), F, True)
        err = max(err, rel_linf(g.get_state(r), ref))
    return err


def main():
    sft.load(B.build(debug=True))
    lib = sft.load()
    out = {"errors": {}}
    ragged = [(33, 64), (20, 100), (41, 70)]        # phi tails off the vector width
    fused = [(36, 100), (57, 520), (41, 70)]        # the fused path, float4 and scalar rows
    out["errors"]["fp64_lie"], _ = case_steps("fp64", ragged, 3, 6.0)
    out["errors"]["fp32_fused"], out["fusion"] = case_steps("fp32", fused, 4, 6.0)
    out["errors"]["fp32_strang_atten_rfe"], _ = case_steps("fp32", fused, 5, 1.0, rfe=True,
                                                           splitting="strang", atten_b0=50.0)
    out["errors"]["fp64_grid_nu_upwind"], _ = case_steps("fp64", ragged, 7, 6.0, nu_grid_alpha=0.5,
                                                         adv_space="upwind")
    out["errors"]["fp32_assim"] = case_assim("fp32")
    first, count = sft.C.c_uint64(), sft.C.c_uint32()
    st = lib.sft_debug_checks(sft.C.byref(first), sft.C.byref(count), 1)
    out["checks_status"], out["first"], out["count"] = st, first.value, count.value
    # the record path: an in-range probe records nothing, out-of-range ones
    # record the first (site, value) and count all
    probes = []
    for site, v in ((5, 7), (9, -3), (4, 20)):
        lib.sft_debug_probe(site, v, 0, 10)
        lib.sft_debug_checks(sft.C.byref(first), sft.C.byref(count), 0)
        probes.append([first.value, count.value])
    lib.sft_debug_checks(sft.C.byref(first), sft.C.byref(count), 1)
    lib.sft_debug_checks(sft.C.byref(first), sft.C.byref(count), 0)
    probes.append([first.value, count.value])
    out["probes"] = probes
    print(json.dumps(out))
    return 0


if __name__ == "__main__":
    sys.exit(main())
