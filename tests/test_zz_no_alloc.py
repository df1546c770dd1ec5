"""The no-allocation diagnostics entry point (sft_flux_diagnostics_noalloc)
against the handle-based sft_flux_diagnostics, through the C-ABI, and on
the smaller map against the FP64 oracle's Sec. 2.6 quantities directly.

This entry point is for callers that cannot allocate device memory while
they run (a solver inside a model whose memory pool already owns the
device, or a real-time pipeline that forbids cudaMalloc after start-up).
The test makes two calls in a row on different maps and shapes, so stale
scratch contents from the first call would show up in the second, then two
more in the other order, across which the device's free memory must not
change (the library's code and array are loaded by the first call).  It sits
in its own file, collected last, and works alone in a fresh process.
"""
import numpy as np
import pytest

import oracle.sft_oracle as O
import sft_inputs as I
from paper_2501_06377_gb300 import build as B
from paper_2501_06377_gb300.sft import Grid, flux_diagnostics_noalloc

pytestmark = pytest.mark.gpu

SUM_FIELDS = ("flux_signed", "flux_pos", "flux_neg", "flux_pole_n", "flux_pole_s",
              "area_pole_n", "area_pole_s", "dipole_axial", "h1", "h2")


def _compare(got, ref):
    for k in SUM_FIELDS:
        scale = max(abs(ref["flux_pos"]), 1.0) if k.startswith(("flux", "area")) else \
            max(abs(ref["brmax"]), 1.0)
        if k.startswith("area"):
            scale = max(abs(ref[k]), 1.0)
        assert abs(got[k] - ref[k]) <= 1e-12 * scale, (k, got[k], ref[k])
    for k in ("brmin", "brmax", "absmin", "nonfinite"):
        assert got[k] == ref[k], k


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_noalloc_diagnostics_match_handle_twice(prec):
    import torch
    B.build()
    assert torch.cuda.is_available()
    dt = torch.float32 if prec == "fp32" else torch.float64
    refs, maps = [], []
    for shape, seed in (((1024, 2048), 1), ((91, 180), 2)):
        m = I.initial_map(*shape, seed=seed)
        g = Grid([shape], prec)
        g.set_state(0, m.astype(g.dtype))
        refs.append(g.diagnostics(lat_cut_deg=60.0)[0])
        maps.append(torch.from_numpy(np.ascontiguousarray(g.get_state(0))).to("cuda", dt))
        g.close()
    torch.cuda.synchronize()
    # two calls in a row on different shapes: the second must not see the first's scratch
    got = [flux_diagnostics_noalloc(maps[0], lat_cut_deg=60.0),
           flux_diagnostics_noalloc(maps[1], lat_cut_deg=60.0)]
    for a, b in zip(got, refs):
        _compare(a, b)
    # the 91 x 180 map against the oracle's definition (the map as the GPU holds it)
    ref = O.diagnostics(O.Grid(91, 180), maps[1].double().cpu().numpy(), 60.0)
    for k in SUM_FIELDS:
        scale = max(abs(ref.flux_pos), 1.0) if k.startswith("flux") else max(abs(ref.brmax), 1.0)
        if k.startswith("area"):
            scale = max(abs(getattr(ref, k)), 1.0)
        assert abs(got[1][k] - getattr(ref, k)) <= 1e-12 * scale, (k, got[1][k], getattr(ref, k))
    for k in ("brmin", "brmax", "absmin"):
        assert got[1][k] == getattr(ref, k), k
    # once the library's device code is loaded (first call in the context),
    # further calls take no device memory: the free figure does not move
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    again = [flux_diagnostics_noalloc(maps[1], lat_cut_deg=60.0),
             flux_diagnostics_noalloc(maps[0], lat_cut_deg=60.0)]
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert again[0] == got[1] and again[1] == got[0]
