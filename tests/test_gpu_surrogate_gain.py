"""What the trained surrogate gains over the method without it, on the GPU.

A network trained briefly (reduced size) on one-day pairs that the batched
solver generates, against the rotation-only control (the same network with
its learned correction switched off: each proposal is the map rotated by the
day's differential rotation), on the same unseen members and days, judged
by the plain solver: the trained network's proposals are closer to the
solver's days (spot-check L2) and more of them are accepted (each accepted
proposal is a member-day the solver does not run), while the ensemble stays
close to the plain solver.  (The control's proposals all fail the judge, so
its ensemble is the plain solver's.)
"""
import numpy as np
import pytest

import sft_inputs as I
from paper_2501_06377_gb300 import build as B

pytestmark = pytest.mark.gpu


def test_trained_network_beats_the_rotation_only_control():
    B.build()
    import torch
    assert torch.cuda.is_available()
    from paper_2501_06377_gb300 import ensemble as E
    from paper_2501_06377_gb300.sft import Grid
    from paper_2501_06377_gb300.surrogate import Surrogate
    nb = 16
    g = Grid([(E.H, E.W)] * nb, "fp32")
    for i in range(nb):
        g.set_state(i, I.initial_map(E.H, E.W, seed=2000 + i).astype(np.float32))
    g.balance_flux()
    base = torch.empty((nb, E.H, E.W), device="cuda")
    g.get_states(np.arange(nb), base)
    torch.cuda.synchronize()
    g.close()
    X, Y, P = E.make_pairs(base, 3072, seed=41)
    net = Surrogate(channels=64, modes=48, blocks=4, max_batch=32, seed=3)
    E.train(net, X, Y, P, epochs=6, batch=32, lr=2e-3)
    del X, Y
    members, days = 64, 6
    rng = np.random.default_rng(43)
    Pm = torch.from_numpy(E.draw_params(members, 44).astype(np.float32)).cuda()
    S0 = E.rolled(base, rng.integers(nb, size=members), rng.integers(E.W, size=members))
    ref, _ = E.plain(S0, Pm, days)
    out, st = E.rollout(net, S0, Pm, days, spot=16)
    ctrl = E.rotation_only(net)
    out_c, st_c = E.rollout(ctrl, S0, Pm, days, spot=16)
    spot_t, spot_c = np.median(st["spot_l2_median"]), np.median(st_c["spot_l2_median"])
    acc_t = st["accepted"] / st["member_days"]
    acc_c = st_c["accepted"] / st_c["member_days"]
    end_t = np.median(net.rel_l2(out, ref))
    end_c = np.median(net.rel_l2(out_c, ref))
    print("spot-check L2 median: trained %.4f, rotation only %.4f; accepted: %.3f vs %.3f; "
          "day-%d L2 vs plain: %.4f vs %.4f" % (spot_t, spot_c, acc_t, acc_c, days, end_t, end_c))
    assert spot_t < 0.5 * spot_c
    assert acc_t > acc_c + 0.25
    assert end_t < 0.05
