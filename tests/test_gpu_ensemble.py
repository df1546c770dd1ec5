"""The surrogate ensemble's judge and fallback (ensemble.rollout) on the GPU.

Two limits with exact answers: when every proposal is rejected, each
member advances with the plain solver, so the rollout equals the plain
batched solver bit for bit; when every proposal is accepted, the rollout
equals repeated surrogate forward passes bit for bit.
"""
import numpy as np
import pytest

import sft_inputs as I
from paper_2501_06377_gb300 import build as B

pytestmark = pytest.mark.gpu

N, DAYS = 8, 2


@pytest.fixture(scope="module")
def setup():
    B.build()
    import torch
    assert torch.cuda.is_available()
    from paper_2501_06377_gb300 import ensemble as E
    P = E.draw_params(N, 21)
    Pt = torch.from_numpy(P.astype(np.float32)).cuda()
    S0 = torch.stack([torch.from_numpy(I.initial_map(256, 512, seed=30 + i).astype(np.float32))
                      for i in range(N)]).cuda().contiguous()
    return torch, E, Pt, S0


def _net(E, seed):
    from paper_2501_06377_gb300.surrogate import Surrogate
    return Surrogate(channels=64, modes=48, blocks=4, max_batch=4, seed=seed)


def test_all_rejected_equals_plain_solver(setup):
    torch, E, Pt, S0 = setup
    net = _net(E, 1)
    # an untrained network misses the day by far more than a 1e-9 L2 bar:
    # every spot check fails, every day is rejected
    out, st = E.rollout(net, S0, Pt, DAYS, l2_tol=1e-9, spot=N)
    ref, _ = E.plain(S0, Pt, DAYS)
    assert st["accepted"] == 0 and st["member_days"] == N * DAYS
    assert torch.equal(out, ref)


def test_all_accepted_equals_repeated_forward(setup):
    torch, E, Pt, S0 = setup
    net = _net(E, 2)
    out, st = E.rollout(net, S0, Pt, DAYS, drift_tol=1e30, l2_tol=1e30, spot=2)
    assert st["accepted"] == N * DAYS - 2 * DAYS  # spot-checked members take the solver's day
    x = S0.clone()
    y = torch.empty_like(x)
    for _ in range(DAYS):
        E.propose(net, x, Pt, y)
        x, y = y, x
    # members never spot-checked carry the pure surrogate trajectory
    seen = np.zeros(N, dtype=bool)
    rng = np.random.default_rng(7)  # rollout's default seed: the same spot draws
    for _ in range(DAYS):
        seen[rng.choice(N, size=2, replace=False)] = True
    for i in np.flatnonzero(~seen):
        assert torch.equal(out[i], x[i]), i
