"""Surrogate-plus-fallback ensemble on 256 x 512 maps (host orchestration).

Every arithmetic step runs in libsft's kernels; this module only decides
which member takes which path:

* ``make_pairs``: one-day (map_t, map_t+1d) training pairs from the batched
  plain solver (sft_step) started from given maps with drawn parameters.
* ``train``: AdamW on the pairs (sfs_train_step), cosine learning rate.
* ``rollout``: members advance one day at a time; the surrogate proposes all
  of them (sfs_forward); a proposal is rejected when its FP64 total-flux
  drift |sum A (B_new - B_old)| / sum A |B_old| exceeds ``drift_tol``
  (sfs_flux), and for a seeded spot-check subset the plain
  solver's own day is computed (queued on the grid's stream before the
  proposals, so the two run at once) and the proposal rejected when their
  relative L2 difference exceeds ``l2_tol`` (sfs_rel_l2).  Rejected members
  advance with the plain solver (the spot-checked ones take the solver's
  result they already have).
* ``plain``: the same members advanced by the plain batched solver only.

Parameters per member: p = (o0, o2, o4) rotation coefficients in deg/day
(relative rate Omega(lat) - 360/27.2753), U meridional amplitude (m/s,
poleward U sin 2 lat), eta (km^2/s).
"""
from __future__ import annotations

import math
import time

import numpy as np

from .sft import FlowParams, Grid
from .surrogate import Surrogate

H, W = 256, 512
DAY = 24.0
FRAME = 360.0 / 27.2753
R_SUN_M = 6.96e8


def flow_params(p):
    """sft_flow_params of one member from (o0, o2, o4, U, eta): Eq. (dr) with
    d_i = (o_i - frame [i=0]) pi/180/86400 R_sun, Eq. (mf) with m1 = 2U."""
    k = math.radians(1.0) / 86400.0 * R_SUN_M
    o0, o2, o4, u, eta = (float(v) for v in p)
    return FlowParams(d0=(o0 - FRAME) * k, d2=o2 * k, d4=o4 * k, m1=2.0 * u, m3=0.0, m5=0.0, nu=eta)


def draw_params(n, seed):
    """Member parameters: rotation coefficients x U[0.9, 1.1], U in [10, 20]
    m/s, eta in [250, 750] km^2/s."""
    rng = np.random.default_rng(seed)
    base = np.array([13.38, -2.30, -1.62])
    p = np.empty((n, 5))
    p[:, :3] = base * rng.uniform(0.9, 1.1, (n, 3))
    p[:, 3] = rng.uniform(10.0, 20.0, n)
    p[:, 4] = rng.uniform(250.0, 750.0, n)
    return p


def _grid(n, params, stream=None):
    g = Grid([(H, W)] * n, "fp32", stream=stream)
    g.set_flows([flow_params(p) for p in params])
    return g


def make_pairs(base_maps, n_pairs, seed=5, chunk=512, max_start_day=9):
    """(X, Y, P): X, Y [n, H, W] float32 CUDA tensors one day apart, P [n, 5]."""
    import torch
    rng = np.random.default_rng(seed)
    X = torch.empty((n_pairs, H, W), device="cuda")
    Y = torch.empty((n_pairs, H, W), device="cuda")
    P = draw_params(n_pairs, seed + 1)
    nb = base_maps.shape[0]
    for c0 in range(0, n_pairs, chunk):
        n = min(chunk, n_pairs - c0)
        g = _grid(n, P[c0:c0 + n])
        for i in range(n):
            m = base_maps[int(rng.integers(nb))]
            g.set_state(i, torch.roll(m, int(rng.integers(W)), dims=1).contiguous())
        d0 = int(rng.integers(0, max_start_day + 1))
        if d0:
            g.step(d0 * DAY)
        for i in range(n):
            g.get_state(i, X[c0 + i])
        g.step((d0 + 1) * DAY)
        for i in range(n):
            g.get_state(i, Y[c0 + i])
        torch.cuda.synchronize()
        g.close()
    return X, Y, torch.from_numpy(P.astype(np.float32)).cuda()


def train(net: Surrogate, X, Y, P, epochs=10, batch=32, lr=2e-3, wd=1e-4, seed=0, log_every=100):
    """Cosine-decayed AdamW; returns the loss history (every log_every steps)."""
    import torch
    n = X.shape[0]
    steps = epochs * (n // batch)
    rng = np.random.default_rng(seed)
    hist = []
    k = 0
    for _ in range(epochs):
        perm = torch.from_numpy(rng.permutation(n)).cuda()
        for b0 in range(0, n - batch + 1, batch):
            idx = perm[b0:b0 + batch]
            xb, yb, pb = X[idx].contiguous(), Y[idx].contiguous(), P[idx].contiguous()
            lr_k = 0.5 * lr * (1.0 + math.cos(math.pi * k / max(steps, 1)))
            want = (k % log_every) == 0
            loss = net.train_step(xb, pb, yb, lr_k, wd, want_loss=want)
            if want:
                hist.append((k, loss))
            k += 1
    return hist


def propose(net: Surrogate, S, P, out):
    for c0 in range(0, S.shape[0], net.max_batch):
        c1 = min(S.shape[0], c0 + net.max_batch)
        net.forward(S[c0:c1], P[c0:c1], out[c0:c1])
    return out


def _fluxes(net: Surrogate, maps):
    return net.flux(maps)


def rollout(net: Surrogate, S0, P, days, drift_tol=1e-4, l2_tol=0.02, spot=32, seed=7, max_fail=0.25):
    """Surrogate + judge + plain-solver fallback.  Returns (final maps, stats).

    A day on which more than ``max_fail`` of the spot checks fail rejects
    every proposal of that day (the unchecked members cannot be trusted
    either); otherwise only the failing members fall back."""
    import torch
    n = S0.shape[0]
    params = P.cpu().numpy().astype(np.float64)
    g = _grid(n, params)
    S = S0.clone()
    prop = torch.empty_like(S)
    rng = np.random.default_rng(seed)
    stats = {"member_days": 0, "accepted": 0, "rejected_drift": 0, "rejected_spot": 0, "spot_checked": 0}
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    phi_old, abs_old = _fluxes(net, S)
    for day in range(days):
        t_day0, t_day1 = day * DAY, (day + 1) * DAY
        chk = rng.choice(n, size=min(spot, n), replace=False)
        run = np.zeros(n, dtype=bool)
        run[chk] = True
        # the plain solver's day for the spot-checked members is queued first
        # (sft_step returns without waiting) so that it runs on the grid's
        # stream while the surrogate proposes on its own
        for i in range(n):
            if run[i]:
                g.set_state(i, S[i])
            g.set_time(t_day0 if run[i] else t_day1, i)
        g.step(t_day1)
        propose(net, S, P, prop)
        phi_new, abs_new = _fluxes(net, prop)
        drift = np.abs(phi_new - phi_old) / np.maximum(abs_old, 1e-300)
        bad = drift > drift_tol
        extra = bad & ~run
        if extra.any():  # drift-rejected members outside the spot check: their own plain day
            for i in range(n):
                if extra[i]:
                    g.set_state(i, S[i])
                g.set_time(t_day0 if extra[i] else t_day1, i)
            g.step(t_day1)
            run |= extra
        plain = torch.empty((int(run.sum()), H, W), device="cuda")
        idx = np.flatnonzero(run)
        for q, i in enumerate(idx):
            g.get_state(int(i), plain[q])
        # spot check: relative L2 of the proposal against the solver's day
        pos = {int(i): q for q, i in enumerate(idx)}
        chk_plain = plain[[pos[int(i)] for i in chk]].contiguous()
        chk_prop = prop[torch.from_numpy(chk).cuda()].contiguous()
        err = net.rel_l2(chk_prop, chk_plain)
        spot_bad = np.zeros(n, dtype=bool)
        spot_bad[chk[err > l2_tol]] = True
        if np.mean(err > l2_tol) > max_fail:
            # untrustworthy day: every member advances with the plain solver
            rest = ~run
            for i in np.flatnonzero(rest):
                g.set_state(int(i), S[int(i)])
                g.set_time(t_day0, int(i))
            for i in np.flatnonzero(run):
                g.set_time(t_day1, int(i))
            g.step(t_day1)
            for i in np.flatnonzero(rest):
                g.get_state(int(i), S[int(i)])
            spot_bad[:] = True
            stats["days_rejected"] = stats.get("days_rejected", 0) + 1
        use_plain = bad | spot_bad | run  # solver result available for every member it ran on
        for q, i in enumerate(idx):
            S[int(i)] = plain[q]
        keep = torch.from_numpy(~use_plain).cuda()
        S[keep] = prop[keep]
        stats["member_days"] += n
        stats["accepted"] += int((~use_plain).sum())
        stats["rejected_drift"] += int(bad.sum())
        stats["rejected_spot"] += int((spot_bad & ~bad).sum())
        stats["spot_checked"] += len(chk)
        stats.setdefault("spot_l2_median", []).append(float(np.median(err)))
        phi_old, abs_old = _fluxes(net, S)
    torch.cuda.synchronize()
    stats["seconds"] = time.perf_counter() - t0
    stats["member_days_per_s"] = stats["member_days"] / stats["seconds"]
    stats["tile_rows"] = g.get_tile_rows(0)  # the autotuner's choice for this grid shape
    g.close()
    return S, stats


def plain(S0, P, days):
    """The plain batched solver over the same members and days."""
    import torch
    n = S0.shape[0]
    g = _grid(n, P.cpu().numpy().astype(np.float64))
    for i in range(n):
        g.set_state(i, S0[i])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for day in range(days):
        g.step((day + 1) * DAY)
        g.diagnostics()  # the same per-day history as the rollout keeps
    torch.cuda.synchronize()
    sec = time.perf_counter() - t0
    out = torch.empty_like(S0)
    for i in range(n):
        g.get_state(i, out[i])
    torch.cuda.synchronize()
    tr = g.get_tile_rows(0)
    g.close()
    return out, {"seconds": sec, "member_days_per_s": n * days / sec, "tile_rows": tr}
