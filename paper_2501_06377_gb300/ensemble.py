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


def rolled(base_maps, which, shifts):
    """base_maps[which[q]] rolled by shifts[q] longitudes (torch.roll along
    phi for every q at once), as one packed [n, H, W] tensor."""
    import torch
    k = torch.arange(W, device=base_maps.device)
    s = torch.as_tensor(np.asarray(shifts), device=base_maps.device)
    cols = (k[None, :] - s[:, None]) % W
    sel = base_maps[torch.as_tensor(np.asarray(which), device=base_maps.device)]
    return torch.gather(sel, 2, cols[:, None, :].expand(-1, H, -1)).contiguous()


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
        members = np.arange(n)
        g.set_states(members, rolled(base_maps, rng.integers(nb, size=n), rng.integers(W, size=n)))
        d0 = int(rng.integers(0, max_start_day + 1))
        if d0:
            g.step(d0 * DAY)
        g.get_states(members, X[c0:c0 + n])
        g.step((d0 + 1) * DAY)
        g.get_states(members, Y[c0:c0 + n])
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


def rotation_only(net: Surrogate):
    """The rotation-only control: a copy of net whose learned correction is
    switched off (decoder Wd, bd zeroed; parameter order of include/sfs.h:
    We[48][C], be[C], Wd[C][16], bd[16], ...), so that it proposes the map
    rotated by the day's differential rotation and nothing else."""
    w = net.get_params()
    C = net.channels
    o = 48 * C + C
    w[o:o + C * 16 + 16] = 0.0
    ctrl = Surrogate(channels=net.channels, modes=net.modes, blocks=net.blocks, max_batch=net.max_batch, seed=0)
    ctrl.set_params(w)
    return ctrl


def propose(net: Surrogate, S, P, out):
    for c0 in range(0, S.shape[0], net.max_batch):
        c1 = min(S.shape[0], c0 + net.max_batch)
        net.forward(S[c0:c1], P[c0:c1], out[c0:c1])
    return out


def _fluxes(net: Surrogate, maps):
    return net.flux(maps)


def _dev_index(a):
    """A host index or mask array on the device without a synchronising copy
    (pinned host buffer, non-blocking upload on the current stream)."""
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).pin_memory().to("cuda", non_blocking=True)


def _warm_merge_ops(S, prop):
    """Run the host-side merge operations of a rollout day once on scratch
    rows (index upload, gather, scatter, masked select), so that loading or
    compiling their torch kernels, done once per process (and once per box
    for a kernel compiled on first use), is not timed as part of the
    rollout."""
    import torch
    n = S.shape[0]
    k = min(2, n)
    idx = _dev_index(np.arange(k, dtype=np.int64))
    rows = S.index_select(0, idx).contiguous()
    scratch = torch.empty_like(rows)
    scratch.index_copy_(0, _dev_index(np.arange(k, dtype=np.int64)), rows)
    keep = _dev_index(np.zeros(k, dtype=bool))
    torch.where(keep[:, None, None], prop[:k], scratch, out=scratch)
    torch.cuda.current_stream().synchronize()


def _advance_subset(g, gs, S, members, t0, t1, sel=None, ready=None):
    """Queue the plain solver's day [t0, t1] for the given members (every
    other member idles at t1) on the grid's stream gs, after the maps of S
    written so far on the current stream.  With ``sel`` (the members' rows of
    S, gathered on the current stream) and ``ready`` (an event recorded after
    that gather), gs waits for the event only, not for later work of the
    current stream."""
    import torch
    g.set_time(t1)
    if len(members):
        if sel is None:
            sel = S.index_select(0, _dev_index(np.asarray(members, dtype=np.int64))).contiguous()
            gs.wait_stream(torch.cuda.current_stream())
        else:
            gs.wait_event(ready)
        sel.record_stream(gs)  # gs reads it: its memory is not reused before that
        g.set_states(members, sel)
        g.set_times(members, t0)
    g.step(t1)


def _fetch(g, gs, members):
    """The grid's maps of the given members as one packed tensor, usable on the
    current stream."""
    import torch
    out = torch.empty((len(members), H, W), device="cuda")
    gs.wait_stream(torch.cuda.current_stream())
    g.get_states(members, out)
    torch.cuda.current_stream().wait_stream(gs)
    return out


def rollout(net: Surrogate, S0, P, days, drift_tol=1e-4, l2_tol=0.02, spot=32, seed=7, max_fail=0.25,
            solver_sms=24, solver_priority=-1):
    """Surrogate + judge + plain-solver fallback.  Returns (final maps, stats).

    A day on which more than ``max_fail`` of the spot checks fail rejects
    every proposal of that day (the unchecked members cannot be trusted
    either); otherwise only the failing members fall back.  stats["phase_s"]
    splits the host time of the days: queueing the spot checks' solver day
    (while the GPU runs the proposals, which are enqueued first), the
    proposals and their flux sums, waiting for and fetching the solver's
    maps, and the rest (spot-check L2, updates, flux sums of the accepted
    maps).  ``solver_sms`` > 0 keeps that many SMs free of the surrogate's
    persistent forward blocks, for the solver's kernels on the grid stream
    (created with ``solver_priority``) to run beside the proposals."""
    import torch
    n = S0.shape[0]
    params = P.cpu().numpy().astype(np.float64)
    gs = torch.cuda.Stream(priority=solver_priority)
    n_sm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    net.set_sm_budget(max(1, n_sm - solver_sms) if solver_sms > 0 else 0)
    g = _grid(n, params, stream=gs)
    S = S0.clone()
    prop = torch.empty_like(S)
    rng = np.random.default_rng(seed)
    stats = {"member_days": 0, "accepted": 0, "rejected_drift": 0, "rejected_spot": 0, "spot_checked": 0}
    ph = {"queue_spot_day": 0.0, "proposals_and_flux": 0.0, "fetch_solver_maps": 0.0, "rest": 0.0}
    _warm_merge_ops(S, prop)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    phi_old, abs_old = _fluxes(net, S)
    for day in range(days):
        ta = time.perf_counter()
        t_day0, t_day1 = day * DAY, (day + 1) * DAY
        chk = np.sort(rng.choice(n, size=min(spot, n), replace=False))
        run = np.zeros(n, dtype=bool)
        run[chk] = True
        # the spot-checked members' rows are gathered, then the proposals are
        # enqueued (cheap on the host) and the plain solver's day for those
        # members is queued on the grid's stream (sft_step returns without
        # waiting; its host work overlaps the proposals on the GPU, and its
        # kernels run beside them)
        sel = S.index_select(0, _dev_index(chk.astype(np.int64))).contiguous()
        ready = torch.cuda.Event()
        ready.record()
        propose(net, S, P, prop)
        tb = time.perf_counter()
        _advance_subset(g, gs, S, chk, t_day0, t_day1, sel=sel, ready=ready)
        tb2 = time.perf_counter()
        phi_new, abs_new = _fluxes(net, prop)
        tc = time.perf_counter()
        drift = np.abs(phi_new - phi_old) / np.maximum(abs_old, 1e-300)
        bad = drift > drift_tol
        extra = bad & ~run
        if extra.any():  # drift-rejected members outside the spot check: their own plain day
            _advance_subset(g, gs, S, np.flatnonzero(extra), t_day0, t_day1)
            run |= extra
        idx = np.flatnonzero(run)
        plain = _fetch(g, gs, idx)
        torch.cuda.current_stream().synchronize()
        td = time.perf_counter()
        # spot check: relative L2 of the proposal against the solver's day
        pos = {int(i): q for q, i in enumerate(idx)}
        chk_plain = plain.index_select(0, _dev_index(np.array([pos[int(i)] for i in chk], dtype=np.int64)))
        chk_prop = prop.index_select(0, _dev_index(chk.astype(np.int64)))
        err = net.rel_l2(chk_prop, chk_plain)
        spot_bad = np.zeros(n, dtype=bool)
        spot_bad[chk[err > l2_tol]] = True
        day_rejected = np.mean(err > l2_tol) > max_fail
        if day_rejected:
            # untrustworthy day: every member advances with the plain solver
            rest = np.flatnonzero(~run)
            if len(rest):
                _advance_subset(g, gs, S, rest, t_day0, t_day1)
                S.index_copy_(0, _dev_index(rest.astype(np.int64)), _fetch(g, gs, rest))
            spot_bad[:] = True
            stats["days_rejected"] = stats.get("days_rejected", 0) + 1
        use_plain = bad | spot_bad | run  # solver result available for every member it ran on
        S.index_copy_(0, _dev_index(idx.astype(np.int64)), plain)
        keep = _dev_index(~use_plain)
        torch.where(keep[:, None, None], prop, S, out=S)
        stats["member_days"] += n
        stats["accepted"] += int((~use_plain).sum())
        stats["rejected_drift"] += int(bad.sum())
        stats["rejected_spot"] += int((spot_bad & ~bad).sum())
        stats["spot_checked"] += len(chk)
        stats.setdefault("spot_l2_median", []).append(float(np.median(err)))
        if day_rejected:
            phi_old, abs_old = _fluxes(net, S)
        else:
            # the new states' fluxes: an accepted member's is its proposal's
            # (computed above), every other member took the solver's map,
            # so only those maps are summed (the same kernel on the same
            # values: the same numbers as summing all of S)
            phi_old, abs_old = phi_new.copy(), abs_new.copy()
            if len(idx):
                fp, fa = _fluxes(net, plain)
                phi_old[idx], abs_old[idx] = fp, fa
        te = time.perf_counter()
        ph["queue_spot_day"] += tb2 - tb
        ph["proposals_and_flux"] += (tb - ta) + (tc - tb2)
        ph["fetch_solver_maps"] += td - tc
        ph["rest"] += te - td
    torch.cuda.synchronize()
    stats["seconds"] = time.perf_counter() - t0
    stats["member_days_per_s"] = stats["member_days"] / stats["seconds"]
    stats["phase_s"] = ph
    stats["tile_rows"] = g.get_tile_rows(0)  # the autotuner's choice for this grid shape
    stats["solver_sms"] = solver_sms
    net.set_sm_budget(0)
    g.close()
    return S, stats


def plain(S0, P, days):
    """The plain batched solver over the same members and days."""
    import torch
    n = S0.shape[0]
    g = _grid(n, P.cpu().numpy().astype(np.float64))
    members = np.arange(n)
    g.set_states(members, S0.contiguous())
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for day in range(days):
        g.step((day + 1) * DAY)
        g.diagnostics()  # the same per-day history as the rollout keeps
    torch.cuda.synchronize()
    sec = time.perf_counter() - t0
    out = torch.empty_like(S0)
    g.get_states(members, out)
    torch.cuda.synchronize()
    tr = g.get_tile_rows(0)
    g.close()
    return out, {"seconds": sec, "member_days_per_s": n * days / sec, "tile_rows": tr}
