"""Benchmark of the batched SFT step (one JSON line on rank 0).

Workload (the batched-ensemble configuration): 64 realizations on a
1024(theta) x 2048(phi) grid, FP32 state, per-realization rotation
coefficients +-10 %, meridional amplitude U[10,20] m/s and eta U[250,750]
km^2/s (seed 3), 8 seeded dipole + active-region start maps, CFL-limited
steps toward a 27-day end time.  One bench "step" = one call of sft_step
advancing every realization by one time step (SSPRK(4,3) WENO3-CS(h)
advection + RKL2 diffusion, ~410-714 stages) plus the flux diagnostics
of every realization (FP64-accurate: compensated FP32 row sums, FP64
across rows).

value: realization-cell-updates/s (sum over realizations of ntheta*nphi per
step / device time), inputs resident in HBM.  e2e: the same step driven
through the C-ABI with pinned host buffers (set_state from host, step,
get_state to host) inside the timed region.  roofline: the RKL2 stages
(the fused eight-stage kernel dominates), algorithmic bytes per pass (20 B
per cell per pass of eight stages: read delta_{j-2}, delta_{j-1}, G, write
two increments; stage 1 3 words) over the CUDA-event time of the RKL2
region.  cpu_baseline: the FP64 oracle on a bounded sample, one
realization per host core (spawned processes).

flux_drift: the largest change of a realization's total signed flux over
the timed steps relative to its unsigned flux (FP64 diagnostics).  c1: the
single-realization FP64 configuration (128x256, 27 days) on the GPU, its
device time and flux drift, and (with the CPU leg) the same run by the FP64
oracle on a host core with the relative L-inf difference of the final maps.
surrogate: the learned-surrogate ensemble (512 members x 27 days at
256x512, surrogate + judge + fallback against the plain solver and a
rotation-only control) with a reduced training set (--sur-pairs,
--sur-epochs; bench.py --surrogate runs the full training alone).

Multi-GPU (torchrun): realizations are independent, so each rank runs its
own 64-realization ensemble (weak scaling, no collective on the data path);
the timing is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

NT, NP, NREAL = 1024, 2048, 64

# DRAM traffic of rkl2_fused_kernel from one ncu capture (16 x 1024x2048
# ensemble, one launch over all 16 realizations, eight stages, 256-row bands,
# pole values from the ring-sum recurrence): dram__bytes_read +
# dram__bytes_write = 0.9734 x the launch's algorithmic bytes (reads +5 %:
# band-overlap rows; writes -14 %: dirty lines still in L2 when the launch
# ends).  Reported per launch as ratio x algorithmic bytes, and only while the
# kernel sources (comments aside) hash to the profiled ones; otherwise null.
FUSED_TRAFFIC = {"ratio": 0.9732, "profile": "profiles/rkl2_fused_kernel_ncu_16x1024x2048.md",
                 "sha256": "e88b676f31c2d5f1368bc6c9e2e3f5ab20b0c7be4215bd84d9213cd848f72840"}
KERNEL_SOURCES = ("paper_2501_06377_gb300/csrc/sft_kernels.cu", "paper_2501_06377_gb300/csrc/sft_device.cuh")


def kernel_sources_sha256():
    """Hash of the kernel sources with comments and blank lines removed
    (a comment edit does not change the profiled kernel)."""
    import hashlib
    import re
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel)) as f:
            text = re.sub(r"/\*.*?\*/", "", f.read(), flags=re.S)
        for line in text.splitlines():
            line = re.sub(r"//.*$", "", line).rstrip()
            if line:
                h.update(line.encode() + b"\n")
    return h.hexdigest()


T_END = 27 * 24.0
WORKLOAD = ("batched ensemble: 64 realizations x 1024(theta) x 2048(phi), FP32 state, "
            "FP64 flux diagnostics, SSPRK(4,3) WENO3-CS(h) + RKL2, eta U[250,750] km^2/s, "
            "rotation +-10%, meridional U[10,20] m/s, 27-day run, CFL-limited steps")


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def make_inputs(nreal, rank, atten_b0=0.0, splitting="lie"):
    import sft_inputs as I
    from paper_2501_06377_gb300.sft import FlowParams
    draws = I.draw_realization_params(nreal, seed=3 + 1000 * rank)
    params = [FlowParams(*d, atten_b0=atten_b0, splitting=splitting) for d in draws]
    maps = [I.initial_map(NT, NP, seed=1 + i + 100 * rank).astype(np.float32) for i in range(8)]
    return params, maps


C1_SHAPE = (128, 256)
C1_WORKLOAD = ("plain SFT: 1 realization, FP64, 128x256, Omega(lat) = 13.38 - 2.30 sin^2 - 1.62 sin^4 "
               "deg/day in the Carrington frame, 15 m/s sin(2 lat) poleward, eta = 500 km^2/s, 10 G dipole "
               "+ 12 seeded pairs flux balanced, 27 days at CFL steps")


def c1_inputs():
    """The single-realization FP64 configuration: flow parameters and start map."""
    import sft_inputs as I
    d = I.omega_to_dr_coeffs(*I.DEFAULT_OMEGA)
    flow = dict(d0=d[0], d2=d[1], d4=d[2], m1=30.0, m3=0.0, m5=0.0, nu=500.0)
    return flow, I.initial_map(*C1_SHAPE, seed=1)


def run_c1_gpu():
    """C1 on the GPU: the 27-day run (second of two; the first builds the step
    graphs), CUDA-event time on the grid's stream, the flux-balanced start map
    and the final map (host FP64)."""
    import torch
    from paper_2501_06377_gb300.sft import FlowParams, Grid
    flow, B0 = c1_inputs()
    st = torch.cuda.Stream()
    g = Grid([C1_SHAPE], "fp64", stream=st)
    g.set_flows([FlowParams(**flow)])
    for _ in range(2):
        g.set_time(0.0)
        g.set_state(0, B0)
        g.balance_flux()
        start = g.get_state(0)
        d0 = g.diagnostics()[0]
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        n = g.step(27 * 24.0)
        e1.record(st)
        st.synchronize()
        d1 = g.diagnostics()[0]
    final = g.get_state(0)
    g.close()
    return {"workload": C1_WORKLOAD, "gpu_ms": e0.elapsed_time(e1), "steps": n,
            "flux_drift": abs(d1["flux_signed"] - d0["flux_signed"]) / d0["flux_pos"]}, start, final


# --------------------------------------------------------------------------
# CPU oracle (baseline / reference arm)
# --------------------------------------------------------------------------
_ORACLE = {}


def oracle_sample(n_stages=16, index=0):
    """Time the FP64 oracle on realization `index` of the workload: one full
    SSPRK(4,3) advection step plus n_stages of its RKL2 stages, and
    extrapolate to a full step.  Returns (cell-updates/s, ms per full step,
    description, seconds timed).  Set-up (tables, limits) is not timed."""
    import oracle as O
    import sft_inputs as I
    if _ORACLE.get("index") != index:
        d = I.draw_realization_params(index + 1, seed=3)[index]
        B0 = I.initial_map(NT, NP, seed=1 + index % 8)
        _ORACLE["r"] = O.Realization(O.Grid(NT, NP), O.Params(*d), B0)
        _ORACLE["index"] = index
    r = _ORACLE["r"]
    dt = min(r.dt_adv, T_END)
    s = O.rkl2_stage_count(dt, r.dt_euler)
    t0 = time.perf_counter()
    B1 = O.ssprk43_advance(r.B, dt, r.FA)
    t1 = time.perf_counter()
    mu, nu, mut, gt = O.rkl2_coefficients(s)
    LY0 = r.L(B1)
    Ym2, Ym1 = B1, B1 + mut[1] * dt * LY0
    for j in range(2, n_stages + 1):
        Y = (mu[j] * Ym1 + nu[j] * Ym2 + (1.0 - mu[j] - nu[j]) * B1
             + mut[j] * dt * r.L(Ym1) + gt[j] * dt * LY0)
        Ym2, Ym1 = Ym1, Y
    t2 = time.perf_counter()
    t_step = (t1 - t0) + (t2 - t1) * s / n_stages
    cells = NT * NP
    desc = ("1 realization of %dx%d: one SSPRK(4,3) advection step + %d of its %d RKL2 stages "
            "timed (%.1f s), full step extrapolated" % (NT, NP, n_stages, s, t2 - t0))
    return cells / t_step, 1e3 * t_step, desc, t2 - t0


def _oracle_worker(job):
    return oracle_sample(job[1], job[0])


def _c1_oracle_worker(start):
    """The FP64 oracle over the C1 run from the given (flux-balanced) map:
    (seconds, final map)."""
    import oracle as O
    flow, _ = c1_inputs()
    r = O.Realization(O.Grid(*C1_SHAPE), O.Params(**flow), start)
    t0 = time.perf_counter()
    r.advance(27 * 24.0)
    return time.perf_counter() - t0, r.B


class OraclePool:
    """The oracle over host cores: one realization per process (the ensemble
    is parallel over realizations), worker processes started with spawn
    (the parent may already hold a CUDA context) and single-threaded numpy.
    A sample: every worker times its own realization at the same time; the
    throughput is the sum over workers."""

    def __init__(self, procs=None):
        import multiprocessing as mp
        self.procs = procs or max(1, min(os.cpu_count() or 1, NREAL))
        for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ[v] = "1"
        self.pool = mp.get_context("spawn").Pool(self.procs)

    def sample(self, n_stages, c1_start=None):
        """One sample over the workers; with c1_start, one more worker task runs
        the C1 oracle from that map alongside (returned as self.c1)."""
        c1 = self.pool.apply_async(_c1_oracle_worker, (c1_start,)) if c1_start is not None else None
        res = self.pool.map(_oracle_worker, [(i, n_stages) for i in range(self.procs)])
        self.c1 = c1.get() if c1 is not None else None
        v = sum(x[0] for x in res)
        ms = statistics.median(x[1] for x in res)
        el = max(x[3] for x in res)
        desc = ("%d realizations of %dx%d, one per process on %d host cores, each: one SSPRK(4,3) "
                "advection step + %d RKL2 stages timed (%.1f s), full step extrapolated; value = sum "
                "over processes" % (self.procs, NT, NP, self.procs, n_stages, el))
        return v, ms, desc, el

    def close(self):
        self.pool.close()
        self.pool.join()


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    n_stages = 16
    pool = OraclePool()
    vals = []
    try:
        for i in range(args.warmup + args.steps):
            v, ms, desc, el = pool.sample(n_stages)
            if i >= args.warmup:
                vals.append((v, ms))
    finally:
        pool.close()
    v = statistics.median(x[0] for x in vals)
    ms = statistics.median(x[1] for x in vals)
    line = {
        "impl": "reference", "metric": "realization-cell-updates/s", "value": v,
        "unit": "cell-updates/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": "per step: " + desc},
        "cpu_baseline": {"value": v, "unit": "cell-updates/s", "cores": pool.procs, "kind": "oracle",
                         "sample": desc},
        "e2e": {"value": v, "unit": "cell-updates/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------
# GPU arm
# --------------------------------------------------------------------------
def run_gpu(args, rank, world, local_rank):
    import torch
    from paper_2501_06377_gb300 import build as B
    from paper_2501_06377_gb300.sft import Grid

    B.build()
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    stream = torch.cuda.Stream()
    nreal = args.nreal
    params, maps = make_inputs(nreal, rank, args.atten_b0, args.splitting)
    g = Grid([(NT, NP)] * nreal, "fp32", stream=stream)
    for r in range(nreal):
        g.set_state(r, maps[r % len(maps)])
    g.balance_flux()
    g.set_flows(params)
    if args.rfe_rate > 0.0:
        from paper_2501_06377_gb300.sft import RfeParams
        g.set_rfe([RfeParams(method=2, rate_mx_per_hour=args.rfe_rate, lifetime_hours=args.rfe_lifetime,
                             seed=7 + r) for r in range(nreal)])
    cells_per_step = float(nreal * NT * NP)

    def one_step():
        n = g.step(T_END, max_steps=1)
        g.diagnostics()
        return n

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    from paper_2501_06377_gb300.sharding import max_over_ranks as _mor

    def max_over_ranks(x):
        return _mor(x, device="cuda") if dist is not None else x

    # warm-up (autotune + graph capture happen in the first step)
    for _ in range(args.warmup):
        one_step()
    g.reset_stats()
    g.set_profiling(True)
    d_start = g.diagnostics()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(local_rank) as clk:
        t_before = sum(g.get_time())
        e0.record(stream)
        steps_done = 0
        for _ in range(args.steps):
            steps_done += one_step()
        e1.record(stream)
        barrier()
    ms = e0.elapsed_time(e1)
    sim_hours = sum(g.get_time()) - t_before  # simulated hours advanced, summed over realizations
    d_end = g.diagnostics()
    # total signed flux drift over the timed steps, FP64 diagnostics, worst realization
    flux_drift = max(abs(b["flux_signed"] - a["flux_signed"]) / a["flux_pos"] for a, b in zip(d_start, d_end))
    st = g.stats()
    ms = max_over_ranks(ms)
    updates = st["cell_updates"] * world
    value = updates / (ms * 1e-3)
    peak, peak_kind = _peaks()
    # per RKL2 pass (a fused pass = 8 stages; the launches of the chains overlap)
    diff_pass_ms = st["diff_ms"] / max(st["diff_launches"], 1)
    diff_pass_bytes = st["diff_bytes"] / max(st["diff_launches"], 1)
    achieved = diff_pass_bytes / (diff_pass_ms * 1e-3) / 1e9
    launches_per_step = st["kernel_launches"] / max(st["global_steps"], 1)
    # e2e: host-resident state, pinned host buffers, copies inside the timing
    g.set_profiling(False)
    e2e_ms = float("nan")
    if not args.no_e2e:
        host = [torch.from_numpy(maps[r % len(maps)].copy()).pin_memory() for r in range(nreal)]
        e2e_steps = max(2, min(args.steps, 6))
        barrier()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            for r in range(nreal):
                g.set_state(r, host[r])
            g.step(T_END, max_steps=1)
            g.diagnostics()
            for r in range(nreal):
                g.get_state(r, host[r])
        barrier()
        e2e_ms = max_over_ranks((time.perf_counter() - t0) * 1e3 / e2e_steps)
    bytes_state = nreal * NT * NP * 4
    c1 = c1_start = c1_final = None
    if rank == 0 and not args.no_c1:
        c1, c1_start, c1_final = run_c1_gpu()
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        pool = OraclePool()
        try:
            v, cms, desc, el = pool.sample(64, c1_start)
        finally:
            pool.close()
        cpu = {"value": v, "unit": "cell-updates/s", "cores": pool.procs, "kind": "oracle", "sample": desc}
        if pool.c1 is not None and c1 is not None:
            c1_s, c1_ref = pool.c1
            c1["oracle_s"] = c1_s
            c1["rel_linf_vs_oracle"] = float(np.abs(c1_final - c1_ref).max() / np.abs(c1_ref).max())
            c1["bar"] = 1e-12
    sur = None
    if rank == 0 and world == 1 and not args.no_surrogate:
        sur = surrogate_eval(args.sur_pairs, args.sur_epochs, args.members, args.days)
        sur["note"] = ("reduced training for the default run (%d pairs x %d epochs; bench.py --surrogate "
                       "trains on %d x %d)" % (args.sur_pairs, args.sur_epochs, args.pairs, args.epochs))
    clocks = clk.summary()
    if rank == 0:
        line = {
            "metric": "realization-cell-updates/s", "value": value, "unit": "cell-updates/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "realizations_per_gpu": nreal, "grid": [NT, NP],
                       "l2": "inputs larger than L2 (537 MB per state array)",
                       "parallelism": "realizations sharded over ranks, no collective",
                       "cell_stage_updates_per_s": (st["diff_cell_stages"] + st["adv_cell_stages"])
                       * world / (ms * 1e-3),
                       "rkl2_stages_per_step": st["diff_cell_stages"] / max(st["cell_updates"], 1),
                       "graph": True, "rkl2_stages_per_launch": g.get_fusion(),
                       "band_rows": g.get_band_rows(0), "tile_rows": g.get_tile_rows(0),
                       "flow_attenuation_b0": args.atten_b0, "splitting": args.splitting,
                       "rfe": ({"method": 2, "rate_mx_per_hour": args.rfe_rate, "lifetime_hours": args.rfe_lifetime}
                               if args.rfe_rate > 0.0 else None),
                       "realization_hours_per_s": sim_hours * world / (ms * 1e-3),
                       "ms_per_step_split": {"rkl2": st["diff_ms"] / args.steps,
                                             "advection": st["adv_ms"] / args.steps,
                                             "rest": (ms - st["diff_ms"] - st["adv_ms"]) / args.steps}},
            "roofline": {"bound": "hbm",
                         "kernel": ("rkl2_fused_kernel (8 RKL2 stages per launch, up to six launch chains)"
                                    if g.get_fusion() > 1 else "rkl2_stage_kernel<float>"),
                         "achieved": achieved,
                         "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "peak_kind": peak_kind + " hbm_gbs",
                         "bytes_per_pass": diff_pass_bytes, "ms_per_pass": diff_pass_ms,
                         "traffic": (FUSED_TRAFFIC["ratio"] * diff_pass_bytes
                                     if g.get_fusion() > 1
                                     and FUSED_TRAFFIC["sha256"] == kernel_sources_sha256() else None),
                         "traffic_source": FUSED_TRAFFIC["profile"]},
            "e2e": {"value": cells_per_step * world / (e2e_ms * 1e-3), "unit": "cell-updates/s",
                    "h2d_bytes_per_step": bytes_state, "d2h_bytes_per_step": bytes_state,
                    "ms_per_step": e2e_ms},
            "flux_drift": flux_drift,
            "gpu_launches": int(st["kernel_launches"] + 2 * st["global_steps"]),
            "gpu_launches_per_step": launches_per_step + 2,
            "clocks": clocks,
        }
        if cpu:
            line["cpu_baseline"] = cpu
        if c1:
            line["c1"] = c1
        if sur:
            line["surrogate"] = sur
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


# --------------------------------------------------------------------------
# learned surrogate + judge + fallback (256 x 512 ensemble, one-day steps)
# --------------------------------------------------------------------------
def surrogate_eval(pairs, epochs, members, days):
    """Train the surrogate on solver-generated one-day pairs, then advance
    an ensemble for `days` days with judge and fallback, against the plain
    batched solver and a rotation-only control (trained correction removed).
    Returns the result record (member-days/s, errors, judge counts, timings)."""
    import torch
    import sft_inputs as I
    from paper_2501_06377_gb300 import ensemble as E
    from paper_2501_06377_gb300.sft import Grid
    from paper_2501_06377_gb300.surrogate import Surrogate

    t_all = time.perf_counter()
    nbase = 64
    g = Grid([(E.H, E.W)] * nbase, "fp32")
    base = torch.empty((nbase, E.H, E.W), device="cuda")
    for i in range(nbase):
        g.set_state(i, I.initial_map(E.H, E.W, seed=1000 + i).astype(np.float32))
    g.balance_flux()
    g.get_states(np.arange(nbase), base)
    torch.cuda.synchronize()
    g.close()
    t0 = time.perf_counter()
    X, Y, P = E.make_pairs(base, pairs, seed=5)
    t_pairs = time.perf_counter() - t0
    net = Surrogate(channels=64, modes=48, blocks=4, max_batch=32, seed=1)
    c0 = net.counters()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hist = E.train(net, X, Y, P, epochs=epochs, batch=32, lr=2e-3)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    c1 = net.counters()
    del X, Y
    # evaluation ensemble: unseen start maps (rolled), unseen parameters
    rng = np.random.default_rng(11)
    Pm = torch.from_numpy(E.draw_params(members, 11).astype(np.float32)).cuda()
    S0 = E.rolled(base, rng.integers(nbase, size=members), rng.integers(E.W, size=members))
    ref, st_plain = E.plain(S0, Pm, days)
    out, st_sur = E.rollout(net, S0, Pm, days)
    err = np.concatenate([net.rel_l2(out[i:i + 32].contiguous(), ref[i:i + 32].contiguous())
                          for i in range(0, members, 32)])
    # control: the same network with its learned correction switched off
    ctrl = E.rotation_only(net)
    out_c, st_ctrl = E.rollout(ctrl, S0, Pm, days)
    err_c = np.concatenate([ctrl.rel_l2(out_c[i:i + 32].contiguous(), ref[i:i + 32].contiguous())
                            for i in range(0, members, 32)])
    return {
        "member_days_per_s": st_sur["member_days_per_s"],
        "plain_member_days_per_s": st_plain["member_days_per_s"],
        "speedup_vs_plain": st_sur["member_days_per_s"] / st_plain["member_days_per_s"],
        "day_rollout_rel_l2_vs_plain": {"days": days, "median": float(np.median(err)),
                                        "p90": float(np.percentile(err, 90)), "max": float(err.max())},
        "accepted_fraction": st_sur["accepted"] / st_sur["member_days"],
        "rejected_drift": st_sur["rejected_drift"], "rejected_spot": st_sur["rejected_spot"],
        "spot_checked": st_sur["spot_checked"],
        "spot_l2_median_by_day": st_sur["spot_l2_median"],
        "rollout_phase_s": st_sur["phase_s"],
        "tile_rows": {"rollout": st_sur.get("tile_rows"), "plain": st_plain.get("tile_rows")},
        "control_rotation_only": {"member_days_per_s": st_ctrl["member_days_per_s"],
                                  "accepted_fraction": st_ctrl["accepted"] / st_ctrl["member_days"],
                                  "spot_l2_median": float(np.median(st_ctrl["spot_l2_median"])),
                                  "rel_l2_median_vs_plain": float(np.median(err_c)),
                                  "note": "its proposals fail the judge, so its members follow the plain solver"},
        "train": {"pairs": pairs, "epochs": epochs, "seconds": t_train,
                  "pair_generation_seconds": t_pairs, "params": net.num_params(),
                  "gemm_tflops": (c1["gemm_flops"] - c0["gemm_flops"]) / t_train / 1e12,
                  "loss_history": hist[::max(1, len(hist) // 12)]},
        "members": members, "days": days,
        "judge": "flux drift > 1e-4 or spot-check L2 > 2% (32 members a day), plain-solver fallback",
        "seconds_total": time.perf_counter() - t_all,
    }


def run_surrogate(args):
    """The learned-surrogate ensemble alone, at the full training size."""
    import torch
    from paper_2501_06377_gb300 import build as B
    B.build()
    torch.cuda.set_device(0)
    r = surrogate_eval(args.pairs, args.epochs, args.members, args.days)
    line = {"metric": "ensemble simulated member-days/s (surrogate + judge + fallback vs plain solver)",
            "value": r["member_days_per_s"], "unit": "member-days/s", **r,
            "config": {"workload": "learned surrogate: %d members x 256x512 FP32, %d days, 1-day proposals, "
                                   "judge: flux drift > 1e-4 or spot-check L2 > 2%%, plain-solver fallback"
                                   % (args.members, args.days),
                       "members": args.members, "days": args.days, "net": "C=64, M=48 modes, L=4, BF16 GEMMs"}}
    print(json.dumps(line), flush=True)
    return 0


def _hh(X, Y):
    """The paper's HH error metric (Sec. 2.6, Eq. hh) in FP64 on the device."""
    X, Y = X.double(), Y.double()
    return float((((X - Y) ** 2).sum() / (X.abs() * Y.abs()).sum()).sqrt())


C4_SHAPES = [((256, 512), 128), ((512, 1024), 96), ((1440, 2880), 32)]


def run_config(args):
    """The long assimilative runs, one JSON line each.

    c2: one 512x1024 FP32 realization started from the dipole, hourly
    mu-weighted flux-balanced assimilation of the hidden-truth stream
    (Earth-facing hemisphere) for args.days days (365), beside a free run
    from the same start without assimilation; reports the final HH against
    the truth, the largest net-flux imbalance seen, and the run time.
    c4: the uneven batch (256 realizations in three grid shapes, 199.8 M
    cells), per-realization parameters, hourly assimilation of one truth
    stream per grid shape, args.days days (90); reports the flux imbalance,
    the HH against the truth per shape, and realization-hours/s."""
    import torch
    import sft_inputs as I
    from paper_2501_06377_gb300 import build as B
    from paper_2501_06377_gb300.sft import AssimParams, FlowParams, Grid
    B.build()
    torch.cuda.set_device(0)
    ap = AssimParams(alpha_mu=4.0, mu_lim=0.1, lat_lim_deg=90.0, flux_balance=True)
    off = AssimParams(alpha_mu=4.0, mu_lim=2.0, lat_lim_deg=90.0, flux_balance=True)  # mu <= 1 < 2: F = 0
    if args.config == "c2":
        days = args.days if args.days != 27 else 365
        shapes = [(512, 1024)] * 2
        d = I.omega_to_dr_coeffs(*I.DEFAULT_OMEGA)
        params = [FlowParams(d0=d[0], d2=d[1], d4=d[2], m1=30.0, m3=0.0, m5=0.0, nu=500.0)] * 2
        aps = [ap, off]
        streams = {(512, 1024): I.ObservationStream(512, 1024, seed=2, days=days + 1)}
        mode = 0
    else:
        days = args.days if args.days != 27 else 90
        shapes = [sh for sh, n in C4_SHAPES for _ in range(n)]
        params = [FlowParams(*dr) for dr in I.draw_realization_params(len(shapes), seed=3)]
        aps = [ap] * len(shapes)
        streams = {sh: I.ObservationStream(*sh, seed=2, days=days + 1) for sh, _ in C4_SHAPES}
        mode = 2
    distinct = list(dict.fromkeys(shapes))
    g = Grid(shapes, "fp32")
    for r, sh in enumerate(shapes):
        g.set_state(r, I.dipole(*sh).astype(np.float32))
    g.set_flows(params)
    worst = 0.0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    t_truth = 0.0
    for hour in range(1, 24 * days + 1):
        g.step(float(hour))
        ta = time.perf_counter()
        obs = torch.cat([streams[sh].truth_torch(float(hour)).float().reshape(-1) for sh in distinct])
        mu = torch.cat([streams[sh].mu_torch(float(hour)).float().reshape(-1) for sh in distinct])
        t_truth += time.perf_counter() - ta
        g.assimilate(obs, mu, mode, aps)
        if hour % 24 == 0:
            for dg in g.diagnostics():
                worst = max(worst, abs(dg["flux_signed"]) / dg["flux_pos"])
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    T = 24.0 * days
    truth = {sh: streams[sh].truth_torch(T).float() for sh in distinct}
    hh = {}
    for r, sh in enumerate(shapes):
        m = torch.from_numpy(g.get_state(r)).cuda()
        hh.setdefault(sh, []).append(_hh(m, truth[sh]))
    st = g.stats()
    line = {"metric": "assimilative run (%s): simulated realization-hours/s" % args.config,
            "value": len(shapes) * T / wall, "unit": "realization-hours/s", "days": days,
            "wall_s": wall, "truth_generation_s": t_truth, "steps": st["global_steps"],
            "max_net_flux_over_unsigned": worst, "dtype": "f32", "data": "synthetic",
            "assimilation": "hourly, alpha_mu = 4, mu_lim = 0.1, no latitude cut, flux balanced (Eq. fluxbal)"}
    if args.config == "c2":
        line["hh_vs_truth"] = {"assimilated": hh[(512, 1024)][0], "free_run": hh[(512, 1024)][1]}
        line["config"] = {"workload": "C2: 512x1024 FP32, 1 realization, %d days, hourly assimilation of a "
                                      "hidden-truth stream (1 new pair/day, Earth-facing hemisphere), from the "
                                      "dipole only; a free run beside it" % days}
    else:
        line["hh_vs_truth_median_by_shape"] = {"%dx%d" % sh: float(np.median(v)) for sh, v in hh.items()}
        line["config"] = {"workload": "C4: 256 realizations (128 x 256x512, 96 x 512x1024, 32 x 1440x2880), "
                                      "FP32, %d days, hourly assimilation of one truth stream per shape" % days}
    print(json.dumps(line), flush=True)
    return 0


def run_sharded_c4(args, rank, world, local_rank):
    """The uneven 256-realization batch sharded over the ranks (one process
    per GPU): realizations bin-packed by cost (LPT over cells x (stages + 4)
    x steps), each rank advancing its own shard for args.hours hours with no
    collective on the data path, then every realization's FP64 diagnostics
    gathered on rank 0.  value: realization-hours / the slowest rank's time
    (grid set-up included); scaling strong (the batch is fixed)."""
    import torch
    import sft_inputs as I
    from paper_2501_06377_gb300 import build as B
    from paper_2501_06377_gb300 import sharding as SH
    from paper_2501_06377_gb300.sft import FlowParams, Grid
    B.build()
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    shapes = [sh for sh, n in C4_SHAPES for _ in range(n)]
    params = [FlowParams(*dr) for dr in I.draw_realization_params(len(shapes), seed=3)]
    # cost of each realization from its own step plan (one small grid per shape)
    costs = []
    plan = {}
    for sh, _ in C4_SHAPES:
        plan[sh] = Grid([sh], "fp32")
    for sh, fp in zip(shapes, params):
        plan[sh].set_flows([fp])
        dt_cfl, _, s = plan[sh].step_plan(0, 1.0)
        steps = max(1, math.ceil(1.0 / min(1.0, dt_cfl) - 1e-12))
        costs.append(SH.shard_costs([sh], [plan[sh].step_plan(0, 1.0 / steps)[2]], steps)[0])
    for gp in plan.values():
        gp.close()
    dip = {}

    def start(sh):
        if sh not in dip:
            dip[sh] = I.dipole(*sh).astype(np.float32)
        return dip[sh]
    advance = SH.grid_advance(shapes, params, start, float(args.hours))
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    shards, recs, sec = SH.run_sharded(costs, advance, world, rank)
    torch.cuda.synchronize()
    sec = SH.max_over_ranks(sec, device="cuda") if dist is not None else sec
    if rank == 0:
        drift = max(abs(d["flux_signed"]) / d["flux_pos"] for _, d in recs)
        loads = [sum(costs[i] for i in s) for s in shards]
        line = {"metric": "sharded uneven batch: realization-hours/s", "value": len(shapes) * args.hours / sec,
                "unit": "realization-hours/s", "n_gpus": world, "scaling": "strong", "dtype": "f32",
                "data": "synthetic", "seconds": sec, "hours": args.hours,
                "records_gathered": len(recs), "max_net_flux_over_unsigned": drift,
                "shard_sizes": [len(s) for s in shards],
                "shard_cost_balance": max(loads) / (sum(loads) / len(loads)),
                "config": {"workload": "C4 uneven batch: 256 realizations (128 x 256x512, 96 x 512x1024, "
                                       "32 x 1440x2880), FP32, sharded by cost over ranks, no data-path "
                                       "collective, FP64 diagnostics gathered on rank 0 (grid set-up timed)"}}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_smoother(args):
    """The flux-preserving map smoother (grid-based diffusivity, Eq. diffgrid):
    a batch of 512x1024 FP32 maps, alpha_nu = 0.5, diffusion only, one hour
    (nu_g t ~ 1/2 grid cell^2: the least smoothing that removes single-cell
    structure).  value: maps/s with the maps resident; e2e: maps/s from
    pinned host maps to smoothed host maps."""
    import torch
    from paper_2501_06377_gb300 import build as B
    from paper_2501_06377_gb300.sft import FlowParams, Grid
    import sft_inputs as I
    B.build()
    nt, np_, n = 512, 1024, args.maps
    g = Grid([(nt, np_)] * n, "fp32")
    maps = [I.initial_map(nt, np_, seed=70 + i).astype(np.float32) for i in range(8)]
    for r in range(n):
        g.set_state(r, maps[r % 8])
    g.set_flows([FlowParams(advection=False, nu_grid_alpha=args.alpha_nu)] * n)
    stages = g.step_plan(0, 1.0)[2]

    def smooth():
        g.set_time(0.0)
        g.step(1.0)

    for _ in range(args.warmup):
        smooth()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        smooth()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    host = [torch.from_numpy(maps[r % 8].copy()).pin_memory() for r in range(n)]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for r in range(n):
            g.set_state(r, host[r])
        smooth()
        for r in range(n):
            g.get_state(r, host[r])
    torch.cuda.synchronize()
    e2e_ms = (time.perf_counter() - t0) * 1e3 / args.steps
    line = {"metric": "smoothed maps/s (512x1024, grid-based diffusivity)", "value": n / (ms * 1e-3),
            "unit": "maps/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": "map smoother: %d maps of 512x1024, alpha_nu = %g /h, 1 h, RKL2 "
                                   "(%d stages)" % (n, args.alpha_nu, stages), "maps": n},
            "e2e": {"value": n / (e2e_ms * 1e-3), "unit": "maps/s", "ms_per_step": e2e_ms,
                    "h2d_bytes_per_step": n * nt * np_ * 4, "d2h_bytes_per_step": n * nt * np_ * 4},
            "paper_context": "0.25 s per 512x1024 map on an RTX 3090Ti (smoothing length not stated)"}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--nreal", type=int, default=NREAL,
                    help="realizations per GPU (smaller only for profiling captures)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--splitting", default="lie", choices=["lie", "strang"],
                    help="operator splitting of a step (Sec. 3.5)")
    ap.add_argument("--rfe-rate", type=float, default=0.0,
                    help="random flux emergence (Sec. 2.4, method 2): unsigned Mx per hour; 0 = off")
    ap.add_argument("--rfe-lifetime", type=float, default=24.0, help="hours between RFE source maps")
    ap.add_argument("--atten-b0", type=float, default=0.0,
                    help="flow attenuation saturation field in G (Eq. flow_attenuation); 0 = off")
    ap.add_argument("--surrogate", action="store_true",
                    help="learned-surrogate ensemble evaluation instead of the solver benchmark")
    ap.add_argument("--pairs", type=int, default=20000)
    ap.add_argument("--members", type=int, default=512)
    ap.add_argument("--days", type=int, default=27)
    ap.add_argument("--epochs", type=int, default=16)
    ap.add_argument("--config", choices=["c2", "c4", "c4s"], default=None,
                    help="a long assimilative run instead of the benchmark (c2: 365 days, c4: 90 days), or "
                         "c4s: the uneven batch sharded over the ranks for --hours")
    ap.add_argument("--hours", type=float, default=6.0, help="simulated hours of --config c4s")
    ap.add_argument("--no-c1", action="store_true", help="skip the single-realization FP64 run")
    ap.add_argument("--no-surrogate", action="store_true",
                    help="skip the (reduced-training) surrogate ensemble of the default run")
    ap.add_argument("--sur-pairs", type=int, default=8000, help="training pairs of the default run's surrogate")
    ap.add_argument("--sur-epochs", type=int, default=12, help="training epochs of the default run's surrogate")
    ap.add_argument("--smoother", action="store_true",
                    help="grid-based-diffusivity map smoother instead of the solver benchmark")
    ap.add_argument("--maps", type=int, default=64)
    ap.add_argument("--alpha-nu", type=float, default=0.5)
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.config == "c4s":
        return run_sharded_c4(args, rank, world, local_rank)
    if args.config:
        return run_config(args)
    if args.surrogate:
        return run_surrogate(args)
    if args.smoother:
        return run_smoother(args)
    return run_gpu(args, rank, world, local_rank)


if __name__ == "__main__":
    sys.exit(main())
