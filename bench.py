#!/usr/bin/env python
"""Benchmark of the W2-FWI likelihood-guidance gradient on GB300.

One step = one pass of the whole hot path over a batch of B synthetic 70x70
models (5 surface shots, 70 receivers, 1000 steps, 40-cell absorbing layer):
observation preparation, forward solve with wavefield record, W2 misfit and
adjoint source, adjoint solve with imaging and fold, and the preconditioned
guided update.  Metric: W2-FWI gradients/s (plus Gcell-updates/s).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--batch B] [--impl ours|reference]
                    [--workload 70x70|256x256|512x1024]

--workload selects the larger grids (256x256: 16 shots, 2000 steps, record
kept, on the cluster propagators; 512x1024: 32 shots, 4000 steps, checkpoints
every 32 steps, on the tiled propagators); the default is the 70x70 workload
above (resident propagators).

Under torchrun (N > 1) every rank owns its own B models (weak scaling, no
data-path collective); the step time is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

DX, DT, NB = 10.0, 1e-3, 40
UNIT = "gradients/s"
# name: physical grid, steps, shots, receivers, model family, default batch,
# checkpoint interval (0: whole record kept); the plan picks the propagator
# family (resident, cluster or tiled) from the grid
WORKLOADS = {
    "70x70": dict(nz=70, nx=70, nt=1000, ns=5, nr=70, kind="layered", batch=152, ckpt=0),
    "256x256": dict(nz=256, nx=256, nt=2000, ns=16, nr=256, kind="curved_faulted", batch=8,
                    ckpt=0),
    "512x1024": dict(nz=512, nx=1024, nt=4000, ns=32, nr=1024, kind="curved_faulted", batch=2,
                     ckpt=32),
}


def metric_of(name):
    w = WORKLOADS[name]
    return f"W2-FWI gradients/s ({w['nz']}x{w['nx']}, {w['ns']} shots, {w['nt']} steps)"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def record_traffic(units, path="resident", workload="70x70", nt=0, what="dram_bytes"):
    """Counts per launch of the two propagators from the committed ncu capture
    of that kernel family (what = "dram_bytes" or "smem_wavefronts"), scaled
    by (model, shot) units (and, for the cluster kernels, captured per time
    step, by the steps); None once the kernel source has changed since the
    capture, or for a workload that was not captured."""
    import hashlib
    name = {"resident": "propagators_traffic.json",
            "cluster": f"cluster_traffic_{workload}.json"}.get(path)
    try:
        with open(os.path.join(ROOT, "profiles", name)) as f:
            rec = json.load(f)
        with open(os.path.join(ROOT, rec["source"]), "rb") as f:
            if hashlib.sha256(f.read()).hexdigest() != rec["sha256"]:
                return None
        if f"{what}_per_unit_step" in rec:
            return {k: v * units * nt for k, v in rec[f"{what}_per_unit_step"].items()}
        return {k: v * units for k, v in rec[f"{what}_per_unit"].items()}
    except Exception:
        return None


def rank_seed0(rank: int, batch: int) -> int:
    """First model seed of a rank: ranks own disjoint blocks of `batch` seeds
    (weak scaling, no data-path collective)."""
    return rank * batch


def max_over_ranks(values, world: int, device=None):
    """Element-wise max of per-rank timings (the slowest rank sets the step
    time); a no-op on one rank."""
    import torch
    t = torch.tensor(values, dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def workload_inputs(wl, B, seed0):
    from paper_2603_16393_gb300 import inputs as I
    vt = I.model_batch(wl["kind"], range(seed0, seed0 + B), wl["nz"], wl["nx"])
    v0 = np.stack([I.linear_initial_model(wl["nz"], wl["nx"])] * B)
    geo = I.surface_geometry(wl["nx"], wl["ns"], wl["nr"])
    return vt, v0, geo


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 8:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[4 + i] == "Active"})
        loaded = sorted(sm)[len(sm) // 2:] if sm else []
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


# ------------------------------------------------------------------ oracle timing
def oracle_sample(n_models, threads, seed0=0, wl=None):
    """Time the FP64 oracle on a bounded sample of the same workload: n_models
    full gradients (forward + W2 misfit + adjoint for each shot)."""
    from oracle import oracle as O
    wl = wl or WORKLOADS["70x70"]
    vt, v0, geo = workload_inputs(wl, n_models, seed0)
    op = O.Problem(nz=wl["nz"], nx=wl["nx"], nb=NB, nt=wl["nt"], dz=DX, dx=DX, dt=DT,
                   src_iz=geo.src_iz, src_ix=geo.src_ix, rec_iz=geo.rec_iz, rec_ix=geo.rec_ix)
    w2p = O.W2Params()
    ctx = O.w2_prepare(O.forward(op, vt, threads=threads), op.dt, w2p)
    t = time.perf_counter()
    O.gradient(op, v0, ctx, w2p, threads=threads)
    return time.perf_counter() - t


def cpu_cores():
    return len(os.sched_getaffinity(0))


def run_reference(args, rank, world):
    """--impl reference: the oracle as it stands, on the host cores, rank 0 only."""
    if rank != 0:
        return
    wl = WORKLOADS["70x70"]
    NS = wl["ns"]
    threads = cpu_cores()
    n_models = max(1, threads // NS + (1 if threads % NS else 0))
    for _ in range(args.warmup):
        oracle_sample(n_models, threads)
    times = [oracle_sample(n_models, threads) for _ in range(args.steps)]
    tstep = statistics.mean(times)
    value = n_models / tstep
    line = {
        "impl": "reference", "metric": metric_of("70x70"), "value": value, "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": tstep * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded layered models)",
        "config": {"workload": f"{n_models} x 70x70 layered models, 5 shots, 70 receivers, "
                               "1000 steps, 40-cell absorbing layer (bounded CPU sample)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": f"{n_models} full gradients per step on {threads} threads"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ our path
def run_ours(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist

    from paper_2603_16393_gb300 import api

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    wl = dict(WORKLOADS[args.workload])
    if args.nt:
        wl["nt"] = args.nt
    NZ_PHYS, NX_PHYS, NT, NS, NR = wl["nz"], wl["nx"], wl["nt"], wl["ns"], wl["nr"]
    B = args.batch or wl["batch"]
    vt, v0, geo = workload_inputs(wl, B, seed0=rank_seed0(rank, B))
    prob = api.Problem(nz=NZ_PHYS, nx=NX_PHYS, nb=NB, nt=NT, dz=DX, dx=DX, dt=DT,
                       src_iz=geo.src_iz, src_ix=geo.src_ix, rec_iz=geo.rec_iz,
                       rec_ix=geo.rec_ix, v_max=4500.0, batch=B, checkpoint_every=wl["ckpt"],
                       absorber=api.ABSORBER_CPML if args.absorber == "cpml" else api.ABSORBER_SPONGE)
    plan = api.Plan(prob, api.W2Params(), device=dev)
    path = {api.KERNELS_RESIDENT: "resident", api.KERNELS_TILED: "tiled",
            api.KERNELS_CLUSTER: "cluster", api.KERNELS_CPML: "cpml"}[plan.kernels]
    # Table 1 (CurveVel-A) rho0, gamma; Sec. 6.3 c, tau, eps; the diffusion's
    # normalised space (v - 3000)/1500 has a unit of 1500 m/s
    gparams = api.GuideParams(rho0=1.15, gamma=0.55, unit=1500.0)
    stream = torch.cuda.current_stream(dev)

    # observed data of the true models (untimed setup), inputs resident in HBM
    vt_d = torch.tensor(vt, dtype=torch.float32, device=dev)
    d_obs, _ = plan.forward(vt_d, store=False)
    d_obs = d_obs.clone()
    v_d = torch.tensor(v0, dtype=torch.float32, device=dev)
    ctx = plan.new_ctx()
    shape = plan.model_shape
    d_syn = torch.empty(plan.data_shape, dtype=torch.float32, device=dev)
    adj = torch.empty(plan.data_shape, dtype=torch.float32, device=dev)
    J = torch.empty(B, dtype=torch.float32, device=dev)
    grad = torch.empty(shape, dtype=torch.float32, device=dev)
    v_out = torch.empty(shape, dtype=torch.float32, device=dev)
    rho = torch.empty(B, dtype=torch.float32, device=dev)
    ev = {k: [] for k in ("fwd0", "fwd1", "adj0", "adj1")}

    def step(v_in, dobs_in, timed, prepare=True):
        # a4 (observation preparation) runs once per observation: the device-
        # timed steps reuse the context; the end-to-end steps take a new
        # observation from the host each step and prepare it
        if prepare:
            api.fwi_w2_prepare(plan.handle, dobs_in, ctx)
        if timed:
            e0 = torch.cuda.Event(enable_timing=True); e0.record(stream)
        api.fwi_forward(plan.handle, v_in, d_syn, plan.snapshots, plan.workspace)
        if timed:
            e1 = torch.cuda.Event(enable_timing=True); e1.record(stream)
        api.fwi_w2_misfit(plan.handle, ctx, d_syn, J, None, adj, plan.workspace)
        if timed:
            e2 = torch.cuda.Event(enable_timing=True); e2.record(stream)
        api.fwi_adjoint_grad(plan.handle, v_in, adj, plan.snapshots, grad, plan.workspace)
        if timed:
            e3 = torch.cuda.Event(enable_timing=True); e3.record(stream)
            ev["fwd0"].append(e0); ev["fwd1"].append(e1); ev["adj0"].append(e2); ev["adj1"].append(e3)
        # preconditioned update (no network: v' = v0hat = v, g = h = dJ/dv)
        api.fwi_guided_step(B, NZ_PHYS, NX_PHYS, gparams, v_in, v_in, grad, grad, v_out, rho)

    # library kernels per timed step: forward, misfit (2), adjoint + shot
    # sum, guided (1); the cluster adjoint adds a fold; the tiled propagators
    # launch once per time step, plus a set-up (and a resume per recomputed
    # segment) and a final gather or fold.  (The observation preparation, 4
    # kernels, is timed apart.)
    if path == "resident":
        kernels_per_step = 1 + 2 + 2 + 1
    elif path == "cpml":
        # set-up 2 + 2 a step (forward); set-up 2 + init + 3 a step (2 at the
        # last) + fold (adjoint), + shot sum
        kernels_per_step = (2 + 2 * NT) + 2 + (2 + 1 + 3 * NT - 2 + 1 + 1) + 1
    elif path == "cluster":
        kernels_per_step = 1 + 2 + 3 + 1
    else:
        K = wl["ckpt"]
        S = -(-NT // K) if K else 0
        fwd_k = 1 + NT + 1
        adj_k = (2 * S + (S - 1) + 2 * NT + 2) if K else (1 + NT + 2)
        kernels_per_step = fwd_k + 2 + adj_k + 1

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    for _ in range(args.warmup):
        step(v_d, d_obs, False)
    barrier()
    # a4 alone: the observation preparation of this batch, amortised per observation
    p0 = torch.cuda.Event(enable_timing=True)
    p1 = torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    for _ in range(args.steps):
        api.fwi_w2_prepare(plan.handle, d_obs, ctx)
    p1.record(stream)
    barrier()
    prep_ms = p0.elapsed_time(p1) / args.steps
    clocks = ClockSampler(local_rank) if rank == 0 else None
    if clocks:
        clocks.start()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.steps):
        step(v_d, d_obs, True, prepare=False)
    t1.record(stream)
    barrier()
    clk = clocks.stop() if clocks else None
    plan.check()
    ms = t0.elapsed_time(t1) / args.steps
    fwd_ms = statistics.mean(a.elapsed_time(b) for a, b in zip(ev["fwd0"], ev["fwd1"]))
    adj_ms = statistics.mean(a.elapsed_time(b) for a, b in zip(ev["adj0"], ev["adj1"]))

    # end to end through the public API with pinned host buffers: every
    # step's inputs go host -> device on a copy stream into one of two buffer
    # sets while the previous step computes (a user's pipeline); the step
    # waits for its copy, and its results come back on the compute stream
    v_h = torch.tensor(v0, dtype=torch.float32).pin_memory()
    dobs_h = d_obs.cpu().pin_memory()
    out_grad_h = torch.empty(shape, dtype=torch.float32).pin_memory()
    out_J_h = torch.empty(B, dtype=torch.float32).pin_memory()
    out_v_h = torch.empty(shape, dtype=torch.float32).pin_memory()
    v_e = [torch.empty_like(v_d) for _ in range(2)]
    dobs_e = [torch.empty_like(d_obs) for _ in range(2)]
    copy_st = torch.cuda.Stream(device=dev)
    loaded = [torch.cuda.Event() for _ in range(2)]
    freed = [torch.cuda.Event() for _ in range(2)]
    used = [False, False]
    barrier()
    e_s = torch.cuda.Event(enable_timing=True)
    e_e = torch.cuda.Event(enable_timing=True)
    e_s.record(stream)
    copy_st.wait_event(e_s)          # every copy falls inside the timed region

    def load(k):
        if used[k]:
            copy_st.wait_event(freed[k])     # the step that read this set is done
        with torch.cuda.stream(copy_st):
            v_e[k].copy_(v_h, non_blocking=True)
            dobs_e[k].copy_(dobs_h, non_blocking=True)
        loaded[k].record(copy_st)
        used[k] = True

    load(0)
    for i in range(args.steps):
        k = i & 1
        if i + 1 < args.steps:
            load(1 - k)
        stream.wait_event(loaded[k])
        step(v_e[k], dobs_e[k], False)
        freed[k].record(stream)
        out_grad_h.copy_(grad, non_blocking=True)
        out_J_h.copy_(J, non_blocking=True)
        out_v_h.copy_(v_out, non_blocking=True)
    e_e.record(stream)
    barrier()
    e2e_ms = e_s.elapsed_time(e_e) / args.steps
    h2d = (v_h.numel() + dobs_h.numel()) * 4
    d2h = (out_grad_h.numel() + out_J_h.numel() + out_v_h.numel()) * 4

    # max over ranks
    ms, e2e_ms, fwd_ms, adj_ms = max_over_ranks([ms, e2e_ms, fwd_ms, adj_ms], world, dev)
    if rank != 0:
        return

    plane = (NZ_PHYS + NB) * (NX_PHYS + 2 * NB)
    cu = B * NS * NT * plane                         # cell-updates of one propagator pass
    cell_updates = 2 * cu                            # forward + adjoint, per step per rank
    small = B * NS * NR * NT * 4 + B * NZ_PHYS * NX_PHYS * 4 * (1 + NS + 1)
    K = wl["ckpt"]
    if path in ("resident", "cluster"):
        # the fields stay on chip (one CTA's, or a cluster's shared memory);
        # the propagators stream the wavefield record (4 B per cell-update:
        # the forward writes it, the adjoint reads it) + traces, models and
        # per-shot gradients
        adj_bytes, fwd_bytes = cu * 4 + small, cu * 4 + B * NS * NR * NT * 4 + B * NZ_PHYS * NX_PHYS * 4
        adj_name, fwd_name = (("adjoint propagator", "forward propagator") if path == "resident"
                              else ("cluster adjoint (+ fold)", "cluster forward"))
    elif path == "cpml":
        # CPML kernels, compulsory bytes per cell-update: forward u read,
        # u' written, increment read + written, record written (20 B) and, in
        # the layer's share f of the cells, psi_x, psi_z, zeta_x, zeta_z read
        # + written (32 B); adjoint mu, nu, imaging sum read + written, record
        # read, h_x, h_z written + read (44 B) and in the layer psi, zeta
        # adjoints read + written and t_x, t_z written + read (48 B); kappa
        # once per model and step
        f = 1.0 - NZ_PHYS * NX_PHYS / plane
        tables = B * NT * plane * 4
        fwd_bytes = int(cu * (20 + 32 * f)) + tables + B * NS * NR * NT * 4
        adj_bytes = int(cu * (44 + 48 * f)) + tables + small
        fwd_name, adj_name = "CPML forward (2 launches a step)", "CPML adjoint (3 launches a step)"
    else:
        # tiled, per cell-update: forward reads u, v and writes u, v (16 B;
        # + 4 B record); adjoint reads psi, w, imaging sum, record and writes
        # psi, w, imaging sum (28 B); the per-model tables kappa A, A B (8 B
        # per cell) are read once per model and step (shots of a model share
        # them); with checkpoints the adjoint call also recomputes the
        # forward with its record
        tables = B * NT * plane * 8
        ck = (2 * B * NS * plane * 4 * -(-NT // K)) if K else 0
        fwd_bytes = cu * (16 if K else 20) + tables + ck + small
        adj_bytes = cu * 28 + tables + ((cu * 20 + tables) if K else 0) + small
        fwd_name = "tiled forward"
        adj_name = "tiled adjoint call (recompute + adjoint)" if K else "tiled adjoint"
    hbm_peak, peak_kind = peaks()
    dom = max((adj_ms, adj_bytes, adj_name, "adjoint"), (fwd_ms, fwd_bytes, fwd_name, "forward"))
    achieved = dom[1] / (dom[0] * 1e-3) / 1e9
    traffic = record_traffic(B * NS, path, args.workload, NT)
    traffic = traffic[dom[3]] if traffic else None
    value = world * B / (ms * 1e-3)
    # the on-chip propagators (fields in shared memory) are bound inside the
    # SM, by the shared-memory pipe: one wavefront (up to 128 B) per clock per
    # SM; the wavefronts per launch come from the committed capture
    roof_smem = None
    if path in ("resident", "cluster"):
        # the shared-memory roof of the on-chip propagators against the
        # algorithmic 24 bytes per cell-update (own column window, x
        # neighbours, old level and table, store; the z neighbours come from
        # registers): 128 B per clock per SM at the sampled clock; the
        # measured wavefronts of the committed capture give the pipe's
        # occupancy beside it
        mhz = (clk or {}).get("sm_mhz") or 2070.0
        n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
        peak_b = 128.0 * n_sm * mhz * 1e6
        per = {k: cu * 24.0 / (t * 1e-3) for k, t in (("forward", fwd_ms), ("adjoint", adj_ms))}
        roof_smem = {"bound": "smem", "kernel": dom[2], "achieved": per[dom[3]] / 1e9,
                     "peak": peak_b / 1e9, "unit": "GB/s", "bytes_per_cell_update": 24,
                     "frac": per[dom[3]] / peak_b,
                     "frac_forward": per["forward"] / peak_b,
                     "frac_adjoint": per["adjoint"] / peak_b,
                     "peak_source": f"128 B per clock per SM x {n_sm} SMs x {mhz:.0f} MHz "
                                    "(sampled clock)"}
        wf = record_traffic(B * NS, path, args.workload, NT, what="smem_wavefronts")
        if wf:
            roof_smem["pipe_occupancy"] = {
                k: wf[k] / (t * 1e-3) / (n_sm * mhz * 1e6)
                for k, t in (("forward", fwd_ms), ("adjoint", adj_ms))}

    cpu = None
    if world == 1 and not args.no_cpu_baseline and args.workload != "512x1024":
        threads = cpu_cores()
        n_models = max(1, (2 * threads + NS - 1) // NS) if args.workload == "70x70" else 1
        t = oracle_sample(n_models, threads, wl=wl)
        cpu = {"value": n_models / t, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"{n_models} full {NZ_PHYS}x{NX_PHYS} gradients ({NS} shots x {NT} "
                         f"steps, FP64) on {threads} threads, {t:.1f} s wall"}
        if args.workload == "70x70":
            # the same oracle on one thread: one full gradient
            t1 = oracle_sample(1, 1, wl=wl)
            cpu["single_thread"] = {"value": 1.0 / t1, "unit": UNIT, "cores": 1,
                                    "sample": f"1 full {NZ_PHYS}x{NX_PHYS} gradient on 1 thread, "
                                              f"{t1:.1f} s wall"}

    record = (f"checkpoints every {K} steps" if K else "store-all wavefield record")
    resident_gb = (B * NS * NT * plane * 4 if not K else B * NS * 6 * plane * 4) / 1e9
    line = {
        "metric": metric_of(args.workload) if not args.nt else metric_of(args.workload).replace(
            f"{WORKLOADS[args.workload]['nt']} steps", f"{NT} steps"), "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": f"synthetic (seeded {wl['kind'].replace('_', '/')} models)",
        "config": {"propagators": path, "workload": f"{B} x {NZ_PHYS}x{NX_PHYS} {wl['kind'].replace('_', '/')} models "
                               f"per GPU, {NS} shots, {NR} receivers, {NT} steps, 40-cell "
                               f"{'CPML' if path == 'cpml' else 'absorbing'} layer, {record}",
                   "batch_per_gpu": B, "global_batch": B * world,
                   "l2": ("inputs larger than L2 (wavefield record %.1f GB per step)" if not K
                          else "inputs larger than L2 (propagator fields %.1f GB)")
                         % resident_gb,
                   "gcell_updates_per_s": world * cell_updates / (ms * 1e-3) / 1e9},
        "roofline": {"bound": "hbm", "kernel": dom[2], "achieved": achieved,
                     "peak": hbm_peak, "unit": "GB/s", "frac": achieved / hbm_peak,
                     "traffic": traffic, "algorithmic_bytes": dom[1],
                     "peak_source": peak_kind, "ms_per_launch": dom[0]},
        "roofline_smem": roof_smem,
        "kernel_ms": {"forward": fwd_ms, "adjoint": adj_ms},
        "obs_prepare_ms": prep_ms,
        "e2e": {"value": world * B / (e2e_ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms},
        "gpu_launches": kernels_per_step * args.steps,
        "clocks": clk,
        "cpu_baseline": cpu,
    }
    if cpu is None and args.workload == "512x1024":
        line["config"]["cpu_baseline_note"] = ("not sampled: one FP64 oracle unit keeps 4000 "
                                               "wavefield levels of 552x1104 cells (19.5 GB)")
    print(json.dumps(line), flush=True)


# the batched uneven workload: (workload, models) -- curved/faulted models,
# observed data with Gaussian noise at 10 dB SNR
MIXED = (("70x70", 64), ("256x256", 8), ("512x1024", 2))


def run_mixed(args, rank, world, local_rank):
    """--mixed: 64 x 70x70 + 8 x 256x256 + 2 x 512x1024 models in one plan
    group; a step (observation preparation, the group's gradients, guided
    step per plan) is captured once into a CUDA graph and replayed.  Also
    times the same work as per-plan calls in sequence on one stream."""
    import torch
    from paper_2603_16393_gb300 import api
    from paper_2603_16393_gb300 import inputs as I
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    plans, dobs, vs, outs = [], [], [], []
    n_models = 0
    for i, (name, B) in enumerate(MIXED):
        wl = dict(WORKLOADS[name], kind="curved_faulted")
        vt, v0, geo = workload_inputs(wl, B, seed0=rank_seed0(rank, B) + 1000 * i)
        prob = api.Problem(nz=wl["nz"], nx=wl["nx"], nb=NB, nt=wl["nt"], dz=DX, dx=DX, dt=DT,
                           src_iz=geo.src_iz, src_ix=geo.src_ix, rec_iz=geo.rec_iz,
                           rec_ix=geo.rec_ix, v_max=4500.0, batch=B,
                           checkpoint_every=wl["ckpt"])
        plan = api.Plan(prob, api.W2Params(), device=dev)
        d, _ = plan.forward(torch.tensor(vt, dtype=torch.float32, device=dev), store=False)
        noise = I.gaussian_noise_like(d.cpu().numpy(), 10.0, seed=77 + i)
        dobs.append(d + torch.tensor(noise, dtype=torch.float32, device=dev))
        vs.append(torch.tensor(v0, dtype=torch.float32, device=dev))
        outs.append((plan.new_ctx(), torch.empty_like(vs[-1]),
                     torch.empty(B, dtype=torch.float32, device=dev)))
        plans.append(plan)
        n_models += B
    group = api.Group(plans)
    gparams = api.GuideParams(rho0=1.15, gamma=0.55, unit=1500.0)
    stream = torch.cuda.current_stream(dev)

    def prepare():
        for plan, d, (ctx, _, _) in zip(plans, dobs, outs):
            plan.w2_prepare(d, ctx)

    def guide(grads):
        for v, g, (_, v_out, rho) in zip(vs, grads, outs):
            api.guided_step(v, v, g, g, gparams, v_out=v_out)

    def step_group():
        prepare()
        _, grads = group.gradient(vs, [o[0] for o in outs])
        guide(grads)

    def step_sequential():
        prepare()
        grads = [plan.gradient(v, o[0])[1] for plan, v, o in zip(plans, vs, outs)]
        guide(grads)

    def timed(fn, steps):
        torch.cuda.synchronize(dev)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(steps):
            fn()
        b.record(stream)
        torch.cuda.synchronize(dev)
        return a.elapsed_time(b) / steps

    for _ in range(args.warmup):
        step_sequential()
    seq_ms = timed(step_sequential, max(1, args.steps // 2))
    side = torch.cuda.Stream(device=dev)
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        for _ in range(2):
            step_group()
    stream.wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        step_group()
    for _ in range(args.warmup):
        graph.replay()
    clocks = ClockSampler(local_rank) if rank == 0 else None
    if clocks:
        clocks.start()
    ms = timed(graph.replay, args.steps)
    clk = clocks.stop() if clocks else None
    for plan in plans:
        plan.check()
    ms = max_over_ranks([ms], world, dev)[0]
    if rank != 0:
        return
    line = {
        "metric": "uneven batch models/s (64x70x70 + 8x256x256 + 2x512x1024, 5/16/32 shots, "
                  "1000/2000/4000 steps)",
        "value": world * n_models / (ms * 1e-3), "unit": "models/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded curved/faulted models, observed data at 10 dB SNR)",
        "config": {"workload": "plan group: 64 x 70x70 (resident kernels), 8 x 256x256 (cluster "
                               "kernels), 2 x 512x1024 (tiled, checkpoints every 32 steps); one "
                               "CUDA graph per step (observation preparation, group gradients "
                               "on forked streams, guided steps)",
                   "propagators": [p.kernels for p in plans],
                   "sequential_ms_per_step": seq_ms,
                   "speedup_vs_sequential": seq_ms / ms},
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)


def run_sampler(args, rank, world, local_rank):
    """--sampler: reverse steps of Algorithm 2 (Sec. 5.2) on B models of the
    70x70 workload: per step the Gaussian-prior score, the clean estimate and
    proposal (fwi_ddpm_proposal), the W2 gradient at the clamped physical
    model (forward -> misfit -> adjoint), the chain rule (fwi_ddpm_guidance)
    and the preconditioned update (fwi_guided_step).  The observation is
    fixed through the sampling, so its preparation runs once, untimed; the
    draws z of every step are on the device before the timed region."""
    import torch
    from paper_2603_16393_gb300 import api
    from paper_2603_16393_gb300 import inputs as I
    from paper_2603_16393_gb300 import sampler as S
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    wl = WORKLOADS["70x70"]
    B = args.batch or wl["batch"]
    nz, nx = wl["nz"], wl["nx"]
    vt, _, geo = workload_inputs(wl, B, seed0=rank_seed0(rank, B))
    prob = api.Problem(nz=nz, nx=nx, nb=NB, nt=args.nt or wl["nt"], dz=DX, dx=DX, dt=DT,
                       src_iz=geo.src_iz, src_ix=geo.src_ix, rec_iz=geo.rec_iz,
                       rec_ix=geo.rec_ix, v_max=4500.0, batch=B)
    plan = api.Plan(prob, api.W2Params(), device=dev)
    d_obs, _ = plan.forward(torch.tensor(vt, dtype=torch.float32, device=dev), store=False)
    ctx = plan.w2_prepare(d_obs)
    # the prior: per-cell moments of 64 seeded models of the same family,
    # disjoint from the models that made the observations
    prior = S.GaussianPrior.from_models(I.model_batch(wl["kind"], range(90_000, 90_064), nz, nx),
                                        device=dev)
    betas = S.linear_betas(1000)
    frac = args.surrogate_fraction
    net = None
    if args.score == "conv":
        from paper_2603_16393_gb300 import score_net as SN
        net = SN.ConvScore((B, nz, nx), betas, device=dev)
    elif args.score == "unet":
        from paper_2603_16393_gb300 import score_net as SN
        net = SN.UNetScore((B, nz, nx), betas, device=dev)
    lowfi = None
    if frac > 0 and args.surrogate == "net":
        # a 3-layer 128-channel convolutional surrogate of dJ/dv (seeded weights: the
        # cost of a trained one; scales as a trained surrogate would use them)
        from paper_2603_16393_gb300 import score_net as SN
        lowfi = S.NetworkSurrogate(SN.ConvScore((B, nz, nx), betas, seed=9, device=dev),
                                   1.0 / 3000.0, 1e-3)
    elif frac > 0:
        lowfi = S.LowFidelity(plan, d_obs)
    smp = S.Sampler(plan, betas, ctx=ctx, prior=None if net else prior, score_fn=net,
                    guide=api.GuideParams(rho0=1.15, gamma=0.55), surrogate=lowfi,
                    surrogate_fraction=frac if frac > 0 else 0.4)
    total = args.warmup + args.steps
    i0 = 400
    gen = torch.Generator(device=dev).manual_seed(1234 + rank)
    zs = torch.randn((total, B, nz, nx), device=dev, generator=gen)
    ab = smp.steps[i0].abar
    v = (ab ** 0.5) * prior.mu + (1 - ab) ** 0.5 * torch.randn((B, nz, nx), device=dev,
                                                                generator=gen)
    bufs = [torch.empty_like(v) for _ in range(2)]
    stream = torch.cuda.current_stream(dev)

    def barrier(world):
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize(dev)

    for w in range(args.warmup):
        v, _ = smp.step(v, i0 - w, zs[w], v_out=bufs[w % 2])
    barrier(world)
    torch.cuda.synchronize(dev)
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local_rank) if rank == 0 else None
    if clocks:
        clocks.start()
    a.record(stream)
    for k in range(args.steps):
        w = args.warmup + k
        v, info = smp.step(v, i0 - w, zs[w], v_out=bufs[w % 2])
    b.record(stream)
    torch.cuda.synchronize(dev)
    barrier(world)
    clk = clocks.stop() if clocks else None
    ms = a.elapsed_time(b) / args.steps
    plan.check()
    ms = max_over_ranks([ms], world, dev)[0]
    ms_sur = None
    if lowfi is not None:
        # the same number of steps inside the surrogate phase (i > i_switch)
        i1 = 1000
        assert smp.uses_surrogate(i1 - total + 1)
        for w in range(args.warmup):
            v, _ = smp.step(v, i1 - w, zs[w], v_out=bufs[w % 2])
        barrier(world)
        a.record(stream)
        for k in range(args.steps):
            w = args.warmup + k
            v, _ = smp.step(v, i1 - w, zs[w], v_out=bufs[w % 2])
        b.record(stream)
        torch.cuda.synchronize(dev)
        barrier(world)
        if isinstance(lowfi, S.LowFidelity):
            lowfi.plan.check()
        ms_sur = max_over_ranks([a.elapsed_time(b) / args.steps], world, dev)[0]

    # the two elementwise kernels alone, at this batch (bytes: v_i, z read,
    # v0hat, v', v_phys written; v0hat, g_phys read, g, h written; the
    # per-cell prior arrays are read once per launch)
    st = smp.steps[i0]
    n = B * nz * nx
    reps = 50

    def per_launch(fn):
        # the launches replayed from one CUDA graph: device time per launch,
        # not the host's launch rate
        side = torch.cuda.Stream(device=dev)
        side.wait_stream(stream)
        with torch.cuda.stream(side):
            fn()
        stream.wait_stream(side)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            for _ in range(reps):
                fn()
        graph.replay()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        graph.replay()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / reps

    t_prop = per_launch(lambda: api.fwi_ddpm_proposal(
        B, nz * nx, st, smp.space, v, None, prior.mu, prior.tau2, zs[0], smp.v0hat, smp.v_prime,
        smp.v_phys))
    t_guid = per_launch(lambda: api.fwi_ddpm_guidance(
        B, nz * nx, st, smp.space, smp.v0hat, smp.g, None, prior.tau2, bufs[0], smp.h))
    net_ms = None
    if net is not None:
        # the score network alone: eps and its vector-Jacobian product
        def net_step():
            net(v, i0)
            net.eps_vjp(smp.g, 1.0)
        net_ms = per_launch(net_step)
    if rank != 0:
        return
    by_prop, by_guid = 20 * n + 8 * nz * nx, 16 * n + 4 * nz * nx
    n_sur = 1000 - smp.i_switch if lowfi is not None else 0
    chain_ms = (n_sur * ms_sur if ms_sur else 0.0) + (1000 - n_sur) * ms
    line = {
        "metric": "Algorithm 2 reverse steps x models/s (70x70, 5 shots, 1000 steps, W2 guidance"
                  + (f"; {'network-surrogate' if args.surrogate == 'net' else 'low-fidelity'} "
                     f"guidance in the first {frac:.0%} of 1000 steps)" if lowfi else ")"),
        "value": world * B * 1000 / (chain_ms * 1e-3), "unit": "model-steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": chain_ms / 1000,
        "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded layered models; Gaussian prior fitted to 64 seeded models)",
        "config": {"workload": f"{B} x 70x70 models per GPU, reverse steps {i0}..{i0 - total + 1} "
                               "of a 1000-step linear schedule; per step: "
                               + ("network score and its vector-Jacobian product"
                                  if net else "prior score")
                               + ", clean estimate, proposal, W2 gradient (5 shots, 1000 steps), "
                               "chain rule, preconditioned update",
                   "batch_per_gpu": B,
                   "l2": "inputs larger than L2 (wavefield record 10 GB per step)",
                   "score": ({"conv": "3-layer 128-channel convolutional noise-prediction "
                                      "network on the tensor cores (seeded weights)",
                              "unet": "4-level U-Net noise-prediction network (widths 32-256) "
                                      "on the tensor cores (seeded weights)"}[args.score]
                             if net else "Gaussian prior fitted to 64 seeded models"),
                   "score_network_ms_per_step": net_ms,
                   "surrogate_fraction": frac,
                   "ms_per_step_full_physics": ms,
                   "ms_per_step_low_fidelity": ms_sur,
                   "chain_ms_1000_steps": chain_ms},
        "elementwise_kernels": {
            "proposal": {"ms": t_prop, "gb_s": by_prop / (t_prop * 1e-3) / 1e9,
                         "bytes": by_prop},
            "guidance": {"ms": t_guid, "gb_s": by_guid / (t_guid * 1e-3) / 1e9,
                         "bytes": by_guid},
            "share_of_step": (t_prop + t_guid) / ms,
            "timing": "50 launches replayed from one CUDA graph; HBM peak "
                      f"{peaks()[0]:.0f} GB/s (of measured)"},
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)


def run_uneven(args, rank, world, local_rank):
    """--uneven: gradients of uneven instances that the resident kernels hold
    -- 64 curved/faulted models of 70 x 70 (5 shots), 48 of 50 x 60 (3 shots)
    and 64 of 30 x 60 (2 shots), dx = 10 m, 1000 steps, a 40-cell layer --
    three ways: each plan's
    gradient in turn, the plans as a group on forked streams (one CUDA graph),
    and the forward and adjoint of all plans each in one persistent launch
    (api.Queue; every (model, shot) unit of every plan on one list that the
    CTAs draw from).  The metric is gradients (models) per second."""
    import torch
    from paper_2603_16393_gb300 import api
    from paper_2603_16393_gb300 import inputs as I
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    sizes = [(70, 70, 40, 5, 64), (50, 60, 40, 3, 48), (30, 60, 40, 2, 64)]
    plans, vs, ctxs = [], [], []
    for k, (nz, nx, nb, ns, B) in enumerate(sizes):
        geo = I.surface_geometry(nx, ns)
        prob = api.Problem(nz=nz, nx=nx, nb=nb, nt=args.nt or 1000, dz=DX, dx=DX, dt=DT,
                           src_iz=geo.src_iz, src_ix=geo.src_ix, rec_iz=geo.rec_iz,
                           rec_ix=geo.rec_ix, v_max=4500.0, batch=B)
        p = api.Plan(prob, api.W2Params(), device=dev)
        seed0 = rank_seed0(rank, 1000) + 1000 * k
        vt = torch.tensor(I.model_batch("curved_faulted", range(seed0, seed0 + B), nz, nx),
                          dtype=torch.float32, device=dev)
        ctxs.append(p.w2_prepare(p.forward(vt, store=False)[0].clone()))
        vs.append(torch.tensor(np.stack([I.linear_initial_model(nz, nx)] * B),
                               dtype=torch.float32, device=dev))
        plans.append(p)
    models = sum(B for *_, B in sizes)
    group = api.Group(plans)
    queue = api.Queue(plans)
    stream = torch.cuda.current_stream(dev)

    def sequential():
        for p, v, c in zip(plans, vs, ctxs):
            p.gradient(v, c)

    def grouped():
        group.gradient(vs, ctxs)

    def queued():
        queue.gradient(vs, ctxs)

    def timed(fn):
        side = torch.cuda.Stream(device=dev)
        side.wait_stream(stream)
        with torch.cuda.stream(side):
            for _ in range(args.warmup):
                fn()
        stream.wait_stream(side)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            fn()
        graph.replay()
        torch.cuda.synchronize(dev)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(args.steps):
            graph.replay()
        b.record(stream)
        torch.cuda.synchronize(dev)
        return a.elapsed_time(b) / args.steps

    clocks = ClockSampler(local_rank) if rank == 0 else None
    if clocks:
        clocks.start()
    ms = {k: timed(f) for k, f in (("sequential", sequential), ("group", grouped),
                                   ("queue", queued))}
    clk = clocks.stop() if clocks else None
    for p in plans:
        p.check()
    ms = dict(zip(ms, max_over_ranks(list(ms.values()), world, dev)))
    if rank != 0:
        return
    line = {
        "metric": "W2-FWI gradients/s of uneven resident instances (64 x 70x70 + 48 x 50x60 + "
                  "64 x 30x60, 1000 steps)",
        "value": world * models / (ms["queue"] * 1e-3), "unit": "gradients/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms["queue"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded curved/faulted models)",
        "config": {"workload": "; ".join(f"{B} x {nz}x{nx}, {ns} shots, {nb}-cell layer"
                                         for nz, nx, nb, ns, B in sizes),
                   "forms": "each form captured in one CUDA graph and replayed",
                   "l2": "inputs larger than L2 (wavefield record 28 GB per step)"},
        "ms": ms,
        "models_per_s": {k: world * models / (t * 1e-3) for k, t in ms.items()},
        "queue_vs_sequential": ms["sequential"] / ms["queue"],
        "queue_vs_group": ms["group"] / ms["queue"],
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)


def run_posterior(args, rank, world, local_rank):
    """--posterior: posterior sampling by Algorithm 2 (Sec. 5.2) on noisy
    observations (10 dB), as the scope table's full guided reverse diffusion
    states it: P posterior samples per observation, N reverse steps, W2
    guidance batched over observations x samples x shots.  Three arms on the
    same draws:
      graph_fd   all-FD guidance, every reverse step replayed from one CUDA
                 graph (sampler.GraphChain)
      graph_sur  the learned forward surrogate in the first 40% of the steps,
                 checked against FD every 10 steps and replaced by FD for good once
                 its gradient error exceeds 5%; trained first on FD pairs of
                 the clean estimates of those steps (training timed apart)
      graph_sur_ungated  the same surrogate phase with the FD check's verdicts
                 recorded but not enforced (what the surrogate would save)
      plain      one plan per posterior sample (batch 1, five shots), eager
                 launches: timed over a few reverse steps of every sample; one
                 sample runs the whole chain and is compared with the batched
                 one bit for bit
    Reported: posterior samples/s of each arm (the headline is graph_fd, whose
    samples are the plain path's bit for bit), velocity RMSE and relative L2
    error of the samples and of each observation's posterior mean against the
    true models, the samples' mean W2 misfit beside the true models', the
    surrogate's W2-gradient error against FD per noise level, and the gate's
    record."""
    import dataclasses as dc
    import torch
    from paper_2603_16393_gb300 import api
    from paper_2603_16393_gb300 import inputs as I
    from paper_2603_16393_gb300 import sampler as S
    from paper_2603_16393_gb300 import surrogate as SG
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    nz = nx = 70
    NT, NS = 1000, 5
    n_obs, P = args.observations, args.samples
    B = n_obs * P
    N = args.reverse_steps
    geo = I.surface_geometry(nx, NS)
    prob = api.Problem(nz=nz, nx=nx, nb=NB, nt=NT, dz=DX, dx=DX, dt=DT, src_iz=geo.src_iz,
                       src_ix=geo.src_ix, rec_iz=geo.rec_iz, rec_ix=geo.rec_ix, v_max=4500.0,
                       batch=B)
    plan = api.Plan(prob, api.W2Params(), device=dev)
    seed0 = 7000 + 100 * rank
    vt = I.model_batch("curved_faulted", range(seed0, seed0 + n_obs), nz, nx)
    vt_rep = np.repeat(vt, P, axis=0)
    d_clean = plan.forward(torch.tensor(vt_rep, dtype=torch.float32, device=dev),
                           store=False)[0].cpu().numpy()
    noise = np.concatenate([np.repeat(I.gaussian_noise_like(d_clean[o * P:o * P + 1], 10.0,
                                                            seed0 + o), P, axis=0)
                            for o in range(n_obs)])
    d_obs = torch.tensor(d_clean + noise, dtype=torch.float32, device=dev)
    ctx = plan.w2_prepare(d_obs)
    if args.prior == "lowrank":
        prior = S.LowRankPrior.from_models(I.model_batch("curved_faulted", range(90_000, 90_512),
                                                         nz, nx), k=32, device=dev)
    else:
        prior = S.GaussianPrior.from_models(I.model_batch("curved_faulted", range(90_000, 90_064),
                                                          nz, nx), device=dev)
    # the 1000-step linear schedule's total noise spread over N steps
    betas = S.linear_betas(N, 1e-4 * 1000 / N, 0.02 * 1000 / N)
    # (rho0, gamma, c): the TV damping exp(-TV / c) is off (c = 1e9) because the
    # Gaussian prior's clean estimates are rough cell by cell; rho0 = 300 brings
    # the samples' misfit down to that of the true model under the noise
    guide = api.GuideParams(rho0=300.0, gamma=0.55, c=1e9)
    gen = torch.Generator(device=dev).manual_seed(4321 + rank)
    zs = torch.randn((N + 1, B, nz, nx), device=dev, generator=gen)
    v_start = torch.randn((B, nz, nx), device=dev, generator=gen)
    stream = torch.cuda.current_stream(dev)
    vt_d = torch.tensor(vt_rep, dtype=torch.float32, device=dev)

    def timed(fn):
        torch.cuda.synchronize(dev)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        out = fn()
        b.record(stream)
        torch.cuda.synchronize(dev)
        return out, a.elapsed_time(b)

    def misfit(v):
        J, _, _ = plan.gradient(v.contiguous(), ctx)
        return float(J.mean())

    def quality(v_state):
        v = (3000.0 + 1500.0 * v_state).clamp(1500.0, 4500.0)
        rmse = float(((v - vt_d) ** 2).mean().sqrt())
        J = misfit(v)
        m = torch.empty((B, 3), dtype=torch.float32, device=dev)
        api.fwi_image_metrics(B, nz, nx, 3000.0, vt_d, v.contiguous(), m)
        pm = v.reshape(n_obs, P, nz, nx).mean(dim=1)
        vt_o = vt_d.reshape(n_obs, P, nz, nx)[:, 0]
        rmse_mean = float(((pm - vt_o) ** 2).mean().sqrt())
        return {"rmse_m_s": rmse, "rel_l2": float(m[:, 0].mean()), "ssim": float(m[:, 2].mean()),
                "posterior_mean_rmse_m_s": rmse_mean, "w2_misfit_mean": J}

    # ---- the learned surrogate: FD pairs of early clean estimates, training
    i_switch = N - int(round(0.4 * N))
    t_data = time.time()
    raw = torch.tensor(I.surrogate_training_models(0, args.surrogate_models).astype(np.float32),
                       device=dev)
    n_early = (args.surrogate_models * 3 // 4) // B * B
    est = SG.early_clean_estimates(raw[:n_early], prior, betas, i_switch + 1, N, B, seed=1)
    fd_plan = plan
    v_tr, d_tr = SG.fd_pairs(fd_plan, torch.cat([est, raw[n_early:]])[:raw.shape[0] // B * B])
    torch.cuda.synchronize(dev)
    t_data = time.time() - t_data
    net = SG.ForwardSurrogate(B, nz, nx, NT, geo.src_ix, geo.rec_ix, SG.trace_amplitude(d_tr),
                              seed=0, device=dev)
    tr = SG.SurrogateTrainer(net)
    sched = [(args.surrogate_steps // 2, 1e-3), (args.surrogate_steps // 4, 3e-4),
             (args.surrogate_steps - args.surrogate_steps // 2 - args.surrogate_steps // 4, 1e-4)]
    log = []

    def train_all():
        for n, lr in sched:
            tr.lr = lr
            log.extend(SG.train(tr, v_tr, d_tr, n, log_every=max(1, n)))
    _, t_train = timed(train_all)
    guid = SG.SurrogateGuidance(net, plan, ctx)
    # W2-gradient error against FD per noise level, on the clean estimates of
    # the true models noised to that step
    levels = []
    for i in sorted({N, int(0.9 * N), int(0.8 * N), int(0.7 * N), i_switch + 1,
                     int(0.5 * N), int(0.3 * N), int(0.1 * N)}, reverse=True):
        v = SG.early_clean_estimates(vt_d, prior, betas, i, i, B, seed=i)
        _, g_fd, _ = plan.gradient(v, ctx)
        g_fd = g_fd.clone()
        d_fd = plan.forward(v, store=False)[0].clone()
        d_s = net.forward(v)
        _, g_s = guid.gradient(v)
        e = SG.rel_error(g_s, g_fd)
        levels.append({"step": i, "abar": float(np.prod(1.0 - np.asarray(betas[:i]))),
                       "data_rel_l2": float((d_s - d_fd).norm() / d_fd.norm()),
                       "grad_rel_l2_median": float(e.median()), "grad_rel_l2_max": float(e.max()),
                       "grad_cosine": float((g_s * g_fd).sum() / (g_s.norm() * g_fd.norm()))})

    # ---- arm graph_fd
    chain_fd = S.GraphChain(plan, betas, ctx, prior, guide, zs)
    chain_fd.capture("fd")
    chain_fd.run(v_start, N, N - 2)          # warm-up replays
    clocks = ClockSampler(local_rank) if rank == 0 else None
    if clocks:
        clocks.start()
    v_fd, ms_fd = timed(lambda: chain_fd.run(v_start).clone())
    q_fd = quality(v_fd)
    # ---- arm graph_sur
    chain_sur = S.GraphChain(plan, betas, ctx, prior, guide, zs, surrogate=guid,
                             surrogate_fraction=0.4, threshold=0.05, check_every=10)
    for k in ("fd", "sur", "check"):
        chain_sur.capture(k)
    v_sur, ms_sur = timed(lambda: chain_sur.run(v_start).clone())
    q_sur = quality(v_sur)
    # ---- arm graph_sur_ungated: the same surrogate phase with the FD check's
    # verdicts recorded but not enforced
    chain_free = S.GraphChain(plan, betas, ctx, prior, guide, zs, surrogate=guid,
                              surrogate_fraction=0.4, threshold=float("inf"), check_every=10)
    for k in ("fd", "sur", "check"):
        chain_free.capture(k)
    v_free, ms_free = timed(lambda: chain_free.run(v_start).clone())
    clk = clocks.stop() if clocks else None
    q_free = quality(v_free)
    plan.check()
    # ---- arm plain: one plan per posterior sample, eager launches
    p1 = api.Plan(dc.replace(prob, batch=1), api.W2Params(), device=dev)
    ctxs = [p1.w2_prepare(d_obs[b:b + 1].contiguous()) for b in range(B)]
    smps = [S.Sampler(p1, betas, ctx=c, prior=prior, guide=guide) for c in ctxs]
    K = args.plain_steps
    vs = [v_start[b:b + 1].clone() for b in range(B)]

    def plain_steps():
        for k in range(K):
            i = N - k
            for b in range(B):
                vs[b], _ = smps[b].step(vs[b], i, zs[i, b:b + 1].contiguous())
    _, ms_plain_k = timed(plain_steps)
    ms_plain = ms_plain_k / K * N
    # one sample through the whole chain on the plain path, against the batched arm
    v1 = v_start[0:1].clone()

    def plain_chain():
        nonlocal v1
        for i in range(N, 0, -1):
            v1, _ = smps[0].step(v1, i, zs[i, 0:1].contiguous())
    timed(plain_chain)
    p1.check()
    bitwise = bool(torch.equal(v1[0], v_fd[0]))
    if rank != 0:
        return
    arms = {
        "graph_fd": {"samples_per_s": B / (ms_fd * 1e-3), "chain_s": ms_fd * 1e-3, **q_fd},
        "graph_sur": {"samples_per_s": B / (ms_sur * 1e-3), "chain_s": ms_sur * 1e-3, **q_sur,
                      "steps": dict(chain_sur.counts),
                      "gate": [{"step": i, "grad_rel_l2_max": e, "accepted": ok}
                               for i, e, ok in chain_sur.records]},
        "graph_sur_ungated": {"samples_per_s": B / (ms_free * 1e-3), "chain_s": ms_free * 1e-3,
                              **q_free, "steps": dict(chain_free.counts),
                              "gate_errors": [e for _, e, _ in chain_free.records]},
        "plain": {"samples_per_s": B / (ms_plain * 1e-3), "chain_s": ms_plain * 1e-3,
                  "timed_reverse_steps": K, "chain_extrapolated_from_timed_steps": True,
                  "one_sample_whole_chain_bitwise_equal_to_graph_fd": bitwise},
    }
    best = "graph_fd"     # the arm whose samples equal the plain path's bit for bit
    line = {
        "metric": f"posterior samples/s (Algorithm 2, 70x70, 5 shots x 1000 FD steps, {N} reverse "
                  "steps, 10 dB observations)",
        "value": arms[best]["samples_per_s"], "unit": "posterior samples/s", "n_gpus": world,
        "steps": 1, "warmup": 1, "ms_per_step": arms[best]["chain_s"] * 1e3 / N,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded curved/faulted true models, Gaussian noise at 10 dB; "
                + ("low-rank Gaussian prior, 32 principal directions of 512 seeded models)"
                   if args.prior == "lowrank" else
                   "diagonal Gaussian prior fitted to 64 seeded models)"),
        "config": {"workload": f"{n_obs} observations x {P} posterior samples = {B} models per "
                               f"GPU, {N} reverse steps, W2 guidance (5 shots, 70 receivers, "
                               "1000 steps, 40-cell layer)",
                   "headline_arm": best,
                   "l2": "inputs larger than L2 (wavefield record 44 GB per reverse step)"},
        "arms": arms,
        "speedup_vs_plain": {k: arms[k]["samples_per_s"] / arms["plain"]["samples_per_s"]
                             for k in ("graph_fd", "graph_sur", "graph_sur_ungated")},
        "guide": {"rho0": guide.rho0, "gamma": guide.gamma, "c": guide.c},
        "true_model_w2_misfit_mean": misfit(vt_d),
        "surrogate": {"training_pairs": int(v_tr.shape[0]),
                      "pairs": "FD seismograms of clean estimates of reverse steps "
                               f"{i_switch + 1}..{N} (3/4) and of seeded models (1/4)",
                      "fd_pairs_s": t_data, "train_s": t_train * 1e-3,
                      "train_steps": args.surrogate_steps,
                      "train_models_per_s": args.surrogate_steps * B / (t_train * 1e-3),
                      "loss_log": log, "error_by_noise_level": levels,
                      "threshold": 0.05, "check_every": 10},
        "gpu_launches": None,
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)


def run_conv(args, rank, world, local_rank):
    """--conv: the tensor-core 3x3 convolution of a convolutional score model
    or surrogate layer on the 70x70 workload's batch: 152 images of 70 x 70,
    128 -> 128 channels, bf16 in and out, bias + SiLU.  Inputs (190 MB) and
    outputs (190 MB) exceed L2.  Reports the tensor roofline against the
    measured bf16 peak and, for context, cuDNN's convolution of the same
    layer through torch."""
    import torch
    from paper_2603_16393_gb300 import api
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    n = args.batch or WORKLOADS["70x70"]["batch"]
    h = w = 70
    c = args.conv_channels
    gen = torch.Generator(device=dev).manual_seed(11 + rank)
    x = torch.randn((n, h, w, c), device=dev, generator=gen).to(torch.bfloat16)
    wt = (torch.randn((c, 3, 3, c), device=dev, generator=gen) / (9 * c) ** 0.5).to(torch.bfloat16)
    bias = torch.randn(c, device=dev, generator=gen)
    y = torch.empty((n, h, w, c), device=dev, dtype=torch.bfloat16)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def launch():
        api.fwi_conv3x3_bf16(x, wt, bias, 1, y, status)

    def timed(fn, steps):
        torch.cuda.synchronize(dev)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(steps):
            fn()
        b.record(stream)
        torch.cuda.synchronize(dev)
        return a.elapsed_time(b) / steps

    for _ in range(args.warmup):
        launch()
    clocks = ClockSampler(local_rank) if rank == 0 else None
    if clocks:
        clocks.start()
    ms = timed(launch, args.steps)
    clk = clocks.stop() if clocks else None
    assert int(status.item()) == 0, "a device-side wait ran out"
    ms = max_over_ranks([ms], world, dev)[0]
    # cuDNN through torch on the same layer (NCHW view of channels-last data)
    xn = x.permute(0, 3, 1, 2)
    wn = wt.permute(0, 3, 1, 2).contiguous(memory_format=torch.channels_last)
    bb = bias.to(torch.bfloat16)

    def cudnn():
        torch.nn.functional.silu(torch.nn.functional.conv2d(xn, wn, bb, padding=1))

    for _ in range(args.warmup):
        cudnn()
    ms_cudnn = timed(cudnn, args.steps)
    if rank != 0:
        return
    flops = 2.0 * n * h * w * c * 9 * c
    byts = 2.0 * n * h * w * c * 2 + wt.numel() * 2
    tf = flops / (ms * 1e-3) / 1e12
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peak, src = float(json.load(f)["bf16_tflops"]), "measured"
    except Exception:
        peak, src = 1900.0, "fallback"
    line = {
        "metric": f"3x3 conv TFLOP/s ({n} x 70x70, {c}->{c} channels, bf16, bias + SiLU)",
        "value": world * tf, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16 (fp32 accumulate)", "data": "synthetic (seeded normal)",
        "config": {"workload": f"{n} x 70x70 x {c} -> {c}, 3x3, stride 1, zero padding",
                   "l2": f"inputs larger than L2 (x and y {n * h * w * c * 2 / 1e6:.0f} MB each)",
                   "tiles": ("192 pixels (8 x 24) as the MMA's N x 128 channels as its M per "
                             "tile; 6 % of the pixels fall outside the 70 x 70 images"
                             if c % 256 != 0 else
                             f"128 pixels (8 x 16) as the MMA's M x {256 if c % 256 == 0 else 64} "
                             "channels as its N per tile; 15 % of the pixels fall outside the "
                             "70 x 70 images") + "; one persistent CTA per SM; outside pixels "
                            "are not credited"},
        "roofline": {"bound": "tensor",
                     "kernel": ("k_conv3x3_tc<256>" if c % 256 == 0 else
                                "k_conv3x3_tc_pn"),
                     "achieved": tf,
                     "peak": peak, "unit": "TFLOP/s", "frac": tf / peak, "peak_source": src,
                     "hbm_gb_s": byts / (ms * 1e-3) / 1e9, "algorithmic_bytes": byts},
        "cudnn_ms": ms_cudnn, "speedup_vs_cudnn": ms_cudnn / ms,
        "gpu_launches": args.steps,
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)


def run_dsm_train(args, rank, world, local_rank):
    """--dsm-train: denoising-score-matching training steps (Eq. L2_rewrite) of
    the convolutional score model (3 layers, --conv-channels wide) on the
    70x70 workload's batch of 152 normalised models: x_t, the network, the
    loss, the parameter gradients and Adam, all in library kernels.  Reports
    training images/s and the FP32 roofline of the weight-gradient kernel,
    timed alone on the middle layer's operands."""
    import numpy as np
    import torch
    from paper_2603_16393_gb300 import api
    from paper_2603_16393_gb300 import score_net as SN
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    n = args.batch or WORKLOADS["70x70"]["batch"]
    h = w = 70
    c, L = args.conv_channels, 3
    betas = [float(b) for b in np.linspace(1e-4, 0.02, 1000)]
    unet = args.score == "unet"
    if unet:
        net = SN.UNetScore((n, h, w), betas, seed=5 + rank, device=dev)
    else:
        net = SN.ConvScore((n, h, w), betas, channels=c, layers=L, seed=5 + rank, device=dev)
    tr = SN.DSMTrainer(net, lr=1e-3)
    gen = torch.Generator(device=dev).manual_seed(13 + rank)
    x0 = 0.3 * torch.randn((n, h, w), device=dev, generator=gen)
    zs = [torch.randn((n, h, w), device=dev, generator=gen) for _ in range(4)]
    rng = np.random.default_rng(17 + rank)
    ts = [int(t) for t in rng.integers(1, 1001, args.warmup + args.steps)]
    stream = torch.cuda.current_stream(dev)
    for k in range(args.warmup):
        tr.step(x0, zs[k % 4], ts[k])
    torch.cuda.synchronize(dev)
    loss0 = float(tr.loss.item())
    clocks = ClockSampler(local_rank) if rank == 0 else None
    if clocks:
        clocks.start()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for k in range(args.steps):
        tr.step(x0, zs[k % 4], ts[args.warmup + k])
    b.record(stream)
    torch.cuda.synchronize(dev)
    clk = clocks.stop() if clocks else None
    ms = a.elapsed_time(b) / args.steps
    loss1 = float(tr.loss.item())
    ms = max_over_ranks([ms], world, dev)[0]
    if unet:
        if rank != 0:
            return
        def conv_flops(layers):
            f = 0.0
            for _, k, ci, co in layers:
                hh, ww = net.sizes[k]
                f += 2.0 * n * hh * ww * 9 * ci * co
            return f
        # executed: the layers as the kernels run them (a 32-channel level in
        # 64-channel blocks); logical: the network's own widths
        flops, flops_logical = conv_flops(net.layers), conv_flops(net.logical_layers)
        print(json.dumps({
            "metric": f"DSM training images/s ({n} x 70x70, 4-level U-Net {net.logical_widths})",
            "value": world * n * 1e3 / ms, "unit": "images/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16 activations, fp32 parameters, gradients and Adam",
            "data": "synthetic (seeded normal models, one seeded t per step)",
            "config": {"workload": f"{n} x 70x70, U-Net widths {net.logical_widths} (kernel "
                                   f"blocks {net.widths}), 15 conv layers, Adam",
                       "conv_tflop_per_step": 3 * flops / 1e12,
                       "conv_tflop_per_step_logical": 3 * flops_logical / 1e12},
            "loss": {"after_warmup": loss0, "last": loss1},
            "conv_tflops_per_s": 3 * flops / (ms * 1e-3) / 1e12,
            "clocks": clk}), flush=True)
        return
    # the weight gradient alone (layer 1: input A[0], output gradient dH), on
    # the tensor cores (staging + k_wgrad_tc + split reduction) and, for
    # context, on the CUDA cores
    X, dP, dW = net.A[0], net.dH[0], tr.grads[1][0]
    reps = max(args.steps, 3)

    def timed(fn):
        fn()
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize(dev)
        return a.elapsed_time(b) / reps

    tc = tr.stage is not None
    ms_tc = timed(lambda: api.fwi_conv3x3_wgrad_tc(X, dP, dW, tr.stage, tr.work)) if tc else None
    ms_cc = timed(lambda: api.fwi_conv3x3_wgrad(X, dP, dW, tr.work))
    ms_f = timed(lambda: api.fwi_conv3x3_bf16(X, net.W[1], net.bias[1][1], 0, net.P[0]))
    if rank != 0:
        return
    flops_w = 2.0 * n * h * w * 9 * c * c
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    if tc:
        splits = api.fwi_conv3x3_wgrad_tc_splits(n, h, w, c, c, tr.work.numel())
        try:
            with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
                peak, src = float(json.load(f)["bf16_tflops"]), "measured (bf16 burst)"
        except Exception:
            peak, src = 1900.0, "fallback"
        ach = flops_w / (ms_tc * 1e-3) / 1e12
        roof = {"bound": "tensor", "kernel": "fwi_conv3x3_wgrad_tc (4 x k_stage_kmajor + "
                                             "k_wgrad_tc + k_wgrad_tc_reduce)",
                "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                "peak_source": src, "splits": splits, "traffic": None}
        per_layer = 4 + 1 + (1 if splits > 1 else 0)
    else:
        splits = api.fwi_conv3x3_wgrad_splits(n, h, w, c, c, tr.work.numel())
        f_mhz = float((clk or {}).get("sm_max_mhz") or 2070.0)
        peak = sms * 128 * 2 * f_mhz * 1e6 / 1e12        # FP32 FMA: 128 lanes per SM
        ach = flops_w / (ms_cc * 1e-3) / 1e12
        roof = {"bound": "alu", "kernel": "k_wgrad", "achieved": ach, "peak": peak,
                "unit": "TFLOP/s", "frac": ach / peak,
                "peak_source": f"{sms} SMs x 128 FP32 lanes x 2 flops x {f_mhz:.0f} MHz",
                "splits": splits, "traffic": None}
        per_layer = 1 + (1 if splits > 1 else 0)
    # x_t; forward; loss (+ ordered sum); per layer the weight gradient, the
    # channel sum (+ ordered sum) and dE, the data gradients; Adam; refresh
    launches = 1 + (2 + L + (L - 1)) + 2 + (1 + (per_layer + 3) * L + 2 * (L - 1)) + 1 + 2 * L
    line = {
        "metric": f"DSM training images/s ({n} x 70x70, {L} conv layers x {c} channels)",
        "value": world * n * 1e3 / ms, "unit": "images/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16 activations, fp32 parameters, gradients and Adam",
        "data": "synthetic (seeded normal models, one seeded t per step)",
        "config": {"workload": f"{n} x 70x70, {L} x conv3x3 {c} -> {c} + SiLU, Adam",
                   "l2": f"activations larger than L2 ({n * h * w * c * 2 / 1e6:.0f} MB each)"},
        "loss": {"after_warmup": loss0, "last": loss1},
        "kernels_ms": {"weight gradient, tensor cores (one layer)": ms_tc,
                       "weight gradient, CUDA cores (one layer)": ms_cc,
                       "conv forward (one layer)": ms_f},
        "roofline": roof,
        "gpu_launches": launches * args.steps,
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--batch", type=int, default=0, help="models per GPU (0: workload default)")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="70x70")
    ap.add_argument("--nt", type=int, default=0,
                    help="time steps (0: the workload's); shorter runs size profiler captures")
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--absorber", choices=["sponge", "cpml"], default="sponge",
                    help="absorbing layer: the damping sponge (default) or the CPML variant")
    ap.add_argument("--mixed", action="store_true",
                    help="the batched uneven workload (64 x 70x70 + 8 x 256x256 + 2 x 512x1024) "
                         "as one graph-captured plan group")
    ap.add_argument("--conv", action="store_true",
                    help="the tensor-core 3x3 convolution of a score-model layer "
                         "(152 x 70x70, 128 -> 128 channels, bf16)")
    ap.add_argument("--score", choices=["prior", "conv", "unet"], default="prior",
                    help="--sampler: the score model (Gaussian prior, a convolutional network "
                         "or the 4-level U-Net); --dsm-train: conv or unet")
    ap.add_argument("--surrogate-fraction", type=float, default=0.0,
                    help="--sampler: low-fidelity guidance (2x coarser grid and time step) in "
                         "this fraction of the first reverse steps")
    ap.add_argument("--surrogate", choices=["lowfi", "net"], default="lowfi",
                    help="--sampler with --surrogate-fraction: the physics-based low-fidelity "
                         "surrogate or a convolutional network surrogate of dJ/dv")
    ap.add_argument("--conv-channels", type=int, default=128,
                    help="--conv: input and output channels (a multiple of 64)")
    ap.add_argument("--dsm-train", action="store_true",
                    help="denoising-score-matching training steps of the convolutional score "
                         "model (152 x 70x70, 3 layers of --conv-channels)")
    ap.add_argument("--uneven", action="store_true",
                    help="uneven resident instances: per-plan gradients, a plan group, and one "
                         "persistent launch per direction (api.Queue)")
    ap.add_argument("--posterior", action="store_true",
                    help="posterior sampling by Algorithm 2 on 10 dB observations: batched "
                         "graph-replayed chains with all-FD and with gated surrogate guidance "
                         "against one eager plan per sample")
    ap.add_argument("--observations", type=int, default=4, help="--posterior: observations")
    ap.add_argument("--prior", choices=["diag", "lowrank"], default="diag",
                    help="--posterior: the Gaussian prior (diagonal, or 32 principal directions)")
    ap.add_argument("--samples", type=int, default=32,
                    help="--posterior: posterior samples per observation")
    ap.add_argument("--reverse-steps", type=int, default=500, help="--posterior: reverse steps")
    ap.add_argument("--plain-steps", type=int, default=2,
                    help="--posterior: reverse steps timed on the plain path")
    ap.add_argument("--surrogate-models", type=int, default=20480,
                    help="--posterior: FD pairs the surrogate trains on")
    ap.add_argument("--surrogate-steps", type=int, default=6000,
                    help="--posterior: Adam steps of the surrogate's training")
    ap.add_argument("--sampler", action="store_true",
                    help="reverse steps of Algorithm 2 (score, proposal, W2 guidance gradient, "
                         "chain rule, preconditioned update) on the 70x70 workload")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1 and args.impl == "ours":
        import torch.distributed as dist
        dist.init_process_group("nccl")
    try:
        if args.impl == "reference":
            run_reference(args, rank, world)
        elif args.mixed:
            run_mixed(args, rank, world, local_rank)
        elif args.sampler:
            run_sampler(args, rank, world, local_rank)
        elif args.posterior:
            run_posterior(args, rank, world, local_rank)
        elif args.uneven:
            run_uneven(args, rank, world, local_rank)
        elif args.conv:
            run_conv(args, rank, world, local_rank)
        elif args.dsm_train:
            run_dsm_train(args, rank, world, local_rank)
        else:
            run_ours(args, rank, world, local_rank)
    finally:
        if world > 1 and args.impl == "ours":
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
