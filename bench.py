"""Throughput of the column-microphysics step on GB300.

Default workload: deep convection, 512x512 columns x 150 stretched levels
(39.3 M grid points), dt = 1 s, mixed FP32/FP64 form; the plain FP64 form is
timed on the same workload for the mixed-vs-FP64 comparison.  One bench step
is one model timestep over the whole domain (one launch of the step kernel),
with the state resident in HBM.  The state (5 GB) is far larger than L2, so
no flush is needed between steps.

Prints one JSON line.  `--impl reference` times the FP64 CPU oracle on a
bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "grid-point updates/s: mixed-precision vs plain FP64, same GB300, at stated error"
UNIT = "grid-point updates/s"
WORKLOAD = "deep_512x512x150"


# DRAM traffic of k_step<PolicyMix> on the deep-convection state, from one
# single-pass ncu capture of the full 262 144-column x 150-level launch
# (dram__bytes_read.sum + dram__bytes_write.sum = 5.0588 + 3.9828 GB for
# 39.32 M points); at another column count it is scaled per point (reads are
# 16 fields per point and writes follow the changed points).  Valid only for
# the kernel source it was taken on.
MEASURED_TRAFFIC = {"kernel": "k_step<PolicyMix>", "bytes_per_launch": 9041585152, "points": 39321600,
                    "bytes_per_point": 229.94,
                    "source": "paper_2010_14823_gb300/csrc/casim_device.cuh",
                    "sha256": "b040dec6cc7b6d47b6f675add1fcc1f4f5979e38b72bbe9ddb8b957d05c32d1c"}


# FP64 arithmetic instructions of k_step<PolicyF64> per point on the same
# state, from one ncu capture of a 16 384-column x 150-level launch
# (smsp__sass_thread_inst_executed_op_{dfma,dadd,dmul}_pred_on.sum =
# 1168.3 M + 296.4 M + 381.0 M for 2.458 M points); the FP64 pipe was 72.9 %
# busy.  Valid only for the kernel source it was taken on.
MEASURED_FP64_OPS = {"kernel": "k_step<PolicyF64>", "inst_per_point": 751.07,
                     "dfma": 475.40, "dadd": 120.63, "dmul": 155.04, "fp64_pipe_active": 0.729,
                     "sha256": "b040dec6cc7b6d47b6f675add1fcc1f4f5979e38b72bbe9ddb8b957d05c32d1c"}


def _host_link_gbs(torch, stream, nbytes: int = 1 << 30):
    """The host link as this run sees it: 1 GB pinned <-> device copies timed with CUDA
    events (one warm-up each), host to device alone, device to host alone, and both at
    once on two streams (GB/s counting both directions).  The host memory and link of
    the box may be shared with other jobs, so the end-to-end rate is read against this."""
    n = nbytes // 8
    h_in = torch.ones(n, dtype=torch.float64).pin_memory()
    h_out = torch.empty(n, dtype=torch.float64).pin_memory()
    d_a = torch.empty(n, dtype=torch.float64, device="cuda")
    d_b = torch.zeros(n, dtype=torch.float64, device="cuda")
    s2 = torch.cuda.Stream()

    def timed(fn, nb):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return nb / (e0.elapsed_time(e1) * 1e-3) / 1e9

    def both():
        start = torch.cuda.Event()
        start.record(stream)
        s2.wait_event(start)
        with torch.cuda.stream(s2):
            h_out.copy_(d_b, non_blocking=True)
        d_a.copy_(h_in, non_blocking=True)
        done = torch.cuda.Event()
        done.record(s2)
        stream.wait_event(done)

    with torch.cuda.stream(stream):
        r = {"h2d": timed(lambda: d_a.copy_(h_in, non_blocking=True), nbytes),
             "d2h": timed(lambda: h_out.copy_(d_b, non_blocking=True), nbytes),
             "both": timed(both, 2 * nbytes)}
    del h_in, h_out, d_a, d_b
    return r


def _kernel_source_sha() -> str:
    import hashlib
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), MEASURED_TRAFFIC["source"])
    with open(path, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()


def _measured_traffic(npts: int):
    """Traffic per launch scaled from the capture, or None if the kernel source changed since."""
    if _kernel_source_sha() != MEASURED_TRAFFIC["sha256"]:
        return None
    if npts == MEASURED_TRAFFIC["points"]:
        return float(MEASURED_TRAFFIC["bytes_per_launch"])
    return MEASURED_TRAFFIC["bytes_per_point"] * npts


def _fp64_roofline(npts: int, fp_ms: float):
    """The FP64 form against the FP64 pipe: counted FP64 arithmetic
    instructions per second over the DFMA rate measured now (probe of
    include/casim_peaks.h); None if the kernel source changed since the count."""
    if _kernel_source_sha() != MEASURED_FP64_OPS["sha256"]:
        return None
    from paper_2010_14823_gb300 import peaks
    peak = peaks.peak_rate("dfma", 1 << 12)
    achieved = MEASURED_FP64_OPS["inst_per_point"] * npts / (fp_ms * 1e-3)
    return {"bound": "fp64", "achieved": achieved, "peak": peak, "unit": "FP64 instructions/s",
            "frac": achieved / peak, "kernel": "k_step<PolicyF64>",
            "inst_per_point": MEASURED_FP64_OPS["inst_per_point"],
            "fp64_pipe_active_ncu": MEASURED_FP64_OPS["fp64_pipe_active"],
            "peak_source": "measured now: DFMA chains on every SM (casim_peak_rate)"}


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_oracle_rate(recipe_fld, dz, ncols_total, dt, target_s=10.0, max_cols=None, nthreads=None):
    """Time the FP64 oracle (as it stands) on host cores (all, or nthreads)
    over a bounded sample of columns of the same workload; returns (points/s,
    threads, sample text, seconds)."""
    import oracle
    nthreads = nthreads or os.cpu_count() or 1
    fld, nlev = recipe_fld, recipe_fld.shape[1]
    cols = 256
    while True:
        cols = min(cols, ncols_total if max_cols is None else min(ncols_total, max_cols))
        sub = np.ascontiguousarray(fld[:, :, :cols])
        pitch = cols
        if pitch % 32:
            pad = np.zeros((16, nlev, (pitch + 31) // 32 * 32))
            pad[:, :, :cols] = sub
            sub = pad
        t0 = time.perf_counter()
        oracle.step(sub, cols, dz, dt, nthreads=nthreads)
        el = time.perf_counter() - t0
        if el >= target_s * 0.5 or cols >= ncols_total or (max_cols and cols >= max_cols):
            return cols * nlev / el, nthreads, f"{cols} columns x {nlev} levels, 1 step, {el:.3f} s", el
        cols = int(cols * min(16.0, max(2.0, target_s / max(el, 1e-3))))


def bench_batch(args, rank, world, local):
    """64 uneven domains (column counts log-uniform 1k-100k, 40-150 levels,
    cloud fraction 5-60 %), mixed form, one persistent launch per step over the
    active-column list, configuration picked by the autotuner, steps replayed
    from a CUDA graph of 10 steps."""
    import torch
    from paper_2010_14823_gb300 import casim, synth
    casim.lib()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2010_14823_gb300 import shard
    doms, dt = synth.batch_workload(64, seed=shard.rank_seed(1237, rank), scale=args.batch_scale)
    dev = [casim.Domain(f, dz, nc) for f, dz, nc, nl in doms]
    del doms
    npts = sum(d.ncols * d.nlev for d in dev)
    stream = torch.cuda.current_stream()

    def sync():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    ctx = casim.casim_init(precision=casim.CASIM_MIXED)
    b = casim.casim_batch_create(ctx, [d.state for d in dev], [d.ncols for d in dev], [d.nlev for d in dev])
    table = casim.casim_batch_tune(ctx, b, dt, steps=2, stream=stream)
    cfg = casim.casim_batch_get_config(b)
    g = 10
    casim.casim_batch_graph(ctx, b, dt, g, stream)
    for _ in range(max(1, args.warmup // g)):
        casim.casim_batch_graph_launch(b, stream)
    nrep = max(1, args.steps // g)
    sync()
    n0 = casim.casim_launch_count(ctx)
    sampler = ClockSampler(local)
    sampler.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(nrep):
        casim.casim_batch_graph_launch(b, stream)
    e1.record(stream)
    sync()
    clocks = sampler.stop()
    ms = shard.max_over_ranks(e0.elapsed_time(e1), dist, "cuda")
    launches = casim.casim_launch_count(ctx) - n0
    rc, fl = casim.casim_get_error(ctx, stream)
    assert rc == 0, (rc, fl)
    steps = nrep * g
    value = world * npts * steps / (ms * 1e-3)
    # the same batch stepped eagerly, one launch pair per step, and the FP64 form
    e0.record(stream)
    for _ in range(g):
        casim.casim_batch_step(ctx, b, dt, stream)
    e1.record(stream)
    sync()
    eager_ms = e0.elapsed_time(e1) / g
    casim.casim_batch_free(b)
    casim.casim_free(ctx)
    ctx64 = casim.casim_init(precision=casim.CASIM_FP64)
    b64 = casim.casim_batch_create(ctx64, [d.state for d in dev], [d.ncols for d in dev], [d.nlev for d in dev])
    casim.casim_batch_step(ctx64, b64, dt, stream)
    sync()
    e0.record(stream)
    casim.casim_batch_step(ctx64, b64, dt, stream)
    e1.record(stream)
    sync()
    fp64_ms = e0.elapsed_time(e1)
    casim.casim_batch_free(b64)
    casim.casim_free(ctx64)
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": steps,
                "warmup": args.warmup, "ms_per_step": ms / steps, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
                "config": {"workload": "batch64", "domains": 64, "grid_points": npts,
                           "columns": int(sum(d.ncols for d in dev)),
                           "form": "mixed, batched persistent launch, CUDA graph of 10 steps",
                           "tuned": {"block": cfg[0], "compact": cfg[1], "persistent": cfg[2]},
                           "tune_table": table, "eager_ms_per_step": eager_ms,
                           "fp64_ms_per_step": fp64_ms, "fp64_value": world * npts / (fp64_ms * 1e-3),
                           "l2": "state %.1f GB > L2, no flush needed" % (16 * 8 * sum(d.nlev * d.pitch for d in dev) / 1e9)},
                "roofline": None, "cpu_baseline": None, "e2e": None,
                "gpu_launches": launches, "clocks": clocks}
        if getattr(args, "emit", True):
            print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return line if rank == 0 else None


def bench_surrogate(args, rank, world, local):
    """The surrogate workload on its own line (see surrogate_run)."""
    line = surrogate_run(args, rank, world, local)
    if rank == 0:
        print(json.dumps(line), flush=True)


def surrogate_run(args, rank, world, local):
    """Learned warm-rain rates on deep convection 512x512x150: training data
    from mixed-form runs (the scheme's own rates), training on the GPU,
    inference through the guarded surrogate step of a batch holding the
    domain (one feature pass, one network launch, one step launch, no host
    synchronisation); errors judged by the plain mixed step (rates on
    held-out points, 100-step surface precipitation).  Returns the line."""
    import torch
    from paper_2010_14823_gb300 import casim, shard, synth
    casim.lib()
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    fld, dz, ncols, nlev, dt, _ = synth.workload("deep_512x512x150", ncols=args.ncols, seed=shard.rank_seed(1240, rank))
    npts = ncols * nlev
    ctx = casim.casim_init(precision=casim.CASIM_MIXED)
    m = casim.casim_mlp_create(seed=5)
    dom = casim.Domain(fld, dz, ncols)
    # training data: 10 M rows sampled evenly from the warm points of 10
    # successive mixed-form states (1 M per state)
    gen_steps = args.gen_steps
    cap = min(10_000_000, gen_steps * npts)
    per = cap // gen_steps
    X = torch.zeros((cap, 12), dtype=torch.float32, device="cuda")
    Y = torch.zeros((cap, 4), dtype=torch.float32, device="cuda")
    M = torch.zeros((cap, 4), dtype=torch.float32, device="cuda")
    Xs = torch.zeros((npts, 12), dtype=torch.float32, device="cuda")
    Ys = torch.zeros((npts, 4), dtype=torch.float32, device="cuda")
    Ms = torch.zeros((npts, 4), dtype=torch.float32, device="cuda")
    have = 0
    gen = torch.Generator(device="cuda")
    gen.manual_seed(17)
    for _ in range(gen_steps):
        rows = casim.casim_mlp_data(ctx, dom.state, ncols, nlev, dt, Xs, Ys, Ms, npts, stream=stream)
        take = min(per, rows)
        idx = torch.randperm(rows, device="cuda", generator=gen)[:take]
        X[have:have + take], Y[have:have + take], M[have:have + take] = Xs[idx], Ys[idx], Ms[idx]
        have += take
        casim.casim_step(ctx, dom.state, ncols, nlev, dt, stream)
    del Xs, Ys, Ms
    # held-out rows from the state after the training window
    Xh = torch.zeros((npts, 12), dtype=torch.float32, device="cuda")
    Yh = torch.zeros((npts, 4), dtype=torch.float32, device="cuda")
    Mh = torch.zeros((npts, 4), dtype=torch.float32, device="cuda")
    hold = casim.casim_mlp_data(ctx, dom.state, ncols, nlev, dt, Xh, Yh, Mh, npts, stream=stream)
    train_steps, batch = args.train_steps, 8192
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hist = casim.casim_mlp_fit(m, X, Y, M, have, train_steps, batch, 1e-3, seed=3, stream=stream, history=False)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    del hist
    stats = casim.casim_mlp_get_norm(m)
    # rate error on held-out points inside the box (linear space, relative)
    sel = np.random.default_rng(0).choice(hold, min(hold, 200_000), replace=False)
    xs, ys, ms = Xh[sel].cpu().numpy(), Yh[sel].cpu().numpy(), Mh[sel].cpu().numpy()
    lo, hi = stats[32:44], stats[44:56]
    inbox = np.all((xs >= lo) & (xs <= hi), axis=1)
    xn = (xs - stats[0:12]) / stats[12:24]
    yp = casim.casim_mlp_forward_host(m, xn.astype(np.float32)) * stats[28:32] + stats[24:28]
    rel = np.abs(np.expm1(yp - ys)) * ms
    rate_err = {}
    for j, name in enumerate(("aut", "acc", "scc", "scr")):
        v = rel[inbox & (ms[:, j] > 0), j]
        rate_err[name] = {"median": float(np.median(v)), "p99": float(np.percentile(v, 99)), "n": int(v.size)}
    # the network alone, through casim_mlp_forward on device rows: 8 M
    # standard-normal standardised inputs (the cost does not depend on the
    # values), 2 warm-up calls, 5 timed; includes the FP32 -> BF16 input pass
    nnet = 8_000_000
    gnet = torch.Generator(device="cuda").manual_seed(1240)
    Xnet = torch.randn((nnet, 12), generator=gnet, device="cuda", dtype=torch.float32)
    Ynet = torch.empty((nnet, 4), device="cuda", dtype=torch.float32)
    for _ in range(2):
        casim.casim_mlp_forward(m, Xnet, Ynet, stream)
    n0 = torch.cuda.Event(enable_timing=True)
    n1 = torch.cuda.Event(enable_timing=True)
    n0.record(stream)
    for _ in range(5):
        casim.casim_mlp_forward(m, Xnet, Ynet, stream)
    n1.record(stream)
    torch.cuda.synchronize()
    net_ms = n0.elapsed_time(n1) / 5
    del Xnet, Ynet
    net_flop = 270336.0 * nnet
    net_tflops = net_flop / (net_ms * 1e-3) / 1e12
    bf16_peak = _peaks().get("bf16_tflops")
    # 100 steps: plain mixed vs surrogate from the same start, surface precipitation judged by the plain run
    nsteps = args.surr_steps
    plain, surr = casim.Domain(fld, dz, ncols), casim.Domain(fld, dz, ncols)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(nsteps):
        casim.casim_step(ctx, plain.state, ncols, nlev, dt, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    plain_ms = e0.elapsed_time(e1) / nsteps
    # the batched surrogate step: warm-up step (counts the served points), then timed steps
    b = casim.casim_batch_create(ctx, [surr.state], [ncols], [nlev])
    served = casim.casim_batch_step_surrogate(ctx, b, m, dt, stream, want_served=True)
    n0 = casim.casim_launch_count(ctx)
    sampler = ClockSampler(local)
    sampler.start()
    e0.record(stream)
    for _ in range(nsteps - 1):
        casim.casim_batch_step_surrogate(ctx, b, m, dt, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    launches = casim.casim_launch_count(ctx) - n0
    surr_ms = e0.elapsed_time(e1) / max(1, nsteps - 1)
    casim.casim_batch_free(b)
    rc, fl = casim.casim_get_error(ctx, stream)
    assert rc == 0, (rc, fl)
    pp, ps = plain.precip[:, :ncols].sum(0).cpu().numpy(), surr.precip[:, :ncols].sum(0).cpu().numpy()
    tot_p, tot_s = float(pp.sum()), float(ps.sum())
    wet = pp > 1e-6 * max(pp.max(), 1e-30)
    col_rel = np.abs(ps[wet] - pp[wet]) / pp[wet]
    casim.casim_mlp_free(m)
    casim.casim_free(ctx)
    value = world * npts / (surr_ms * 1e-3)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": nsteps - 1, "warmup": 1,
                "ms_per_step": surr_ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "bf16 network + f32/f64 step", "data": "synthetic",
                "config": {"workload": "surrogate_deep_512x512x150", "train_rows": have, "gen_steps": gen_steps,
                           "train_steps": train_steps, "batch": batch, "train_s": train_s,
                           "path": "casim_batch_step_surrogate: feature pass, network, step; no host sync",
                           "rate_rel_error_heldout": rate_err, "heldout_inbox_frac": float(inbox.mean()),
                           "served_points_per_step": served, "plain_ms_per_step": plain_ms,
                           "surrogate_ms_per_step": surr_ms, "precip_total_rel_error": abs(tot_s - tot_p) / tot_p,
                           "precip_column_rel_error": {"median": float(np.median(col_rel)),
                                                       "p99": float(np.percentile(col_rel, 99))}},
                "roofline": {"bound": "tensor", "achieved": net_tflops, "peak": bf16_peak, "unit": "TFLOP/s",
                             "frac": net_tflops / bf16_peak if bf16_peak else None, "traffic": None,
                             "kernel": "k_mlp_umma (network alone via casim_mlp_forward, 8 M rows, with its "
                                       "FP32 -> BF16 input pass)",
                             "algorithmic_flop_per_launch": net_flop, "ms_per_launch": net_ms,
                             "peak_source": "MEASURED_PEAKS.json bf16_tflops (burst cuBLAS GEMM)"},
                "cpu_baseline": None, "e2e": None, "gpu_launches": launches, "clocks": clocks}
    return line


def bench_peaks(args, rank, world, local):
    """Instruction-throughput probes of this GPU (include/casim_peaks.h): FP32
    and FP64 fused multiply-adds and the special-function unit's ex2, lg2, rcp
    and tanh, each over 8 independent chains per thread on every SM; rates
    per second and per SM per clock (at the median SM clock sampled during
    the probes)."""
    import torch
    from paper_2010_14823_gb300 import peaks
    torch.cuda.set_device(local)
    iters = {"ffma": 1 << 18, "dfma": 1 << 12, "ex2": 1 << 16, "lg2": 1 << 15, "rcp": 1 << 15, "tanh": 1 << 15,
             "tanh_bf16x2": 1 << 15}
    nsm = torch.cuda.get_device_properties(local).multi_processor_count
    sampler = ClockSampler(local)
    sampler.start()
    rates = {k: peaks.peak_rate(k, n) for k, n in iters.items()}
    clocks = sampler.stop()
    mhz = clocks.get("sm_mhz") if isinstance(clocks, dict) else None
    per = {k: (v / (nsm * mhz * 1e6) if mhz else None) for k, v in rates.items()}
    if rank == 0:
        print(json.dumps({"workload": "peaks", "unit": "operations/s (one FMA = one operation)", "sms": nsm,
                          "rates": rates, "per_sm_per_clock": per, "iters": iters, "clocks": clocks}), flush=True)


def bench_tendency(args, rank, world, local):
    """The source-term mode on deep convection 512x512x150: the state is left
    unchanged and (x_after - x_before) / dt of the 13 prognostic fields goes to
    a separate array at every point, the parent model's interface.  `value` is
    the mixed form; the roofline counts 16 fields read and 13 source terms
    written per point (every point's, zero where nothing changes)."""
    import torch
    from paper_2010_14823_gb300 import casim, synth, shard
    casim.lib()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    fld, dz, ncols, nlev, dt, _ = synth.workload(WORKLOAD, ncols=args.ncols, seed=shard.rank_seed(1236, rank))
    npts = ncols * nlev
    stream = torch.cuda.current_stream()
    dom = casim.Domain(fld, dz, ncols)
    tend = torch.empty((13, nlev, dom.pitch), dtype=torch.float64, device=dom.fld.device)

    def sync():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def run(precision, steps, warmup):
        ctx = casim.casim_init(precision=precision)
        for _ in range(warmup):
            casim.casim_step_tendency(ctx, dom.state, ncols, nlev, dt, tend, stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        sync()
        n0 = casim.casim_launch_count(ctx)
        e0.record(stream)
        for _ in range(steps):
            casim.casim_step_tendency(ctx, dom.state, ncols, nlev, dt, tend, stream)
        e1.record(stream)
        sync()
        rc, fl = casim.casim_get_error(ctx, stream)
        assert rc == 0, (rc, fl)
        launches = casim.casim_launch_count(ctx) - n0
        casim.casim_free(ctx)
        return shard.max_over_ranks(e0.elapsed_time(e1), dist, "cuda") / steps, launches

    sampler = ClockSampler(local)
    sampler.start()
    mix_ms, launches = run(casim.CASIM_MIXED, args.steps, args.warmup)
    clocks = sampler.stop()
    fp_ms, _ = run(casim.CASIM_FP64, args.fp64_steps, 1)
    peak = _peaks().get("hbm_gbs")
    alg = (128.0 + 104.0) * npts
    achieved = alg / (mix_ms * 1e-3) / 1e9
    if rank == 0:
        v = lambda ms: world * npts / (ms * 1e-3)
        line = {"metric": METRIC, "value": v(mix_ms), "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": mix_ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
                "config": {"workload": WORKLOAD + " source-term mode", "ncols": ncols, "nlev": nlev, "dt_s": dt,
                           "path": "casim_step_tendency: state unchanged, 13 source-term rows written",
                           "l2": "state 5 GB and source terms 4 GB > L2, no flush needed",
                           "fp64_value": v(fp_ms), "fp64_ms_per_step": fp_ms},
                "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                             "frac": achieved / peak if peak else None, "traffic": None,
                             "kernel": "k_step<PolicyMix, tendency>", "algorithmic_bytes_per_launch": alg,
                             "peak_source": "MEASURED_PEAKS.json hbm_gbs (burst copy)"},
                "cpu_baseline": None, "e2e": None, "gpu_launches": launches, "clocks": clocks}
        if getattr(args, "emit", True):
            print(json.dumps(line), flush=True)
    return line if rank == 0 else None


def bench_warm(args, rank, world, local):
    """The warm configuration (liquid water only) against the cold one on the
    same 512x512x150 stratus state, mixed and FP64 forms.  `value` is the warm
    mixed step; the roofline is the warm kernel's (10 fields read, 7 written
    where the step changes a point)."""
    import torch
    from paper_2010_14823_gb300 import casim, synth, shard
    casim.lib()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    name = "stratus_512x512x150"
    fld, dz, ncols, nlev, dt, _ = synth.workload(name, ncols=args.ncols, seed=shard.rank_seed(1238, rank))
    npts = ncols * nlev
    stream = torch.cuda.current_stream()
    dom = casim.Domain(fld, dz, ncols)
    fld0 = dom.fld.clone()

    def sync():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def run(precision, flags, steps, warmup):
        ctx = casim.casim_init(precision=precision, flags=flags)
        dom.fld.copy_(fld0)
        dom.precip.zero_()
        for _ in range(warmup):
            casim.casim_step(ctx, dom.state, ncols, nlev, dt, stream)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        sync()
        n0 = casim.casim_launch_count(ctx)
        for i in range(steps):
            evs[i][0].record(stream)
            casim.casim_step(ctx, dom.state, ncols, nlev, dt, stream)
            evs[i][1].record(stream)
        sync()
        rc, fl = casim.casim_get_error(ctx, stream)
        assert rc == 0, (rc, fl)
        launches = casim.casim_launch_count(ctx) - n0
        casim.casim_free(ctx)
        total = evs[0][0].elapsed_time(evs[-1][1])
        per = float(np.mean([a.elapsed_time(b) for a, b in evs]))
        return shard.max_over_ranks(total, dist, "cuda") / steps, per, launches

    # points the warm step changes (for the algorithmic bytes)
    ctx = casim.casim_init(precision=casim.CASIM_MIXED, flags=casim.CASIM_WARM)
    before = dom.fld[:13].clone()
    casim.casim_step(ctx, dom.state, ncols, nlev, dt, stream)
    torch.cuda.synchronize()
    changed = int((dom.fld[:13] != before).any(dim=0)[:, :ncols].sum().item())
    del before
    casim.casim_free(ctx)
    sampler = ClockSampler(local)
    sampler.start()
    warm_ms, warm_per, launches = run(casim.CASIM_MIXED, casim.CASIM_WARM, args.steps, args.warmup)
    clocks = sampler.stop()
    cold_ms, _, _ = run(casim.CASIM_MIXED, 0, args.steps, args.warmup)
    w64_ms, _, _ = run(casim.CASIM_FP64, casim.CASIM_WARM, args.fp64_steps, 1)
    c64_ms, _, _ = run(casim.CASIM_FP64, 0, args.fp64_steps, 1)
    # the warm step with activated-aerosol mass: 19 fields (free aerosol
    # ~100 cm^-3 of 0.05 um particles; aerosol in cloud and rain at 1e-5 of
    # their water)
    aero = torch.zeros((19, nlev, dom.pitch), dtype=torch.float64, device=dom.fld.device)
    aero[:16] = fld0
    aero[16] = 3e-9
    aero[17] = 1e-5 * fld0[2]
    aero[18] = 1e-5 * fld0[3]

    def time_ext(ext, flags):
        d = casim.Domain(ext, dz, ncols)
        ctx = casim.casim_init(precision=casim.CASIM_MIXED, flags=flags)
        for _ in range(args.warmup):
            casim.casim_step(ctx, d.state, ncols, nlev, dt, stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        sync()
        e0.record(stream)
        for _ in range(args.steps):
            casim.casim_step(ctx, d.state, ncols, nlev, dt, stream)
        e1.record(stream)
        sync()
        rc, fl = casim.casim_get_error(ctx, stream)
        assert rc == 0, (rc, fl)
        casim.casim_free(ctx)
        return e0.elapsed_time(e1) / args.steps

    aero_ms = time_ext(aero, casim.CASIM_WARM | casim.CASIM_AEROSOL)
    del aero
    # the cold chain with aerosol mass also in ice, snow and graupel (22
    # fields, each at 1e-5 of its species' water)
    aero = torch.zeros((22, nlev, dom.pitch), dtype=torch.float64, device=dom.fld.device)
    aero[:16] = fld0
    aero[16] = 3e-9
    for f, q in ((17, 2), (18, 3), (19, 4), (20, 5), (21, 6)):
        aero[f] = 1e-5 * fld0[q]
    aero_cold_ms = time_ext(aero, casim.CASIM_AEROSOL)
    del aero
    # triple-moment rain: 17 fields, the rain's sixth moment that of a gamma
    # distribution of shape uniform in [0, 8] at every rainy point
    tri = torch.zeros((17, nlev, dom.pitch), dtype=torch.float64, device=dom.fld.device)
    tri[:16] = fld0
    g = torch.Generator(device=dom.fld.device).manual_seed(1239)
    mu = 8.0 * torch.rand((nlev, dom.pitch), generator=g, dtype=torch.float64, device=dom.fld.device)
    gmu = (mu + 4) * (mu + 5) * (mu + 6) / ((mu + 1) * (mu + 2) * (mu + 3))
    qr, nr = fld0[3], fld0[8]
    rainy = (qr > 1e-14) & (nr > 0)
    tri[16] = torch.where(rainy, gmu * (qr / casim.casim_default_params().a[1]) ** 2 / nr.clamp_min(1e-300), 0.0)
    del mu, gmu, rainy
    tri_ms = time_ext(tri, casim.CASIM_WARM | casim.CASIM_THREE_MOMENT)
    del tri
    # the cold chain with triple-moment r, i, s, g: 20 fields, every species'
    # sixth moment that of a gamma distribution of shape uniform in [0, 8]
    tri = torch.zeros((20, nlev, dom.pitch), dtype=torch.float64, device=dom.fld.device)
    tri[:16] = fld0
    a_sp = casim.casim_default_params().a
    for x, (qf, nf) in enumerate(((3, 8), (4, 9), (5, 10), (6, 11))):
        mu = 8.0 * torch.rand((nlev, dom.pitch), generator=g, dtype=torch.float64, device=dom.fld.device)
        gmu = (mu + 4) * (mu + 5) * (mu + 6) / ((mu + 1) * (mu + 2) * (mu + 3))
        q, n = fld0[qf], fld0[nf]
        has = (q > 1e-14) & (n > 0)
        tri[16 + x] = torch.where(has, gmu * (q / a_sp[1 + x]) ** 2 / n.clamp_min(1e-300), 0.0)
        del mu, gmu, has
    tri_cold_ms = time_ext(tri, casim.CASIM_THREE_MOMENT)
    del tri
    peak = _peaks().get("hbm_gbs")
    alg = 80.0 * npts + 56.0 * changed
    achieved = alg / (warm_per * 1e-3) / 1e9
    if rank == 0:
        v = lambda ms: world * npts / (ms * 1e-3)
        line = {"metric": METRIC, "value": v(warm_ms), "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": warm_ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
                "config": {"workload": name + " warm configuration", "ncols": ncols, "nlev": nlev, "dt_s": dt,
                           "form": "mixed, warm configuration (liquid water only: 10 fields read, 7 written)",
                           "l2": "state 5 GB > L2, no flush needed",
                           "cold_mixed_value": v(cold_ms), "cold_mixed_ms_per_step": cold_ms,
                           "warm_over_cold": cold_ms / warm_ms,
                           "warm_fp64_value": v(w64_ms), "cold_fp64_value": v(c64_ms),
                           "warm_aerosol_mixed_value": v(aero_ms), "warm_aerosol_mixed_ms_per_step": aero_ms,
                           "cold_aerosol_mixed_value": v(aero_cold_ms),
                           "cold_aerosol_mixed_ms_per_step": aero_cold_ms,
                           "warm_three_moment_mixed_value": v(tri_ms),
                           "warm_three_moment_mixed_ms_per_step": tri_ms,
                           "cold_three_moment_mixed_value": v(tri_cold_ms),
                           "cold_three_moment_mixed_ms_per_step": tri_cold_ms,
                           "changed_points_frac": changed / npts},
                "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                             "frac": achieved / peak if peak else None, "traffic": None,
                             "kernel": "k_step<PolicyMixWarm>", "algorithmic_bytes_per_launch": alg,
                             "peak_source": "MEASURED_PEAKS.json hbm_gbs (burst copy)"},
                "cpu_baseline": None, "e2e": None, "gpu_launches": launches, "clocks": clocks}
        if getattr(args, "emit", True):
            print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return line if rank == 0 else None


FIELD_NAMES = ("T", "qv", "qc", "qr", "qi", "qs", "qg", "nc", "nr", "ni", "ns", "ng", "na")


def _compare(torch, a, b, x0, pa, pb):
    """Per-field differences of the mixed state a against the FP64 state b
    (both [13][nlev][ncols] on the device), x0 the common starting state."""
    out = {"fields": {}}
    for f, name in enumerate(FIELD_NAMES):
        diff = (a[f] - b[f]).abs()
        rec = {"max_abs": float(diff.max().item()), "rms_abs": float(diff.square().mean().sqrt().item())}
        # floors: any amount, and a significant amount (1e-6 kg/kg, 1e3 /kg)
        floors = (0.0, 0.0) if name == "T" else ((1.0, 1e3) if name[0] == "n" else (1e-12, 1e-6))
        for tag, floor in zip(("", "_significant"), floors):
            sel = b[f].abs() > floor
            rel = diff[sel] / b[f].abs()[sel]
            rec["max_rel" + tag] = float(rel.max().item()) if rel.numel() else 0.0
            rec["rms_rel" + tag] = float(rel.square().mean().sqrt().item()) if rel.numel() else 0.0
        if name[0] == "q" and name != "qv":
            # presence decisions (q > q_min) taken differently by the two forms
            rec["presence_flips"] = int(((a[f] > 1e-14) != (b[f] > 1e-14)).sum().item())
        out["fields"][name] = rec
    # the scales the scheme conserves: cloud water against total water
    # (qv + qc: the adjustment moves water between them), the aerosol number
    # against the aerosol population (n_a + n_c: activation moves number
    # between them); activation decisions: points where n_a changed in one
    # form only
    na, nc, qv, qc = 12, 7, 1, 2
    out["qc_max_rel_to_total_water"] = float(((a[qc] - b[qc]).abs() / (b[qv] + b[qc])).max().item())
    out["na_max_rel_to_population"] = float(((a[na] - b[na]).abs() / (b[na] + b[nc]).clamp_min(1.0)).max().item())
    out["activation_decision_flips"] = int(((a[na] != x0[na]) != (b[na] != x0[na])).sum().item())
    wet = pb > 1e-6 * float(pb.max().item())
    out["precip_column_max_rel"] = float(((pa - pb).abs()[wet] / pb[wet]).max().item()) if wet.any() else 0.0
    return out


def mixed_vs_fp64(casim, torch, fld0, dz, ncols, nlev, dt, nsteps, stream):
    """The mixed form against the FP64 form on the GPU, both advanced from the
    same state, compared after one step and after nsteps: per prognostic
    field the largest and rms absolute difference, and the largest and rms
    relative difference over points where the FP64 value exceeds a floor
    (1e-12 kg/kg for masses, 1 /kg for numbers; and a significant floor,
    1e-6 kg/kg and 1e3 /kg); cloud water relative to total water, aerosol
    number relative to the aerosol population, activation decisions taken
    differently; per form the drift of total water (vapour + condensate in
    the air + accumulated surface precipitation) per step, relative."""
    doms, drift, one = {}, {}, {}
    for name, prec in (("mixed", casim.CASIM_MIXED), ("fp64", casim.CASIM_FP64)):
        ctx = casim.casim_init(precision=prec)
        d = casim.Domain(fld0, dz, ncols)
        bud = torch.zeros((2, ncols), dtype=torch.float64, device=d.fld.device)
        casim.casim_budget(ctx, d.state, ncols, nlev, bud, stream)
        w0 = float(bud[0].sum().item())
        for i in range(nsteps):
            casim.casim_step(ctx, d.state, ncols, nlev, dt, stream)
            if i == 0:
                one[name] = (d.fld[:13, :, :ncols].clone(), d.precip[:, :ncols].sum(0))
        casim.casim_budget(ctx, d.state, ncols, nlev, bud, stream)
        rc, fl = casim.casim_get_error(ctx, stream)
        assert rc == 0, (rc, fl)
        w1 = float(bud[0].sum().item()) + float(d.precip[:, :ncols].sum().item())
        drift[name] = abs(w1 - w0) / w0 / nsteps
        casim.casim_free(ctx)
        doms[name] = d
    x0 = fld0[:13, :, :ncols]
    out = {"steps": nsteps, "water_drift_per_step": drift}
    out["after_one_step"] = _compare(torch, one["mixed"][0], one["fp64"][0], x0, one["mixed"][1], one["fp64"][1])
    del one
    last = _compare(torch, doms["mixed"].fld[:13, :, :ncols], doms["fp64"].fld[:13, :, :ncols], x0,
                    doms["mixed"].precip[:, :ncols].sum(0), doms["fp64"].precip[:, :ncols].sum(0))
    out.update(last)
    del doms
    torch.cuda.empty_cache()
    return out


def reference_arm(args, world, base_fld, dz, ncols, nlev, dt):
    """The reference arm: the FP64 oracle as it stands, on all host cores,
    stepping a sample of the workload's columns.  The sample is the first C
    columns of the domain (the generator draws every column independently, so
    they are a fair sample), C a multiple of 32 sized from one untimed
    calibration step so that the W + K steps take about a minute in all.  It
    runs W untimed steps, then K timed steps of that sample in sequence (the
    sample's state advances like a real run), and reports exactly that:
    config.ncols = C, steps = K, ms_per_step = the mean measured time of one
    step of the C columns, value = C * nlev / that time."""
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    budget_s = 60.0
    per_step_s = min(0.5, budget_s / max(1, args.steps + args.warmup))

    def sample(c):
        return np.ascontiguousarray(base_fld[:, :, :c]), np.zeros((4, c))

    c = min(256, ncols // 32 * 32 or 32)
    sub, pr = sample(c)
    t0 = time.perf_counter()
    oracle.step(sub, c, dz, dt, precip=pr, nthreads=cores)
    rate = c / max(time.perf_counter() - t0, 1e-6)
    c = int(max(32, min(ncols // 32 * 32, rate * per_step_s // 32 * 32)))
    sub, pr = sample(c)
    for _ in range(args.warmup):
        _, _, err = oracle.step(sub, c, dz, dt, precip=pr, nthreads=cores)
        assert err == 0, err
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        _, _, err = oracle.step(sub, c, dz, dt, precip=pr, nthreads=cores)
        times.append(time.perf_counter() - t0)
        assert err == 0, err
    ms = 1e3 * float(np.mean(times))
    v = c * nlev / (ms * 1e-3)
    text = (f"first {c} of the {ncols} columns of {args.workload} x {nlev} levels, {args.warmup} untimed + "
            f"{args.steps} timed steps in sequence, {ms:.2f} ms per step")
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": args.workload, "ncols": c, "nlev": nlev, "dt_s": dt,
                       "sample_of_ncols": ncols, "timed_s": float(np.sum(times)),
                       "form": "FP64 CPU oracle, OpenMP over columns (schedule guided)"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": text},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--ncols", type=int, default=None, help="override the workload's column count")
    ap.add_argument("--forms", default="mixed,fp64", help="forms to time: mixed and/or fp64")
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--acc-steps", type=int, default=100,
                    help="steps of the mixed-vs-FP64 accuracy comparison (0: skip)")
    ap.add_argument("--batch-scale", type=float, default=1.0, help="batch64: scale of the column counts")
    ap.add_argument("--surr-steps", type=int, default=100, help="surrogate: steps compared with the plain step")
    ap.add_argument("--gen-steps", type=int, default=10, help="surrogate: states the training rows come from")
    ap.add_argument("--train-steps", type=int, default=4000, help="surrogate: Adam steps")
    ap.add_argument("--no-more-workloads", action="store_true",
                    help="default run: skip the short batch64, warm_vs_cold and tendency runs")
    ap.add_argument("--no-surrogate", action="store_true",
                    help="leave the surrogate run (training + 100 steps) out of the main line's config")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    from paper_2010_14823_gb300 import synth
    if args.workload == "batch64":
        return bench_batch(args, rank, world, local)
    if args.workload == "surrogate":
        return bench_surrogate(args, rank, world, local)
    if args.workload == "peaks":
        return bench_peaks(args, rank, world, local)
    if args.workload == "warm_vs_cold":
        return bench_warm(args, rank, world, local)
    if args.workload == "tendency":
        return bench_tendency(args, rank, world, local)
    from paper_2010_14823_gb300 import shard
    base_fld, dz, ncols, nlev, dt, _ = synth.workload(args.workload, ncols=args.ncols,
                                                      seed=shard.rank_seed(1236, rank))
    forms = set(args.forms.split(","))
    npts = ncols * nlev

    if args.impl == "reference":
        if rank != 0:
            return
        return reference_arm(args, world, base_fld, dz, ncols, nlev, dt)

    import torch
    from paper_2010_14823_gb300 import casim
    casim.lib()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(x):
        return shard.max_over_ranks(x, dist, "cuda")

    stream = torch.cuda.current_stream()
    dom = casim.Domain(base_fld, dz, ncols)
    fld0 = dom.fld.clone()

    def time_form(precision, steps, warmup):
        ctx = casim.casim_init(precision=precision)
        dom.fld.copy_(fld0)
        dom.precip.zero_()
        for _ in range(warmup):
            casim.casim_step(ctx, dom.state, ncols, nlev, dt, stream)
        rc, fl = casim.casim_get_error(ctx, stream)
        assert rc == 0, (rc, fl)
        barrier()
        n0 = casim.casim_launch_count(ctx)
        t_start = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        t_start.record(stream)
        for i in range(steps):
            casim.casim_step(ctx, dom.state, ncols, nlev, dt, stream)
        t_end.record(stream)
        barrier()
        launches = casim.casim_launch_count(ctx) - n0
        total_ms = t_start.elapsed_time(t_end)
        # the average launch duration over the timed region (one launch per
        # step on this stream, back to back; the gaps between launches are
        # included, so the roofline figure is conservative)
        per = [total_ms / steps]
        rc, fl = casim.casim_get_error(ctx, stream)
        assert rc == 0, (rc, fl)
        casim.casim_free(ctx)
        return total_ms, per, launches

    # algorithmic bytes: 16 fields read per point; 13 written per point the step changes
    ctx = casim.casim_init(precision=casim.CASIM_MIXED)
    before = dom.fld[:13].clone()
    casim.casim_step(ctx, dom.state, ncols, nlev, dt, stream)
    torch.cuda.synchronize()
    changed = int((dom.fld[:13] != before).any(dim=0)[:, :ncols].sum().item())
    # the in-place host step's stores: per field, level and warp (32 columns)
    # the whole 256-byte row where any value's bits changed
    flips = dom.fld[:13].view(torch.int64) != before.view(torch.int64)
    line_rows = int(flips.view(13, nlev, dom.pitch // 32, 32).any(dim=-1).sum().item())
    del before, flips
    casim.casim_free(ctx)

    value = fp64_value = None
    mix_ms = fp_ms = None
    launches = 0
    clocks = None
    mix_per = [float("nan")]
    if "mixed" in forms:
        sampler = ClockSampler(local)
        sampler.start()
        mix_ms, mix_per, launches = time_form(casim.CASIM_MIXED, args.steps, args.warmup)
        clocks = sampler.stop()
        mix_ms = max_over_ranks(mix_ms)
        value = world * npts * args.steps / (mix_ms * 1e-3)
    if "fp64" in forms and args.fp64_steps > 0:
        fp_ms, fp_per, fp_launches = time_form(casim.CASIM_FP64, args.fp64_steps, 1)
        fp_ms = max_over_ranks(fp_ms)
        fp64_value = world * npts * args.fp64_steps / (fp_ms * 1e-3)
        if value is None:
            value, launches, mix_ms, args.steps = fp64_value, fp_launches, fp_ms, args.fp64_steps

    # end to end through the host entry point: pinned host state, copies inside the timed region
    e2e = None
    link = _host_link_gbs(torch, stream) if args.e2e_steps > 0 else None
    if args.e2e_steps > 0:
        pitch = dom.pitch
        hfld = torch.from_numpy(base_fld).pin_memory()
        hdz = torch.from_numpy(dz).pin_memory()
        hpr = torch.zeros((4, pitch), dtype=torch.float64).pin_memory()
        hstate = casim.make_state(hfld.data_ptr(), pitch, hdz.data_ptr(), hpr.data_ptr())
        ctx = casim.casim_init(precision=casim.CASIM_MIXED if "mixed" in forms else casim.CASIM_FP64)
        casim.casim_step_host(ctx, hstate, ncols, nlev, dt, stream)
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            casim.casim_step_host(ctx, hstate, ncols, nlev, dt, stream)
        barrier()
        e2e_s = max_over_ranks(time.perf_counter() - t0)
        # the same call on a pinned state 128 bytes off the 256-byte alignment,
        # which casim_step_host moves by its chunked copy pipeline instead
        # (rows still 128-byte aligned for the copy engines)
        big = torch.empty(hfld.numel() + 16, dtype=torch.float64).pin_memory()
        hfld_c = big[16:].view(hfld.shape)
        hfld_c.copy_(torch.from_numpy(base_fld))
        hpr.zero_()
        cstate = casim.make_state(hfld_c.data_ptr(), pitch, hdz.data_ptr(), hpr.data_ptr())
        casim.casim_step_host(ctx, cstate, ncols, nlev, dt, stream)
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            casim.casim_step_host(ctx, cstate, ncols, nlev, dt, stream)
        barrier()
        copy_s = max_over_ranks(time.perf_counter() - t0)
        del hfld_c, big
        casim.casim_free(ctx)
        # bytes over the host link: every input of the ncols columns, dz and the
        # precipitation rows in; the changed fields' whole warp rows (as the
        # first step wrote them) and the precipitation rows out
        h2d = 16 * nlev * ncols * 8 + hdz.numel() * 8 + 4 * ncols * 8
        d2h = line_rows * 256 + 4 * ncols * 8
        e2e = {"value": world * npts * args.e2e_steps / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "steps": args.e2e_steps,
               "path": "casim_step_host on pinned host state: the step kernel loads every input over the host "
                       "link and stores, per field and warp, whole rows where a value changed, in place; "
                       "equal to the device step bit for bit",
               "copy_pipeline": {"value": world * npts * args.e2e_steps / copy_s, "unit": UNIT,
                                 "ms_per_step": copy_s / args.e2e_steps * 1e3,
                                 "path": "casim_step_host on a pinned state 128 bytes off the 256-byte alignment: "
                                         "65 536-column chunks copied in, stepped and copied back on 3 streams",
                                 "h2d_bytes_per_step": 16 * nlev * ncols * 8 + hdz.numel() * 8 + 4 * ncols * 8,
                                 "d2h_bytes_per_step": 13 * nlev * ncols * 8 + 4 * ncols * 8},
               "host_link_gbs": link,
               "copy_gbs": (h2d + d2h) * args.e2e_steps / e2e_s / 1e9,
               "link_frac": (h2d + d2h) * args.e2e_steps / e2e_s / 1e9 / link["both"] if link else None}

    accuracy = None
    if args.acc_steps > 0 and {"mixed", "fp64"} <= forms:
        accuracy = mixed_vs_fp64(casim, torch, fld0, dz, ncols, nlev, dt, args.acc_steps, stream)

    peaks = _peaks()
    peak = peaks.get("hbm_gbs")
    alg_bytes = 128.0 * npts + 104.0 * changed
    kern_ms = float(np.mean(mix_per))
    achieved = alg_bytes / (kern_ms * 1e-3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak if peak else None,
                "traffic": _measured_traffic(npts) if args.workload.startswith("deep") else None,
                "kernel": "k_step<PolicyMix>", "algorithmic_bytes_per_launch": alg_bytes,
                "changed_points_frac": changed / npts, "ms_per_launch": kern_ms,
                "duration": "average launch over the timed region (CUDA events on the launching stream)",
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (burst copy)"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        r, cores, sample, _ = cpu_oracle_rate(base_fld, dz, ncols, dt, target_s=12.0)
        r1, _, sample1, _ = cpu_oracle_rate(base_fld, dz, ncols, dt, target_s=3.0, nthreads=1)
        cpu = {"value": r, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
               "single_thread_value": r1, "single_thread_sample": sample1}

    surrogate = None
    if not args.no_surrogate and args.workload.startswith("deep") and "mixed" in forms:
        # the learned warm-rain rates on the same workload (their own seed):
        # training, then the batched surrogate step against the plain step
        del dom, fld0
        torch.cuda.empty_cache()
        sl = surrogate_run(args, rank, world, local)
        c = sl["config"]
        surrogate = {"workload": c["workload"], "value": sl["value"], "ms_per_step": sl["ms_per_step"],
                     "plain_ms_per_step": c["plain_ms_per_step"], "path": c["path"],
                     "served_points_per_step": c["served_points_per_step"], "train_rows": c["train_rows"],
                     "train_steps": c["train_steps"], "train_s": c["train_s"],
                     "rate_rel_error_heldout": c["rate_rel_error_heldout"],
                     "precip_total_rel_error": c["precip_total_rel_error"],
                     "precip_column_rel_error": c["precip_column_rel_error"], "network_roofline": sl["roofline"],
                     "gpu_launches": sl["gpu_launches"]}

    more = None
    if not args.no_more_workloads and world == 1 and args.workload.startswith("deep") and "mixed" in forms:
        # the other single-GPU workloads, shortly (20 steps each), each with its
        # own state: the batch of 64 uneven domains, the warm configuration
        # against the cold one on stratus, the source-term mode
        import copy
        torch.cuda.empty_cache()
        sub = copy.copy(args)
        sub.emit, sub.steps, sub.warmup, sub.fp64_steps = False, 20, 3, 1
        more = {}
        for key, fn in (("batch64", bench_batch), ("warm_vs_cold", bench_warm), ("tendency", bench_tendency)):
            ln = fn(sub, rank, world, local)
            c = ln["config"]
            more[key] = {"workload": c["workload"], "value": ln["value"], "ms_per_step": ln["ms_per_step"],
                         "steps": ln["steps"], "fp64_ms_per_step": c.get("fp64_ms_per_step"),
                         "roofline_frac": ln["roofline"]["frac"] if ln["roofline"] else None,
                         "gpu_launches": ln["gpu_launches"]}
            for extra in ("eager_ms_per_step", "tuned", "cold_mixed_ms_per_step", "warm_over_cold",
                          "warm_aerosol_mixed_ms_per_step", "cold_aerosol_mixed_ms_per_step",
                          "warm_three_moment_mixed_ms_per_step", "cold_three_moment_mixed_ms_per_step"):
                if extra in c:
                    more[key][extra] = c[extra]
            torch.cuda.empty_cache()

    if rank == 0:
        cfg = {"workload": args.workload, "ncols": ncols, "nlev": nlev, "dt_s": dt,
               "form": "mixed FP32 rates / FP64 state and transfers" if "mixed" in forms else "FP64",
               "l2": "state 5 GB > L2, no flush needed",
               "parallelism": f"{world} independent domain(s), one per GPU"}
        if fp64_value is not None:
            cfg.update({"fp64_value": fp64_value, "fp64_ms_per_step": fp_ms / args.fp64_steps,
                        "speedup_mixed_vs_fp64": value / fp64_value})
            if args.workload.startswith("deep"):
                cfg["fp64_roofline"] = _fp64_roofline(npts, fp_ms / args.fp64_steps)
        if accuracy is not None:
            cfg["mixed_vs_fp64"] = accuracy
        if surrogate is not None:
            cfg["surrogate"] = surrogate
        if more is not None:
            cfg["more_workloads"] = more
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": mix_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": "f32+f64" if "mixed" in forms else "f64", "data": "synthetic",
                "config": cfg, "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": launches, "clocks": clocks}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
