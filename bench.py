#!/usr/bin/env python
"""Benchmark: trajectory-steps/s of the relic-overdensity hot path on GB300.

One step = one batched launch of the precision-sweep workload (NFW halo
1e13 Msun, mass history M0 exp(-0.8 z), 4 relic masses {0.01, 0.05, 0.1, 0.3}
eV, 64 radii log 1 kpc - 1 Mpc, 200 log q x 64 Gauss-Legendre mu, 800 RK4
steps from z = 0 to 4: 3,276,800 trajectories, 2.62e9 trajectory-steps),
mixed precision (FP32 state and force, FP64-built tables, FP64 sums).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  Under torchrun the job is N copies of the
workload whose requests are partitioned over the N ranks (weak scaling, no
data-path collective); the timing is the max over ranks.  --impl reference times the FP64 CPU oracle on
a bounded sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2410_08267_gb300 import workloads as W  # noqa: E402

METRIC = "trajectory-steps/s"
UNIT = "trajectory-steps/s"
WORKLOAD = ("precision_sweep_mixed: NFW M=1e13 Msun c=7.15 xi=exp(-0.8z), m_nu in "
            "{0.01,0.05,0.1,0.3} eV, 64 radii log 1-1000 kpc, 200 log q (0.01-10 T0) x 64 GL mu, "
            "800 RK4 steps z 0->4")
# Algorithmic FP32 work (FMA = 2 flops, one flop per special function),
# counted from the force + RK4 formulation.  The force has three branches
# (App. A), so its work is data dependent and is counted exactly per run by
# the library's branch tallies (nu_batch_branch_counts):
#   force evaluation beyond R (gradient 0): r^2                          3
#   in the compensating shell: + rsqrt 1, r^-3 2, sel/r^3 - 1/R^3 2      8
#   in the NFW part: + y = r S 2, I(y) = log1p(y) - y/(1+y) 4, /I(c) 1   15
#   RK4 combination per trajectory-step: three stage updates 9 each (27),
#   last force scale (1), positions 2 x 7 (14), velocities 2 x 9 + 1 (19) 61
# A full evaluation everywhere would be 4 x 15 + 61 = 121 per trajectory-step.
# Trajectories that are finished (beyond R and receding: their velocity can no
# longer change) are not integrated further; their remaining steps are counted
# in the workload's nominal trajectory-steps (the metric) but not as executed
# work in the roofline.
FLOPS_EVAL = (3, 8, 15, 15)
FLOPS_COMBINE = 61
FLOPS_FULL = 121
SMS, FP32_LANES_PER_SM = 152, 128
# DRAM bytes (read + write) per launch of the trajectory kernel at the tuned
# shape 128x3xg on this workload: mean of two launches of one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum), recorded in
# profiles/traj_kernel_precision_sweep_mixed.md.  Must be reset to None
# whenever the kernel changes, until it is captured again.
NCU_TRAFFIC_BYTES = {"128x3xg": 1229568.0}
# Pipe utilisation of the same kernel and shape on this workload, from one-pass
# ncu captures (sm__pipe_fma_cycles_active, smsp__issue_active), also recorded
# in that profile summary; reset together with the traffic when the kernel changes.
NCU_PIPES = {"128x3xg": {"fma_pipe_cycles_active": 0.668, "issue_slots_active": 0.630}}
SAMPLE_RADII = (0, 9, 18, 27, 36, 45, 54, 63)   # oracle sample: ~1 s on 16 cores
SAMPLE_MASS_INDEX = 2          # 0.1 eV


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def fp32_peak_tflops(mhz: float) -> float:
    return 2.0 * FP32_LANES_PER_SM * SMS * mhz * 1e6 / 1e12


class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self, max_mhz_fallback: float = 2070.0) -> dict:
        rows = []
        if self.path and os.path.exists(self.path):
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
                except ValueError:
                    continue
            os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": max_mhz_fallback, "reasons": ["unsampled"], "samples": 0}
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({names[i] for _, _, flags in rows for i, f in enumerate(flags)
                          if f.lower() in ("active", "1", "yes")})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def run_oracle_sample(problems, n_threads: int = 0):
    """FP64 oracle on the bounded sample: one mass, four radii (the oracle as is)."""
    import oracle
    pb = problems[SAMPLE_MASS_INDEX].replace(precision=W.FP64)
    t0 = time.perf_counter()
    out = oracle.profile(pb, radius_sel=list(SAMPLE_RADII), n_threads=n_threads)
    dt = time.perf_counter() - t0
    traj_steps = len(SAMPLE_RADII) * pb.n_q * pb.n_mu * pb.n_steps
    return out, dt, traj_steps, oracle.max_threads() if n_threads <= 0 else n_threads


def bench_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    problems = W.precision_sweep(precision=W.MIXED)
    sample = (f"m_nu=0.1 eV, radii {list(SAMPLE_RADII)} of 64 "
              f"({len(SAMPLE_RADII)} x 12800 trajectories x 800 steps)")
    for _ in range(args.warmup):
        run_oracle_sample(problems)
    times, ts, cores = [], 0, 1
    for _ in range(args.steps):
        _, dt, ts, cores = run_oracle_sample(problems)
        times.append(dt)
    total = sum(times)
    value = ts * len(times) / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": sample, "parallelism": "host cores"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def drive_stream(nu, srv, reqs, poll_sleep=2e-4, timeout_s=600.0):
    """Submit each request at its arrival time and collect results; returns
    (wall seconds from first arrival to last result, latencies ms, failures)."""
    t0 = time.perf_counter()
    outstanding = {}
    lat, failed = [], 0
    i = 0
    while (i < len(reqs) or outstanding) and time.perf_counter() - t0 < timeout_s:
        now = time.perf_counter() - t0
        while i < len(reqs) and reqs[i].t_arrival <= now:
            outstanding[nu.nu_server_submit(srv, reqs[i].problem)] = reqs[i].problem.n_radii
            i += 1
        for t in list(outstanding):
            r = nu.nu_server_poll(srv, t, outstanding[t])
            if r is None:
                continue
            del outstanding[t]
            if r[0] == nu.NU_OK:
                lat.append(r[3])
            else:
                failed += 1
        time.sleep(poll_sleep)
    return time.perf_counter() - t0, lat, failed + len(outstanding)


def mass_reuse_once(nu, torch, stream, block, tpt, tflags, steps, flush):
    """The precision sweep as one mass-reuse request (trajectories of the
    heaviest mass read for all four masses): kernel time per step with the
    same launch shape, L2 flush and CUDA events as the main measurement."""
    pb = W.precision_sweep_reuse(precision=W.MIXED)
    with torch.cuda.stream(stream):
        h = nu.create(pb, stream=stream)
    o = nu.nu_opts()
    o.flags = nu.NU_FLAG_TIMING | tflags
    o.stream = stream.cuda_stream
    o.block, o.tpt = block, tpt
    b = nu.nu_batch_create([h], o)
    try:
        for _ in range(3):
            nu.nu_batch_run(b, stream)
        ms = []
        for _ in range(steps):
            with torch.cuda.stream(stream):
                flush.zero_()
            nu.nu_batch_run(b, stream)
            ms.append(nu.nu_batch_kernel_ms(b))
        out = nu.nu_profile_result(h, pb.n_out)[0].reshape(len(pb.masses), pb.n_radii)
    finally:
        nu.nu_batch_destroy(b)
        nu.nu_profile_destroy(h)
    kms = float(np.mean(ms))
    return pb, kms, out


def paper_grid_once(nu, torch, stream, reps=10):
    """The paper's production grid (Sec. III) as one request through the public
    API, end to end (create + run + result + destroy, host buffers), next to
    the paper's own statement that a profile takes seconds."""
    pb = W.paper_production_grid(precision=W.MIXED)
    t = []
    for i in range(reps + 2):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            out, _ = nu.profile(pb, stream=stream, block=128, tpt=3, flags=nu.NU_FLAG_GTAB)
        t.append(time.perf_counter() - t0)
    t = np.array(t[2:]) * 1e3
    return {"workload": ("paper production grid: 20 radii log 10 kpc-50 Mpc x 200 log q (0.01-400 "
                         "k_B T0 at 0.3 eV) x 10 GL mu, 15 masses 0.01-0.5 eV from one trajectory "
                         "set, M=1e12 Msun, linear growth, 800 steps to z_i"),
            "e2e_ms_median": float(np.median(t)), "e2e_ms_min": float(t.min()),
            "profiles_per_request": len(pb.masses),
            "finite": bool(np.all(np.isfinite(out))),
            "paper_statement": ("'within seconds' per profile on GPUs whose model is not stated; "
                                "the C version 'a few seconds' per mass on a laptop CPU")}


def serve_once(nu, rate, n_requests, seed=2412, batched=True, chunk=0, budget=8 << 30,
               resident=False, linger_ms=0.0):
    """The serving workload (Poisson arrivals, mixed requests) through the
    continuous-batching server, or through its one-request-per-launch form.
    chunk 0: whole runs, requests join at the next launch; chunk > 0: each
    launch advances every request by that many steps, so requests also join
    ones already part-way through; resident: whole runs, and requests that
    arrive while a launch runs join it through the device work queue."""
    reqs = W.serving_stream(rate=rate, n_requests=n_requests, seed=seed)
    srv = (nu.nu_server_create(device_bytes=budget, chunk_steps=chunk, max_active=64,
                               resident=resident, linger_ms=linger_ms) if batched
           else nu.nu_server_create(device_bytes=budget, chunk_steps=0, max_active=1))
    try:
        wall, lat, failed = drive_stream(nu, srv, reqs)
        st = nu.nu_server_stats(srv)
    finally:
        nu.nu_server_destroy(srv)
    lat = np.asarray(lat)
    mode = ("one_per_launch" if not batched else
            (f"resident_linger{linger_ms:g}" if resident else
             "continuous" if chunk == 0 else f"continuous_chunk{chunk}"))
    return {"rate_per_s": rate, "requests": n_requests, "mode": mode,
            "profiles_per_s": len(lat) / wall, "p50_ms": float(np.percentile(lat, 50)) if len(lat) else None,
            "p99_ms": float(np.percentile(lat, 99)) if len(lat) else None, "failed": failed,
            "launches": st["iterations"], "max_active": st["max_active_seen"],
            "joined_running_launch": st["joined"], "queue_expired": st["queue_expired"],
            "traj_steps_per_s": st["traj_steps"] / wall, "gpu_busy_frac": st["busy_ms"] / 1e3 / wall}


def roofline_flops(counts):
    """Algorithmic FP32 flops of one launch from its branch tallies."""
    return FLOPS_COMBINE * counts[4] + sum(f * c for f, c in zip(FLOPS_EVAL, counts[:4]))


def batch_leg(nu, torch, stream, problems, block, tpt, tflags, steps, flush, sample, peak, tol):
    """One of the batch workloads (uneven halos, new physics) at the tuned
    launch shape: kernel time per step (CUDA events, L2 flushed), nominal and
    executed trajectory-steps/s, the roofline fraction, one end-to-end pass
    through the public API, and the oracle on a sample of (halo, radius)."""
    import oracle
    with torch.cuda.stream(stream):
        hs = [nu.create(pb, stream=stream) for pb in problems]
    o = nu.nu_opts()
    o.flags = nu.NU_FLAG_TIMING | tflags
    o.stream = stream.cuda_stream
    o.block, o.tpt = block, tpt
    b = nu.nu_batch_create(hs, o)
    try:
        nu.nu_batch_run(b, stream)
        ms = []
        for _ in range(steps):
            with torch.cuda.stream(stream):
                flush.zero_()
            nu.nu_batch_run(b, stream)
            ms.append(nu.nu_batch_kernel_ms(b))
        got = [nu.nu_profile_result(h, pb.n_radii)[0] for h, pb in zip(hs, problems)]
        counts = nu.nu_batch_branch_counts(b, stream)
    finally:
        nu.nu_batch_destroy(b)
        for h in hs:
            nu.nu_profile_destroy(h)
    kms = float(np.mean(ms))
    nominal = sum(pb.traj_steps for pb in problems)
    flops = roofline_flops(counts)
    # end to end through the public API: create (host tables to device),
    # batch, run, result, destroy
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    with torch.cuda.stream(stream):
        hh = [nu.create(pb, stream=stream) for pb in problems]
        o2 = nu.nu_opts()
        o2.stream = stream.cuda_stream
        o2.block, o2.tpt, o2.flags = block, tpt, tflags
        b2 = nu.nu_batch_create(hh, o2)
        nu.nu_batch_run(b2, stream)
        for h, pb in zip(hh, problems):
            nu.nu_profile_result(h, pb.n_radii)
        nu.nu_batch_destroy(b2)
        for h in hh:
            nu.nu_profile_destroy(h)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    errs, misses = [], []
    for i, sel in sample:
        pb = problems[i]
        ref = oracle.profile(pb.replace(precision=W.FP64), radius_sel=sel)
        for r in sel:
            # (a relic cold enough to vanish from the core gives n/nbar = 0 in both)
            e = 0.0 if got[i][r] == ref[r] else abs(got[i][r] - ref[r]) / abs(ref[r])
            errs.append(e)
            if e > tol:
                # the oracle's own spread at this radius under FP32 state rounding,
                # rounding-size step noise and a relative force error of the same
                # size (two seeds, one of each sign): where it reaches the
                # tolerance the radius is chaotic under the mode's rounding
                spr = max(abs(oracle.profile_perturbed(pb, 2.0 ** -22, seed, radius_sel=[r],
                                                       step_noise=True, force_noise=True,
                                                       round_state=True)[r]
                              - ref[r]) / abs(ref[r]) for seed in (1, 2))
                misses.append({"request": i, "radius": r, "rel_err": e, "oracle_spread": spr})
    return {"kernel_ms_per_step": kms, "traj_steps_per_step": nominal,
            "traj_steps_per_s": nominal / (kms / 1e3),
            "executed_traj_steps_per_s": counts[4] / (kms / 1e3),
            "e2e_traj_steps_per_s": nominal / e2e_s,
            "roofline_frac": flops / (kms / 1e3) / 1e12 / peak,
            "accuracy": {"sampled": len(errs), "max_rel_err": float(max(errs)),
                         "within_tol": int(sum(e <= tol for e in errs)), "tol": tol,
                         "misses": misses}}


def bench_ours(args):
    import torch

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        dist = None
        torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    from paper_2410_08267_gb300 import nuprof as nu

    from paper_2410_08267_gb300 import sharding

    dev = torch.cuda.current_device()
    stream = torch.cuda.Stream()
    prec = W.FP64 if args.precision == "fp64" else W.MIXED
    one = W.precision_sweep(precision=prec)
    if args.case == "small":            # profiling case: one mass, 24 radii (fills every SM)
        one = [one[SAMPLE_MASS_INDEX].replace(radii=np.geomspace(1.0, 1000.0, 24))]
    elif args.case == "medium":         # profiling case: every mass, every 4th radius
        one = [pb.replace(radii=pb.radii[::4]) for pb in one]
    elif args.case == "uneven":         # 1024 halos of uneven sizes in one launch
        one = W.batched_uneven(precision=prec)
    elif args.case == "new_physics":    # 256 halos, relic kinds and couplings
        one = W.new_physics(precision=prec)
    # The job at N GPUs is N copies of the workload (weak scaling); its
    # requests are partitioned over the ranks by trajectory-steps, with no
    # collective on the data path.
    job = one * world
    mine = sharding.partition_problems(job, world)[rank]
    problems = [job[i] for i in mine]
    traj_steps = sum(pb.traj_steps for pb in problems)
    job_traj_steps = sum(pb.traj_steps for pb in job)

    with torch.cuda.stream(stream):
        hs = [nu.create(pb, stream=stream) for pb in problems]
    # launch shape: autotuned (untimed) unless given as BLOCKxTPT
    if args.shape == "auto":
        tune = nu.nu_autotune(hs, stream)
        block, tpt, tflags = tune["block"], tune["tpt"], tune["flags"]
    else:
        parts = args.shape.lower().split("x")
        block, tpt = int(parts[0]), int(parts[1])
        tflags = nu.NU_FLAG_GTAB if len(parts) > 2 and parts[2] == "g" else 0
        tune = None
    opts = nu.nu_opts()
    opts.flags = nu.NU_FLAG_TIMING | tflags
    opts.stream = stream.cuda_stream
    opts.block, opts.tpt = block, tpt
    batch = nu.nu_batch_create(hs, opts)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)   # > 129 MB L2

    for _ in range(args.warmup):
        nu.nu_batch_run(batch, stream)
    stream.synchronize()

    # ---- timed region: K steps, L2 flushed between steps ----
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    kernel_ms = []
    launches0 = nu.nu_kernel_launches()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(dev) as clocks:
        wall0 = time.perf_counter()
        for i in range(args.steps):
            with torch.cuda.stream(stream):
                flush.zero_()
            starts[i].record(stream)
            nu.nu_batch_run(batch, stream)
            ends[i].record(stream)
            kernel_ms.append(nu.nu_batch_kernel_ms(batch))
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
    launches = nu.nu_kernel_launches() - launches0
    grid = nu.nu_batch_info(batch)["grid"]
    # results of the last timed run (read before the counting run overwrites them)
    timed_results = {i: nu.nu_profile_result(h, pb.n_radii)[0] for i, h, pb in zip(mine, hs, problems)}
    counts = nu.nu_batch_branch_counts(batch, stream)     # untimed counting run
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    ms_total = sharding.max_over_ranks(float(sum(step_ms)), dist)
    ms_per_step = ms_total / args.steps
    value = job_traj_steps / (ms_per_step / 1e3)
    clock = clocks.summary()

    # results of the last timed run, gathered in job order (for the accuracy record)
    results = sharding.gather_profiles(timed_results, len(job), dist)

    # ---- end to end through the public API with host buffers ----
    # Every step creates its requests (host tables, upload from page-locked
    # staging), batches and runs them, and reads the results back.  Pipelined
    # (the value): the next step's creates and uploads run on a second stream
    # while this step's kernel runs, as a user scanning many profiles would
    # do; every step's copies stay inside the timed region.  Sequential: the
    # same steps one after the other.
    e2e_steps = max(2, min(args.steps, 5))
    up = torch.cuda.Stream()

    def e2e_prepare(st):
        with torch.cuda.stream(st):
            hh = [nu.create(pb, stream=st) for pb in problems]
            o2 = nu.nu_opts()
            o2.stream = st.cuda_stream
            o2.block, o2.tpt, o2.flags = block, tpt, tflags     # the tuned launch shape
            return hh, nu.nu_batch_create(hh, o2)

    def e2e_finish(hh, b2):
        outs = [nu.nu_profile_result(h, pb.n_radii) for h, pb in zip(hh, problems)]
        nu.nu_batch_destroy(b2)
        for h in hh:
            nu.nu_profile_destroy(h)
        return outs

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        hh, b2 = e2e_prepare(stream)
        bh2d = nu.nu_batch_info(b2)["h2d_bytes"]
        nu.nu_batch_run(b2, stream)
        e2e_finish(hh, b2)
    torch.cuda.synchronize()
    e2e_seq_s = sharding.max_over_ranks((time.perf_counter() - t0) / e2e_steps, dist)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    nxt = e2e_prepare(up)
    for i in range(e2e_steps):
        hh, b2 = nxt
        nu.nu_batch_run(b2, stream)
        nxt = e2e_prepare(up) if i + 1 < e2e_steps else None
        e2e_finish(hh, b2)
    torch.cuda.synchronize()
    e2e_s = sharding.max_over_ranks((time.perf_counter() - t0) / e2e_steps, dist)
    h2d = d2h = 0
    for pb in problems:
        h2d += nu.plan(pb)["h2d_bytes"]
        d2h += 2 * 8 * pb.n_radii
    h2d += bh2d                               # batch descriptor upload

    nu.nu_batch_destroy(batch)
    for h in hs:
        nu.nu_profile_destroy(h)

    # ---- the paper's own production grid, end to end ----
    paper_grid = None
    if args.case == "full" and not args.main_only and prec == W.MIXED:
        paper_grid = paper_grid_once(nu, torch, stream)

    # ---- the same four masses from one trajectory set (Sec. III mass reuse) ----
    reuse = None
    if args.case == "full" and not args.main_only and prec == W.MIXED:
        rpb, rms, rout = mass_reuse_once(nu, torch, stream, block, tpt, tflags,
                                         max(3, min(args.steps, 10)), flush)
        kms_main = float(np.mean(kernel_ms))
        reuse = {"workload": (f"one request: trajectories of m={rpb.m_eV} eV read for masses "
                              f"{list(rpb.masses)}; {rpb.n_radii} radii, {rpb.n_q} log q "
                              f"({rpb.q_min}-{rpb.q_max:g} k_B T0 of the fiducial mass) x "
                              f"{rpb.n_mu} GL mu, {rpb.n_steps} steps"),
                 "kernel_ms_per_step": rms,
                 "profiles_per_s": len(rpb.masses) * world / (rms / 1e3),
                 "per_mass_requests_kernel_ms": kms_main,
                 "speedup_vs_per_mass_requests": kms_main / rms,
                 "note": "a different momentum discretisation from the per-mass grids of the metric"}

    # ---- serving: the request stream, continuous batching vs one launch per request,
    #      at a rate the GPU keeps up with and at a saturating one ----
    serving = None
    if args.serve_rate > 0 and args.case == "full" and not args.main_only and prec == W.MIXED:
        serving = {}
        for key, rate, n_req in (("at_rate", args.serve_rate, args.serve_requests),
                                 ("saturated", args.serve_saturated_rate, args.serve_saturated_requests)):
            if rate <= 0:
                continue
            serving[key] = {"continuous": serve_once(nu, rate, n_req, batched=True),
                            "continuous_chunk100": serve_once(nu, rate, n_req, batched=True, chunk=100),
                            "resident": serve_once(nu, rate, n_req, batched=True, resident=True),
                            "one_per_launch": serve_once(nu, rate, n_req, batched=False)}

    # ---- the two batch workloads (1024 uneven halos; 256 halos of new physics) ----
    batch_legs = None
    if args.case == "full" and not args.main_only and prec == W.MIXED and world == 1:
        peak_leg = fp32_peak_tflops(2070.0)
        uneven = W.batched_uneven(precision=prec)
        npx = W.new_physics(precision=prec)
        batch_legs = {
            "uneven": {"workload": ("1024 halos (seed 2410), log10 M ~ U[11,15], c lognormal 0.15 dex, "
                                    "n_r ~ U{8..128} log 1e-3-2 r200, n_q ~ U{32..256}, "
                                    "n_mu ~ U{16..64}, m ~ U[0.01,0.3] eV, 400 steps; one launch"),
                       "oracle_sample": "every 64th halo, innermost and outermost radius",
                       **batch_leg(nu, torch, stream, uneven, block, tpt, tflags, 3, flush,
                                   [(i, [0, uneven[i].n_radii - 1]) for i in range(0, 1024, 64)],
                                   peak_leg, 1e-4)},
            "new_physics": {"workload": ("256 halos (seed 2411), 128 radii x 256 log q x 64 GL mu, "
                                         "FD eta in {-1,0,1} or q^-1/2 e^-q at 1-10 keV, "
                                         "kappa = (1+z)^gamma, 400 steps; one launch"),
                            "oracle_sample": "every 32nd halo, innermost and outermost radius",
                            **batch_leg(nu, torch, stream, npx, block, tpt, tflags, 3, flush,
                                        [(i, [0, 127]) for i in range(0, 256, 32)], peak_leg, 1e-4)},
            "note": ("kernel-only rates at the tuned launch shape, L2 flushed between steps; "
                     "roofline_frac against the FP32 peak at 2070 MHz; misses are sampled radii "
                     "beyond 1e-4 of the FP64 oracle")}

    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    if rank != 0:
        return 0

    # ---- roofline of the trajectory kernel ----
    kms = float(np.mean(kernel_ms))
    live_steps = counts[4]
    flops = roofline_flops(counts)
    achieved = flops / (kms / 1e3) / 1e12
    peak_mhz = clock["sm_max_mhz"] or 2070.0
    if prec == W.FP64:
        # FP64 mode: no unit count for GB300's FP64 pipe is at hand, so the
        # peak is the measured FP64 FMA rate of this GPU (nu_measure_peaks)
        peak = nu.nu_measure_peaks(stream)["dfma_tflops"]
        peak_basis = "measured FP64 FMA rate (nu_measure_peaks)"
    else:
        peak = fp32_peak_tflops(peak_mhz)
        peak_basis = f"152 SMs x 128 FP32 lanes x 2 flop/FMA x {peak_mhz:.0f} MHz"
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak,
                "traffic": (NCU_TRAFFIC_BYTES.get(f"{block}x{tpt}{'xg' if tflags else ''}")
                            if args.case == "full" and prec == W.MIXED else None),
                "ncu_pipes": (NCU_PIPES.get(f"{block}x{tpt}{'xg' if tflags else ''}")
                              if args.case == "full" and prec == W.MIXED else None),
                "kernel": (f"traj_kernel<{'double' if prec == W.FP64 else 'float'},{min(tpt, 2)},"
                           f"packed={tpt == 3},l1_table={bool(tflags)}>"),
                "kernel_ms": kms,
                "flops_per_launch": flops, "flops_per_executed_traj_step": flops / live_steps,
                "executed_traj_steps": live_steps,
                "finished_early_frac": 1.0 - live_steps / traj_steps,
                "lane_steps_run": counts[5], "needed_lane_frac": live_steps / counts[5],
                "branch_counts": {"beyond_R": counts[0], "shell": counts[1],
                                  "nfw_rational_or_series": counts[2], "nfw_log": counts[3]},
                "full_eval_equiv_tflops": FLOPS_FULL * traj_steps / (kms / 1e3) / 1e12,
                "peak_basis": peak_basis}

    # ---- CPU baseline: the oracle on a bounded sample, and the accuracy check ----
    full = W.precision_sweep(precision=W.MIXED)
    ref, dt, ts, cores = run_oracle_sample(full)
    tol = 1e-5 if prec == W.FP64 else 1e-4
    accuracy = None
    if args.case == "full":
        import oracle as _oracle
        sel = list(SAMPLE_RADII)
        accuracy = {"tol": tol, "sample": f"radii {sel} of 64, all four masses", "per_mass": {}}
        for a, pb in enumerate(full):
            r = ref if a == SAMPLE_MASS_INDEX else _oracle.profile(pb.replace(precision=W.FP64),
                                                                    radius_sel=sel)
            rel = np.abs(results[a][sel] - r[sel]) / np.abs(r[sel])
            misses = []
            for i, e in zip(sel, rel):
                if e > tol:
                    # the oracle's own spread at this radius under rounding-size step
                    # noise and a relative force error of the same size (two seeds, one
                    # of each sign), with the state rounded to FP32 in the mixed mode
                    mixed = prec == W.MIXED
                    spr = max(abs(_oracle.profile_perturbed(pb, 2.0 ** -22 if mixed else 2.0 ** -50,
                                                            seed, radius_sel=[i], step_noise=True,
                                                            force_noise=True, round_state=mixed)[i]
                                  - r[i]) / abs(r[i]) for seed in (1, 2))
                    misses.append({"radius": int(i), "rel_err": float(e), "oracle_spread": spr})
            accuracy["per_mass"][f"{pb.m_eV:g} eV"] = {
                "max_rel_err": float(rel.max()), "per_radius": [float(x) for x in rel],
                "misses": misses}
        accuracy["max_rel_err"] = max(v["max_rel_err"] for v in accuracy["per_mass"].values())
        accuracy["misses"] = sum(len(v["misses"]) for v in accuracy["per_mass"].values())
    # per-core rate: one thread on the outermost sampled radius
    import oracle
    pb1 = full[SAMPLE_MASS_INDEX].replace(precision=W.FP64)
    t1 = time.perf_counter()
    oracle.profile(pb1, radius_sel=[SAMPLE_RADII[-1]], n_threads=1)
    dt1 = time.perf_counter() - t1
    cpu = {"value": ts / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"m_nu=0.1 eV, radii {list(SAMPLE_RADII)} of 64, FP64, {dt:.1f} s wall",
           "per_core_value": pb1.n_q * pb1.n_mu * pb1.n_steps / dt1}

    if args.case == "small":
        WORKLOAD_USED = "small profiling case of " + WORKLOAD + " (m_nu=0.1 eV, 24 radii)"
    elif args.case == "medium":
        WORKLOAD_USED = "medium profiling case of " + WORKLOAD + " (every 4th radius: 16 of 64)"
    elif args.case == "uneven":
        WORKLOAD_USED = ("batched_uneven: 1024 halos (seed 2410), log10 M ~ U[11,15], n_r ~ U{8..128} "
                         "x n_q ~ U{32..256} x n_mu ~ U{16..64}, linear growth, 400 RK4 steps z 0->4")
    elif args.case == "new_physics":
        WORKLOAD_USED = ("new_physics: 256 halos (seed 2411), 128 radii x 256 log q x 64 GL mu each, "
                         "FD eta in {-1,0,1} or freeze-in at 1-10 keV, kappa = (1+z)^gamma, 400 steps")
    else:
        WORKLOAD_USED = WORKLOAD
    executed = {"traj_steps_per_s": value * live_steps / traj_steps,
                "frac_of_nominal": live_steps / traj_steps,
                "note": ("trajectory-steps actually integrated; the rest belong to trajectories "
                         "that are finished (beyond R on a path that never re-enters), whose "
                         "velocity can no longer change")}
    line = {"metric": METRIC, "value": value, "executed": executed, "unit": UNIT, "n_gpus": world,
            "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if prec == W.FP64 else "f32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD_USED + (" (FP64 mode)" if prec == W.FP64 else ""),
                       "traj_steps_per_step": job_traj_steps,
                       "precision": ("FP64 state, force, f and sums" if prec == W.FP64 else
                                     "mixed: FP32 state/force, FP64 tables and sums"),
                       "l2": "flushed (256 MiB write) between timed steps",
                       "launch": f"one persistent batched launch per step: grid {grid} CTAs x {block} "
                                 f"threads, shape {block}x{tpt}{'xg' if tflags else ''} "
                                 "(tpt 3 = two trajectories/thread in packed FP32x2; g = table via L1)",
                       "autotune": (None if tune is None else
                                    {f"{b_}x{t_}{'xg' if f_ else ''}": round(ms, 4)
                                     for b_, t_, f_, ms in tune["candidates"]}),
                       "parallelism": (f"{world} ranks, each {len(one)} requests of a job of {world} "
                                       "copies of the workload (partitioned, no collective)")},
            "e2e": {"value": job_traj_steps / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d * world,
                    "d2h_bytes_per_step": d2h * world,
                    "sequential_value": job_traj_steps / e2e_seq_s,
                    "path": ("create (host tables -> device) + batch + run + result + destroy every "
                             "step; value: the next step's create and upload on a second stream "
                             "overlap this step's kernel; sequential_value: steps one after another")},
            "gpu_launches": launches, "wall_s": wall,
            "step_ms": {"mean": ms_per_step, "median": float(np.median(step_ms)),
                        "min": float(np.min(step_ms)), "max": float(np.max(step_ms))}, "serving": serving, "mass_reuse": reuse, "paper_grid": paper_grid,
            "roofline": roofline, "cpu_baseline": cpu, "clocks": clock,
            "accuracy": accuracy, "batch_workloads": batch_legs}
    print(json.dumps(line), flush=True)
    return 0


def bench_serve_sweep(args):
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    from paper_2410_08267_gb300 import nuprof as nu
    rates = [float(r) for r in args.serve_rates.split(",")]
    for rate in rates:
        n_req = int(min(args.serve_requests, max(20, rate * 2)))
        for batched, chunk, res, linger in ((True, 0, False, 0.0), (True, 100, False, 0.0),
                                            (True, 0, True, 0.0), (True, 0, True, 2.0),
                                            (False, 0, False, 0.0)):
            r = serve_once(nu, rate, n_req, batched=batched, chunk=chunk, resident=res,
                           linger_ms=linger)
            print(json.dumps({"metric": "served profiles/s", **r}), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--shape", default="auto",
                    help="launch shape BLOCKxTPT[xg] (e.g. 256x1, 256x3xg), or auto (autotuner)")
    ap.add_argument("--case", choices=("full", "small", "medium", "uneven", "new_physics"), default="full",
                    help="small: one mass x 24 radii of the same workload; medium: all four masses, "
                         "every 4th radius (the full workload's branch mix), both for profiler captures; "
                         "uneven / new_physics: the 1024-halo and 256-halo batch workloads")
    ap.add_argument("--serve-rate", type=float, default=300.0,
                    help="request rate of the serving leg (0: skip it)")
    ap.add_argument("--serve-requests", type=int, default=200)
    ap.add_argument("--serve-saturated-rate", type=float, default=3000.0,
                    help="request rate of the saturating serving leg (0: skip it)")
    ap.add_argument("--serve-saturated-requests", type=int, default=400)
    ap.add_argument("--precision", choices=("mixed", "fp64"), default="mixed",
                    help="fp64: the verification mode (FP64 state and force)")
    ap.add_argument("--main-only", action="store_true",
                    help="skip the serving and mass-reuse legs (profiler runs)")
    ap.add_argument("--serve-rates", default="10,30,100,300,1000,3000,5000",
                    help="request rates of --serve-sweep")
    ap.add_argument("--serve-sweep", action="store_true",
                    help="only the serving workload at rates 10..5000 /s, one JSON line per rate and mode")
    args = ap.parse_args()
    if args.serve_sweep:
        return bench_serve_sweep(args)
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        return bench_reference(args)
    return bench_ours(args)


if __name__ == "__main__":
    sys.exit(main())
