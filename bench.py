"""Benchmark of the implicit SPH thermal-radiative-transfer step on GB300.

One benchmark "step" is one pass of the whole hot path over one job of the 3-D
manufactured workload mms3d-128^3 (128^3 = 2,097,152 interior particles on a
jittered lattice plus 308,952 Dirichlet ghosts, h = 1.5 dx, sigma = 1, no
limiter): set the particles (Morton sort, cell list, neighbour search, operator
sparsity) and advance 50 backward-Euler steps of dt = 1e-3 (material data,
assembly, AMG set-up, preconditioned Krylov solves inside the
nonlinear-elimination loop, per-particle Newton).  The metric is
particle-steps/s = interior particles x time steps / device time.

The same jobs run in both arithmetic forms, one after the other:
  value       the mixed-precision form (FP32 operator copy, FP32 AMG hierarchy
              and V-cycle inside an FP64 Krylov solve with FP64 residuals)
  fp64        the plain FP64 form, with mixed_over_fp64 = value / fp64 value and
              the largest relative difference of the two forms' final energies
  e2e         the mixed form through the host-pointer C ABI: particle arrays and
              per-step sources copied from pinned host memory, final energies
              copied back, all inside the timed region
  roofline    the fine-operator SpMV-class kernels (CG product, residual and
              smoother sweeps on the finest level), CUDA-event time per launch
              against the measured HBM copy bandwidth
  cpu_baseline / --impl reference   the CPU oracle (tests only otherwise) on a
              bounded sample of the same workload, on the host cores

Multi-GPU (torchrun): replicas only -- every rank runs its own job, the
metric is the sum over ranks, timing is the max over ranks.
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

from paper_2001_11606_gb300 import inputs as I  # noqa: E402

L2_BYTES = 129 * 1024 * 1024


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 7:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4)
                          if r[3 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.rows)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def aggregate_ranks(t_local: float, work_local: float):
    """Replicas: every rank ran its own job.  Returns (t_max, total_work) over
    ranks; with one process this is (t_local, work_local).  Uses whatever
    process group is initialised (NCCL on GPUs, gloo in the CPU tests)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return t_local, work_local
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" \
        else torch.device("cpu")
    t = torch.tensor([t_local], dtype=torch.float64, device=dev)
    wk = torch.tensor([work_local], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(wk, op=dist.ReduceOp.SUM)
    return float(t.item()), float(wk.item())


# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum) from one
# ncu capture of the kernel at the workload, keyed (workload, precision, kernel);
# the profiles/ summary named in the second field holds the capture.
# At 128^3 the traffic is that of the same kernel's capture on the 64^3 instance
# of the workload, scaled by the algorithmic bytes of a launch (traffic grows
# with the stored entries and rows a launch processes): FP32 V-cycle residual
# 225.6 MB for 219.1 MB (x1.029), FP64 residual 342.2 MB for 332.9 MB (x1.028).
NCU_TRAFFIC = {
    ("mms3d-lp-64^3", "fp64", "resid"): (338.3e6, "profiles/fine_sweeps_mms3d-lp-64.md"),
    ("mms3d-lp-64^3", "fp64", "spmv_pq"): (341.8e6, "profiles/fine_sweeps_mms3d-lp-64.md"),
    ("mms3d-lp-64^3", "fp64", "post_ap"): (115.1e6, "profiles/fine_sweeps_mms3d-lp-64.md"),
    ("mms3d-128^3", "mixed", "resid"): (1850.8e6, "profiles/fine_sweeps_mms3d-mixed.md"),
    ("mms3d-128^3", "mixed", "true_resid"): (2819.4e6, "profiles/fine_sweeps_mms3d-mixed.md"),
}


# Solver settings: unless given on the command line (--fine-post-smooth,
# --reliable-drop), each form's timed solver tunes them itself on its first
# warm-up step (config.autotune = 1: finest-level post-smoothing on or off,
# Chebyshev degree, the mixed form's reliable-update threshold); the kernel-
# timing and end-to-end passes then run the chosen settings (autotune = 2: the
# SpMV loads in flight only).  The choice and the trial times are in the line's
# config.solver.


def make_workload(name: str):
    if name == "mms3d-lp-64":
        return I.mms_3d_lp(n=64, steps=100)
    if name == "mms3d-lp-32":
        return I.mms_3d_lp(n=32, steps=20)
    if name == "mms2d-32":
        return I.mms_2d(n=32, steps=10)
    if name.startswith("mms3d-") and name[6:].isdigit():
        # 3-D manufactured problem, sigma = 1, no limiter: 50 steps of 1e-3
        return I.mms_3d(n=int(name[6:]), steps=50)
    if name.startswith("sphere-"):
        # heterogeneous sphere problem, 20 steps of 1e-4 (n^3 interior particles)
        return I.sphere_3d(n=int(name.split("-")[1]), steps=20, dt=1e-4)
    raise SystemExit(f"unknown workload {name}")


def sample_block(w, m: int):
    """A bounded sample of workload w for the CPU oracle: the interior lattice
    points of the corner block [0, m)^d, with every particle of the workload
    within the ghost layers around the block as a Dirichlet ghost (holding the
    workload's values there).  The sample's particles, masses, smoothing
    lengths and per-step inputs are the workload's own at those positions."""
    P = w.particles
    if np.any(P.kind == I.COPY):
        raise ValueError("sample_block needs a workload without copy ghosts")
    idx = np.floor(P.pos / P.dx).astype(np.int64)  # lattice cell (jitter < dx / 2)
    g = I.GHOST_LAYERS
    inner = np.all((idx >= 0) & (idx < m), axis=1)
    near = np.all((idx >= -g) & (idx < m + g), axis=1)
    sel = np.flatnonzero(near)
    kind = np.where(inner[sel], I.INTERIOR, I.DIRICHLET).astype(np.int32)
    S = I.Particles(dim=P.dim, dx=P.dx, counts=(m,) * P.dim, pos=np.ascontiguousarray(P.pos[sel]),
                    kind=kind, copy_of=np.full(len(sel), -1, dtype=np.int64),
                    mass=P.mass[sel].copy(), rho=P.rho[sel].copy(), h=P.h[sel].copy(),
                    sigma0=P.sigma0[sel].copy())
    return I.Workload(name=f"{w.name} corner {m}^{P.dim} block", particles=S,
                      params=dict(w.params), dt=w.dt, steps=w.steps, mms=w.mms,
                      e0=w.e0[sel].copy(), E0=w.E0[sel].copy())


def cpu_block(w) -> int:
    """Edge of the sampled block: about 2.6e5 interior particles in 3-D."""
    return min(64 if w.particles.dim == 3 else 512, min(w.particles.counts))


def cpu_sample(w, steps: int = 1):
    """Oracle timing on a bounded sample: neighbour set-up plus `steps` steps."""
    import oracle as O

    t0 = time.perf_counter()
    pb = O.Problem(w.particles, w.params)
    t1 = time.perf_counter()
    e, E = w.e0.copy(), w.E0.copy()
    t_steps = 0.0
    for n in range(1, steps + 1):
        ins = w.step_inputs(n)
        ts = time.perf_counter()
        rc, e, E, _ = pb.step(e, E, w.dt, *ins)
        t_steps += time.perf_counter() - ts
    return dict(setup_s=t1 - t0, step_s=t_steps / steps, cores=O.num_threads())


def run_reference(args, w):
    """The oracle on a bounded sample of the workload (sample_block): its
    neighbour set-up amortised over the job's time steps plus the timed steps."""
    rank, world, _ = dist_env()
    if world > 1 and rank != 0:
        return
    import oracle as O

    O.build()
    ws = sample_block(w, cpu_block(w))
    n_int = ws.particles.n_interior
    t0 = time.perf_counter()
    pb = O.Problem(ws.particles, ws.params)
    setup_s = time.perf_counter() - t0
    e, E = ws.e0.copy(), ws.E0.copy()
    inputs = [ws.step_inputs(n) for n in range(1, args.warmup + args.steps + 1)]
    for n in range(args.warmup):
        rc, e, E, _ = pb.step(e, E, ws.dt, *inputs[n])
    t0 = time.perf_counter()
    for n in range(args.warmup, args.warmup + args.steps):
        rc, e, E, _ = pb.step(e, E, ws.dt, *inputs[n])
    steps_s = time.perf_counter() - t0
    dt_s = steps_s + setup_s * args.steps / w.steps
    value = n_int * args.steps / dt_s
    sample = (f"{ws.name}: {n_int} interior particles; one backward-Euler step per benchmark "
              f"step plus the neighbour set-up ({setup_s:.1f} s) amortised over the job's "
              f"{w.steps} steps")
    line = {"impl": "reference", "metric": "particle-steps/s", "value": value,
            "unit": "particle-steps/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * dt_s / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": w.name, "precision": "fp64",
                                            "sample": ws.name},
            "cpu_baseline": {"value": value, "unit": "particle-steps/s", "cores": O.num_threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "particle-steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_serving(args):
    """Serving stream: Poisson arrivals of heating-wave problems (2-D/3-D,
    1k..256k particles, 20 steps each) through the continuous-batching loop.
    Measures the saturated service rate mu (all requests queued at once), then
    replays the stream at 0.5, 0.8 and 1.2 mu and reports p50/p99 latency."""
    from paper_2001_11606_gb300 import sphrt

    n_req = args.requests
    descs = I.serving_stream(n_req, seed=4)
    problems = []
    for d in descs:
        w = I.heating_wave(d["dim"], d["n_target"], d["sigma0"], seed=d["seed"], steps=20)
        problems.append(w)
    total_ps = sum(w.particles.n_interior * w.steps for w in problems)
    cfgs = [sphrt.config_from_params(w.params) for w in problems]

    def play(rate, workers):
        srv = sphrt.Server(workers=workers, max_resident=args.max_resident,
                           hbm_budget_bytes=120e9)
        gaps = np.diff([0.0] + [d["arrival"] for d in descs])  # mean 1
        t0 = time.perf_counter()
        ids, t_arr = [], []
        t_next = t0
        for k, w in enumerate(problems):
            if rate is not None:
                t_next += gaps[k] / rate
                delay = t_next - time.perf_counter()
                if delay > 0:
                    time.sleep(delay)
            t_arr.append(time.perf_counter())
            ids.append(srv.submit(cfgs[k], w.particles, w.e0, w.E0, w.steps, w.dt))
        lat = []
        for k, rid in enumerate(ids):
            rc = srv.wait(rid)
            if rc != sphrt.OK:
                raise RuntimeError(f"request {k} failed: {rc}")
            st, t = srv.poll(rid)
            lat.append(t[2] - t[1] + (t[1] - t[0]))  # done - submit
        info = srv.info()
        makespan = info.t_last_done - info.t_first_submit
        srv.close()
        lat = np.array(lat)
        return dict(p50_s=float(np.percentile(lat, 50)), p99_s=float(np.percentile(lat, 99)),
                    mean_s=float(lat.mean()), makespan_s=makespan,
                    throughput=total_ps / makespan, req_per_s=n_req / makespan,
                    peak_resident=info.peak_resident, peak_bytes=info.peak_bytes,
                    fused_requests=info.fused_requests, fused_batches=info.fused_batches)

    sat = play(None, args.workers)
    mu = sat["req_per_s"]
    loads = {}
    for f in (0.5, 0.8, 1.2):
        loads[str(f)] = play(f * mu, args.workers)
    line = {"metric": "serving p99 latency", "value": loads["0.8"]["p99_s"], "unit": "s",
            "higher_is_better": False, "n_gpus": 1, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"serving stream: {n_req} heating-wave requests, 2-D/3-D, "
                                   "1k..256k particles, 20 steps of dt = 1e-5",
                       "workers": args.workers, "max_resident": args.max_resident,
                       "hbm_budget_bytes": 120e9, "particle_steps": total_ps},
            "saturated": sat, "mu_req_per_s": mu, "loads": loads}
    print(json.dumps(line), flush=True)


def batch_problems(k: int, seed: int = 7):
    """The serving stream's fusable requests: k heating-wave problems (2-D/3-D
    50/50, 1k..20k particles log-uniform, sigma0 log-uniform in [1, 100], 20
    steps of dt = 1e-5)."""
    descs = I.serving_stream(k, seed=seed, n_min=1000, n_max=20000)
    return [I.heating_wave(d["dim"], d["n_target"], d["sigma0"], seed=d["seed"], steps=20)
            for d in descs]


def batch_bytes(info, dim, krylov, degree, steps):
    """Algorithmic bytes of one batched run of `steps` steps of one problem:
    every operator sweep (one residual a step -- later outer iterations take
    the residual from the B x the CG carries -- and degree sweeps a Krylov
    iteration: the CG product and degree - 1 inside the Chebyshev
    application) streams the operator's values and columns once (12 B an
    entry) and 32 B per row (row pointer, diagonal, the row's own x, y
    written); every step's assembly reads G and the columns and writes the
    values (20 B an entry) and its limiter gradient reads the neighbour
    columns and the dim per-pair weights (4 + 8 dim B an entry)."""
    nnz, ni, nbr = info["nnz_operator"], info["n_interior"], info["nnz_neighbours"]
    return ((steps + degree * krylov) * (12 * nnz + 32 * ni)
            + steps * (20 * nnz + (4 + 8 * dim) * nbr))


def run_batch(args):
    """Batched form: the serving stream's small problems, one batch per dimension,
    each advanced 20 steps by one CUDA-graph launch (per step, one batched-step
    launch per cluster size).  The launch shape of each batch is picked by the
    library's autotuner."""
    import torch

    from paper_2001_11606_gb300 import sphrt

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    streams = {d: torch.cuda.Stream(device=local) for d in (2, 3)}
    stream = streams[3]
    probs = batch_problems(args.batch_k)
    groups = {d: [w for w in probs if w.particles.dim == d] for d in (2, 3)}
    groups = {d: g for d, g in groups.items() if g}
    dt, T = probs[0].dt, probs[0].steps
    hbm, peak_src = peaks()
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=local)

    def make(d, shape=None):
        g = groups[d]
        cfg = sphrt.config_from_params(g[0].params, device=local, stream=streams[d].cuda_stream)
        B = sphrt.Batch(cfg)
        B.add_many([(w.particles, w.e0, w.E0) for w in g], threads=4)
        if shape is not None:
            B.set_shape(*shape)
        return B

    t0 = time.perf_counter()
    batches = {d: make(d) for d in groups}
    setup_s = time.perf_counter() - t0
    tuned, tables, tune_s = {}, {}, {}
    for d, B in batches.items():
        t0 = time.perf_counter()
        if args.batch_shape:
            B.set_shape(*[int(a) for a in args.batch_shape.split(",")])
            tuned[d], tables[d] = B.get_shape(), {}
        else:
            tuned[d], tables[d] = B.autotune(dt)
        tune_s[d] = time.perf_counter() - t0
    infos = {d: [B.problem_info(k) for k in range(len(groups[d]))] for d, B in batches.items()}
    ps_run = sum(i["n_interior"] * T for d in infos for i in infos[d])
    # the batches run side by side, each on its own stream from its own host
    # thread (the library's calls release the interpreter lock), as the serving
    # loop's workers run fused batches; the run's time is from a start event
    # both streams wait on to the later of the two end events
    ev0 = torch.cuda.Event(enable_timing=True)
    ev_end = {d: torch.cuda.Event(enable_timing=True) for d in batches}

    def one_run():
        main = streams[3]
        with torch.cuda.stream(main):
            flush.zero_()  # inputs are larger than L2, and L2 is flushed between runs
        ev0.record(main)
        for d in batches:
            streams[d].wait_event(ev0)
        res = {}

        def go(d):
            rc, st, ou, kr = batches[d].run(dt, T)
            ev_end[d].record(streams[d])
            res[d] = (st, ou, kr)

        th = [threading.Thread(target=go, args=(d,)) for d in batches]
        for t in th:
            t.start()
        for t in th:
            t.join()
        for d in batches:
            streams[d].synchronize()
        ms = {d: ev0.elapsed_time(ev_end[d]) for d in batches}
        return res, ms

    for _ in range(args.warmup):
        one_run()
    clocks = ClockSampler(local)
    clocks.start()
    runs = [one_run() for _ in range(args.steps)]
    clk = clocks.stop()
    ms_tot = [max(ms.values()) for _, ms in runs]
    t_ms = statistics.mean(ms_tot)
    t_max, work = aggregate_ranks(t_ms * 1e-3 * args.steps, ps_run * args.steps)
    per_dim = {}
    byt_all = 0.0
    for d in batches:
        deg = tuned[d][1]
        byt = []
        for res, ms in runs:
            st, ou, kr = res[d]
            assert np.all(st == 0), f"batched {d}-D run did not converge"
            byt.append(sum(batch_bytes(infos[d][k], d, int(kr[k]), deg, T)
                           for k in range(len(groups[d]))))
        mean_ms = statistics.mean(ms[d] for _, ms in runs)
        mean_b = statistics.mean(byt)
        byt_all += mean_b
        res0 = runs[-1][0][d]
        per_dim[f"{d}d"] = {
            "problems": len(groups[d]),
            "interior_particles": sum(i["n_interior"] for i in infos[d]),
            "problems_per_cluster_size": {str(c): sum(i["cluster"] == c for i in infos[d])
                                          for c in (1, 2, 4, 8)},
            "operator_entries": sum(i["nnz_operator"] for i in infos[d]),
            "shape": dict(zip(("lanes_per_row", "cheb_degree", "blocks_per_sm", "rows_per_cta"),
                              tuned[d])),
            "autotune_s": tune_s[d],
            "autotune_ms": {f"W{k[0]}-deg{k[1]}-b{k[2]}-r{k[3]}": v for k, v in tables[d].items()},
            "ms_to_end": mean_ms, "gbs_own_time": mean_b / (mean_ms * 1e-3) / 1e9,
            "outer_per_step": float(np.mean(res0[1])) / T,
            "krylov_per_step": float(np.mean(res0[2])) / T}
    achieved = byt_all / (t_ms * 1e-3) / 1e9  # both batches' bytes over the run's time
    value = work / t_max

    # end to end through the public API from host arrays: set-up of every problem
    # (neighbours, operator), the runs with the tuned shapes, and every result read back
    h2d = sum(w.particles.pos.nbytes + 5 * 8 * w.particles.n + 4 * w.particles.n
              + (8 * w.particles.n if np.any(w.particles.kind == sphrt.COPY) else 0)
              for w in probs)
    d2h = sum(16 * w.particles.n for w in probs)
    e_ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    e_ev[0].record(stream)
    fresh = {d: make(d, tuned[d]) for d in groups}
    for d, B in fresh.items():
        B.run(dt, T)
        for k in range(len(groups[d])):
            B.get_energies(k)
    e_ev[1].record(stream)
    stream.synchronize()
    e2e_s = e_ev[0].elapsed_time(e_ev[1]) * 1e-3
    for B in list(fresh.values()) + list(batches.values()):
        B.close()
    if rank != 0:
        return
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        small = sorted(probs, key=lambda w: w.particles.n)[:3]
        import oracle as O

        O.build()
        t0 = time.perf_counter()
        for w in small:
            pb = O.Problem(w.particles, w.params)
            e, E = w.e0.copy(), w.E0.copy()
            rc, e, E, _ = pb.step(e, E, w.dt)
        cpu_s = time.perf_counter() - t0
        n_s = sum(w.particles.n_interior for w in small)
        cpu = {"value": n_s / cpu_s, "unit": "particle-steps/s", "cores": O.num_threads(),
               "kind": "oracle",
               "sample": f"the 3 smallest problems of the batch ({n_s} interior particles), "
                         "neighbour set-up plus one backward-Euler step each"}
    line = {"metric": "particle-steps/s (batched form)", "value": value,
            "unit": "particle-steps/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"batched serving problems: {args.batch_k} heating-wave "
                                   "problems, 2-D/3-D, 1k..20k particles, one batch per "
                                   f"dimension, {T} steps of dt = {dt:g} per run",
                       "step": "one CUDA-graph run of each batch (20 steps), the two batches "
                               "side by side on two streams",
                       "l2": "flushed between runs (a 258 MB write)",
                       "setup_s": setup_s},
            "batches": per_dim,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": achieved / hbm, "traffic": None,
                         "kernel": "batch_step_kernel (the two batches' graph runs, side by "
                                   "side: run time from the common start to the later end)",
                         "peak_source": peak_src},
            "e2e": {"value": ps_run / e2e_s, "unit": "particle-steps/s",
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "includes": "set-up of every problem from host arrays, the runs, results"},
            "gpu_launches": args.steps * T * sum(
                1 + len({i["cluster"] for i in infos[d]}) for d in batches),
            "clocks": clk,
            "cpu_baseline": cpu}
    print(json.dumps(line), flush=True)


def fine_roofline(k_kinds, k_ms, k_bytes, hbm, src, workload, precision):
    """Roofline object of the fine kernel with the largest total event time."""
    dom = max(k_kinds, key=lambda k: k_kinds[k][1])
    d_n, d_ms, d_by = k_kinds[dom]
    achieved = (d_by / (d_ms / 1e3)) / 1e9 if d_ms > 0 else None
    traffic = NCU_TRAFFIC.get((workload, precision, dom))
    return {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
            "frac": achieved / hbm if achieved else None,
            "traffic": traffic[0] if traffic else None,
            "kernel": f"{dom} (fine level, {precision})",
            "timing": "CUDA events per launch on the solver stream, the same jobs in a second "
                      "timed pass with the host-driven loop",
            "launches": d_n, "bytes_per_launch": d_by / d_n if d_n else None,
            "us_per_launch": 1e3 * d_ms / d_n if d_n else None,
            "traffic_source": traffic[1] if traffic else None,
            "peak_source": src,
            "fine_kernels": {k: {"launches": v[0],
                                 "GB/s": (v[2] / (v[1] / 1e3)) / 1e9 if v[1] > 0 else None,
                                 "us_per_launch": 1e3 * v[1] / v[0] if v[0] else None,
                                 "share_of_timed": v[1] / k_ms if k_ms > 0 else None}
                             for k, v in k_kinds.items() if v[0] > 0},
            "all_fine_GB/s": (k_bytes / (k_ms / 1e3)) / 1e9 if k_ms > 0 else None}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="mms3d-128")
    ap.add_argument("--time-steps", type=int, default=None,
                    help="backward-Euler steps per job (default: the workload's)")
    ap.add_argument("--precision", default="both", choices=["fp64", "mixed", "both"],
                    help="both: the mixed form is the value, the FP64 form is timed beside it")
    ap.add_argument("--precond", default="amg", choices=["jacobi", "chebyshev", "amg"])
    ap.add_argument("--fine-post-smooth", type=int, default=None, choices=[0, 1],
                    help="AMG finest-level post-smoothing (default: the library's)")
    ap.add_argument("--reliable-drop", type=float, default=None)
    ap.add_argument("--krylov-start", type=int, default=None, choices=[0, 1, 2, 3],
                    help="start of each step's first solve: 0 E^{n-1}, p > 0 extrapolated in time (order p)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-kernel-timing", action="store_true")
    ap.add_argument("--no-graphs", action="store_true",
                    help="host-driven outer loop instead of the per-step CUDA graph")
    ap.add_argument("--check-every", type=int, default=None,
                    help="host-driven loop: Krylov iterations queued per convergence read "
                         "(1: no launch after convergence, the graph's kernel sequence)")
    ap.add_argument("--requests", type=int, default=512, help="serving: number of requests")
    ap.add_argument("--batch-k", type=int, default=512,
                    help="batch: number of problems (both dimensions)")
    ap.add_argument("--batch-shape", default=None,
                    help="batch: W,degree,blocks_per_sm,rows_per_cta instead of the autotuner")
    ap.add_argument("--workers", type=int, default=8, help="serving: worker threads")
    ap.add_argument("--max-resident", type=int, default=32, help="serving: resident cap")
    args = ap.parse_args()
    if args.workload == "serving":
        run_serving(args)
        return
    if args.workload == "batch":
        run_batch(args)
        return

    w = make_workload(args.workload)
    if args.time_steps:
        w.steps = args.time_steps
    if args.impl == "reference":
        run_reference(args, w)
        return

    import torch

    from paper_2001_11606_gb300 import sphrt

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    P = w.particles
    n, n_int, T = P.n, P.n_interior, w.steps
    stream = torch.cuda.Stream(device=dev)
    precond = {"jacobi": sphrt.PRECOND_JACOBI, "chebyshev": sphrt.PRECOND_CHEBYSHEV,
               "amg": sphrt.PRECOND_AMG}[args.precond]
    forms = {"both": ["mixed", "fp64"], "mixed": ["mixed"], "fp64": ["fp64"]}[args.precision]
    head = forms[0]
    prec_of = {"mixed": sphrt.MIXED, "fp64": sphrt.FP64}
    extra = {"check_every": args.check_every} if args.check_every else {}
    if args.fine_post_smooth is not None:
        extra["fine_post_smooth"] = args.fine_post_smooth
    if args.reliable_drop is not None:
        extra["reliable_drop"] = args.reliable_drop
    if args.krylov_start is not None:
        extra["krylov_start"] = args.krylov_start
    tune = args.fine_post_smooth is None and args.reliable_drop is None
    chosen = {f: {} for f in forms}  # the timed solver's tuned settings, per form
    trials = {}

    def make_cfg(form, **kw):
        settings = dict(extra, **chosen[form])
        settings["autotune"] = 1 if tune and not chosen[form] else 2
        settings.update(kw)
        return sphrt.config_from_params(w.params, device=local, stream=stream.cuda_stream,
                                        precond=precond, precision=prec_of[form], **settings)

    # ---- inputs resident in HBM --------------------------------------------
    f64 = dict(dtype=torch.float64, device=dev)
    d_pos = torch.as_tensor(P.pos, **f64)
    d_part = [torch.as_tensor(a, **f64) for a in (P.mass, P.rho, P.h, P.sigma0)]
    d_kind = torch.as_tensor(P.kind, dtype=torch.int32, device=dev)
    d_e0, d_E0 = torch.as_tensor(w.e0, **f64), torch.as_tensor(w.E0, **f64)
    # per-step sources and ghost values (manufactured problems); problems without
    # sources keep their initial ghost values and pass NULL (no per-step inputs)
    if w.mms is not None:
        host_inputs = [w.step_inputs(k) for k in range(1, T + 1)]
        d_inputs = [[torch.as_tensor(a, **f64) for a in ins] for ins in host_inputs]
        d_ptrs = [[a.data_ptr() for a in ins] for ins in d_inputs]
    else:
        host_inputs = None
        d_ptrs = [[0, 0, 0, 0] for _ in range(T)]
    d_out = {f: (torch.empty(n, **f64), torch.empty(n, **f64)) for f in forms}
    torch.cuda.synchronize(dev)

    def job_device(S, form):
        S.set_particles_device(n, d_pos.data_ptr(), *[a.data_ptr() for a in d_part],
                               d_kind.data_ptr(), 0, d_e0.data_ptr(), d_E0.data_ptr())
        outer = krylov = 0
        for k in range(T):
            _, st = S.step_device(w.dt, *d_ptrs[k])
            outer += st.outer_iters
            krylov += st.krylov_iters_total
        S.get_energies_device(d_out[form][0].data_ptr(), d_out[form][1].data_ptr())
        return outer, krylov

    def barrier():
        if world > 1:
            import torch.distributed as dist

            dist.barrier()

    # ---- timed passes: each form warmed up, then K jobs between events -----
    sampler = ClockSampler(local)
    timed = {}
    sampler.start()
    for form in forms:
        S = sphrt.Solver(make_cfg(form, graphs=int(not args.no_graphs)))
        for _ in range(args.warmup):
            job_device(S, form)
        barrier()
        torch.cuda.synchronize(dev)
        launches0 = S.launch_count()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        iters = [job_device(S, form) for _ in range(args.steps)]
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        barrier()
        gpu_ms = ev0.elapsed_time(ev1)
        t_max, work = aggregate_ranks(gpu_ms / 1e3, float(n_int * T * args.steps))
        timed[form] = dict(value=work / t_max, t_max=t_max, launches=S.launch_count() - launches0,
                           outer=sum(i[0] for i in iters) / (args.steps * T),
                           krylov=sum(i[1] for i in iters) / (args.steps * T))
        c = S.get_config()
        chosen[form] = dict(fine_post_smooth=c.fine_post_smooth, cheb_degree=c.cheb_degree,
                            reliable_drop=c.reliable_drop)
        trials[form] = S.solver_tuning()
        S.close()
    clocks = sampler.stop()

    # ---- kernel timing: the same jobs with CUDA events around every fine-operator
    # SpMV-class launch (per-launch events need the host-driven loop) --------------
    kt = {}
    if not args.no_kernel_timing:
        for form in forms:
            S_t = sphrt.Solver(make_cfg(form, kernel_timing=1))
            job_device(S_t, form)
            S_t.kernel_stats(reset=True)
            barrier()
            for _ in range(args.steps):
                job_device(S_t, form)
            torch.cuda.synchronize(dev)
            kt[form] = (S_t.kernel_stats(), S_t.kernel_stats_by_kind())
            S_t.close()

    # ---- end to end through the host-pointer C ABI (the headline form) -------
    e2e = None
    if not args.no_e2e:
        S = sphrt.Solver(make_cfg(head, graphs=int(not args.no_graphs)))
        pin = dict(dtype=torch.float64, pin_memory=True)
        h_pos = torch.as_tensor(P.pos, dtype=torch.float64).pin_memory()
        h_part = [torch.as_tensor(a, dtype=torch.float64).pin_memory() for a in
                  (P.mass, P.rho, P.h, P.sigma0, w.e0, w.E0)]
        h_kind = torch.as_tensor(P.kind, dtype=torch.int32).pin_memory()
        h_inputs = ([[torch.as_tensor(a, dtype=torch.float64).pin_memory() for a in ins]
                     for ins in host_inputs] if host_inputs is not None else None)
        h_ptrs = ([[a.data_ptr() for a in ins] for ins in h_inputs] if h_inputs is not None
                  else [[0, 0, 0, 0] for _ in range(T)])
        h_e = torch.empty(n, **pin)
        h_E = torch.empty(n, **pin)
        L = sphrt.load()
        import ctypes as C

        def job_host():
            rc = L.sph_rt_set_particles(S._h, n, C.c_void_p(h_pos.data_ptr()),
                                        *[C.c_void_p(a.data_ptr()) for a in h_part[:4]],
                                        C.c_void_p(h_kind.data_ptr()), None,
                                        C.c_void_p(h_part[4].data_ptr()),
                                        C.c_void_p(h_part[5].data_ptr()))
            if rc != 0:
                raise RuntimeError(S.last_error())
            for k in range(T):
                S.step_host_ptrs(w.dt, *h_ptrs[k])
            S.get_energies_host_ptrs(h_e.data_ptr(), h_E.data_ptr())

        job_host()
        barrier()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            job_host()
        torch.cuda.synchronize(dev)
        t_e2e, work_e2e = aggregate_ranks(time.perf_counter() - t0, float(n_int * T * args.steps))
        h2d = (P.pos.nbytes + 6 * n * 8 + n * 4) + (T * 4 * n * 8 if h_inputs is not None else 0)
        e2e = {"value": work_e2e / t_e2e, "unit": "particle-steps/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(2 * n * 8),
               "precision": head}
        S.close()

    if rank != 0:
        return
    hbm, src = peaks()
    roof = None
    if kt:
        (k_launch, k_ms, k_bytes), k_kinds = kt[head]
        roof = fine_roofline(k_kinds, k_ms, k_bytes, hbm, src, w.name, head)
        for form in forms[1:]:
            (_, ms2, by2), kinds2 = kt[form]
            roof[f"{form}_form"] = fine_roofline(kinds2, ms2, by2, hbm, src, w.name, form)
    cpu = None
    if not args.no_cpu_baseline:
        import oracle as O

        O.build()
        ws = sample_block(w, cpu_block(w))
        cs = cpu_sample(ws, steps=1)
        per = cs["setup_s"] / T + cs["step_s"]
        cpu = {"value": ws.particles.n_interior / per, "unit": "particle-steps/s",
               "cores": cs["cores"], "kind": "oracle",
               "sample": (f"{ws.name} ({ws.particles.n_interior} interior particles): oracle "
                          f"neighbour set-up ({cs['setup_s']:.1f} s, amortised over {T} steps) "
                          f"plus one backward-Euler step ({cs['step_s']:.1f} s)")}
    mask = P.kind == I.INTERIOR
    hd = timed[head]
    line = {"metric": "particle-steps/s", "value": hd["value"], "unit": "particle-steps/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * hd["t_max"] / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if head == "fp64" else "f32+f64",
            "data": "synthetic",
            "config": {"workload": w.name, "interior_particles": n_int, "ghosts": n - n_int,
                       "time_steps_per_job": T, "dt": w.dt, "precision": head,
                       "precond": args.precond, "parallelism": f"replicas{world}",
                       "krylov_start": make_cfg(head).krylov_start,
                       "outer_loop": "host" if args.no_graphs else "cuda-graph",
                       "l2": "inputs larger than L2 (operator > 129 MB)",
                       "outer_iters_per_step": hd["outer"], "krylov_iters_per_step": hd["krylov"],
                       "ms_per_time_step": 1e3 * hd["t_max"] / (args.steps * T),
                       "solver": {f: dict(chosen[f], tuned=tune,
                                          trials_ms=[{"fine_post_smooth": t[0], "cheb_degree": t[1],
                                                      "reliable_drop": t[2], "ms": t[3]}
                                                     for t in trials.get(f, [])])
                                  for f in forms}},
            "clocks": clocks, "e2e": e2e, "gpu_launches": hd["launches"], "roofline": roof,
            "cpu_baseline": cpu}
    if len(forms) > 1:
        other = forms[1]
        od = timed[other]
        eh = d_out[head][0].cpu().numpy()[mask]
        Eh = d_out[head][1].cpu().numpy()[mask]
        eo = d_out[other][0].cpu().numpy()[mask]
        Eo = d_out[other][1].cpu().numpy()[mask]
        diff = max(float(np.max(np.abs(eh - eo) / np.abs(eo))),
                   float(np.max(np.abs(Eh - Eo) / np.abs(Eo))))
        line[other] = {"value": od["value"], "unit": "particle-steps/s",
                       "ms_per_step": 1e3 * od["t_max"] / args.steps,
                       "ms_per_time_step": 1e3 * od["t_max"] / (args.steps * T),
                       "outer_iters_per_step": od["outer"], "krylov_iters_per_step": od["krylov"],
                       "gpu_launches": od["launches"]}
        line[f"{head}_over_{other}"] = hd["value"] / od["value"]
        line[f"{head}_vs_{other}_max_rel_diff"] = diff
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
