"""Benchmark of the modified Hermite hot path on GB300.

Workload (one GPU): SMBH disc, M_bh = 1 plus N = 65536 equal-mass stars of total
mass 0.01, surface density ~ r^-1.5 on [0.1, 1], e and i Rayleigh (0.05, 0.025),
Plummer eps = 1e-4, 8th-order modified Hermite in FP64, shared step
dt = 2 pi 1e-3, P(EC)^3.  A step is one Taylor prediction plus three
evaluate/correct passes over all bodies; its work is 3 N (N - 1) pair
interactions (N = 65537 bodies).  The FP32-pair precision form is measured on
the same workload and reported under "forms".

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Timing: W untimed warm-up steps, then K steps, each bracketed by CUDA events
on the simulation's stream with an L2 flush (a 256 MB device write) between
steps, outside the events; barrier + synchronize around the timed region;
max over ranks.  For N > 1 (torchrun) every rank advances its own replica of
the workload (the single-system path does not shard; replicas only).

--impl reference times the CPU oracle (plain C, FP64, OpenMP over bodies) on
the host cores: each step is one 8th-order evaluation of a bounded sample of
bodies against all N bodies of the same disc.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "pair-interactions/s, particle-steps/s vs plain FP64 at equal ecc-vector error"
UNIT = "pair-interactions/s"
N_STARS = 65536
ORDER = 8
N_ITER = 3
DT = 2 * np.pi * 1e-3
EPS = 1e-4
SEED = 2
# Algorithmic flops per pair interaction at 8th order: the conventional count
# used for 4th/6th/8th-order Hermite codes (60/97/144).
FLOPS_PER_PAIR = {4: 60, 6: 97, 8: 144}
# The FP64 headline kernel evaluates each unordered pair once and accumulates
# its terms into both bodies: per unordered pair the conventional count of one
# direction plus one multiply-add (2 flops) per accumulated component of the
# second body, 3 (p + 1) of them.
FLOPS_PER_UNORDERED_PAIR = {o: FLOPS_PER_PAIR[o] + 2 * 3 * (o // 2) for o in (4, 6, 8)}
# Peaks from unit counts and the maximum SM clock (2070 MHz), 152 SMs:
#   FP32: 128 FMA lanes/SM x 2 flops; FP64: 2 DFMA lanes/SM x 2 flops (ncu's
#   peak of 304 DFMA thread-instructions per cycle on 152 SMs; the GB300
#   nominal figure is 1.25 TFLOP/s).  mh.measure_peaks() measures both on the
#   box and the JSON line reports them beside these.
SM_MAX_MHZ = 2070.0
N_SM = 152
PEAK_FP32 = N_SM * 128 * 2 * SM_MAX_MHZ * 1e6
PEAK_FP64 = N_SM * 2 * 2 * SM_MAX_MHZ * 1e6
# DRAM traffic per launch of the dominant kernel from one ncu capture
# (profiles/); valid only while the kernel source is the one captured.
TRAFFIC = {"files": ["paper_2006_02501_gb300/csrc/pair_sym.cu", "paper_2006_02501_gb300/csrc/pair_math.cuh"],
           "sha256": ["9bb18f03603bf070ab67a7690021637658f34ee289fa7f8943c02ba8300861e2",
                      "7b05f4cd731085ffd18547e017c5352bbda74f8e674505c0fb411285746659be"],
           # profiles/k_pair_fp64_sym_disc_N65536_order8_dram.md: 11.32 MB read + 38.03 MB written
           "bytes_per_launch": 11.32e6 + 38.03e6}


# FP64 instructions per pair interaction (ordered pair) of the double-double
# evaluation kernel at 4096 bodies, k_dd_pair_sym<3> (each unordered pair once),
# from one ncu capture (profiles/), valid while its source is the one captured.
DD_INSTR = {"files": ["paper_2006_02501_gb300/csrc/dd.cu", "paper_2006_02501_gb300/csrc/dd.cuh"],
            "sha256": ["35a3a503fc226f03d335d5dbb94d40af14ca79471c0ad7aec442c2df68240110",
                       "f43f2591663c27103bf9ee43e6dda962e4fc0d99eef95b3953edd99ba0cb6c9a"],
            # profiles/k_dd_pair_sym_disc_N4096_order8.md: 15.85e9 FP64 thread
            # instructions for 4096 x 4095 pair interactions
            "fp64_thread_instr_per_interaction": 945.0}
FP64_LANE_INSTR_PER_S = N_SM * 2 * SM_MAX_MHZ * 1e6


def _sha(path):
    with open(os.path.join(ROOT, path), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.3)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [t.strip() for t in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def workload():
    from paper_2006_02501_gb300 import inputs
    return inputs.smbh_disc(seed=SEED, N=N_STARS)


def cpu_oracle_rate(m, x, v, target_s: float, min_i: int = 64):
    """Pair interactions per second of the oracle's 8th-order evaluation over a
    sample of bodies (all N sources), sized to take about target_s seconds."""
    import oracle
    from paper_2006_02501_gb300 import inputs  # noqa: F401  (same inputs module as the GPU path)
    N = len(m)
    traj = np.zeros((N, 4, 3))
    traj[:, 0], traj[:, 1] = x, v
    # a and a-dot inputs: any values are valid for timing; use the Kepler field
    r = x - x[0]
    d = np.linalg.norm(r, axis=1)
    d[0] = 1.0
    traj[:, 2] = -r / d[:, None] ** 3
    oracle.evaluate(m, traj, EPS, i0=0, i1=min_i)                  # warm-up and calibration
    t0 = time.perf_counter()
    oracle.evaluate(m, traj, EPS, i0=0, i1=min_i)
    dt = time.perf_counter() - t0
    n_i = int(min(N, max(min_i, min_i * target_s / max(dt, 1e-6))))
    t0 = time.perf_counter()
    oracle.evaluate(m, traj, EPS, i0=0, i1=n_i)
    dt = time.perf_counter() - t0
    return n_i * (N - 1) / dt, n_i, dt


def omp_threads():
    v = os.environ.get("OMP_NUM_THREADS")
    return int(v) if v and v.isdigit() else (os.cpu_count() or 1)


def run_reference(args, rank):
    if rank != 0:
        return
    m, x, v = workload()
    N = len(m)
    rate0, n_i, _ = cpu_oracle_rate(m, x, v, target_s=3.0)
    import oracle
    traj = np.zeros((N, 4, 3))
    traj[:, 0], traj[:, 1] = x, v
    for _ in range(args.warmup):
        oracle.evaluate(m, traj, EPS, i0=0, i1=n_i)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.evaluate(m, traj, EPS, i0=0, i1=n_i)
    el = time.perf_counter() - t0
    value = args.steps * n_i * (N - 1) / el
    sample = f"8th-order evaluation of bodies 0..{n_i - 1} against all {N} bodies per step"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": config_dict(N, "reference"),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": omp_threads(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def config_dict(N, impl):
    return {"workload": f"smbh_disc_N{N_STARS}_order{ORDER}_fp64_shared_pec{N_ITER}",
            "bodies": N, "order": ORDER, "n_iter": N_ITER, "dt": DT, "eps": EPS, "seed": SEED,
            "pair_interactions_per_step": N_ITER * N * (N - 1),
            "l2": "flushed between timed steps (256 MB device write)" if impl == "ours" else "n/a",
            "parallelism": "replicas (one system per GPU)"}


def time_steps(sim, stream, torch, steps, flush):
    """Per-step device times (ms) with CUDA events on the simulation's stream."""
    times = []
    for _ in range(steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.step(DT, N_ITER)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    return times


def time_steps_batch(b, stream, torch, steps):
    """Seconds of one persistent batched launch of `steps` steps (CUDA events)."""
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    b.step(steps, 2)
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) * 1e-3


def reduce_max(val: float, world: int) -> float:
    """Maximum of a per-rank value over all ranks (the job's time is the slowest
    rank's); the tensor lives where the process group's backend wants it."""
    if world == 1:
        return val
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([val], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world: int, units_per_rank: float, seconds_max: float) -> float:
    """Whole-job throughput: every rank advances its own replica (weak scaling),
    so the job processes world x units in the slowest rank's time."""
    return world * units_per_rank / seconds_max


def run_ours(args, rank, world, local_rank):
    import torch
    import paper_2006_02501_gb300 as mh
    from paper_2006_02501_gb300.build import build
    if rank == 0:
        build()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.set_device(local_rank)
    stream = torch.cuda.Stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    m, x, v = workload()
    N = len(m)
    units = N_ITER * N * (N - 1)

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    # ---- FP64 form: the headline ----
    sim = mh.Simulation(ORDER, m, x, v, EPS, stream=stream)
    for _ in range(args.warmup):
        sim.step(DT, N_ITER)
    c0 = sim.counters()
    barrier()
    sim.set_timing(True)
    with ClockSampler(local_rank) as clk:
        times = time_steps(sim, stream, torch, args.steps, flush)
    barrier()
    sim.set_timing(False)
    c1 = sim.counters()
    elapsed_ms = reduce_max(sum(times), world)
    value = job_rate(world, args.steps * units, elapsed_ms * 1e-3)
    pair_launches = c1["pair_kernel_timed"] - c0["pair_kernel_timed"]
    pair_ms = (c1["pair_kernel_ms"] - c0["pair_kernel_ms"]) / max(pair_launches, 1)
    gpu_launches = c1["kernel_launches"] - c0["kernel_launches"]
    achieved = FLOPS_PER_UNORDERED_PAIR[ORDER] * N * (N - 1) / 2 / (pair_ms * 1e-3)
    same_src = all(_sha(f) == h for f, h in zip(TRAFFIC["files"], TRAFFIC["sha256"]))
    traffic = TRAFFIC["bytes_per_launch"] if same_src else None

    # ---- end to end through the public API: state in from host, step, state out ----
    _, hx, hv, hd = sim.sync()
    pin = lambda a: torch.from_numpy(a).pin_memory().numpy()
    hx, hv, hd = pin(hx), pin(hv), pin(hd)
    e2e_steps = max(1, args.steps)
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        sim.set_state(hx, hv, hd, t=0.0)
        sim.step(DT, N_ITER)
        _, hx2, hv2, hd2 = sim.sync()
    barrier()
    e2e_s = reduce_max(time.perf_counter() - t0, world)
    h2d = hx.nbytes + hv.nbytes + hd.nbytes
    d2h = hx2.nbytes + hv2.nbytes + hd2.nbytes
    sim.close()

    # ---- FP64 form with the ordered-pair kernel (every i, j evaluated), same workload ----
    simo = mh.Simulation(ORDER, m, x, v, EPS, stream=stream, symmetric=False)
    simo.step(DT, N_ITER)
    ko = 2
    o0 = simo.counters()
    barrier()
    simo.set_timing(True)
    to = time_steps(simo, stream, torch, ko, flush)
    barrier()
    o1 = simo.counters()
    simo.close()
    elo = reduce_max(sum(to), world)
    pairo_ms = (o1["pair_kernel_ms"] - o0["pair_kernel_ms"]) / max(o1["pair_kernel_timed"] - o0["pair_kernel_timed"], 1)
    acho = FLOPS_PER_PAIR[ORDER] * N * (N - 1) / (pairo_ms * 1e-3)

    # ---- FP32-pair precision form, same workload ----
    sim32 = mh.Simulation(ORDER, m, x, v, EPS, stream=stream, precision=mh.MH_PREC_FP32PAIR)
    for _ in range(max(3, args.warmup)):
        sim32.step(DT, N_ITER)
    k32 = max(10, args.steps)
    d0 = sim32.counters()
    barrier()
    sim32.set_timing(True)
    t32 = time_steps(sim32, stream, torch, k32, flush)
    barrier()
    d1 = sim32.counters()
    sim32.close()
    variant32 = d1["pair_variant"]
    kernel32 = {1: "k_pair_fp32<3,1>", 2: "k_pair_fp32<3,2>", 3: "k_pair_fp32x2<3>",
                4: "k_pair_fp32_sym<3>"}.get(variant32, "?")
    el32 = reduce_max(sum(t32), world)
    pair32_ms = (d1["pair_kernel_ms"] - d0["pair_kernel_ms"]) / max(d1["pair_kernel_timed"] - d0["pair_kernel_timed"], 1)
    flops32 = FLOPS_PER_UNORDERED_PAIR[ORDER] * N * (N - 1) / 2 if d1["pair_variant"] == 4 \
        else FLOPS_PER_PAIR[ORDER] * N * (N - 1)
    ach32 = flops32 / (pair32_ms * 1e-3)

    # ---- FP32-pair form with the ordered-pair packed kernel (variant 3), same workload ----
    simp = mh.Simulation(ORDER, m, x, v, EPS, stream=stream, precision=mh.MH_PREC_FP32PAIR, fp32_variant=3)
    for _ in range(3):
        simp.step(DT, N_ITER)
    kp = 5
    p0 = simp.counters()
    barrier()
    simp.set_timing(True)
    tp = time_steps(simp, stream, torch, kp, flush)
    barrier()
    p1 = simp.counters()
    simp.close()
    elp = reduce_max(sum(tp), world)
    pairp_ms = (p1["pair_kernel_ms"] - p0["pair_kernel_ms"]) / max(p1["pair_kernel_timed"] - p0["pair_kernel_timed"], 1)
    achp = FLOPS_PER_PAIR[ORDER] * N * (N - 1) / (pairp_ms * 1e-3)

    # ---- batched form: 4096 planetary systems, 6th order, 10^4 steps in one launch ----
    from paper_2006_02501_gb300 import inputs as _inp
    off, bm, bx, bv, pmin = _inp.planetary_systems(seed=4, S=4096)
    with mh.Batch(6, off, bm, bx, bv, pmin / 128.0, 1e-8, stream=stream) as b:
        b.tune(probe_steps=16, n_iter=2)
        b.step(10, 2)
        g0 = b.counters()
        barrier()
        tb = reduce_max(time_steps_batch(b, stream, torch, 10000), world)
        barrier()
        g1 = b.counters()
    sizes = np.diff(off)
    batch_pairs = float((sizes * (sizes - 1)).sum()) * 2 * 10000
    batch_ps = (g1["particle_steps"] - g0["particle_steps"]) / tb

    # ---- double-double form: the same disc cut to 4096 stars (8th order), and a
    # 65-body planetesimal ring at 10th order (the few-body regime it is for) ----
    from paper_2006_02501_gb300 import inputs as _inp2
    dd_out = {}
    for tag, (dm, dx, dv), d_order, d_eps, d_steps in (
            ("disc4096_order8", _inp2.smbh_disc(seed=2, N=4095), 8, EPS, 3),
            ("ring65_order10", _inp2.planetesimal_ring(seed=1, n=64, m=1e-9), 10, 0.0, 50)):
        dN = len(dm)
        with mh.DDSimulation(d_order, dm, dx, dv, d_eps, stream=stream) as dsim:
            dsim.step(DT, N_ITER, nsteps=2)
            dsim.sync()
            q0 = dsim.counters()
            barrier()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            dsim.step(DT, N_ITER, nsteps=d_steps)
            e1.record(stream)
            e1.synchronize()
            q1 = dsim.counters()
        dms = reduce_max(e0.elapsed_time(e1), world)
        dd_out[tag] = {"bodies": dN, "order": d_order, "steps": d_steps, "ms_per_step": dms / d_steps,
                       "pair_interactions_per_s": world * d_steps * N_ITER * dN * (dN - 1) / (dms * 1e-3),
                       "particle_steps_per_s": world * d_steps * dN / (dms * 1e-3),
                       "gpu_launches": q1["kernel_launches"] - q0["kernel_launches"]}
    # batched double-double: the 4096 planetary systems of the batched form, 6th order
    from paper_2006_02501_gb300 import inputs as _inp3
    boff, bbm, bbx, bbv, bpmin = _inp3.planetary_systems(seed=4, S=4096)
    with mh.DDBatch(6, boff, bbm, bbx, bbv, bpmin / 128.0, 1e-8, stream=stream) as db:
        db.step(2, 2)
        db.sync()
        r0 = db.counters()
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        db.step(20, 2)
        e1.record(stream)
        e1.synchronize()
        r1 = db.counters()
    bms = reduce_max(e0.elapsed_time(e1), world)
    bsz = np.diff(boff)
    dd_out["batched4096_order6"] = {
        "workload": "the batched form's 4096 planetary systems (3..64 bodies), 6th order, P(EC)^2, "
                    "dt_s = P_min/128, 20 steps replayed from a CUDA graph",
        "ms_per_step": bms / 20,
        "particle_steps_per_s": world * 20 * int(boff[-1]) / (bms * 1e-3),
        "pair_interactions_per_s": world * 20 * 2 * float((bsz * (bsz - 1)).sum()) / (bms * 1e-3),
        "gpu_launches": r1["kernel_launches"] - r0["kernel_launches"]}
    dd_pair_rate = dd_out["disc4096_order8"]["pair_interactions_per_s"] / world
    dd_src = all(_sha(f) == h for f, h in zip(DD_INSTR["files"], DD_INSTR["sha256"]))
    dd_instr = DD_INSTR["fp64_thread_instr_per_interaction"] if dd_src else None
    dd_out["pair_kernel"] = "k_dd_pair_sym<3> (each unordered pair once)"
    dd_out["fp64_thread_instr_per_interaction"] = dd_instr
    dd_out["fp64_pipe_frac"] = (dd_pair_rate * dd_instr / FP64_LANE_INSTR_PER_S) if dd_instr else None
    dd_out["fp64_pipe_frac_basis"] = ("pair-interactions/s of the 4096-body step x FP64 thread "
                                      "instructions per interaction (ncu, profiles/) / (152 SMs x 2 FP64 "
                                      "lanes x 2070 MHz); null once dd.cu or dd.cuh changes")

    peaks = mh.measure_peaks()       # measured ALU rates of this GPU, reported beside the unit-count peaks
    if rank != 0:
        return
    cpu = None
    if world == 1:
        rate, n_i, dt_cpu = cpu_oracle_rate(m, x, v, target_s=10.0)
        cpu = {"value": rate, "unit": UNIT, "cores": omp_threads(), "kind": "oracle",
               "sample": f"one 8th-order evaluation of bodies 0..{n_i - 1} against all {N} bodies "
                         f"({dt_cpu:.1f} s)"}
    clocks = clk.summary()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_dict(N, "ours"),
        "particle_steps_per_s": world * args.steps * N / (elapsed_ms * 1e-3),
        "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": PEAK_FP64 / 1e12,
                     "unit": "TFLOP/s", "frac": achieved / PEAK_FP64, "traffic": traffic,
                     "kernel": "k_pair_fp64_sym<3>",
                     "flops_per_unordered_pair": FLOPS_PER_UNORDERED_PAIR[ORDER],
                     "unordered_pairs_per_launch": N * (N - 1) // 2,
                     "peak_source": "152 SMs x 2 FP64 lanes x 2 flops x 2070 MHz (nominal 1.25 TFLOP/s)",
                     "launch_ms": pair_ms, "launches": pair_launches},
        "cpu_baseline": cpu,
        "e2e": {"value": world * e2e_steps * units / e2e_s, "unit": UNIT,
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "clocks": clocks,
        "measured_alu_peaks": peaks,
        "gpu_launches": gpu_launches,
        "forms": {"fp64_ordered": {
            "value": world * ko * units / (elo * 1e-3), "unit": UNIT, "ms_per_step": elo / ko,
            "steps": ko, "pair_kernel": "k_pair_fp64<3>", "launch_ms": pairo_ms,
            "achieved_tflops": acho / 1e12, "peak_tflops": PEAK_FP64 / 1e12, "frac": acho / PEAK_FP64,
            "flops_per_pair": FLOPS_PER_PAIR[ORDER]},
            "fp32pair": {
            "value": world * k32 * units / (el32 * 1e-3), "unit": UNIT, "ms_per_step": el32 / k32,
            "steps": k32, "pair_kernel": kernel32, "launch_ms": pair32_ms,
            "flops_per_launch": flops32,
            "achieved_tflops": ach32 / 1e12, "peak_tflops": PEAK_FP32 / 1e12,
            "frac": ach32 / PEAK_FP32,
            "peak_source": "152 SMs x 128 FP32 lanes x 2 flops x 2070 MHz"},
            "fp32pair_ordered_packed": {
            "value": world * kp * units / (elp * 1e-3), "unit": UNIT, "ms_per_step": elp / kp, "steps": kp,
            "pair_kernel": "k_pair_fp32x2<3>", "launch_ms": pairp_ms, "achieved_tflops": achp / 1e12,
            "peak_tflops": PEAK_FP32 / 1e12, "frac": achp / PEAK_FP32, "flops_per_pair": FLOPS_PER_PAIR[ORDER]},
            "double_double": dd_out,
            "batched": {
            "workload": "4096 planetary systems (3..64 bodies), 6th order FP64, P(EC)^2, dt_s = P_min/128, "
                        "10^4 steps in one launch",
            "particle_steps_per_s": world * batch_ps, "pair_interactions_per_s": world * batch_pairs / tb,
            "seconds": tb}},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    try:
        run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
