"""Measurements across the forms of the integrator (one GPU).

    python -m paper_2006_02501_gb300.compare_forms ecc      # FP64 vs FP32-pair at equal ecc-vector error
    python -m paper_2006_02501_gb300.compare_forms block    # block steps, FP32-pair vs FP64, N = 262144
    python -m paper_2006_02501_gb300.compare_forms batch    # 4096 planetary systems, 10^4 steps
    python -m paper_2006_02501_gb300.compare_forms learned  # learned predictor on the N = 65536 disc
    python -m paper_2006_02501_gb300.compare_forms table1   # Section 3.3 disc, time-symmetric steps

Each prints JSON lines.  Throughputs are timed with CUDA events on the
simulation's stream; pair interactions and particle steps come from the
library's counters.  Eccentricity-vector error: the median over the stars of
|e_i - e_i^ref| at the end time, e about the SMBH (Appendix A, Eq. A1), with the
reference an 8th-order FP64 run at a quarter of the step and P(EC)^4.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np


def _setup():
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch
    import paper_2006_02501_gb300 as mh
    from paper_2006_02501_gb300 import inputs
    mh.build_library()
    torch.cuda.set_device(0)
    return torch, mh, inputs


def _timed(torch, stream, fn):
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) * 1e-3


def _ecc_err(e, e_ref):
    return float(np.median(np.linalg.norm(e[1:] - e_ref[1:], axis=1)))


def run_ecc(args):
    """SMBH disc (N stars + SMBH), 8th order, shared steps P(EC)^3: FP64 and
    FP32-pair forms at dt0 and dt0/2 over the same time, against a reference."""
    torch, mh, I = _setup()
    st = torch.cuda.Stream()
    m, x, v = I.smbh_disc(seed=2, N=args.N)
    eps, dt0, nst = 1e-4, 2 * np.pi * 1e-3, args.steps
    T = nst * dt0
    with mh.Simulation(8, m, x, v, eps, stream=st) as ref:
        ref.step(dt0 / 4, args.ref_passes, nsteps=4 * nst)
        _, e_ref = ref.diagnostics(central=0)
    rows = []
    for prec, name in ((mh.MH_PREC_FP64, "fp64"), (mh.MH_PREC_FP32PAIR, "fp32pair")):
        for div in (args.fp64_divs if name == "fp64" else (1, 2)):
            dt = dt0 / div
            with mh.Simulation(8, m, x, v, eps, stream=st, precision=prec) as s:
                c0 = s.counters()
                sec = _timed(torch, st, lambda: s.step(dt, 3, nsteps=nst * div))
                c1 = s.counters()
                E, e = s.diagnostics(central=0)
            row = {"form": name, "dt": dt, "steps": nst * div, "time_s": sec,
                   "particle_steps_per_s": (c1["particle_steps"] - c0["particle_steps"]) / sec,
                   "pair_interactions_per_s": (c1["pair_interactions"] - c0["pair_interactions"]) / sec,
                   "ecc_err_median": _ecc_err(e, e_ref), "N": len(m), "t_end": T}
            rows.append(row)
            print(json.dumps(row), flush=True)
    # equal-error comparison: the error each form reaches at dt0 and dt0/2, and the
    # throughput of each at the finer step that reaches the FP64 error at dt0
    target = [r for r in rows if r["form"] == "fp64" and r["dt"] == dt0][0]["ecc_err_median"]
    summary = {"equal_error_target": target}
    for name in ("fp64", "fp32pair"):
        ok = [r for r in rows if r["form"] == name and r["ecc_err_median"] <= target * 1.05]
        best = max(ok, key=lambda r: r["particle_steps_per_s"]) if ok else None
        summary[name] = None if best is None else {k: best[k] for k in ("dt", "particle_steps_per_s",
                                                                          "ecc_err_median")}
    print(json.dumps({"summary": summary}), flush=True)


def run_block(args):
    """Block time steps on the SMBH disc (N stars + SMBH, total star mass 0.01,
    seed 3): FP32-pair and FP64 forms from the same start over
    args.dtmax_units x dt_max (dt_max = 2^-5, levels k <= 12, eta = 0.05),
    8th and 6th order."""
    torch, mh, I = _setup()
    st = torch.cuda.Stream()
    m, x, v = I.smbh_disc(seed=3, N=args.N)
    eps = 1e-4
    blk = dict(dt_max=2.0 ** -5, k_max=12, eta=0.05)
    span = args.dtmax_units * blk["dt_max"]
    forms = [(p, n) for p, n in ((mh.MH_PREC_FP32PAIR, "fp32pair"), (mh.MH_PREC_FP64, "fp64")) if n in args.forms]
    for order in args.orders:
        out = {}
        for prec, name in forms:
            with mh.Simulation(order, m, x, v, eps, stream=st, precision=prec, block=blk) as s:
                lv = s.levels()
                E0 = s.energy()
                c0 = s.counters()
                if args.chunk_dtmax > 0:
                    # progress lines every chunk_dtmax x dt_max (long runs)
                    sec, done = 0.0, 0
                    while done < args.dtmax_units:
                        k = min(args.chunk_dtmax, args.dtmax_units - done)
                        sec += _timed(torch, st, lambda: s.step(k * blk["dt_max"], 3))
                        done += k
                        print(json.dumps({"progress": name, "order": order, "dtmax_done": done, "seconds": sec,
                                          "dE_rel": s.energy() / E0 - 1}), flush=True)
                else:
                    sec = _timed(torch, st, lambda: s.step(span, 3))
                c1 = s.counters()
                E1, e = s.diagnostics(central=0)
            out[name] = {"time_s": sec, "particle_steps": c1["particle_steps"] - c0["particle_steps"],
                         "particle_steps_per_s": (c1["particle_steps"] - c0["particle_steps"]) / sec,
                         "pair_interactions_per_s": (c1["pair_interactions"] - c0["pair_interactions"]) / sec,
                         "block_steps": c1["steps"] - c0["steps"], "dE_rel": E1 / E0 - 1,
                         "levels": np.bincount(lv, minlength=blk["k_max"] + 1).tolist(), "e": e}
        row = {"order": order, "N": len(m), "span": span}
        if len(out) == 2:
            row["dE_rel_difference"] = abs(out["fp32pair"]["dE_rel"] - out["fp64"]["dE_rel"])
            row["ecc_median_difference_fp32_vs_fp64"] = _ecc_err(out["fp32pair"]["e"], out["fp64"]["e"])
        for name in out:
            out[name].pop("e")
            row[name] = out[name]
        print(json.dumps(row), flush=True)


def run_batch(args):
    """4096 planetary systems (3..64 bodies), 6th order, P(EC)^2, dt_s = P_min/128,
    10^4 steps in one launch; the single-system path on a subset for comparison."""
    torch, mh, I = _setup()
    st = torch.cuda.Stream()
    off, m, x, v, pmin = I.planetary_systems(seed=4, S=args.S)
    dt = pmin / 128.0
    eps = 1e-8
    with mh.Batch(6, off, m, x, v, dt, eps, stream=st) as b:
        t0 = time.perf_counter()
        w, o = b.tune(probe_steps=16, n_iter=2)
        tune_s = time.perf_counter() - t0
        E0 = b.energies()
        c0 = b.counters()
        sec = _timed(torch, st, lambda: b.step(args.steps, 2))
        c1 = b.counters()
        E1 = b.energies()
    sizes = np.diff(off)
    pairs = float((sizes * (sizes - 1)).sum()) * 2 * args.steps
    dE = np.abs(E1 / E0 - 1)
    row = {"form": "batched", "systems": args.S, "bodies": int(off[-1]), "steps": args.steps, "time_s": sec,
           "particle_steps_per_s": (c1["particle_steps"] - c0["particle_steps"]) / sec,
           "pair_interactions_per_s": pairs / sec, "autotune": {"warps": w, "order": o, "seconds": tune_s},
           "dE_rel_median": float(np.median(dE)), "dE_rel_max": float(dE.max())}
    print(json.dumps(row), flush=True)
    # the single-system path (one simulation per system) on a subset
    k_sub, n_sub = args.subset, args.subset_steps
    tot_ps, tot_s = 0.0, 0.0
    for k in range(k_sub):
        sl = slice(off[k], off[k + 1])
        with mh.Simulation(6, m[sl], x[sl], v[sl], eps, stream=st) as s:
            s.step(dt[k], 2, nsteps=5)
            sec = _timed(torch, st, lambda: s.step(dt[k], 2, nsteps=n_sub))
            tot_ps += (off[k + 1] - off[k]) * n_sub
            tot_s += sec
    print(json.dumps({"form": "single-system path (subset)", "systems": k_sub, "steps": n_sub,
                      "particle_steps_per_s": tot_ps / tot_s}), flush=True)


def run_learned(args):
    """Learned predictor: trained on converged steps of N-star discs (seeds 100+),
    evaluated on a fresh seed-1000 disc: fraction of bodies converged to 1e-13
    (relative to the 16-pass result) after n passes, plain vs learned.  A global
    max-norm criterion is not reachable on this disc: star-star passages faster
    than dt keep a few bodies from contracting at all."""
    torch, mh, I = _setup()
    from paper_2006_02501_gb300 import train_predictor as tp
    st = torch.cuda.Stream()
    eps, dt, tol = 1e-4, 2 * np.pi * 1e-3, 1e-13
    Fs, Ts = [], []
    rows = 0
    seed = 100
    t0 = time.perf_counter()
    while rows < args.samples:
        m, x, v = I.smbh_disc(seed=seed, N=args.N)
        with mh.Simulation(8, m, x, v, eps, stream=st) as s:
            steps = min(args.steps_per_disc, -(-(args.samples - rows) // len(m)))
            F, T = tp.collect(s, dt, steps=steps, n_iter=10)
        Fs.append(F)
        Ts.append(T)
        rows += F.shape[0]
        seed += 1
    collect_s = time.perf_counter() - t0
    F, T = torch.cat(Fs), torch.cat(Ts)
    t0 = time.perf_counter()
    net = tp.fit((F, T), epochs=args.epochs, seed=0)
    train_s = time.perf_counter() - t0
    # evaluation: a fresh disc, a few plain steps so the stack holds interpolated
    # derivatives, then from one state: the fraction of bodies whose position after
    # n passes is within tol (relative) of the 16-pass result, plain vs learned
    m, x, v = I.smbh_disc(seed=1000, N=args.N)
    with mh.Simulation(8, m, x, v, eps, stream=st) as s:
        s.step(dt, 3, nsteps=3)
        t, x0, v0, d0 = s.sync()
        s.step(dt, 16)
        _, xr, _, _ = s.sync()
    scale = np.linalg.norm(xr, axis=1)
    res = {"n": list(range(1, args.max_passes + 1))}
    for name, use in (("plain", False), ("learned", True)):
        frac = []
        for n in res["n"]:
            with mh.Simulation(8, m, x0, v0, eps, stream=st) as s:
                s.set_state(x0, v0, d0, t=t)
                if use:
                    s.set_predictor(net)
                s.step(dt, n)
                _, xs, _, _ = s.sync()
            err = np.linalg.norm(xs - xr, axis=1)
            frac.append(float(np.mean(err <= tol * scale)))
        res[name + "_fraction_converged"] = frac
    print(json.dumps({"N": len(m), "training_rows": int(F.shape[0]), "collect_s": collect_s, "train_s": train_s,
                      "tol": tol, **res}), flush=True)
    # equal-error comparison: eccentricity-vector error after K steps from the
    # same state (reference: dt/4, P(EC)^4) and particle-steps/s, plain P(EC)^n
    # against learned P(EC)^n, on fresh discs.  The eccentricity vectors are
    # relative to the SMBH, so an error of the SMBH's own trajectory moves
    # every star's vector; the error is also given with the SMBH's state taken
    # from the reference ("stars_only"), and the SMBH's position error itself.
    def ecc_rows(m_, x_, v_, xc, vc):
        mu = m_[0] + m_[1:]
        r, u = x_[1:] - xc, v_[1:] - vc
        rn = np.linalg.norm(r, axis=1)[:, None]
        return ((u * u).sum(1)[:, None] / mu[:, None] - 1.0 / rn) * r - (r * u).sum(1)[:, None] * u / mu[:, None]
    for eval_seed in args.eval_seeds:
        m, x, v = I.smbh_disc(seed=eval_seed, N=args.N)
        with mh.Simulation(8, m, x, v, eps, stream=st) as s:
            s.step(dt, 3, nsteps=3)
            t, x0, v0, d0 = s.sync()
        for K in args.ecc_steps:
            with mh.Simulation(8, m, x0, v0, eps, stream=st) as s:
                s.set_state(x0, v0, d0, t=t)
                s.step(dt / 4, 4, nsteps=4 * K)
                _, xr, vr, _ = s.sync()
            e_ref = ecc_rows(m, xr, vr, xr[0], vr[0])
            rows = []
            for name, use in (("plain", False), ("learned", True)):
                for n in (1, 2, 3, 4):
                    if use and n == 4:
                        continue
                    with mh.Simulation(8, m, x0, v0, eps, stream=st) as s:
                        s.set_state(x0, v0, d0, t=t)
                        if use:
                            s.set_predictor(net)
                        s.step(dt, n)                       # warm-up (graphs, tuner)
                        s.set_state(x0, v0, d0, t=t)
                        sec = _timed(torch, st, lambda: s.step(dt, n, nsteps=K))
                        _, xs, vs, _ = s.sync()
                    e = ecc_rows(m, xs, vs, xs[0], vs[0])
                    e_st = ecc_rows(m, xs, vs, xr[0], vr[0])
                    rows.append({"predictor": name, "n": n,
                                 "ecc_error": float(np.median(np.linalg.norm(e - e_ref, axis=1))),
                                 "ecc_error_stars_only": float(np.median(np.linalg.norm(e_st - e_ref, axis=1))),
                                 "smbh_dx": float(np.linalg.norm(xs[0] - xr[0])),
                                 "particle_steps_per_s": K * len(m) / sec, "ms_per_step": 1e3 * sec / K})
            print(json.dumps({"N": len(m), "seed": eval_seed, "steps": K, "dt": dt, "ecc_vs_reference": rows}),
                  flush=True)


def run_table1(args):
    """Section 3.3 N-body test: 100 bodies of 1e-5 around a unit mass, a
    log-spaced in [0.1, 10], Rayleigh e, i with sigma_i = 2 sigma_e = 0.12,
    eps = 1e-6, 8th order, time-symmetric variable shared step (Eq. 24), run to
    t = 100 pi; the median |E - E0|/|E0| over the last time unit, per (n, eta)."""
    torch, mh, I = _setup()
    st = torch.cuda.Stream()
    m, x, v = I.disc_100(seed=args.seed)
    t_end = args.t_end
    for n_iter in args.n:
        for eta in args.eta:
            with mh.Simulation(args.order, m, x, v, 1e-6, stream=st, timesym_eta=eta) as sim:
                E0 = sim.energy()
                t, steps, samples = 0.0, 0, []
                w0 = time.perf_counter()
                while t < t_end:
                    # coarse chunks until just before the last time unit (sized from the
                    # mean step so far), then sample every few steps
                    if t < t_end - 1.2 and steps > 0:
                        chunk = int(min(args.chunk, max(args.sample_every, (t_end - 1.2 - t) / (t / steps))))
                    elif t < t_end - 1.2:
                        chunk = args.sample_every
                    else:
                        chunk = args.sample_every
                    sim.step_timesym(chunk, n_iter)
                    steps += chunk
                    t = sim.sync()[0]
                    if t >= t_end - 1.0:
                        samples.append(abs(sim.energy() / E0 - 1))
                wall = time.perf_counter() - w0
            print(json.dumps({"case": "table1", "order": args.order, "n": n_iter, "eta": eta, "t": t,
                              "steps": steps, "median_dE_last_unit": float(np.median(samples)),
                              "samples": len(samples), "seconds": wall, "us_per_step": wall / steps * 1e6,
                              "seed": args.seed}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    sub = ap.add_subparsers(dest="cmd", required=True)
    a = sub.add_parser("ecc")
    a.add_argument("--N", type=int, default=16384)
    a.add_argument("--steps", type=int, default=40)
    a.add_argument("--ref-passes", type=int, default=4)
    a.add_argument("--fp64-divs", type=int, nargs="+", default=[1, 2])
    b = sub.add_parser("block")
    b.add_argument("--N", type=int, default=262144)
    b.add_argument("--dtmax-units", type=int, default=1)
    b.add_argument("--chunk-dtmax", type=int, default=0)
    b.add_argument("--orders", type=int, nargs="+", default=[8, 6])
    b.add_argument("--forms", nargs="+", default=["fp32pair", "fp64"], choices=["fp32pair", "fp64"])
    c = sub.add_parser("batch")
    c.add_argument("--S", type=int, default=4096)
    c.add_argument("--steps", type=int, default=10000)
    c.add_argument("--subset", type=int, default=16)
    c.add_argument("--subset-steps", type=int, default=200)
    d = sub.add_parser("learned")
    d.add_argument("--N", type=int, default=65536)
    d.add_argument("--samples", type=int, default=1_000_000)
    d.add_argument("--steps-per-disc", type=int, default=8)
    d.add_argument("--epochs", type=int, default=30)
    d.add_argument("--max-passes", type=int, default=6)
    d.add_argument("--ecc-steps", type=int, nargs="+", default=[10])
    d.add_argument("--eval-seeds", type=int, nargs="+", default=[1000])
    t1 = sub.add_parser("table1")
    t1.add_argument("--n", type=int, nargs="+", default=[3, 4])
    t1.add_argument("--eta", type=float, nargs="+", default=[0.08, 0.04, 0.02, 0.01, 0.005])
    t1.add_argument("--order", type=int, default=8)
    t1.add_argument("--t-end", type=float, default=100 * np.pi)
    t1.add_argument("--seed", type=int, default=5)
    t1.add_argument("--chunk", type=int, default=4000)
    t1.add_argument("--sample-every", type=int, default=20)
    args = ap.parse_args()
    {"ecc": run_ecc, "block": run_block, "batch": run_batch, "learned": run_learned,
     "table1": run_table1}[args.cmd](args)


if __name__ == "__main__":
    main()
