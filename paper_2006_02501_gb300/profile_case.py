"""Run one small disc case through the library, for profilers.

    python -m paper_2006_02501_gb300.profile_case --N 16384 --precision fp64 --order 8 --steps 1

Creates an SMBH disc of N stars (same recipe as the benchmark workload, seed 2),
runs the initialisation and `steps` shared P(EC)^3 steps, then exits.  The
initialisation launches one evaluation per pass (p passes), so a profiler that
wants the first step's evaluation skips those.  FP64 evaluations use the
pair-symmetric kernel (k_pair_fp64_sym) for P <= 3 unless --ordered is given;
the 8th-order initialisation's last pass (P = 5) always runs k_pair_fp64.
--precision dd runs the double-double form (mh_dd_*) on the same disc; its
initialisation also launches one evaluation per pass (k_dd_pair_sym from 2048
bodies up, k_dd_pair with --ordered or below).
--precision all runs one step of every form on the same small disc (for a
memory checker): FP64 with the pair-symmetric and the ordered kernel, the
FP32-pair form with both (orders up to 8), the double-double form, and a
double-double batch of three systems cut from the disc.
--precision batch runs the batched form instead: --N planetary systems of 3 to
64 bodies (the bench's recipe, seed 4), 6th order, P(EC)^2, dt = P_min/128,
--steps steps in one launch after a fixed configuration (6 warps per CTA,
largest systems first), so that the profiled launch is the first k_batch one.
"""
import argparse
import os
import sys

import numpy as np


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--N", type=int, default=16384)
    ap.add_argument("--precision", choices=["fp64", "fp32pair", "dd", "all", "batch"], default="fp64")
    ap.add_argument("--order", type=int, default=8)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--n-iter", type=int, default=3)
    ap.add_argument("--ordered", action="store_true",
                    help="FP64: evaluate every ordered pair instead of each unordered pair once")
    a = ap.parse_args()
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import paper_2006_02501_gb300 as mh
    from paper_2006_02501_gb300 import inputs
    mh.build_library()
    if a.precision == "batch":
        off, m, x, v, pmin = inputs.planetary_systems(seed=4, S=a.N)
        with mh.Batch(6, off, m, x, v, pmin / 128.0, 1e-8) as b:
            b.step(a.steps, 2)
            ok = bool(np.isfinite(b.sync()[1]).all())
        print(f"ok batch systems {a.N} bodies {int(off[-1])} steps {a.steps} finite={ok}")
        return
    m, x, v = inputs.smbh_disc(seed=2, N=a.N)
    dt = 2 * np.pi * 1e-3
    if a.precision == "all":
        runs = [("fp64 pair-symmetric", mh.MH_PREC_FP64, 2), ("fp64 ordered", mh.MH_PREC_FP64, 0)]
        if a.order <= 8:
            runs += [("fp32pair pair-symmetric", mh.MH_PREC_FP32PAIR, 2), ("fp32pair ordered", mh.MH_PREC_FP32PAIR, 0)]
        for name, prec, sym in runs:
            with mh.Simulation(a.order, m, x, v, 1e-4, precision=prec, symmetric=sym) as sim:
                sim.step(dt, a.n_iter, nsteps=a.steps)
                sim.diagnostics(central=0)
                ok = bool(np.isfinite(sim.sync()[1]).all())
            print(f"ok {name} N={len(m)} order {a.order} finite={ok}")
        with mh.DDSimulation(a.order, m, x, v, 1e-4) as sim:
            sim.step(dt, a.n_iter, nsteps=a.steps)
            sim.diagnostics(central=0)
            print(f"ok dd N={len(m)} order {a.order} finite={bool(np.isfinite(sim.sync()[1]).all())}")
        off = np.array([0, 1, 3, min(len(m), 64)], dtype=np.int64)
        k = int(off[-1])
        with mh.DDBatch(a.order, off, m[:k], x[:k], v[:k], np.full(3, dt), 1e-4) as b:
            b.step(a.steps, a.n_iter)
            b.energies()
            print(f"ok dd batch systems {np.diff(off).tolist()} finite={bool(np.isfinite(b.sync()[1]).all())}")
        return
    if a.precision == "dd":
        with mh.DDSimulation(a.order, m, x, v, 1e-4, symmetric=0 if a.ordered else 1) as sim:
            sim.step(2 * np.pi * 1e-3, a.n_iter, nsteps=a.steps)
            t2, x2, v2, d2 = sim.sync()
        print(f"ok N={len(m)} dd order {a.order} steps {a.steps} t={t2[0]:.6f} "
              f"finite={bool(np.isfinite(x2).all())}")
        return
    prec = mh.MH_PREC_FP64 if a.precision == "fp64" else mh.MH_PREC_FP32PAIR
    with mh.Simulation(a.order, m, x, v, 1e-4, precision=prec, symmetric=not a.ordered) as sim:
        sim.step(2 * np.pi * 1e-3, a.n_iter, nsteps=a.steps)
        t, xs, vs, ds = sim.sync()
    print(f"ok N={len(m)} {a.precision} order {a.order} steps {a.steps} t={t:.6f} "
          f"finite={bool(np.isfinite(xs).all())}")


if __name__ == "__main__":
    main()
