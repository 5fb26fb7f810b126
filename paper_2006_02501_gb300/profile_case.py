"""Run one small disc case through the library, for profilers.

    python -m paper_2006_02501_gb300.profile_case --N 16384 --precision fp64 --order 8 --steps 1

Creates an SMBH disc of N stars (same recipe as the benchmark workload, seed 2),
runs the initialisation and `steps` shared P(EC)^3 steps, then exits.  The
initialisation launches one evaluation per pass (p passes), so a profiler that
wants the first step's evaluation skips those.  FP64 evaluations use the
pair-symmetric kernel (k_pair_fp64_sym) for P <= 3 unless --ordered is given;
the 8th-order initialisation's last pass (P = 5) always runs k_pair_fp64.
--precision dd runs the double-double form (mh_dd_*) on the same disc; its
initialisation also launches one evaluation (k_dd_pair) per pass.
"""
import argparse
import os
import sys

import numpy as np


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--N", type=int, default=16384)
    ap.add_argument("--precision", choices=["fp64", "fp32pair", "dd"], default="fp64")
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
    m, x, v = inputs.smbh_disc(seed=2, N=a.N)
    if a.precision == "dd":
        with mh.DDSimulation(a.order, m, x, v, 1e-4) as sim:
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
