"""Write tests/golden/c2_trajectory_fp64.txt: the FP64 oracle's run of the
1024 x 1024, n = 3 workload (sign-split iid N(0,1) field projected by the
oracle, tau = 3 h^2) for 200 steps of Algorithm 1 at the stationarity
tolerance 1e-4, one line per step: step, E^tau(A_s), max |A_{s+1} - A_s|,
det-sign flips.  Calls only the oracle; run from the repository root:

    python tests/golden/make_c2_trajectory.py
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
from paper_1711_01365_gb300 import inputs as I  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "c2_trajectory_fp64.txt")
MAX_STEPS, TOL = 200, 1e-4


def main():
    O.build()
    threads = O.set_threads(0)
    F, n, tau = I.config_field("C2")
    A0 = O.project(F, n)
    t0 = time.time()
    _, info = O.run(A0, n, tau, MAX_STEPS, TOL)
    dt = time.time() - t0
    s = info["steps"]
    with open(OUT, "w") as f:
        f.write("# FP64 oracle run of the 1024x1024 n=3 sign-split workload, tau=3h^2, "
                f"max_steps={MAX_STEPS}, tol={TOL:g}\n")
        f.write(f"# steps={s} stationary={int(info['stationary'])} "
                f"(oracle threads {threads}, {dt:.0f} s)\n")
        f.write("# step energy max_delta det_flips  (energy of A_s; last line: energy of the final field)\n")
        for k in range(s):
            f.write(f"{k} {info['energies'][k]:.17e} {info['max_deltas'][k]:.17e} "
                    f"{int(info['det_flips'][k])}\n")
        f.write(f"{s} {info['energies'][s]:.17e} nan -1\n")
    print(OUT, s, info["stationary"], f"{dt:.0f} s")


if __name__ == "__main__":
    main()
