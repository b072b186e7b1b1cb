"""Writes the stored expected values under tests/golden/ using only the oracle and the seeded
workload generator (never the CUDA path).

  python tests/golden/make_golden.py headline     # ~15 min on 8 cores: M=1000, k=(40,60,80)
  python tests/golden/make_golden.py mixed4000    # ~2 h on 8 cores: M=4000, r=0.004, GMRES(500)

Output: <name>_bragg.txt with one line per propagating order: side (c|d), n, Re, Im; and a
header with the GMRES iteration count, final relative residual and flux error.
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import workloads as W  # noqa: E402
from oracle import solver as S  # noqa: E402


# GMRES restart length per workload: GMRES(200) is enough at M = 1000; the denser M = 4000
# geometry is solved with GMRES(500), the restart the GPU solver uses.
RESTART = {"headline": 200, "mixed4000": 500}


def main(name: str):
    cfg = W.config(name)
    t0 = time.time()
    prob = S.setup(cfg["grating"], cfg["theta"], cfg["disks"])
    restart = RESTART.get(name, 200)
    beta, its, hist, _ = S.solve_gmres(prob, tol=min(cfg["tol"], 1e-12), restart=restart, maxit=3000)
    _, br, fe = prob.recover(beta)
    out = os.path.join(HERE, f"{name}_bragg.txt")
    with open(out, "w") as f:
        f.write(f"# workload {name} (workloads.config('{name}'), seed 1); oracle GMRES its {its}, "
                f"relres {hist[-1]:.3e}, flux error {fe:.3e}, GMRES({restart}), {time.time() - t0:.0f} s\n")
        for side, ns, vals in (("c", br["n_top"], br["c"]), ("d", br["n_bot"], br["d"])):
            for n, v in zip(ns, vals):
                f.write(f"{side} {int(n)} {v.real:.17e} {v.imag:.17e}\n")
    print("wrote", out)


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else "headline")
