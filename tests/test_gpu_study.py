"""Disk analogues of the paper's experiments (Sec. 6, Example 1 and Table 3 of Example 3) run
through the library: every configuration conserves flux, and the qualitative findings the paper
reports hold for disks too -- a layered background does not change the iteration count much
against a homogeneous one (the multiple scattering is dominated by the inclusions), and the count
grows with the middle wavenumber k2 (the paper: 13, 15, 43, 83 iterations for k2 = 1, 10, 20, 30).
Iteration counts themselves are not compared with the paper's (its inclusions are stars)."""
import os
import sys

import pytest

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_paper_experiment_analogues():
    sys.path.insert(0, ROOT)
    import bench
    out = bench.run_study(0)
    print(out)
    for row in out["example1"] + out["example3"]:
        assert row["relres"] <= 1e-10 and row["flux_err"] < 1e-9, row
    ex1 = {(r["M"], r["background"]): r["iters"] for r in out["example1"]}
    for M in (100, 500, 1000):
        h, l = ex1[(M, "homogeneous")], ex1[(M, "layered")]
        assert abs(h - l) <= 0.5 * max(h, l), (M, h, l)
    its = [r["iters"] for r in out["example3"]]
    assert its[-1] > its[0], its
