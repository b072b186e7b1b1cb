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


@pytest.mark.parametrize("case", ["example1_homogeneous", "example1_layered", "example3_k2_20"])
def test_study_configurations_against_oracle(case):
    """Study configurations solved by the library against the oracle: Example 1 with M = 100 disks
    (k_p = 30, p = 10) in the homogeneous k = (10, 10, 10) and layered k = (10, 8, 10) backgrounds
    near the k1 = 10 Wood angle, and Example 3 at k2 = 20 with disks crossing the walls.  The
    reference is the oracle's matrix-free GMRES solution to 1e-13: on Example 1 the dense
    preconditioned matrix has a condition number near 1e24 (the products s_n H_q(k2 R) of tiny
    high-order disk coefficients and huge close-pair Hankel values span ~30 decades), and the
    oracle's own LU and GMRES solutions differ by 2.5e-9 in the Bragg amplitudes there, whatever
    the GMRES tolerance.  Bragg amplitudes to 1e-9 norm-wise; element-wise to 1e-8 on Example 1
    (weakest order 1e-2 of the norm), 1e-9 on Example 3."""
    import math

    import workloads as W
    from bragg import check as check_bragg
    from oracle import solver as S
    from paper_1412_7466_gb300 import GratingSolver
    base = W.grating("small")
    g = dict(base)
    if case.startswith("example1"):
        g["k"] = (10.0, 10.0, 10.0) if case.endswith("homogeneous") else (10.0, 8.0, 10.0)
        theta = -math.acos(1.0 - 2.0 * math.pi / 10.0) + 0.1
        dk = W.disks(100, 0.025, 0.0125, 3.0, 10.0, seed=100, p=10)
    else:
        g["k"] = (5.0, 20.0, 5.0)
        theta = -math.pi / 5
        dk = W.disks(100, 0.025, 0.0125, 1.6, 5.0, seed=3, p=10)
    gs = GratingSolver(0)
    gs.set_layers(g)
    gs.set_incidence([theta])
    gs.set_inclusions(dk)
    gs.factor()
    gs.solve(tol=1e-12, maxit=4000, restart=500)
    got = gs.bragg()
    gs.close()
    prob = S.setup(g, theta, dk)
    beta, _, _, _ = S.solve_gmres(prob, tol=1e-13, restart=500, maxit=4000)
    _, ref, _ = prob.recover(beta)
    nw, ew = check_bragg(got, ref, 1e-9, 1e-8 if case.startswith("example1") else 1e-9)
    print(case, "Bragg error vs oracle", nw, ew)
