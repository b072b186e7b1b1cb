"""The multi-angle lockstep solve (gs_solve_angles) through the C-ABI: one geometry at several
incidence angles -- one of them the Wood anomaly of k1, one normal incidence -- solved together with
FP64 refinement and either inner translation (the tensor-core product of all angles, GS_MIXED_BF16,
or each angle from the complex64 pair table, GS_C64), against the oracle's dense LU solution at each
angle (Bragg amplitudes 1e-9, norm-wise and element-wise), and against the single-angle mixed solve
of the same context."""
import math

import numpy as np
import pytest

import workloads as W
from bragg import check as check_bragg
from oracle import solver as S

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("inner", ["bf16", "c64"])
def test_angles_small_against_oracle(inner):
    from paper_1412_7466_gb300 import GS_C64, GS_MIXED_BF16, GratingSolver
    cfg = W.config("small")
    g, dk = cfg["grating"], cfg["disks"]
    thetas = [-math.pi / 5, -1.2, W.wood_angle(g["k"][0], g["d"]), -math.pi / 2, -2.2]
    gs = GratingSolver(0)
    gs.set_layers(g)
    gs.set_incidence(thetas)
    gs.set_inclusions(dk)
    gs.factor()
    gs.solve_angles(tol=1e-12, maxit=2000, restart=200, precision=GS_MIXED_BF16 if inner == "bf16" else GS_C64)
    got = [gs.bragg(angle=q) for q in range(len(thetas))]
    stats = [gs.stats(angle=q) for q in range(len(thetas))]
    for q, th in enumerate(thetas):
        prob = S.setup(g, th, dk)
        beta, _, _ = S.solve_dense(prob)
        _, ref, _ = prob.recover(beta)
        nw, ew = check_bragg(got[q], ref)
        assert stats[q][1] <= 1e-12, (q, stats[q])
        assert got[q]["flux_err"] < 1e-10
        print(f"{inner} angle {th:+.4f}: inner iterations {stats[q][0]}, sweeps {gs.refinement_sweeps(q)}, "
              f"Bragg error {nw:.1e} / {ew:.1e}")
    # the same context's single-angle mixed solve agrees
    for q in (0, 2):
        gs.solve(angle=q, tol=1e-12, maxit=2000, precision=GS_C64)
        check_bragg(gs.bragg(angle=q), got[q])
    gs.close()


@pytest.mark.parametrize("inner", ["c64", "bf16"])
def test_angles_medium_against_oracle(inner):
    """150 disks, p = 8, eight angles spread over [-pi/3, pi/3] from the downward normal, the
    Wood angle among them; sampled angles against the oracle's dense solve."""
    from paper_1412_7466_gb300 import GratingSolver
    g = W.grating("small")
    dk = W.disks(150, 0.012, 0.006, 2.0, g["k"][0], seed=71, p=8)
    phis = list(np.linspace(-math.pi / 3, math.pi / 3, 7))
    thetas = [-math.pi / 2 + f for f in phis] + [W.wood_angle(g["k"][0], g["d"])]
    gs = GratingSolver(0)
    gs.set_layers(g)
    gs.set_incidence(thetas)
    gs.set_inclusions(dk)
    gs.factor()
    from paper_1412_7466_gb300 import GS_C64, GS_MIXED_BF16
    gs.solve_angles(tol=1e-12, maxit=4000, restart=300, precision=GS_C64 if inner == "c64" else GS_MIXED_BF16)
    for q in (0, 3, 7):
        prob = S.setup(g, thetas[q], dk)
        beta, _, _ = S.solve_dense(prob)
        _, ref, _ = prob.recover(beta)
        got = gs.bragg(angle=q)
        nw, ew = check_bragg(got, ref)
        its, rr = gs.stats(angle=q)
        print(f"angle {thetas[q]:+.4f}: inner iterations {its}, sweeps {gs.refinement_sweeps(q)}, "
              f"Bragg error {nw:.1e} / {ew:.1e}")
        assert rr <= 1e-12
    gs.close()


def test_angles_refuses_fp64_and_needs_factor():
    from paper_1412_7466_gb300 import GS_ERR_ARG, GS_ERR_STATE, GS_FP64, GratingSolver, GsError, gs_solve_opts
    import ctypes
    gs = GratingSolver(0)
    g = W.grating("tiny")
    gs.set_layers(g)
    gs.set_incidence([-1.0, -0.8])
    with pytest.raises(GsError) as e:
        gs.solve_angles()
    assert e.value.status == GS_ERR_STATE
    gs.set_inclusions(W.disks(5, 0.02, 0.01, 2.0, g["k"][0], seed=2, p=4))
    gs.factor()
    o = gs_solve_opts(tol=1e-10, maxit=100, restart=50, precision=GS_FP64, inner_tol=1e-6, max_sweeps=0)
    assert gs.lib.gs_solve_angles(gs.ctx, ctypes.byref(o)) == GS_ERR_ARG
    # the complex64-table form needs the table: refused when the budget allows none
    from paper_1412_7466_gb300 import GS_C64, GS_ERR_OOM
    gs.lib.gs_set_table_budget(gs.ctx, 0.0)
    o.precision = GS_C64
    assert gs.lib.gs_solve_angles(gs.ctx, ctypes.byref(o)) == GS_ERR_OOM
    gs.close()
