"""GPU parity: every step of the CUDA path (called through the C-ABI) against the oracle on the
same seeded inputs.  Floating-point tolerances: assembled matrices agree to 1e-10 of each block's
largest entry (two independent FP64 evaluations of the same formulas, with different Bessel
implementations); the translation and the operator to 1e-12 relative (norm); Bragg amplitudes to
the stated 1e-9 relative (the FP64 path's target), norm-wise over the propagating orders and for
every single amplitude (element-wise), with the propagating orders equal."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import inclusions as I
from oracle import layers as L
from oracle import solver as S
from bragg import check as check_bragg

pytestmark = pytest.mark.gpu

BRAGG_TOL = 1e-9


def _solver():
    from paper_1412_7466_gb300 import GratingSolver
    return GratingSolver(0)


def _setup_gpu(cfg_grating, theta, disks):
    gs = _solver()
    gs.set_layers(cfg_grating)
    gs.set_incidence([theta])
    gs.set_inclusions(disks)
    gs.factor()
    return gs


@pytest.fixture(scope="module")
def small():
    cfg = W.config("small")
    prob = S.setup(cfg["grating"], cfg["theta"], cfg["disks"])
    gs = _setup_gpu(cfg["grating"], cfg["theta"], cfg["disks"])
    yield cfg, prob, gs
    gs.close()


def _np(t):
    return t.detach().cpu().numpy()


def _blocks(eg):
    return [(rn, rs, cn, cs) for rn, rs in eg.rows.items() for cn, cs in eg.cols.items()]


def test_assembled_A_matches_oracle(small):
    cfg, prob, gs = small
    A = _np(gs.get_A())
    Ao = prob.eg.A
    assert A.shape == Ao.shape
    for rn, rs, cn, cs in _blocks(prob.eg):
        blk_o = Ao[rs, cs]
        scale = np.max(np.abs(blk_o))
        err = np.max(np.abs(A[rs, cs] - blk_o))
        assert err <= 1e-10 * max(scale, 1e-300), (rn, cn, err, scale)


def test_rhs_f_matches_oracle(small):
    cfg, prob, gs = small
    np.testing.assert_allclose(_np(gs.get_f()), prob.eg.f, atol=1e-13)


def test_scattering_diagonal(small):
    cfg, prob, gs = small
    s = _np(gs.get_scattering())
    np.testing.assert_allclose(s, prob.s, rtol=1e-11, atol=1e-300)


def test_coupling_B_C(small):
    cfg, prob, gs = small
    B, Cm = gs.get_coupling()
    B, Cm = _np(B), _np(Cm)
    nB = B.shape[1]
    Bo = prob.B[:, :nB]
    assert np.all(prob.B[:, nB:] == 0)
    for blk in ("mu1", "sigma1", "mu2", "sigma2", "a2"):
        sl = prob.eg.cols[blk]
        sc = np.max(np.abs(Bo[:, sl]))
        assert np.max(np.abs(B[:, sl] - Bo[:, sl])) <= 1e-11 * sc, blk
    nC = Cm.shape[0]
    Co = prob.C[:nC]
    assert np.all(prob.C[nC:] == 0)
    sc = np.max(np.abs(Co))
    assert np.max(np.abs(Cm - Co)) <= 1e-11 * sc


def test_empty_grating_pseudo_inverse(small):
    """A^+ f from the GPU Jacobi SVD gives the oracle's empty-grating Bragg amplitudes."""
    cfg, prob, gs = small
    x = _np(gs.pinv_apply(gs.get_f()))
    xo = prob.pinv.apply(prob.eg.f)
    for blk in ("c", "d"):
        a, b = x[prob.eg.cols[blk]], xo[prob.eg.cols[blk]]
        assert np.linalg.norm(a - b) <= 1e-10 * np.linalg.norm(b)
    res = np.linalg.norm(prob.eg.A @ x - prob.eg.f) / np.linalg.norm(prob.eg.f)
    assert res < 1e-10


def test_translate_matches_oracle(small):
    cfg, prob, gs = small
    rng = np.random.default_rng(0)
    n = prob.M * prob.nc
    beta = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    got = _np(gs.translate(beta))
    ref = prob.translate(beta)
    assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)


def test_operator_and_rhs_match_oracle(small):
    cfg, prob, gs = small
    rng = np.random.default_rng(1)
    n = prob.M * prob.nc
    x = (rng.standard_normal(n) + 1j * rng.standard_normal(n)) * np.tile(0.3 ** np.abs(np.arange(-prob.disks["p"], prob.disks["p"] + 1)), prob.M)
    got = _np(gs.apply(x))
    ref = prob.apply(x)
    assert np.linalg.norm(got - ref) <= 1e-11 * np.linalg.norm(ref)
    b = _np(gs.rhs())
    bo = prob.rhs()
    assert np.linalg.norm(b - bo) <= 1e-10 * np.linalg.norm(bo)


def test_solve_small_bragg(small):
    cfg, prob, gs = small
    gs.solve(tol=cfg["tol"], maxit=500)
    its, rr = gs.stats()
    assert rr <= 10 * cfg["tol"]
    got = gs.bragg()
    beta, _, _ = S.solve_dense(prob)
    _, ref, fe = prob.recover(beta)
    check_bragg(got, ref, BRAGG_TOL)
    assert got["flux_err"] < 1e-10
    bg = _np(gs.get_beta())
    assert np.linalg.norm(bg - beta) <= 1e-8 * np.linalg.norm(beta)


@pytest.mark.parametrize("M,p", [(1, 3), (7, 5), (13, 8)])
def test_translate_ragged_and_orders(M, p):
    """Single disk (images only), ragged M (not a multiple of the warps per block), other orders."""
    g = W.grating("tiny")
    dk = W.disks(M, 0.02, 0.01, 2.0, g["k"][0], seed=100 + M, p=p)
    gs = _setup_gpu(g, -0.9, dk)
    rng = np.random.default_rng(M)
    n = M * (2 * p + 1)
    beta = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    alpha = np.exp(1j * g["k"][0] * math.cos(-0.9) * g["d"])
    T = I.translation_matrix(dk["xy"], g["k"][1], p, g["d"], alpha)
    ref = T @ beta
    got = _np(gs.translate(beta))
    assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)
    gs.close()


def test_wood_anomaly_solve():
    """At the Wood angle of k1 the GPU path keeps matching the oracle and conserving flux."""
    cfg = W.config("small")
    g = cfg["grating"]
    theta = W.wood_angle(g["k"][0], g["d"])
    dk = cfg["disks"]
    prob = S.setup(g, theta, dk)
    beta, _, _ = S.solve_dense(prob)
    _, ref, _ = prob.recover(beta)
    gs = _setup_gpu(g, theta, dk)
    gs.solve(tol=1e-12, maxit=500)
    got = gs.bragg()
    check_bragg(got, ref, BRAGG_TOL)
    gs.close()


def test_geometry_and_state_errors():
    from paper_1412_7466_gb300 import GS_ERR_GEOMETRY, GS_ERR_STATE, GsError
    g = W.grating("tiny")
    gs = _solver()
    gs.set_layers(g)
    gs.set_incidence([-0.8])
    bad = {"xy": np.array([[0.0, 0.0], [0.01, 0.0]]), "radius": np.array([0.01, 0.01]),
           "kp": np.array([10.0, 10.0]), "p": 3}
    with pytest.raises(GsError) as e:
        gs.set_inclusions(bad)
    assert e.value.status == GS_ERR_GEOMETRY
    # overlap across the wall (minimum image)
    bad["xy"] = np.array([[-0.499, 0.0], [0.4985, 0.0]])
    with pytest.raises(GsError) as e:
        gs.set_inclusions(bad)
    assert e.value.status == GS_ERR_GEOMETRY
    with pytest.raises(GsError) as e:
        gs.solve()
    assert e.value.status == GS_ERR_STATE
    gs.close()


def test_factor_stats(small):
    """gs_factor_stats: the factorisation's Jacobi sweeps ended with a sweep that rotated nothing
    (the convergence test of the one-sided Jacobi method), its phase times are positive and add up to
    less than the whole factorisation could take, and the call is refused before any factorisation."""
    from paper_1412_7466_gb300 import GS_ERR_STATE, GsError
    cfg, prob, gs = small
    st = gs.factor_stats(0)
    assert st["sweeps_fp32"] >= 1 and st["sweeps_fp64"] >= 1
    assert len(st["rotations_fp32"]) == st["sweeps_fp32"] and len(st["rotations_fp64"]) == st["sweeps_fp64"]
    assert st["rotations_fp64"][-1] == 0 and st["rotations_fp64"][0] > 0
    n = prob.eg.A.shape[1]
    assert max(st["rotations_fp64"]) <= n * (n - 1) // 2
    # the polar step stopped at the FP64 floor: each Newton-Schulz step squared the defect until then
    d = st["newton_schulz_defects"]
    assert 1 <= st["newton_schulz_steps"] <= 6 and d[-1] < 1e-10
    assert all(b < a for a, b in zip(d, d[1:]))
    ph = st["phase_ms"]
    assert set(ph) == {"assemble", "qr", "jacobi_fp32", "polar_step", "jacobi_fp64", "u_v"}
    assert all(v > 0 for v in ph.values()) and sum(ph.values()) < 60e3
    fresh = _solver()
    fresh.set_layers(cfg["grating"])
    fresh.set_incidence([cfg["theta"]])
    with pytest.raises(GsError) as e:
        fresh.factor_stats(0)
    assert e.value.status == GS_ERR_STATE
    fresh.close()


def test_translate_c64_matches_oracle(small):
    """complex64 translation: FP32 products and Hankel recurrence; the operator agrees with the
    FP64 oracle to single-precision accuracy (1e-5 relative in norm, from ~1e-7 unit roundoff
    accumulated over ~30 source images and up to 2p recurrence steps per pair)."""
    from paper_1412_7466_gb300 import GS_C64
    cfg, prob, gs = small
    rng = np.random.default_rng(4)
    n = prob.M * prob.nc
    w = np.tile(0.3 ** np.abs(np.arange(-prob.disks["p"], prob.disks["p"] + 1)), prob.M)
    beta = (rng.standard_normal(n) + 1j * rng.standard_normal(n)) * w
    got = _np(gs.translate(beta, precision=GS_C64))
    ref = prob.translate(beta)
    assert np.linalg.norm(got - ref) <= 1e-5 * np.linalg.norm(ref)


def test_operator_c64_matches_oracle(small):
    """complex64 inner operator: complex64 translation and a complex64 copy of B_phys with FP32
    products, C x, U^* and V Sigma in double-float arithmetic: single-precision accuracy, 1e-5
    relative in norm."""
    from paper_1412_7466_gb300 import GS_C64
    cfg, prob, gs = small
    rng = np.random.default_rng(6)
    n = prob.M * prob.nc
    x = (rng.standard_normal(n) + 1j * rng.standard_normal(n)) * np.tile(0.3 ** np.abs(np.arange(-prob.disks["p"], prob.disks["p"] + 1)), prob.M)
    got = _np(gs.apply(x, precision=GS_C64))
    ref = prob.apply(x)
    assert np.linalg.norm(got - ref) <= 1e-5 * np.linalg.norm(ref)


def test_operator_c64_lowrank_part(small):
    """The low-rank correction S B_phys A^+ C x inside the complex64 operator, isolated as
    L32 x - x + S T32 x: C x in double-float arithmetic feeds A^+ (whose clipped Sigma^+ amplifies
    rounding in its near-null directions), so a plain FP32 C x would show here; only the complex64
    copy of B_phys (applied after A^+) rounds at single precision.  1e-5 relative in norm."""
    from paper_1412_7466_gb300 import GS_C64
    cfg, prob, gs = small
    rng = np.random.default_rng(16)
    n = prob.M * prob.nc
    x = (rng.standard_normal(n) + 1j * rng.standard_normal(n)) * np.tile(0.3 ** np.abs(np.arange(-prob.disks["p"], prob.disks["p"] + 1)), prob.M)
    s = prob.s.ravel()
    got = _np(gs.apply(x, precision=GS_C64)) - x + s * _np(gs.translate(x, precision=GS_C64))
    ref = prob.lowrank(x)
    assert np.linalg.norm(got - ref) <= 1e-5 * np.linalg.norm(ref)


def test_mixed_solve_small_bragg(small):
    """Mixed form (complex64 inner GMRES + FP64 refinement) reaches the same 1e-9 Bragg target."""
    from paper_1412_7466_gb300 import GS_C64
    cfg, prob, gs = small
    gs.solve(tol=cfg["tol"], maxit=2000, precision=GS_C64)
    its, rr = gs.stats()
    assert rr <= cfg["tol"]
    assert gs.refinement_sweeps() >= 1
    got = gs.bragg()
    beta, _, _ = S.solve_dense(prob)
    _, ref, _ = prob.recover(beta)
    check_bragg(got, ref, BRAGG_TOL)


def test_new_geometry_keeps_grating_factorisation():
    """gs_set_inclusions after gs_factor keeps the per-angle grating factorisation: a second
    geometry solved on the same context matches a fresh context."""
    cfg = W.config("small")
    g, th = cfg["grating"], cfg["theta"]
    d2 = W.disks(7, 0.04, 0.02, 2.0, g["k"][0], seed=77, p=10)
    gs = _setup_gpu(g, th, cfg["disks"])
    gs.set_inclusions(d2)
    gs.factor()
    gs.solve(tol=1e-12, maxit=500)
    a = gs.bragg()
    gs.close()
    gs2 = _setup_gpu(g, th, d2)
    gs2.solve(tol=1e-12, maxit=500)
    b = gs2.bragg()
    gs2.close()
    np.testing.assert_allclose(np.r_[a["c"], a["d"]], np.r_[b["c"], b["d"]], rtol=0, atol=1e-12)


def test_new_geometry_after_mixed_solve():
    """A mixed solve, then gs_set_inclusions with another geometry and a second mixed solve on the
    same context (the geometry's scratch, which the double-float low-rank products use, is rebuilt
    in between): the second solve matches the same geometry's mixed solve on a fresh context."""
    from paper_1412_7466_gb300 import GS_C64
    cfg = W.config("small")
    g, th = cfg["grating"], cfg["theta"]
    d2 = W.disks(7, 0.04, 0.02, 2.0, g["k"][0], seed=77, p=10)
    gs = _setup_gpu(g, th, cfg["disks"])
    gs.solve(tol=1e-12, maxit=500, precision=GS_C64)
    gs.set_inclusions(d2)
    gs.factor()
    gs.solve(tol=1e-12, maxit=500, precision=GS_C64)
    a = gs.bragg()
    gs.close()
    gs2 = _setup_gpu(g, th, d2)
    gs2.solve(tol=1e-12, maxit=500, precision=GS_C64)
    b = gs2.bragg()
    gs2.close()
    np.testing.assert_allclose(np.r_[a["c"], a["d"]], np.r_[b["c"], b["d"]], rtol=0, atol=1e-11)


@pytest.mark.parametrize("budget", [0.0, -1.0])
def test_translate_with_and_without_pair_table(budget):
    """The FP64 translation from the precomputed pair table (default) and recomputed in the kernel
    (table budget 0) both match the oracle's dense translation."""
    g = W.grating("tiny")
    dk = W.disks(37, 0.02, 0.01, 2.0, g["k"][0], seed=41, p=8)
    from paper_1412_7466_gb300 import GratingSolver
    gs = GratingSolver(0)
    gs.set_table_budget(budget)
    gs.set_layers(g)
    gs.set_incidence([-1.1])
    gs.set_inclusions(dk)
    gs.factor()
    rng = np.random.default_rng(9)
    n = 37 * 17
    beta = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    alpha = np.exp(1j * g["k"][0] * math.cos(-1.1) * g["d"])
    ref = I.translation_matrix(dk["xy"], g["k"][1], 8, g["d"], alpha) @ beta
    got = _np(gs.translate(beta))
    assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)
    gs.close()


def test_disks_across_the_walls_match_oracle():
    """Disks that straddle the period walls (Remark "cancel": the wall rows see only far copies),
    Bragg amplitudes against the oracle's dense solution."""
    g = W.grating("small")
    rng = np.random.default_rng(12)
    xy = np.array([[-0.49, 0.1], [0.495, -0.2], [0.0, 0.0], [-0.2, 0.25], [0.3, -0.05]])
    dk = {"xy": xy, "radius": np.full(5, 0.03), "kp": np.full(5, 20.0), "p": 8}
    th = -math.pi / 5
    prob = S.setup(g, th, dk)
    beta, _, _ = S.solve_dense(prob)
    _, ref, _ = prob.recover(beta)
    gs = _setup_gpu(g, th, dk)
    gs.solve(tol=1e-12, maxit=500)
    got = gs.bragg()
    check_bragg(got, ref, BRAGG_TOL)
    assert got["flux_err"] < 1e-10
    gs.close()


def test_degenerate_inputs_are_refused():
    from paper_1412_7466_gb300 import GS_ERR_ARG, GsError
    g = W.grating("tiny")
    gs = _solver()
    gs.set_layers(g)
    gs.set_incidence([-0.8])
    empty = {"xy": np.zeros((0, 2)), "radius": np.zeros(0), "kp": np.zeros(0), "p": 4}
    with pytest.raises(GsError) as e:
        gs.set_inclusions(empty)
    assert e.value.status == GS_ERR_ARG
    bad_p = {"xy": np.array([[0.0, 0.0]]), "radius": np.array([0.02]), "kp": np.array([10.0]), "p": 9}
    with pytest.raises(GsError) as e:
        gs.set_inclusions(bad_p)
    assert e.value.status == GS_ERR_ARG
    nan_xy = {"xy": np.array([[np.nan, 0.0]]), "radius": np.array([0.02]), "kp": np.array([10.0]), "p": 4}
    with pytest.raises(GsError):
        gs.set_inclusions(nan_xy)
    gs.close()


@pytest.mark.parametrize("prec_name,tol,gap", [("fp64", 1e-12, 0.01), ("c64", 1e-5, 0.2)])
@pytest.mark.parametrize("p", [1, 16])
def test_translate_extreme_orders(p, prec_name, tol, gap):
    """The smallest and the largest supported multipole order, both translation precisions (the
    complex64 case on well-separated disks: see the next test)."""
    from paper_1412_7466_gb300 import GS_C64, GS_FP64
    g = W.grating("tiny")
    M = 8
    dk = W.disks(M, 0.02, gap, 2.0, g["k"][0], seed=300 + p, p=p)
    gs = _setup_gpu(g, -1.0, dk)
    rng = np.random.default_rng(p)
    n = M * (2 * p + 1)
    w = np.tile(0.5 ** np.abs(np.arange(-p, p + 1)), M)
    beta = (rng.standard_normal(n) + 1j * rng.standard_normal(n)) * w
    alpha = np.exp(1j * g["k"][0] * math.cos(-1.0) * g["d"])
    ref = I.translation_matrix(dk["xy"], g["k"][1], p, g["d"], alpha) @ beta
    got = _np(gs.translate(beta, precision=GS_FP64 if prec_name == "fp64" else GS_C64))
    assert np.linalg.norm(got - ref) <= tol * np.linalg.norm(ref)
    gs.close()


def test_c64_translation_refused_outside_fp32_range():
    """p = 16 with disks 0.05 apart at k2 = 8: |H_32(0.4)| ~ 1e56 would overflow FP32, so the
    complex64 translation is refused (GS_ERR_ARG); the FP64 one still runs."""
    from paper_1412_7466_gb300 import GS_C64, GS_ERR_ARG, GsError
    g = W.grating("tiny")
    dk = W.disks(8, 0.02, 0.01, 2.0, g["k"][0], seed=5, p=16)
    gs = _setup_gpu(g, -1.0, dk)
    beta = np.ones(8 * 33, dtype=complex)
    with pytest.raises(GsError) as e:
        gs.translate(beta, precision=GS_C64)
    assert e.value.status == GS_ERR_ARG
    assert np.all(np.isfinite(_np(gs.translate(beta))))
    gs.close()


def test_several_angles_in_one_context():
    """gs_set_incidence with four angles (one at a Wood anomaly, one at normal incidence, alpha = 1):
    each angle's factorisation, coupling and solve, against the oracle at that angle."""
    cfg = W.config("small")
    g, dk = cfg["grating"], cfg["disks"]
    thetas = [-math.pi / 5, -1.2, W.wood_angle(g["k"][0], g["d"]), -math.pi / 2]   # ..., normal incidence
    from paper_1412_7466_gb300 import GratingSolver
    gs = GratingSolver(0)
    gs.set_layers(g)
    gs.set_incidence(thetas)
    gs.set_inclusions(dk)
    gs.factor()
    for q, th in enumerate(thetas):
        prob = S.setup(g, th, dk)
        beta, _, _ = S.solve_dense(prob)
        _, ref, _ = prob.recover(beta)
        gs.solve(angle=q, tol=1e-12, maxit=500)
        got = gs.bragg(angle=q)
        check_bragg(got, ref, BRAGG_TOL)
    gs.close()


def test_flat_interfaces():
    """Flat interfaces (no Fourier terms) with inclusions, against the oracle."""
    g = dict(W.grating("small"))
    g["gamma1"] = {"h0": 0.5, "cos": [], "sin": []}
    g["gamma2"] = {"h0": -0.5, "cos": [], "sin": []}
    dk = W.disks(6, 0.04, 0.02, 2.0, g["k"][0], seed=8, p=8)
    th = -math.pi / 5
    prob = S.setup(g, th, dk)
    beta, _, _ = S.solve_dense(prob)
    _, ref, _ = prob.recover(beta)
    gs = _setup_gpu(g, th, dk)
    gs.solve(tol=1e-12, maxit=500)
    got = gs.bragg()
    check_bragg(got, ref, BRAGG_TOL)
    assert got["flux_err"] < 1e-10
    gs.close()
