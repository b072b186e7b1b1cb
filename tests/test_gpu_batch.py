"""Batched form: geometries of uneven size on one factored grating, one persistent translation
launch, grouped low-rank products, lockstep GMRES replayed from a CUDA graph.  Each geometry's
operator and Bragg amplitudes must match the single-geometry path (and the oracle) on the same
inputs: FP64 operator 1e-12, complex64 operator 1e-5, Bragg amplitudes 1e-9 (relative, norm)."""
import numpy as np
import pytest

import workloads as W
from bragg import check as check_bragg
from oracle import solver as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def batch():
    from paper_1412_7466_gb300 import GratingSolver
    cfg = W.config("small")
    g, th = cfg["grating"], cfg["theta"]
    geos = [W.disks(M, 0.02, 0.01, 2.0, g["k"][0], seed=300 + M, p=8) for M in (41, 7, 23)]
    gs = GratingSolver(0)
    gs.set_layers(g)
    gs.set_incidence([th])
    gs.set_inclusions_batch(geos)
    gs.factor_batch()
    single = []
    for dk in geos:
        s1 = GratingSolver(0)
        s1.set_layers(g)
        s1.set_incidence([th])
        s1.set_inclusions(dk)
        s1.factor()
        single.append(s1)
    yield cfg, geos, gs, single
    for s1 in single:
        s1.close()
    gs.close()


def _split(v, sizes):
    out, o = [], 0
    for n in sizes:
        out.append(v[o:o + n])
        o += n
    return out


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 1e-5)])
def test_batched_operator_matches_single(batch, prec, tol):
    cfg, geos, gs, single = batch
    sizes = gs.batch_sizes
    rng = np.random.default_rng(7)
    x = rng.standard_normal(sum(sizes)) + 1j * rng.standard_normal(sum(sizes))
    y = gs.apply_batch(x, precision=prec).cpu().numpy()
    for xg, yg, s1 in zip(_split(x, sizes), _split(y, sizes), single):
        ref = s1.apply(xg, precision=prec).cpu().numpy()
        assert np.linalg.norm(yg - ref) <= tol * np.linalg.norm(ref)


@pytest.mark.parametrize("prec", [0, 1])
def test_batched_solve_matches_single_and_oracle(batch, prec):
    cfg, geos, gs, single = batch
    gs.solve_batch(tol=1e-12, maxit=2000, precision=prec)
    for q, (dk, s1) in enumerate(zip(geos, single)):
        its, rr = gs.batch_stats(q)
        assert rr <= 1e-11
        got = gs.bragg_batch(q)
        s1.solve(tol=1e-12, maxit=2000)
        check_bragg(got, s1.bragg())
    # geometry 1 (M = 7) against the oracle's dense LU
    prob = S.setup(cfg["grating"], cfg["theta"], geos[1])
    beta, _, _ = S.solve_dense(prob)
    _, ref, _ = prob.recover(beta)
    check_bragg(gs.bragg_batch(1), ref)


def test_autotuned_tiles_are_candidates(batch):
    cfg, geos, gs, single = batch
    chunk, bps = gs.batch_tuning()
    assert chunk in (512, 1024, 2048) and bps in (2, 4, 8)


def test_batched_two_angles_match_single():
    """One batch factored at two angles: each angle's batched mixed solve matches the
    single-geometry solve at that angle."""
    from paper_1412_7466_gb300 import GS_C64, GratingSolver
    cfg = W.config("small")
    g = cfg["grating"]
    thetas = [-1.3, -0.7]
    geos = [W.disks(M, 0.02, 0.01, 2.0, g["k"][0], seed=500 + M, p=6) for M in (19, 5)]
    gb = GratingSolver(0)
    gb.set_layers(g)
    gb.set_incidence(thetas)
    gb.set_inclusions_batch(geos)
    gb.factor_batch()
    for q, th in enumerate(thetas):
        gb.solve_batch(angle=q, tol=1e-12, precision=GS_C64)
        for k, dk in enumerate(geos):
            got = gb.bragg_batch(k, angle=q)
            s1 = GratingSolver(0)
            s1.set_layers(g)
            s1.set_incidence([th])
            s1.set_inclusions(dk)
            s1.factor()
            s1.solve(tol=1e-12, maxit=500)
            ref = s1.bragg()
            s1.close()
            check_bragg(got, ref)
    gb.close()
