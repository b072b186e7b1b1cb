"""General inclusion shapes through the C-ABI (gs_set_inclusions_star), against the oracle: the
rotated star matrices from the GPU boundary integral equation (1e-11 of the largest entry: two
FP64 Nystrom solves of the same discretisation with different Bessel implementations), a circle
through the same route against the closed-form disk coefficients, and full solves with rotated
stars -- FP64, mixed, TE, many angles -- against the oracle's dense LU (Bragg amplitudes 1e-9,
norm-wise and element-wise)."""
import math

import numpy as np
import pytest

import workloads as W
from bragg import check as check_bragg
from oracle import inclusions as I
from oracle import shapes as SH
from oracle import solver as S

pytestmark = pytest.mark.gpu


def _stars(M, seed, a1, a2, p, kp, N=128):
    dk = W.disks(M, a1 + a2, 0.5 * (a1 + a2), 1.0, kp, seed=seed, p=p)
    rng = np.random.default_rng(seed + 1)
    dk["kp"] = np.full(M, kp)
    dk["phi"] = rng.uniform(0, 2 * math.pi, M)
    dk["shape"] = {"a1": a1, "a2": a2, "a3": 3, "N": N}
    return dk


def _gpu(g, thetas, dk):
    from paper_1412_7466_gb300 import GratingSolver
    gs = GratingSolver(0)
    gs.set_layers(g)
    gs.set_incidence(thetas)
    gs.set_inclusions(dk)
    gs.factor()
    return gs


@pytest.mark.parametrize("pol", ["TM", "TE"])
def test_star_blocks_match_oracle(pol):
    cfg = W.config("small")
    g = dict(cfg["grating"], pol=pol)
    dk = _stars(8, 5, 0.03, 0.01, 8, 30.0)
    gs = _gpu(g, [cfg["theta"]], dk)
    got = gs.get_scattering_blocks().cpu().numpy()
    gs.close()
    ref = SH.scattering_blocks(dk, g["k"][1], pol)
    assert np.max(np.abs(got - ref)) <= 1e-11 * np.max(np.abs(ref))


def test_circle_through_the_shape_route():
    cfg = W.config("small")
    g = cfg["grating"]
    dk = _stars(4, 6, 0.04, 0.0, 8, 20.0, N=96)
    gs = _gpu(g, [cfg["theta"]], dk)
    got = gs.get_scattering_blocks().cpu().numpy()
    gs.close()
    m = I.mie_coefficients(8, 0.04, g["k"][1], 20.0)
    for blk in got:
        np.testing.assert_allclose(np.diag(blk), m, rtol=0, atol=1e-12 * np.abs(m).max())
        assert np.max(np.abs(blk - np.diag(np.diag(blk)))) < 1e-13 * np.abs(m).max()


@pytest.mark.parametrize("pol,prec_name", [("TM", "fp64"), ("TM", "c64"), ("TE", "fp64")])
def test_solve_with_rotated_stars_matches_oracle(pol, prec_name):
    from paper_1412_7466_gb300 import GS_C64, GS_FP64
    cfg = W.config("small")
    g = dict(cfg["grating"], pol=pol)
    dk = _stars(8, 5, 0.03, 0.01, 8, 30.0)
    gs = _gpu(g, [cfg["theta"]], dk)
    gs.solve(tol=1e-12, maxit=2000, precision=GS_FP64 if prec_name == "fp64" else GS_C64)
    got = gs.bragg()
    gs.close()
    prob = S.setup(g, cfg["theta"], dk)
    beta, _, _ = S.solve_dense(prob)
    _, ref, _ = prob.recover(beta)
    nw, ew = check_bragg(got, ref)
    assert got["flux_err"] < 1e-10
    print(pol, prec_name, "stars: Bragg error vs oracle", nw, ew)


def test_many_angles_with_stars_match_oracle():
    cfg = W.config("small")
    g = cfg["grating"]
    dk = _stars(6, 7, 0.03, 0.01, 8, 30.0)
    thetas = [-math.pi / 5, W.wood_angle(g["k"][0], g["d"])]
    gs = _gpu(g, thetas, dk)
    gs.solve_angles(tol=1e-12, maxit=2000, restart=200)
    got = [gs.bragg(angle=q) for q in range(2)]
    gs.close()
    for q, th in enumerate(thetas):
        prob = S.setup(g, th, dk)
        beta, _, _ = S.solve_dense(prob)
        check_bragg(got[q], prob.recover(beta)[1])


def test_warm_start_refuses_stars():
    from paper_1412_7466_gb300 import GS_ERR_STATE, GsError
    cfg = W.config("small")
    dk = _stars(4, 8, 0.03, 0.01, 8, 30.0)
    gs = _gpu(cfg["grating"], [cfg["theta"]], dk)
    gs.mlp_set_params(8, W.mlp_init(8, 1).tolist() + [0.0] * 64 + [1.0] * 64 + [1.0] * 17)
    with pytest.raises(GsError) as e:
        gs.warm_start()
    assert e.value.status == GS_ERR_STATE
    gs.close()
