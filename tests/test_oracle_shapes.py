"""Pins of the oracle's general inclusion shapes (Sec. 4.1 Eqs. intg1-intg2 and the moment
integral; Sec. 4.2 rotations), against mathematics the oracle does not share: a circle reproduces
the closed-form disk coefficients; the partial S-matrix I + 2 S of a lossless star is unitary; the
matrix of a rotated star computed from its own boundary equals the rotated matrix; the multipole
expansion reproduces the scattered field evaluated directly from the densities; a star rotated by
one petal period is the same inclusion; solves with stars conserve flux and LU agrees with GMRES."""
import math

import numpy as np
import pytest
from scipy.special import hankel1

import workloads as W
from oracle import inclusions as I
from oracle import layers as L
from oracle import shapes as SH
from oracle import solver as S


@pytest.mark.parametrize("pol", ["TM", "TE"])
@pytest.mark.parametrize("R,k2,kp", [(0.04, 15.0, 20.0), (0.3, 5.0, 11.0)])
def test_circle_reproduces_disk_coefficients(pol, R, k2, kp):
    Smat = SH.scattering_matrix(R, 0.0, 3, 96, 8, k2, kp, pol)
    m = I.mie_coefficients(8, R, k2, kp, pol)
    np.testing.assert_allclose(np.diag(Smat), m, rtol=0, atol=1e-13 * np.abs(m).max())
    assert np.max(np.abs(Smat - np.diag(np.diag(Smat)))) < 1e-14 * np.abs(m).max()


@pytest.mark.parametrize("pol", ["TM", "TE"])
def test_star_partial_s_matrix_unitary(pol):
    """Energy conservation for a lossless inclusion: (I + 2S)^* (I + 2S) = I (to the truncation of
    the expansion, which the star's small size makes negligible at p = 10)."""
    Smat = SH.scattering_matrix(0.0309, 0.0103, 3, 300, 10, 8.0, 30.0, pol)
    U = np.eye(21) + 2 * Smat
    assert np.max(np.abs(U.conj().T @ U - np.eye(21))) < 1e-12
    assert np.max(np.abs(Smat - np.diag(np.diag(Smat)))) > 1e-6     # genuinely non-diagonal


def test_rotation_phase_factors():
    """Rotation by phi (counter-clockwise) multiplies s_ln by e^{i phi (n - l)} (Sec. 4.2, printed
    with the clockwise angle): the matrix of the rotated star computed from its own discretised
    boundary agrees with the rotated matrix, and not with the opposite sign."""
    S0 = SH.scattering_matrix(0.04, 0.015, 3, 200, 8, 15.0, 26.0)
    for phi in (0.3, -1.1, 2.5):
        Sr = SH.scattering_matrix(0.04, 0.015, 3, 200, 8, 15.0, 26.0, phi=phi)
        assert np.max(np.abs(Sr - SH.rotate(S0, phi))) < 1e-13 * np.max(np.abs(S0))
        assert np.max(np.abs(Sr - SH.rotate(S0, -phi))) > 1e-4 * np.max(np.abs(S0))
    # one petal period (2 pi / 3) maps the star onto itself
    S3 = SH.rotate(S0, 2 * math.pi / 3)
    assert np.max(np.abs(S3 - S0)) < 1e-12 * np.max(np.abs(S0))


def test_multipole_expansion_matches_direct_field():
    """Outside the circumscribing circle, sum_l s_ln H_l(k2 r) e^{i l th} equals the scattered field
    S^{k2} sigma_n + D^{k2} mu_n evaluated from the boundary densities by the (spectrally accurate)
    trapezoid rule: checks the moment integral, its i/4 and its conjugate waves.  The expansion is
    taken to |l| <= 24 so that its truncation stays below the comparison (a star couples order n to
    n +- 3, n +- 6, ...)."""
    k2, p = 15.0, 24
    Smat, cv, mu, sigma = SH.scattering_matrix(0.04, 0.015, 3, 200, p, k2, 26.0, return_densities=True)
    rng = np.random.default_rng(0)
    rr = rng.uniform(0.09, 0.2, 20)
    th = rng.uniform(0, 2 * math.pi, 20)
    pts = np.stack([rr * np.cos(th), rr * np.sin(th)], axis=1)
    w = (2 * math.pi / cv["N"]) * cv["speed"]
    K = L.kernels(pts, np.tile([1.0, 0.0], (20, 1)), cv["pos"], cv["nrm"], k2)
    scale = None
    for n in (0, -5, -3, 2, 4, 6):
        direct = (K["S"] * w[None, :]) @ sigma[:, n + p] + (K["D"] * w[None, :]) @ mu[:, n + p]
        series = SH.exterior_field(Smat[:, n + p], k2, pts)
        scale = np.max(np.abs(direct)) if scale is None else scale     # the n = 0 field's size
        assert np.max(np.abs(direct - series)) < 1e-10 * scale, n


def test_scattering_matrix_converges_in_nodes():
    a = SH.scattering_matrix(0.0309, 0.0103, 3, 300, 10, 8.0, 30.0)
    b = SH.scattering_matrix(0.0309, 0.0103, 3, 160, 10, 8.0, 30.0)
    assert np.max(np.abs(a - b)) < 1e-12 * np.max(np.abs(a))


def _stars(M, seed, a1, a2, p, kp, N=128):
    dk = W.disks(M, a1 + a2, 0.5 * (a1 + a2), 1.0, kp, seed=seed, p=p)
    rng = np.random.default_rng(seed + 1)
    dk["kp"] = np.full(M, kp)
    dk["phi"] = rng.uniform(0, 2 * math.pi, M)
    dk["shape"] = {"a1": a1, "a2": a2, "a3": 3, "N": N}
    return dk


@pytest.mark.parametrize("pol", ["TM", "TE"])
def test_solve_with_stars_conserves_flux_and_lu_matches_gmres(pol):
    cfg = W.config("small")
    g = dict(cfg["grating"], pol=pol)
    dk = _stars(8, 5, 0.03, 0.01, 8, 30.0)
    prob = S.setup(g, cfg["theta"], dk)
    beta, _, _ = S.solve_dense(prob)
    _, br, fe = prob.recover(beta)
    assert fe < 1e-10
    bg, its, hist, _ = S.solve_gmres(prob, tol=1e-13, restart=200, maxit=500)
    _, br2, _ = prob.recover(bg)
    a = np.r_[br["c"], br["d"]]
    b = np.r_[br2["c"], br2["d"]]
    assert np.linalg.norm(a - b) < 1e-10 * np.linalg.norm(a)


def test_petal_rotation_leaves_the_solution_unchanged():
    cfg = W.config("small")
    dk = _stars(5, 9, 0.03, 0.01, 8, 30.0)
    out = []
    for shift in (0.0, 2 * math.pi / 3):
        d2 = dict(dk, phi=dk["phi"] + shift)
        prob = S.setup(cfg["grating"], cfg["theta"], d2)
        beta, _, _ = S.solve_dense(prob)
        out.append(prob.recover(beta)[1])
    a = np.r_[out[0]["c"], out[0]["d"]]
    b = np.r_[out[1]["c"], out[1]["d"]]
    assert np.linalg.norm(a - b) < 1e-11 * np.linalg.norm(a)
