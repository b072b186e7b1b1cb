"""Pins of the oracle's coupled solve (Sec. 5): energy conservation with inclusions, LU against
GMRES, convergence in the multipole order p, invariance under a shift of the whole structure
(which moves disks across the unit-cell walls), invisibility of interfaces between equal media,
B against a projection of the directly evaluated layer field onto a circle, and the wall rows of
C against the uncancelled discrepancy."""
import math

import numpy as np
import pytest
from scipy.special import jv

import workloads as W
from oracle import inclusions as I
from oracle import layers as L
from oracle import solver as S


@pytest.fixture(scope="module")
def small():
    cfg = W.config("small")
    prob = S.setup(cfg["grating"], cfg["theta"], cfg["disks"])
    beta, Ld, b = S.solve_dense(prob)
    return cfg, prob, beta


def _bragg_vec(prob, beta):
    a, br, fe = prob.recover(beta)
    return np.concatenate([br["c"], br["d"]]), fe


def test_flux_with_inclusions(small):
    cfg, prob, beta = small
    _, fe = _bragg_vec(prob, beta)
    assert fe < 1e-11


def test_lu_and_gmres_agree(small):
    cfg, prob, beta = small
    bg, its, hist, _ = S.solve_gmres(prob, tol=1e-13)
    assert np.linalg.norm(bg - beta) <= 1e-11 * np.linalg.norm(beta)
    assert its < 60


def test_convergence_in_multipole_order():
    """Bragg amplitudes converge geometrically as p grows (Sec. 4.2: truncation to 2p+1 terms)."""
    cfg = W.config("small")
    out = {}
    for p in (3, 5, 7, 10):
        dk = dict(cfg["disks"])
        dk["p"] = p
        prob = S.setup(cfg["grating"], cfg["theta"], dk)
        beta, _, _ = S.solve_dense(prob)
        out[p], _ = _bragg_vec(prob, beta)
    ref = out[10]
    e = [np.linalg.norm(out[p] - ref) / np.linalg.norm(ref) for p in (3, 5, 7)]
    assert e[0] > e[1] > e[2]
    assert e[2] < 1e-9


def _shifted(g, disks, delta):
    w = 2 * math.pi / g["d"]
    g2 = dict(g)
    for key in ("gamma1", "gamma2"):
        a = g[key]["cos"][0]
        g2[key] = {"h0": g[key]["h0"], "cos": [a * math.cos(w * delta)], "sin": [a * math.sin(w * delta)]}
    d2 = dict(disks)
    xy = disks["xy"].copy()
    xy[:, 0] = (xy[:, 0] + delta + 0.5 * g["d"]) % g["d"] - 0.5 * g["d"]
    d2["xy"] = xy
    return g2, d2


def test_shift_invariance_with_wall_crossing():
    """Shifting grating and disks by delta (disks wrapped into the cell, so some straddle a wall)
    multiplies each Bragg amplitude by exp(-2 pi i n delta/d) (Remark "cancel": walls are
    invisible to the particles)."""
    g = W.grating("small")
    dk = W.disks(6, 0.03, 0.02, 2.0, g["k"][0], seed=11, p=8)
    theta = -0.7
    delta = 0.5 - dk["xy"][0, 0] - 0.01          # puts disk 0 across the right wall
    prob0 = S.setup(g, theta, dk)
    b0, _, _ = S.solve_dense(prob0)
    g2, d2 = _shifted(g, dk, delta)
    prob1 = S.setup(g2, theta, d2)
    b1, _, _ = S.solve_dense(prob1)
    xr = d2["xy"][0, 0]
    assert 0.5 - xr < 0.03 or xr + 0.5 < 0.03     # disk 0 straddles a wall
    a0, br0, _ = prob0.recover(b0)
    a1, br1, f1 = prob1.recover(b1)
    assert f1 < 1e-10
    w = 2 * math.pi / g["d"]
    np.testing.assert_allclose(br1["c"], br0["c"] * np.exp(-1j * w * br0["n_top"] * delta), atol=1e-9)
    np.testing.assert_allclose(br1["d"], br0["d"] * np.exp(-1j * w * br0["n_bot"] * delta), atol=1e-9)


def test_interfaces_between_equal_media_are_invisible():
    """With k1 = k2 = k3 the interfaces carry no physics: two different interface shapes give the
    same Bragg amplitudes for the same disks (checks the signs and images of B and C)."""
    g = dict(W.grating("small"))
    g["k"] = (15.0, 15.0, 15.0)
    dk = W.disks(5, 0.03, 0.02, 1.5, 15.0, seed=4, p=8)
    theta = -1.0
    res = []
    for amp in (0.05, 0.03):
        g2 = dict(g)
        g2["gamma1"] = {"h0": 0.5, "cos": [amp], "sin": []}
        g2["gamma2"] = {"h0": -0.5, "cos": [], "sin": [amp]}
        prob = S.setup(g2, theta, dk)
        beta, _, _ = S.solve_dense(prob)
        res.append(_bragg_vec(prob, beta)[0])
    np.testing.assert_allclose(res[0], res[1], atol=1e-10)


def test_B_matches_projection_of_layer_field(small):
    """Incoming coefficients from B_phys equal the Fourier projection, on a small circle about a
    disk centre, of the middle-layer field of the layer unknowns (Eq. repre3) evaluated directly."""
    cfg, prob, _ = small
    eg = prob.eg
    rng = np.random.default_rng(8)
    x = np.zeros(eg.A.shape[1], dtype=complex)
    for blk in ("mu1", "sigma1", "mu2", "sigma2"):
        sl = eg.cols[blk]
        x[sl] = rng.standard_normal(sl.stop - sl.start) + 1j * rng.standard_normal(sl.stop - sl.start)
    sl = eg.cols["a2"]
    Q2 = eg.g["Q"][1]
    x[sl] = (rng.standard_normal(2 * Q2 + 1) + 1j * rng.standard_normal(2 * Q2 + 1)) * 0.5 ** np.abs(np.arange(-Q2, Q2 + 1))
    coeff = (prob.B @ x).reshape(prob.M, prob.nc)
    k2 = eg.k[1]
    p = prob.disks["p"]
    ntheta = 128
    th = 2 * np.pi * np.arange(ntheta) / ntheta
    for i in (0, 3, 7):
        c = prob.disks["xy"][i]
        rho = 0.03
        pts = c + rho * np.stack([np.cos(th), np.sin(th)], axis=1)
        nrm = np.tile([0.0, 1.0], (ntheta, 1))
        u = np.zeros(ntheta, dtype=complex)
        for cv, cm, cs in ((eg.c1, "mu1", "sigma1"), (eg.c2, "mu2", "sigma2")):
            P = L.near_potentials(pts, nrm, cv, eg.d, eg.alpha, k2)
            u += P["S"] @ x[eg.cols[cs]] + P["D"] @ x[eg.cols[cm]]
        v, _ = L.jexp_columns(pts, nrm, eg.centers[1], k2, Q2)
        u += v @ x[eg.cols["a2"]]
        for m in range(-5, 6):
            proj = np.mean(u * np.exp(-1j * m * th)) / jv(m, k2 * rho)
            assert abs(proj - coeff[i, m + p]) <= 1e-9 * max(1.0, abs(proj))


def test_C_wall_rows_equal_uncancelled_discrepancy():
    """For disks away from the walls, the cancelled wall rows of C equal alpha u(L) - u(R) summed
    over the three near copies (Remark "cancel")."""
    g = W.grating("small")
    eg = L.build_empty_grating(g, -0.6)
    dk = {"xy": np.array([[0.1, 0.2], [-0.25, -0.1]]), "radius": np.array([0.02, 0.02]),
          "kp": np.array([20.0, 20.0]), "p": 6}
    C = I.coupling_C(eg, dk)
    ys = eg.wall_y[1]
    d = eg.d
    Lp = np.stack([np.full_like(ys, -0.5 * d), ys], axis=1)
    Rp = np.stack([np.full_like(ys, 0.5 * d), ys], axis=1)
    direct_v = 0
    direct_n = 0
    for l in (-1, 0, 1):
        cen = dk["xy"] + np.array([l * d, 0.0])
        vL, fxL, _ = I._outgoing_fields(Lp, cen, eg.k[1], dk["p"])
        vR, fxR, _ = I._outgoing_fields(Rp, cen, eg.k[1], dk["p"])
        direct_v = direct_v + eg.alpha ** l * (eg.alpha * vL - vR)
        direct_n = direct_n + eg.alpha ** l * (eg.alpha * fxL - fxR)
    n = ys.size
    np.testing.assert_allclose(C[eg.rows["w2v"]], direct_v.reshape(n, -1), atol=1e-12)
    np.testing.assert_allclose(C[eg.rows["w2n"]], direct_n.reshape(n, -1), atol=1e-10)
