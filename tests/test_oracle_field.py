"""Pins of the middle-layer field oracle: (1) a transparent grating (k1 = k2 = k3) with an
invisible inclusion (k_p = k2, so s = 0) carries exactly the incident plane wave through the
middle layer; (2) on a circle just outside an inclusion the field's Fourier modes are
alpha_n J_n(k2 rho) + beta_n H_n(k2 rho) with beta the solution and alpha its incoming
coefficients w + t (the empty grating's field plus T beta - B_phys A^+ C beta) -- direct Hankel
sums and layer potentials on one side, the Graf translation and the B_phys projection on the
other."""
import math

import numpy as np
import pytest
from scipy.special import hankel1, jv

import workloads as W
from oracle import field as F
from oracle import solver as S
from oracle import warmstart as WS


def test_transparent_grating_carries_the_plane_wave():
    g = dict(W.grating("small"))
    k = 10.0
    g["k"] = (k, k, k)
    th = -math.pi / 5
    dk = W.disks(1, 0.04, 0.02, 1.0, k, seed=2, p=6)          # k_p = k2: invisible
    prob = S.setup(g, th, dk)
    beta, _, _ = S.solve_dense(prob)
    assert np.max(np.abs(beta)) < 1e-12
    rng = np.random.default_rng(0)
    pts = np.stack([rng.uniform(-0.5, 0.5, 40), rng.uniform(-0.3, 0.3, 40)], axis=1)
    u = F.middle_field(prob, beta, pts)
    ref = np.exp(1j * k * (math.cos(th) * pts[:, 0] + math.sin(th) * pts[:, 1]))
    ok = ~np.isnan(u)
    assert ok.sum() >= 38
    assert np.max(np.abs(u[ok] - ref[ok])) < 1e-9


def test_field_modes_around_an_inclusion():
    cfg = W.config("small")
    prob = S.setup(cfg["grating"], cfg["theta"], cfg["disks"])
    beta, _, _ = S.solve_dense(prob)
    p = prob.disks["p"]
    nc = 2 * p + 1
    alpha = WS.incoming_empty(prob) + WS.scattered_incoming(prob, beta)
    B = beta.reshape(prob.M, nc)
    k2 = prob.eg.k[1]
    nth = 64
    th = 2 * np.pi * np.arange(nth) / nth
    for j in (0, 4, 9):
        c = prob.disks["xy"][j]
        rho = 1.05 * prob.disks["radius"][j]
        pts = c + rho * np.stack([np.cos(th), np.sin(th)], axis=1)
        u = F.middle_field(prob, beta, pts)
        modes = np.fft.fft(u) / nth                        # u = sum_n u_n e^{i n th}
        for n in range(-4, 5):
            got = modes[n % nth]
            ref = alpha[j, n + p] * jv(n, k2 * rho) + B[j, n + p] * hankel1(n, k2 * rho)
            assert abs(got - ref) <= 1e-8 * max(1.0, abs(ref)), (j, n, got, ref)


def _slab_field(k, theta, a_top, b_bot, pts):
    """Textbook three-layer slab field: u1 = e^{i(kx x - q1 y)} + r e^{i(kx x + q1 y)},
    u2 = (A e^{-i q2 y} + B e^{i q2 y}) e^{i kx x}, u3 = t e^{i(kx x - q3 y)}, with continuity of u
    and u_y at the flat interfaces y = a_top, y = b_bot."""
    k1, k2, k3 = k
    kx = k1 * math.cos(theta)
    q1, q2, q3 = [np.sqrt(complex(kk * kk - kx * kx)) for kk in k]
    ea = lambda qq, s: np.exp(1j * s * qq * a_top)
    eb = lambda qq, s: np.exp(1j * s * qq * b_bot)
    M = np.array([[ea(q1, 1), -ea(q2, -1), -ea(q2, 1), 0],
                  [1j * q1 * ea(q1, 1), 1j * q2 * ea(q2, -1), -1j * q2 * ea(q2, 1), 0],
                  [0, eb(q2, -1), eb(q2, 1), -eb(q3, -1)],
                  [0, -1j * q2 * eb(q2, -1), 1j * q2 * eb(q2, 1), 1j * q3 * eb(q3, -1)]], dtype=complex)
    rhs = np.array([-ea(q1, -1), 1j * q1 * ea(q1, -1), 0, 0], dtype=complex)
    r, A, B, t = np.linalg.solve(M, rhs)
    x, y = pts[:, 0], pts[:, 1]
    ex = np.exp(1j * kx * x)
    return np.where(y > a_top, ex * (np.exp(-1j * q1 * y) + r * np.exp(1j * q1 * y)),
                    np.where(y > b_bot, ex * (A * np.exp(-1j * q2 * y) + B * np.exp(1j * q2 * y)),
                             ex * t * np.exp(-1j * q3 * y)))


def _away_from_interfaces(g, pts, dist):
    from oracle import layers as L
    h1 = L.iface_eval(g["gamma1"], g["d"], pts[:, 0])[0]
    h2 = L.iface_eval(g["gamma2"], g["d"], pts[:, 0])[0]
    return (np.abs(pts[:, 1] - h1) > dist) & (np.abs(pts[:, 1] - h2) > dist)


def test_all_layer_field_transparent_grating():
    """k1 = k2 = k3 over corrugated interfaces with an invisible inclusion: the total field is the
    incident plane wave in every layer, including the Rayleigh-Bloch regions beyond +-y0."""
    g = dict(W.grating("small"))
    k = 10.0
    g["k"] = (k, k, k)
    th = -math.pi / 5
    dk = W.disks(1, 0.04, 0.02, 1.0, k, seed=2, p=6)
    prob = S.setup(g, th, dk)
    beta, _, _ = S.solve_dense(prob)
    rng = np.random.default_rng(1)
    pts = np.stack([rng.uniform(-0.5, 0.5, 300), rng.uniform(-1.6, 1.6, 300)], axis=1)
    pts = pts[_away_from_interfaces(g, pts, 0.05)]
    u = F.field(prob, beta, pts)
    ref = np.exp(1j * k * (math.cos(th) * pts[:, 0] + math.sin(th) * pts[:, 1]))
    ok = ~np.isnan(u)
    assert ok.sum() >= pts.shape[0] - 2
    for sel in (pts[:, 1] > 1.0, pts[:, 1] < -1.0, np.abs(pts[:, 1]) < 1.0):
        assert (ok & sel).sum() > 20
    assert np.max(np.abs(u[ok] - ref[ok])) < 1e-9


def test_all_layer_field_flat_slab():
    """Flat interfaces at y = +-0.5 with an invisible inclusion: the field in all three layers and
    beyond +-y0 is the textbook slab solution (reflected and transmitted plane waves)."""
    g = dict(W.grating("small"))
    g["gamma1"] = {"h0": 0.5, "cos": [], "sin": []}
    g["gamma2"] = {"h0": -0.5, "cos": [], "sin": []}
    th = -0.9
    dk = W.disks(1, 0.04, 0.02, 1.5, g["k"][0], seed=2, p=6)
    dk["kp"] = np.array([g["k"][1]])                             # k_p = k2: invisible
    prob = S.setup(g, th, dk)
    beta, _, _ = S.solve_dense(prob)
    rng = np.random.default_rng(2)
    pts = np.stack([rng.uniform(-0.5, 0.5, 300), rng.uniform(-1.6, 1.6, 300)], axis=1)
    pts = pts[_away_from_interfaces(g, pts, 0.05)]
    u = F.field(prob, beta, pts)
    ref = _slab_field(g["k"], th, 0.5, -0.5, pts)
    ok = ~np.isnan(u)
    assert ok.sum() >= pts.shape[0] - 2
    assert np.max(np.abs(u[ok] - ref[ok])) < 1e-9 * np.max(np.abs(ref))


def test_field_continuous_across_gamma_u_and_gamma_d():
    """With inclusions on a corrugated grating, the potential/J-expansion representation below
    Gamma_u (above Gamma_d) and the Rayleigh-Bloch expansion on the other side agree at y = +-y0
    (the Gamma_u/Gamma_d rows of A impose it at the n_bound nodes; in between, to the scheme's
    accuracy)."""
    cfg = W.config("small")
    prob = S.setup(cfg["grating"], cfg["theta"], cfg["disks"])
    beta, _, _ = S.solve_dense(prob)
    y0 = cfg["grating"]["y0"]
    xs = np.linspace(-0.49, 0.49, 37)
    for yy in (y0, -y0):
        above = F.field(prob, beta, np.stack([xs, np.full_like(xs, yy + 1e-9)], 1))
        below = F.field(prob, beta, np.stack([xs, np.full_like(xs, yy - 1e-9)], 1))
        assert np.max(np.abs(above - below)) < 1e-7 * np.max(np.abs(above)), yy
