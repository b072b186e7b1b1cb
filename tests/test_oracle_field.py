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
