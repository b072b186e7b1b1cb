"""Pins of the oracle's TE polarisation and lossy inclusions (Sec. 2 names TE; Sec. 7 leaves TE and
complex permittivities to future work).  TE: u is the magnetic field, [u] = 0 and
[(1/eps) d_n u] = 0 on every interface, eps proportional to k^2 (constant permeability).  Lossy:
complex interior wavenumber kp (Im kp > 0).  Checked against mathematics the oracle does not share:
the transmission conditions of the disk coefficients evaluated directly, unitarity and absorption of
the partial S-matrix, the textbook TE slab (transfer matrix with 1/eps-weighted derivatives), energy
conservation (the TE flux identity) on corrugated gratings with and without inclusions, TM = TE when
all permittivities agree, and the weighted singular operators against an independent graded
Gauss-Legendre quadrature of the lattice integral."""
import math

import numpy as np
import pytest
from scipy.special import h1vp, hankel1, jv, jvp

import workloads as W
from oracle import inclusions as I
from oracle import layers as L
from oracle import solver as S


@pytest.mark.parametrize("pol", ["TM", "TE"])
@pytest.mark.parametrize("R,k2,kp", [(0.04, 15.0, 20.0), (0.008, 60.0, 80.0 + 3.0j), (0.3, 5.0, 11.0 + 0.5j)])
def test_disk_coefficients_transmission_conditions(pol, R, k2, kp):
    """Outside J_n + s_n H_n at k2, inside t_n J_n at kp: the values match and so do the radial
    derivatives weighted by 1 (TM) or 1/eps ~ 1/k^2 (TE), also for complex kp."""
    s = I.mie_coefficients(12, R, k2, kp, pol)
    n = np.arange(-12, 13)
    t = (jv(n, k2 * R) + s * hankel1(n, k2 * R)) / jv(n, kp * R)
    w2, wp = (1.0, 1.0) if pol == "TM" else (1.0 / k2 ** 2, 1.0 / kp ** 2)
    lhs = w2 * k2 * (jvp(n, k2 * R) + s * h1vp(n, k2 * R))
    rhs = wp * kp * t * jvp(n, kp * R)
    np.testing.assert_allclose(lhs, rhs, rtol=1e-9, atol=1e-300)
    np.testing.assert_allclose(s, s[::-1], rtol=1e-12)


def test_disk_partial_s_matrix_unitary_or_absorbing():
    """|1 + 2 s_n| = 1 for a lossless disk in both polarisations, < 1 for a lossy one, and the
    TE coefficients differ from the TM ones."""
    for pol in ("TM", "TE"):
        for (R, k2, kp) in ((0.04, 15.0, 20.0), (0.3, 5.0, 11.0)):
            s = I.mie_coefficients(10, R, k2, kp, pol)
            np.testing.assert_allclose(np.abs(1 + 2 * s), 1.0, atol=1e-13)
            sl = I.mie_coefficients(10, R, k2, kp + 0.8j, pol)
            assert np.all(np.abs(1 + 2 * sl[8:13]) < 1.0 - 1e-6)
    a = I.mie_coefficients(6, 0.3, 5.0, 11.0, "TM")
    b = I.mie_coefficients(6, 0.3, 5.0, 11.0, "TE")
    assert np.max(np.abs(a - b)) > 1e-3 * np.max(np.abs(a))


def _te_slab(k, theta, a_top, b_bot):
    """TE slab by the transfer matrix: u1 = e^{i(kx x - q1 y)} + r e^{i(kx x + q1 y)},
    u2 = A e^{-i q2 y} + B e^{i q2 y}, u3 = t e^{-i q3 y}; u and (1/k^2) u_y continuous."""
    kx = k[0] * math.cos(theta)
    q1, q2, q3 = [np.sqrt(complex(kk * kk - kx * kx)) for kk in k]
    e1, e2, e3 = [1.0 / (kk * kk) for kk in k]
    ea = lambda qq, s: np.exp(1j * s * qq * a_top)
    eb = lambda qq, s: np.exp(1j * s * qq * b_bot)
    M = np.array([[ea(q1, 1), -ea(q2, -1), -ea(q2, 1), 0],
                  [e1 * 1j * q1 * ea(q1, 1), e2 * 1j * q2 * ea(q2, -1), -e2 * 1j * q2 * ea(q2, 1), 0],
                  [0, eb(q2, -1), eb(q2, 1), -eb(q3, -1)],
                  [0, -e2 * 1j * q2 * eb(q2, -1), e2 * 1j * q2 * eb(q2, 1), e3 * 1j * q3 * eb(q3, -1)]], dtype=complex)
    rhs = np.array([-ea(q1, -1), e1 * 1j * q1 * ea(q1, -1), 0, 0], dtype=complex)
    r, A, B, t = np.linalg.solve(M, rhs)
    return r, t, q1, q3


def _solve_empty(g, theta):
    eg = L.build_empty_grating(g, theta)
    return eg, L.factor(eg).apply(eg.f)


def test_te_flat_slab_matches_transfer_matrix():
    g = dict(W.grating("small"))
    g["gamma1"] = {"h0": 0.5, "cos": [], "sin": []}
    g["gamma2"] = {"h0": -0.5, "cos": [], "sin": []}
    g["pol"] = "TE"
    theta = -0.9
    eg, a = _solve_empty(g, theta)
    r, t, q1, q3 = _te_slab(g["k"], theta, 0.5, -0.5)
    K = g["K_rb"]
    c, d = a[eg.cols["c"]], a[eg.cols["d"]]
    y0 = g["y0"]
    assert abs(c[K] - r * np.exp(1j * q1 * y0)) < 1e-10
    assert abs(d[K] - t * np.exp(1j * q3 * y0)) < 1e-10
    others = np.r_[np.arange(K), np.arange(K + 1, 2 * K + 1)]
    assert np.max(np.abs(c[others])) < 1e-10 and np.max(np.abs(d[others])) < 1e-10
    # and the TM slab gives different amplitudes (the weights matter)
    rm, _, _, _ = _te_slab((1.0, 1.0, 1.0), theta, 0.5, -0.5)
    assert abs(r) > 1e-3


@pytest.mark.parametrize("name,theta", [("small", -math.pi / 5), ("tiny", -1.3), ("small", None)])
def test_te_flux_conservation_corrugated(name, theta):
    """TE energy identity sum k_{1,n}|c_n|^2/eps1 + sum k_{3,n}|d_n|^2/eps3 = k1|sin theta|/eps1 on
    corrugated interfaces (theta None: the k1 Wood anomaly)."""
    g = dict(W.grating(name))
    g["pol"] = "TE"
    th = W.wood_angle(g["k"][0], g["d"]) if theta is None else theta
    eg, a = _solve_empty(g, th)
    assert L.flux_error(eg, a) < 1e-10


def test_te_flux_with_inclusions_and_absorption():
    """TE with the 10-disk workload: flux conserved for lossless disks; with lossy disks the outgoing
    flux falls below the incident one (absorption), and tends to the lossless value as Im kp -> 0."""
    cfg = W.config("small")
    g = dict(cfg["grating"])
    g["pol"] = "TE"
    dk = cfg["disks"]
    prob = S.setup(g, cfg["theta"], dk)
    beta, _, _ = S.solve_dense(prob)
    a, _, fe = prob.recover(beta)
    assert fe < 1e-11
    out0, inc = L.flux_balance(prob.eg, a)
    prev = None
    for eps in (1.0, 1e-2, 1e-4):
        lossy = dict(dk, kp=dk["kp"] + 1j * eps)
        pl = S.setup(g, cfg["theta"], lossy)
        bl, _, _ = S.solve_dense(pl)
        al, _, _ = pl.recover(bl)
        out, _ = L.flux_balance(pl.eg, al)
        assert out < inc * (1 - 1e-12)
        gap = inc - out
        if prev is not None:
            assert gap < prev
        prev = gap
    assert abs(out - out0) < 1e-3 * inc


def test_te_equals_tm_for_equal_permittivities():
    """With k1 = k2 = k3 the TE weights are all 1 and the TE system is the TM one."""
    g = dict(W.grating("tiny"))
    g["k"] = (8.0, 8.0, 8.0)
    dk = W.disks(5, 0.03, 0.015, 1.5, 8.0, seed=4, p=6)
    sols = []
    for pol in ("TM", "TE"):
        gg = dict(g, pol=pol)
        prob = S.setup(gg, -1.0, dk)
        beta, _, _ = S.solve_dense(prob)
        sols.append(prob.recover(beta)[0])
    # the disk coefficients differ (TE weighs the interior by 1/kp^2), so compare the empty grating
    egm = L.build_empty_grating(dict(g, pol="TM"), -1.0)
    ege = L.build_empty_grating(dict(g, pol="TE"), -1.0)
    assert np.max(np.abs(egm.A - ege.A)) == 0.0 and np.max(np.abs(egm.f - ege.f)) == 0.0
    assert np.all(np.isfinite(sols[1]))


def _ref_kernels_weighted(gr, t, s, shift, ka, kb, wa, wb, key):
    """(wa K^{ka} - wb K^{kb})(gamma(t), gamma(s) + shift) |gamma'(s)| for K = S or D, with R.n_y from
    Taylor remainders at short range; the double layer keeps its k-independent pole part
    (wa - wb) (R.n_y) / (2 pi r^2), bounded on the smooth curve."""
    from test_oracle_special import _y1_plus_pole
    ht, hs = gr.deriv(t, 0), gr.deriv(s, 0)
    hps = gr.deriv(s, 1)
    sps = np.sqrt(1 + hps ** 2)
    Rx = t - s - shift
    Ry = ht - hs
    RnyN = gr.remainder(s, t - s) if shift == 0 else Ry - hps * Rx
    Rny = RnyN / sps
    r = np.hypot(Rx, Ry)
    out = 0
    for k, w in ((ka, wa), (kb, -wb)):
        z = k * r
        if key == "S":
            v = 0.25j * hankel1(0, z)
        else:
            E1 = np.where(np.abs(z) < 2.0, 0.25j * k * (jv(1, z) + 1j * _y1_plus_pole(z)),
                          0.25j * k * hankel1(1, z) - 1 / (2 * np.pi * r))
            v = E1 * Rny / r + Rny / (2 * np.pi * r * r)
        out = out + w * v
    return out * sps


def _ref_apply_weighted(iface, xi, sig, alpha, ka, kb, wa, wb, key, d, lmax):
    from test_oracle_special import _Graph, _graded_nodes
    gr = _Graph(iface, d)
    tot = 0
    t64, w64 = np.polynomial.legendre.leggauss(64)
    for l in range(-lmax, lmax + 1):
        sing = xi - l * d
        if -0.5 * d - 0.2 < sing < 0.5 * d + 0.2:
            cc = min(max(sing, -0.5 * d), 0.5 * d)
            parts = []
            if cc > -0.5 * d:
                parts.append(_graded_nodes(-0.5 * d, cc, cc))
            if cc < 0.5 * d:
                parts.append(_graded_nodes(cc, 0.5 * d, cc))
        else:
            edges = np.linspace(-0.5 * d, 0.5 * d, 9)
            parts = [(0.5 * (a + b) + 0.5 * (b - a) * t64, 0.5 * (b - a) * w64) for a, b in zip(edges[:-1], edges[1:])]
        for s_, w in parts:
            tot += alpha ** l * np.sum(w * _ref_kernels_weighted(gr, xi, s_, l * d, ka, kb, wa, wb, key) * sig(s_))
    return tot


@pytest.mark.parametrize("key", ["S", "D"])
def test_weighted_self_operators_on_decaying_lattice(key):
    """wa K^{ka} - wb K^{kb} for the single and double layer with unequal weights (the TE value rows:
    the log singularity of S no longer cancels, and D keeps the Laplace double layer's curvature
    term): the Kress-corrected near operator plus the far copies against the lattice integral by
    graded Gauss-Legendre quadrature, whose kernels carry the weights explicitly."""
    g = W.grating("small")
    d = 1.0
    ka, kb = 10 + 8j, 6 + 9j
    wa, wb = 0.6, 1.45
    kap = 3.3
    alpha = np.exp(1j * kap * d)
    lmax = 5

    def sig(s):
        return np.exp(1j * kap * s) * (1 + 0.3 * np.cos(2 * np.pi * s / d) + 0.2j * np.sin(4 * np.pi * s / d))

    N = 256
    c = L.discretise_curve(g["gamma1"], d, N)
    ops = L.self_difference_operators(c, d, alpha, ka, kb, wa, wb)
    far = [l for l in range(-lmax, lmax + 1) if abs(l) >= 2]
    Fa = L.near_potentials(c.pos, c.nrm, c, d, alpha, ka, shifts=far)
    Fb = L.near_potentials(c.pos, c.nrm, c, d, alpha, kb, shifts=far)
    disc = (ops[key] + wa * Fa[key] - wb * Fb[key]) @ sig(c.x)
    for i in (0, 85, N - 1):
        ref = _ref_apply_weighted(g["gamma1"], c.x[i], sig, alpha, ka, kb, wa, wb, key, d, lmax)
        assert abs(disc[i] - ref) <= 1e-11 * abs(ref), (key, i, disc[i], ref)
