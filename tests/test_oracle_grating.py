"""Pins of the oracle's empty-grating block A against closed forms and the paper's printed values:
a transparent grating (exact plane wave), the flat three-layer slab (transfer matrix), the
paper's Fig. 2 matrix size and flux accuracy, and the Wood-anomaly branch."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import layers as L


def _solve(g, theta):
    eg = L.build_empty_grating(g, theta)
    pinv = L.factor(eg)
    a = pinv.apply(eg.f)
    return eg, a


def test_fig2_matrix_size_and_flux():
    """Sec. 6: N=120, 50 points on Gamma_u/Gamma_d, 2Q+1=73, 41 Rayleigh-Bloch modes give A of
    size 1020 x 781 (the paper prints exactly this); Fig. 2 reports a flux error near 1e-13."""
    g = W.grating("fig2")
    eg, a = _solve(g, -math.pi / 5)
    assert eg.A.shape == (1020, 781)
    assert L.flux_error(eg, a) < 1e-10


def test_transparent_corrugated_grating_is_a_plane_wave():
    """k1 = k2 = k3 with corrugated interfaces: no reflection, c = 0, and the field below is the
    incident plane wave, d_0 = exp(i k_{3,0} y0), all other d_n = 0."""
    g = dict(W.grating("tiny"))
    g["k"] = (8.0, 8.0, 8.0)
    theta = -1.1
    eg, a = _solve(g, theta)
    c = a[eg.cols["c"]]
    d = a[eg.cols["d"]]
    K = g["K_rb"]
    d_exact = np.zeros(2 * K + 1, dtype=complex)
    d_exact[K] = np.exp(1j * eg.k3n[K] * g["y0"])
    assert np.max(np.abs(c)) < 1e-11
    assert np.max(np.abs(d - d_exact)) < 1e-11


def _slab(k, theta, a_top, b_bot):
    """Textbook three-layer slab: u1 = e^{i(kx x - q1 y)} + r e^{i(kx x + q1 y)},
    u2 = A e^{-i q2 y} + B e^{i q2 y}, u3 = t e^{-i q3 y}; continuity of u, u_y at y = a, b."""
    k1, k2, k3 = k
    kx = k1 * math.cos(theta)
    q = [np.sqrt(complex(kk * kk - kx * kx)) for kk in k]
    q1, q2, q3 = q
    M = np.zeros((4, 4), dtype=complex)
    rhs = np.zeros(4, dtype=complex)
    ea = lambda qq, s: np.exp(1j * s * qq * a_top)
    eb = lambda qq, s: np.exp(1j * s * qq * b_bot)
    # unknowns r, A, B, t
    M[0] = [ea(q1, 1), -ea(q2, -1), -ea(q2, 1), 0]
    rhs[0] = -ea(q1, -1)
    M[1] = [1j * q1 * ea(q1, 1), 1j * q2 * ea(q2, -1), -1j * q2 * ea(q2, 1), 0]
    rhs[1] = 1j * q1 * ea(q1, -1)
    M[2] = [0, eb(q2, -1), eb(q2, 1), -eb(q3, -1)]
    M[3] = [0, -1j * q2 * eb(q2, -1), 1j * q2 * eb(q2, 1), 1j * q3 * eb(q3, -1)]
    r, A, B, t = np.linalg.solve(M, rhs)
    return r, t, q1, q3


def test_flat_slab_matches_transfer_matrix():
    """Flat interfaces y = 0.5, y = -0.5: only order 0 is excited, c_0 = r e^{i q1 y0},
    d_0 = t e^{i q3 y0}, all other orders vanish (Sec. 2 Eqs. rad1-rad2)."""
    g = dict(W.grating("small"))
    g["gamma1"] = {"h0": 0.5, "cos": [], "sin": []}
    g["gamma2"] = {"h0": -0.5, "cos": [], "sin": []}
    theta = -0.9
    eg, a = _solve(g, theta)
    r, t, q1, q3 = _slab(g["k"], theta, 0.5, -0.5)
    K = g["K_rb"]
    c = a[eg.cols["c"]]
    d = a[eg.cols["d"]]
    y0 = g["y0"]
    assert abs(c[K] - r * np.exp(1j * q1 * y0)) < 1e-10
    assert abs(d[K] - t * np.exp(1j * q3 * y0)) < 1e-10
    others = np.r_[np.arange(K), np.arange(K + 1, 2 * K + 1)]
    assert np.max(np.abs(c[others])) < 1e-10
    assert np.max(np.abs(d[others])) < 1e-10


@pytest.mark.parametrize("name", ["small", "tiny"])
def test_flux_conservation_corrugated(name):
    """Sec. 6: for real wavenumbers the Bragg powers add up to the incident power."""
    g = W.grating(name)
    for theta in (-math.pi / 5, -1.3):
        eg, a = _solve(g, theta)
        assert L.flux_error(eg, a) < 1e-10


def test_flux_at_wood_anomaly():
    """Sec. 2 and Ex. 2: at a Wood anomaly (k_{1,n} = 0 for one order) the scheme stays accurate."""
    g = dict(W.grating("small"))
    theta = W.wood_angle(g["k"][0], g["d"])
    eg, a = _solve(g, theta)
    assert np.any(eg.k1n == 0)
    assert L.flux_error(eg, a) < 1e-9


def test_kvert_branch():
    """k_{j,n} = +sqrt(k^2 - kappa^2): positive real or positive imaginary, snapped to 0."""
    kap = np.array([-12.0, -10.0 * (1 + 1e-14), 0.0, 3.0, 11.0])
    v = L.kvert(10.0, kap)
    assert v[0].real == 0 and v[0].imag > 0
    assert v[1] == 0
    assert v[2] == 10.0
    assert v[3].real > 0 and v[3].imag == 0
    assert v[4].imag > 0


def test_shift_invariance_of_bragg_magnitudes():
    """Shifting the whole grating by delta in x multiplies c_n, d_n by exp(-2 pi i n delta / d)."""
    g = dict(W.grating("tiny"))
    theta = -0.8
    eg0, a0 = _solve(g, theta)
    delta = 0.137
    w = 2 * math.pi / g["d"]
    g2 = dict(g)
    # cos(w (x - delta)) = cos(w delta) cos(w x) + sin(w delta) sin(w x)
    for key in ("gamma1", "gamma2"):
        a = g[key]["cos"][0]
        g2[key] = {"h0": g[key]["h0"], "cos": [a * math.cos(w * delta)], "sin": [a * math.sin(w * delta)]}
    eg1, a1 = _solve(g2, theta)
    n = np.arange(-g["K_rb"], g["K_rb"] + 1)
    ph = np.exp(-1j * w * n * delta)
    for blk in ("c", "d"):
        np.testing.assert_allclose(a1[eg1.cols[blk]], a0[eg0.cols[blk]] * ph, atol=1e-10)
