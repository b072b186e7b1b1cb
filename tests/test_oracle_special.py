"""Pins of the oracle's building blocks against mathematics that does not come from the oracle:
Bessel identities, Graf's addition theorem by direct evaluation, the disk transmission conditions,
S-matrix unitarity, exactness of the Kress weights, and the singular Nystrom operators against an
independent graded Gauss-Legendre quadrature on a decaying (complex-k) lattice."""
import math

import numpy as np
import pytest
from scipy.special import digamma, factorial, h1vp, hankel1, jv, jvp, yv

import workloads as W
from oracle import inclusions as I
from oracle import layers as L


def test_wronskian_of_library_bessel():
    # DLMF 10.5.2: J_{n+1}(z) Y_n(z) - J_n(z) Y_{n+1}(z) = 2/(pi z)
    z = np.linspace(0.05, 60.0, 400)
    for n in range(0, 30):
        w = jv(n + 1, z) * yv(n, z) - jv(n, z) * yv(n + 1, z)
        np.testing.assert_allclose(w, 2.0 / (np.pi * z), rtol=1e-10)


def test_graf_m2l_by_direct_evaluation():
    """Outgoing wave of particle j (and its +-d images, phases alpha^l) expanded about particle i
    with the oracle's translation matrix equals the directly evaluated wave (Sec. 4.2, Eq. trans)."""
    rng = np.random.default_rng(3)
    k, p, d = 17.0, 24, 1.0
    alpha = np.exp(1j * 0.7)
    xy = np.array([[0.1, 0.05], [-0.25, -0.2]])
    T = I.translation_matrix(xy, k, p, d, alpha)
    nc = 2 * p + 1
    for n_src in (-3, 0, 5):
        e = np.zeros(2 * nc, dtype=complex)
        e[nc + n_src + p] = 1.0                     # beta^j with j = particle 1, order n_src
        a = (T @ e)[:nc]                             # incoming coefficients at particle 0
        for _ in range(5):
            r, th = 0.02 * rng.random(), 2 * np.pi * rng.random()
            x = xy[0] + r * np.array([np.cos(th), np.sin(th)])
            direct = 0.0
            for l in (-1, 0, 1):
                v = x - (xy[1] + np.array([l * d, 0.0]))
                direct += alpha ** l * hankel1(n_src, k * np.hypot(*v)) * np.exp(1j * n_src * np.arctan2(v[1], v[0]))
            m = np.arange(-p, p + 1)
            series = np.sum(a * jv(m, k * r) * np.exp(1j * m * th))
            assert abs(series - direct) < 1e-12 * abs(direct)


def test_translation_excludes_only_self_l0():
    """A single particle sees its own +-d images but not itself (reading of Eq. repre3_mod)."""
    k, p, d = 9.0, 3, 1.0
    alpha = np.exp(0.4j)
    xy = np.array([[0.2, 0.1]])
    T = I.translation_matrix(xy, k, p, d, alpha)
    nc = 2 * p + 1
    m = np.arange(-p, p + 1)
    expect = np.zeros((nc, nc), dtype=complex)
    for l in (-1, 1):
        R = abs(l) * d
        Th = 0.0 if l == -1 else np.pi              # polar(c - (c + l d))
        q = m[None, :] - m[:, None]
        expect += alpha ** l * hankel1(q, k * R) * np.exp(1j * q * Th)
    np.testing.assert_allclose(T, expect, rtol=1e-13, atol=1e-13)


def test_graf_l2l_by_direct_evaluation():
    """The a2 columns of B: J_n about x2 re-expanded about a particle centre (Graf for J)."""
    g = W.grating("tiny")
    eg = L.build_empty_grating(g, -0.6)
    disks = {"xy": np.array([[0.13, -0.21]]), "radius": np.array([0.01]), "kp": np.array([12.0]), "p": 30}
    B = I.coupling_B(eg, disks)
    k = g["k"][1]
    Q2 = g["Q"][1]
    x2 = eg.centers[1]
    rng = np.random.default_rng(5)
    for ncol in (-Q2, -3, 0, 7, Q2):
        col = B[:, eg.cols["a2"]][:, ncol + Q2]
        for _ in range(4):
            r, th = 0.05 * rng.random(), 2 * np.pi * rng.random()
            x = disks["xy"][0] + r * np.array([np.cos(th), np.sin(th)])
            v = x - x2
            direct = jv(ncol, k * np.hypot(*v)) * np.exp(1j * ncol * np.arctan2(v[1], v[0]))
            m = np.arange(-30, 31)
            series = np.sum(col * jv(m, k * r) * np.exp(1j * m * th))
            assert abs(series - direct) < 1e-12 * max(1e-3, abs(direct))


def test_mie_transmission_conditions():
    """Sec. 4.1: J_n(k2 r) + s_n H_n(k2 r) outside and t_n J_n(kp r) inside match in value and
    radial derivative at r = R; and kp = k2 gives no scattering."""
    for (R, k2, kp) in ((0.04, 15.0, 20.0), (0.008, 60.0, 80.0), (0.3, 5.0, 11.0)):
        s = I.mie_coefficients(12, R, k2, kp)
        n = np.arange(-12, 13)
        t = (jv(n, k2 * R) + s * hankel1(n, k2 * R)) / jv(n, kp * R)
        lhs = k2 * (jvp(n, k2 * R) + s * h1vp(n, k2 * R))
        rhs = kp * t * jvp(n, kp * R)
        np.testing.assert_allclose(lhs, rhs, rtol=1e-9, atol=1e-300)
        np.testing.assert_allclose(s, s[::-1], rtol=1e-12)     # s_{-n} = s_n
    assert np.all(np.abs(I.mie_coefficients(10, 0.1, 7.0, 7.0)) < 1e-15)


def test_mie_unitarity_lossless():
    """A lossless disk: each partial S-matrix element 1 + 2 s_n has modulus one."""
    for (R, k2, kp) in ((0.04, 15.0, 20.0), (0.3, 5.0, 11.0), (0.02, 30.0, 75.0)):
        s = I.mie_coefficients(10, R, k2, kp)
        np.testing.assert_allclose(np.abs(1 + 2 * s), 1.0, atol=1e-13)


def test_cylinder_wave_gradients_by_finite_differences():
    """d_x f_n = (k/2)(f_{n-1} - f_{n+1}), d_y f_n = (ik/2)(f_{n-1} + f_{n+1}) as used for the
    J-expansion normal derivatives in A (checked on J and H waves)."""
    k, Q = 7.3, 6
    x0 = np.array([0.1, -0.2])
    pts = np.array([[0.5, 0.3], [-0.2, 0.6]])
    nx = np.array([[1.0, 0.0], [1.0, 0.0]])
    ny = np.array([[0.0, 1.0], [0.0, 1.0]])
    val, dnx = L.jexp_columns(pts, nx, x0, k, Q)
    _, dny = L.jexp_columns(pts, ny, x0, k, Q)
    h = 1e-6
    vxp, _ = L.jexp_columns(pts + [h, 0], nx, x0, k, Q)
    vxm, _ = L.jexp_columns(pts - [h, 0], nx, x0, k, Q)
    vyp, _ = L.jexp_columns(pts + [0, h], nx, x0, k, Q)
    vym, _ = L.jexp_columns(pts - [0, h], nx, x0, k, Q)
    np.testing.assert_allclose(dnx, (vxp - vxm) / (2 * h), rtol=1e-7, atol=1e-9)
    np.testing.assert_allclose(dny, (vyp - vym) / (2 * h), rtol=1e-7, atol=1e-9)


def test_kress_weights_exact_on_trig_polynomials():
    """int_0^{2pi} log(4 sin^2((t-s)/2)) e^{iqs} ds = -2pi/|q| e^{iqt} (q != 0), 0 (q = 0)."""
    N = 32
    R = L.kress_weights(N)
    s = 2 * np.pi * np.arange(N) / N
    for i in (0, 5, 17):
        t = s[i]
        for q in range(-N // 2 + 1, N // 2):
            approx = np.sum(R[(i - np.arange(N)) % N] * np.exp(1j * q * s))
            exact = 0.0 if q == 0 else -2 * np.pi / abs(q) * np.exp(1j * q * t)
            assert abs(approx - exact) < 1e-12


# ----------------------------------------------------------------------------------------------
# Singular Nystrom operators vs an independent quadrature on a decaying lattice (complex k)
# ----------------------------------------------------------------------------------------------

def _y1_plus_pole(z):
    """Y1(z) + 2/(pi z) computed without cancellation (ascending series for |z| < 2, DLMF 10.8.1)."""
    z = np.asarray(z, dtype=complex)
    out = np.empty_like(z)
    small = np.abs(z) < 2.0
    zs = z[small]
    ser = np.zeros_like(zs)
    for m in range(30):
        ser += (digamma(m + 1) + digamma(m + 2)) * (-zs * zs / 4) ** m * (zs / 2) / (factorial(m) * factorial(m + 1))
    out[small] = (2 / np.pi) * jv(1, zs) * np.log(zs / 2) - ser / np.pi
    out[~small] = yv(1, z[~small]) + 2 / (np.pi * z[~small])
    return out


class _Graph:
    """Exact geometry of a Fourier graph, with R.n computed from Taylor remainders at short range."""

    def __init__(self, iface, d):
        self.f, self.d = iface, d

    def deriv(self, x, m):
        out = np.zeros_like(x) + (self.f["h0"] if m == 0 else 0.0)
        for j, a in enumerate(self.f.get("cos", []), start=1):
            w = 2 * np.pi * j / self.d
            out = out + a * w ** m * np.cos(w * x + m * np.pi / 2)
        for j, b in enumerate(self.f.get("sin", []), start=1):
            w = 2 * np.pi * j / self.d
            out = out + b * w ** m * np.sin(w * x + m * np.pi / 2)
        return out

    def remainder(self, x, delta):
        """h(x + delta) - h(x) - h'(x) delta, accurate for small delta."""
        direct = self.deriv(x + delta, 0) - self.deriv(x, 0) - self.deriv(x, 1) * delta
        ser = np.zeros_like(delta)
        for m in range(2, 40):
            ser = ser + self.deriv(x, m) * delta ** m / math.factorial(m)
        return np.where(np.abs(delta) < 0.05, ser, direct)


def _ref_kernels(gr, t, s, shift, ka, kb, key):
    """(K^{ka} - K^{kb})(gamma(t), gamma(s) + shift) * |gamma'(s)| for K in S, D, N, T."""
    ht, hs = gr.deriv(t, 0), gr.deriv(s, 0)
    hpt, hps = gr.deriv(t, 1), gr.deriv(s, 1)
    spt, sps = np.sqrt(1 + hpt ** 2), np.sqrt(1 + hps ** 2)
    Rx = t - s - shift
    if shift == 0:
        # Ry - h'(t) Rx = -(h(s) - h(t) - h'(t)(s - t));  Ry - h'(s) Rx = h(t) - h(s) - h'(s)(t - s)
        RnxN = -gr.remainder(t, s - t)
        RnyN = gr.remainder(s, t - s)
        Ry = ht - hs
    else:
        Ry = ht - hs
        RnxN = Ry - hpt * Rx
        RnyN = Ry - hps * Rx
    Rnx, Rny = RnxN / spt, RnyN / sps
    nn = (hpt * hps + 1) / (spt * sps)
    r = np.hypot(Rx, Ry)
    out = 0
    for k, sg in ((ka, 1), (kb, -1)):
        z = k * r
        H0 = hankel1(0, z)
        # E1 = (ik/4) H1(kr) - 1/(2 pi r): series near 0, Hankel function elsewhere (J and Y
        # separately grow for complex z); the pole part is k-independent and cancels below
        E1 = np.where(np.abs(z) < 2.0, 0.25j * k * (jv(1, z) + 1j * _y1_plus_pole(z)),
                      0.25j * k * hankel1(1, z) - 1 / (2 * np.pi * r))
        if key == "S":
            v = 0.25j * H0
        elif key == "D":
            v = E1 * Rny / r
        elif key == "N":
            v = -E1 * Rnx / r
        else:
            # T = (ik^2/4) H0 P/r^2 + ((ik/4)H1)(-2P/r^3 + nn/r); the pole part is k-independent
            P = Rnx * Rny
            v = 0.25j * k * k * H0 * P / r ** 2 + E1 * (-2 * P / r ** 3 + nn / r)
        out = out + sg * v
    return out * sps


def _graded_nodes(a, b, sing, nlev=45, npan=16):
    """Composite Gauss-Legendre on [a, b] graded geometrically towards `sing` (an end point)."""
    t, w = np.polynomial.legendre.leggauss(npan)
    xs, ws = [], []
    L_ = b - a
    for j in range(nlev):
        hi, lo = L_ * 2.0 ** (-j), L_ * 2.0 ** (-j - 1)
        x = 0.5 * (hi + lo) + 0.5 * (hi - lo) * t
        xs.append(x)
        ws.append(0.5 * (hi - lo) * w)
    x = np.concatenate(xs)
    wt = np.concatenate(ws)
    return (a + x, wt) if sing == a else (b - x, wt)


def _ref_apply(gr, xi, sig, alpha, ka, kb, key, d, lmax):
    tot = 0
    t64, w64 = np.polynomial.legendre.leggauss(64)
    for l in range(-lmax, lmax + 1):
        sing = xi - l * d
        if -0.5 * d - 0.2 < sing < 0.5 * d + 0.2:
            c = min(max(sing, -0.5 * d), 0.5 * d)
            parts = []
            if c > -0.5 * d:
                parts.append(_graded_nodes(-0.5 * d, c, c))
            if c < 0.5 * d:
                parts.append(_graded_nodes(c, 0.5 * d, c))
        else:
            edges = np.linspace(-0.5 * d, 0.5 * d, 9)
            parts = [(0.5 * (a + b) + 0.5 * (b - a) * t64, 0.5 * (b - a) * w64) for a, b in zip(edges[:-1], edges[1:])]
        for s, w in parts:
            tot += alpha ** l * np.sum(w * _ref_kernels(gr, xi, s, l * d, ka, kb, key) * sig(s))
    return tot


@pytest.mark.parametrize("key", ["S", "D", "N", "T"])
def test_self_operators_spectral_on_decaying_lattice(key):
    """With Im k > 0 the lattice sum converges; the Kress-corrected near operator plus the plain
    trapezoid far copies must equal the lattice integral computed by graded Gauss-Legendre."""
    g = W.grating("small")
    d = 1.0
    ka, kb = 10 + 8j, 6 + 9j
    kap = 3.3
    alpha = np.exp(1j * kap * d)
    lmax = 5

    def sig(s):
        return np.exp(1j * kap * s) * (1 + 0.3 * np.cos(2 * np.pi * s / d) + 0.2j * np.sin(4 * np.pi * s / d))

    gr = _Graph(g["gamma1"], d)
    N = 256
    c = L.discretise_curve(g["gamma1"], d, N)
    ops = L.self_difference_operators(c, d, alpha, ka, kb)
    far = [l for l in range(-lmax, lmax + 1) if abs(l) >= 2]
    Fa = L.near_potentials(c.pos, c.nrm, c, d, alpha, ka, shifts=far)
    Fb = L.near_potentials(c.pos, c.nrm, c, d, alpha, kb, shifts=far)
    disc = (ops[key] + Fa[key] - Fb[key]) @ sig(c.x)
    for i in (0, 85, N - 1):
        ref = _ref_apply(gr, c.x[i], sig, alpha, ka, kb, key, d, lmax)
        assert abs(disc[i] - ref) <= 1e-11 * abs(ref), (key, i, disc[i], ref)


def test_self_operator_diagonal_is_load_bearing():
    """Planting a 1e-6 error in the T diagonal limit must break the lattice pin (sensitivity check)."""
    g = W.grating("small")
    d = 1.0
    ka, kb = 10 + 8j, 6 + 9j
    alpha = np.exp(3.3j)
    c = L.discretise_curve(g["gamma1"], d, 256)
    good = L.self_difference_operators(c, d, alpha, ka, kb)["T"]
    orig = L.diag_limits

    def planted(a, b, wa=1.0, wb=1.0):
        out = orig(a, b, wa, wb)
        out["T"] = (out["T"][0], out["T"][1] * (1 + 1e-6))
        return out

    L.diag_limits = planted
    try:
        bad = L.self_difference_operators(c, d, alpha, ka, kb)["T"]
    finally:
        L.diag_limits = orig
    x = np.ones(256)
    assert np.max(np.abs((bad - good) @ x)) > 1e-9 * np.max(np.abs(good @ x))


def test_c_direct_sum_matches_dense_translation():
    """The oracle's C direct sum (recurrence-based Hankel orders) equals the dense translation
    matrix built from scipy's Hankel functions order by order."""
    from oracle import m2l
    dk = W.disks(40, 0.01, 0.005, 2.0, 40.0, seed=3, p=12)
    al = np.exp(0.77j)
    T = I.translation_matrix(dk["xy"], 60.0, 12, 1.0, al)
    rng = np.random.default_rng(1)
    b = rng.standard_normal(T.shape[0]) + 1j * rng.standard_normal(T.shape[0])
    r1 = T @ b
    r2 = m2l.apply(dk["xy"], 60.0, 12, 1.0, al, b)
    assert np.linalg.norm(r1 - r2) <= 1e-13 * np.linalg.norm(r1)


def test_translation_rows_by_direct_field_modes():
    """translation_apply_rows (the reference of the sampled-row GPU checks) against the field it
    stands for: around target i, the directly summed outgoing waves of every other particle and of
    every +-d image (phases alpha^l, i's own l = 0 wave left out) have Fourier modes
    alpha_m J_m(k r) on a circle of radius r about c_i (Graf, Sec. 4.2 Eq. trans).  The modes come
    from an FFT of the directly evaluated field, not from any translation formula."""
    k, p, d = 60.0, 12, 1.0
    alpha = np.exp(-0.83j)
    dk = W.disks(40, 0.01, 0.005, 2.0, 40.0, seed=8, p=p)
    xy = dk["xy"]
    M, nc = xy.shape[0], 2 * p + 1
    rng = np.random.default_rng(4)
    w = np.tile(0.5 ** np.abs(np.arange(-p, p + 1)), M)
    beta = (rng.standard_normal(M * nc) + 1j * rng.standard_normal(M * nc)) * w
    B = beta.reshape(M, nc)
    rows = [0, 17, 39]
    got = I.translation_apply_rows(xy, k, p, d, alpha, beta, rows)
    n = np.arange(-p, p + 1)
    npts = 256
    t = 2 * np.pi * np.arange(npts) / npts
    for row, i in zip(got, rows):
        srcs = [(j, l) for l in (-1, 0, 1) for j in range(M) if not (l == 0 and j == i)]
        dist = min(np.hypot(*(xy[i] - xy[j] - [l * d, 0.0])) for j, l in srcs)
        r = 0.6 * dist
        x = xy[i][None, :] + r * np.stack([np.cos(t), np.sin(t)], axis=1)
        u = np.zeros(npts, dtype=complex)
        for j, l in srcs:
            v = x - (xy[j] + [l * d, 0.0])
            rho, ph = np.hypot(v[:, 0], v[:, 1]), np.arctan2(v[:, 1], v[:, 0])
            u += alpha ** l * (hankel1(n[None, :], k * rho[:, None]) * np.exp(1j * n[None, :] * ph[:, None])) @ B[j]
        modes = np.fft.fft(u) / npts            # mode m at index m mod npts
        c = modes[n % npts]
        expect = row * jv(n, k * r)
        scale = np.max(np.abs(u))
        assert np.max(np.abs(c - expect)) <= 1e-11 * scale, i
        # the check is not vacuous: the highest orders carry a visible share of the field
        assert np.abs(expect[[0, -1]]).max() > 1e-6 * scale


def test_translation_rows_match_dense_matrix_and_c_direct_sum():
    """translation_apply_rows equals the rows of the dense matrix and of the C direct sum
    (three independent evaluations of Eq. trans), for first, middle and last targets: on a dense
    40-disk geometry, and entry by entry on a sparse one whose +-d images carry a large share of
    every entry (so a wrong image phase or self-image mask cannot hide under near-pair terms)."""
    from oracle import m2l
    k, p, d = 60.0, 12, 1.0
    nc = 2 * p + 1
    al = np.exp(0.41j)
    for M, gap, wdec in ((40, 0.005, 1.0), (6, 0.25, 0.3)):
        dk = W.disks(M, 0.01, gap, 2.0, 40.0, seed=5, p=p)
        rng = np.random.default_rng(6)
        w = np.tile(wdec ** np.abs(np.arange(-p, p + 1)), M)
        b = (rng.standard_normal(M * nc) + 1j * rng.standard_normal(M * nc)) * w
        rows = [0, 1, M // 2, M - 2, M - 1]
        got = I.translation_apply_rows(dk["xy"], k, p, d, al, b, rows)
        dense = (I.translation_matrix(dk["xy"], k, p, d, al) @ b).reshape(M, nc)[rows]
        csum = m2l.apply(dk["xy"], k, p, d, al, b).reshape(M, nc)[rows]
        if M > 10:
            assert np.linalg.norm(got - dense) <= 1e-13 * np.linalg.norm(dense)
            assert np.linalg.norm(got - csum) <= 1e-13 * np.linalg.norm(dense)
        else:
            np.testing.assert_allclose(got, dense, rtol=1e-12, atol=0)
            np.testing.assert_allclose(got, csum, rtol=1e-12, atol=0)
