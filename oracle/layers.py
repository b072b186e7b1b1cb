"""Oracle for the empty layered grating: discretisation, the block matrix A, its pseudo-inverse.

TEST INFRASTRUCTURE (see the package docstring): never used by the product path.

Follows Sec. 3 of the paper (Eqs. repre1-repre3, slp, dlp, jr1-jr4, bound1-bound3, matA, Arhs),
Sec. 5 (Eq. applypA and the remark after it) and Sec. 6 (flux identity).  Readings taken where the
paper is silent or garbled:

  * The unknown vector is [mu1, sigma1, mu2, sigma2, a2, a1, a3, c, d] (Eq. matA) and the block
    A11 acts on [mu; sigma] as [[I + D1-D2, S1-S2], [T1-T2, -I + N1-N2]] (the printed block has the
    off-diagonal entries swapped with respect to Eqs. intg1-intg2; this order follows from the jump
    relations).
  * Jump relations with the normal pointing to the + side: (S s)_n^{+-} = (-+1/2 + N) s and
    (D m)^{+-} = (+-1/2 + D) m.  Interface and Gamma_u/Gamma_d normals point up (+y); wall normals
    are +x on both walls.
  * The Gamma1 rows carry the a1 J-expansion and the Gamma2 rows the a3 J-expansion (both are part
    of u1 and u3 by Eqs. repre1 and repre2, although Eq. matA prints zeros there).
  * The last row of Eq. bound3 is read with u3: d_y u3 + sum_n i k_{3,n} d_n e^{i kappa_n x} = 0.
  * Wall discrepancies use the cancelled form (Remark "cancel"): alpha u(L) - u(R) over the three
    near copies equals alpha^2 u_{+1}(L) - alpha^{-1} u_{-2}(L), so walls never see a near source.
  * Singular quadrature: the paper's 16th-order Alpert tables are not reproduced; instead the
    periodic log-singular product rule of Kress (1991) is applied to a windowed log coefficient
    (a C-infinity flat-top window in the parameter), with the Bloch phase applied to neighbours
    that wrap around the period end.  Only kernel differences k_a - k_b enter (Sec. 3, A11).
  * J-expansion columns are rescaled to unit 2-norm before the SVD (Sec. 3, Fig. 2a remark).
  * Sigma^+ = min(1/sigma_j, 1/eps) taken literally (a clip, not a truncation), eps absolute.
  * Wood branch: k_{j,n} = +sqrt(k_j^2 - kappa_n^2), principal branch; |k_j^2-kappa_n^2| <
    1e-12 k_j^2 is set to 0.
  * TE polarisation (Sec. 2 names it and Sec. 7 leaves it to future work; g["pol"] = "TE"): u is the
    magnetic field and the flux condition on every interface carries the inverse permittivity,
    [u] = 0, [(1/eps) d_n u] = 0, with eps_j proportional to k_j^2 (constant permeability, Sec. 2).
    Relative to the middle layer, w_j = eps_j / eps_2 = (k_j / k_2)^2.  Each layer's potentials are
    scaled by its w_j (u_j = w_j (D mu + S sigma) + J-expansions, Mueller's choice), which keeps the
    system of the second kind: the value rows of an interface carry (w_a + w_b)/2 I + w_a D_a - w_b D_b
    and w_a S_a - w_b S_b, the flux rows (1/w_j) d_n of each side, where the potentials' hypersingular
    parts still cancel (T_a - T_b, N_a - N_b).  The J-expansion and Rayleigh-Bloch unknowns absorb
    the scaling.  TM is w_j = 1.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
from scipy.special import hankel1, jv

EULER = float(np.euler_gamma)
WINDOW_A = 0.05   # flat-top half-width of the log-coefficient window (fraction of a period)
WINDOW_B = 0.45   # the window vanishes beyond this half-width
SNAP_REL = 1e-12  # Wood branch snapping threshold (relative to k_j^2)


# ----------------------------------------------------------------------------------------------
# Geometry and discretisation (Sec. 3, "We discretize the four interfaces ...")
# ----------------------------------------------------------------------------------------------

def iface_eval(iface: dict, d: float, x):
    """h(x), h'(x), h''(x) of the graph y = h0 + sum_m a_m cos(2 pi m x/d) + b_m sin(2 pi m x/d)."""
    x = np.asarray(x, dtype=np.float64)
    h = np.full_like(x, iface["h0"])
    hp = np.zeros_like(x)
    hpp = np.zeros_like(x)
    for m, a in enumerate(iface.get("cos", []), start=1):
        w = 2.0 * math.pi * m / d
        h += a * np.cos(w * x)
        hp += -a * w * np.sin(w * x)
        hpp += -a * w * w * np.cos(w * x)
    for m, b in enumerate(iface.get("sin", []), start=1):
        w = 2.0 * math.pi * m / d
        h += b * np.sin(w * x)
        hp += b * w * np.cos(w * x)
        hpp += -b * w * w * np.sin(w * x)
    return h, hp, hpp


@dataclass
class Curve:
    """N equispaced parameter nodes x_i = -d/2 + (i+1/2) d/N on one period of an interface."""
    x: np.ndarray
    pos: np.ndarray      # (N,2)
    nrm: np.ndarray      # (N,2) upward unit normal
    speed: np.ndarray    # |gamma'(x)|
    w: np.ndarray        # periodic trapezoid weights h*speed
    h: float
    curv: np.ndarray = None   # signed curvature h'' / (1 + h'^2)^{3/2} (with respect to the upward normal)


def discretise_curve(iface: dict, d: float, N: int) -> Curve:
    hstep = d / N
    x = -0.5 * d + (np.arange(N) + 0.5) * hstep
    y, yp, ypp = iface_eval(iface, d, x)
    speed = np.sqrt(1.0 + yp * yp)
    nrm = np.stack([-yp / speed, 1.0 / speed], axis=1)
    pos = np.stack([x, y], axis=1)
    return Curve(x=x, pos=pos, nrm=nrm, speed=speed, w=hstep * speed, h=hstep, curv=ypp / speed**3)


def gauss_legendre(n: int, lo: float, hi: float) -> np.ndarray:
    t, _ = np.polynomial.legendre.leggauss(n)
    return 0.5 * (hi + lo) + 0.5 * (hi - lo) * t


# ----------------------------------------------------------------------------------------------
# Kernels (Sec. 3, Eqs. slp, dlp and the N, T operators; G_k = (i/4) H_0(k |x-y|))
# ----------------------------------------------------------------------------------------------

def kernels(tpos, tnrm, spos, snrm, k):
    """S, D, N, T kernels between targets (T,2) and sources (S,2); R = x - y.

    S = (i/4) H0(kr);  D = dG/dn_y = (ik/4) H1(kr) R.n_y / r;  N = dG/dn_x = -(ik/4) H1(kr) R.n_x / r;
    T = d2G/dn_x dn_y = (ik/4) [k H0 R.n_x R.n_y / r^2 - 2 H1 R.n_x R.n_y / r^3 + H1 n_x.n_y / r].
    """
    Rx = tpos[:, None, 0] - spos[None, :, 0]
    Ry = tpos[:, None, 1] - spos[None, :, 1]
    r = np.hypot(Rx, Ry)
    kr = k * r
    H0 = hankel1(0, kr)
    H1 = hankel1(1, kr)
    Rnx = Rx * tnrm[:, None, 0] + Ry * tnrm[:, None, 1]
    Rny = Rx * snrm[None, :, 0] + Ry * snrm[None, :, 1]
    nn = tnrm[:, None, 0] * snrm[None, :, 0] + tnrm[:, None, 1] * snrm[None, :, 1]
    S = 0.25j * H0
    D = 0.25j * k * H1 * Rny / r
    N = -0.25j * k * H1 * Rnx / r
    T = 0.25j * k * (k * H0 * Rnx * Rny / r**2 - 2.0 * H1 * Rnx * Rny / r**3 + H1 * nn / r)
    return {"S": S, "D": D, "N": N, "T": T}


def diag_limits(ka, kb, wa=1.0, wb=1.0):
    """Limits at coincidence of the kernel differences, per unit arc length: wa S_ka - wb S_kb and
    wa D_ka - wb D_kb for S and D, plain differences (ka - kb) for N and T.

    Returns (K1, Krest) for each of S, D, N, T where K = K1 log r + Krest + o(1) as y -> x on a
    smooth curve.  Small-argument forms: H0(z) = 1 + (2i/pi)(log(z/2) + gamma) + ..., and
    H1(z) = -2i/(pi z) + z/2 + (iz/pi) log(z/2) - (iz/(2 pi))(1 - 2 gamma) + ...; the curvature
    terms of N and the hypersingular part of T do not depend on k and cancel in the differences.
    D's limit is (wa - wb) kappa / (4 pi), kappa the curvature (the Laplace double layer's
    (R.n_y)/(2 pi r^2) tends to kappa/(4 pi)): it is returned per unit curvature.
    """
    ka = complex(ka)
    kb = complex(kb)
    la = np.log(ka / 2.0)
    lb = np.log(kb / 2.0)
    def s_rest(k_log):
        return 0.25j - (k_log + EULER) / (2.0 * math.pi)
    S = (-(wa - wb) / (2.0 * math.pi), wa * s_rest(la) - wb * s_rest(lb))
    D = (0.0, (wa - wb) / (4.0 * math.pi))
    N = (0.0, 0.0)
    dk2 = ka * ka - kb * kb
    T = (-dk2 / (4.0 * math.pi),
         1j * dk2 / 8.0 - (ka * ka * la - kb * kb * lb) / (4.0 * math.pi)
         + dk2 * (1.0 - 2.0 * EULER) / (8.0 * math.pi))
    return {"S": S, "D": D, "N": N, "T": T}


def window(u, a=WINDOW_A, b=WINDOW_B):
    """C-infinity flat-top window: 1 for |u| <= a, 0 for |u| >= b, smooth step in between."""
    u = np.abs(np.asarray(u, dtype=np.float64))
    out = np.zeros_like(u)
    out[u <= a] = 1.0
    mid = (u > a) & (u < b)
    v = (u[mid] - a) / (b - a)
    f1 = np.exp(-1.0 / v)
    f2 = np.exp(-1.0 / (1.0 - v))
    out[mid] = f2 / (f1 + f2)
    return out


def kress_weights(N: int) -> np.ndarray:
    """R_m, m = 0..N-1: weights of the periodic rule int_0^{2pi} log(4 sin^2((t-s)/2)) f(s) ds ~
    sum_j R_{(i-j) mod N} f(s_j) on N equispaced nodes with t = s_i (Kress 1991), exact for
    trigonometric polynomials of degree <= N/2."""
    m = np.arange(N)
    q = np.arange(1, N // 2)
    R = -(4.0 * math.pi / N) * (np.cos(2.0 * math.pi * np.outer(m, q) / N) / q).sum(axis=1)
    R -= (4.0 * math.pi / N**2) * np.cos(math.pi * m)
    return R


def self_difference_operators(c: Curve, d: float, alpha: complex, ka, kb, wa=1.0, wb=1.0):
    """Nystrom matrices of wa S^{ka} - wb S^{kb}, wa D^{ka} - wb D^{kb}, N^{ka} - N^{kb},
    T^{ka} - T^{kb} on one interface, summed over the near copies l = -1, 0, 1 with Bloch phases
    alpha^l (Sec. 3, A11 and Eq. qGreen2 with P = 1; the weights are the TE permittivity ratios,
    1 for TM).

    A_ij = h F_ij + (W_ij - h log(4 sin^2(pi (i-j)/N))) L_ij   (j != i)
    A_ii = h F_ii + W_ii L_ii + h speed_i [ (K1_ii/2) log(speed_i^2 d^2/(4 pi^2)) + Krest_ii ]
    with F the near-copy kernel sum times speed (the l=0 diagonal left out), L the windowed log
    coefficient (K1/2 times speed, on the copy of node j within half a period of node i, times
    that copy's phase), W the Kress weights in the parameter."""
    N = c.x.size
    h = c.h
    out = {}
    F = {key: np.zeros((N, N), dtype=np.complex128) for key in "SDNT"}
    for l in (-1, 0, 1):
        spos = c.pos + np.array([l * d, 0.0])
        with np.errstate(divide="ignore", invalid="ignore"):   # l = 0 diagonal is left out
            Ka = kernels(c.pos, c.nrm, spos, c.nrm, ka)
            Kb = kernels(c.pos, c.nrm, spos, c.nrm, kb)
        ph = alpha ** l
        for key in "SDNT":
            wgt_a, wgt_b = (wa, wb) if key in "SD" else (1.0, 1.0)
            diff = wgt_a * Ka[key] - wgt_b * Kb[key]
            if l == 0:
                np.fill_diagonal(diff, 0.0)
            F[key] += ph * diff
    # windowed log coefficient on the nearest copy
    dx = (c.x[None, :] - c.x[:, None]) / d
    lstar = -np.round(dx)                      # copy of node j nearest to node i
    u = dx + lstar
    psi = window(u)
    spos_near_x = c.pos[None, :, 0] + lstar * d
    Rx = c.pos[:, None, 0] - spos_near_x
    Ry = c.pos[:, None, 1] - c.pos[None, :, 1]
    # log coefficients evaluated pair by pair on the chosen copy
    r = np.hypot(Rx, Ry)
    np.fill_diagonal(r, 1.0)
    Rnx = Rx * c.nrm[:, None, 0] + Ry * c.nrm[:, None, 1]
    Rny = Rx * c.nrm[None, :, 0] + Ry * c.nrm[None, :, 1]
    nn = c.nrm[:, None, 0] * c.nrm[None, :, 0] + c.nrm[:, None, 1] * c.nrm[None, :, 1]
    K1 = {}
    for key in "SDNT":
        K1[key] = np.zeros((N, N), dtype=np.complex128)
    for k, sgn, wsd in ((ka, 1.0, wa), (kb, -1.0, wb)):
        kr = k * r
        J0 = jv(0, kr)
        J1 = jv(1, kr)
        cc = -1.0 / (2.0 * math.pi)
        K1["S"] += sgn * wsd * cc * J0
        K1["D"] += sgn * wsd * cc * k * J1 * Rny / r
        K1["N"] += sgn * (-cc) * k * J1 * Rnx / r
        K1["T"] += sgn * cc * k * (k * J0 * Rnx * Rny / r**2 - 2.0 * J1 * Rnx * Rny / r**3
                                   + J1 * nn / r)
    phase = alpha ** lstar
    R = kress_weights(N)
    idx = (np.arange(N)[:, None] - np.arange(N)[None, :]) % N
    W = (d / (2.0 * math.pi)) * R[idx]
    with np.errstate(divide="ignore"):
        logt = np.log(4.0 * np.sin(math.pi * idx / N) ** 2)
    np.fill_diagonal(logt, 0.0)
    lim = diag_limits(ka, kb, wa, wb)
    for key in "SDNT":
        L = psi * 0.5 * K1[key] * phase * c.speed[None, :]
        np.fill_diagonal(L, 0.5 * lim[key][0] * c.speed)
        A = h * F[key] * c.speed[None, :] + (W - h * logt) * L
        rest = lim[key][1] * (c.curv if key == "D" else 1.0)
        diag = (h * np.diag(F[key]) * c.speed + W[0, 0] * 0.5 * lim[key][0] * c.speed
                + h * c.speed * (0.5 * lim[key][0] * np.log(c.speed**2 * d * d / (4.0 * math.pi**2))
                                 + rest))
        np.fill_diagonal(A, diag)
        out[key] = A
    return out


def near_potentials(tpos, tnrm, c: Curve, d: float, alpha: complex, k, shifts=(-1, 0, 1),
                    phases=None):
    """Plain-trapezoid layer potentials at off-curve targets: sum over copies l of
    phase_l * K(x, y_j + l d) w_j, for K in S, D, N, T (target normal tnrm)."""
    if phases is None:
        phases = [alpha ** l for l in shifts]
    out = {key: np.zeros((tpos.shape[0], c.x.size), dtype=np.complex128) for key in "SDNT"}
    for l, ph in zip(shifts, phases):
        spos = c.pos + np.array([l * d, 0.0])
        K = kernels(tpos, tnrm, spos, c.nrm, k)
        for key in "SDNT":
            out[key] += ph * K[key] * c.w[None, :]
    return out


# ----------------------------------------------------------------------------------------------
# Cylindrical waves C_n(k|x-c|) e^{i n theta} and their gradients
# ----------------------------------------------------------------------------------------------

def jexp_columns(tpos, tnrm, center, k, Q):
    """Values and normal derivatives of J_n(k|x-x0|) e^{i n theta_{x-x0}}, n = -Q..Q, using
    d_x f_n = (k/2)(f_{n-1} - f_{n+1}) and d_y f_n = (ik/2)(f_{n-1} + f_{n+1})."""
    Rx = tpos[:, 0] - center[0]
    Ry = tpos[:, 1] - center[1]
    rho = np.hypot(Rx, Ry)
    th = np.arctan2(Ry, Rx)
    n = np.arange(-Q - 1, Q + 2)
    f = jv(n[None, :], k * rho[:, None]) * np.exp(1j * n[None, :] * th[:, None])
    val = f[:, 1:-1]
    fx = 0.5 * k * (f[:, :-2] - f[:, 2:])
    fy = 0.5j * k * (f[:, :-2] + f[:, 2:])
    dn = tnrm[:, 0:1] * fx + tnrm[:, 1:2] * fy
    return val, dn


# ----------------------------------------------------------------------------------------------
# Bloch and Rayleigh-Bloch quantities (Sec. 2, Eqs. quasi, rad1, rad2)
# ----------------------------------------------------------------------------------------------

def kappa_n(k1, theta, d, K):
    n = np.arange(-K, K + 1)
    return k1 * math.cos(theta) + 2.0 * math.pi * n / d


def kvert(kj, kap):
    """k_{j,n} = +sqrt(k_j^2 - kappa_n^2), positive real or positive imaginary, snapped to 0."""
    s = kj * kj - kap * kap
    out = np.where(s >= 0, np.sqrt(np.abs(s)) + 0j, 1j * np.sqrt(np.abs(s)))
    out = np.where(np.abs(s) < SNAP_REL * kj * kj, 0.0 + 0j, out)
    return out


# ----------------------------------------------------------------------------------------------
# The block matrix A (Eq. matA) and right-hand side f (Eq. Arhs)
# ----------------------------------------------------------------------------------------------

COL_BLOCKS = ("mu1", "sigma1", "mu2", "sigma2", "a2", "a1", "a3", "c", "d")
ROW_BLOCKS = ("g1v", "g1n", "g2v", "g2n", "w2v", "w2n", "w1v", "w1n", "w3v", "w3n",
              "uv", "un", "dv", "dn")


@dataclass
class EmptyGrating:
    g: dict
    theta: float
    d: float
    k: tuple
    alpha: complex
    kappa: np.ndarray
    k1n: np.ndarray
    k3n: np.ndarray
    c1: Curve
    c2: Curve
    centers: tuple
    wall_y: tuple           # GL nodes on walls of layers 1, 2, 3
    bound_x: np.ndarray     # nodes on Gamma_u / Gamma_d
    cols: dict = field(default_factory=dict)
    rows: dict = field(default_factory=dict)
    A: np.ndarray = None
    f: np.ndarray = None

    @property
    def shape(self):
        return self.A.shape


def _offsets(sizes: dict, order) -> dict:
    out, o = {}, 0
    for name in order:
        out[name] = slice(o, o + sizes[name])
        o += sizes[name]
    return out


def layer_weights(g: dict):
    """(w1, w3): the permittivities of the top and bottom layers relative to the middle layer,
    (k_j / k_2)^2, for TE polarisation; (1, 1) for TM (g["pol"], TM when absent)."""
    pol = g.get("pol", "TM")
    if pol == "TM":
        return 1.0, 1.0
    if pol != "TE":
        raise ValueError(f"unknown polarisation {pol!r}")
    k1, k2, k3 = g["k"]
    return (k1 / k2) ** 2, (k3 / k2) ** 2


def build_empty_grating(g: dict, theta: float) -> EmptyGrating:
    """Assemble A and f for the grating g at incidence theta (Sec. 3, Eqs. bound1-bound3, matA)."""
    d = g["d"]
    k1, k2, k3 = g["k"]
    N = g["N"]
    Q1, Q2, Q3 = g["Q"]
    K = g["K_rb"]
    y0 = g["y0"]
    nw1, nw2, nw3 = g["n_wall"]
    nb = g["n_bound"]
    kap0 = k1 * math.cos(theta)
    alpha = np.exp(1j * kap0 * d)
    kap = kappa_n(k1, theta, d, K)
    k1n = kvert(k1, kap)
    k3n = kvert(k3, kap)
    c1 = discretise_curve(g["gamma1"], d, N)
    c2 = discretise_curve(g["gamma2"], d, N)
    h10 = g["gamma1"]["h0"]
    h20 = g["gamma2"]["h0"]
    x1 = np.array([0.0, 0.5 * (h10 + y0)])
    x2 = np.array([0.0, 0.5 * (h10 + h20)])
    x3 = np.array([0.0, 0.5 * (h20 - y0)])
    yL1 = iface_eval(g["gamma1"], d, np.array([-0.5 * d]))[0][0]
    yL2 = iface_eval(g["gamma2"], d, np.array([-0.5 * d]))[0][0]
    wall1 = gauss_legendre(nw1, yL1, y0)
    wall2 = gauss_legendre(nw2, yL2, yL1)
    wall3 = gauss_legendre(nw3, -y0, yL2)
    bx = -0.5 * d + (np.arange(nb) + 0.5) * d / nb

    eg = EmptyGrating(g=g, theta=theta, d=d, k=(k1, k2, k3), alpha=alpha, kappa=kap, k1n=k1n,
                      k3n=k3n, c1=c1, c2=c2, centers=(x1, x2, x3), wall_y=(wall1, wall2, wall3),
                      bound_x=bx)
    w1, w3 = layer_weights(g)
    csz = dict(mu1=N, sigma1=N, mu2=N, sigma2=N, a2=2 * Q2 + 1, a1=2 * Q1 + 1, a3=2 * Q3 + 1,
               c=2 * K + 1, d=2 * K + 1)
    rsz = dict(g1v=N, g1n=N, g2v=N, g2n=N, w2v=nw2, w2n=nw2, w1v=nw1, w1n=nw1, w3v=nw3, w3n=nw3,
               uv=nb, un=nb, dv=nb, dn=nb)
    eg.cols = _offsets(csz, COL_BLOCKS)
    eg.rows = _offsets(rsz, ROW_BLOCKS)
    nrow = sum(rsz.values())
    ncol = sum(csz.values())
    A = np.zeros((nrow, ncol), dtype=np.complex128)
    C, R = eg.cols, eg.rows

    def put(rv, rn, cm, cs, P, wgt=1.0):
        """value rows get D (mu) and S (sigma); derivative rows get T (mu) and N (sigma); all scaled
        by the layer's TE weight wgt."""
        A[R[rv], C[cm]] += wgt * P["D"]
        A[R[rv], C[cs]] += wgt * P["S"]
        A[R[rn], C[cm]] += wgt * P["T"]
        A[R[rn], C[cs]] += wgt * P["N"]

    # --- Gamma1 rows: u1 - u2 = -u_inc, d_n u1 - d_n u2 = -d_n u_inc (Eq. bound1) -------------
    # u1 = w1 (D mu1 + S sigma1) + J(a1) + u_inc above, u2 = D mu1 + S sigma1 + ... below; the flux
    # rows take (1/w1) d_n u1 - d_n u2
    s1 = self_difference_operators(c1, d, alpha, k1, k2, w1, 1.0)
    I = np.eye(N)
    A[R["g1v"], C["mu1"]] = 0.5 * (w1 + 1.0) * I + s1["D"]
    A[R["g1v"], C["sigma1"]] = s1["S"]
    A[R["g1n"], C["mu1"]] = s1["T"]
    A[R["g1n"], C["sigma1"]] = -I + s1["N"]
    P = near_potentials(c1.pos, c1.nrm, c2, d, alpha, k2)          # Gamma2 sources at k2
    put("g1v", "g1n", "mu2", "sigma2", {key: -v for key, v in P.items()})
    v, dn = jexp_columns(c1.pos, c1.nrm, x2, k2, Q2)
    A[R["g1v"], C["a2"]] = -v
    A[R["g1n"], C["a2"]] = -dn
    v, dn = jexp_columns(c1.pos, c1.nrm, x1, k1, Q1)
    A[R["g1v"], C["a1"]] = v
    A[R["g1n"], C["a1"]] = dn / w1

    # --- Gamma2 rows: u2 - u3 = 0, d_n u2 - d_n u3 = 0 ------------------------------------------
    s2 = self_difference_operators(c2, d, alpha, k2, k3, 1.0, w3)
    A[R["g2v"], C["mu2"]] = 0.5 * (1.0 + w3) * I + s2["D"]
    A[R["g2v"], C["sigma2"]] = s2["S"]
    A[R["g2n"], C["mu2"]] = s2["T"]
    A[R["g2n"], C["sigma2"]] = -I + s2["N"]
    P = near_potentials(c2.pos, c2.nrm, c1, d, alpha, k2)          # Gamma1 sources at k2
    put("g2v", "g2n", "mu1", "sigma1", P)
    v, dn = jexp_columns(c2.pos, c2.nrm, x2, k2, Q2)
    A[R["g2v"], C["a2"]] = v
    A[R["g2n"], C["a2"]] = dn
    v, dn = jexp_columns(c2.pos, c2.nrm, x3, k3, Q3)
    A[R["g2v"], C["a3"]] = -v
    A[R["g2n"], C["a3"]] = -dn / w3

    # --- wall rows: alpha u(L) - u(R), alpha d_x u(L) - d_x u(R) (Eq. bound2, cancelled form) ----
    ex = np.array([1.0, 0.0])

    def wall(rv, rn, ys, curves, kk, center, ca, Qc, wgt):
        L = np.stack([np.full_like(ys, -0.5 * d), ys], axis=1)
        Rt = np.stack([np.full_like(ys, 0.5 * d), ys], axis=1)
        tn = np.tile(ex, (ys.size, 1))
        for cv, cm, cs in curves:
            P = near_potentials(L, tn, cv, d, alpha, kk, shifts=(1, -2),
                                phases=(alpha ** 2, -alpha ** -1))
            put(rv, rn, cm, cs, P, wgt)
        vL, dL = jexp_columns(L, tn, center, kk, Qc)
        vR, dR = jexp_columns(Rt, tn, center, kk, Qc)
        A[R[rv], C[ca]] = alpha * vL - vR
        A[R[rn], C[ca]] = alpha * dL - dR

    wall("w2v", "w2n", wall2, [(c1, "mu1", "sigma1"), (c2, "mu2", "sigma2")], k2, x2, "a2", Q2, 1.0)
    wall("w1v", "w1n", wall1, [(c1, "mu1", "sigma1")], k1, x1, "a1", Q1, w1)
    wall("w3v", "w3n", wall3, [(c2, "mu2", "sigma2")], k3, x3, "a3", Q3, w3)

    # --- Gamma_u / Gamma_d rows (Eq. bound3) ------------------------------------------------------
    ey = np.array([0.0, 1.0])
    tn = np.tile(ey, (nb, 1))
    U = np.stack([bx, np.full_like(bx, y0)], axis=1)
    Dd = np.stack([bx, np.full_like(bx, -y0)], axis=1)
    P = near_potentials(U, tn, c1, d, alpha, k1)
    put("uv", "un", "mu1", "sigma1", P, w1)
    v, dn = jexp_columns(U, tn, x1, k1, Q1)
    A[R["uv"], C["a1"]] = v
    A[R["un"], C["a1"]] = dn
    E = np.exp(1j * np.outer(bx, kap))
    A[R["uv"], C["c"]] = -E
    A[R["un"], C["c"]] = -1j * E * k1n[None, :]
    P = near_potentials(Dd, tn, c2, d, alpha, k3)
    put("dv", "dn", "mu2", "sigma2", P, w3)
    v, dn = jexp_columns(Dd, tn, x3, k3, Q3)
    A[R["dv"], C["a3"]] = v
    A[R["dn"], C["a3"]] = dn
    A[R["dv"], C["d"]] = -E
    A[R["dn"], C["d"]] = 1j * E * k3n[None, :]

    # --- right-hand side (Eq. Arhs) ---------------------------------------------------------------
    f = np.zeros(nrow, dtype=np.complex128)
    kv = np.array([kap0, k1 * math.sin(theta)])
    uinc = np.exp(1j * (c1.pos @ kv))
    dninc = 1j * (c1.nrm @ kv) * uinc
    f[R["g1v"]] = -uinc
    f[R["g1n"]] = -dninc / w1
    eg.A = A
    eg.f = f
    return eg


# ----------------------------------------------------------------------------------------------
# Pseudo-inverse (Sec. 5, Eq. applypA)
# ----------------------------------------------------------------------------------------------

@dataclass
class PInv:
    U: np.ndarray
    s: np.ndarray
    Vh: np.ndarray
    colscale: np.ndarray
    eps: float

    @property
    def sinv(self):
        return 1.0 / np.maximum(self.s, self.eps)

    def apply(self, g):
        """A^+ g = D V Sigma^+ (U^* g); g may be a vector or a matrix of columns."""
        w = self.U.conj().T @ g
        w = (self.sinv[:, None] * w) if w.ndim == 2 else self.sinv * w
        x = self.Vh.conj().T @ w
        return (self.colscale[:, None] * x) if x.ndim == 2 else self.colscale * x


def jcolumn_scale(eg: EmptyGrating) -> np.ndarray:
    """Unit 2-norm scaling of the J-expansion columns (a2, a1, a3); 1 elsewhere."""
    D = np.ones(eg.A.shape[1])
    for blk in ("a2", "a1", "a3"):
        sl = eg.cols[blk]
        D[sl] = 1.0 / np.linalg.norm(eg.A[:, sl], axis=0)
    return D


def factor(eg: EmptyGrating, eps=None, lapack_driver: str = "gesdd") -> PInv:
    """SVD of the column-scaled A (Sec. 5): A D = U Sigma V^*."""
    eps = eg.g["eps_pinv"] if eps is None else eps
    D = jcolumn_scale(eg)
    As = eg.A * D[None, :]
    if lapack_driver == "gesdd":
        U, s, Vh = np.linalg.svd(As, full_matrices=False)
    else:
        import scipy.linalg
        U, s, Vh = scipy.linalg.svd(As, full_matrices=False, lapack_driver=lapack_driver)
    return PInv(U=U, s=s, Vh=Vh, colscale=D, eps=eps)


# ----------------------------------------------------------------------------------------------
# Bragg amplitudes and flux (Sec. 2 Eqs. rad1-rad2, Sec. 6 flux identity)
# ----------------------------------------------------------------------------------------------

def bragg(eg: EmptyGrating, avec: np.ndarray):
    """Propagating orders (k_{j,n} > 0 real after snapping) and their amplitudes c_n, d_n."""
    K = eg.g["K_rb"]
    n = np.arange(-K, K + 1)
    c = avec[eg.cols["c"]]
    dd = avec[eg.cols["d"]]
    pt = (eg.k1n.imag == 0) & (eg.k1n.real > 0)
    pb = (eg.k3n.imag == 0) & (eg.k3n.real > 0)
    return {"n_top": n[pt], "c": c[pt], "n_bot": n[pb], "d": dd[pb],
            "k1n": eg.k1n[pt].real, "k3n": eg.k3n[pb].real}


def flux_balance(eg: EmptyGrating, avec: np.ndarray):
    """(outgoing, incident) vertical energy fluxes: sum k_{1,n}|c_n|^2 / w1 + sum k_{3,n}|d_n|^2 / w3
    over the propagating orders and k1 |sin theta| / w1 (TE weights w_j; 1 for TM)."""
    b = bragg(eg, avec)
    w1, w3 = layer_weights(eg.g)
    out = np.sum(b["k1n"] * np.abs(b["c"]) ** 2) / w1 + np.sum(b["k3n"] * np.abs(b["d"]) ** 2) / w3
    return float(out), eg.k[0] * abs(math.sin(eg.theta)) / w1


def flux_error(eg: EmptyGrating, avec: np.ndarray) -> float:
    """|outgoing - incident| / incident of flux_balance (Sec. 6; zero for lossless media)."""
    out, inc = flux_balance(eg, avec)
    return float(abs(out - inc) / inc)
