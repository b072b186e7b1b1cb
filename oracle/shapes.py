"""Oracle: scattering matrices of general (non-circular) inclusions.

TEST INFRASTRUCTURE (see the package docstring): never used by the product path.

Sec. 4.1: for an inclusion with a smooth closed boundary, the exterior scattered field and the
interior field are represented as u^s = S^{k2} sigma + D^{k2} mu and u = S^{kp} sigma + D^{kp} mu
(Eqs. rep1-rep2); the transmission conditions give the second-kind system of Eqs. intg1-intg2,
  mu + (S^{k2} - S^{kp}) sigma + (D^{k2} - D^{kp}) mu = -u_inc,
  -sigma + (N^{k2} - N^{kp}) sigma + (T^{k2} - T^{kp}) mu = -d_n u_inc,
with the normal pointing out of the inclusion.  For u_inc = J_n(k2 r) e^{i n theta} the outgoing
coefficients follow from Graf's theorem, H_0(k|x-y|) = sum_l H_l(k|x|) e^{i l th_x} J_l(k|y|)
e^{-i l th_y} for |y| < |x|:
  s_ln = (i/4) int [J_l(k2|y|) e^{-i l th_y} sigma_n(y) + n(y) . grad(J_l(k2|y|) e^{-i l th_y}) mu_n(y)] ds
(the factor i/4 of the kernel G = (i/4) H_0, which the printed formula leaves implicit).  Sec. 4.2:
a copy rotated about its centre has phase factors e^{+-i phi (l - n)} s_ln; with phi measured
counter-clockwise (x towards y) the factor is e^{i phi (n - l)}, the printed e^{i phi (l - n)} being
the same rotation with phi measured clockwise (the matrix of a rotated star computed from its own
boundary decides the sign).

TE polarisation (flux condition [(1/eps) d_n u] = 0, eps ~ k^2): the interior potentials are scaled
by wp = (kp/k2)^2 (as for the layers), so the first equation reads ((1 + wp)/2) mu + (S^{k2} - wp
S^{kp}) sigma + (D^{k2} - wp D^{kp}) mu = -u_inc and the second is unchanged.

Discretisation: the star r(t) = a1 + a2 cos(a3 t) (Eq. par1), t in [0, 2 pi), N equispaced nodes;
the Nystrom matrices use Kress's product rule for the log-singular part (the coefficient of log r,
obtained by replacing H_n by (2i/pi) J_n) and the trapezoid rule for the rest, with the diagonal
limits of the kernel differences (as for the interfaces; D keeps the Laplace double layer's
curvature term (wa - wb) gamma''.n / (4 pi |gamma'|^2) when the weights differ).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import hankel1, jv

from .layers import EULER, kernels, kress_weights


def star(a1: float, a2: float, a3: int, N: int, phi: float = 0.0):
    """Nodes of the star r(t) = a1 + a2 cos(a3 t) rotated by phi: positions, outward unit normals,
    speed |gamma'(t)|, and gamma''.n / |gamma'|^2 (the curvature term of the double layer)."""
    t = 2.0 * math.pi * np.arange(N) / N
    r = a1 + a2 * np.cos(a3 * t)
    rp = -a2 * a3 * np.sin(a3 * t)
    rpp = -a2 * a3 * a3 * np.cos(a3 * t)
    c, s = np.cos(t + phi), np.sin(t + phi)
    pos = np.stack([r * c, r * s], axis=1)
    d1 = np.stack([rp * c - r * s, rp * s + r * c], axis=1)
    d2 = np.stack([rpp * c - 2 * rp * s - r * c, rpp * s + 2 * rp * c - r * s], axis=1)
    speed = np.hypot(d1[:, 0], d1[:, 1])
    nrm = np.stack([d1[:, 1], -d1[:, 0]], axis=1) / speed[:, None]     # outward for counter-clockwise t
    kap = (d2[:, 0] * nrm[:, 0] + d2[:, 1] * nrm[:, 1]) / speed ** 2
    return {"t": t, "pos": pos, "nrm": nrm, "speed": speed, "kappa": kap, "N": N}


def _log_coeffs(tpos, tnrm, spos, snrm, k):
    """Coefficient of log r in the S, D, N, T kernels (H_n -> (2i/pi) J_n)."""
    Rx = tpos[:, None, 0] - spos[None, :, 0]
    Ry = tpos[:, None, 1] - spos[None, :, 1]
    r = np.hypot(Rx, Ry)
    np.fill_diagonal(r, 1.0)
    kr = k * r
    J0, J1 = jv(0, kr), jv(1, kr)
    Rnx = Rx * tnrm[:, None, 0] + Ry * tnrm[:, None, 1]
    Rny = Rx * snrm[None, :, 0] + Ry * snrm[None, :, 1]
    nn = tnrm[:, None, 0] * snrm[None, :, 0] + tnrm[:, None, 1] * snrm[None, :, 1]
    c = -1.0 / (2.0 * math.pi)
    return {"S": c * J0, "D": c * k * J1 * Rny / r, "N": -c * k * J1 * Rnx / r,
            "T": c * k * (k * J0 * Rnx * Rny / r ** 2 - 2.0 * J1 * Rnx * Rny / r ** 3 + J1 * nn / r)}


def closed_difference_operators(cv, ka, kb, wa=1.0, wb=1.0):
    """Nystrom matrices of wa S^{ka} - wb S^{kb}, wa D^{ka} - wb D^{kb}, N^{ka} - N^{kb},
    T^{ka} - T^{kb} on the closed curve cv (Kress product rule on the log part)."""
    N = cv["N"]
    pos, nrm, sp = cv["pos"], cv["nrm"], cv["speed"]
    h = 2.0 * math.pi / N
    with np.errstate(divide="ignore", invalid="ignore"):
        Ka = kernels(pos, nrm, pos, nrm, ka)
        Kb = kernels(pos, nrm, pos, nrm, kb)
    La = _log_coeffs(pos, nrm, pos, nrm, ka)
    Lb = _log_coeffs(pos, nrm, pos, nrm, kb)
    R = kress_weights(N)
    idx = (np.arange(N)[:, None] - np.arange(N)[None, :]) % N
    W = R[idx]
    with np.errstate(divide="ignore"):
        logt = np.log(4.0 * np.sin(math.pi * idx / N) ** 2)
    np.fill_diagonal(logt, 0.0)
    la, lb = np.log(complex(ka) / 2.0), np.log(complex(kb) / 2.0)
    dk2 = complex(ka) ** 2 - complex(kb) ** 2
    out = {}
    for key in "SDNT":
        u, v = (wa, wb) if key in "SD" else (1.0, 1.0)
        K = (u * Ka[key] - v * Kb[key]) * sp[None, :]
        K1 = (0.5 * (u * La[key] - v * Lb[key]) * sp[None, :]).astype(complex)   # coefficient of log(4 sin^2)
        # diagonal limits per unit length: K = K1' log r + Krest
        if key == "S":
            k1d = -(u - v) / (2.0 * math.pi)
            rest = u * (0.25j - (la + EULER) / (2.0 * math.pi)) - v * (0.25j - (lb + EULER) / (2.0 * math.pi))
        elif key == "D":
            k1d, rest = 0.0, (u - v) * cv["kappa"] / (4.0 * math.pi)
        elif key == "N":
            k1d, rest = 0.0, 0.0
        else:
            k1d = -dk2 / (4.0 * math.pi)
            rest = (1j * dk2 / 8.0 - (complex(ka) ** 2 * la - complex(kb) ** 2 * lb) / (4.0 * math.pi)
                    + dk2 * (1.0 - 2.0 * EULER) / (8.0 * math.pi))
        np.fill_diagonal(K1, 0.5 * k1d * sp)
        A = W * K1 + h * (K - K1 * logt)
        # log r = (1/2) log(4 sin^2((t-s)/2)) + log|gamma'| at coincidence
        np.fill_diagonal(A, W[0, 0] * 0.5 * k1d * sp + h * sp * (k1d * np.log(sp) + rest))
        out[key] = A
    return out


def scattering_matrix(a1, a2, a3, N, p, k2, kp, pol="TM", phi=0.0, return_densities=False):
    """The (2p+1) x (2p+1) matrix s_ln (l, n = -p..p) of the star rotated by phi (Sec. 4.1)."""
    cv = star(a1, a2, a3, N, phi)
    wp = 1.0 if pol == "TM" else (kp / k2) ** 2
    ops = closed_difference_operators(cv, k2, kp, 1.0, wp)
    I = np.eye(N)
    A = np.block([[0.5 * (1.0 + wp) * I + ops["D"], ops["S"]],
                  [ops["T"], -I + ops["N"]]])
    pos, nrm, sp = cv["pos"], cv["nrm"], cv["speed"]
    rho = np.hypot(pos[:, 0], pos[:, 1])
    th = np.arctan2(pos[:, 1], pos[:, 0])
    n = np.arange(-p - 1, p + 2)
    f = jv(n[None, :], k2 * rho[:, None]) * np.exp(1j * n[None, :] * th[:, None])     # J_n e^{in th}
    fx = 0.5 * k2 * (f[:, :-2] - f[:, 2:])
    fy = 0.5j * k2 * (f[:, :-2] + f[:, 2:])
    val = f[:, 1:-1]
    dn = nrm[:, 0:1] * fx + nrm[:, 1:2] * fy
    sol = np.linalg.solve(A, -np.vstack([val, dn]))          # columns: incident orders n = -p..p
    mu, sigma = sol[:N], sol[N:]
    # moments with the conjugate waves J_l e^{-i l th}: value and normal derivative
    g = jv(n[None, :], k2 * rho[:, None]) * np.exp(-1j * n[None, :] * th[:, None])    # J_n e^{-in th}
    gx = 0.5 * k2 * (g[:, :-2] - g[:, 2:])
    gy = -0.5j * k2 * (g[:, :-2] + g[:, 2:])
    gv = g[:, 1:-1]
    gn = nrm[:, 0:1] * gx + nrm[:, 1:2] * gy
    w = (2.0 * math.pi / N) * sp
    S = 0.25j * ((gv * w[:, None]).T @ sigma + (gn * w[:, None]).T @ mu)
    return (S, cv, mu, sigma) if return_densities else S


def scattering_blocks(disks: dict, k2: float, pol: str = "TM") -> np.ndarray:
    """(M, 2p+1, 2p+1) blocks of the preconditioner S for inclusions of one star shape
    (disks["shape"] = {a1, a2, a3, N}) rotated by disks["phi"] about their centres (Sec. 4.2)."""
    sh, p = disks["shape"], disks["p"]
    S0 = scattering_matrix(sh["a1"], sh["a2"], sh["a3"], sh["N"], p, k2, disks["kp"][0], pol)
    return np.stack([rotate(S0, ph) for ph in disks["phi"]])


def rotate(S: np.ndarray, phi: float) -> np.ndarray:
    """The matrix of the inclusion rotated counter-clockwise by phi about its centre (Sec. 4.2):
    e^{i phi (n - l)} s_ln."""
    p = (S.shape[0] - 1) // 2
    l = np.arange(-p, p + 1)
    return np.exp(1j * phi * (l[None, :] - l[:, None])) * S


def exterior_field(S_col_n: np.ndarray, k2: float, pts: np.ndarray) -> np.ndarray:
    """sum_l s_ln H_l(k2 r) e^{i l th} at pts (the outgoing expansion of one incident order)."""
    p = (S_col_n.size - 1) // 2
    l = np.arange(-p, p + 1)
    r = np.hypot(pts[:, 0], pts[:, 1])
    th = np.arctan2(pts[:, 1], pts[:, 0])
    return (hankel1(l[None, :], k2 * r[:, None]) * np.exp(1j * l[None, :] * th[:, None])) @ S_col_n
