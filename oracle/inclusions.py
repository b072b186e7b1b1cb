"""Oracle for the inclusions: disk scattering coefficients, the translation operator, and the
coupling matrices between the inclusions and the layered grating.

TEST INFRASTRUCTURE (see the package docstring): never used by the product path.

Follows Sec. 4.1 (disk scattering matrix, diagonal, closed form), Sec. 4.2 (Eq. trans: M2L
translation; Eq. scattmatrix), Sec. 5 (Eq. repre3_mod: particle field with the +-d near copies;
Eqs. matB, matC; the L2L lemma; Remark "cancel").  Readings:

  * Eq. repre3_mod mixes the indices j and m; it is read as
    sum_l alpha^l sum_j sum_n beta^j_n H_n(k2 r^l_j) e^{i n theta^l_j}; a particle's own field is
    left out only for l = 0, its +-d images are included.
  * The paper's B equals minus the physical map B_phys from layer unknowns to incoming
    coefficients (Eq. finalsys with D = S^{-1} - T); this module builds B_phys.
  * The L2L lemma as printed is garbled; Graf's theorem for J is used:
    J_n(k|x-x0|) e^{in th_{x-x0}} = sum_m J_{n-m}(k|c-x0|) e^{i(n-m) th_{c-x0}} J_m(k|x-c|) e^{im th_{x-c}}.
  * M2L (Graf): H_n(k|x-c_j|) e^{in th_{x-c_j}} = sum_m H_{n-m}(k R) e^{i(n-m) Th} J_m(k|x-c_i|)
    e^{im th_{x-c_i}} with (R, Th) = polar(c_i - c_j), |x - c_i| < R.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import h1vp, hankel1, jv, jvp

from .layers import Curve, EmptyGrating


def mie_coefficients(p: int, R: float, k2: float, kp, pol: str = "TM") -> np.ndarray:
    """s_n, n = -p..p, of a disk of radius R (inside kp, outside k2): incoming J_n(k2 r)e^{in th}
    -> outgoing s_n H_n(k2 r) e^{in th}, from continuity of u and of w d_r u at r = R (Sec. 4.1),
    w = 1 for TM and w = 1/eps, proportional to 1/k^2, for TE (Sec. 2).  kp may be complex
    (a lossy inclusion, Im kp > 0: complex permittivity, Sec. 7)."""
    n = np.arange(-p, p + 1)
    a, b = k2 * R, kp * R
    # weights of the radial derivative terms: k (TM) or k / k^2 = 1 / k (TE), from d_r J_n(k r) = k J_n'
    wp, w2 = (kp, k2) if pol == "TM" else (1.0 / kp, 1.0 / k2)
    num = wp * jvp(n, b) * jv(n, a) - w2 * jv(n, b) * jvp(n, a)
    den = w2 * jv(n, b) * h1vp(n, a) - wp * jvp(n, b) * hankel1(n, a)
    return num / den


def scattering_diagonal(disks: dict, k2: float, pol: str = "TM") -> np.ndarray:
    """(M, 2p+1) diagonal of the block-diagonal preconditioner S (Sec. 4.2, Remark on several
    particle types: one diagonal per disk).  disks["kp"] may be complex (lossy inclusions)."""
    p = disks["p"]
    M = disks["xy"].shape[0]
    out = np.empty((M, 2 * p + 1), dtype=np.complex128)
    cache = {}
    for i in range(M):
        key = (float(disks["radius"][i]), complex(disks["kp"][i]))
        if key not in cache:
            cache[key] = mie_coefficients(p, key[0], k2, key[1], pol)
        out[i] = cache[key]
    return out


def _image_shifts():
    return (-1, 0, 1)


def translation_matrix(xy: np.ndarray, k: float, p: int, d: float, alpha: complex) -> np.ndarray:
    """Dense T (Eqs. trans, scattmatrix, repre3_mod): block (i, j) maps beta^j to its
    contribution to the incoming coefficients of particle i, summed over the images l = -1,0,1 of
    particle j with phase alpha^l; the block (i, i, l = 0) is left out.
    Entry [(i, m), (j, n)] = sum_l alpha^l H_{n-m}(k R) e^{i (n-m) Th}, (R,Th) = polar(c_i - c_j - l d)."""
    M = xy.shape[0]
    nc = 2 * p + 1
    T = np.zeros((M, nc, M, nc), dtype=np.complex128)
    q = np.arange(-2 * p, 2 * p + 1)
    m = np.arange(-p, p + 1)
    qidx = (m[None, :] - m[:, None]) + 2 * p       # index of n - m, [m, n]
    for l in _image_shifts():
        dx = xy[:, None, 0] - (xy[None, :, 0] + l * d)
        dy = xy[:, None, 1] - xy[None, :, 1]
        R = np.hypot(dx, dy)
        Th = np.arctan2(dy, dx)
        if l == 0:
            R[np.arange(M), np.arange(M)] = 1.0
        Hq = hankel1(q[None, None, :], k * R[:, :, None]) * np.exp(1j * q[None, None, :] * Th[:, :, None])
        if l == 0:
            Hq[np.arange(M), np.arange(M), :] = 0.0
        # T[i, m, j, n] += alpha^l Hq[i, j, n - m]
        T += (alpha ** l) * np.transpose(Hq[:, :, qidx], (0, 2, 1, 3))
    return T.reshape(M * nc, M * nc)


def translation_apply_rows(xy, k, p, d, alpha, beta, rows):
    """(T beta) for the target particles listed in `rows`, by direct summation (one by one)."""
    M = xy.shape[0]
    nc = 2 * p + 1
    B = beta.reshape(M, nc)
    q = np.arange(-2 * p, 2 * p + 1)
    m = np.arange(-p, p + 1)
    qidx = (m[None, :] - m[:, None]) + 2 * p
    out = np.zeros((len(rows), nc), dtype=np.complex128)
    for t, i in enumerate(rows):
        for l in _image_shifts():
            dx = xy[i, 0] - (xy[:, 0] + l * d)
            dy = xy[i, 1] - xy[:, 1]
            R = np.hypot(dx, dy)
            Th = np.arctan2(dy, dx)
            mask = np.ones(M, dtype=bool)
            if l == 0:
                mask[i] = False
            Hq = hankel1(q[None, :], k * R[mask, None]) * np.exp(1j * q[None, :] * Th[mask, None])
            # out[m] += alpha^l sum_j sum_n Hq[j, n - m] B[j, n]
            out[t] += (alpha ** l) * np.einsum("jmn,jn->m", Hq[:, qidx], B[mask])
    return out


def _outgoing_fields(tpos, centers, k, p, nrm=None):
    """f_n = H_n(k|x-c|) e^{in th_{x-c}} for n = -p-1..p+1 at targets (T) and centres (M);
    returns values (T, M, 2p+1) and gradients (x, y components) when nrm is None, or the
    derivative along nrm (T,2)."""
    Rx = tpos[:, None, 0] - centers[None, :, 0]
    Ry = tpos[:, None, 1] - centers[None, :, 1]
    rho = np.hypot(Rx, Ry)
    th = np.arctan2(Ry, Rx)
    n = np.arange(-p - 1, p + 2)
    f = hankel1(n[None, None, :], k * rho[:, :, None]) * np.exp(1j * n[None, None, :] * th[:, :, None])
    val = f[:, :, 1:-1]
    fx = 0.5 * k * (f[:, :, :-2] - f[:, :, 2:])
    fy = 0.5j * k * (f[:, :, :-2] + f[:, :, 2:])
    return val, fx, fy


def coupling_C(eg: EmptyGrating, disks: dict) -> np.ndarray:
    """C (Eq. matC): particle multipoles (three copies, phases alpha^l) -> Gamma1 rows (with a minus
    sign, since u2 enters u1 - u2), Gamma2 rows (plus), and the middle-layer wall discrepancy in the
    cancelled form alpha^2 f_{+1}(L) - alpha^{-1} f_{-2}(L) (Remark "cancel")."""
    d = eg.d
    k2 = eg.k[1]
    alpha = eg.alpha
    xy = disks["xy"]
    p = disks["p"]
    M = xy.shape[0]
    nc = 2 * p + 1
    C = np.zeros((eg.A.shape[0], M * nc), dtype=np.complex128)
    R = eg.rows

    def add(rv, rn, tpos, tnrm, shifts, phases, sign):
        for l, ph in zip(shifts, phases):
            cen = xy + np.array([l * d, 0.0])
            val, fx, fy = _outgoing_fields(tpos, cen, k2, p)
            dn = tnrm[:, None, 0:1] * fx + tnrm[:, None, 1:2] * fy
            C[R[rv], :] += sign * ph * val.reshape(tpos.shape[0], M * nc)
            C[R[rn], :] += sign * ph * dn.reshape(tpos.shape[0], M * nc)

    sh = (-1, 0, 1)
    phs = [alpha ** l for l in sh]
    add("g1v", "g1n", eg.c1.pos, eg.c1.nrm, sh, phs, -1.0)
    add("g2v", "g2n", eg.c2.pos, eg.c2.nrm, sh, phs, +1.0)
    ys = eg.wall_y[1]
    L = np.stack([np.full_like(ys, -0.5 * d), ys], axis=1)
    tn = np.tile(np.array([1.0, 0.0]), (ys.size, 1))
    add("w2v", "w2n", L, tn, (1, -2), (alpha ** 2, -alpha ** -1), +1.0)
    return C


def coupling_B(eg: EmptyGrating, disks: dict) -> np.ndarray:
    """B_phys (Eq. matB, with the sign of the physical map): layer densities on Gamma1, Gamma2
    (k2, three copies, trapezoid weights) and the middle J-expansion a2 -> incoming coefficients
    alpha^i_m of every particle.

    single layer at y:  (i/4) H_m(k|y-c|) e^{-im phi_y} w;
    double layer at y:  (i/4) n_y . grad_y [H_m(k|y-c|) e^{-im phi_y}] w, using
        d_x g_m = (k/2)(g_{m-1} - g_{m+1}), d_y g_m = -(ik/2)(g_{m-1} + g_{m+1});
    a2 column n:        J_{n-m}(k|c-x2|) e^{i(n-m) th_{c-x2}}."""
    d = eg.d
    k = eg.k[1]
    alpha = eg.alpha
    xy = disks["xy"]
    p = disks["p"]
    M = xy.shape[0]
    nc = 2 * p + 1
    B = np.zeros((M * nc, eg.A.shape[1]), dtype=np.complex128)
    Cc = eg.cols
    mm = np.arange(-p - 1, p + 2)
    for cv, cm, cs in ((eg.c1, "mu1", "sigma1"), (eg.c2, "mu2", "sigma2")):
        Sblk = np.zeros((M, nc, cv.x.size), dtype=np.complex128)
        Dblk = np.zeros((M, nc, cv.x.size), dtype=np.complex128)
        for l in (-1, 0, 1):
            sp = cv.pos + np.array([l * d, 0.0])
            Rx = sp[None, :, 0] - xy[:, None, 0]
            Ry = sp[None, :, 1] - xy[:, None, 1]
            rho = np.hypot(Rx, Ry)
            phi = np.arctan2(Ry, Rx)
            g = hankel1(mm[None, None, :], k * rho[:, :, None]) * np.exp(-1j * mm[None, None, :] * phi[:, :, None])
            gv = g[:, :, 1:-1]
            gx = 0.5 * k * (g[:, :, :-2] - g[:, :, 2:])
            gy = -0.5j * k * (g[:, :, :-2] + g[:, :, 2:])
            gn = cv.nrm[None, :, 0, None] * gx + cv.nrm[None, :, 1, None] * gy
            ph = (alpha ** l) * 0.25j * cv.w[None, :, None]
            Sblk += np.transpose(ph * gv, (0, 2, 1))
            Dblk += np.transpose(ph * gn, (0, 2, 1))
        B[:, Cc[cs]] = Sblk.reshape(M * nc, -1)
        B[:, Cc[cm]] = Dblk.reshape(M * nc, -1)
    x2 = eg.centers[1]
    Q2 = eg.g["Q"][1]
    n = np.arange(-Q2, Q2 + 1)
    m = np.arange(-p, p + 1)
    Rc = np.hypot(xy[:, 0] - x2[0], xy[:, 1] - x2[1])
    Tc = np.arctan2(xy[:, 1] - x2[1], xy[:, 0] - x2[0])
    q = n[None, None, :] - m[None, :, None]      # (1, nc, nQ)
    Jb = jv(q, k * Rc[:, None, None]) * np.exp(1j * q * Tc[:, None, None])
    B[:, Cc["a2"]] = Jb.reshape(M * nc, -1)
    return B
