"""Oracle: the total field at given points of one period, in all three layers.

TEST INFRASTRUCTURE (see the package docstring): never used by the product path.

The layer unknowns are those of the converged solution, a = A^+ (f - C beta) (Sec. 5).
  * Middle layer (Sec. 3 Eq. repre3, Sec. 5 Eq. repre3_mod): single- and double-layer potentials of
    both interfaces at k2 with the +-d near copies, the J-expansion about the layer's centre x2 for
    the far copies, and the inclusions' outgoing fields with their +-d near copies, read as
    sum_l alpha^l sum_j sum_n beta^j_n H_n(k2 r^l_j) e^{i n theta^l_j}.
  * Top layer (Eq. repre1): the incident plane wave plus the potentials of Gamma1's densities at k1
    (near copies; times w1 = (k1/k2)^2 in TE polarisation) and the J-expansion a1 about x1; above Gamma_u (y >= y0) the Rayleigh-Bloch
    expansion (Eq. rad1) u_inc + sum_n c_n e^{i (kappa_n x + k_{1,n} (y - y0))}, all 2K+1 orders.
  * Bottom layer (Eq. repre2): the potentials of Gamma2's densities at k3 (times w3 = (k3/k2)^2 in
    TE) and the J-expansion a3 about x3; below Gamma_d (y <= -y0) sum_n d_n e^{i (kappa_n x - k_{3,n} (y + y0))} (Eq. rad2).
The signs follow from the interface rows of A (u1 - u2 = -u_inc on Gamma1, u2 - u3 = 0 on Gamma2,
with the jump relations of the double layer).  The representation holds inside one period,
-d/2 <= x <= d/2; potentials are plain trapezoid sums, accurate for points a few node spacings away
from the interfaces.  Points outside the period or inside an inclusion are returned as NaN.
"""
from __future__ import annotations

import numpy as np
from scipy.special import hankel1

from . import layers as L


def middle_field(prob, beta: np.ndarray, pts: np.ndarray, a=None) -> np.ndarray:
    eg = prob.eg
    pts = np.asarray(pts, dtype=np.float64)
    if a is None:
        a, _, _ = prob.recover(beta)
    nrm = np.tile([0.0, 1.0], (pts.shape[0], 1))      # the S and D kernels ignore the target normal
    u = np.zeros(pts.shape[0], dtype=np.complex128)
    for cv, cm, cs in ((eg.c1, "mu1", "sigma1"), (eg.c2, "mu2", "sigma2")):
        P = L.near_potentials(pts, nrm, cv, eg.d, eg.alpha, eg.k[1])
        u += P["S"] @ a[eg.cols[cs]] + P["D"] @ a[eg.cols[cm]]
    v, _ = L.jexp_columns(pts, nrm, eg.centers[1], eg.k[1], eg.g["Q"][1])
    u += v @ a[eg.cols["a2"]]
    xy = prob.disks["xy"]
    p = prob.disks["p"]
    n = np.arange(-p, p + 1)
    B = beta.reshape(prob.M, 2 * p + 1)
    inside = np.zeros(pts.shape[0], dtype=bool)
    for l in (-1, 0, 1):
        dx = pts[:, None, 0] - (xy[None, :, 0] + l * eg.d)
        dy = pts[:, None, 1] - xy[None, :, 1]
        r = np.hypot(dx, dy)
        inside |= np.any(r < prob.disks["radius"][None, :], axis=1)
        th = np.arctan2(dy, dx)
        H = hankel1(n[None, None, :], eg.k[1] * r[:, :, None]) * np.exp(1j * n[None, None, :] * th[:, :, None])
        u += eg.alpha ** l * np.einsum("tjn,jn->t", H, B)
    u[inside] = np.nan
    return u


def _layer_field(eg, a, pts, curve, cm, cs, k, center, col_a, Q, wgt):
    """Potentials of one interface's densities (near copies, scaled by the layer's TE weight) plus a
    J-expansion, at wavenumber k."""
    nrm = np.tile([0.0, 1.0], (pts.shape[0], 1))
    P = L.near_potentials(pts, nrm, curve, eg.d, eg.alpha, k)
    u = wgt * (P["S"] @ a[eg.cols[cs]] + P["D"] @ a[eg.cols[cm]])
    v, _ = L.jexp_columns(pts, nrm, center, k, Q)
    return u + v @ a[eg.cols[col_a]]


def field(prob, beta: np.ndarray, pts: np.ndarray) -> np.ndarray:
    """Total field at pts (npts, 2) in whichever layer each point lies."""
    eg = prob.eg
    g = eg.g
    pts = np.asarray(pts, dtype=np.float64)
    a, _, _ = prob.recover(beta)
    x, y = pts[:, 0], pts[:, 1]
    h1 = L.iface_eval(g["gamma1"], eg.d, x)[0]
    h2 = L.iface_eval(g["gamma2"], eg.d, x)[0]
    y0 = g["y0"]
    u = np.full(pts.shape[0], np.nan + 0j)
    inper = np.abs(x) <= 0.5 * eg.d
    kv = np.array([eg.kappa[g["K_rb"]], eg.k[0] * np.sin(eg.theta)])
    uinc = np.exp(1j * (pts @ kv))
    top_rb = inper & (y >= y0)
    top = inper & (y > h1) & (y < y0)
    mid = inper & (y < h1) & (y > h2)
    bot = inper & (y < h2) & (y > -y0)
    bot_rb = inper & (y <= -y0)
    c = a[eg.cols["c"]]
    d = a[eg.cols["d"]]
    if top_rb.any():
        E = np.exp(1j * (np.outer(x[top_rb], eg.kappa) + np.outer(y[top_rb] - y0, eg.k1n)))
        u[top_rb] = uinc[top_rb] + E @ c
    if bot_rb.any():
        E = np.exp(1j * (np.outer(x[bot_rb], eg.kappa) - np.outer(y[bot_rb] + y0, eg.k3n)))
        u[bot_rb] = E @ d
    w1, w3 = L.layer_weights(g)
    if top.any():
        u[top] = uinc[top] + _layer_field(eg, a, pts[top], eg.c1, "mu1", "sigma1", eg.k[0], eg.centers[0], "a1",
                                          g["Q"][0], w1)
    if bot.any():
        u[bot] = _layer_field(eg, a, pts[bot], eg.c2, "mu2", "sigma2", eg.k[2], eg.centers[2], "a3", g["Q"][2],
                              w3)
    if mid.any():
        u[mid] = middle_field(prob, beta, pts[mid], a=a)
    return u
