"""Oracle: the total field in the layer that holds the inclusions, at given points.

TEST INFRASTRUCTURE (see the package docstring): never used by the product path.

Follows Sec. 3 Eq. repre3 (the middle-layer field of the layer unknowns: single- and double-layer
potentials of both interfaces with the +-d near copies, and the J-expansion about the layer's
centre for the far copies) and Sec. 5 Eq. repre3_mod (the inclusions' outgoing fields with their
+-d near copies, read as sum_l alpha^l sum_j sum_n beta^j_n H_n(k2 r^l_j) e^{i n theta^l_j}).  The
layer unknowns are those of the converged solution, a = A^+ (f - C beta) (Sec. 5).  The
representation holds inside one period, -d/2 <= x <= d/2, between the interfaces; potentials are
plain trapezoid sums, accurate for points a few node spacings away from the interfaces.  The
incident field lives in the top layer only, so it does not appear here.  Points inside an
inclusion are returned as NaN.
"""
from __future__ import annotations

import numpy as np
from scipy.special import hankel1

from . import layers as L


def middle_field(prob, beta: np.ndarray, pts: np.ndarray) -> np.ndarray:
    eg = prob.eg
    pts = np.asarray(pts, dtype=np.float64)
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
