"""Oracle for the full solve: the preconditioned Schur-complement system over the inclusions'
outgoing coefficients, and the Bragg amplitudes recovered from it.

TEST INFRASTRUCTURE (see the package docstring): never used by the product path.

Sec. 5: with alpha = A^+ (f - C beta) (applypA) substituted into Eq. finalsys, and the left
preconditioner S (Sec. 4.2), the system is (I - S T + S B_phys A^+ C) beta = S B_phys A^+ f
(the paper writes B = -B_phys).  For small M it is formed densely and solved by LU
(numpy.linalg.solve); for large M it is solved matrix-free by restarted GMRES (Sec. 5 "We can use
GMRES on this system"), with the translation applied by direct summation.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass

import numpy as np

from . import inclusions as inc
from . import layers as lay


@dataclass
class Problem:
    eg: lay.EmptyGrating
    pinv: lay.PInv
    disks: dict
    s: np.ndarray        # (M, nc) disk scattering diagonal, or (M, nc, nc) blocks of general shapes
    B: np.ndarray        # B_phys, (M nc, ncols of A)
    C: np.ndarray        # (nrows of A, M nc)
    timings: dict

    @property
    def M(self):
        return self.disks["xy"].shape[0]

    @property
    def nc(self):
        return 2 * self.disks["p"] + 1

    def apply_s(self, v):
        """S v: the diagonal (disks) or the per-inclusion blocks (general shapes, Sec. 4.2), for a
        vector or for the columns of a matrix."""
        V = v.reshape(self.M, self.nc, -1)
        out = self.s[:, :, None] * V if self.s.ndim == 2 else np.einsum("imn,inr->imr", self.s, V)
        return out.reshape(v.shape)

    def lowrank(self, beta):
        """S B_phys A^+ C beta (the Schur-complement correction, Sec. 5)."""
        return self.apply_s(self.B @ self.pinv.apply(self.C @ beta))

    def rhs(self):
        return self.apply_s(self.B @ self.pinv.apply(self.eg.f))

    def translate(self, beta):
        return translation_apply(self.disks, self.eg.k[1], self.eg.d, self.eg.alpha, beta)

    def apply(self, beta):
        """L beta = beta - S (T beta) + S B_phys A^+ C beta."""
        return beta - self.apply_s(self.translate(beta)) + self.lowrank(beta)

    def recover(self, beta):
        """alpha = A^+ (f - C beta) (Sec. 5) and the Bragg amplitudes / flux error (Sec. 6)."""
        a = self.pinv.apply(self.eg.f - self.C @ beta)
        return a, lay.bragg(self.eg, a), lay.flux_error(self.eg, a)


def setup(g: dict, theta: float, disks: dict, eps=None, lapack_driver="gesdd") -> Problem:
    t0 = time.perf_counter()
    eg = lay.build_empty_grating(g, theta)
    t1 = time.perf_counter()
    pinv = lay.factor(eg, eps=eps, lapack_driver=lapack_driver)
    t2 = time.perf_counter()
    if "shape" in disks:
        from . import shapes
        s = shapes.scattering_blocks(disks, eg.k[1], g.get("pol", "TM"))
    else:
        s = inc.scattering_diagonal(disks, eg.k[1], g.get("pol", "TM"))
    B = inc.coupling_B(eg, disks)
    C = inc.coupling_C(eg, disks)
    t3 = time.perf_counter()
    return Problem(eg=eg, pinv=pinv, disks=disks, s=s, B=B, C=C,
                   timings={"assemble": t1 - t0, "factor": t2 - t1, "couple": t3 - t2})


_M2L = None


def translation_apply(disks, k, d, alpha, beta):
    """T beta by direct summation over all pairs and the three images (Eq. trans)."""
    global _M2L
    M = disks["xy"].shape[0]
    p = disks["p"]
    if M <= 64:
        T = inc.translation_matrix(disks["xy"], k, p, d, alpha)
        return T @ beta
    if _M2L is None:
        from . import m2l as _m
        _M2L = _m
    return _M2L.apply(disks["xy"], k, p, d, alpha, beta)


def dense_operator(prob: Problem) -> np.ndarray:
    T = inc.translation_matrix(prob.disks["xy"], prob.eg.k[1], prob.disks["p"], prob.eg.d, prob.eg.alpha)
    BAC = prob.B @ prob.pinv.apply(prob.C)
    return np.eye(T.shape[0]) - prob.apply_s(T) + prob.apply_s(BAC)


def solve_dense(prob: Problem):
    L = dense_operator(prob)
    b = prob.rhs()
    beta = np.linalg.solve(L, b)
    return beta, L, b


def gmres(apply, b, tol=1e-12, restart=200, maxit=2000, x0=None):
    """Restarted GMRES (Saad-Schultz) with modified Gram-Schmidt applied twice and Givens
    rotations; stops when ||b - A x|| <= tol ||b||.  Returns (x, iterations, relres history)."""
    n = b.size
    x = np.zeros(n, dtype=np.complex128) if x0 is None else x0.astype(np.complex128).copy()
    bnorm = np.linalg.norm(b)
    if bnorm == 0:
        return x, 0, [0.0]
    hist = []
    it = 0
    while it < maxit:
        r = b - apply(x) if (x0 is not None or it > 0) else b.copy()
        beta = np.linalg.norm(r)
        hist.append(beta / bnorm)
        if beta <= tol * bnorm:
            break
        V = np.zeros((restart + 1, n), dtype=np.complex128)
        H = np.zeros((restart + 1, restart), dtype=np.complex128)
        cs = np.zeros(restart, dtype=np.complex128)
        sn = np.zeros(restart, dtype=np.complex128)
        g = np.zeros(restart + 1, dtype=np.complex128)
        g[0] = beta
        V[0] = r / beta
        j_end = 0
        for j in range(restart):
            w = apply(V[j])
            it += 1
            for _ in range(2):
                for i in range(j + 1):
                    h = np.vdot(V[i], w)
                    H[i, j] += h
                    w = w - h * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] != 0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -np.conj(sn[i]) * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            a, bb = H[j, j], H[j + 1, j]
            rr = math.hypot(abs(a), abs(bb))
            if rr == 0:
                cs[j], sn[j] = 1.0, 0.0
            elif a == 0:
                cs[j], sn[j] = 0.0, np.conj(bb) / abs(bb)
            else:
                cs[j] = abs(a) / rr
                sn[j] = (a / abs(a)) * np.conj(bb) / rr
            H[j, j] = cs[j] * a + sn[j] * bb
            H[j + 1, j] = 0.0
            g[j + 1] = -np.conj(sn[j]) * g[j]
            g[j] = cs[j] * g[j]
            j_end = j + 1
            hist.append(abs(g[j + 1]) / bnorm)
            if abs(g[j + 1]) <= tol * bnorm or it >= maxit:
                break
        y = np.linalg.solve(np.triu(H[:j_end, :j_end]), g[:j_end])
        x = x + V[:j_end].T @ y
        x0 = x
        if hist[-1] <= tol:
            r = b - apply(x)
            hist.append(np.linalg.norm(r) / bnorm)
            if hist[-1] <= 10 * tol:
                break
    return x, it, hist


def solve_gmres(prob: Problem, tol=1e-12, restart=200, maxit=2000, x0=None):
    b = prob.rhs()
    beta, its, hist = gmres(prob.apply, b, tol=tol, restart=restart, maxit=maxit, x0=x0)
    return beta, its, hist, b
