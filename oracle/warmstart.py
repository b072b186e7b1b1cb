"""Oracle for the learned warm start of the inclusion solve.

TEST INFRASTRUCTURE (see the package docstring): never used by the product path.

The paper has no learned component; the warm start is an addition to the method of Sec. 5
(the iterative solve of the preconditioned Schur system for the outgoing coefficients beta).  What
it computes, stated here in plain FP64 so that the kernels can be checked against it:

  * Features of inclusion i (64 values): its centre (x, y); sin and cos of 2 pi j x / d, j = 1..4
    (the quasi-periodic direction); the incidence angle theta and the top wavenumber k1; the real
    and imaginary parts of the empty grating's field at the centre, which is the n = 0 entry of the
    incoming coefficients w = B_phys A^+ f (Sec. 5: B_phys maps the layer unknowns to the
    J-expansion coefficients about each centre, and J_n(0) = delta_n0); zeros up to 64.
  * Network: standardise the features, (x - mu) / sd, then Linear 64->128, SiLU, Linear 128->128,
    SiLU, Linear 128->2(2p+1).  Output row = [Re of orders -p..p, Im of orders -p..p].
  * Coefficients: the network predicts the part of the incoming coefficients that the empty-grating
    field does not give, per order scaled by a fixed scale_n >= 0 (0: the order is not predicted):
    alpha_hat = w + scale (.) (Re + i Im),
    and beta_0 = s (.) alpha_hat (Sec. 4.1: beta = s (.) alpha for each disk).  The converged
    solution gives the training target t / scale, t = T beta - B_phys A^+ C beta (= beta / s - w).
  * Loss: mean of the squared output errors over all rows and the 2(2p+1) outputs; Adam.
  * The zero start is kept unless ||b - L beta_0|| < ||b||.

Storage precision of the kernels (bfloat16 weights and activations, FP32 accumulation) is
emulated on request (``bf16=True``) by rounding the same quantities to bfloat16 (round to nearest
even) at the same points, so that the kernels can be compared tightly; without it everything is
FP64.
"""
from __future__ import annotations

import math

import numpy as np

N_IN = 64
N_HID = 128


def n_out(p: int) -> int:
    return 2 * (2 * p + 1)


def weight_shapes(p: int):
    """Shapes of the trainable tensors in their flat order: W1, b1, W2, b2, W3, b3 (W[in][out])."""
    no = n_out(p)
    return [(N_IN, N_HID), (N_HID,), (N_HID, N_HID), (N_HID,), (N_HID, no), (no,)]


def n_weights(p: int) -> int:
    return int(sum(np.prod(s) for s in weight_shapes(p)))


def n_params(p: int) -> int:
    """Flat parameter vector: the weights, then mu (64), sd (64), scale (2p+1)."""
    return n_weights(p) + 2 * N_IN + (2 * p + 1)


def unpack(params: np.ndarray, p: int):
    out, o = [], 0
    for s in weight_shapes(p):
        n = int(np.prod(s))
        out.append(params[o:o + n].reshape(s))
        o += n
    mu = params[o:o + N_IN]
    sd = params[o + N_IN:o + 2 * N_IN]
    scale = params[o + 2 * N_IN:o + 2 * N_IN + 2 * p + 1]
    return out, mu, sd, scale


def bf16(x: np.ndarray) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def features(xy: np.ndarray, theta: float, k1: float, w0: np.ndarray, d: float = 1.0) -> np.ndarray:
    """(M, 64) features of each inclusion (see the module docstring)."""
    M = xy.shape[0]
    F = np.zeros((M, N_IN))
    x, y = xy[:, 0], xy[:, 1]
    F[:, 0] = x
    F[:, 1] = y
    for j in range(1, 5):
        F[:, 2 * j] = np.sin(2 * math.pi * j * x / d)
        F[:, 2 * j + 1] = np.cos(2 * math.pi * j * x / d)
    F[:, 10] = theta
    F[:, 11] = k1
    F[:, 12] = w0.real
    F[:, 13] = w0.imag
    return F


def standardisation(X0: np.ndarray, theta_range, k_range):
    """(mu, sd) of the 64 features: mean and population standard deviation over one geometry's
    inclusions, except theta (column 10) and k1 (column 11), which take the sweep's ranges read as
    uniform distributions (mean (lo + hi)/2, sd (hi - lo)/sqrt(12)); a constant column gets sd = 1."""
    X0 = np.asarray(X0, dtype=np.float64)
    mu, sd = X0.mean(0), X0.std(0)
    for col, (lo, hi) in ((10, theta_range), (11, k_range)):
        mu[col] = 0.5 * (lo + hi)
        sd[col] = (hi - lo) / math.sqrt(12.0)
    sd[~(sd > 1e-12)] = 1.0
    return mu, sd


def order_scale(ms_t: np.ndarray, ms_st: np.ndarray, share: float = 1e-4) -> np.ndarray:
    """Per-order output scale from (mean |t_n|^2, mean |s_n t_n|^2) of one solved point: rms(t_n)
    where the order's share of beta, rms(s_n t_n), exceeds `share` times the largest order's, else 0
    (the order is left to the empty grating's field)."""
    rt = np.sqrt(np.asarray(ms_t, dtype=np.float64))
    rst = np.sqrt(np.asarray(ms_st, dtype=np.float64))
    top = rst.max() if np.isfinite(rst.max()) else 0.0
    keep = (rst > share * top) & (rt > 0) & np.isfinite(rt)
    return np.where(keep, rt, 0.0)


def incoming_empty(prob) -> np.ndarray:
    """w = B_phys A^+ f: the empty grating's incoming coefficients about every centre, (M, 2p+1)."""
    return (prob.B @ prob.pinv.apply(prob.eg.f)).reshape(prob.M, prob.nc)


def silu(z):
    return z / (1.0 + np.exp(-z))


def dsilu(z):
    g = 1.0 / (1.0 + np.exp(-z))
    return g * (1.0 + z * (1.0 - g))


def forward(params: np.ndarray, X: np.ndarray, p: int, bf16_storage: bool = False):
    """Network output (rows, 2(2p+1)) and the intermediate values kept for the backward pass."""
    (W1, b1, W2, b2, W3, b3), mu, sd, _ = unpack(params, p)
    r = bf16 if bf16_storage else (lambda v: v)
    x0 = r((X - mu) / sd)
    W1, W2, W3 = r(W1), r(W2), r(W3)
    z1 = x0 @ W1 + b1
    a1 = r(silu(z1))
    z2 = a1 @ W2 + b2
    a2 = r(silu(z2))
    out = a2 @ W3 + b3
    return out, {"x0": x0, "z1": z1, "a1": a1, "z2": z2, "a2": a2, "W1": W1, "W2": W2, "W3": W3}


def loss_and_grad(params: np.ndarray, X: np.ndarray, Y: np.ndarray, p: int, bf16_storage: bool = False):
    """Mean squared error and its gradient with respect to the weights (flat, weight order)."""
    out, c = forward(params, X, p, bf16_storage)
    diff = out - Y
    loss = float(np.mean(diff ** 2))
    G3 = 2.0 * diff / diff.size
    gW3 = c["a2"].T @ G3
    gb3 = G3.sum(0)
    G2 = (G3 @ c["W3"].T) * dsilu(c["z2"])
    gW2 = c["a1"].T @ G2
    gb2 = G2.sum(0)
    G1 = (G2 @ c["W2"].T) * dsilu(c["z1"])
    gW1 = c["x0"].T @ G1
    gb1 = G1.sum(0)
    return loss, np.concatenate([g.ravel() for g in (gW1, gb1, gW2, gb2, gW3, gb3)])


def adam_step(params: np.ndarray, grad: np.ndarray, m: np.ndarray, v: np.ndarray, t: int, p: int,
              lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
    """One Adam update (Kingma & Ba 2015) of the weight part of params; returns the new (params, m, v)."""
    nw = n_weights(p)
    m = beta1 * m + (1 - beta1) * grad
    v = beta2 * v + (1 - beta2) * grad * grad
    mh = m / (1 - beta1 ** t)
    vh = v / (1 - beta2 ** t)
    new = params.copy()
    new[:nw] = params[:nw] - lr * mh / (np.sqrt(vh) + eps)
    return new, m, v


def scattered_incoming(prob, beta: np.ndarray) -> np.ndarray:
    """t = T beta - B_phys A^+ C beta, (M, 2p+1): the incoming field about each centre from the
    other inclusions and their images (Eq. trans) minus the layers' response to them (Sec. 5).
    At a converged beta, beta = s (.) (w + t); forming beta / s - w instead loses every digit where
    s is tiny (high orders)."""
    t = prob.translate(beta) - prob.B @ prob.pinv.apply(prob.C @ beta)
    return t.reshape(prob.M, prob.nc)


def targets(prob, beta: np.ndarray, scale: np.ndarray) -> np.ndarray:
    """Training targets (rows, 2(2p+1)) from a converged beta: t / scale split as [Re, Im]; an order
    with scale 0 is not predicted (target 0)."""
    scale = np.asarray(scale, dtype=np.float64)
    t = scattered_incoming(prob, beta)
    t = np.where(scale > 0, t / np.where(scale > 0, scale, 1.0), 0.0)
    return np.concatenate([t.real, t.imag], axis=1)


def moments(prob, beta: np.ndarray):
    """Per order: mean over the inclusions of |t_n|^2 and of |s_n t_n|^2 (chooses `scale`)."""
    t = scattered_incoming(prob, beta)
    return np.mean(np.abs(t) ** 2, axis=0), np.mean(np.abs(prob.s * t) ** 2, axis=0)


def guess(prob, params: np.ndarray, theta: float, k1: float):
    """beta_0 = s (.) (w + scale (.) network output), its relative residual, and the start kept
    (beta_0 if ||b - L beta_0|| < ||b||, else zero)."""
    p = prob.disks["p"]
    nc = 2 * p + 1
    w = incoming_empty(prob)
    X = features(prob.disks["xy"], theta, k1, w[:, p], prob.eg.d)
    out, _ = forward(params, X, p)
    _, _, _, scale = unpack(params, p)
    ah = w + scale * (out[:, :nc] + 1j * out[:, nc:])
    beta0 = (prob.s * ah).ravel()
    b = prob.rhs()
    rel = float(np.linalg.norm(b - prob.apply(beta0)) / np.linalg.norm(b))
    return beta0, rel, (beta0 if rel < 1.0 else np.zeros_like(beta0))
