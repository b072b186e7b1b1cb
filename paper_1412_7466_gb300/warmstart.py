"""Learned warm start: the training driver over a design sweep.

Host orchestration only: features, targets, the network's forward and backward passes, Adam and
the start itself run in the library's kernels (gs_ws_*, gs_mlp_*, gs_warm_start).  The two
normalisations are fixed before training: the feature standardisation (mu, sd) from one
geometry's features and the sweep's ranges of theta and k1 (uniform: mean and width / sqrt(12)),
and the per-order output scale from the target moments of one solved sweep point (orders with a
negligible share of beta are not predicted, see ``order_scale``).
"""
from __future__ import annotations

import math

import numpy as np

N_IN = 64


def standardisation(X0: np.ndarray, theta_range, k_range):
    """(mu, sd) of the 64 features: sample moments over one geometry's inclusions, except theta
    (column 10) and k1 (column 11), which take the sweep's uniform ranges; constant columns get
    sd = 1."""
    X0 = np.asarray(X0, dtype=np.float64)
    mu, sd = X0.mean(0), X0.std(0)
    for col, (lo, hi) in ((10, theta_range), (11, k_range)):
        mu[col] = 0.5 * (lo + hi)
        sd[col] = (hi - lo) / math.sqrt(12.0)
    sd[~(sd > 1e-12)] = 1.0
    return mu, sd


def order_scale(ms_t: np.ndarray, ms_st: np.ndarray, share: float = 1e-4) -> np.ndarray:
    """Per-order output scale from the moments of one solved point (mean |t_n|^2, mean |s_n t_n|^2).

    The start's error is s (.) (t_hat - t): an order matters in proportion to its share of beta,
    rms(s_n t_n).  Orders whose share is below `share` times the largest are not predicted
    (scale 0: the empty grating's field alone), since any error the network makes there is
    multiplied by the translation's large high-order entries; the others take the root mean square
    target rms(t_n), so that their normalised targets have unit size."""
    rt = np.sqrt(np.asarray(ms_t, dtype=np.float64))
    rst = np.sqrt(np.asarray(ms_st, dtype=np.float64))
    top = rst.max() if np.isfinite(rst.max()) else 0.0
    keep = (rst > share * top) & (rt > 0) & np.isfinite(rt)
    return np.where(keep, rt, 0.0)


def pack(weights: np.ndarray, mu, sd, scale) -> np.ndarray:
    return np.concatenate([np.asarray(weights, np.float64), mu, sd, scale]).astype(np.float32)


class SweepTrainer:
    """Collects (features, targets) from solved sweep points and trains the network on them.

    Usage: after the first solved point call ``begin(weights0, theta_range, k_range)`` (fixes the
    normalisations from that point), then ``add()`` after every solved training point, then
    ``fit(epochs, lr)``; ``gs.warm_start()`` then gives the start for new points."""

    def __init__(self, gs, p: int):
        self.gs, self.p = gs, p
        self.nc = 2 * p + 1
        self.X, self.Y = [], []

    def begin(self, weights0: np.ndarray, theta_range, k_range, angle: int = 0):
        gs, nc = self.gs, self.nc
        # provisional network (unit normalisation) so that the feature and moment calls can run
        gs.mlp_set_params(self.p, pack(weights0, np.zeros(N_IN), np.ones(N_IN), np.ones(nc)))
        X0 = gs.ws_features(angle).cpu().numpy()
        self.mu, self.sd = standardisation(X0, theta_range, k_range)
        self.scale = order_scale(*gs.ws_moments(angle))
        gs.mlp_set_params(self.p, pack(weights0, self.mu, self.sd, self.scale))

    def add(self, angle: int = 0):
        self.X.append(self.gs.ws_features(angle))
        self.Y.append(self.gs.ws_targets(angle))

    def fit(self, epochs: int, lr: float, lr_final: float | None = None):
        """Full-batch Adam over everything collected; cosine decay from lr to lr_final.  Returns the
        loss history (before each step)."""
        torch = self.gs.torch
        X = torch.cat(self.X).contiguous()
        Y = torch.cat(self.Y).contiguous()
        lo = lr if lr_final is None else lr_final
        hist = []
        for e in range(epochs):
            r = lo + 0.5 * (lr - lo) * (1.0 + math.cos(math.pi * e / max(epochs - 1, 1)))
            hist.append(self.gs.mlp_train_step(X, Y, r))
        return hist
