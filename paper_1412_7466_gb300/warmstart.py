"""Learned warm start: the training driver over a design sweep.

Host orchestration only: features, targets, the normalisations, the network's forward and
backward passes, Adam and the start itself run in the library's kernels (gs_ws_*, gs_mlp_*,
gs_warm_start).  The two normalisations are fixed by gs_ws_normalise after the first solved sweep
point: the feature standardisation from that geometry's features and the sweep's ranges of theta
and k1, and the per-order output scale from that point's target moments (orders with a
negligible share of beta are not predicted).
"""
from __future__ import annotations

import math

import numpy as np

N_IN = 64


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
        # initial weights with a provisional unit normalisation, then the library fixes mu, sd and
        # the per-order scale from this solved point
        gs.mlp_set_params(self.p, pack(weights0, np.zeros(N_IN), np.ones(N_IN), np.ones(nc)))
        gs.ws_normalise(theta_range, k_range, share=1e-4, angle=angle)

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
