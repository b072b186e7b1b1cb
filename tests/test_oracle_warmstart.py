"""Pins of the warm-start oracle (CPU): the network gradient against central finite differences,
the bfloat16 rounding helper against hand-worked cases and torch's conversion, Adam's first step
against its closed form, the features' field value against the directly evaluated empty-grating
field, the training targets against the solution they must rebuild, and the start with an exact one-inclusion network and a planted bad one."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import layers as L
from oracle import solver as S
from oracle import warmstart as WS


def _params(p, seed=3, scale=None):
    rng = np.random.default_rng(seed)
    w = W.mlp_init(p, seed).astype(np.float64)
    w += 0.05 * rng.standard_normal(w.size)          # non-zero biases too
    mu = 0.1 * rng.standard_normal(64)
    sd = 0.5 + rng.random(64)
    sc = np.ones(2 * p + 1) if scale is None else scale
    return np.concatenate([w, mu, sd, sc])


def test_gradient_matches_finite_differences():
    p = 2
    rng = np.random.default_rng(0)
    prm = _params(p)
    X = rng.standard_normal((7, 64))
    Y = rng.standard_normal((7, WS.n_out(p)))
    loss, g = WS.loss_and_grad(prm, X, Y, p)
    nw = WS.n_weights(p)
    assert g.shape == (nw,)
    idx = np.concatenate([rng.choice(nw, 60, replace=False),
                          [WS.n_weights(p) - 1, 64 * 128, 64 * 128 + 128 + 5]])   # a b3, b1, W2 entry
    h = 1e-6
    for e in idx:
        a, b = prm.copy(), prm.copy()
        a[e] += h
        b[e] -= h
        fd = (WS.loss_and_grad(a, X, Y, p)[0] - WS.loss_and_grad(b, X, Y, p)[0]) / (2 * h)
        assert abs(fd - g[e]) <= 1e-7 * max(1.0, abs(g[e])) + 1e-9, (e, fd, g[e])


def test_bf16_rounding():
    v = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -9, -2.5, 3.0e38, 1e-40])
    r = WS.bf16(v)
    assert r[0] == 1.0
    assert r[1] == 1.0                       # halfway: ties to even
    assert r[2] == 1.0 + 2.0 ** -7           # above halfway
    assert r[3] == -2.5                      # exact
    torch = pytest.importorskip("torch")
    x = np.random.default_rng(1).standard_normal(1000).astype(np.float32) * 37.0
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(WS.bf16(x), ref)


def test_adam_first_step_closed_form():
    p = 1
    prm = _params(p)
    nw = WS.n_weights(p)
    g = np.random.default_rng(2).standard_normal(nw)
    new, m, v = WS.adam_step(prm, g, np.zeros(nw), np.zeros(nw), 1, p, lr=1e-3)
    # t = 1: m_hat = g, v_hat = g^2, update = -lr g / (|g| + eps)
    np.testing.assert_allclose(new[:nw] - prm[:nw], -1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=1e-18)
    np.testing.assert_array_equal(new[nw:], prm[nw:])      # mu, sd, scale are not trained


@pytest.fixture(scope="module")
def small():
    cfg = W.config("small")
    prob = S.setup(cfg["grating"], cfg["theta"], cfg["disks"])
    beta, _, _ = S.solve_dense(prob)
    return cfg, prob, beta


def test_features_and_field_at_centre(small):
    """Feature 12/13 is the empty grating's field at the centre, evaluated here directly from the
    layer densities and the middle J-expansion (Eq. repre3) at the centre point."""
    cfg, prob, _ = small
    eg = prob.eg
    w = WS.incoming_empty(prob)
    X = WS.features(prob.disks["xy"], cfg["theta"], eg.k[0], w[:, prob.disks["p"]], eg.d)
    a = prob.pinv.apply(eg.f)
    pts = prob.disks["xy"]
    nrm = np.tile([0.0, 1.0], (pts.shape[0], 1))
    u = np.zeros(pts.shape[0], dtype=complex)
    for cv, cm, cs in ((eg.c1, "mu1", "sigma1"), (eg.c2, "mu2", "sigma2")):
        P = L.near_potentials(pts, nrm, cv, eg.d, eg.alpha, eg.k[1])
        u += P["S"] @ a[eg.cols[cs]] + P["D"] @ a[eg.cols[cm]]
    v, _ = L.jexp_columns(pts, nrm, eg.centers[1], eg.k[1], eg.g["Q"][1])
    u += v @ a[eg.cols["a2"]]
    np.testing.assert_allclose(X[:, 12] + 1j * X[:, 13], u, rtol=1e-9, atol=1e-12)
    x = pts[:, 0]
    np.testing.assert_allclose(X[:, 8], np.sin(8 * math.pi * x), atol=1e-15)      # sin(2 pi 3 x)... j = 4
    np.testing.assert_allclose(X[:, 9], np.cos(8 * math.pi * x), atol=1e-15)
    np.testing.assert_allclose(X[:, 2], np.sin(2 * math.pi * x), atol=1e-15)
    assert np.all(X[:, 14:] == 0) and np.all(X[:, 10] == cfg["theta"]) and np.all(X[:, 11] == eg.k[0])


def test_targets_rebuild_the_solution(small):
    """At a converged beta the targets (T beta - B_phys A^+ C beta) give back beta = s (.) (w + t),
    i.e. L beta = b rewritten; scale only divides."""
    cfg, prob, beta = small
    p = prob.disks["p"]
    nc = 2 * p + 1
    scale = 0.5 + np.arange(nc) * 0.1
    Y = WS.targets(prob, beta, scale)
    t = (Y[:, :nc] + 1j * Y[:, nc:]) * scale
    rebuilt = (prob.s * (WS.incoming_empty(prob) + t)).ravel()
    assert np.linalg.norm(rebuilt - beta) <= 1e-12 * np.linalg.norm(beta)
    mt, mst = WS.moments(prob, beta)
    np.testing.assert_allclose(mt, np.mean(np.abs(t) ** 2, axis=0), rtol=1e-12)
    # s t is beta - s (.) w = beta - b (which cancels where beta is tiny: absolute floor)
    np.testing.assert_allclose(mst, np.mean(np.abs((beta - prob.rhs()).reshape(prob.M, nc)) ** 2, axis=0),
                               rtol=1e-9, atol=1e-12 * mst.max())


def test_guess_exact_network_and_fallback():
    """One inclusion: a network whose last layer outputs the exact (scaled) target reproduces the
    solution; a planted network with huge outputs is rejected (zero start)."""
    g = W.grating("small")
    th = -math.pi / 5
    dk = W.disks(1, 0.05, 0.02, 2.0, g["k"][0], seed=5, p=4)
    prob = S.setup(g, th, dk)
    beta, _, _ = S.solve_dense(prob)
    p = 4
    scale = np.full(2 * p + 1, 0.7)
    Y = WS.targets(prob, beta, scale)
    prm = _params(p, scale=scale)
    (W1, b1, W2, b2, W3, b3), _, _, _ = WS.unpack(prm, p)
    W3[:] = 0.0
    b3[:] = Y[0]
    b0, rel, kept = WS.guess(prob, prm, th, g["k"][0])
    assert np.linalg.norm(b0 - beta) <= 1e-10 * np.linalg.norm(beta)
    assert rel < 1e-10 and np.array_equal(kept, b0)
    b3[:] = 1e12
    b0, rel, kept = WS.guess(prob, prm, th, g["k"][0])
    assert rel > 1.0 and np.all(kept == 0)
