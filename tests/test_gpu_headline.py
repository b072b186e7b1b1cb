"""GPU parity at the headline size (M = 1000 disks, k = (40, 60, 80), p = 12), in the launch
configuration bench.py times: translation rows sampled one by one against the oracle's direct sum,
the full FP64 solve's Bragg amplitudes against the stored oracle values (tests/golden, written by
tests/golden/make_golden.py from the oracle only) to 1e-9, and flux conservation."""
import os

import numpy as np
import pytest

import workloads as W
from oracle import inclusions as I

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def headline():
    from paper_1412_7466_gb300 import GratingSolver
    cfg = W.config("headline")
    gs = GratingSolver(0)
    gs.set_layers(cfg["grating"])
    gs.set_incidence([cfg["theta"]])
    gs.set_inclusions(cfg["disks"])
    gs.factor()
    yield cfg, gs
    gs.close()


def test_translate_sampled_rows(headline):
    cfg, gs = headline
    dk = cfg["disks"]
    g = cfg["grating"]
    M, p = dk["xy"].shape[0], dk["p"]
    rng = np.random.default_rng(2)
    beta = (rng.standard_normal(M * (2 * p + 1)) + 1j * rng.standard_normal(M * (2 * p + 1)))
    got = gs.translate(beta).cpu().numpy().reshape(M, -1)
    alpha = np.exp(1j * g["k"][0] * np.cos(cfg["theta"]) * g["d"])
    rows = [0, 1, 2, 3, 499, 997, 998, 999]
    ref = I.translation_apply_rows(dk["xy"], g["k"][1], p, g["d"], alpha, beta, rows)
    assert np.linalg.norm(got[rows] - ref) <= 1e-12 * np.linalg.norm(ref)


def test_headline_solve_matches_golden(headline):
    cfg, gs = headline
    gs.solve(tol=cfg["tol"], maxit=2000, restart=200)
    its, rr = gs.stats()
    assert rr <= 10 * cfg["tol"]
    br = gs.bragg()
    ref = {}
    for ln in open(os.path.join(HERE, "golden", "headline_bragg.txt")):
        if ln.startswith("#"):
            continue
        s, n, a, b = ln.split()
        ref[(s, int(n))] = complex(float(a), float(b))
    got = {("c", int(n)): v for n, v in zip(br["n_top"], br["c"])}
    got.update({("d", int(n)): v for n, v in zip(br["n_bot"], br["d"])})
    assert set(got) == set(ref)
    keys = sorted(ref)
    a = np.array([got[k] for k in keys])
    b = np.array([ref[k] for k in keys])
    assert np.linalg.norm(a - b) <= 1e-9 * np.linalg.norm(b)
    assert br["flux_err"] < 1e-10


def test_headline_mixed_solve_matches_golden(headline):
    from paper_1412_7466_gb300 import GS_C64
    cfg, gs = headline
    gs.solve(tol=cfg["tol"], maxit=4000, restart=200, precision=GS_C64)
    its, rr = gs.stats()
    assert rr <= cfg["tol"]
    br = gs.bragg()
    ref = {}
    for ln in open(os.path.join(HERE, "golden", "headline_bragg.txt")):
        if ln.startswith("#"):
            continue
        s, n, a, b = ln.split()
        ref[(s, int(n))] = complex(float(a), float(b))
    got = {("c", int(n)): v for n, v in zip(br["n_top"], br["c"])}
    got.update({("d", int(n)): v for n, v in zip(br["n_bot"], br["d"])})
    keys = sorted(ref)
    a = np.array([got[k] for k in keys])
    b = np.array([ref[k] for k in keys])
    assert np.linalg.norm(a - b) <= 1e-9 * np.linalg.norm(b)
