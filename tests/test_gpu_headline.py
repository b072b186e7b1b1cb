"""GPU parity at the headline size (M = 1000 disks, k = (40, 60, 80), p = 12), in the launch
configuration bench.py times: translation rows sampled one by one against the oracle's direct sum,
the full FP64 and mixed solves' Bragg amplitudes against the stored oracle values (tests/golden,
written by tests/golden/make_golden.py from the oracle only) to 1e-9, norm-wise and element-wise,
and flux conservation."""

import numpy as np
import pytest

import workloads as W
from oracle import inclusions as I
from bragg import check as check_bragg, load_golden

pytestmark = pytest.mark.gpu


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
    nw, ew = check_bragg(br, load_golden("headline"))
    print("headline FP64: Bragg error norm-wise", nw, "element-wise", ew)
    assert br["flux_err"] < 1e-10


def test_headline_mixed_solve_matches_golden(headline):
    from paper_1412_7466_gb300 import GS_C64
    cfg, gs = headline
    gs.solve(tol=cfg["tol"], maxit=4000, restart=200, precision=GS_C64)
    its, rr = gs.stats()
    assert rr <= cfg["tol"]
    nw, ew = check_bragg(gs.bragg(), load_golden("headline"))
    print("headline mixed: Bragg error norm-wise", nw, "element-wise", ew)
