"""TE polarisation and lossy inclusions through the C-ABI, against the oracle on the same seeded
inputs: the assembled TE matrix and right-hand side (1e-10 of each block's largest entry, as for
TM), the TE and lossy disk coefficients (1e-11), full solves in both precisions (Bragg amplitudes
1e-9 norm-wise and element-wise), the flux error (energy conservation for lossless TE; the absorbed
fraction for lossy disks, equal to the oracle's), and the all-layer field in TE."""
import math

import numpy as np
import pytest

import workloads as W
from bragg import check as check_bragg
from oracle import field as F
from oracle import layers as L
from oracle import solver as S

pytestmark = pytest.mark.gpu


def _np(t):
    return t.detach().cpu().numpy()


def _gpu(g, theta, dk):
    from paper_1412_7466_gb300 import GratingSolver
    gs = GratingSolver(0)
    gs.set_layers(g)
    gs.set_incidence([theta])
    gs.set_inclusions(dk)
    gs.factor()
    return gs


@pytest.fixture(scope="module")
def te_small():
    cfg = W.config("small")
    g = dict(cfg["grating"], pol="TE")
    prob = S.setup(g, cfg["theta"], cfg["disks"])
    gs = _gpu(g, cfg["theta"], cfg["disks"])
    yield cfg, g, prob, gs
    gs.close()


def test_te_assembly_matches_oracle(te_small):
    cfg, g, prob, gs = te_small
    A = _np(gs.get_A())
    Ao = prob.eg.A
    for rn, rs in prob.eg.rows.items():
        for cn, cs in prob.eg.cols.items():
            blk = Ao[rs, cs]
            scale = np.max(np.abs(blk))
            assert np.max(np.abs(A[rs, cs] - blk)) <= 1e-10 * max(scale, 1e-300), (rn, cn)
    np.testing.assert_allclose(_np(gs.get_f()), prob.eg.f, atol=1e-13)
    np.testing.assert_allclose(_np(gs.get_scattering()), prob.s, rtol=1e-11, atol=1e-300)


@pytest.mark.parametrize("prec_name", ["fp64", "c64"])
def test_te_solve_matches_oracle(te_small, prec_name):
    from paper_1412_7466_gb300 import GS_C64, GS_FP64
    cfg, g, prob, gs = te_small
    gs.solve(tol=1e-12, maxit=2000, precision=GS_FP64 if prec_name == "fp64" else GS_C64)
    got = gs.bragg()
    beta, _, _ = S.solve_dense(prob)
    _, ref, _ = prob.recover(beta)
    nw, ew = check_bragg(got, ref)
    assert got["flux_err"] < 1e-10
    print("TE", prec_name, "Bragg error vs oracle", nw, ew, "flux", got["flux_err"])


@pytest.mark.parametrize("pol", ["TM", "TE"])
def test_lossy_inclusions_match_oracle(pol):
    """Disks with kp = 20 + 1.5i (|kp R| = 0.8): coefficients, solve and absorbed fraction."""
    cfg = W.config("small")
    g = dict(cfg["grating"], pol=pol)
    dk = dict(cfg["disks"])
    dk["kp"] = dk["kp"] + 1.5j
    prob = S.setup(g, cfg["theta"], dk)
    beta, _, _ = S.solve_dense(prob)
    a, ref, fe = prob.recover(beta)
    gs = _gpu(g, cfg["theta"], dk)
    np.testing.assert_allclose(_np(gs.get_scattering()), prob.s, rtol=1e-11, atol=1e-300)
    gs.solve(tol=1e-12, maxit=2000)
    got = gs.bragg()
    gs.close()
    check_bragg(got, ref)
    out, inc = L.flux_balance(prob.eg, a)
    assert out < inc and fe > 1e-6                       # the disks absorb
    assert abs(got["flux_err"] - fe) <= 1e-8 * fe
    print(pol, "lossy: absorbed fraction", fe, got["flux_err"])


def test_te_field_all_layers_matches_oracle(te_small):
    cfg, g, prob, gs = te_small
    gs.solve(tol=1e-13, maxit=2000)
    beta, _, _ = S.solve_dense(prob)
    xs, ys = np.meshgrid(np.linspace(-0.5, 0.5, 21), np.linspace(-1.3, 1.3, 41))
    pts = np.stack([xs.ravel(), ys.ravel()], axis=1)
    h1 = L.iface_eval(g["gamma1"], g["d"], pts[:, 0])[0]
    h2 = L.iface_eval(g["gamma2"], g["d"], pts[:, 0])[0]
    xy, r = cfg["disks"]["xy"], cfg["disks"]["radius"]
    dmin = np.min([np.hypot(pts[:, 0, None] - (xy[None, :, 0] + l), pts[:, 1, None] - xy[None, :, 1]) / r[None, :]
                   for l in (-1, 0, 1)], axis=(0, 2))
    keep = (np.minimum(np.abs(pts[:, 1] - h1), np.abs(pts[:, 1] - h2)) > 0.05) & (dmin >= 1.5)
    pts = pts[keep]
    got = _np(gs.field(pts))
    ref = F.field(prob, beta, pts)
    ok = ~np.isnan(ref)
    assert np.array_equal(np.isnan(got), np.isnan(ref)) and ok.sum() > 500
    assert np.max(np.abs(got[ok] - ref[ok])) <= 1e-8 * np.max(np.abs(ref[ok]))


def test_polarisation_and_loss_refusals():
    from paper_1412_7466_gb300 import GS_ERR_ARG, GratingSolver
    gs = GratingSolver(0)
    assert gs.lib.gs_set_polarization(gs.ctx, 7) == GS_ERR_ARG
    g = W.grating("tiny")
    gs.set_layers(g)
    gs.set_incidence([-1.0])
    dk = W.disks(3, 0.02, 0.01, 2.0, g["k"][0], seed=2, p=4)
    gs.set_inclusions(dk)
    import ctypes
    bad = (ctypes.c_double * 3)(0.1, -0.1, 0.0)
    assert gs.lib.gs_set_inclusion_loss(gs.ctx, bad) == GS_ERR_ARG
    big = (ctypes.c_double * 3)(1e4, 0.0, 0.0)             # |kp R| > 12
    assert gs.lib.gs_set_inclusion_loss(gs.ctx, big) == GS_ERR_ARG
    gs.close()
