"""The allocation-free translation entry point (gs_translate_noalloc), called through the C-ABI.

Callers that cannot allocate device memory where they need the operation -- a framework whose pool
owns the device heap, a loop that may not allocate after start-up, code without a gs_ctx -- use
this entry point; it keeps its scratch in a fixed array inside the library.  Checked here, for both
precisions: two calls in a row with different inputs against the oracle's dense translation and
against the context path (gs_translate), within the tolerances of the other parity tests (FP64
1e-12, complex64 1e-5, relative in norm); the complex64 layout near the array's size limit against
the oracle's direct sum on sampled rows; and the refusals (too large for the array, a geometry
whose Hankel values overflow FP32 in the complex64 form, malformed tensors).  The file is collected
last on purpose."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import inclusions as I

pytestmark = pytest.mark.gpu


def _dev(a, dtype):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype).contiguous()


@pytest.mark.parametrize("prec_name,tol", [("fp64", 1e-12), ("c64", 1e-5)])
def test_noalloc_translate_matches_oracle_and_context_path_twice(prec_name, tol):
    import torch
    from paper_1412_7466_gb300 import GS_C64, GS_FP64, GS_OK, GratingSolver, translate_noalloc

    prec = GS_FP64 if prec_name == "fp64" else GS_C64
    g = W.grating("tiny")
    theta = -0.9
    dk = W.disks(150, 0.01, 0.005, 2.0, g["k"][0], seed=5, p=8)
    gs = GratingSolver(0)
    gs.set_layers(g)
    gs.set_incidence([theta])
    gs.set_inclusions(dk)
    gs.factor()
    M, p = dk["xy"].shape[0], dk["p"]
    n = M * (2 * p + 1)
    xy = _dev(dk["xy"], torch.float64)
    alpha = np.exp(1j * g["k"][0] * math.cos(theta) * g["d"])
    T = I.translation_matrix(dk["xy"], g["k"][1], p, g["d"], alpha)
    rng = np.random.default_rng(3)
    w = np.tile(0.3 ** np.abs(np.arange(-p, p + 1)), M)
    for call in range(2):
        bh = (rng.standard_normal(n) + 1j * rng.standard_normal(n)) * w
        beta = _dev(bh, torch.complex128)
        ref = T @ bh
        ctx = gs.translate(beta, precision=prec).cpu().numpy()
        out = torch.full_like(beta, float("nan"))
        st = translate_noalloc(xy, beta, out, p, g["k"][1], g["d"], alpha, precision=prec)
        assert st == GS_OK
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.linalg.norm(got - ref) <= tol * np.linalg.norm(ref), (call, "oracle")
        assert np.linalg.norm(got - ctx) <= tol * np.linalg.norm(ref), (call, "context path")
    gs.close()


def test_noalloc_c64_near_the_size_limit():
    """M = 12945 at p = 12: the largest complex64 problem the fixed array holds (partials,
    converted coefficients, image coordinates and the range check's slot), sampled rows against
    the oracle's direct sum; M = 12946 is refused before any device work."""
    import torch
    from paper_1412_7466_gb300 import GS_C64, GS_ERR_ARG, GS_OK, translate_noalloc

    M, p, k2, d = 12945, 12, 300.0, 1.0
    dk = W.disks(M, 0.002, 0.001, 2.0, 40.0, seed=21, p=p)
    n = M * (2 * p + 1)
    rng = np.random.default_rng(8)
    w = np.tile(0.3 ** np.abs(np.arange(-p, p + 1)), M)
    bh = (rng.standard_normal(n) + 1j * rng.standard_normal(n)) * w
    alpha = np.exp(0.63j)
    xy = _dev(dk["xy"], torch.float64)
    beta = _dev(bh, torch.complex128)
    out = torch.full_like(beta, float("nan"))
    assert translate_noalloc(xy, beta, out, p, k2, d, alpha, precision=GS_C64) == GS_OK
    torch.cuda.synchronize()
    got = out.cpu().numpy().reshape(M, -1)
    rows = [0, M // 2, M - 1]
    ref = I.translation_apply_rows(dk["xy"], k2, p, d, alpha, bh, rows)
    for r, row in zip(rows, ref):
        assert np.linalg.norm(got[r] - row) <= 1e-5 * np.linalg.norm(row), r
    big = M + 1
    st = translate_noalloc(torch.zeros((big, 2), dtype=torch.float64, device="cuda"),
                           torch.zeros(big * 25, dtype=torch.complex128, device="cuda"),
                           torch.zeros(big * 25, dtype=torch.complex128, device="cuda"), p, k2, d, alpha,
                           precision=GS_C64)
    assert st == GS_ERR_ARG


def test_noalloc_refusals():
    """FP64 above the array's 2^19 values; complex64 on a geometry whose |H_2p(k2 R_min)| would
    overflow FP32 (p = 16, disks 0.05 apart at k2 = 8), while the FP64 form still runs; malformed
    tensors are refused by the binding before the library sees them."""
    import torch
    from paper_1412_7466_gb300 import GS_C64, GS_ERR_ARG, GS_FP64, GS_OK, translate_noalloc

    alpha = np.exp(0.3j)
    big = 524288 // 17 + 1
    st = translate_noalloc(torch.zeros((big, 2), dtype=torch.float64, device="cuda"),
                           torch.zeros(big * 17, dtype=torch.complex128, device="cuda"),
                           torch.zeros(big * 17, dtype=torch.complex128, device="cuda"), 8, 8.0, 1.0, alpha)
    assert st == GS_ERR_ARG
    g = W.grating("tiny")
    dk = W.disks(8, 0.02, 0.01, 2.0, g["k"][0], seed=5, p=16)
    xy = _dev(dk["xy"], torch.float64)
    beta = torch.ones(8 * 33, dtype=torch.complex128, device="cuda")
    out = torch.empty_like(beta)
    assert translate_noalloc(xy, beta, out, 16, g["k"][1], 1.0, alpha, precision=GS_C64) == GS_ERR_ARG
    assert translate_noalloc(xy, beta, out, 16, g["k"][1], 1.0, alpha, precision=GS_FP64) == GS_OK
    torch.cuda.synchronize()
    assert bool(torch.isfinite(out).all())
    with pytest.raises(ValueError):
        translate_noalloc(xy.float(), beta, out, 16, g["k"][1], 1.0, alpha)
    with pytest.raises(ValueError):
        translate_noalloc(xy, beta[:-1], out[:-1], 16, g["k"][1], 1.0, alpha)
    with pytest.raises(ValueError):
        translate_noalloc(xy, beta, beta, 16, g["k"][1], 1.0, alpha)
    with pytest.raises(ValueError):
        translate_noalloc(xy.cpu(), beta, out, 16, g["k"][1], 1.0, alpha)
