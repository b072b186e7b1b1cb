"""The allocation-free translation entry point (gs_translate_noalloc), called through the C-ABI.

Callers that cannot allocate device memory where they need the operation -- a framework whose pool
owns the device heap, a loop that may not allocate after start-up, code without a gs_ctx -- use
this entry point; it keeps its scratch in a fixed array inside the library.  The test checks it
against the context path (gs_translate) on two calls in a row with different inputs, within the
FP64 translation tolerance used by the other parity tests (1e-12 relative in norm), and that an
oversized problem is refused before any device work.  The file is collected last on purpose."""
import math

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def test_noalloc_translate_matches_context_path_twice():
    import torch
    from paper_1412_7466_gb300 import GS_ERR_ARG, GS_FP64, GS_OK, GratingSolver, translate_noalloc

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
    xy = torch.tensor(dk["xy"], dtype=torch.float64, device="cuda").contiguous()
    alpha = complex(math.cos(g["k"][0] * math.cos(theta) * g["d"]), math.sin(g["k"][0] * math.cos(theta) * g["d"]))
    gen = torch.Generator(device="cuda").manual_seed(3)
    for call in range(2):
        beta = torch.randn(n, dtype=torch.complex128, device="cuda", generator=gen)
        ref = gs.translate(beta, precision=GS_FP64)
        out = torch.full_like(beta, float("nan"))
        st = translate_noalloc(xy, beta, out, p, g["k"][1], g["d"], alpha, precision=GS_FP64)
        assert st == GS_OK
        torch.cuda.synchronize()
        err = (torch.linalg.norm(out - ref) / torch.linalg.norm(ref)).item()
        assert err <= 1e-12, (call, err)
    # M (2p+1) above the fixed capacity of 2^19 values is refused before any launch
    big = 524288 // 17 + 1
    st = translate_noalloc(torch.zeros((big, 2), dtype=torch.float64, device="cuda"),
                           torch.zeros(big * 17, dtype=torch.complex128, device="cuda"),
                           torch.zeros(big * 17, dtype=torch.complex128, device="cuda"), 8, g["k"][1], g["d"], alpha)
    assert st == GS_ERR_ARG
    gs.close()
