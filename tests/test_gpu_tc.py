"""Tensor-core (tcgen05) product C = A B^T, bfloat16 in, FP32 accumulate, against the same product
of the same bfloat16 values in FP64 on the host.  Each product of two bfloat16 numbers is exact in
FP32, so the only difference is FP32 accumulation over K terms: |err| <= K 2^-24 sum |a||b|, i.e.
about 1e-5 relative in norm for K <= 1024 with random data."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("M,N,K", [(128, 256, 64), (256, 256, 640), (384, 512, 1024)])
def test_tc_gemm_matches_host(M, N, K):
    import torch
    from paper_1412_7466_gb300 import GratingSolver
    g = torch.Generator().manual_seed(M + N + K)
    A = torch.randn(M, K, generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, generator=g).to(torch.bfloat16)
    ref = A.double() @ B.double().T
    gs = GratingSolver(0)
    C = gs.tc_gemm_bf16(A.cuda(), B.cuda()).cpu().double()
    gs.close()
    err = torch.linalg.norm(C - ref) / torch.linalg.norm(ref)
    assert float(err) <= 1e-5, float(err)
    # element-wise bound: K 2^-24 sum |a||b|
    bound = K * 2.0 ** -24 * (A.double().abs() @ B.double().abs().T)
    assert bool(((C - ref).abs() <= bound + 1e-30).all())


def test_tc_gemm_rejects_bad_shapes():
    import torch
    from paper_1412_7466_gb300 import GS_ERR_ARG, GratingSolver, GsError
    gs = GratingSolver(0)
    A = torch.zeros(100, 64, dtype=torch.bfloat16, device="cuda")
    B = torch.zeros(256, 64, dtype=torch.bfloat16, device="cuda")
    with pytest.raises(GsError) as e:
        gs.tc_gemm_bf16(A, B)
    assert e.value.status == GS_ERR_ARG
    gs.close()


@pytest.mark.parametrize("M,p,R", [(37, 8, 5), (130, 12, 300)])
def test_translate_multi_matches_oracle(M, p, R):
    """R angles of one geometry through the tensor-core translation, against the oracle's dense
    translation per angle.  bfloat16 operands (2^-9 relative rounding of each operator entry and
    coefficient, FP32 accumulation): ~3e-3 relative in norm; bound 1e-2.  R = 300 spans two
    256-column tiles; M = 130, p = 12 gives ragged row and column tails."""
    import math
    import workloads as W
    from oracle import inclusions as I
    from paper_1412_7466_gb300 import GratingSolver
    g = W.grating("tiny")
    dk = W.disks(M, 0.01, 0.005, 2.0, g["k"][0], seed=50 + M, p=p)
    gs = GratingSolver(0)
    gs.set_layers(g)
    gs.set_incidence([-1.0])
    gs.set_inclusions(dk)
    gs.factor()
    rng = np.random.default_rng(M)
    nc = 2 * p + 1
    n = M * nc
    thetas = -math.pi / 2 + rng.uniform(-math.pi / 3, math.pi / 3, R)
    alphas = np.exp(1j * g["k"][0] * np.cos(thetas) * g["d"])
    w = np.tile(0.5 ** np.abs(np.arange(-p, p + 1)), M)
    betas = (rng.standard_normal((R, n)) + 1j * rng.standard_normal((R, n))) * w
    got = gs.translate_multi(alphas, betas).cpu().numpy()
    gs.close()
    for r in sorted({0, 1, R // 2, R - 1}):
        T = I.translation_matrix(dk["xy"], g["k"][1], p, g["d"], alphas[r])
        ref = T @ betas[r]
        err = np.linalg.norm(got[r] - ref) / np.linalg.norm(ref)
        assert err <= 1e-2, (r, err)


@pytest.mark.parametrize("M,p,R", [(37, 8, 5), (130, 12, 140)])
def test_translate_multi_split_matches_oracle(M, p, R):
    """The inner operator of the multi-angle solve: operator and coefficients each split into three
    bfloat16 parts (~24 significant bits together), the six products of parts whose orders add up to
    at most 2 accumulated in FP32.  Per entry the dropped products and the rounding of the last parts
    are ~2^-24 relative, so FP32 accumulation over 6n terms dominates: bound 1e-5 relative in norm
    (the complex64 translation's bound), against the oracle's dense translation per angle.  R = 140
    spans several 256-column tiles of the stacked coefficient parts."""
    import math
    import workloads as W
    from oracle import inclusions as I
    from paper_1412_7466_gb300 import GratingSolver
    g = W.grating("tiny")
    dk = W.disks(M, 0.01, 0.005, 2.0, g["k"][0], seed=60 + M, p=p)
    gs = GratingSolver(0)
    gs.set_layers(g)
    gs.set_incidence([-1.0])
    gs.set_inclusions(dk)
    gs.factor()
    rng = np.random.default_rng(M + 1)
    nc = 2 * p + 1
    n = M * nc
    thetas = -math.pi / 2 + rng.uniform(-math.pi / 3, math.pi / 3, R)
    alphas = np.exp(1j * g["k"][0] * np.cos(thetas) * g["d"])
    w = np.tile(0.5 ** np.abs(np.arange(-p, p + 1)), M)
    betas = (rng.standard_normal((R, n)) + 1j * rng.standard_normal((R, n))) * w
    got = gs.translate_multi_split(alphas, betas).cpu().numpy()
    gs.close()
    errs = []
    for r in sorted({0, 1, R // 2, R - 1}):
        T = I.translation_matrix(dk["xy"], g["k"][1], p, g["d"], alphas[r])
        ref = T @ betas[r]
        errs.append(np.linalg.norm(got[r] - ref) / np.linalg.norm(ref))
    print("three-part tensor-core translation, relative errors", errs)
    assert max(errs) <= 1e-5, errs
