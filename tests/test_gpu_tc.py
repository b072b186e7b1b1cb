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
