"""The tcgen05 BF16 GEMM (the tensor-core building block of the candidate
ranker) against a float64 CPU product of the same bf16 values: ragged M, N
and K, several tiles, split-K, bias and ReLU epilogues."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def gsp():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2110_12749_gb300 import build, gsp as g
    build.build()
    g.lib()
    return g


@pytest.mark.parametrize("M,N,K,splitk,bias,relu", [
    (128, 16, 64, 1, False, False),       # one tile, one K step
    (200, 40, 136, 1, True, False),       # ragged M, N, K
    (300, 130, 512, 1, True, True),       # several tiles in M and N
    (64, 9, 4096, 8, False, False),       # split-K (weight-gradient shape)
    (1024, 64, 2048, 1, True, True),      # fully connected layer shape
    (4096, 96, 2048, 1, True, True),      # fc1 of an inference batch (narrow column blocks)
    (89600, 8, 16, 1, True, True),        # first conv layer shape: CTAs loop over M tiles
    (40000, 72, 32, 1, False, False),     # conv input-gradient shape
])
def test_gemm_matches_float64(gsp, M, N, K, splitk, bias, relu):
    g = torch.Generator().manual_seed(M * 7 + N * 3 + K)
    lda = (K + 7) // 8 * 8 + 8
    A = torch.zeros((M, lda), dtype=torch.bfloat16)
    B = torch.zeros((N, lda), dtype=torch.bfloat16)
    A[:, :K] = torch.randn((M, K), generator=g).to(torch.bfloat16)
    B[:, :K] = torch.randn((N, K), generator=g).to(torch.bfloat16)
    bvec = torch.randn(N, generator=g, dtype=torch.float32) if bias else None
    ref = A[:, :K].double() @ B[:, :K].double().T
    if bias:
        ref = ref + bvec.double()
    if relu:
        ref = ref.clamp_min(0.0)
    C = torch.full((M, N + 3), 0.0 if splitk > 1 else -9.0, dtype=torch.float32, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    gsp.gsp_gemm_bf16(A.cuda(), B.cuda(), C, M, N, K,
                      bias=bvec.cuda() if bias else None, relu=relu, splitk=splitk, err=err)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    got = C[:, :N].double().cpu()
    # FP32 accumulation of K products of bf16 values: error <= K * 2^-24 * sum|a b|
    bound = (A[:, :K].double().abs() @ B[:, :K].double().abs().T) * (K * 2.0 ** -24) + 1e-6
    assert ((got - ref).abs() <= bound).all(), float((got - ref).abs().max())
    if splitk == 1:
        assert (C[:, N:] == -9.0).all()
