"""The tcgen05 BF16 GEMM against an FP64 product of the same BF16-rounded
inputs.  Products of two BF16 numbers are exact in FP32, so the only error is
the FP32 accumulation: bound |C - C_ref| <= K * 2^-23 * sum|a||b| (loose)."""
import numpy as np
import pytest

from paper_2503_06757_gb300 import prrtc as P

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2503_06757_gb300 import build
    build.build()


def _case(M, N, K, bias=False, relu=False, seed=0, splits=None, rows=None):
    g = torch.Generator(device="cpu").manual_seed(seed)
    A = torch.randn(M, K, generator=g).to(torch.bfloat16).cuda()
    B = torch.randn(N, K, generator=g).to(torch.bfloat16).cuda()
    bv = torch.randn(N, generator=g).float().cuda() if bias else None
    c32 = torch.zeros(M, N, dtype=torch.float32, device="cuda")
    c16 = torch.zeros(M, N, dtype=torch.bfloat16, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    if splits is None:
        P.prrtc_gemm_bf16(A.data_ptr(), B.data_ptr(), M, N, K, bv.data_ptr() if bias else 0, relu, c32.data_ptr(),
                          c16.data_ptr(), stream)
    else:
        P.prrtc_gemm_bf16_splitk(A.data_ptr(), B.data_ptr(), M, N, K, bv.data_ptr() if bias else 0, relu,
                                 c32.data_ptr(), c16.data_ptr(), splits, stream)
    torch.cuda.synchronize()
    assert P.prrtc_gemm_error() == 0
    rows = np.arange(M) if rows is None else rows
    a = A.float().cpu().numpy().astype(np.float64)[rows]
    b = B.float().cpu().numpy().astype(np.float64)
    ref = a @ b.T
    if bias:
        ref = ref + bv.cpu().numpy()[None, :]
    if relu:
        ref = np.maximum(ref, 0.0)
    bound = K * 2.0 ** -23 * (np.abs(a) @ np.abs(b).T) + 1e-6
    got = c32.cpu().numpy()[rows]
    c16 = c16[torch.as_tensor(rows, device="cuda")]
    c32 = c32[torch.as_tensor(rows, device="cuda")]
    assert np.all(np.abs(got - ref) <= bound), float(np.max(np.abs(got - ref) - bound))
    # the BF16 output is the FP32 result rounded once
    np.testing.assert_array_equal(c16.float().cpu().numpy(), c32.to(torch.bfloat16).float().cpu().numpy())
    return got, ref


@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (256, 256, 512), (200, 1024, 4160), (130, 136, 72),
                                   (1, 8, 8), (512, 512, 1024), (37, 256, 200)])
def test_gemm_matches_fp64(M, N, K):
    _case(M, N, K)


def test_gemm_bias_relu():
    _case(300, 232, 512, bias=True, relu=True, seed=3)


def test_gemm_rejects_bad_shapes():
    A = torch.zeros(16, 12, dtype=torch.bfloat16, device="cuda")
    c = torch.zeros(16, 16, dtype=torch.float32, device="cuda")
    with pytest.raises(P.PrrtcError):
        P.prrtc_gemm_bf16(A.data_ptr(), A.data_ptr(), 16, 16, 12, 0, False, c.data_ptr(), 0)


@pytest.mark.parametrize("splits", [1, 2, 3, 5, 16])
@pytest.mark.parametrize("M,N,K", [(200, 1024, 4160), (130, 264, 1000)])
def test_gemm_split_k_matches_fp64(M, N, K, splits):
    """K split into ranges (65 and 16 k-tiles: uneven ranges) summed in order."""
    _case(M, N, K, bias=True, relu=True, seed=splits, splits=splits)


def test_gemm_split_k_deterministic():
    g = torch.Generator(device="cpu").manual_seed(9)
    A = torch.randn(256, 4160, generator=g).to(torch.bfloat16).cuda()
    B = torch.randn(512, 4160, generator=g).to(torch.bfloat16).cuda()
    outs = []
    for _ in range(3):
        c = torch.zeros(256, 512, dtype=torch.float32, device="cuda")
        P.prrtc_gemm_bf16_splitk(A.data_ptr(), B.data_ptr(), 256, 512, 4160, 0, False, c.data_ptr(), 0, 8,
                                 torch.cuda.current_stream().cuda_stream)
        outs.append(c.cpu())
    assert torch.equal(outs[0], outs[1]) and torch.equal(outs[0], outs[2])


def test_gemm_many_tiles_per_cta():
    """More than two output tiles per CTA: both tensor-memory accumulators are
    reused several times (sampled rows against FP64)."""
    rows = np.random.default_rng(0).choice(4096, 96, replace=False)
    _case(4096, 4096, 256, bias=True, seed=11, rows=np.sort(rows))


def test_gemm_large_k_sampled():
    rows = np.sort(np.random.default_rng(1).choice(1024, 64, replace=False))
    _case(1024, 2048, 8192, seed=12, rows=rows)
