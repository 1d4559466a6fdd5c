"""The tcgen05 BF16 GEMM through the C ABI against an FP64 matmul of the same
bf16-rounded operands (FP32 accumulation: relative tolerance 2e-6 * sqrt(K)
of the row's magnitude)."""
import numpy as np
import pytest

import paper_1501_03450_b300 as st

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("M,N,K", [(128, 256, 64), (256, 256, 256), (384, 128, 192), (128, 16, 256),
                                   (256, 64, 512), (128, 32, 64), (1024, 256, 1024), (32768, 256, 256)])
@pytest.mark.parametrize("with_bias", [False, True])
def test_gemm_matches_fp64_reference(M, N, K, with_bias):
    torch = pytest.importorskip("torch")
    g = torch.Generator().manual_seed(M * 7 + N * 13 + K)
    A = torch.randn(M, K, generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, generator=g).to(torch.bfloat16)
    bias = torch.randn(N, generator=g, dtype=torch.float32)
    ref = A.double() @ B.double().T
    if with_bias:
        ref = ref + bias.double()
    Ad, Bd = A.cuda(), B.cuda()
    D = torch.full((M, N), float("nan"), dtype=torch.float32, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    bd = bias.cuda()
    st.st_gemm_bf16(Ad.data_ptr(), Bd.data_ptr(), D.data_ptr(), M, N, K, bd.data_ptr() if with_bias else None,
                    status.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    Dh = D.cpu().double()
    scale = (A.double().abs() @ B.double().abs().T).max()
    assert torch.isfinite(Dh).all()
    assert (Dh - ref).abs().max() / scale < 2e-6 * np.sqrt(K) + 1e-7


def test_gemm_with_a_bias_that_is_not_16_byte_aligned():
    """The epilogue reads the bias as 16-byte vectors when it can and element
    by element otherwise: a bias starting one float into its buffer gives
    the same result."""
    torch = pytest.importorskip("torch")
    M, N, K = 256, 128, 128
    g = torch.Generator().manual_seed(5)
    A = torch.randn(M, K, generator=g).to(torch.bfloat16).cuda()
    B = torch.randn(N, K, generator=g).to(torch.bfloat16).cuda()
    buf = torch.randn(N + 1, generator=g, dtype=torch.float32).cuda()
    aligned = buf[1:].clone()
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    D1 = torch.empty((M, N), dtype=torch.float32, device="cuda")
    D2 = torch.empty((M, N), dtype=torch.float32, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    st.st_gemm_bf16(A.data_ptr(), B.data_ptr(), D1.data_ptr(), M, N, K, buf.data_ptr() + 4, status.data_ptr(), s)
    st.st_gemm_bf16(A.data_ptr(), B.data_ptr(), D2.data_ptr(), M, N, K, aligned.data_ptr(), status.data_ptr(), s)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    assert torch.equal(D1, D2)


def test_gemm_rejects_bad_shapes():
    torch = pytest.importorskip("torch")
    A = torch.zeros(100, 64, dtype=torch.bfloat16, device="cuda")
    D = torch.zeros(100, 16, dtype=torch.float32, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(st.SpinTrackError) as e:
        st.st_gemm_bf16(A.data_ptr(), A.data_ptr(), D.data_ptr(), 100, 16, 64, None, status.data_ptr())
    assert e.value.code == st.ST_EINVAL
