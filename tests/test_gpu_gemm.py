"""The tcgen05 BF16 GEMM through the C ABI against an FP64 matmul of the same
bf16-rounded operands (FP32 accumulation: relative tolerance 2e-6 * sqrt(K)
of the row's magnitude)."""
import numpy as np
import pytest

import paper_1501_03450_b300 as st

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("M,N,K", [(128, 256, 64), (256, 256, 256), (384, 128, 192), (128, 16, 256),
                                   (256, 64, 512), (128, 32, 64), (1024, 256, 1024)])
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


def test_gemm_rejects_bad_shapes():
    torch = pytest.importorskip("torch")
    A = torch.zeros(100, 64, dtype=torch.bfloat16, device="cuda")
    D = torch.zeros(100, 16, dtype=torch.float32, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(st.SpinTrackError) as e:
        st.st_gemm_bf16(A.data_ptr(), A.data_ptr(), D.data_ptr(), 100, 16, 64, None, status.data_ptr())
    assert e.value.code == st.ST_EINVAL
