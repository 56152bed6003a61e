"""Measurement support on the device: the FP64 throughput probe and the
kernel timing of the tensor-core products (the roofline denominators and
numerators of bench.py)."""
import pytest

pytestmark = pytest.mark.gpu


def test_fp64_peak_is_in_the_parts_range(lrs):
    from paper_2105_01271_gb300 import binding as b
    t = lrs.fp64_peak(2048)
    # GB300: 152 SMs x 2 FP64 FMA per clock at up to 2.07 GHz = 1.26 TFLOP/s nominal
    assert 0.3 <= t <= 1.6, t
    with pytest.raises(b.LrsError, match="iters"):
        lrs.fp64_peak(1)


def test_kernel_timing_covers_the_generic_tensor_core_product(lrs):
    import torch
    from paper_2105_01271_gb300 import binding as b
    M, N, K = 384, 4096, 512            # M > 256: the generic product, not the TMA A-pass
    X = torch.randn((K, M), dtype=torch.float64, device="cuda")
    A = torch.randn((K, N), dtype=torch.float32, device="cuda")
    C = torch.empty((M, N), dtype=torch.float32, device="cuda")
    lrs.set_kernel_timing(True)
    lrs.gemm_tn(M, N, K, X, b.LRS_F64, M, A, b.LRS_F32, N, C, 0, 0, N, b.LRS_PREC_SPLIT_BF16)
    ms = lrs.last_kernel_ms()
    lrs.set_kernel_timing(False)
    assert ms > 0.0
    ref = (X.T @ A.double()).float()
    assert torch.allclose(C, ref, rtol=0, atol=1e-3 * float(ref.abs().max()))
