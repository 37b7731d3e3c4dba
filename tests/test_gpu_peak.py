"""GPU test of the tensor-pipe peak probe (hz_tensor_peak): the measured dense MMA rates are in
the range the hardware allows (TF32 at half the bf16 rate; neither above the SM clock limit; the
same TF32 rate with the A operand in tensor memory), and bad arguments come back as statuses."""
import ctypes as ct

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_tensor_peak_probe():
    from paper_1801_08655_gb300 import build, hz
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    tf32, ms = hz.tensor_peak("tf32", 128, 0.3)
    bf16, _ = hz.tensor_peak("bf16", 128, 0.3)
    assert ms > 100.0
    # 152 SMs x 2070 MHz x 8192 (bf16) / 4096 (tf32) flops per SM and cycle bound the rates
    assert 300.0 < tf32 < 1.05 * 152 * 2.07e9 * 4096 / 1e12
    assert 600.0 < bf16 < 1.05 * 152 * 2.07e9 * 8192 / 1e12
    assert 0.4 < tf32 / bf16 < 0.6
    # the A operand read from tensor memory instead of shared memory: the same rate
    tmem_a, _ = hz.tensor_peak("tf32_tmem_a", 128, 0.3)
    assert 0.9 < tmem_a / tf32 < 1.1
    lib = hz.load()
    out = ct.c_double()
    assert lib.hz_tensor_peak(3, 128, 0.1, ct.byref(out), None) == hz.HZ_ERR_ARG
    assert lib.hz_tensor_peak(0, 96, 0.1, ct.byref(out), None) == hz.HZ_ERR_ARG
