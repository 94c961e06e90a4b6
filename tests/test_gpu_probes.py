"""The measurement probes behind profiles/peaks.txt: fk_fma_probe (CUDA-core
multiply-add chains) and fk_mma_probe (back-to-back BF16 tcgen05.mma of
128 x N x 16).  They run, report a plausible count and leave no device error;
the rates themselves are measurements, recorded by bench.py --case peaks."""
import ctypes

import pytest
import torch

from paper_1909_10547_b300 import _lib

pytestmark = pytest.mark.gpu


def stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


@pytest.mark.parametrize("fill", [0, 1])
@pytest.mark.parametrize("n", [16, 64, 240, 256])
def test_mma_probe_counts_cycles(n, fill):
    cyc = torch.zeros(1, dtype=torch.int64, device="cuda")
    _lib.call("fk_mma_probe", n, 2048, fill, ctypes.c_void_p(cyc.data_ptr()), stream())
    torch.cuda.synchronize()
    per = cyc.item() / 2048
    # one instruction of 128 x n x 16 BF16 multiply-adds: at least the
    # nominal dense rate allows (8192 flops per SM cycle), at most a few
    # hundred cycles
    assert 2 * 128 * n * 16 / 8192 * 0.9 <= per < 2000, per
    assert _lib.load().fk_device_status(1) == 0


def test_fma_probe_runs():
    sink = torch.zeros(148, dtype=torch.float64, device="cuda")
    _lib.call("fk_fma_probe", _lib.FK_FP64, 148, 64, ctypes.c_void_p(sink.data_ptr()), stream())
    torch.cuda.synchronize()
    assert torch.count_nonzero(sink) == 0  # the sink condition is never met
