"""Bounded waits: a wait that runs out stops the kernel, raises the device
error word read by fk_device_status, and leaves the device usable.

The wait is made to run out on a barrier nothing arrives on (fk_wait_selftest),
through the same wait the tensor-core kernels use; nothing faults or hangs.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1909_10547_b300 as fk
from paper_1909_10547_b300 import _lib
from paper_1909_10547_b300 import workloads as W

pytestmark = pytest.mark.gpu


def test_bounded_wait_reports_and_device_stays_usable():
    lib = _lib.load()
    assert lib.fk_device_status(1) == 0
    assert lib.fk_wait_selftest(20000) == 0        # ran out after 20 ms and was reported
    assert lib.fk_device_status(0) == 0            # the self-test cleared the flag
    # the device still computes correctly afterwards
    t, F = W.config1(R=3, ndata=20, nc=10, nx=12)
    tab = fk.Table.from_workload(t, precs=("fp64", "bf16x3"))
    O_ref, S = oracle.had(t, F)
    O = fk.conv(tab, torch.tensor(F, device="cuda"), "fp64").cpu().numpy()
    assert np.all(np.abs(O - O_ref) <= 1e-12 * S)
    O3 = fk.conv(tab, torch.tensor(F, dtype=torch.float32, device="cuda"), "bf16x3")
    torch.cuda.synchronize()
    assert lib.fk_device_status(1) == 0


def test_wait_selftest_rejects_bad_limits():
    lib = _lib.load()
    assert lib.fk_wait_selftest(0) == _lib.FK_EINVAL
    assert lib.fk_wait_selftest(2000000) == _lib.FK_EINVAL
