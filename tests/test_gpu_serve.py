"""Serving loop: continuous batching over resident tables.

Each served result must equal the same request run alone through fk_*_conv:
bit for bit in FP64/FP32 (the coalescing never changes a replica's kernel or
summation order) and within the mode's error in the tensor-core modes (where
replica rows are independent too, so equality is checked as well).
"""
import time

import numpy as np
import pytest
import torch

import oracle
import paper_1909_10547_b300 as fk
from paper_1909_10547_b300 import workloads as W

pytestmark = pytest.mark.gpu


def alone(tab, F, prec):
    dt = torch.float64 if prec == "fp64" else torch.float32
    O = fk.conv(tab, torch.tensor(F, dtype=dt, device="cuda"), prec)
    torch.cuda.synchronize()
    return O.cpu().numpy()


@pytest.fixture(scope="module")
def setup():
    g = W.config3(R=8, scale=0.1)
    tabs, kinds = [], []
    for t in g.tables[:10]:
        had = hasattr(t, "ca")
        precs = ("fp64", "fp32", "bf16", "bf16x3", "tf32")
        tabs.append(fk.Table.from_workload(t, precs=precs))
        kinds.append(had)
    return g, tabs, kinds


def test_served_results_equal_alone(setup):
    g, tabs, kinds = setup
    srv = fk.Server(budget_bytes=8 << 30, max_inflight=4)
    ids = [srv.add_table(t) for t in tabs]
    rng = np.random.default_rng(0)
    reqs = []
    for n in range(60):
        k = int(rng.integers(len(tabs)))
        precs = ["fp64", "fp32", "bf16", "bf16x3", "tf32"]
        prec = precs[int(rng.integers(len(precs)))]
        R = int(rng.choice([1, 2, 3, 7, 40, 130]))
        F = W.pdf_replicas(g.x, g.params, R, np.random.default_rng(1000 + n))
        reqs.append((k, prec, F, srv.submit(ids[k], F, prec)))
    for k, prec, F, tk in reqs:
        O = srv.wait(tk, 60000)
        ref = alone(tabs[k], F, prec)
        assert np.array_equal(O, ref), (k, prec, F.shape[0], np.abs(O - ref).max())
    st = srv.stats()
    assert st["completed"] == len(reqs)
    assert st["launches"] <= len(reqs)
    srv.close()


def test_served_matches_oracle(setup):
    g, tabs, kinds = setup
    srv = fk.Server(budget_bytes=8 << 30, max_inflight=2)
    k = kinds.index(True)
    tid = srv.add_table(tabs[k])
    F = W.pdf_replicas(g.x, g.params, 5, np.random.default_rng(5))
    O = srv.wait(srv.submit(tid, F, "fp64"))
    ref, S = oracle.conv(g.tables[k], F)
    assert np.all(np.abs(O - ref) <= 1e-12 * S)
    srv.close()


def test_budget_admission_serialises_but_completes(setup):
    g, tabs, kinds = setup
    k = kinds.index(True)
    t = tabs[k]
    budget = t.device_bytes() + (12 << 20)  # room for about one request at a time
    srv = fk.Server(budget_bytes=budget, max_inflight=4)
    tid = srv.add_table(t)
    F = W.pdf_replicas(g.x, g.params, 64, np.random.default_rng(9))
    tks = [srv.submit(tid, F, "fp32") for _ in range(6)]
    outs = [srv.wait(tk) for tk in tks]
    for O in outs[1:]:
        assert np.array_equal(O, outs[0])
    assert srv.stats()["peak_bytes"] <= budget
    srv.close()


def test_serve_errors(setup):
    g, tabs, kinds = setup
    k = kinds.index(True)
    srv = fk.Server(budget_bytes=tabs[k].device_bytes() + (1 << 20), max_inflight=1)
    tid = srv.add_table(tabs[k])
    with pytest.raises(fk.FKError, match="budget"):
        srv.submit(tid, W.pdf_replicas(g.x, g.params, 4000, None), "fp32")
    with pytest.raises(fk.FKError, match="not found"):
        srv.submit(7, W.pdf_replicas(g.x, g.params, 1, None), "fp32")
    with pytest.raises(fk.FKError, match="not found"):
        srv.poll(12345)
    # a precision the table does not store
    d = next(t for t in g.tables if not hasattr(t, "ca"))
    only64 = fk.Table.from_workload(d, precs=("fp64",))
    small = fk.Server(budget_bytes=1 << 30, max_inflight=1)
    tid2 = small.add_table(only64)
    with pytest.raises(fk.FKError, match="unsupported"):
        small.submit(tid2, W.pdf_replicas(g.x, g.params, 1, None), "bf16")
    small.close()
    srv.close()


def test_poll_reports_pending_then_done(setup):
    g, tabs, kinds = setup
    k = kinds.index(True)
    srv = fk.Server(budget_bytes=8 << 30, max_inflight=1)
    tid = srv.add_table(tabs[k])
    F = W.pdf_replicas(g.x, g.params, 128, np.random.default_rng(3))
    tk = srv.submit(tid, F, "fp64")
    t0 = time.time()
    done, O = srv.poll(tk)
    while not done and time.time() - t0 < 60:
        time.sleep(0.001)
        done, O = srv.poll(tk)
    assert done
    assert np.array_equal(O, alone(tabs[k], F, "fp64"))
    srv.close()
