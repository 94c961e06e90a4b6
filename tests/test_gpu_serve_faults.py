"""Failure detection in the serving loop, with every fault made on the host.

Injected faults (fk_serve_inject / FK_FAULT): a failed pinned staging
allocation, a failed device allocation, a failed convolution launch and a
lost completion message; plus a cancelled ticket and a server destroyed with
requests queued and running.  Each must end in its own per-ticket status
within a bounded time, leave the server usable and return the budget.  No
kernel is made to fault, trap or hang.
"""
import os
import subprocess
import sys
import time

import numpy as np
import pytest

import paper_1909_10547_b300 as fk
from paper_1909_10547_b300 import _lib
from paper_1909_10547_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    g = W.config3(R=4, scale=0.1)
    k = next(i for i, t in enumerate(g.tables) if hasattr(t, "ca"))
    tab = fk.Table.from_workload(g.tables[k], precs=("fp64", "fp32"))
    return g, tab


def status_of(fn):
    with pytest.raises(fk.FKError) as e:
        fn()
    return e.value.status


def test_injected_faults_end_in_ticket_status(setup):
    g, tab = setup
    srv = fk.Server(budget_bytes=8 << 30, max_inflight=2)
    tid = srv.add_table(tab)
    F = W.pdf_replicas(g.x, g.params, 3, None)
    ok = srv.wait(srv.submit(tid, F, "fp64"))
    # pinned staging fails at submit
    srv.inject("pinned", 1)
    assert status_of(lambda: srv.submit(tid, F, "fp64")) == _lib.FK_ENOMEM
    # device allocation of the batch fails
    srv.inject("device", 1)
    tk = srv.submit(tid, F, "fp64")
    assert status_of(lambda: srv.wait(tk, 10000)) == _lib.FK_ENOMEM
    # the convolution launch fails
    srv.inject("launch", 1)
    tk = srv.submit(tid, F, "fp64")
    assert status_of(lambda: srv.wait(tk, 10000)) == _lib.FK_ECUDA
    # the completion message is lost: the watchdog ends the ticket
    srv.inject("drop", 1)
    tk = srv.submit(tid, F, "fp64")
    t0 = time.time()
    assert status_of(lambda: srv.wait(tk, 10000)) == _lib.FK_ETIMEDOUT
    assert time.time() - t0 < 5.0
    # the server is still usable, results unchanged, budget returned
    assert np.array_equal(srv.wait(srv.submit(tid, F, "fp64")), ok)
    st = srv.stats()
    assert st["queued"] == 0
    srv.close()


def test_cancel_queued_and_running(setup):
    g, tab = setup
    srv = fk.Server(budget_bytes=8 << 30, max_inflight=1)
    tid = srv.add_table(tab)
    big = W.pdf_replicas(g.x, g.params, 2000, None)
    small = W.pdf_replicas(g.x, g.params, 2, None)
    t_big = srv.submit(tid, big, "fp64")      # occupies the only slot
    t_q = [srv.submit(tid, small, "fp64") for _ in range(3)]
    srv.cancel(t_q[1])                        # still queued
    srv.cancel(t_big)                         # running (or done)
    assert status_of(lambda: srv.wait(t_q[1], 60000)) == _lib.FK_ECANCELED
    st_big = None
    try:
        srv.wait(t_big, 60000)
    except fk.FKError as e:
        st_big = e.status
    assert st_big in (None, _lib.FK_ECANCELED)
    ref = srv.wait(t_q[0], 60000)
    assert np.array_equal(srv.wait(t_q[2], 60000), ref)
    assert status_of(lambda: srv.cancel(123456789)) == _lib.FK_ENOTFOUND
    srv.close()


def test_destroy_with_requests_in_flight(setup):
    g, tab = setup
    srv = fk.Server(budget_bytes=8 << 30, max_inflight=2)
    tid = srv.add_table(tab)
    F = W.pdf_replicas(g.x, g.params, 500, None)
    for _ in range(20):
        srv.submit(tid, F, "fp64")
    t0 = time.time()
    srv.close()                               # queued ones cancelled, running ones finish
    assert time.time() - t0 < 60.0


def test_fault_environment_variable():
    """FK_FAULT arms faults at fk_serve_create (a fresh process)."""
    code = (
        "import numpy as np, paper_1909_10547_b300 as fk\n"
        "from paper_1909_10547_b300 import workloads as W, _lib\n"
        "g = W.config3(R=2, scale=0.1)\n"
        "t = next(t for t in g.tables if hasattr(t, 'ca'))\n"
        "tab = fk.Table.from_workload(t, precs=('fp32',))\n"
        "s = fk.Server(1 << 32, 1); tid = s.add_table(tab)\n"
        "F = W.pdf_replicas(g.x, g.params, 2, None)\n"
        "try:\n"
        "    s.wait(s.submit(tid, F, 'fp32'), 10000); print('no fault')\n"
        "except fk.FKError as e:\n"
        "    print('status', e.status)\n"
        "s.wait(s.submit(tid, F, 'fp32'), 10000); print('second ok')\n"
        "s.close()\n")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, FK_FAULT="device:1")
    out = subprocess.run([sys.executable, "-c", code], cwd=root, env=env, capture_output=True, text=True,
                         timeout=600)
    assert out.returncode == 0, out.stderr
    assert f"status {_lib.FK_ENOMEM}" in out.stdout and "second ok" in out.stdout, out.stdout
