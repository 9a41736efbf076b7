"""Failure detection without a GPU fault: a bounded device wait that nothing
completes gives up, the host reads DDEL_ETIMEOUT, and the device stays usable."""
import time

import numpy as np
import pytest

import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_bounded_wait_reports_timeout_and_device_stays_usable():
    from paper_1501_06211_gb300 import ddel
    t0 = time.perf_counter()
    code, status = ddel.ddel_selftest_wait_timeout(2000)
    assert code == ddel.DDEL_OK and status == ddel.DDEL_ETIMEOUT
    assert time.perf_counter() - t0 < 10.0
    assert ddel.ddel_selftest_wait_timeout(0)[0] == ddel.DDEL_EINVAL
    # a solve afterwards runs normally
    cfg = workloads.config("c0")
    s = ddel.Solver(cfg, tol=1e-8)
    s.assemble(workloads.density(cfg))
    s.factor()
    u, st = s.solve()
    assert st.status == ddel.DDEL_OK and st.relres <= 1e-8 and np.isfinite(u).all()
