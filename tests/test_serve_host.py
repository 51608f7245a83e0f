"""The re-planning server's host logic with a fake plan and fake CUDA hooks (no GPU):
admission keeps the in-flight device footprint under the budget, oversized requests are
refused, a failing request does not take its worker down, and warm start hands a patient's
last x to the next solve."""
import threading
import time
import types

import numpy as np
import pytest
import torch

from paper_0908_4421_gb300 import _lib as L
from paper_0908_4421_gb300 import serve


class FakePlan:
    lock = threading.Lock()
    live = 0
    max_live = 0
    x0s = []

    def __init__(self, row_ptr, col, val, mask, thresholds, weights, m, n, options):
        if getattr(mask, "fail", False):
            raise RuntimeError("planted failure")
        self.n, self.options = n, options

    def __enter__(self):
        with FakePlan.lock:
            FakePlan.live += 1
            FakePlan.max_live = max(FakePlan.max_live, FakePlan.live)
        return self

    def __exit__(self, *exc):
        with FakePlan.lock:
            FakePlan.live -= 1

    def solve(self, x0=None, raise_on_error=True):
        FakePlan.x0s.append((None if x0 is None else x0.copy(), self.options.x_init))
        time.sleep(0.02)
        return types.SimpleNamespace(objective=1.0, iterations=3, status=0)

    def get_x(self):
        return np.full(self.n, 2.0, np.float32)

    def dose(self, x):
        return np.zeros(4, np.float32)


class Mask(np.ndarray):
    fail = False


def case(n=10, fail=False):
    mask = np.zeros(4, np.uint8).view(Mask)
    mask.fail = fail
    return types.SimpleNamespace(m=100, n=n, nnz=1000, row_ptr=None, col=None, val=None, mask=mask,
                                 thresholds=None, weights=None)


@pytest.fixture
def fake_cuda(monkeypatch):
    FakePlan.live = FakePlan.max_live = 0
    FakePlan.x0s = []
    need = serve.plan_footprint_bytes(100, 10, 1000, L.FP32)
    free = int((2 * need + 10) / 0.8) + 1  # a budget for exactly two requests in flight
    monkeypatch.setattr(torch.cuda, "set_device", lambda d: None)
    monkeypatch.setattr(torch.cuda, "mem_get_info", lambda d=None: (free, 2 * free))
    monkeypatch.setattr(torch.cuda, "Stream", lambda device=None: types.SimpleNamespace(cuda_stream=0))
    monkeypatch.setattr(serve, "Plan", FakePlan)
    return need


def test_admission_keeps_in_flight_bytes_under_the_budget(fake_cuda):
    srv = serve.ReplanServer(workers=4)
    futs = [srv.submit(case()) for _ in range(8)]
    res = [f.result(timeout=10) for f in futs]
    srv.close()
    assert len(res) == 8 and all(r.status == 0 for r in res)
    assert srv.peak_in_flight <= srv.budget < 3 * fake_cuda
    assert FakePlan.max_live == 2  # four workers, but the budget holds two plans
    assert srv.in_flight == 0


def test_oversized_request_is_refused(fake_cuda):
    srv = serve.ReplanServer(workers=1)
    with pytest.raises(ValueError, match="HBM budget"):
        srv.submit(types.SimpleNamespace(m=10**7, n=10, nnz=10**9))
    srv.close()


def test_failed_request_keeps_the_worker(fake_cuda):
    srv = serve.ReplanServer(workers=1)
    bad = srv.submit(case(fail=True))
    good = srv.submit(case())
    with pytest.raises(RuntimeError, match="planted"):
        bad.result(timeout=10)
    assert good.result(timeout=10).status == 0
    srv.close()
    assert srv.in_flight == 0


def test_warm_start_passes_the_last_x(fake_cuda):
    srv = serve.ReplanServer(workers=1, warm_start=True)
    srv.submit(case(), patient="p1").result(timeout=10)
    srv.submit(case(), patient="p1").result(timeout=10)
    srv.submit(case(n=12), patient="p1").result(timeout=10)  # another beamlet count: cold start
    srv.close()
    (x0a, ia), (x0b, ib), (x0c, ic) = FakePlan.x0s
    assert x0a is None and x0c is None
    np.testing.assert_array_equal(x0b, np.full(10, 2.0, np.float32))
    assert ib == 2 and ic != 2
