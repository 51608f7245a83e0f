"""The re-planning server's host logic with a fake plan, a fake batched solve and fake CUDA
hooks (no GPU): admission keeps the reserved device bytes under the budget and switches to
the measured plan size, oversized requests are refused, a failing request does not take its
worker down, warm start hands a patient's last x to the next solve, requests that arrive
while a launch runs are batched into the next one, and resident plans are rebuilt in place
and evicted least recently used first."""
import threading
import time
import types

import numpy as np
import pytest
import torch

from paper_0908_4421_gb300 import _lib as L
from paper_0908_4421_gb300 import serve
from paper_0908_4421_gb300.api import Options

NEED = serve.plan_footprint_bytes(100, 10, 1000, L.FP32)


class FakePlan:
    lock = threading.Lock()
    live = 0
    max_live = 0
    created = 0
    updates = 0
    x0s = []

    def __init__(self, row_ptr, col, val, mask, thresholds, weights, m, n, options):
        if getattr(mask, "fail", False):
            raise RuntimeError("planted failure")
        self.n, self.options, self.closed = n, options, False
        with FakePlan.lock:
            FakePlan.live += 1
            FakePlan.created += 1
            FakePlan.max_live = max(FakePlan.max_live, FakePlan.live)

    def info(self):
        return {"device_bytes": NEED // 2}  # the measured size replaces the estimate

    def update(self, row_ptr, col, val, mask, thresholds, weights, m, n):
        FakePlan.updates += 1
        self.n = n

    def set_options(self, **kw):
        import dataclasses
        self.options = dataclasses.replace(self.options, **kw)

    def close(self):
        if not self.closed:
            self.closed = True
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


BATCHES = []


def fake_solve_batch(plans, x0s=None, stream=0, raise_on_error=True):
    BATCHES.append(len(plans))
    time.sleep(0.05)
    for p, x0 in zip(plans, x0s or [None] * len(plans)):
        FakePlan.x0s.append((None if x0 is None else x0.copy(), p.options.x_init))
    return [types.SimpleNamespace(objective=1.0, iterations=3, status=0) for _ in plans]


class Mask(np.ndarray):
    fail = False


def case(n=10, fail=False):
    mask = np.zeros(4, np.uint8).view(Mask)
    mask.fail = fail
    return types.SimpleNamespace(m=100, n=n, nnz=1000, row_ptr=None, col=None, val=None, mask=mask,
                                 thresholds=None, weights=None)


@pytest.fixture
def fake_cuda(monkeypatch):
    FakePlan.live = FakePlan.max_live = FakePlan.created = FakePlan.updates = 0
    FakePlan.x0s = []
    BATCHES.clear()
    free = int((2 * NEED + 10) / 0.8) + 1  # a budget for exactly two estimated requests in flight
    monkeypatch.setattr(torch.cuda, "set_device", lambda d: None)
    monkeypatch.setattr(torch.cuda, "mem_get_info", lambda d=None: (free, 2 * free))
    monkeypatch.setattr(torch.cuda, "Stream", lambda device=None: types.SimpleNamespace(cuda_stream=0))
    monkeypatch.setattr(serve, "Plan", FakePlan)
    monkeypatch.setattr(serve, "solve_batch", fake_solve_batch)
    return NEED


def test_admission_keeps_reserved_bytes_under_the_budget(fake_cuda):
    srv = serve.ReplanServer(workers=6, batched=False)
    futs = [srv.submit(case()) for _ in range(12)]
    res = [f.result(timeout=10) for f in futs]
    srv.close()
    assert len(res) == 12 and all(r.status == 0 for r in res)
    assert srv.peak_in_flight <= srv.budget < 3 * fake_cuda
    # the estimate admits two at a time; measured plans of half that size let a third one in
    assert 2 <= FakePlan.max_live <= 4
    assert srv.in_flight == 0 and FakePlan.live == 0


def test_oversized_request_is_refused(fake_cuda):
    srv = serve.ReplanServer(workers=1, batched=False)
    with pytest.raises(ValueError, match="HBM budget"):
        srv.submit(types.SimpleNamespace(m=10**7, n=10, nnz=10**9))
    srv.close()


@pytest.mark.parametrize("batched", [False, True])
def test_failed_request_keeps_the_worker(fake_cuda, batched):
    srv = serve.ReplanServer(workers=1, batched=batched)
    bad = srv.submit(case(fail=True))
    good = srv.submit(case())
    with pytest.raises(RuntimeError, match="planted"):
        bad.result(timeout=10)
    assert good.result(timeout=10).status == 0
    srv.close()
    assert srv.in_flight == 0


@pytest.mark.parametrize("batched", [False, True])
def test_warm_start_passes_the_last_x(fake_cuda, batched):
    srv = serve.ReplanServer(workers=1, warm_start=True, batched=batched)
    srv.submit(case(), patient="p1").result(timeout=10)
    srv.submit(case(), patient="p1").result(timeout=10)
    srv.submit(case(n=12), patient="p1").result(timeout=10)  # another beamlet count: cold start
    srv.close()
    (x0a, ia), (x0b, ib), (x0c, ic) = FakePlan.x0s
    assert x0a is None and x0c is None
    np.testing.assert_array_equal(x0b, np.full(10, 2.0, np.float32))
    assert ib == 2 and ic != 2


def test_requests_arriving_during_a_launch_join_the_next(fake_cuda):
    srv = serve.ReplanServer(workers=4, batched=True, hbm_fraction=1e6)
    futs = [srv.submit(case()) for _ in range(3)]
    time.sleep(0.02)
    futs += [srv.submit(case()) for _ in range(9)]
    res = [f.result(timeout=10) for f in futs]
    srv.close()
    assert sorted(r.request_id for r in res) == list(range(12))
    assert sum(BATCHES) == 12 and max(BATCHES) > 1
    assert srv.stats()["launches"] == len(BATCHES)
    assert max(r.batch for r in res) == max(BATCHES)


def test_resident_plans_are_rebuilt_in_place_and_evicted_lru(fake_cuda):
    srv = serve.ReplanServer(workers=1, batched=True, resident=True)
    srv.submit(case(), patient="a").result(timeout=10)
    srv.submit(case(), patient="a").result(timeout=10)  # the same plan, rebuilt
    assert FakePlan.created == 1 and FakePlan.updates == 1
    assert srv.in_flight == NEED // 2  # the resident plan's measured bytes stay reserved
    # more patients: b and c fit beside a (measured plans are half the estimate); d does not, so
    # the least recently used idle plan (a) is evicted
    srv.submit(case(), patient="b").result(timeout=10)
    srv.submit(case(), patient="c").result(timeout=10)
    assert FakePlan.live == 3
    srv.submit(case(), patient="d").result(timeout=10)
    assert FakePlan.live == 3 and "a" not in srv._residents
    assert srv.in_flight == 3 * (NEED // 2) <= srv.budget
    srv.close()
    assert FakePlan.created == 4
    assert FakePlan.live == 0
