"""Re-planning server: continuous batching of plan requests on one GPU.

The paper's motivation is online adaptive re-planning: while the patient lies on
the couch, a new plan must be optimised for the day's anatomy (Sec. 1). Here a
request carries a patient's new dose-deposition matrix D (and structures) and is
answered with the optimised intensities x and the dose z.

* Workers: W host threads, each with its own CUDA stream. A worker takes the
  oldest admitted request, creates the plan from the request's host arrays
  (plan_create copies D to the device and builds its layouts there), solves it
  (plan_solve: one CUDA graph with the Armijo controller on the device), reads x
  and z back, and destroys the plan. Requests that arrive while others are on
  the GPU start as soon as a worker and device memory are free, and their
  kernels run concurrently with the others' on the device (one stream each).
  Plan creation and destruction are stream-ordered, so they never stall the
  other requests' work.
* Admission: a request's device footprint is estimated from its size before it
  is created; it is admitted while the in-flight total stays under the HBM
  budget (a fraction, 0.8 by default, of the memory free when the server
  starts). Requests wait in arrival order.
* Resident state: a patient's last solution is kept and seeds its next request
  (x_init = 2) when `warm_start` is on.
* Metrics: per request, time-to-plan = completion - arrival; p50 / p99 and
  plans per second over a run.

The kernels are deterministic (fixed reduction orders, schedule-independent
partials), so a request's result is the same alone and in the mix.
"""
from __future__ import annotations

import concurrent.futures
import dataclasses
import queue
import statistics
import threading
import time
from typing import Dict, List, Optional

import numpy as np

from . import _lib as L
from .api import Options, Plan


@dataclasses.dataclass
class ServeResult:
    request_id: int
    patient: Optional[str]
    x: np.ndarray
    z: np.ndarray
    objective: float
    iterations: int
    status: int
    arrival: float
    start: float
    done: float

    @property
    def time_to_plan(self) -> float:
        return self.done - self.arrival


def plan_footprint_bytes(m: int, n: int, nnz: int, precision: int) -> int:
    """Upper estimate of a plan's device memory (both FP32 copies of D, a reduced copy,
    9 buffer sets of x / z / r, build temporaries), used for admission."""
    per_nnz = 8 * 1.05 + 8 + (8 if precision != L.FP32 else 0) + 12  # + build temporaries (CSR copy)
    m_pad = (m + 31) // 32 * 32
    return int(nnz * per_nnz + m_pad * (9 * 8 + 24) + n * 200 + (64 << 20))


class _Request:
    __slots__ = ("rid", "patient", "case", "arrival", "future", "bytes")

    def __init__(self, rid, patient, case, arrival, bytes_):
        self.rid, self.patient, self.case, self.arrival = rid, patient, case, arrival
        self.future = concurrent.futures.Future()
        self.bytes = bytes_


class ReplanServer:
    """Continuous-batching plan server (see the module docstring)."""

    def __init__(self, workers: int = 4, options: Optional[Options] = None, hbm_fraction: float = 0.8,
                 warm_start: bool = False, device: int = 0):
        import torch
        torch.cuda.set_device(device)
        self.options = options or Options()
        self.warm_start = warm_start
        free, total = torch.cuda.mem_get_info(device)
        self.budget = int(hbm_fraction * free)
        self.in_flight = 0
        self.peak_in_flight = 0
        self._cv = threading.Condition()
        self._pending: List[_Request] = []
        self._closed = False
        self._next_id = 0
        self._last_x: Dict[str, np.ndarray] = {}
        self._results: List[ServeResult] = []
        self._streams = [torch.cuda.Stream(device=device) for _ in range(workers)]
        self._threads = [threading.Thread(target=self._worker, args=(i,), daemon=True) for i in range(workers)]
        for t in self._threads:
            t.start()

    # -- client side -------------------------------------------------------
    def submit(self, case, patient: Optional[str] = None) -> concurrent.futures.Future:
        """Queues one request (a phantom.Case or any object with the same arrays)."""
        need = plan_footprint_bytes(case.m, case.n, case.nnz, self.options.precision)
        if need > self.budget:
            raise ValueError(f"request needs ~{need} bytes, more than the HBM budget {self.budget}")
        with self._cv:
            rid = self._next_id
            self._next_id += 1
            req = _Request(rid, patient, case, time.perf_counter(), need)
            self._pending.append(req)
            self._cv.notify_all()
        return req.future

    def close(self) -> None:
        with self._cv:
            self._closed = True
            self._cv.notify_all()
        for t in self._threads:
            t.join()

    def results(self) -> List[ServeResult]:
        return list(self._results)

    def stats(self, results: Optional[List[ServeResult]] = None) -> dict:
        res = results if results is not None else self._results
        if not res:
            return {"n": 0}
        lat = sorted(r.time_to_plan for r in res)
        span = max(r.done for r in res) - min(r.arrival for r in res)
        return {"n": len(res), "p50_s": lat[len(lat) // 2], "p99_s": lat[min(len(lat) - 1, int(0.99 * len(lat)))],
                "mean_s": statistics.mean(lat), "plans_per_s": len(res) / span if span > 0 else float("nan"),
                "peak_in_flight_bytes": self.peak_in_flight, "budget_bytes": self.budget,
                "failed": sum(1 for r in res if r.status != 0)}

    # -- server side -------------------------------------------------------
    def _admit(self) -> Optional[_Request]:
        with self._cv:
            while True:
                if self._pending:
                    req = self._pending[0]
                    if self.in_flight + req.bytes <= self.budget:
                        self._pending.pop(0)
                        self.in_flight += req.bytes
                        self.peak_in_flight = max(self.peak_in_flight, self.in_flight)
                        return req
                elif self._closed:
                    return None
                self._cv.wait(timeout=0.05)

    def _release(self, req: _Request) -> None:
        with self._cv:
            self.in_flight -= req.bytes
            self._cv.notify_all()

    def _worker(self, index: int) -> None:
        import torch
        stream = self._streams[index]
        while True:
            req = self._admit()
            if req is None:
                return
            start = time.perf_counter()
            try:
                opts = dataclasses.replace(self.options, stream=stream.cuda_stream)
                x0 = None
                if self.warm_start and req.patient is not None and req.patient in self._last_x:
                    x0 = self._last_x[req.patient]
                    if x0.shape[0] != req.case.n:
                        x0 = None
                if x0 is not None:
                    opts = dataclasses.replace(opts, x_init=2)
                c = req.case
                with Plan(c.row_ptr, c.col, c.val, c.mask, c.thresholds, c.weights, m=c.m, n=c.n,
                          options=opts) as plan:
                    res = plan.solve(x0=x0, raise_on_error=False)
                    x = plan.get_x()
                    z = plan.dose(x)
                done = time.perf_counter()
                if req.patient is not None:
                    self._last_x[req.patient] = x
                out = ServeResult(req.rid, req.patient, x, z, res.objective, res.iterations, res.status,
                                  req.arrival, start, done)
                self._results.append(out)
                req.future.set_result(out)
            except BaseException as e:  # a failed request must not take the worker down
                req.future.set_exception(e)
            finally:
                self._release(req)


def poisson_stream(server: ReplanServer, cases, rate_hz: float, seed: int = 0, patients=None):
    """Submits `cases` with exponential inter-arrival times (mean 1/rate_hz); returns the futures."""
    rng = np.random.Generator(np.random.PCG64(seed))
    futures = []
    t_next = time.perf_counter()
    for i, c in enumerate(cases):
        t_next += float(rng.exponential(1.0 / rate_hz))
        delay = t_next - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        futures.append(server.submit(c, patient=None if patients is None else patients[i]))
    return futures


def _main():
    """Serving benchmark: Poisson arrivals of re-planning requests (PTV shifted by up to
    +-5 mm, D regenerated), sequential FP32 solves against the concurrent FP16 form."""
    import argparse
    import json

    from . import phantom
    ap = argparse.ArgumentParser()
    ap.add_argument("--requests", type=int, default=1000)
    ap.add_argument("--rate", type=float, default=20.0)
    ap.add_argument("--workers", type=int, default=8)
    ap.add_argument("--seed", type=int, default=0)
    args = ap.parse_args()
    # requests: the tiny-phantom geometry with the PTV shifted, D regenerated per request
    specs = [phantom.jittered_spec(args.seed * 100000 + i, shift_mm=5.0, vary=False) for i in range(args.requests)]
    cases = [phantom.make_case(s) for s in specs]
    out = {}
    for name, workers, prec in (("sequential_fp32", 1, L.FP32), ("concurrent_fp16", args.workers, L.FP16)):
        srv = ReplanServer(workers=workers, options=Options(precision=prec))
        fut = poisson_stream(srv, cases, args.rate, seed=args.seed)
        concurrent.futures.wait(fut)
        srv.close()
        out[name] = srv.stats()
    print(json.dumps({"metric": "re-plan time-to-plan", "unit": "s", "requests": args.requests,
                      "rate_hz": args.rate, "workers": args.workers, **out}))


if __name__ == "__main__":
    _main()
