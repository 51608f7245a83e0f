"""Re-planning server: continuous batching of plan requests on one GPU.

The paper's motivation is online adaptive re-planning: while the patient lies on the
couch, a new plan must be optimised for the day's anatomy (Sec. 1), and re-optimisation
starts from the original plan (Sec. 2.1). A request carries a patient's new
dose-deposition matrix D (and structures) and is answered with the optimised intensities
x and the dose z.

* Builders: W host threads, each with its own CUDA stream, admit the oldest waiting
  request when its device footprint fits the HBM budget and build its plan on the
  device: a patient's resident plan is rebuilt in place from the new D (plan_update, the
  memory stays with the patient), otherwise a plan is created. Building is
  stream-ordered and never stalls the plans being solved.
* Scheduler (batched form): one thread takes every plan that is ready and solves them
  all in one persistent launch of the team solver (plan_solve_batch): requests that
  arrived while the GPU was busy join the next launch, uneven plans share the GPU's
  CTAs, and every plan's result is the same as alone (the team solver's results do not
  depend on the batch). The sequential form solves each request on its builder thread
  as soon as it is built.
* Admission: a request reserves an estimate of its footprint (its patient's measured
  plan size when the patient is resident); once built, the reservation becomes the plan's
  measured device bytes (plan_info). Resident plans stay counted; the least recently
  used idle ones are evicted when a request does not fit.
* Warm start: a patient's last x seeds the next request (x_init = 2) when the beamlet
  count matches.
* Metrics: per request, time-to-plan = completion - arrival; p50 / p99 and plans per
  second over a run.
"""
from __future__ import annotations

import collections
import concurrent.futures
import dataclasses
import statistics
import threading
import time
from typing import Dict, List, Optional

import numpy as np

from . import _lib as L
from .api import Options, Plan, solve_batch


@dataclasses.dataclass
class ServeResult:
    request_id: int
    patient: Optional[str]
    x: np.ndarray
    z: Optional[np.ndarray]
    objective: float
    iterations: int
    status: int
    arrival: float
    start: float
    done: float
    batch: int = 1  # plans in the launch that solved this request
    x0: Optional[np.ndarray] = None  # the warm start used (None: the x_init rule)

    @property
    def time_to_plan(self) -> float:
        return self.done - self.arrival


def plan_footprint_bytes(m: int, n: int, nnz: int, precision: int) -> int:
    """Upper estimate of a plan's device memory before it exists (both FP32 copies of D, a reduced
    copy, 9 buffer sets of x / z / r, build temporaries); replaced by the measured size once built."""
    per_nnz = 8 * 1.05 + 8 + (8 if precision != L.FP32 else 0) + 12  # + build temporaries (CSR copy)
    m_pad = (m + 31) // 32 * 32
    return int(nnz * per_nnz + m_pad * (9 * 8 + 24) + n * 200 + (64 << 20))


class _Request:
    __slots__ = ("rid", "patient", "case", "arrival", "future", "reserved", "plan", "x0", "start")

    def __init__(self, rid, patient, case, arrival):
        self.rid, self.patient, self.case, self.arrival = rid, patient, case, arrival
        self.future = concurrent.futures.Future()
        self.reserved = 0
        self.plan = None
        self.x0 = None
        self.start = 0.0


class _Resident:
    __slots__ = ("plan", "bytes", "x", "busy", "last_used")

    def __init__(self, plan, nbytes):
        self.plan, self.bytes, self.x, self.busy, self.last_used = plan, nbytes, None, True, 0.0


class ReplanServer:
    """Continuous-batching plan server (see the module docstring).

    workers: builder threads; batched: one scheduler launches all ready plans together (default
    when options.solver is the team solver); resident: keep each patient's plan on the device
    and rebuild it in place for the patient's next request."""

    def __init__(self, workers: int = 4, options: Optional[Options] = None, hbm_fraction: float = 0.8,
                 warm_start: bool = False, device: int = 0, batched: Optional[bool] = None,
                 resident: bool = False, want_dose: bool = True, max_batch: int = 1024):
        import torch
        torch.cuda.set_device(device)
        self.options = options or Options()
        self.batched = (self.options.solver == L.SOLVER_TEAM) if batched is None else batched
        self.warm_start, self.resident, self.want_dose, self.max_batch = warm_start, resident, want_dose, max_batch
        free, total = torch.cuda.mem_get_info(device)
        self.budget = int(hbm_fraction * free)
        self.in_flight = 0          # reserved bytes: requests being built or solved, and resident plans
        self.peak_in_flight = 0
        self.launches = 0
        self._cv = threading.Condition()
        self._pending: List[_Request] = []
        self._ready: List[_Request] = []
        self._building = 0
        self._closed = False
        self._next_id = 0
        self._last_x: Dict[str, np.ndarray] = {}
        self._residents: "collections.OrderedDict[str, _Resident]" = collections.OrderedDict()
        self._active = set()  # patients with a request being built or solved
        self._results: List[ServeResult] = []
        self._streams = [torch.cuda.Stream(device=device) for _ in range(workers + 1)]
        self._threads = [threading.Thread(target=self._builder, args=(i,), daemon=True) for i in range(workers)]
        if self.batched:
            self._threads.append(threading.Thread(target=self._scheduler, daemon=True))
        for t in self._threads:
            t.start()

    # -- client side -------------------------------------------------------
    def submit(self, case, patient: Optional[str] = None) -> concurrent.futures.Future:
        """Queues one request (a phantom.Case or any object with the same arrays)."""
        need = plan_footprint_bytes(case.m, case.n, case.nnz, self.options.precision)
        if need > self.budget:
            raise ValueError(f"request needs ~{need} bytes, more than the HBM budget {self.budget}")
        with self._cv:
            req = _Request(self._next_id, patient, case, time.perf_counter())
            self._next_id += 1
            self._pending.append(req)
            self._cv.notify_all()
        return req.future

    def close(self) -> None:
        with self._cv:
            self._closed = True
            self._cv.notify_all()
        for t in self._threads:
            t.join()
        for r in self._residents.values():
            r.plan.close()
        self._residents.clear()

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
                "launches": self.launches, "mean_batch": statistics.mean(r.batch for r in res),
                "failed": sum(1 for r in res if r.status != 0),
                "failed_status": sorted({L.STATUS_NAMES.get(r.status, r.status) for r in res if r.status != 0})}

    # -- admission ---------------------------------------------------------
    def _estimate(self, req: _Request) -> int:
        r = self._residents.get(req.patient) if req.patient is not None else None
        if r is not None:  # rebuilt in place: only growth beyond its measured size is new
            est = plan_footprint_bytes(req.case.m, req.case.n, req.case.nnz, self.options.precision)
            return max(0, min(est, 2 * r.bytes) - r.bytes)
        return plan_footprint_bytes(req.case.m, req.case.n, req.case.nnz, self.options.precision)

    def _evict_for(self, need: int, keep: Optional[str]) -> None:
        """Destroys idle resident plans, least recently used first, until `need` bytes fit."""
        for pid in list(self._residents):
            if self.in_flight + need <= self.budget:
                return
            r = self._residents[pid]
            if r.busy or pid == keep:
                continue
            r.plan.close()
            self.in_flight -= r.bytes
            del self._residents[pid]

    def _admit(self) -> Optional[_Request]:
        """The oldest waiting request that can start: its patient has no request in progress
        (requests of one patient keep their order, so warm starts follow it) and its footprint
        fits the budget, after evicting idle resident plans if needed. A request that does not
        fit holds back the ones behind it (no overtaking on memory)."""
        with self._cv:
            while True:
                blocked = set()
                for idx, req in enumerate(self._pending):
                    if req.patient is not None and (req.patient in blocked or req.patient in self._active):
                        blocked.add(req.patient)
                        continue
                    res = self._residents.get(req.patient) if req.patient is not None else None
                    need = self._estimate(req)
                    if self.in_flight + need > self.budget:
                        self._evict_for(need, req.patient)
                    if self.in_flight + need > self.budget:
                        break
                    self._pending.pop(idx)
                    self.in_flight += need
                    self.peak_in_flight = max(self.peak_in_flight, self.in_flight)
                    req.reserved = need
                    if res is not None:
                        res.busy = True
                    if req.patient is not None:
                        self._active.add(req.patient)
                    self._building += 1
                    return req
                if self._closed and not self._pending:
                    return None
                self._cv.wait(timeout=0.05)

    # -- building ----------------------------------------------------------
    def _build(self, req: _Request, stream) -> None:
        c = req.case
        opts = dataclasses.replace(self.options, stream=stream.cuda_stream)
        x0 = None
        if self.warm_start and req.patient is not None and req.patient in self._last_x:
            x0 = self._last_x[req.patient]
            if x0.shape[0] != c.n:
                x0 = None
        opts = dataclasses.replace(opts, x_init=2 if x0 is not None else self.options.x_init)
        res = self._residents.get(req.patient) if (self.resident and req.patient is not None) else None
        if res is not None:
            res.plan.update(c.row_ptr, c.col, c.val, c.mask, c.thresholds, c.weights, m=c.m, n=c.n)
            res.plan.set_options(**{f.name: getattr(opts, f.name) for f in dataclasses.fields(opts)})
            plan = res.plan
        else:
            plan = Plan(c.row_ptr, c.col, c.val, c.mask, c.thresholds, c.weights, m=c.m, n=c.n, options=opts)
        measured = int(plan.info()["device_bytes"])
        with self._cv:
            if res is not None:  # the resident's bytes were already counted
                self.in_flight += measured - res.bytes - req.reserved
                res.bytes = measured
            else:
                self.in_flight += measured - req.reserved
                if self.resident and req.patient is not None:
                    self._residents[req.patient] = _Resident(plan, measured)
                    self._residents.move_to_end(req.patient)
            self.peak_in_flight = max(self.peak_in_flight, self.in_flight)
            req.reserved = 0 if (self.resident and req.patient is not None) else measured
        req.plan, req.x0 = plan, x0

    def _finish(self, req: _Request, objective: float, iterations: int, status: int, launch: int) -> None:
        plan = req.plan
        x = plan.get_x()
        z = plan.dose(x) if self.want_dose else None
        done = time.perf_counter()
        out = ServeResult(req.rid, req.patient, x, z, objective, iterations, status, req.arrival, req.start, done,
                          launch, req.x0)
        with self._cv:
            if req.patient is not None:
                self._last_x[req.patient] = x
                self._active.discard(req.patient)
                self._cv.notify_all()
            r = self._residents.get(req.patient) if req.patient is not None else None
            if r is not None and r.plan is plan:
                r.busy = False
                r.last_used = done
                self._residents.move_to_end(req.patient)
            self._results.append(out)
        if r is None or r.plan is not plan:
            plan.close()
            self._release(req)
        req.future.set_result(out)

    def _release(self, req: _Request) -> None:
        with self._cv:
            self.in_flight -= req.reserved
            req.reserved = 0
            self._cv.notify_all()

    def _fail(self, req: _Request, exc: BaseException) -> None:
        with self._cv:
            if req.patient is not None:
                self._active.discard(req.patient)
            r = self._residents.get(req.patient) if req.patient is not None else None
            if r is not None and (req.plan is None or r.plan is req.plan):  # drop a half-rebuilt resident
                r.plan.close()
                self.in_flight -= r.bytes
                del self._residents[req.patient]
            elif req.plan is not None:
                req.plan.close()
        self._release(req)
        req.future.set_exception(exc)

    def _builder(self, index: int) -> None:
        stream = self._streams[index]
        while True:
            req = self._admit()
            if req is None:
                return
            req.start = time.perf_counter()
            try:
                self._build(req, stream)
            except BaseException as e:  # a failed request must not take the worker down
                with self._cv:
                    self._building -= 1
                    self._cv.notify_all()
                self._fail(req, e)
                continue
            if self.batched:
                with self._cv:
                    self._building -= 1
                    self._ready.append(req)
                    self._cv.notify_all()
                continue
            try:
                r = req.plan.solve(x0=req.x0, raise_on_error=False)
                with self._cv:
                    self._building -= 1
                    self.launches += 1
                self._finish(req, r.objective, r.iterations, r.status, 1)
            except BaseException as e:
                with self._cv:
                    self._building -= 1
                self._fail(req, e)

    # -- batched solving ---------------------------------------------------
    def _scheduler(self) -> None:
        stream = self._streams[-1]
        while True:
            with self._cv:
                while not self._ready and not (self._closed and not self._pending and not self._building):
                    self._cv.wait(timeout=0.05)
                if not self._ready:
                    return
                batch, self._ready = self._ready[:self.max_batch], self._ready[self.max_batch:]
                self.launches += 1
            try:
                res = solve_batch([r.plan for r in batch], x0s=[r.x0 for r in batch], stream=stream.cuda_stream,
                                  raise_on_error=False)
            except BaseException as e:
                for r in batch:
                    self._fail(r, e)
                continue
            for r, rr in zip(batch, res):
                try:
                    self._finish(r, rr.objective, rr.iterations, rr.status, len(batch))
                except BaseException as e:
                    self._fail(r, e)


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


FORMS = {
    # the plain FP32 solver, one request after another
    "sequential_fp32": dict(workers=1, batched=False, options=Options()),
    # mixed precision (FP16 D, FP32 polish) in the team solver with continuous batching
    "batched_fp16": dict(workers=4, batched=True, resident=True, options=Options(precision=L.FP16,
                                                                                   solver=L.SOLVER_TEAM)),
}


def run_stream(form: str, cases, rate_hz: float, seed: int = 0, patients=None, warm_start: bool = False) -> dict:
    """One Poisson stream through one serving form; returns its stats."""
    kw = dict(FORMS[form])
    srv = ReplanServer(warm_start=warm_start, **kw)
    try:
        futs = poisson_stream(srv, cases, rate_hz, seed=seed, patients=patients)
        concurrent.futures.wait(futs)
    finally:
        srv.close()
    return srv.stats()


def _main():
    """Serving benchmark: Poisson arrivals of re-planning requests (PTV shifted by up to +-5 mm,
    D regenerated), sequential plain FP32 solves against the batched mixed-precision form."""
    import argparse
    import json

    from . import phantom
    ap = argparse.ArgumentParser()
    ap.add_argument("--requests", type=int, default=1000)
    ap.add_argument("--rates", default="2,20,200")
    ap.add_argument("--seed", type=int, default=0)
    args = ap.parse_args()
    specs = [phantom.jittered_spec(args.seed * 100000 + i, shift_mm=5.0, vary=False) for i in range(args.requests)]
    cases = [phantom.make_case(s) for s in specs]
    patients = [f"patient{i % 50}" for i in range(args.requests)]
    out = {}
    for rate in [float(r) for r in args.rates.split(",")]:
        for form in FORMS:
            out[f"{form}@{rate:g}Hz"] = run_stream(form, cases, rate, seed=args.seed, patients=patients)
    print(json.dumps({"metric": "re-plan time-to-plan", "unit": "s", "requests": args.requests, **out}))


if __name__ == "__main__":
    _main()
