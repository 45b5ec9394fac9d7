"""Request loop for HFX force/stress evaluations (serving).

A seeded stream of structures arrives as a Poisson process; each structure
is a relaxation-like driver that issues `steps` evaluations one after the
other (step k + 1 is issued as soon as step k's result is back, its
positions moved by a small seeded displacement).  The server

  * keeps one device-resident plan per active structure: its templates, D,
    pair lists and operand stores stay on the device across the structure's
    steps and are freed after its last step;
  * admits structures in arrival order while the device bytes of the
    resident plans plus the new structure's estimate stay within an HBM
    budget (a structure whose estimate alone exceeds the budget is
    rejected); the estimate is refined from the measured plan sizes of the
    shapes already seen;
  * runs the requests of the admitted structures on `workers` host threads,
    each plan on its own CUDA stream, so that evaluations of different
    structures overlap on the GPU;
  * records per request its arrival (issue time), start and end, and
    reports throughput with p50 / p99 latency (issue -> result on the host)
    and the admission wait;
  * optionally re-evaluates a sample of requests alone, on a fresh plan of
    the same structure, after the stream has drained, and reports the
    largest relative difference to the in-the-mix result (only the order of
    the FP64 atomic additions differs between the two).

Every evaluation runs through the C ABI (hfx.Plan); this module only
schedules.  The scheduling logic takes a backend object, so that it can be
tested on the CPU with a stand-in.
"""
from __future__ import annotations

import argparse
import collections
import dataclasses
import heapq
import json
import threading
import time
from typing import Callable, Dict, List, Optional

import numpy as np

from . import inputs

# shapes a request may carry: name -> (generator, n_rep)
SHAPES: Dict[str, Callable] = {
    "si8": lambda seed, strain: inputs.si_supercell(1, seed=seed, strain_amp=strain),
    "si64": lambda seed, strain: inputs.si_supercell(2, seed=seed, strain_amp=strain),
    "si216": lambda seed, strain: inputs.si_supercell(3, seed=seed, strain_amp=strain),
    "si512": lambda seed, strain: inputs.si_supercell(4, seed=seed, strain_amp=strain),
    "si1000": lambda seed, strain: inputs.si_supercell(5, seed=seed, strain_amp=strain),
    "perovskite5": lambda seed, strain: inputs.perovskite_supercell(1, seed=seed, strain_amp=strain),
    "perovskite40": lambda seed, strain: inputs.perovskite_supercell(2, seed=seed, strain_amp=strain),
    "perovskite135": lambda seed, strain: inputs.perovskite_supercell(3, seed=seed, strain_amp=strain),
    "perovskite320": lambda seed, strain: inputs.perovskite_supercell(4, seed=seed, strain_amp=strain),
}


@dataclasses.dataclass
class Structure:
    sid: int
    shape: str
    arrival: float                # seconds after the start of the stream
    workload: object              # an inputs.Workload (or any object the backend accepts)
    geoms: List[np.ndarray]       # positions of its steps


@dataclasses.dataclass
class Record:
    sid: int
    shape: str
    step: int
    precision: str
    issued: float
    start: float
    end: float
    plan_ms: float                # plan creation inside this request (first step only)
    result: Optional[tuple] = None
    device: Optional[tuple] = None   # (start, end) of its GPU work in s on the server's device clock

    @property
    def latency(self) -> float:
        return self.end - self.issued


def make_stream(seed: int, rate: float, n_structures: int, shapes: List[str], steps: int,
                strain: float = 0.03, make: Optional[Callable] = None) -> List[Structure]:
    """Seeded Poisson arrivals (mean `rate` structures per second), shapes
    drawn uniformly from `shapes`; each structure gets its own workload seed,
    a random strain of amplitude `strain` and `steps` geometries 0.01 A apart
    (jitter per step)."""
    rng = np.random.Generator(np.random.Philox(seed))
    make = make or (lambda shape, s: SHAPES[shape](s, strain))
    t = 0.0
    out = []
    for sid in range(n_structures):
        t += rng.exponential(1.0 / rate)
        shape = shapes[int(rng.integers(len(shapes)))]
        w = make(shape, seed * 1000 + sid)
        geoms = inputs.geometry_sequence(w, steps, seed=seed * 1000 + sid)
        out.append(Structure(sid, shape, t, w, geoms))
    return out


class Server:
    """Admission, per-structure plans and worker threads (see the module
    docstring).  `backend` provides create(structure) -> plan (with
    .evaluate(lattice, positions) -> (E, F, sigma), .device_bytes(), .close()
    and .precision), and estimate_bytes(structure, known) -> bytes."""

    def __init__(self, backend, budget_bytes: float, workers: int = 4, keep_results: bool = True):
        self.backend = backend
        self.budget = float(budget_bytes)
        self.workers = int(workers)
        self.keep_results = keep_results

    def run(self, structures: List[Structure]) -> dict:
        arrivals = sorted(structures, key=lambda s: s.arrival)
        cond = threading.Condition()
        ready: List[tuple] = []          # heap of (issued, seq, structure, step)
        seq = [0]
        known: Dict[str, float] = {}      # measured plan bytes per shape
        resident: Dict[int, float] = {}   # admitted sid -> bytes accounted
        plans: Dict[int, object] = {}
        records: List[Record] = []
        admitted_at: Dict[int, float] = {}
        rejected: List[int] = []
        peak = [0.0]
        done = [0]
        errors: List[str] = []
        n_total = sum(len(s.geoms) for s in structures)
        t0 = time.perf_counter()
        clock = lambda: time.perf_counter() - t0

        def push(item):
            heapq.heappush(ready, (item[0], seq[0]) + item[1:])
            seq[0] += 1

        def worker():
            while True:
                with cond:
                    while not ready and done[0] < n_total and not errors:
                        cond.wait(0.05)
                    if done[0] >= n_total or errors:
                        return
                    issued, _, s, k = heapq.heappop(ready)
                start = clock()
                plan_ms = 0.0
                try:
                    if k == 0:
                        tp = time.perf_counter()
                        plans[s.sid] = self.backend.create(s)
                        plan_ms = (time.perf_counter() - tp) * 1e3
                    plan = plans[s.sid]
                    res = plan.evaluate(s.workload.lattice, s.geoms[k])
                    dev_iv = plan.last_device_interval() if hasattr(plan, "last_device_interval") else None
                except Exception as e:   # a failed request ends the run with its message
                    with cond:
                        errors.append(f"structure {s.sid} step {k}: {e}")
                        cond.notify_all()
                    return
                end = clock()
                rec = Record(s.sid, s.shape, k, plan.precision, issued, start, end, plan_ms,
                             res if self.keep_results else None, dev_iv)
                last = k + 1 == len(s.geoms)
                if k == 0:
                    b = float(plan.device_bytes())
                    with cond:
                        known[s.shape] = max(known.get(s.shape, 0.0), b)
                        resident[s.sid] = b     # the measured size replaces the estimate
                        peak[0] = max(peak[0], sum(resident.values()))
                if last:
                    plan.close()
                    del plans[s.sid]
                with cond:
                    records.append(rec)
                    done[0] += 1
                    if last:
                        resident.pop(s.sid, None)
                    else:
                        push((end, s, k + 1))   # the driver issues its next step at once
                    cond.notify_all()

        threads = [threading.Thread(target=worker, daemon=True) for _ in range(self.workers)]
        for t in threads:
            t.start()
        waiting = collections.deque()
        i = 0
        with cond:
            while done[0] < n_total and not errors:
                now = clock()
                while i < len(arrivals) and arrivals[i].arrival <= now:
                    waiting.append(arrivals[i])
                    i += 1
                # admission in arrival order within the budget
                while waiting:
                    s = waiting[0]
                    est = float(self.backend.estimate_bytes(s, known))
                    if est > self.budget:
                        waiting.popleft()
                        rejected.append(s.sid)
                        n_total -= len(s.geoms)
                        continue
                    if resident and sum(resident.values()) + est > self.budget:
                        break
                    waiting.popleft()
                    resident[s.sid] = est
                    peak[0] = max(peak[0], sum(resident.values()))
                    admitted_at[s.sid] = now
                    push((s.arrival, s, 0))
                    cond.notify_all()
                nxt = arrivals[i].arrival - now if i < len(arrivals) else 0.05
                cond.wait(max(1e-4, min(nxt, 0.05)))
            cond.notify_all()
        for t in threads:
            t.join()
        if errors:
            raise RuntimeError(errors[0])
        makespan = max((r.end for r in records), default=0.0)
        return {"records": records, "makespan": makespan, "rejected": rejected, "peak_bytes": peak[0],
                "admission_wait": {sid: admitted_at[sid] - next(s.arrival for s in structures if s.sid == sid)
                                   for sid in admitted_at}, "known_bytes": known}


def device_overlap(records: List[Record]) -> Optional[dict]:
    """Concurrency of the requests' GPU work, from their device intervals:
    the sum of the intervals over the time the GPU had at least one request
    in flight (1 = no overlap; k = k requests in flight on average while
    busy)."""
    iv = sorted(r.device for r in records if r.device is not None)
    if not iv:
        return None
    union, cur_s, cur_e = 0.0, iv[0][0], iv[0][1]
    for s, e in iv[1:]:
        if s > cur_e:
            union += cur_e - cur_s
            cur_s, cur_e = s, e
        else:
            cur_e = max(cur_e, e)
    union += cur_e - cur_s
    total = sum(e - s for s, e in iv)
    return {"busy_s": union, "sum_of_request_device_s": total, "mean_requests_in_flight": total / union
            if union > 0 else 0.0, "first_start_s": iv[0][0], "last_end_s": max(e for _, e in iv)}


def summarize(out: dict, structures: List[Structure]) -> dict:
    recs: List[Record] = out["records"]
    lat = np.array([r.latency for r in recs]) * 1e3
    by_shape = {}
    for shape in sorted({r.shape for r in recs}):
        ls = np.array([r.latency for r in recs if r.shape == shape]) * 1e3
        ev = np.array([r.end - r.start - r.plan_ms / 1e3 for r in recs if r.shape == shape]) * 1e3
        by_shape[shape] = {"requests": int(ls.size), "p50_ms": float(np.percentile(ls, 50)),
                           "p99_ms": float(np.percentile(ls, 99)), "eval_ms_median": float(np.median(ev)),
                           "precision": sorted({r.precision for r in recs if r.shape == shape})}
    waits = np.array(list(out["admission_wait"].values())) * 1e3 if out["admission_wait"] else np.zeros(1)
    span = out["makespan"]
    last_arrival = max(s.arrival for s in structures) if structures else 0.0
    ov = device_overlap(recs)
    served = {r.sid for r in recs}
    return {"requests": len(recs), "structures": len(structures), "rejected": len(out["rejected"]),
            "makespan_s": span, "last_arrival_s": last_arrival,
            "throughput_req_s": len(recs) / span if span > 0 else 0.0,
            "device_overlap": ov,
            # the arrival rate this mix of shapes can be served at: the served
            # structures over the time the GPU was busy with them (above it the
            # queue grows without bound)
            "sustainable_structures_per_s": len(served) / ov["busy_s"] if ov and ov["busy_s"] > 0 else None,
            "p50_ms": float(np.percentile(lat, 50)) if lat.size else None,
            "p99_ms": float(np.percentile(lat, 99)) if lat.size else None,
            "admission_wait_ms_p50": float(np.percentile(waits, 50)),
            "admission_wait_ms_max": float(waits.max()),
            "peak_resident_gb": out["peak_bytes"] / 1e9, "by_shape": by_shape}


def rel_diff(a: tuple, b: tuple) -> float:
    """Largest of |dE|/|E|, max|dF|/max|F|, max|dsigma|/max|sigma|."""
    out = abs(a[0] - b[0]) / max(abs(b[0]), 1e-300)
    for x, y in ((a[1], b[1]), (a[2], b[2])):
        x, y = np.asarray(x, float), np.asarray(y, float)
        out = max(out, float(np.max(np.abs(x - y)) / max(np.max(np.abs(y)), 1e-300)))
    return out


def alone_vs_mix(backend, structures: List[Structure], records: List[Record], n_check: int) -> float:
    """Re-evaluate up to n_check requests alone (a fresh plan of the same
    structure, the GPU otherwise idle) and return the largest relative
    difference to the results they had in the mix."""
    by_sid = {s.sid: s for s in structures}
    worst = 0.0
    for r in sorted(records, key=lambda r: (r.sid, r.step))[::max(1, len(records) // max(1, n_check))][:n_check]:
        s = by_sid[r.sid]
        plan = backend.create(s)
        try:
            res = plan.evaluate(s.workload.lattice, s.geoms[r.step])
        finally:
            plan.close()
        worst = max(worst, rel_diff(res, r.result))
    return worst


class GpuBackend:
    """Plans through the C ABI, one CUDA stream per plan, every shape in the
    requested precision (shapes with n_ao > 16, the perovskite Cs blocks, take
    the library's wide split-precision kernels)."""

    # device bytes per atom before any plan of a shape has been measured
    # (si64: 139 MB per atom in FP64, 367 MB with BF16X6); refined online
    DEFAULT_BYTES_PER_ATOM = {"fp64": 1.6e8, "bf16x3": 3.0e8, "bf16x6": 4.0e8}

    def __init__(self, precision: str, device: int = 0):
        import torch
        from . import hfx
        self.torch, self.hfx = torch, hfx
        self.precision = precision
        self.code = {"fp64": hfx.HFX_FP64, "bf16x3": hfx.HFX_BF16X3, "bf16x6": hfx.HFX_BF16X6}[precision]
        self.device = device
        self.clock0 = _DeviceClock(torch, device)

    def estimate_bytes(self, s: Structure, known: Dict[str, float]) -> float:
        if s.shape in known:
            return known[s.shape]
        n = len(s.workload.species)
        return n * self.DEFAULT_BYTES_PER_ATOM[self.precision]

    def create(self, s: Structure):
        torch, hfx = self.torch, self.hfx
        stream = torch.cuda.Stream(device=self.device)
        code, name = self.code, self.precision
        plan = hfx.Plan(s.workload, precision=code, stream=stream.cuda_stream, device=self.device)
        return _GpuPlan(plan, stream, name, self.clock0)


class _DeviceClock:
    """A CUDA event recorded once on the device: the time origin of every
    request's device interval (elapsed time between events of different
    streams of one device is well defined)."""

    def __init__(self, torch, device):
        self.torch = torch
        with torch.cuda.device(device):
            self.e = torch.cuda.Event(enable_timing=True)
            self.e.record(torch.cuda.current_stream(device))
            self.e.synchronize()

    def since(self, ev) -> float:
        return self.e.elapsed_time(ev) / 1e3


class _GpuPlan:
    def __init__(self, plan, stream, precision, clock0):
        self.plan, self.stream, self.precision = plan, stream, precision
        self._bytes = None
        self._clock0 = clock0
        self._iv = None

    def evaluate(self, lattice, positions):
        torch = self._clock0.torch
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(self.stream)
        E, F, S = self.plan.evaluate(lattice, positions, stats=self._bytes is None)
        e1.record(self.stream)
        e1.synchronize()
        self._iv = (self._clock0.since(e0), self._clock0.since(e1))
        if self._bytes is None:
            self._bytes = int(self.plan.stats.device_bytes)
        return E, F, S

    def last_device_interval(self):
        """(start, end) of the last evaluation's GPU work, in s on the device
        clock shared by every plan of the backend."""
        return self._iv

    def device_bytes(self) -> int:
        return self._bytes or 0

    def close(self):
        self.plan.close()


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--rate", type=float, default=20.0, help="structure arrivals per second (Poisson)")
    ap.add_argument("--structures", type=int, default=40)
    ap.add_argument("--steps", type=int, default=5, help="relaxation steps (requests) per structure")
    ap.add_argument("--shapes", default="si8,si64,perovskite5,perovskite40")
    ap.add_argument("--precision", default="bf16x6", choices=["bf16x6", "bf16x3", "fp64"])
    ap.add_argument("--workers", type=int, default=4)
    ap.add_argument("--budget-gb", type=float, default=200.0)
    ap.add_argument("--check", type=int, default=8, help="requests re-evaluated alone after the stream")
    ap.add_argument("--seed", type=int, default=7)
    args = ap.parse_args(argv)
    import torch
    if not torch.cuda.is_available():
        raise SystemExit("serving needs a CUDA GPU")
    free, _ = torch.cuda.mem_get_info()
    budget = min(args.budget_gb * 1e9, 0.85 * free)
    t = time.perf_counter()
    structures = make_stream(args.seed, args.rate, args.structures, args.shapes.split(","), args.steps)
    gen_s = time.perf_counter() - t
    backend = GpuBackend(args.precision)
    out = Server(backend, budget, args.workers).run(structures)
    summ = summarize(out, structures)
    summ.update({"precision": args.precision, "rate_structures_per_s": args.rate, "steps": args.steps,
                 "workers": args.workers, "budget_gb": budget / 1e9, "shapes": args.shapes.split(","),
                 "seed": args.seed, "input_generation_s": gen_s,
                 "latency": "issue of a request (arrival, or the previous step's result) -> its result on the host"})
    if args.check > 0:
        summ["alone_vs_mix_max_rel_diff"] = alone_vs_mix(backend, structures, out["records"], args.check)
        summ["alone_vs_mix_checked"] = min(args.check, len(out["records"]))
    print(json.dumps(summ))
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
