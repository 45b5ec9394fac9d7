"""Serving loop (paper_2412_11081_gb300/serve.py): scheduling, admission and
latency bookkeeping with a stand-in backend on the CPU, and one short
stream on the GPU through the C ABI with the alone-vs-in-the-mix check."""
import threading
import time
import types

import numpy as np
import pytest

from paper_2412_11081_gb300 import serve


class FakePlan:
    """Stands in for a device plan: sleeps for a size-dependent time and
    returns a deterministic result of the geometry; records concurrency."""

    def __init__(self, backend, s):
        self.backend, self.s = backend, s
        self.precision = "fake"
        self.steps_seen = []

    def evaluate(self, lattice, positions):
        b = self.backend
        with b.lock:
            b.active += 1
            b.max_active = max(b.max_active, b.active)
        time.sleep(b.eval_s * len(self.s.workload.species))
        with b.lock:
            b.active -= 1
            b.evals.append((self.s.sid, time.perf_counter()))
        p = np.asarray(positions, float)
        return float(p.sum()), p * 2.0, np.eye(3) * p.mean()

    def device_bytes(self):
        return self.backend.bytes_per_atom * len(self.s.workload.species)

    def close(self):
        with self.backend.lock:
            self.backend.closed.append(self.s.sid)


class FakeBackend:
    def __init__(self, eval_s=0.002, bytes_per_atom=1.0, estimate_scale=1.0):
        self.eval_s, self.bytes_per_atom, self.estimate_scale = eval_s, bytes_per_atom, estimate_scale
        self.lock = threading.Lock()
        self.active = self.max_active = 0
        self.evals, self.closed, self.created = [], [], []

    def estimate_bytes(self, s, known):
        return known.get(s.shape, self.estimate_scale * self.bytes_per_atom * len(s.workload.species))

    def create(self, s):
        with self.lock:
            self.created.append(s.sid)
        return FakePlan(self, s)


def fake_stream(n, rate, steps, sizes=(2, 5, 9), seed=3):
    def make(shape, sd):
        n_at = int(shape[1:])
        rng = np.random.default_rng(sd)
        return types.SimpleNamespace(species=np.zeros(n_at, np.int32), lattice=np.eye(3) * 5.0,
                                     positions=rng.normal(size=(n_at, 3)))
    return serve.make_stream(seed, rate, n, [f"x{k}" for k in sizes], steps, make=make)


def test_stream_is_seeded_poisson_with_relaxation_steps():
    a = fake_stream(50, 100.0, 4)
    b = fake_stream(50, 100.0, 4)
    assert [s.arrival for s in a] == [s.arrival for s in b]
    assert [s.shape for s in a] == [s.shape for s in b]
    gaps = np.diff([0.0] + [s.arrival for s in a])
    assert np.all(gaps > 0) and 0.3 / 100 < gaps.mean() < 3.0 / 100
    for s in a:
        assert len(s.geoms) == 4
        d = np.abs(s.geoms[1] - s.workload.positions)
        assert 0 < d.max() < 0.1   # small displacement per step


def test_every_request_runs_once_in_step_order_and_plans_are_freed():
    st = fake_stream(12, 400.0, 3)
    be = FakeBackend()
    out = serve.Server(be, budget_bytes=1e9, workers=3).run(st)
    recs = out["records"]
    assert len(recs) == 12 * 3 and not out["rejected"]
    for s in st:
        mine = sorted((r for r in recs if r.sid == s.sid), key=lambda r: r.start)
        assert [r.step for r in mine] == [0, 1, 2]
        # step k + 1 is issued when step k's result is back
        for r0, r1 in zip(mine, mine[1:]):
            assert r1.issued == pytest.approx(r0.end) and r1.start >= r0.end
        assert mine[0].issued == pytest.approx(s.arrival)
        assert mine[0].start >= s.arrival
    assert sorted(be.created) == sorted(be.closed) == sorted(s.sid for s in st)
    assert be.max_active > 1   # structures overlap
    # results belong to the request's own geometry
    for r in recs:
        s = st[r.sid]
        assert r.result[0] == pytest.approx(float(np.asarray(s.geoms[r.step]).sum()))


def test_admission_keeps_resident_bytes_within_budget():
    st = fake_stream(16, 1000.0, 2, sizes=(4, 6))
    be = FakeBackend(eval_s=0.002)
    budget = 12.0   # at most two 6-atom or three 4-atom structures at once
    out = serve.Server(be, budget_bytes=budget, workers=8).run(st)
    assert out["peak_bytes"] <= budget + 1e-9
    # reconstruct residency from the records: first start -> last end per structure
    spans = {}
    for r in out["records"]:
        a, b = spans.get(r.sid, (r.start, r.end))
        spans[r.sid] = (min(a, r.start), max(b, r.end))
    size = {s.sid: len(s.workload.species) for s in st}
    for sid, (a, b) in spans.items():
        t = (a + b) / 2
        live = sum(size[k] for k, (x, y) in spans.items() if x <= t <= y)
        assert live <= budget + 1e-9
    assert max(out["admission_wait"].values()) > 0   # the budget made some structures wait


def test_structure_larger_than_budget_is_rejected_not_stalled():
    st = fake_stream(6, 500.0, 2, sizes=(3, 20))
    be = FakeBackend()
    out = serve.Server(be, budget_bytes=10.0, workers=2).run(st)
    big = {s.sid for s in st if len(s.workload.species) == 20}
    assert set(out["rejected"]) == big
    assert {r.sid for r in out["records"]} == {s.sid for s in st} - big


def test_summary_percentiles_and_alone_vs_mix():
    st = fake_stream(10, 300.0, 3)
    be = FakeBackend()
    out = serve.Server(be, budget_bytes=1e9, workers=4).run(st)
    summ = serve.summarize(out, st)
    assert summ["requests"] == 30 and summ["p50_ms"] <= summ["p99_ms"]
    assert summ["throughput_req_s"] > 0
    assert set(summ["by_shape"]) == {s.shape for s in st}
    assert serve.alone_vs_mix(be, st, out["records"], 5) == 0.0   # the stand-in is deterministic


def test_device_overlap_from_request_intervals():
    """Requests in flight on the GPU at once: the sum of their device
    intervals over the union of them."""
    rec = lambda a, b: serve.Record(0, "x", 0, "p", 0.0, 0.0, 0.0, 0.0, None, (a, b))
    ov = serve.device_overlap([rec(0.0, 1.0), rec(0.5, 1.5), rec(2.0, 3.0), rec(2.2, 2.4)])
    assert ov["busy_s"] == pytest.approx(2.5)
    assert ov["sum_of_request_device_s"] == pytest.approx(3.2)
    assert ov["mean_requests_in_flight"] == pytest.approx(3.2 / 2.5)
    assert serve.device_overlap([rec(0.0, 1.0)])["mean_requests_in_flight"] == pytest.approx(1.0)
    assert serve.device_overlap([]) is None


def test_failed_request_ends_the_run_with_its_message():
    st = fake_stream(4, 500.0, 2)

    class Broken(FakeBackend):
        def create(self, s):
            if s.sid == 2:
                raise RuntimeError("no plan")
            return super().create(s)

    with pytest.raises(RuntimeError, match="structure 2 step 0: no plan"):
        serve.Server(Broken(), budget_bytes=1e9, workers=2).run(st)


@pytest.mark.gpu
def test_gpu_stream_alone_vs_mix():
    """A short mixed stream of small cells through the C ABI: every request
    completes, and requests re-evaluated alone on a fresh plan agree with
    their in-the-mix results to 1e-12 (only the order of FP64 atomic
    additions differs)."""
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available()
    st = serve.make_stream(11, 50.0, 6, ["si8", "perovskite5"], 3)
    be = serve.GpuBackend("bf16x6")
    out = serve.Server(be, budget_bytes=50e9, workers=3).run(st)
    assert len(out["records"]) == 18 and not out["rejected"]
    precs = {r.shape: r.precision for r in out["records"]}
    assert precs.get("si8", "bf16x6") == "bf16x6"
    assert precs.get("perovskite5", "bf16x6") == "bf16x6"   # n_ao 18: the wide split kernels
    assert serve.alone_vs_mix(be, st, out["records"], 6) <= 1e-12
    summ = serve.summarize(out, st)
    ov = summ["device_overlap"]
    assert ov is not None and ov["busy_s"] > 0 and ov["mean_requests_in_flight"] >= 1.0 - 1e-9
    assert summ["sustainable_structures_per_s"] > 0
