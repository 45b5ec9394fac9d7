"""Benchmark: HFX force+stress evaluations per second on the 1000-atom
Si-like supercell (5x5x5 diamond, n_ao 13, n_abf 50, r_c 3.7 A, 3 % random
strain, thresholds 1e-10), the configuration the mixed-precision target is
quoted on.

One step = one full evaluation of the hot path (block norms, two-step
screening, Y build, both exchange products in passes of 128 home atoms,
force/stress/energy reduction) on a warm plan, at a new geometry (small
seeded jitter within the pair-list skin, so every block, norm and screening
decision is recomputed).  The headline precision is HFX_BF16X6 (the split
that meets the 1e-5 contract on every tested geometry; HFX_BF16X3 misses it
on some, see tests/test_gpu_mixed.py); FP64 and BF16X3 are reported beside
it, each with its error against the FP64 GPU result of the same geometry.
Plans run one after another (FP64, the headline, the other split), each
freed before the next, so that one holds the GPU's memory at a time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (torchrun, one rank per GPU) each rank's plan takes a contiguous
range of home atoms and an all-reduce of E, F and sigma finishes each step
(home-atom sharding; total work fixed, "scaling": "strong").
`--impl reference` times the CPU oracle (the only reference that exists:
the paper has no code) on bounded samples of the same per-atom work.
Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "HFX force+stress evals/s & %tensor roofline, mixed vs FP64 at 1e-5 rel; p99 latency"
UNIT = "evals/s"
WORKLOAD_NAME = "si1000"
N_ATOMS = 1000
WORKLOAD = ("si1000: 5x5x5 diamond supercell, 1000 atoms, n_ao 13, n_abf 50, r_c 3.7 A, 3 % random strain, "
            "theta 1e-10")
SI64_TRIPLETS = 828423   # kept triplets of si64, the case the first product's DRAM traffic was scaled to


def _env_rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


def max_over_ranks(values, dist=None, device=None):
    """Each value's maximum over the ranks of the process group (the job's
    time is the slowest rank's); the values themselves on one process."""
    if dist is None:
        return [float(v) for v in values]
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t]


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""
    FIELDS = ["clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.hw_slowdown",
              "clocks_event_reasons.hw_thermal_slowdown", "clocks_event_reasons.sw_thermal_slowdown",
              "clocks_event_reasons.sw_power_cap"]

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + ",".join(self.FIELDS),
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) != len(self.FIELDS):
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def t1_traffic(precision):
    """DRAM bytes per si64 launch of the first-product kernel at `precision`
    ("bf16x3" or "bf16x6") from its ncu summary, or None once the kernel's
    sources differ from the captured ones."""
    import hashlib
    path = os.path.join(ROOT, "profiles", f"k_t1_umma_si8_{precision}.md")
    try:
        text = open(path).read()
    except OSError:
        return None
    vals = {}
    for line in text.splitlines():
        k, _, v = line.strip().partition(": ")
        if k in ("kernel_sources_sha256_16", "traffic_bytes_per_si64_launch"):
            vals[k] = v.strip()
    h = hashlib.sha256()
    for f in ("hfx_t1umma.cu", "hfx_device.cuh"):
        with open(os.path.join(ROOT, "paper_2412_11081_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    if vals.get("kernel_sources_sha256_16") != h.hexdigest()[:16] or "traffic_bytes_per_si64_launch" not in vals:
        return None
    return float(vals["traffic_bytes_per_si64_launch"])


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def fp64_gemm_peak(torch, dev):
    """FP64 reference peak on this GPU: cuBLAS DGEMM 4096^3, best of 3
    (the FP64 counterpart of the bf16 cuBLAS figure in MEASURED_PEAKS)."""
    n = 4096
    a = torch.randn(n, n, dtype=torch.float64, device=dev)
    b = torch.randn(n, n, dtype=torch.float64, device=dev)
    torch.matmul(a, b)
    torch.cuda.synchronize()
    best = 1e30
    for _ in range(3):
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        torch.matmul(a, b)
        e.record()
        torch.cuda.synchronize()
        best = min(best, s.elapsed_time(e) / 1e3)
    del a, b
    return 2.0 * n ** 3 / best / 1e12


def cpu_baseline_sample(name="si64"):
    """Time the oracle, as it stands, on a bounded sample with the per-atom
    work of the benchmark's workload: si64 has the same species, basis sizes,
    thresholds and per-atom pair counts as si1000 (the lattice sums cover
    every image, so the work per atom does not depend on the supercell).
    One evaluation costs a per-structure part (the plan's D norms, then the
    blocks, norms and Cauchy-Schwarz factors of every atom: OraclePlan and
    evaluate(homes=[])) and a part per home atom (evaluate(homes=[k]) minus
    evaluate(homes=[])).  The per-home part builds every Y block that home
    atom's items read, blocks a full evaluation shares among home atoms, so
    N times it overstates the oracle's time on a full evaluation."""
    from oracle import OraclePlan
    from paper_2412_11081_gb300 import inputs
    w = inputs.workload_by_name(name)
    t0 = time.time()
    plan = OraclePlan(w)
    t_ctor = time.time() - t0
    t1 = time.time()
    plan.evaluate(homes=[])
    t_pre = time.time() - t1
    t2 = time.time()
    plan.evaluate(homes=[0])
    t_one = time.time() - t2
    return {"n_atoms": w.n_atoms, "t_ctor": t_ctor, "t_pre": t_pre, "t_one": t_one, "wall": time.time() - t0}


def oracle_rate(sample, n_atoms):
    """Oracle evals/s on n_atoms atoms: the per-structure part scaled by
    atoms plus n_atoms times one home atom's part."""
    per_atom_pre = (sample["t_ctor"] + sample["t_pre"]) / sample["n_atoms"]
    per_home = max(sample["t_one"] - sample["t_pre"], 0.0)
    return 1.0 / (n_atoms * (per_atom_pre + per_home)), per_atom_pre, per_home


def cpu_baseline(n_atoms):
    s = cpu_baseline_sample()
    rate, pa, ph = oracle_rate(s, n_atoms)
    return {"value": rate, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"oracle on si64 (same per-atom shapes and pair counts as {WORKLOAD_NAME}): per-structure "
                      f"part {s['t_ctor'] + s['t_pre']:.1f} s for 64 atoms, one home atom {ph:.1f} s; estimate for "
                      f"{n_atoms} atoms = {n_atoms} x ({pa:.3f} + {ph:.2f}) s (each home atom's Y blocks counted "
                      f"in full: an upper bound of a full evaluation's time); {s['wall']:.1f} s of CPU work; "
                      f"numpy/OpenBLAS threads = cores"}


def run_reference(args):
    """The oracle (the reference arm: the paper ships no code) on bounded
    samples of the workload.  Step k evaluates home atom k of si64 (the same
    per-atom work as si1000); the line's value is the oracle's evals/s on
    si1000 from the per-structure part (timed once before the steps) plus
    the mean per-home-atom time of the steps; ms_per_step is the measured
    wall time of one step."""
    rank, world, _ = _env_rank()
    if rank != 0:
        return 0
    from oracle import OraclePlan
    from paper_2412_11081_gb300 import inputs
    w = inputs.workload_by_name("si64")
    t0 = time.time()
    plan = OraclePlan(w)
    t_ctor = time.time() - t0
    t1 = time.time()
    plan.evaluate(homes=[])
    t_pre = time.time() - t1
    for k in range(args.warmup):
        plan.evaluate(homes=[k % w.n_atoms])
    times = []
    for k in range(args.steps):
        t = time.time()
        plan.evaluate(homes=[k % w.n_atoms])
        times.append(time.time() - t)
    step = statistics.mean(times)
    rate, pa, ph = oracle_rate({"n_atoms": w.n_atoms, "t_ctor": t_ctor, "t_pre": t_pre, "t_one": step}, N_ATOMS)
    sample = (f"step k = home atom k of si64 (same per-atom shapes and pair counts as {WORKLOAD_NAME}); "
              f"value = 1 / ({N_ATOMS} x ({pa:.3f} s per-structure part per atom + {ph:.2f} s per home atom)), "
              f"the per-structure part ({t_ctor + t_pre:.1f} s for 64 atoms) timed once before the steps, the "
              f"per-home part = mean step minus it; each home atom's Y blocks counted in full (an upper bound "
              f"of a full evaluation's time)")
    line = {"metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": WORKLOAD, "sample": sample},
            "cpu_baseline": {"value": rate, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _time_device(plan, w, d_pos, d_out, first, steps, stream, torch, reduce=None):
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for k in range(steps):
        plan.evaluate_device(w.lattice, d_pos[first + k].data_ptr(), d_out.data_ptr())
        if reduce is not None:
            reduce(d_out)
    ev1.record(stream)
    torch.cuda.synchronize()
    return ev0.elapsed_time(ev1) / 1e3


def _rel(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _errs(got, ref):
    return {"errE": abs(got[0] - ref[0]) / abs(ref[0]), "errF": _rel(got[1], ref[1]), "errS": _rel(got[2], ref[2])}


PEROVSKITE = ("perovskite320: 4x4x4 CsSnI3-shaped cubic perovskite, 320 atoms, n_ao 18/13/13, n_abf 75/60/60 "
              "(Cs/Sn/I), r_c 4.2 A, jittered, theta 1e-10")


def perovskite_line(torch, dev, stream, local, steps=3):
    """The 320-atom three-species perovskite in BF16X6 (the split kernels for
    n_ao > 16) against the FP64 GPU path on the same GB300: rate of each,
    the errors of the split result on the first geometry, per-stage times."""
    from paper_2412_11081_gb300 import hfx, inputs
    w = inputs.workload_by_name("perovskite320")
    n = w.n_atoms
    geoms = inputs.geometry_sequence(w, steps + 3, seed=23)
    d_pos = [torch.tensor(g, dtype=torch.float64, device=dev) for g in geoms]
    d_out = torch.zeros(1 + 3 * n + 9, dtype=torch.float64, device=dev)

    def result(plan, k):
        plan.evaluate_device(w.lattice, d_pos[k].data_ptr(), d_out.data_ptr())
        v = d_out.cpu().numpy()
        return float(v[0]), v[1:1 + 3 * n].reshape(n, 3).copy(), v[1 + 3 * n:].reshape(3, 3).copy()

    out = {"workload": PEROVSKITE, "precision": "bf16x6"}
    with hfx.Plan(w, precision=hfx.HFX_FP64, stream=stream.cuda_stream, device=local) as p:
        ref = result(p, 0)
        out["fp64_evals_per_s"] = 1.0 / _time_device(p, w, d_pos, d_out, 1, 1, stream, torch)
    with hfx.Plan(w, precision=hfx.HFX_BF16X6, stream=stream.cuda_stream, device=local) as p:
        out.update(_errs(result(p, 0), ref))
        p.evaluate_device(w.lattice, d_pos[1].data_ptr(), d_out.data_ptr())
        t = _time_device(p, w, d_pos, d_out, 2, steps, stream, torch) / steps
        out["evals_per_s"] = 1.0 / t
        out["speedup_over_fp64"] = out["evals_per_s"] / out["fp64_evals_per_s"]
        p.set_timing(True)
        p.evaluate_device(w.lattice, d_pos[2].data_ptr(), d_out.data_ptr(), stats=True)
        st = p.stats.as_dict()
        out["stages_ms"] = {k: st[k] for k in ("ms_blocks", "ms_screen", "ms_y", "ms_term1", "ms_term2", "ms_total")}
        out["gflop_per_eval"] = st["flops_total"] / 1e9
        out["achieved_tflops"] = st["flops_total"] / t / 1e12
        out["kernels"] = "k_ybuild_w, k_term1_w, k_term2_w, k_q2_w (warp-level MMAs on bf16 pieces, n_ao up to 32)"
    return out


def run_ours(args):
    import torch
    rank, world, local = _env_rank()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2412_11081_gb300 import hfx, inputs, shard
    w = inputs.workload_by_name(WORKLOAD_NAME)
    stream = torch.cuda.current_stream(dev)
    n = w.n_atoms
    home = shard.home_ranges(n, world)[rank] if world > 1 else None
    geoms = inputs.geometry_sequence(w, args.warmup + args.steps + 4)
    d_pos = [torch.tensor(g, dtype=torch.float64, device=dev) for g in geoms]
    d_out = torch.zeros(1 + 3 * n + 9, dtype=torch.float64, device=dev)
    PREC = {"bf16x6": hfx.HFX_BF16X6, "bf16x3": hfx.HFX_BF16X3, "fp64": hfx.HFX_FP64}
    reduce = None
    if dist is not None:
        def reduce(t):   # the sum of the ranks' shares (home-atom sharding): the one exchange
            dist.all_reduce(t, op=dist.ReduceOp.SUM)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize(dev)

    def new_plan(name):
        return hfx.Plan(w, precision=PREC[name], stream=stream.cuda_stream, device=local, home=home)

    def whole(plan, k):
        """E, F, sigma of geometry k (the shares summed over the ranks)."""
        plan.evaluate_device(w.lattice, d_pos[k].data_ptr(), d_out.data_ptr())
        if reduce is not None:
            reduce(d_out)
        v = d_out.cpu().numpy()
        return float(v[0]), v[1:1 + 3 * n].reshape(n, 3).copy(), v[1 + 3 * n:].reshape(3, 3).copy()

    # ---- the FP64 GPU path (parity-tested against the oracle to 1e-10) on the
    #      first geometry: the reference of the split precisions' errors, and its rate
    pl = new_plan("fp64")
    pl.set_timing(True)
    barrier()
    t = time.perf_counter()
    ref = whole(pl, 0)
    barrier()
    t_fp64 = time.perf_counter() - t
    pl.evaluate_device(w.lattice, d_pos[0].data_ptr(), d_out.data_ptr(), stats=True)
    fp64_stats = pl.stats.as_dict()
    pl.close()

    head = args.precision if args.precision != "auto" else "bf16x6"
    # ---- headline precision
    plan = new_plan(head)
    head_err = _errs(whole(plan, 0), ref) if head != "fp64" else {"errE": 0.0, "errF": 0.0, "errS": 0.0}
    tuned = {}
    if head != "fp64" and not args.no_autotune:   # launch shapes by the library's autotuner (untimed)
        tuned[head] = plan.autotune(w.lattice, geoms[1], reps=2)
    for k in range(args.warmup):
        plan.evaluate_device(w.lattice, d_pos[1 + k].data_ptr(), d_out.data_ptr(), stats=True)
        if reduce is not None:
            reduce(d_out)
    st = plan.stats.as_dict()

    # device-resident timing (value)
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    first = 1 + args.warmup
    t_dev = _time_device(plan, w, d_pos, d_out, first, args.steps, stream, torch, reduce)
    barrier()
    ck = clocks.stop()
    launches = st["kernel_launches"] * args.steps

    # end to end through the host entry point (H2D positions, D2H results)
    pin_pos = [torch.tensor(g, dtype=torch.float64).pin_memory().numpy() for g in geoms]
    barrier()
    t0 = time.perf_counter()
    lat = []   # per request: host positions in -> E, F, sigma back on the host (the call is synchronous)
    for k in range(args.steps):
        tk = time.perf_counter()
        E, F, S = plan.evaluate(w.lattice, pin_pos[first + k])
        if reduce is not None:
            v = torch.from_numpy(shard.pack(E, F, S)).to(dev)
            reduce(v)
            v.cpu()
        lat.append(time.perf_counter() - tk)
    barrier()
    t_e2e = time.perf_counter() - t0

    # per-stage and per-kernel times (CUDA events on the plan's stream)
    plan.set_timing(True)
    keys = ("ms_blocks", "ms_screen", "ms_y", "ms_term1", "ms_term2", "ms_reduce", "ms_term1_kernel",
            "ms_term2_kernel", "ms_total")
    stage = {k: [] for k in keys}
    for k in range(min(3, args.steps)):
        plan.evaluate_device(w.lattice, d_pos[first + k].data_ptr(), d_out.data_ptr(), stats=True)
        flops = plan.stats.as_dict()
        for key in keys:
            stage[key].append(flops[key])
    plan.set_timing(False)
    stage_ms = {k: statistics.mean(v) for k, v in stage.items()}
    plan.close()

    # ---- graph replay (hfx_options.graph): frozen plans of the headline
    #      precision with and without it, the same steps
    graph_cmp = {}
    if not args.no_graph:
        m = min(args.steps, 3)
        for use_graph in (False, True):
            pl = hfx.Plan(w, precision=PREC[head], stream=stream.cuda_stream, device=local, home=home,
                          freeze_lists=True, graph=use_graph)
            for k in range(2):   # the first call fixes the decisions, the second records the graph
                pl.evaluate_device(w.lattice, d_pos[1 + k].data_ptr(), d_out.data_ptr())
            barrier()
            tt = _time_device(pl, w, d_pos, d_out, first, m, stream, torch, reduce) / m
            pl.evaluate_device(w.lattice, d_pos[first].data_ptr(), d_out.data_ptr(), stats=True)
            graph_cmp["graph" if use_graph else "direct"] = {"ms_per_eval": tt * 1e3,
                                                             "graph_replayed": pl.stats.graph_replayed}
            pl.close()
        graph_cmp["what"] = ("frozen plans (screening decisions of the first call kept), the headline precision, "
                             f"{m} steps each: every kernel launched per call vs one CUDA graph launch per call")

    # ---- the other split precision (secondary line item)
    other = {}
    for name in ("bf16x6", "bf16x3"):
        if name == head:
            continue
        pl = new_plan(name)
        e = _errs(whole(pl, 0), ref)
        pl.evaluate_device(w.lattice, d_pos[1].data_ptr(), d_out.data_ptr())
        m = min(args.steps, 3)
        tt = _time_device(pl, w, d_pos, d_out, first, m, stream, torch, reduce) / m
        pl.close()
        other[name] = {"evals_per_s": 1.0 / tt, **e}

    t_max, t_e2e_max = max_over_ranks([t_dev, t_e2e], dist, dev)
    value = args.steps / t_max          # whole evaluations of the structure per second
    e2e_value = args.steps / t_e2e_max

    if rank == 0:
        peaks = measured_peaks()
        fp64_peak = fp64_gemm_peak(torch, dev)
        # the dominant kernel: the first exchange product's contraction (one launch per pass)
        kflops = flops["flops_term1"]
        kms = stage_ms["ms_term1_kernel"]
        passes = flops["passes"]
        achieved = kflops / (kms / 1e3) / 1e12
        if head == "fp64":
            roofline = {"kernel": "k_term1", "bound": "alu", "achieved": achieved, "peak": fp64_peak,
                        "unit": "TFLOP/s", "frac": achieved / fp64_peak, "traffic": None,
                        "peak_source": "FP64 cuBLAS DGEMM 4096^3 measured in this run (FP64 pipe)"}
        else:
            pk = peaks.get("bf16_tflops_sustained") or 1717.3
            pieces = 6 if head == "bf16x6" else 3
            tr = t1_traffic(head)
            # DRAM bytes per launch: the capture's bytes per kept triplet times one launch's kept triplets
            traffic = tr / SI64_TRIPLETS * (flops["triplets"] / passes) if tr is not None else None
            roofline = {"kernel": "k_t1_umma", "bound": "tensor", "achieved": achieved, "peak": pk,
                        "unit": "TFLOP/s", "frac": achieved / pk, "traffic": traffic,
                        "launches_per_step": passes,
                        "per_launch": f"{kflops / passes / 1e12:.3f} TFLOP algorithmic ({flops['triplets'] // passes} "
                                      f"kept triplets) in {kms / passes:.1f} ms",
                        "traffic_source": f"profiles/k_t1_umma_si8_{head}.md: DRAM read+write per kept triplet of "
                                          "the capture, times the kept triplets of one launch (one pass)",
                        "peak_source": "bf16 dense, sustained, of measured (MEASURED_PEAKS.json)",
                        "note": f"achieved counts algorithmic FLOPs only; the {pieces} bf16 piece products per "
                                f"multiply and the 13->16 / 50->64 tile padding are not counted",
                        "tensor_issue_tflops": achieved * pieces}
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            cpu = cpu_baseline(n)
        perov = None
        if world == 1 and not args.no_perovskite:
            perov = perovskite_line(torch, dev, stream, local)
        h2d = 3 * n * 8
        d2h = (1 + 3 * n + 9) * 8
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": t_max / args.steps * 1e3, "higher_is_better": True,
                "scaling": "strong" if world > 1 else "weak", "vs_baseline": None,
                "dtype": "bf16" if head != "fp64" else "f64",
                "data": "synthetic",
                "config": {"workload": WORKLOAD, "precision": head,
                           "arithmetic": "bf16 pieces on tensor cores, fp32 accumulate, fp64 screening/reduction"
                           if head != "fp64" else "fp64",
                           "parallelism": f"home-atom shards x{world} + all-reduce of E, F, sigma" if world > 1
                           else "single",
                           "passes": passes,
                           "l2": "working set > L2 (Y stores of over 100 GB and per-pass operand stores each step)"},
                "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
                "latency": {"p50_ms": float(np.percentile(lat, 50)) * 1e3, "p99_ms": float(np.percentile(lat, 99)) * 1e3,
                            "requests": len(lat), "what": "one evaluation through the host entry point on an "
                            "otherwise idle GPU, rank 0; a loaded request stream is reported by the serving loop"},
                "gpu_launches": launches,
                "roofline": roofline,
                "cpu_baseline": cpu,
                "clocks": ck,
                "error_vs_fp64": head_err,
                "fp64": {"evals_per_s": 1.0 / t_fp64, "speedup_of_headline": value * t_fp64,
                         "term1_kernel_tflops": fp64_stats["flops_term1"] / fp64_stats["ms_term1_kernel"] / 1e9
                         if fp64_stats["ms_term1_kernel"] > 0 else None},
                "other_precisions": other,
                "perovskite320": perov,
                "graph_replay": graph_cmp,
                "stages_ms": stage_ms,
                "autotune": tuned,
                "gflop_per_eval": flops["flops_total"] / 1e9,
                "achieved_tflops_total": flops["flops_total"] / (t_max / args.steps) / 1e12,
                "counts": {k: flops[k] for k in ("c_pairs", "v_pairs", "triplets", "term1_pairs",
                                                 "term2_pairs", "y_blocks", "device_bytes", "passes")},
                "peaks": {"hbm_gbs": peaks.get("hbm_gbs"), "bf16_tflops": peaks.get("bf16_tflops"),
                          "bf16_tflops_sustained": peaks.get("bf16_tflops_sustained"),
                          "fp64_dgemm_tflops": fp64_peak}}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--precision", default="auto", choices=["auto", "bf16x6", "bf16x3", "fp64"],
                    help="headline precision; auto = bf16x6")
    ap.add_argument("--no-autotune", action="store_true", help="keep the plans' initial launch shapes")
    ap.add_argument("--no-graph", action="store_true", help="skip the frozen-plan graph replay comparison")
    ap.add_argument("--no-perovskite", action="store_true", help="skip the 320-atom perovskite line (BF16X6 vs FP64)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
