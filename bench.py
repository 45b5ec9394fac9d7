"""Benchmark: HFX force+stress evaluations per second on the 64-atom Si-like
supercell (2x2x2 diamond, n_ao 13, n_abf 50, r_c 3.7 A, thresholds 1e-10).

One step = one full evaluation of the hot path (block generation, two-step
screening, Y build, both exchange products, force/stress/energy reduction)
on a warm plan, at a new geometry (small seeded jitter within the pair-list
skin, so every block, norm and screening decision is recomputed).  The
headline precision (`--precision auto`, the default) is HFX_BF16X3 if its
energy, force and stress errors against the FP64 GPU results of the first
four geometries of the sequence are all within 1e-5 relative, else
HFX_BF16X6; the other split and FP64 are reported beside it, each with its
measured (largest) error.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

`--impl reference` times the CPU oracle (the only reference that exists:
the paper has no code) on a bounded sample of the same workload.
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
WORKLOAD = "si64: 2x2x2 diamond supercell, 64 atoms, n_ao 13, n_abf 50, r_c 3.7 A, theta 1e-10"


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


def job_rates(steps_per_rank, world, t_dev, t_e2e, dist=None, device=None):
    """Whole-job throughput: the units all ranks processed over the slowest
    rank's time, device-timed and end to end."""
    t_max, t_e2e_max = max_over_ranks([t_dev, t_e2e], dist, device)
    return world * steps_per_rank / t_max, world * steps_per_rank / t_e2e_max, t_max


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


def cpu_baseline(w, homes, reps=1):
    """Time the oracle, as it stands, on `homes` home atoms of the workload.
    Its work is a sum over home atoms, so evals/s = 1 / (t * N / k)."""
    from oracle import OraclePlan
    plan = OraclePlan(w)
    t = time.time()
    for _ in range(reps):
        plan.evaluate(homes=list(range(homes)))
    dt = (time.time() - t) / reps
    per_eval = dt * w.n_atoms / homes
    return {"value": 1.0 / per_eval, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{homes} of {w.n_atoms} home atoms of {w.name} ({dt:.1f} s), scaled by N/k; "
                      f"numpy/OpenBLAS threads = cores"}


def run_reference(args):
    rank, world, _ = _env_rank()
    if rank != 0:
        return 0
    from paper_2412_11081_gb300 import inputs
    w = inputs.si_supercell(2)
    from oracle import OraclePlan
    plan = OraclePlan(w)
    homes = 1
    for _ in range(args.warmup):
        plan.evaluate(homes=[0])
    times = []
    for k in range(args.steps):
        t = time.time()
        plan.evaluate(homes=[k % w.n_atoms])
        times.append(time.time() - t)
    per_eval = statistics.mean(times) * w.n_atoms / homes
    value = 1.0 / per_eval
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": per_eval * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": WORKLOAD, "sample": "one home atom per step, scaled by 64"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"{homes} of 64 home atoms per step ({statistics.mean(times):.1f} s)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _time_device(plan, w, d_pos, d_out, first, steps, stream, torch):
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for k in range(steps):
        plan.evaluate_device(w.lattice, d_pos[first + k].data_ptr(), d_out.data_ptr())
    ev1.record(stream)
    torch.cuda.synchronize()
    return ev0.elapsed_time(ev1) / 1e3


def _rel(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


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
    from paper_2412_11081_gb300 import hfx, inputs
    w = inputs.si_supercell(2)
    stream = torch.cuda.current_stream(dev)
    n = w.n_atoms
    geoms = inputs.geometry_sequence(w, args.warmup + args.steps + 8)
    d_pos = [torch.tensor(g, dtype=torch.float64, device=dev) for g in geoms]
    d_out = torch.zeros(1 + 3 * n + 9, dtype=torch.float64, device=dev)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize(dev)

    # ---- reference result of the same geometry on the FP64 GPU path (parity-tested
    #      against the CPU oracle to 1e-10): the error of the mixed path is taken here
    fp64 = hfx.Plan(w, precision=hfx.HFX_FP64, stream=stream.cuda_stream, device=local)
    n_chk = 4   # geometries the split precisions are checked on
    refs = [fp64.evaluate(w.lattice, geoms[k]) for k in range(n_chk)]
    fp64_steps = max(1, min(2, args.steps))
    fp64.evaluate_device(w.lattice, d_pos[1].data_ptr(), d_out.data_ptr())
    barrier()
    t_fp64 = _time_device(fp64, w, d_pos, d_out, 2, fp64_steps, stream, torch) / fp64_steps
    fp64.close()

    variants = {}
    for name, prec in (("bf16x6", hfx.HFX_BF16X6), ("bf16x3", hfx.HFX_BF16X3)):
        pl = hfx.Plan(w, precision=prec, stream=stream.cuda_stream, device=local)
        errs = []
        for k in range(n_chk):
            E, F, S = pl.evaluate(w.lattice, geoms[k])
            ref = refs[k]
            errs.append((abs(E - ref[0]) / abs(ref[0]), _rel(F, ref[1]), _rel(S, ref[2])))
        variants[name] = dict(plan=pl, errE=max(e[0] for e in errs), errF=max(e[1] for e in errs),
                              errS=max(e[2] for e in errs))
    auto = args.precision == "auto"
    if auto:
        # BF16X3 runs half the piece products of BF16X6: it is the headline
        # only if it meets the 1e-5 contract on every checked geometry
        x3 = variants["bf16x3"]
        args.precision = "bf16x3" if max(x3["errE"], x3["errF"], x3["errS"]) <= 1e-5 else "bf16x6"
    plan = variants[args.precision]["plan"] if args.precision != "fp64" else \
        hfx.Plan(w, precision=hfx.HFX_FP64, stream=stream.cuda_stream, device=local)
    # the split plans pick their launch shapes with the library's autotuner
    # (hfx_plan_autotune, untimed; the arithmetic does not change)
    tuned = {}
    if not args.no_autotune:
        for name, v in variants.items():
            tuned[name] = v["plan"].autotune(w.lattice, geoms[0], reps=3)

    for k in range(args.warmup):
        plan.evaluate_device(w.lattice, d_pos[k].data_ptr(), d_out.data_ptr(), stats=True)
    st = plan.stats.as_dict()

    # ---- device-resident timing of the headline precision (value)
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    t_dev = _time_device(plan, w, d_pos, d_out, args.warmup, args.steps, stream, torch)
    barrier()
    ck = clocks.stop()
    launches = st["kernel_launches"] * args.steps

    # ---- end-to-end through the host entry point (H2D positions, D2H results)
    pin_pos = [torch.tensor(g, dtype=torch.float64).pin_memory().numpy() for g in geoms]
    barrier()
    t0 = time.perf_counter()
    lat = []   # per request: host positions in -> E, F, sigma back on the host (the call is synchronous)
    for k in range(args.steps):
        tk = time.perf_counter()
        plan.evaluate(w.lattice, pin_pos[args.warmup + k])
        lat.append(time.perf_counter() - tk)
    barrier()
    t_e2e = time.perf_counter() - t0

    # ---- the other split precision (secondary line items)
    other = {}
    for name, v in variants.items():
        if name == args.precision:
            continue
        pl = v["plan"]
        pl.evaluate_device(w.lattice, d_pos[0].data_ptr(), d_out.data_ptr())
        tt = _time_device(pl, w, d_pos, d_out, args.warmup, min(args.steps, 5), stream, torch) / min(args.steps, 5)
        other[name] = {"evals_per_s": 1.0 / tt, "errE": v["errE"], "errF": v["errF"], "errS": v["errS"]}

    # ---- per-stage times (CUDA events on the plan's stream)
    plan.set_timing(True)
    stage = {k: [] for k in ("ms_blocks", "ms_screen", "ms_y", "ms_term1", "ms_term2", "ms_reduce")}
    flops = None
    for k in range(min(3, args.steps)):
        plan.evaluate_device(w.lattice, d_pos[k].data_ptr(), d_out.data_ptr(), stats=True)
        flops = plan.stats.as_dict()
        for key in stage:
            stage[key].append(flops[key])
    plan.set_timing(False)
    stage_ms = {k: statistics.mean(v) for k, v in stage.items()}

    value, e2e_value, t_max = job_rates(args.steps, world, t_dev, t_e2e, dist, dev)

    if rank == 0:
        peaks = measured_peaks()
        fp64_peak = fp64_gemm_peak(torch, dev)
        dom = max(("y", "term1", "term2"), key=lambda k: stage_ms["ms_" + k])
        dom_flops = flops["flops_" + dom]
        dom_ms = stage_ms["ms_" + dom]
        achieved = dom_flops / (dom_ms / 1e3) / 1e12
        kname = {"y": "k_ybuild", "term1": "k_term1", "term2": "k_term2"}[dom]
        if args.precision != "fp64":
            kname = {"y": "k_ybuild_umma", "term1": "k_t1_umma", "term2": "k_term2_pairs+k_q2_umma"}[dom]
        if args.precision == "fp64":
            roofline = {"kernel": kname, "bound": "alu", "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s",
                        "frac": achieved / fp64_peak, "traffic": None,
                        "peak_source": "FP64 cuBLAS DGEMM 4096^3 measured in this run (FP64 pipe)"}
        else:
            pk = peaks.get("bf16_tflops_sustained") or 1717.3
            pieces = 6 if args.precision == "bf16x6" else 3
            roofline = {"kernel": kname, "bound": "tensor", "achieved": achieved, "peak": pk,
                        "unit": "TFLOP/s", "frac": achieved / pk,
                        "traffic": t1_traffic(args.precision) if kname == "k_t1_umma" else None,
                        "traffic_source": f"profiles/k_t1_umma_si8_{args.precision}.md: dram read+write of one si8 "
                                          "launch, scaled to si64 by kept triplets (bytes per launch)",
                        "peak_source": "bf16 dense, sustained, of measured (MEASURED_PEAKS.json)",
                        "note": f"achieved counts algorithmic FLOPs only; the {pieces} bf16 piece products per "
                                f"multiply and the 13->16 / 50->64 tile padding are not counted",
                        "tensor_issue_tflops": achieved * pieces}
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            cpu = cpu_baseline(w, homes=1)
        h2d = 3 * n * 8 + 9 * 8
        d2h = (1 + 3 * n + 9) * 8
        head = variants.get(args.precision, {})
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": t_max / args.steps * 1e3, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": "bf16" if args.precision != "fp64" else "f64",
                "data": "synthetic",
                "config": {"workload": WORKLOAD, "precision": args.precision,
                           "headline_rule": "bf16x3 if max(errE, errF, errS) <= 1e-5 vs FP64 GPU on 4 geometries, else bf16x6"
                           if auto else "fixed by --precision",
                           "arithmetic": "bf16 pieces on tensor cores, fp32 accumulate, fp64 screening/reduction"
                           if args.precision != "fp64" else "fp64",
                           "parallelism": f"replicas{world}" if world > 1 else "single",
                           "l2": "working set > L2 (block, Y and Z stores of several GB per step)"},
                "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
                "latency": {"p50_ms": float(np.percentile(lat, 50)) * 1e3, "p99_ms": float(np.percentile(lat, 99)) * 1e3,
                            "requests": len(lat), "what": "one evaluation through the host entry point on an "
                            "otherwise idle GPU, rank 0; a loaded request stream is reported by the serving loop"},
                "gpu_launches": launches,
                "roofline": roofline,
                "cpu_baseline": cpu,
                "clocks": ck,
                "error_vs_fp64": {k: head.get(k) for k in ("errE", "errF", "errS")} if head else None,
                "fp64": {"evals_per_s": 1.0 / t_fp64, "speedup_of_headline": value / world * t_fp64},
                "other_precisions": other,
                "stages_ms": stage_ms,
                "autotune": tuned,
                "gflop_per_eval": flops["flops_total"] / 1e9,
                "achieved_tflops_total": flops["flops_total"] / (t_max / args.steps) / 1e12,
                "counts": {k: flops[k] for k in ("c_pairs", "v_pairs", "triplets", "term1_pairs",
                                                 "term2_pairs", "y_blocks", "device_bytes")},
                "peaks": {"hbm_gbs": peaks.get("hbm_gbs"), "bf16_tflops": peaks.get("bf16_tflops"),
                          "bf16_tflops_sustained": peaks.get("bf16_tflops_sustained"),
                          "fp64_dgemm_tflops": fp64_peak}}
        print(json.dumps(line), flush=True)
    for v in variants.values():
        v["plan"].close()
    if args.precision == "fp64":
        plan.close()
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
    ap.add_argument("--precision", default="auto", choices=["auto", "bf16x6", "bf16x3", "fp64"])
    ap.add_argument("--no-autotune", action="store_true", help="keep the plans' initial launch shapes")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
