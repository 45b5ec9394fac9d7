"""Command-line entry point: run one synthetic workload through the C ABI
and print its stage times and counts.

  python -m paper_2412_11081_gb300.run_case [--cell NAME] [--precision fp64|bf16x3|bf16x6]
        [--evals N] [--home-chunk K] [--autotune]

NAME is one of diamond8, si8, si64, si216, si1000, perovskite, perovskite320,
perovskite1080.  The plan is created once and evaluated N times at the same
geometry; the last evaluation's stage times (CUDA events on the plan's
stream) and counts are printed as one JSON line.  Used to profile a single
plan (for example under ncu with -k on one kernel).
"""
from __future__ import annotations

import argparse
import json

from . import hfx, inputs

CELLS = {
    "diamond8": lambda: inputs.diamond8(),
    "si8": lambda: inputs.si_supercell(1),
    "si64": lambda: inputs.si_supercell(2),
    "si216": lambda: inputs.si_supercell(3),
    "si1000": lambda: inputs.workload_by_name("si1000"),
    "perovskite": lambda: inputs.perovskite_supercell(1),
    "perovskite40": lambda: inputs.perovskite_supercell(2),
    "perovskite135": lambda: inputs.perovskite_supercell(3),
    "perovskite320": lambda: inputs.workload_by_name("perovskite320"),
    "perovskite1080": lambda: inputs.workload_by_name("perovskite1080"),
}
PRECISIONS = {"fp64": hfx.HFX_FP64, "bf16x3": hfx.HFX_BF16X3, "bf16x6": hfx.HFX_BF16X6}


def lri_case(batch: int) -> int:
    """Wall time of hfx_lri_fit (host in, host out) on `batch` Si-like pairs,
    after one warm-up call, with its algorithmic FLOPs: per pair the Cholesky
    factor (n^3 / 3), the four substitutions of w columns (4 * 2 n^2 w) and
    the three dA X products (3 * 2 n^2 w)."""
    import time
    import numpy as np
    d, A, B, dA, dB, _ = inputs.lri_pairs(batch, 50, 50, 13, 13, seed=6)
    hfx.lri_fit(A[:2], B[:2], dA[:2], dB[:2])
    t = time.perf_counter()
    X, dX = hfx.lri_fit(A, B, dA, dB)
    dt = time.perf_counter() - t
    n, w = B.shape[1], B.shape[2]
    flops = batch * (n ** 3 / 3 + 14 * n * n * w)
    moved = A.nbytes + B.nbytes + dA.nbytes + dB.nbytes + X.nbytes + dX.nbytes
    print(json.dumps({"lri_batch": batch, "n": n, "w": w, "seconds": dt, "gflop": flops / 1e9,
                      "gflops_per_s": flops / dt / 1e9, "host_bytes_copied": moved,
                      "finite": bool(np.isfinite(X).all() and np.isfinite(dX).all())}))
    return 0


def main(argv=None) -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--cell", default="si8", choices=sorted(CELLS))
    ap.add_argument("--precision", default="bf16x3", choices=sorted(PRECISIONS))
    ap.add_argument("--evals", type=int, default=2)
    ap.add_argument("--autotune", action="store_true", help="run hfx_plan_autotune before the evaluations")
    ap.add_argument("--home-chunk", type=int, default=0, help="home atoms per pass (0 = the library's default)")
    ap.add_argument("--lri-batch", type=int, default=0,
                    help="instead: time hfx_lri_fit on this many Si-like pairs (n_abf 50 + 50, n_ao 13 x 13)")
    args = ap.parse_args(argv)
    if args.lri_batch > 0:
        return lri_case(args.lri_batch)
    w = CELLS[args.cell]()
    tune = None
    with hfx.Plan(w, precision=PRECISIONS[args.precision], home_chunk=args.home_chunk) as p:
        if args.autotune:
            tune = p.autotune(w.lattice, w.positions, reps=2)
        p.set_timing(True)
        for _ in range(max(1, args.evals)):
            E, F, S = p.evaluate(w.lattice, w.positions, stats=True)
        st = p.stats.as_dict()
    keep = ("ms_blocks", "ms_screen", "ms_y", "ms_term1", "ms_term2", "ms_reduce", "ms_total", "ms_term1_kernel",
            "ms_term2_kernel", "triplets", "term1_pairs", "term2_pairs", "y_blocks", "flops_y", "flops_term1",
            "flops_term2", "flops_total", "kernel_launches", "device_bytes", "passes")
    print(json.dumps({"cell": args.cell, "precision": args.precision, "E": E, **{k: st[k] for k in keep},
                      "autotune": tune}))
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
