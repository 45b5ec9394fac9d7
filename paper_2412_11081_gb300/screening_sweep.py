"""Screening sweep on a synthetic workload: error and time of the force and
stress evaluation against the block-screening thresholds.

This is the analogue of the paper's threshold study (Sec. 4.2, the effect
of filtering the individual tensors C, V, D, grad C, grad V, and Sec. 4.3,
the Cauchy-Schwarz screening of items with and without that pre-screening):

  * one family per tensor: "C+dC" (theta_C = theta_dC), "V+dV" (theta_V =
    theta_dV) and "D" take each value of the sweep while every other
    threshold, theta_CS included, is 0.  A pair's block and its gradient
    are kept or dropped together (kept if either norm is above its
    threshold, so that E, F and sigma come from one item set), so C and
    grad C (V and grad V) are swept as one family: theta_C alone, with
    theta_dC at 0, could drop only pairs whose gradient is exactly zero;
  * "CS": theta_CS alone (all tensor thresholds 0);
  * "CS+pre": theta_CS with every tensor threshold at `pre` (1e-10).

The reference is the evaluation with every threshold 0 (nothing screened
beyond the exact zeros of the model and the D blocks present in the
input).  Errors are the FP64 results against that reference, per output:
|dE|/|E|, max|dF|/max|F|, max|dsigma|/max|sigma|.  Times are CUDA-event
totals of one evaluation on a warm plan, FP64 and the BF16X6 split.  Kept
item counts (term-1 triplets, term-2 pairs) come with each point.

Every evaluation runs through the C ABI; this module only varies the
options and collects the numbers.
"""
from __future__ import annotations

import argparse
import json
import statistics

import numpy as np

from . import hfx, inputs

TENSORS = ("C", "dC", "V", "dV", "D")
FAMILIES = ("C+dC", "V+dV", "D", "CS", "CS+pre")


def _thetas(family: str, value: float, pre: float) -> dict:
    th = {k: 0.0 for k in TENSORS + ("CS",)}
    if family in ("C+dC", "V+dV", "D"):
        for k in family.split("+"):
            th[k] = value
    elif family == "CS":
        th["CS"] = value
    elif family == "CS+pre":
        th.update({k: pre for k in TENSORS})
        th["CS"] = value
    elif family != "reference":
        raise ValueError(family)
    return th


def _errors(out, ref) -> dict:
    E, F, S = out
    E0, F0, S0 = ref
    F, F0, S, S0 = (np.asarray(x, float) for x in (F, F0, S, S0))
    return {"errE": abs(E - E0) / abs(E0), "errF": float(np.max(np.abs(F - F0)) / np.max(np.abs(F0))),
            "errS": float(np.max(np.abs(S - S0)) / np.max(np.abs(S0)))}


def _run(w, precision: int, theta: dict, reps: int):
    with hfx.Plan(w, precision=precision, theta=theta) as p:
        out = p.evaluate(w.lattice, w.positions)
        p.set_timing(True)
        ms = []
        for _ in range(reps):
            p.evaluate(w.lattice, w.positions, stats=True)
            ms.append(p.stats.ms_total)
        st = p.stats.as_dict()
    return out, statistics.median(ms), st


def sweep(w, values, pre: float = 1e-10, families=FAMILIES, reps: int = 3,
          split: bool = True):
    ref, ref_ms, ref_st = _run(w, hfx.HFX_FP64, _thetas("reference", 0.0, pre), reps)
    rows = [{"family": "reference", "theta": 0.0, "ms_fp64": ref_ms, "triplets": ref_st["triplets"],
             "term2_pairs": ref_st["term2_pairs"], "errE": 0.0, "errF": 0.0, "errS": 0.0}]
    if split:
        _, ms, _ = _run(w, hfx.HFX_BF16X6, _thetas("reference", 0.0, pre), reps)
        rows[0]["ms_bf16x6"] = ms
    for fam in families:
        for v in values:
            th = _thetas(fam, v, pre)
            out, ms, st = _run(w, hfx.HFX_FP64, th, reps)
            row = {"family": fam, "theta": v, "ms_fp64": ms, "triplets": st["triplets"],
                   "term2_pairs": st["term2_pairs"]}
            row.update(_errors(out, ref))
            if split:
                _, ms6, _ = _run(w, hfx.HFX_BF16X6, th, reps)
                row["ms_bf16x6"] = ms6
            rows.append(row)
    return rows


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--cell", default="si8", choices=["si8", "si64", "diamond8"])
    ap.add_argument("--values", default="1e-10,1e-8,1e-6,1e-4,1e-2")
    ap.add_argument("--pre", type=float, default=1e-10)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--no-split", action="store_true", help="time the FP64 path only")
    args = ap.parse_args(argv)
    w = {"si8": lambda: inputs.si_supercell(1), "si64": lambda: inputs.si_supercell(2),
         "diamond8": inputs.diamond8}[args.cell]()
    values = [float(x) for x in args.values.split(",")]
    for row in sweep(w, values, args.pre, reps=args.reps, split=not args.no_split):
        row["cell"] = args.cell
        print(json.dumps(row), flush=True)
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
