"""Write the oracle's E, F and sigma for the full-size workloads.

Calls only oracle/ (and the seeded input generator for its inputs); the
stored values are what the GPU parity tests compare against at sizes the
oracle takes minutes for.  Run from the repository root:

    python tests/golden/make_golden.py si64
    python tests/golden/make_golden.py si1000:0:4 perovskite1080:0:5

NAME:B:E stores the share of home atoms [B, E) (the sum over the home atom A
of Eq. exx_expand restricted to that range, OraclePlan.evaluate(homes=...)):
the oracle's per-structure part alone takes minutes at 1000 atoms, and a full
evaluation would take hours, so the 1000-atom cells are checked on a sample
of home atoms, compared with a plan over the same range.  Such a file is
named NAME_homes_B_E_oracle.json.
"""
import json
import os
import platform
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import OraclePlan  # noqa: E402
from paper_2412_11081_gb300 import inputs  # noqa: E402


def main(specs):
    for spec in specs:
        name, *rng = spec.split(":")
        w = inputs.workload_by_name(name)
        homes = list(range(int(rng[0]), int(rng[1]))) if rng else None
        t = time.time()
        r = OraclePlan(w).evaluate(homes=homes)
        dt = time.time() - t
        out = dict(workload=name, seed=w.seed, n_atoms=w.n_atoms, theta=w.theta, E=r.E,
                   F=r.F.tolist(), sigma=r.sigma.tolist(), counts=r.counts, flops=r.flops,
                   oracle_seconds=round(dt, 1), host=platform.machine())
        fname = f"{name}_oracle.json"
        if homes is not None:
            out["homes"] = [homes[0], homes[-1] + 1]
            fname = f"{name}_homes_{homes[0]}_{homes[-1] + 1}_oracle.json"
        path = os.path.join(HERE, fname)
        with open(path, "w") as f:
            json.dump(out, f, indent=1)
        print(spec, f"{dt:.1f} s", "->", path, flush=True)


if __name__ == "__main__":
    main(sys.argv[1:] or ["si64"])
