"""Write the oracle's E, F and sigma for the full-size workloads.

Calls only oracle/ (and the seeded input generator for its inputs); the
stored values are what the GPU parity tests compare against at sizes the
oracle takes minutes for.  Run from the repository root:

    python tests/golden/make_golden.py si64
"""
import json
import os
import platform
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import evaluate  # noqa: E402
from paper_2412_11081_gb300 import inputs  # noqa: E402


def main(names):
    for name in names:
        w = inputs.workload_by_name(name)
        t = time.time()
        r = evaluate(w)
        dt = time.time() - t
        out = dict(workload=name, seed=w.seed, n_atoms=w.n_atoms, theta=w.theta, E=r.E,
                   F=r.F.tolist(), sigma=r.sigma.tolist(), counts=r.counts, flops=r.flops,
                   oracle_seconds=round(dt, 1), host=platform.machine())
        path = os.path.join(HERE, f"{name}_oracle.json")
        with open(path, "w") as f:
            json.dump(out, f, indent=1)
        print(name, f"{dt:.1f} s", "->", path)


if __name__ == "__main__":
    main(sys.argv[1:] or ["si64"])
