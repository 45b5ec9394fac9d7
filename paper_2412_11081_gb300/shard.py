"""Home-atom sharding of one evaluation over processes, one GPU each.

Eq. exx_expand sums over the atom A of the home cell, and every item (an
(A, B, F) triplet or an (A, B) pair) belongs to one A.  The paper
distributes the atom quartets over processes, redistributes the tensors
once and sums the forces at the end, with no communication inside the loop
(Sec. 3.3).  Here each rank's plan takes a contiguous range of home atoms
(hfx_options home_begin / home_end): it regenerates every block it needs
from the positions and the model, evaluates its share of E, F and sigma, and
one all-reduce (sum) of the 1 + 3 n_atoms + 9 doubles finishes the step.
That all-reduce is the only exchange.
"""
from __future__ import annotations

from typing import Callable, List, Optional, Tuple

import numpy as np


def home_ranges(n_atoms: int, world: int) -> List[Tuple[int, int]]:
    """Contiguous, near-equal ranges of home atoms, one per rank, covering
    [0, n_atoms) in order.  Every range is non-empty (world <= n_atoms)."""
    if world < 1 or n_atoms < world:
        raise ValueError(f"cannot split {n_atoms} home atoms over {world} ranks")
    return [(n_atoms * r // world, n_atoms * (r + 1) // world) for r in range(world)]


def pack(E: float, F, sigma) -> np.ndarray:
    """[E, F (n x 3, row-major), sigma (3 x 3, row-major)] as one vector."""
    return np.concatenate([[float(E)], np.asarray(F, float).ravel(), np.asarray(sigma, float).ravel()])


def unpack(v, n_atoms: int):
    v = np.asarray(v, float)
    return float(v[0]), v[1:1 + 3 * n_atoms].reshape(n_atoms, 3), v[1 + 3 * n_atoms:].reshape(3, 3)


class ShardedPlan:
    """One rank's share of a structure: a plan over its home-atom range and
    the all-reduce that sums the shares.

    `group` is a torch.distributed process group (None = the default one);
    with the NCCL backend the sum runs on the rank's GPU, with gloo on the
    host.  `plan_factory(w, home=(begin, end), **plan_kw)` makes the plan
    (hfx.Plan by default)."""

    def __init__(self, w, rank: int, world: int, *, group=None, plan_factory: Optional[Callable] = None,
                 **plan_kw):
        if plan_factory is None:
            from . import hfx
            plan_factory = hfx.Plan
        self.n_atoms = int(np.asarray(w.species).shape[0])
        self.rank, self.world, self.group = rank, world, group
        self.home = home_ranges(self.n_atoms, world)[rank]
        self.plan = plan_factory(w, home=self.home, **plan_kw)

    def share(self, lattice, positions):
        """This rank's share (E, F, sigma), before the sum."""
        return self.plan.evaluate(lattice, positions)

    def evaluate(self, lattice, positions):
        """E, F, sigma of the whole structure: the shares summed over the ranks."""
        import torch
        import torch.distributed as dist
        v = torch.from_numpy(pack(*self.share(lattice, positions)))
        if dist.get_backend(self.group) == "nccl":
            v = v.cuda()
        dist.all_reduce(v, op=dist.ReduceOp.SUM, group=self.group)
        return unpack(v.cpu().numpy(), self.n_atoms)

    def close(self):
        self.plan.close()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
