"""Deterministic reduction (hfx_options.deterministic).

The force and stress are sums over pairs of the pair gradients of Eq. Fexx1
(Sec. 2, Eq. stress); on the GPU many CTAs add to the same sums.  With the
option set, every such sum is an exact fixed-point integer, so the result
must not depend on how the work is split or ordered: repeated calls, other
passes of home atoms, the launch shapes the autotuner picks and a replayed
CUDA graph must all give the same bits, and the values must agree with the
FP64 atomic sums to rounding.
"""
import numpy as np
import pytest

from paper_2412_11081_gb300 import hfx, inputs

pytestmark = pytest.mark.gpu


def rel(a, ref):
    a, ref = np.asarray(a, float), np.asarray(ref, float)
    return float(np.max(np.abs(a - ref)) / np.max(np.abs(ref)))


def same_bits(x, y):
    return all(np.array_equal(np.asarray(a, float).view(np.int64), np.asarray(b, float).view(np.int64))
               for a, b in zip(x, y))


CASES = [
    ("diamond8 fp64", inputs.diamond8, hfx.HFX_FP64, {}),
    ("si8 bf16x6", lambda: inputs.si_supercell(1), hfx.HFX_BF16X6, {}),
    # the warp-level first product and R2 / Z kernels (their shared-memory
    # partial sums go straight into the exact cells)
    ("si8 bf16x6 warp-level", lambda: inputs.si_supercell(1), hfx.HFX_BF16X6,
     {"HFX_T1_KERNEL": "mma", "HFX_T2_KERNEL": "mma"}),
    ("perovskite bf16x6 wide", lambda: inputs.perovskite_supercell(1), hfx.HFX_BF16X6, {}),
]


@pytest.mark.parametrize("name,make,prec,env", CASES, ids=[c[0] for c in CASES])
def test_same_bits_for_any_split_or_order(name, make, prec, env, monkeypatch):
    for k, v in env.items():
        monkeypatch.setenv(k, v)
    w = make()
    pos = inputs.geometry_sequence(w, 2, seed=11)[1]
    with hfx.Plan(w, precision=prec) as p:
        ref = p.evaluate(w.lattice, pos)
    with hfx.Plan(w, precision=prec, deterministic=True) as p:
        a1 = p.evaluate(w.lattice, pos)
        a2 = p.evaluate(w.lattice, pos)
    assert same_bits(a1, a2), name
    # one pass per home atom (the sums collect their parts in another order)
    with hfx.Plan(w, precision=prec, deterministic=True, home_chunk=1) as p:
        b = p.evaluate(w.lattice, pos, stats=True)
        assert p.stats.passes == len(w.species)
    assert same_bits(a1, b), name
    # launch shapes of the autotuner (ring shape, item order, tiles per CTA)
    with hfx.Plan(w, precision=prec, deterministic=True) as p:
        p.autotune(w.lattice, pos, reps=1)
        c = p.evaluate(w.lattice, pos)
    assert same_bits(a1, c), name
    E, F, S = a1
    assert abs(E - ref[0]) <= 1e-13 * abs(ref[0])
    assert rel(F, ref[1]) <= 1e-13 and rel(S, ref[2]) <= 1e-13


def test_graph_replay_same_bits():
    w = inputs.si_supercell(1)
    seq = inputs.geometry_sequence(w, 4, seed=12)
    with hfx.Plan(w, precision=hfx.HFX_BF16X6, deterministic=True, freeze_lists=True) as p:
        direct = [p.evaluate(w.lattice, x) for x in seq]
    with hfx.Plan(w, precision=hfx.HFX_BF16X6, deterministic=True, freeze_lists=True, graph=True) as p:
        replayed = [p.evaluate(w.lattice, x, stats=True) for x in seq]
        assert p.stats.graph_replayed == 1
    for d, r in zip(direct, replayed):
        assert same_bits(d, r)
