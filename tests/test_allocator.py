"""hfx_options alloc / free: a plan whose device memory comes from
PyTorch's caching allocator gives the same results as one on cudaMalloc,
and its memory shows up in, and goes back to, that allocator."""
import numpy as np
import pytest

from paper_2412_11081_gb300 import hfx, inputs

pytestmark = pytest.mark.gpu


def rel(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("prec", [hfx.HFX_FP64, hfx.HFX_BF16X6])
def test_torch_allocator_plan(prec):
    torch = pytest.importorskip("torch")
    w = inputs.diamond8()
    with hfx.Plan(w, precision=prec) as p:
        ref = p.evaluate(w.lattice, w.positions)
    torch.cuda.synchronize()
    base = torch.cuda.memory_allocated()
    p = hfx.Plan(w, precision=prec, allocator="torch")
    try:
        for _ in range(2):   # the second call reuses the grown stores
            E, F, S = p.evaluate(w.lattice, w.positions, stats=True)
        used = torch.cuda.memory_allocated() - base
        assert used >= 0.9 * p.stats.device_bytes > 0
    finally:
        p.close()
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == base
    assert abs(E - ref[0]) <= 1e-12 * abs(ref[0]) and rel(F, ref[1]) <= 1e-12 and rel(S, ref[2]) <= 1e-12


def test_alloc_without_free_is_rejected():
    import ctypes as ct
    lib = hfx.load_library()
    hooks = hfx._torch_hooks(0)
    o = hfx.default_options()
    o.alloc = hooks[0]      # free left NULL
    h = ct.c_void_p()
    st = lib.hfx_plan_create(None, None, ct.byref(o), ct.byref(h))
    assert st == 1 and not h.value
