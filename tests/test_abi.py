"""The C-ABI library loads and exports every symbol include/hfx.h declares;
argument validation that happens before any CUDA call (no GPU needed)."""
import ctypes as ct
import os
import re

import numpy as np
import pytest

from paper_2412_11081_gb300 import hfx, inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(hfx.LIB_PATH):
        from paper_2412_11081_gb300 import build
        build.build()
    return hfx.load_library()


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "hfx.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(hfx_\w+)\s*\(", txt)))


def test_header_declares_the_abi():
    names = declared_symbols()
    for must in ("hfx_plan_create", "hfx_energy_force_stress", "hfx_plan_destroy"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing
    # the binding binds exactly the declared set
    assert set(hfx._SIGNATURES) == set(declared_symbols())


def test_status_strings(lib):
    for s in range(7):
        assert lib.hfx_status_string(s)
    assert lib.hfx_status_string(99) == b"unknown status"


def test_default_options(lib):
    o = hfx.default_options()
    assert o.theta_CS == 1e-10 and o.precision == hfx.HFX_FP64 and o.terms == 3 and o.skin == 0.5
    assert o.home_begin == 0 and o.home_end == 0 and o.home_chunk == 0
    assert o.graph == 0 and o.deterministic == 0
    # the binding's copy of hfx_options ends where the C struct does: a
    # default-filled struct with a canary after it keeps the canary
    import ctypes as ct

    class Guarded(ct.Structure):
        _fields_ = [("o", hfx.HfxOptions), ("canary", ct.c_uint64)]

    g = Guarded()
    g.canary = 0x5A5A5A5A5A5A5A5A
    assert lib.hfx_default_options(ct.byref(g.o)) == 0 and g.canary == 0x5A5A5A5A5A5A5A5A
    assert lib.hfx_default_options(None) == 1


def _create(lib, w, **kw):
    """hfx_plan_create with optional corruption of the marshalled inputs."""
    species = np.ascontiguousarray(w.species, dtype=np.int32)
    pos = np.ascontiguousarray(w.positions, dtype=np.float64)
    if "positions" in kw:
        pos = np.ascontiguousarray(kw.pop("positions"), dtype=np.float64)
    sysm = hfx.HfxSystem(n_atoms=species.shape[0], species=species.ctypes.data_as(hfx._ip),
                         lattice=(ct.c_double * 9)(*np.asarray(kw.pop("lattice", w.lattice)).ravel()),
                         positions=pos.ctypes.data_as(hfx._dp))
    S = w.n_ao.shape[0]
    G = [np.ascontiguousarray(g) for g in w.G]
    M = [np.ascontiguousarray(m) for m in w.M]
    n_ao = np.ascontiguousarray(w.n_ao, dtype=np.int32)
    n_abf = np.ascontiguousarray(w.n_abf, dtype=np.int32)
    model = hfx.HfxModel(n_species=S, n_ao=n_ao.ctypes.data_as(hfx._ip), n_abf=n_abf.ctypes.data_as(hfx._ip),
                         r_c=kw.pop("r_c", w.r_c), omega=w.omega,
                         G=(hfx._dp * (S * S))(*[g.ctypes.data_as(hfx._dp) for g in G]),
                         M=(hfx._dp * (S * S))(*[m.ctypes.data_as(hfx._dp) for m in M]))
    opts = hfx.default_options(**kw)
    h = ct.c_void_p()
    st = lib.hfx_plan_create(ct.byref(sysm), ct.byref(model), ct.byref(opts), ct.byref(h))
    if st == 0:
        lib.hfx_plan_destroy(h)
    return st


def test_invalid_arguments_rejected_before_any_device_work(lib):
    w = inputs.cut_density(inputs.diamond8(), 4.0)
    assert lib.hfx_plan_create(None, None, None, None) == 1
    assert _create(lib, w, theta_CS=-1.0) == 1                    # negative threshold
    assert _create(lib, w, terms=0) == 1                          # no exchange product
    assert _create(lib, w, precision=7) == 6                      # unknown precision
    assert _create(lib, w, precision=1) == 6                      # unassigned precision value
    assert _create(lib, w, home_begin=3, home_end=3) == 1         # empty home-atom range
    assert _create(lib, w, home_begin=0, home_end=9) == 1         # range past n_atoms (8)
    assert _create(lib, w, home_begin=-1, home_end=4) == 1
    assert _create(lib, w, home_chunk=-2) == 1
    assert _create(lib, w, r_c=float("nan")) == 1                 # non-finite model
    bad = w.positions.copy()
    bad[2, 1] = float("inf")
    assert _create(lib, w, positions=bad) == 1                    # non-finite positions
    assert _create(lib, w, lattice=np.zeros(9)) == 1              # singular lattice
    assert b"singular" in lib.hfx_last_error(None)


def test_destroy_null_is_ok(lib):
    assert lib.hfx_plan_destroy(None) == 0
