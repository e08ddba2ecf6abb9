"""C-ABI library checks that need no GPU: it builds, loads, exports every
symbol include/pf.h declares, and its host-side logic (tableau, argument
validation) is right."""
import os
import re

import numpy as np
import pytest

import paper_2609_36100_gb300 as pfg
from tests.order_conditions import max_violation

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    pfg.build()
    return pfg.lib()


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "pf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pf_[a-z_]+)\s*\(", src)))


def test_header_symbols_exported(L):
    names = declared_symbols()
    assert "pf_create" in names and "pf_batch_advance" in names
    for n in names:
        assert hasattr(L, n), n
    # the binding declares every header entry point
    assert set(names) == set(pfg.SIGNATURES)


def test_build_compiles_every_translation_unit():
    # every .cu under csrc/ is one translation unit of libpf.so, and the
    # source list names no missing file
    import importlib
    B = importlib.import_module("paper_2609_36100_gb300.build")
    units = sorted(f for f in os.listdir(B.CSRC) if f.endswith(".cu"))
    assert sorted(B.SOURCES) == units


def test_library_tableau_order_conditions(L):
    AE, AI, bE, bI, btE, btI = pfg.method_tableau("ark4")
    assert AE.shape == (6, 6)
    assert max_violation(AE, AI, bE, bI, 4) < 1e-14
    assert max_violation(AE, AI, btE, btI, 3) < 1e-14
    AE, AI, bE, bI, _, _ = pfg.method_tableau("euler")
    assert max_violation(AE, AI, bE, bI, 1) < 1e-15
    for name, p in [("ark2", 2), ("ark3", 3)]:
        AE, AI, bE, bI, btE, btI = pfg.method_tableau(name)
        assert AE.shape == ({"ark2": 3, "ark3": 4}[name],) * 2
        assert max_violation(AE, AI, bE, bI, p) < 1e-14
        assert max_violation(AE, AI, btE, btI, p - 1) < 1e-14
        assert max_violation(AE, AI, btE, btI, p) > 1e-3


def test_library_and_oracle_tables_agree(L):
    """The two typed copies of every table (library and oracle) agree to
    rounding: a mistyped digit in either shows here as well as in the order
    conditions."""
    import oracle
    for name in ("euler", "ark2", "ark3", "ark4"):
        AE, AI, bE, bI, btE, btI = pfg.method_tableau(name)
        t = oracle.TABLES[name]()
        assert np.max(np.abs(AE - t.AE)) <= 4e-16 and np.max(np.abs(AI - t.AI)) <= 4e-16
        assert np.max(np.abs(bE - t.bE)) <= 4e-16 and np.max(np.abs(bI - t.bI)) <= 4e-16
        if t.btE is not None:
            assert np.max(np.abs(btE - t.btE)) <= 4e-16 and np.max(np.abs(btI - t.btI)) <= 4e-16


def test_batch_round_cap_query_and_set(L):
    prev = pfg.batch_round_cap(0)
    assert prev == 1 << 20
    assert pfg.batch_round_cap(5) == prev
    assert pfg.batch_round_cap(0) == 5
    pfg.batch_round_cap(prev)
    assert pfg.batch_round_cap(0) == prev


def test_unknown_method_rejected(L):
    import ctypes as C
    bufs = [(C.c_double * 64)() for _ in range(6)]
    assert L.pf_method_tableau(7, *[C.cast(b, C.POINTER(C.c_double)) for b in bufs]) == pfg.PF_EUNSUPPORTED


@pytest.mark.parametrize("shape", [(64, 64, 7), (64, 14, 64), (2, 8, 8), (2048, 8, 8), (8, 8, 22)])
def test_create_rejects_unsupported_sizes(L, params, shape):
    import ctypes as C
    nz, ny, nx = shape
    g = pfg.PFGrid(nx, ny, nz, 0.5, 0.5, 0.5)
    prm = pfg.make_params(params)
    ctx = C.c_void_p()
    rc = L.pf_create(C.byref(g), C.byref(prm), None, C.byref(ctx))
    assert rc == pfg.PF_EUNSUPPORTED
    assert ctx.value is None
    assert b"2,3,5-smooth" in L.pf_last_error(None)


def test_create_rejects_bad_parameters(L, params):
    import ctypes as C
    g = pfg.PFGrid(8, 8, 8, 0.5, 0.5, 0.5)
    prm = pfg.make_params(params)
    prm.precision = 9
    ctx = C.c_void_p()
    assert L.pf_create(C.byref(g), C.byref(prm), None, C.byref(ctx)) == pfg.PF_EINVAL
    prm = pfg.make_params(params)
    prm.A_m = -1.0
    assert L.pf_create(C.byref(g), C.byref(prm), None, C.byref(ctx)) == pfg.PF_EINVAL
    g2 = pfg.PFGrid(8, 8, 8, 0.0, 0.5, 0.5)
    assert L.pf_create(C.byref(g2), C.byref(pfg.make_params(params)), None, C.byref(ctx)) == pfg.PF_EINVAL


def test_null_arguments_rejected(L):
    assert L.pf_create(None, None, None, None) == pfg.PF_EINVAL
    assert L.pf_set_state(None, None, 0) == pfg.PF_EINVAL
    assert L.pf_step(None, 1.0, None) == pfg.PF_EINVAL
