"""The allocation-free inverse transform (pf_state_to_real_noalloc) against
the context path (pf_set_state_hat + pf_get_state) through the C ABI.

It exists for callers that cannot allocate device memory and so cannot create
a context.  This file is collected last on purpose: its entry point shares
file-scope device arrays across calls, and the test must hold both when run
alone in a fresh process and after every other test."""
import ctypes as C

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pfg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2609_36100_gb300 as m
    m.build()
    return m


def _reference(pfg, shape, params, y):
    with pfg.Simulation(shape, params, "euler", "fp64") as s:
        s.set_state(y)
        yh = s.state_hat()
        ref = s.get_state()
    return yh, ref


@pytest.mark.parametrize("shape", [(12, 10, 20), (64, 64, 64)])
def test_noalloc_matches_context_path_twice(pfg, params, shape):
    import torch
    L = pfg.lib()
    nz, ny, nx = shape
    grid = pfg.PFGrid(nx, ny, nz, params["dx"], params["dx"], params["dx"])
    stream = torch.cuda.current_stream()
    for seed in (21, 22):  # two calls in a row, different inputs
        y = synth.random_state(shape, seed)
        yh, ref = _reference(pfg, shape, params, y)
        out = torch.full((4,) + shape, np.nan, dtype=torch.float64, device="cuda")
        rc = L.pf_state_to_real_noalloc(C.byref(grid), C.c_void_p(yh.data_ptr()), C.c_void_p(out.data_ptr()),
                                        C.c_void_p(stream.cuda_stream))
        assert rc == pfg.PF_OK, L.pf_last_error(None)
        got = out.cpu().numpy()
        # the transform tolerance of the parity tests
        assert np.max(np.abs(got - ref)) <= 1e-13
        assert np.max(np.abs(got - y)) <= 1e-13


def test_noalloc_rejects_oversize_grid(pfg, params):
    import torch
    L = pfg.lib()
    grid = pfg.PFGrid(72, 72, 72, 0.5, 0.5, 0.5)  # 72*72*37 > 135168
    dummy = torch.zeros(8, dtype=torch.float64, device="cuda")
    rc = L.pf_state_to_real_noalloc(C.byref(grid), C.c_void_p(dummy.data_ptr()), C.c_void_p(dummy.data_ptr()), None)
    assert rc == pfg.PF_EINVAL
    assert b"too large" in L.pf_last_error(None)
