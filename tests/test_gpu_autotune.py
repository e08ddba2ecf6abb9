"""Autotuner: it keeps the fastest schedule it timed, the tuned schedule
computes the same step (to rounding), schedules round-trip through
get/set, and invalid radix orders are refused."""
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


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-13), ("fp32bulk", 1e-6)])
def test_autotune_keeps_results(pfg, params, prec, tol):
    y0 = synth.ic_spheres(48, 3, 3.0, 5.0, 4, params)
    shape = y0.shape[1:]
    with pfg.Simulation(shape, params, "ark4", prec) as a:
        a.set_state(y0)
        e_ref = a.step(0.5)
        ref = a.state_hat().cpu().numpy()
    with pfg.Simulation(shape, params, "ark4", prec) as b:
        b.set_state(y0)
        rec = b.autotune(reps=1)
        assert rec["ms_after"] <= rec["ms_before"] * 1.0001
        e = b.step(0.5)
        got = b.state_hat().cpu().numpy()
        cfg = b.tuning()
        b.set_tuning(cfg)
        assert b.tuning() == cfg
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= tol
    assert e == pytest.approx(e_ref, rel=1e-4 if prec == "fp32bulk" else 1e-8)


def test_bad_radix_order_refused(pfg, params):
    with pfg.Simulation((16, 16, 16), params, "ark4", "fp64") as s:
        cfg = s.tuning()
        cfg[4:4 + 11] = [2, 8, 4] + [0] * 8  # 8 * 4 = 32 != 16
        with pytest.raises(pfg.PFError):
            s.set_tuning(cfg)
