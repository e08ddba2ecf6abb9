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


@pytest.mark.parametrize("prec,orders,tol", [
    ("fp64", ([16, 4], [16], [2, 16]), 1e-11),
    ("fp64", ([4, 16], [2, 8], [16, 2]), 1e-11),
    ("fp32bulk", ([16, 4], [16], [2, 16]), 1e-5),
    ("fp32bulk", ([4, 16], [4, 4], [8, 4]), 1e-5),
])
def test_radix_orders_match_oracle(pfg, params, prec, orders, tol):
    """Every radix order (radix-16 stages first, last or alone) gives the
    oracle's step on a grid with unequal axes."""
    import oracle
    y0 = synth.ic_spheres(16, 2, 3.0, 4.0, 6, params)
    y0 = np.concatenate([y0, y0], axis=1)[:, :, :, :]           # nz = 32
    y0 = np.concatenate([y0, y0[:, :, :, ::-1]], axis=3)        # nx = 32
    y0 = np.concatenate([y0, y0[:, :, :, ::-1]], axis=3)        # nx = 64
    shape = y0.shape[1:]
    assert shape == (32, 16, 64)
    m = oracle.Model(shape, params)
    ref, _, _ = oracle.ark_step(m, m.to_k(y0), 0.5, oracle.ark436l2sa())
    with pfg.Simulation(shape, params, "ark4", prec) as s:
        cfg = s.tuning()
        for a, order in enumerate(orders):
            cfg[4 + 11 * a:4 + 11 * (a + 1)] = [len(order)] + order + [0] * (10 - len(order))
        s.set_tuning(cfg)
        assert s.tuning() == cfg
        s.set_state(y0)
        s.step(0.5)
        got = s.state_hat().cpu().numpy()
    for f in range(4):
        # a variant absent from this state is compared against the whole state
        den = np.linalg.norm(ref[f]) or np.linalg.norm(ref)
        err = np.linalg.norm(got[f] - ref[f]) / den
        assert err <= tol, (f, err)


@pytest.mark.parametrize("tx", [8, 16])
def test_compiled_plans_match_oracle(pfg, params, tx):
    """The kernels compiled for fixed lengths and radix orders (the FP32-bulk
    defaults of the workload sizes: z 96 = 8*4*3, y 64 = 16*4, x 128 = 16*8,
    and 256 = 16*16 along z in the second grid) against the oracle, for both
    tile widths that have compiled variants."""
    import oracle
    for shape in [(96, 64, 128), (256, 16, 32)]:
        nz, ny, nx = shape
        rng = np.random.default_rng(7)
        nuc = synth.draw_nuclei(shape, 6, rng, lambda r, v: (3.5, 3.5, 3.5))
        y0 = synth.nuclei_ic(shape, params, nuc, x_inside=params["B_v"])
        m = oracle.Model(shape, params)
        ref, _, _ = oracle.ark_step(m, m.to_k(y0), 0.5, oracle.ark436l2sa())
        with pfg.Simulation(shape, params, "ark4", "fp32bulk") as s:
            cfg = s.tuning()
            cfg[0], cfg[1], cfg[2], cfg[37] = tx, tx, 8, tx  # z, y, elastic and forward-z tile widths
            s.set_tuning(cfg)
            s.set_state(y0)
            s.step(0.5)
            got = s.state_hat().cpu().numpy()
        for f in range(4):
            den = np.linalg.norm(ref[f]) or np.linalg.norm(ref)
            err = np.linalg.norm(got[f] - ref[f]) / den
            assert err <= 1e-5, (shape, f, err)


def test_compiled_x_plans_fp64_match_oracle(pfg, params):
    """FP64 x passes with the compiled radix-8 plans (256 = 8*8*4, 128 =
    8*4*4, 160 = 8*4*5) against the oracle at the FP64 bar."""
    import oracle
    for nx in (256, 128, 160):
        shape = (12, 16, nx)
        rng = np.random.default_rng(nx)
        nuc = synth.draw_nuclei(shape, 3, rng, lambda r, v: (3.0, 3.0, 3.0))
        y0 = synth.nuclei_ic(shape, params, nuc, x_inside=params["B_v"])
        m = oracle.Model(shape, params)
        ref, _, _ = oracle.ark_step(m, m.to_k(y0), 0.5, oracle.ark436l2sa())
        with pfg.Simulation(shape, params, "ark4", "fp64") as s:
            s.set_state(y0)
            s.step(0.5)
            got = s.state_hat().cpu().numpy()
        for f in range(4):
            den = np.linalg.norm(ref[f]) or np.linalg.norm(ref)
            err = np.linalg.norm(got[f] - ref[f]) / den
            assert err <= 1e-11, (shape, f, err)
