"""Ensemble batching (pf_batch_advance): members of uneven grids and
temperatures advanced together (one device-looped graph launch, or the
host-polled round graph) must give what each member's own pf_advance gives
(same attempt counts, same states to rounding), and an FP64 member must
still match the oracle."""
import numpy as np
import pytest

import oracle
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


def members(params, n=4):
    out = []
    specs = [((16, 16, 16), 0.0), ((24, 20, 30), 12.0), ((32, 32, 32), -15.0), ((12, 10, 20), 5.0)][:n]
    for k, (shape, dT) in enumerate(specs):
        p = dict(params)
        p["T"] = p["T0"] + dT
        y0 = synth.random_state(shape, 40 + k, phi_scale=0.9) if shape[0] != shape[1] else \
            synth.ic_spheres(shape[0], 2, 3.0, 4.5, 50 + k, p)
        out.append((shape, p, y0))
    return out


def relerr(a, b):
    return max(np.linalg.norm((a[f] - b[f]).ravel()) / max(np.linalg.norm(b[f].ravel()), 1e-300)
               for f in range(a.shape[0]))


@pytest.mark.parametrize("prec", ["fp64", "fp32bulk"])
def test_batch_equals_individual_advance(pfg, params, prec):
    ms = members(params)
    t_final = 4.0
    singles = []
    for shape, p, y0 in ms:
        with pfg.Simulation(shape, p, "ark4", prec) as s:
            s.set_state(y0)
            st = s.advance(t_final, 1e-4, 1e-8)
            singles.append((s.state_hat().cpu().numpy(), st))
    sims = [pfg.Simulation(shape, p, "ark4", prec) for shape, p, _ in ms]
    try:
        for s, (_, _, y0) in zip(sims, ms):
            s.set_state(y0)
        stats = pfg.batch_advance(sims, t_final, 1e-4, 1e-8)
        for s, st, (ref, st1) in zip(sims, stats, singles):
            assert st["t"] == pytest.approx(t_final, rel=1e-14)
            assert st["steps_accepted"] == st1["steps_accepted"]
            assert st["steps_rejected"] == st1["steps_rejected"]
            assert st["rhs_evals"] == st1["rhs_evals"]
            # FP64: rounding-level agreement; FP32-bulk: the device and host
            # controllers may differ in the last bit of dt, which FP32
            # transforms turn into FP32-level differences
            assert relerr(s.state_hat().cpu().numpy(), ref) <= (1e-12 if prec == "fp64" else 1e-5)
    finally:
        for s in sims:
            s.close()


def test_batch_member_matches_oracle(pfg, params):
    ms = members(params, 2)
    sims = [pfg.Simulation(shape, p, "ark4", "fp64") for shape, p, _ in ms]
    try:
        for s, (_, _, y0) in zip(sims, ms):
            s.set_state(y0)
        pfg.batch_advance(sims, 3.0, 1e-4, 1e-8)
        for s, (shape, p, y0) in zip(sims, ms):
            m = oracle.Model(shape, p)
            yh, t, log = oracle.advance(m, m.to_k(y0), 0.0, 3.0, oracle.ark436l2sa(), p, 1e-4, 1e-8)
            assert t == pytest.approx(3.0, rel=1e-14)
            assert relerr(s.state_hat().cpu().numpy(), yh) <= 1e-11
    finally:
        for s in sims:
            s.close()


def test_batch_euler_fixed_steps(pfg, params):
    p = dict(params, h0=0.25)
    ms = members(p, 3)
    sims = [pfg.Simulation(shape, q, "euler", "fp64") for shape, q, _ in ms]
    try:
        for s, (_, _, y0) in zip(sims, ms):
            s.set_state(y0)
        stats = pfg.batch_advance(sims, 2.0)
        for s, st, (shape, q, y0) in zip(sims, stats, ms):
            assert st["steps_accepted"] == 8 and st["steps_rejected"] == 0
            m = oracle.Model(shape, q)
            yh = m.to_k(y0)
            for _ in range(8):
                yh, _, _ = oracle.ark_step(m, yh, 0.25, oracle.euler())
            assert relerr(s.state_hat().cpu().numpy(), yh) <= 1e-11
    finally:
        for s in sims:
            s.close()


def test_batch_rejects_mixed_methods(pfg, params):
    a = pfg.Simulation((8, 8, 8), params, "ark4", "fp64")
    b = pfg.Simulation((8, 8, 8), params, "euler", "fp64")
    try:
        with pytest.raises(pfg.PFError):
            pfg.batch_advance([a, b], 1.0)
    finally:
        a.close()
        b.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32bulk"])
def test_batch_device_looped_equals_polled(pfg, params, prec):
    """The device-looped driver runs the same rounds as the host-polled one
    and gives bitwise the same states; members that finish early skip their
    rounds (attempt counts per member unchanged)."""
    ms = members(params)
    out = {}
    for polled in (False, True):
        sims = [pfg.Simulation(shape, p, "ark4", prec) for shape, p, _ in ms]
        try:
            for s, (_, _, y0) in zip(sims, ms):
                s.set_state(y0)
            stats = pfg.batch_advance(sims, 4.0, 1e-4, 1e-8, polled=polled)
            rounds, looped = pfg.batch_last()
            out[polled] = ([s.state_hat().cpu().numpy() for s in sims], stats, rounds, looped)
        finally:
            for s in sims:
                s.close()
    states_l, stats_l, rounds_l, looped_l = out[False]
    states_p, stats_p, rounds_p, looped_p = out[True]
    assert looped_l and not looped_p
    attempts = [st["steps_accepted"] + st["steps_rejected"] for st in stats_l]
    assert rounds_l == max(attempts)          # the loop ends with the last live member
    assert rounds_p >= rounds_l               # the polled driver checks every two rounds
    for a, b, sa, sb in zip(states_l, states_p, stats_l, stats_p):
        assert np.array_equal(a, b)
        assert sa["steps_accepted"] == sb["steps_accepted"] and sa["steps_rejected"] == sb["steps_rejected"]


def test_batch_with_cluster_elastic_pass(pfg, params):
    """FP32-bulk members whose z length has a compiled plan, each running the
    elastic pass as a three-CTA cluster (tuning slot 40 = 2): batched, with
    members that finish early skipping their rounds (whole clusters return
    together), they give what each member's own pf_advance gives."""
    specs = [((64, 8, 12), 0), ((96, 10, 16), 1), ((64, 6, 20), 2)]
    t_final = 6.0

    def prepared(shape, k):
        s = pfg.Simulation(shape, params, "ark4", "fp32bulk")
        cfg = s.tuning()
        cfg[38] = {64: 5, 96: 8}[shape[0]]  # compiled plans of length nz
        cfg[40] = 2
        s.set_tuning(cfg)
        assert s.tuning()[40] == 2
        s.set_state(synth.random_state(shape, 70 + k, phi_scale=0.9))
        return s

    singles = []
    for shape, k in specs:
        with prepared(shape, k) as s:
            st = s.advance(t_final, 1e-4, 1e-8)
            singles.append((s.state_hat().cpu().numpy(), st))
    sims = [prepared(shape, k) for shape, k in specs]
    try:
        stats = pfg.batch_advance(sims, t_final, 1e-4, 1e-8)
        for s, st, (ref, st1) in zip(sims, stats, singles):
            assert st["steps_accepted"] == st1["steps_accepted"]
            assert st["steps_rejected"] == st1["steps_rejected"]
            assert relerr(s.state_hat().cpu().numpy(), ref) <= 1e-5
    finally:
        for s in sims:
            s.close()
