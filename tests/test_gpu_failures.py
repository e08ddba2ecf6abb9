"""Failure detection and checkpoint/resume through the C ABI (errors made on
the host side: bad input, impossible tolerances, a capped batch loop; no GPU
fault is provoked)."""
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


def to_np(t):
    return t.detach().cpu().numpy()


@pytest.mark.parametrize("prec", ["fp64", "fp32bulk"])
def test_nonfinite_input_refused_state_kept(pfg, params, prec):
    y0 = synth.ic_spheres(16, 2, 2.5, 3.5, 4, params)
    with pfg.Simulation(y0.shape[1:], params, "ark4", prec) as s:
        s.set_state(y0)
        before = to_np(s.state_hat())
        bad = y0.copy()
        bad[2, 3, 4, 5] = np.nan
        with pytest.raises(pfg.PFError) as ei:
            s.set_state(bad)
        assert ei.value.code == pfg.PF_ENONFINITE
        bad[2, 3, 4, 5] = np.inf
        with pytest.raises(pfg.PFError) as ei:
            s.set_state(bad)
        assert ei.value.code == pfg.PF_ENONFINITE
        yb = before.copy()
        yb[1, 2, 3, 4] = complex(np.nan, 0.0)
        with pytest.raises(pfg.PFError) as ei:
            s.set_state_hat(yb)
        assert ei.value.code == pfg.PF_ENONFINITE
        assert np.array_equal(to_np(s.state_hat()), before)
        s.step(0.25)  # the context is still usable


@pytest.mark.parametrize("prec", ["fp64", "fp32bulk"])
def test_impossible_tolerance_fails_with_state_intact(pfg, params, prec):
    """rtol = 0 and atol = 1e-30 make every attempt fail its error test: after
    max_rejects rejections the call returns PF_ESTEPFAIL with the last
    accepted state and clock untouched, and the context keeps working."""
    y0 = synth.ic_spheres(16, 2, 2.5, 3.5, 4, params)
    with pfg.Simulation(y0.shape[1:], params, "ark4", prec) as s:
        s.set_state(y0)
        s.advance(2.0, 1e-4, 1e-8)
        t0, _ = s.time()
        before = to_np(s.state_hat())
        with pytest.raises(pfg.PFError) as ei:
            s.advance(10.0, 0.0, 1e-30)
        assert ei.value.code == pfg.PF_ESTEPFAIL
        att = s.attempts()
        assert len(att) == params["max_rejects"] + 1 and not any(ok for *_, ok in att)
        assert s.time()[0] == t0
        assert np.array_equal(to_np(s.state_hat()), before)
        st = s.advance(3.0, 1e-4, 1e-8)
        assert st["t"] == pytest.approx(3.0, rel=1e-14)


@pytest.mark.parametrize("prec", ["fp64", "fp32bulk"])
def test_checkpoint_resume_bitwise(pfg, params, prec):
    """Adaptive run to t = 12 s in one go, against a run checkpointed at
    t = 5 s (k-space state, clock, controller history) and resumed in a fresh
    context: identical attempts and a bitwise-identical final state."""
    y0 = synth.ic_spheres(24, 3, 2.5, 4.0, 6, params)
    with pfg.Simulation(y0.shape[1:], params, "ark4", prec) as a:
        a.set_state(y0)
        a.set_time(0.0, 0.5)
        a.advance(5.0, 1e-4, 1e-8)
        ck = a.checkpoint()
        a.advance(12.0, 1e-4, 1e-8)
        att_a = a.attempts()
        ya = to_np(a.state_hat())
    with pfg.Simulation(y0.shape[1:], params, "ark4", prec) as b:
        b.restore(ck)
        b.advance(12.0, 1e-4, 1e-8)
        att_b = b.attempts()
        yb = to_np(b.state_hat())
    assert att_a == att_b
    assert np.array_equal(ya, yb)


def test_fixed_steps_resume_bitwise(pfg, params):
    y0 = synth.ic_ellipsoids(32, 1, params, count=4)
    with pfg.Simulation(y0.shape[1:], params, "euler", "fp64") as a:
        a.set_state(y0)
        for _ in range(10):
            a.step(0.25, want_lte=False)
        ya = to_np(a.state_hat())
    with pfg.Simulation(y0.shape[1:], params, "euler", "fp64") as b:
        b.set_state(y0)
        for _ in range(4):
            b.step(0.25, want_lte=False)
        ck = b.checkpoint()
    with pfg.Simulation(y0.shape[1:], params, "euler", "fp64") as c:
        c.restore(ck)
        for _ in range(6):
            c.step(0.25, want_lte=False)
        yc = to_np(c.state_hat())
        assert c.time()[0] == pytest.approx(2.5, rel=1e-15)
    assert np.array_equal(ya, yc)


@pytest.mark.parametrize("polled", [False, True])
def test_batch_round_cap_times_out_and_resumes(pfg, params, polled):
    """A batch stopped by the round cap returns PF_ETIMEOUT with every member
    at its last accepted state and clock; continuing it to t_final gives the
    same states, bitwise, as one uninterrupted batch."""
    ys = [synth.ic_spheres(n, 2, 2.5, 3.5, 20 + n, params) for n in (16, 24, 16)]

    def make():
        sims = []
        for y in ys:
            s = pfg.Simulation(y.shape[1:], params, "ark4", "fp32bulk")
            s.set_state(y)
            s.set_time(0.0, 0.5)
            sims.append(s)
        return sims

    ref = make()
    pfg.batch_advance(ref, 20.0, 1e-4, 1e-8, polled=polled)
    want = [to_np(s.state_hat()) for s in ref]
    for s in ref:
        s.close()
    sims = make()
    prev = pfg.batch_round_cap(3)
    try:
        with pytest.raises(pfg.PFError) as ei:
            pfg.batch_advance(sims, 20.0, 1e-4, 1e-8, polled=polled)
        assert ei.value.code == pfg.PF_ETIMEOUT
    finally:
        pfg.batch_round_cap(prev)
    ts = [s.time()[0] for s in sims]
    assert all(0.0 < t < 20.0 for t in ts), ts
    pfg.batch_advance(sims, 20.0, 1e-4, 1e-8, polled=polled)
    for s, w in zip(sims, want):
        assert s.time()[0] == pytest.approx(20.0, rel=1e-14)
        assert np.array_equal(to_np(s.state_hat()), w)
        s.close()


def test_checkpoint_resume_with_hu_chen_warm_start(pfg, params):
    """With the phase-dependent stiffness and its warm start the carried
    eps(u) is not part of a checkpoint: a resumed context starts its first
    solve cold.  The resumed run then continues within the elastic
    tolerance's reach of the uninterrupted one, not bitwise; with el_warm = 0
    it is bitwise again."""
    base = dict(params, el_inhom=1, C11_v=1.3 * params["C11"], C12_v=1.1 * params["C12"],
                C44_v=1.2 * params["C44"], el_tol=1e-8, el_max_iter=100)
    y0 = synth.ic_spheres(16, 2, 2.5, 3.5, 7, params)
    for warm in (1, 0):
        p = dict(base, el_warm=warm)
        with pfg.Simulation(y0.shape[1:], p, "ark4", "fp64") as a:
            a.set_state(y0)
            a.set_time(0.0, 0.5)
            a.advance(2.0, 1e-4, 1e-8)
            ck = a.checkpoint()
            a.advance(4.0, 1e-4, 1e-8)
            ya = to_np(a.state_hat())
        with pfg.Simulation(y0.shape[1:], p, "ark4", "fp64") as b:
            b.restore(ck)
            b.advance(4.0, 1e-4, 1e-8)
            yb = to_np(b.state_hat())
        if warm:
            d = np.linalg.norm((ya - yb).ravel()) / np.linalg.norm(ya.ravel())
            assert d <= 1e-6, d
        else:
            assert np.array_equal(ya, yb)
