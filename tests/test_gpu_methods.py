"""The second- and third-order members of the ImEx-ARK family (Sec. 4.4:
ARK2 of Giraldo et al. and ARK3(2)4L[2]SA) through the C ABI against the FP64
oracle, and the FP32-bulk error estimate against the FP64 one."""
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


def relerr(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return np.array([np.linalg.norm((a[f] - b[f]).ravel()) / max(np.linalg.norm(b[f].ravel()), 1e-300)
                     for f in range(a.shape[0])])


def to_np(t):
    return t.detach().cpu().numpy()


@pytest.mark.parametrize("meth", ["ark2", "ark3"])
@pytest.mark.parametrize("shape", [(32, 32, 32), (24, 20, 30)])
def test_steps_and_lte_vs_oracle(pfg, params, meth, shape):
    """Four fixed steps of 0.5 s: state rel L2 <= 1e-11 per field, the WRMS
    norms of the embedded error estimates to 1e-9 relative (FP64)."""
    if shape[0] == shape[1] == shape[2]:
        y0 = synth.ic_spheres(shape[0], 3, 3.0, 5.0, 9, params)
    else:
        y0 = synth.random_state(shape, 5, phi_scale=0.9)
    m = oracle.Model(shape, params)
    yh = m.to_k(y0)
    tab = oracle.TABLES[meth]()
    errs = []
    for _ in range(4):
        yh, e, _ = oracle.ark_step(m, yh, 0.5, tab, params["rtol"], params["atol"])
        errs.append(e)
    with pfg.Simulation(shape, params, meth, "fp64") as s:
        s.set_state(y0)
        dc = to_np(s.state_hat())[0, 0, 0, 0]
        got_e = [s.step(0.5) for _ in range(4)]
        got = to_np(s.state_hat())
        st = s.stats()
    assert got[0, 0, 0, 0] == dc
    assert np.all(relerr(got, yh) <= 1e-11), relerr(got, yh)
    np.testing.assert_allclose(got_e, errs, rtol=1e-9)
    assert st["rhs_evals"] == 4 * {"ark2": 3, "ark3": 4}[meth]  # Sec. 4.4: 3 and 4 per step


@pytest.mark.parametrize("meth", ["ark2", "ark3"])
def test_fp32bulk_steps(pfg, params, meth):
    y0 = synth.ic_spheres(32, 3, 3.0, 5.0, 9, params)
    m = oracle.Model(y0.shape[1:], params)
    yh = m.to_k(y0)
    for _ in range(4):
        yh, _, _ = oracle.ark_step(m, yh, 0.5, oracle.TABLES[meth]())
    with pfg.Simulation(y0.shape[1:], params, meth, "fp32bulk") as s:
        s.set_state(y0)
        for _ in range(4):
            s.step(0.5)
        got = to_np(s.state_hat())
    assert np.all(relerr(got, yh) <= 1e-5), relerr(got, yh)


def test_ark3_adaptive_replayed(pfg, params):
    """Adaptive ARK3(2)4L[2]SA at rtol 1e-4 (controller exponent q = 3): the
    oracle replays the GPU's attempts; errors agree to 1e-6 relative,
    decisions wherever |e - 1| > 1e-6, and the final state to 1e-11."""
    y0 = synth.ic_spheres(32, 3, 3.0, 5.0, 9, params)
    with pfg.Simulation(y0.shape[1:], params, "ark3", "fp64") as s:
        s.set_state(y0)
        st = s.advance(8.0, 1e-4, 1e-8)
        att = s.attempts()
        got = to_np(s.state_hat())
    assert st["t"] == pytest.approx(8.0, rel=1e-14)
    m = oracle.Model(y0.shape[1:], params)
    replay = [(h, ok) for (_, h, _, ok) in att]
    yh, t, log = oracle.advance(m, m.to_k(y0), 0.0, 8.0, oracle.ark324l2sa(), params, 1e-4, 1e-8, replay=replay)
    for (tg, hg, eg, okg), (to, ho, eo, _) in zip(att, log):
        assert tg == pytest.approx(to, rel=1e-12, abs=1e-12)
        assert eg == pytest.approx(eo, rel=1e-6)
        if abs(eo - 1.0) > 1e-6:
            assert okg == (eo <= 1.0)
    assert np.all(relerr(got, yh) <= 1e-11)


def test_fp32bulk_error_estimate_tracks_fp64(pfg, params):
    """The FP32-bulk form accumulates its local error estimate in FP32 and
    transforms it in FP32 before the FP64 WRMS norm.  Along an adaptive
    FP32-bulk run, every attempt is repeated in the FP64 path from the same
    state with the same step: the two norms agree to 1e-2 relative (1e-2 of
    0.05 absolute where the norm is small), so the accept/reject decisions
    agree wherever ||LTE|| is more than 1 % away from 1."""
    import torch
    y0 = synth.ic_spheres(32, 3, 3.0, 5.0, 9, params)
    with pfg.Simulation(y0.shape[1:], params, "ark4", "fp32bulk") as s32, \
            pfg.Simulation(y0.shape[1:], params, "ark4", "fp64") as s64:
        s32.set_state(y0)
        s32.set_time(0.0, 0.5)
        n = 0
        while n < 12:
            before = s32.state_hat()
            s32.advance_attempts(1)
            (t, h, e32, ok), = s32.attempts()
            s64.set_state_hat(before)
            e64 = s64.step(h)
            assert abs(e32 - e64) <= 1e-2 * max(e64, 0.05), (n, h, e32, e64)
            if abs(e64 - 1.0) > 1e-2:
                assert ok == (e64 <= 1.0)
            n += 1
        torch.cuda.synchronize()


@pytest.mark.parametrize("meth,nrhs", [("euler", 1), ("ark2", 3), ("ark3", 4), ("ark4", 6)])
def test_rhs_evaluations_per_step_match_paper(pfg, params, meth, nrhs):
    """Sec. 2.3 prints 1, 3, 4 and 6 explicit RHS evaluations per step for the
    first- through fourth-order methods (tests/golden/rhs_per_step.txt): the
    library's counter over three fixed steps, both precisions."""
    y0 = synth.ic_spheres(16, 2, 2.0, 3.0, 4, params)
    for prec in ("fp64", "fp32bulk"):
        with pfg.Simulation((16, 16, 16), params, meth, prec) as s:
            s.set_state(y0)
            r0 = s.stats()["rhs_evals"]
            for _ in range(3):
                s.step(0.25)
            assert s.stats()["rhs_evals"] - r0 == 3 * nrhs


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32bulk", 2e-5)])
def test_unequal_curvature_kks_matches_oracle(pfg, params, prec, tol):
    """KKS with parabolic phases of different curvature (A^v = 2.5 A^m, B^v =
    0.2; Eqs. f_ch_p, x_sum, equal_mu): the explicit right-hand side on a
    ragged grid (the fused x passes at 64, the staged ones elsewhere) and
    three ARK4 steps against the oracle.  Order parameters stay at or below
    0.4 so that sum_v h(phi_v) <= 1, where the mixture is well posed."""
    import torch
    p = dict(params, A_v=2.5 * params["A_m"], B_v=0.2)
    for shape in ((16, 12, 64), (10, 12, 20)):
        y = synth.random_state(shape, 55)
        y[1:] *= 0.4
        m = oracle.Model(shape, p)
        yh = m.to_k(y)
        ref = m.rhs_explicit(yh)
        with pfg.Simulation(shape, p, "ark4", prec) as s:
            got = s.rhs_explicit(torch.from_numpy(yh).to("cuda")).cpu().numpy()
            assert np.all(relerr(got, ref) <= tol), (shape, relerr(got, ref))
            s.set_state(y)
            ref_y = yh
            for _ in range(3):
                ref_y, _, _ = oracle.ark_step(m, ref_y, 0.5, oracle.ark436l2sa(), p["rtol"], p["atol"])
                s.step(0.5)
            got_y = s.state_hat().cpu().numpy()
            assert np.all(relerr(got_y, ref_y) <= (1e-11 if prec == "fp64" else 1e-5)), (shape, relerr(got_y, ref_y))


@pytest.mark.parametrize("prec,tol,stol", [("fp64", 1e-12, 1e-11), ("fp32bulk", 2e-5, 1e-5)])
def test_obstacle_barrier_matches_oracle(pfg, params, prec, tol, stol):
    """The literal obstacle term of Eq. f_b (barrier = 1): the explicit
    right-hand side, then three ARK4 steps, each followed by the projection of
    the order parameters onto [0, 1] in real space, against the oracle's
    steps and projections; the composition mean stays exact and the real-space
    order parameters end inside [0, 1] (to the transforms' rounding)."""
    import torch
    p = dict(params, barrier=1)
    for shape in ((16, 12, 64), (10, 12, 20)):
        y = synth.random_state(shape, 57)
        y[1:] = np.clip(1.4 * y[1:] - 0.2, 0.0, 1.0)  # bulk regions at the bounds, where the force pushes out
        m = oracle.Model(shape, p)
        yh = m.to_k(y)
        ref = m.rhs_explicit(yh)
        with pfg.Simulation(shape, p, "ark4", prec) as s:
            got = s.rhs_explicit(torch.from_numpy(yh).to("cuda")).cpu().numpy()
            assert np.all(relerr(got, ref) <= tol), (shape, relerr(got, ref))
            s.set_state(y)
            dc = s.state_hat()[0, 0, 0, 0].item()
            ref_y = yh
            for _ in range(3):
                ref_y, _, _ = oracle.ark_step(m, ref_y, 0.25, oracle.ark436l2sa(), p["rtol"], p["atol"])
                ref_y = m.project(ref_y)
                s.step(0.25)
            got_y = s.state_hat().cpu().numpy()
            assert np.all(relerr(got_y, ref_y) <= stol), (shape, relerr(got_y, ref_y))
            assert got_y[0, 0, 0, 0] == dc
            real = s.get_state()
            assert real[1:].min() >= -1e-12 and real[1:].max() <= 1 + 1e-12


def test_batch_refuses_obstacle(pfg, params):
    p = dict(params, barrier=1)
    y0 = synth.ic_spheres(16, 2, 2.5, 3.5, 7, p)
    with pfg.Simulation(y0.shape[1:], p, "ark4", "fp32bulk") as s:
        s.set_state(y0)
        with pytest.raises(pfg.PFError) as ei:
            pfg.batch_advance([s], 2.0)
        assert ei.value.code == pfg.PF_EUNSUPPORTED
