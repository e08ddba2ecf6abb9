"""GPU path vs the FP64 oracle, element by element, through the C ABI.

Bar (FP64 path): relative L2 per field <= 1e-11 after the configured steps
(transforms and single RHS evaluations are held to 1e-12); the composition
mean is conserved bitwise.  FP32-bulk errors against the FP64 oracle are
bounded by what single-precision transforms give (rel L2 <= 1e-5 for the
state after a few steps)."""
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
    """Relative L2 error per field of arrays [4, ...]."""
    a = np.asarray(a)
    b = np.asarray(b)
    out = []
    for f in range(a.shape[0]):
        den = np.linalg.norm(b[f].ravel())
        out.append(np.linalg.norm((a[f] - b[f]).ravel()) / (den if den > 0 else 1.0))
    return np.array(out)


def to_np(t):
    return t.detach().cpu().numpy()


def to_dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


SHAPES = [(8, 8, 8), (12, 10, 20), (6, 16, 4), (32, 32, 32)]


@pytest.mark.parametrize("shape", SHAPES)
def test_transforms_roundtrip_and_vs_oracle(pfg, params, shape):
    y = synth.random_state(shape, 1)
    m = oracle.Model(shape, params)
    with pfg.Simulation(shape, params, "euler", "fp64") as s:
        s.set_state(y)
        yh = to_np(s.state_hat())
        ref = m.to_k(y)
        assert np.max(np.abs(yh - ref)) <= 1e-14 * np.max(np.abs(ref))
        back = s.get_state()
        assert np.max(np.abs(back - y)) <= 1e-13


@pytest.mark.parametrize("shape", SHAPES + [(64, 64, 64)])
@pytest.mark.parametrize("elastic", [True, False])
def test_rhs_explicit_fp64(pfg, params, shape, elastic):
    p = params if elastic else synth.load_params(eps_c=0.0, eps_a=0.0)
    y = synth.random_state(shape, 2)
    m = oracle.Model(shape, p)
    yh = m.to_k(y)
    ref = m.rhs_explicit(yh)
    with pfg.Simulation(shape, p, "ark4", "fp64") as s:
        got = to_np(s.rhs_explicit(to_dev(yh)))
    err = relerr(got, ref)
    assert np.all(err <= 1e-12), err


@pytest.mark.parametrize("shape", [(12, 10, 20), (32, 32, 32)])
def test_rhs_explicit_fp32bulk(pfg, params, shape):
    y = synth.random_state(shape, 3)
    m = oracle.Model(shape, params)
    yh = m.to_k(y)
    ref = m.rhs_explicit(yh)
    with pfg.Simulation(shape, params, "ark4", "fp32bulk") as s:
        got = to_np(s.rhs_explicit(to_dev(yh)))
    err = relerr(got, ref)
    assert np.all(err <= 2e-5), err


def test_solve_implicit(pfg, params):
    shape = (12, 10, 20)
    m = oracle.Model(shape, params)
    rng = np.random.default_rng(4)
    r = rng.standard_normal((4, 12, 10, 11)) + 1j * rng.standard_normal((4, 12, 10, 11))
    with pfg.Simulation(shape, params, "ark4", "fp64") as s:
        got = to_np(s.solve_implicit(0.37, to_dev(r)))
    ref = m.solve_implicit(0.37, r)
    assert np.max(np.abs(got - ref)) <= 1e-15 * np.max(np.abs(ref))


def test_euler_ellipsoids_64_50_steps(pfg, params):
    """Plain method, FP64, 64^3, 8 ellipsoidal nuclei, ImEx Euler, 50 fixed
    steps of 0.25 s (rel L2 <= 1e-11 per field; composition mean bitwise)."""
    y0 = synth.ic_ellipsoids(64, 1, params)
    m = oracle.Model(y0.shape[1:], params)
    yh = m.to_k(y0)
    tab = oracle.euler()
    for _ in range(50):
        yh, _, _ = oracle.ark_step(m, yh, 0.25, tab)
    with pfg.Simulation(y0.shape[1:], params, "euler", "fp64") as s:
        s.set_state(y0)
        dc = to_np(s.state_hat())[0, 0, 0, 0]
        for _ in range(50):
            s.step(0.25, want_lte=False)
        got = to_np(s.state_hat())
        assert got[0, 0, 0, 0] == dc
    err = relerr(got, yh)
    assert np.all(err <= 1e-11), err
    # the hand-written Chen-Shen form of the same method (Sec. 2.3 check)
    yc = m.to_k(y0)
    for _ in range(50):
        yc = oracle.chen_shen_euler(m, yc, 0.25)
    assert np.all(relerr(got, yc) <= 1e-11)


@pytest.mark.parametrize("shape", [(32, 32, 32), (24, 20, 30)])
def test_ark4_steps_and_lte(pfg, params, shape):
    y0 = synth.ic_spheres(shape[0], 3, 3.0, 5.0, 9, params) if shape[0] == shape[1] == shape[2] else None
    if y0 is None:
        y0 = synth.random_state(shape, 5, phi_scale=0.9)
    m = oracle.Model(shape, params)
    yh = m.to_k(y0)
    tab = oracle.ark436l2sa()
    errs = []
    for _ in range(4):
        yh, e, _ = oracle.ark_step(m, yh, 0.5, tab, params["rtol"], params["atol"])
        errs.append(e)
    with pfg.Simulation(shape, params, "ark4", "fp64") as s:
        s.set_state(y0)
        got_e = [s.step(0.5) for _ in range(4)]
        got = to_np(s.state_hat())
    assert np.all(relerr(got, yh) <= 1e-11)
    np.testing.assert_allclose(got_e, errs, rtol=1e-9)


def test_adaptive_advance_replayed(pfg, params):
    """Adaptive ARK4 at rtol 1e-4: the oracle replays the GPU's attempt
    sequence.  ||LTE|| is a difference of stage terms ~1e4 times smaller than
    the terms, so the two FP64 implementations agree on it to ~1e-8 relative;
    decisions must agree wherever |e - 1| > 1e-6, and the final state matches."""
    y0 = synth.ic_spheres(32, 3, 3.0, 5.0, 9, params)
    with pfg.Simulation(y0.shape[1:], params, "ark4", "fp64") as s:
        s.set_state(y0)
        st = s.advance(12.0, 1e-4, 1e-8)
        att = s.attempts()
        got = to_np(s.state_hat())
    assert st["t"] == pytest.approx(12.0, rel=1e-14)
    assert len(att) >= 3
    m = oracle.Model(y0.shape[1:], params)
    replay = [(h, ok) for (_, h, _, ok) in att]
    yh, t, log = oracle.advance(m, m.to_k(y0), 0.0, 12.0, oracle.ark436l2sa(), params, 1e-4, 1e-8, replay=replay)
    for (tg, hg, eg, okg), (to, ho, eo, _) in zip(att, log):
        assert tg == pytest.approx(to, rel=1e-12, abs=1e-12)
        assert eg == pytest.approx(eo, rel=1e-6)
        if abs(eo - 1.0) > 1e-6:
            assert okg == (eo <= 1.0)
    assert np.all(relerr(got, yh) <= 1e-11)


def test_free_energy(pfg, params):
    y0 = synth.ic_ellipsoids(32, 1, params)
    m = oracle.Model(y0.shape[1:], params)
    with pfg.Simulation(y0.shape[1:], params, "ark4", "fp64") as s:
        s.set_state(y0)
        F = s.free_energy()
    assert F == pytest.approx(m.free_energy(m.to_k(y0)), rel=1e-12)


def test_fp32bulk_state_error_after_steps(pfg, params):
    y0 = synth.ic_spheres(32, 3, 3.0, 5.0, 9, params)
    m = oracle.Model(y0.shape[1:], params)
    yh = m.to_k(y0)
    for _ in range(4):
        yh, _, _ = oracle.ark_step(m, yh, 0.5, oracle.ark436l2sa())
    with pfg.Simulation(y0.shape[1:], params, "ark4", "fp32bulk") as s:
        s.set_state(y0)
        dc = to_np(s.state_hat())[0, 0, 0, 0]
        for _ in range(4):
            s.step(0.5)
        got = to_np(s.state_hat())
    assert got[0, 0, 0, 0] == dc  # composition mean stays FP64-exact
    err = relerr(got, yh)
    assert np.all(err <= 1e-5), err


def test_fp32bulk_keeps_increments_below_fp32_resolution(pfg, params):
    """The FP32-bulk form keeps the state and the stage combination at
    (close to) FP64 precision: over many tiny steps whose increments are far
    below one FP32 ulp of the state, its accumulated change matches the FP64
    path's to FP32-relative accuracy of the increment itself.  A state or a
    combination carried in FP32 would drop these increments entirely."""
    y0 = synth.ic_spheres(32, 3, 3.0, 5.0, 9, params)
    d = {}
    for prec in ("fp64", "fp32bulk"):
        with pfg.Simulation(y0.shape[1:], params, "ark4", prec) as s:
            s.set_state(y0)
            h0 = to_np(s.state_hat())
            for _ in range(40):
                s.step(2e-9)
            d[prec] = to_np(s.state_hat()) - h0
    scale = np.linalg.norm(h0)
    n64 = np.linalg.norm(d["fp64"])
    assert 0 < n64 < 1e-8 * scale  # far below FP32 resolution of the state
    assert np.linalg.norm(d["fp32bulk"] - d["fp64"]) <= 1e-4 * n64
