"""Phase-dependent stiffness (Eq. u_gov with the Reuss-mixed C(r), solved by
Hu-Chen iterations in FP64) through the C ABI against the oracle's
independent formulation (oracle/elastic.py: full fourth-order tensors,
Mandel inversion, numpy FFTs)."""
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
    """Relative L2 error per field (absolute where the reference field is zero)."""
    out = []
    for f in range(a.shape[0]):
        den = np.linalg.norm(b[f].ravel())
        out.append(np.linalg.norm((a[f] - b[f]).ravel()) / (den if den > 0 else 1.0))
    return np.array(out)


def contrast(params, tol=1e-12, it=200):
    return dict(params, el_inhom=1, C11_v=1.3 * params["C11"], C12_v=1.1 * params["C12"], C44_v=1.2 * params["C44"],
                el_tol=tol, el_max_iter=it)


def state(shape, seed):
    """Precipitate-like fields with sum_v h(phi_v) <= 1 (a valid compliance mix)."""
    y = synth.random_state(shape, seed)
    y[1:] *= 0.4
    return y


@pytest.mark.parametrize("shape", [(16, 16, 16), (12, 10, 20)])
@pytest.mark.parametrize("tol", [1e-12, 1e-2])
def test_rhs_fp64_matches_oracle(pfg, params, shape, tol):
    """Converged (1e-12) and loose (1e-2: a few iterations) tolerances: the
    same iteration count as the oracle and the explicit right-hand side to
    1e-11 per field."""
    import torch
    p = contrast(params, tol)
    y = state(shape, 31)
    m = oracle.Model(shape, p)
    yh = m.to_k(y)
    ref = m.rhs_explicit(yh)
    its = m.hc.solve(oracle.h_interp(m.to_r(yh)[1:]))[4]
    with pfg.Simulation(shape, p, "ark4", "fp64") as s:
        got = s.rhs_explicit(torch.from_numpy(yh).to("cuda")).cpu().numpy()
        assert s.elastic_iterations() == its
    assert its >= 2
    assert np.all(relerr(got, ref) <= 1e-11), relerr(got, ref)


def test_rhs_fp32bulk_matches_oracle(pfg, params):
    import torch
    p = contrast(params)
    shape = (16, 16, 16)
    y = state(shape, 32)
    m = oracle.Model(shape, p)
    yh = m.to_k(y)
    ref = m.rhs_explicit(yh)
    with pfg.Simulation(shape, p, "ark4", "fp32bulk") as s:
        got = s.rhs_explicit(torch.from_numpy(yh).to("cuda")).cpu().numpy()
    assert np.all(relerr(got, ref) <= 2e-5), relerr(got, ref)


def test_ark4_step_and_free_energy(pfg, params):
    p = contrast(params)
    y0 = synth.ic_spheres(16, 2, 2.5, 3.5, 7, p)
    m = oracle.Model(y0.shape[1:], p)
    F0 = m.free_energy(m.to_k(y0))  # the same order of solves as below (warm start)
    yh, e, _ = oracle.ark_step(m, m.to_k(y0), 0.5, oracle.ark436l2sa(), p["rtol"], p["atol"])
    with pfg.Simulation(y0.shape[1:], p, "ark4", "fp64") as s:
        s.set_state(y0)
        F = s.free_energy()
        eg = s.step(0.5)
        got = s.state_hat().cpu().numpy()
    assert F == pytest.approx(F0, rel=1e-12)
    assert np.all(relerr(got, yh) <= 1e-11), relerr(got, yh)
    assert eg == pytest.approx(e, rel=1e-8)


def test_warm_start_sequence_matches_oracle(pfg, params):
    """Three ARK4 steps at the loose tolerance (1e-6): with the warm start
    every solve continues from the previous one's eps(u) across stages and
    steps, in the library as in the oracle; the iteration count of each
    step's last solve and the state after each step agree, and the warm
    start needs fewer iterations than cold solves (el_warm = 0), which the
    library reproduces as well."""
    y0 = synth.ic_spheres(16, 2, 2.5, 3.5, 7, params)
    counts = {}
    for warm in (1, 0):
        p = dict(contrast(params, 1e-6), el_warm=warm)
        m = oracle.Model(y0.shape[1:], p)
        yh = m.to_k(y0)
        its, states = [], []
        for _ in range(3):
            yh, _, _ = oracle.ark_step(m, yh, 0.5, oracle.ark436l2sa(), p["rtol"], p["atol"])
            its.append(m.hc_last_iters)
            states.append(yh)
        with pfg.Simulation(y0.shape[1:], p, "ark4", "fp64") as s:
            s.set_state(y0)
            for i in range(3):
                s.step(0.5)
                assert s.elastic_iterations() == its[i], (warm, i)
                got = s.state_hat().cpu().numpy()
                assert np.all(relerr(got, states[i]) <= 1e-10), (warm, i, relerr(got, states[i]))
        counts[warm] = its
    assert all(w < c for w, c in zip(counts[1], counts[0])), counts


def test_batch_refuses_phase_contrast(pfg, params):
    p = contrast(params)
    y0 = synth.ic_spheres(16, 2, 2.5, 3.5, 7, p)
    with pfg.Simulation(y0.shape[1:], p, "ark4", "fp32bulk") as s:
        s.set_state(y0)
        with pytest.raises(pfg.PFError) as ei:
            pfg.batch_advance([s], 2.0)
        assert ei.value.code == pfg.PF_EUNSUPPORTED
