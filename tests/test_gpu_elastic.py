"""The fused elastic pass (last forward z stage, Green's contraction of
Eq. u_gov and first inverse stage in registers; the inverse runs the forward
radix order reversed), its form without a fused stage (every stage over the
three fields in place) and its three-CTA cluster form (one h field per CTA,
the contraction through distributed shared memory; tuning slot 40 = 0, 1, 2)
against the FP64 oracle's explicit right-hand side, for every compiled radix
plan of each length and every tile width, on grids whose half-spectrum rows
leave a ragged last tile."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

# compiled plans (id: length) of the library
PLANS = {1: 256, 2: 256, 3: 128, 4: 128, 5: 64, 6: 64, 7: 160, 8: 96, 9: 120, 10: 192, 11: 640}


@pytest.fixture(scope="module")
def pfg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2609_36100_gb300 as m
    m.build()
    return m


def relerr(a, b):
    return np.array([np.linalg.norm((a[f] - b[f]).ravel()) / np.linalg.norm(b[f].ravel()) for f in range(4)])


@pytest.mark.parametrize("pid", sorted(PLANS))
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32bulk", 2e-5)])
def test_fused_elastic_plan_matches_oracle(pfg, params, pid, prec, tol):
    import torch
    n = PLANS[pid]
    shape = (n, 6, 10)  # nz = n; nx/2 + 1 = 6 columns: every tile width leaves a ragged tail
    y = synth.random_state(shape, 40 + pid)
    m = oracle.Model(shape, params)
    yh = m.to_k(y)
    ref = m.rhs_explicit(yh)
    dev = torch.from_numpy(yh).to("cuda")
    with pfg.Simulation(shape, params, "ark4", prec) as s:
        for tx in (2, 4, 8, 16):
            for unfused in (0, 1, 2):
                cfg = s.tuning()
                cfg[2] = tx
                cfg[38] = pid
                cfg[40] = unfused
                s.set_tuning(cfg)
                assert s.tuning()[38] == pid
                got = s.rhs_explicit(dev).cpu().numpy()
                err = relerr(got, ref)
                assert np.all(err <= tol), (tx, unfused, err)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32bulk", 2e-5)])
def test_generic_elastic_pass_selectable(pfg, params, prec, tol):
    """Plan value -1 selects the elastic pass without a fused stage (forward
    transforms, contraction, inverse transforms as separate steps of one
    kernel), also where a compiled plan exists."""
    import torch
    shape = (256, 12, 30)
    y = synth.random_state(shape, 91)
    m = oracle.Model(shape, params)
    yh = m.to_k(y)
    ref = m.rhs_explicit(yh)
    dev = torch.from_numpy(yh).to("cuda")
    with pfg.Simulation(shape, params, "ark4", prec) as s:
        cfg = s.tuning()
        cfg[38] = -1
        s.set_tuning(cfg)
        assert s.tuning()[38] == -1
        got = s.rhs_explicit(dev).cpu().numpy()
        assert np.all(relerr(got, ref) <= tol)


@pytest.mark.parametrize("shape", [(256, 10, 40), (64, 18, 90), (640, 6, 36)])
@pytest.mark.parametrize("shear", [False, True])
def test_cluster_elastic_pass(pfg, shape, shear):
    """The cluster form over several ky rows (the launch order pairs ky with
    ny - ky), several column tiles with a ragged last one, and 640-point
    columns.  With
    diagonal eigenstrains it reads B(k)/N from the octant table; with a shear
    component the kernel is no longer even in each wave-number component, no
    table is built and every wave number forms B itself."""
    import torch
    e = [[0.004, 0.004, 0.02, 0.0, 0.0, 0.0], [0.004, 0.02, 0.004, 0.0, 0.0, 0.0],
         [0.02, 0.004, 0.004, 0.0, 0.0, 0.0]]
    if shear:
        e[0][5] = 0.003
        e[2][3] = -0.002
    p = synth.load_params(eps_star=e)
    y = synth.random_state(shape, 7 + shape[1])
    m = oracle.Model(shape, p)
    yh = m.to_k(y)
    ref = m.rhs_explicit(yh)
    dev = torch.from_numpy(yh).to("cuda")
    with pfg.Simulation(shape, p, "ark4", "fp32bulk") as s:
        for tx in (8, 16):
            cfg = s.tuning()
            cfg[2] = tx
            cfg[38] = {256: 1, 64: 5, 640: 11}[shape[0]]
            cfg[40] = 2
            s.set_tuning(cfg)
            assert s.tuning()[40] == 2
            got = s.rhs_explicit(dev).cpu().numpy()
            err = relerr(got, ref)
            assert np.all(err <= 2e-5), (tx, err)


def test_elastic_form_out_of_range_refused(pfg, params):
    with pfg.Simulation((64, 8, 8), params, "ark4", "fp32bulk") as s:
        cfg = s.tuning()
        cfg[40] = 3
        with pytest.raises(pfg.PFError):
            s.set_tuning(cfg)


def test_elastic_plan_of_wrong_length_refused(pfg, params):
    with pfg.Simulation((64, 8, 8), params, "ark4", "fp64") as s:
        cfg = s.tuning()
        cfg[38] = 1  # length 256
        with pytest.raises(pfg.PFError):
            s.set_tuning(cfg)


@pytest.mark.parametrize("n", [96, 120, 160, 192, 640])
@pytest.mark.parametrize("axis", ["y", "z"])
def test_column_passes_three_stage_plans(pfg, params, n, axis):
    """y and z column transforms of three-stage compiled plans, whose middle
    stage runs in place in one shared buffer: one FP32-bulk RHS evaluation
    against the oracle's, for every tile width the autotuner can choose."""
    import torch
    shape = (6, n, 10) if axis == "y" else (n, 6, 10)
    y = synth.random_state(shape, 80 + n)
    m = oracle.Model(shape, params)
    yh = m.to_k(y)
    ref = m.rhs_explicit(yh)
    dev = torch.from_numpy(yh).to("cuda")
    order = {96: [8, 4, 3], 120: [8, 3, 5], 160: [8, 4, 5], 192: [16, 4, 3], 640: [16, 8, 5]}[n]
    a = 1 if axis == "y" else 2
    with pfg.Simulation(shape, params, "ark4", "fp32bulk") as s:
        for tx in (4, 8, 16):
            cfg = s.tuning()
            cfg[0] = cfg[1] = cfg[37] = tx
            cfg[4 + 11 * a:4 + 11 * (a + 1)] = [3] + order + [0] * 7
            s.set_tuning(cfg)
            got = s.rhs_explicit(dev).cpu().numpy()
            err = relerr(got, ref)
            assert np.all(err <= 2e-5), (tx, err)
