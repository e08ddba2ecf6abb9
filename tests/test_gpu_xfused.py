"""The fused FP32 x passes (last inverse stage, real-space physics and first
forward stage in registers; C2R packing folded into the first inverse stage,
R2C unpacking into the store) against the FP64 oracle, for every line length
that has a fused plan, on grids whose row-pair count leaves a ragged last CTA;
the staged kernel (tuning slot 39), the right-hand-side pass with its real
fields copied into shared memory (slot 41) and the passes with every stage in
place in one buffer (slot 42) must agree as well."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

LENGTHS = [64, 96, 120, 128, 160, 192, 256, 640]


@pytest.fixture(scope="module")
def pfg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2609_36100_gb300 as m
    m.build()
    return m


def relerr(a, b):
    return np.array([np.linalg.norm((a[f] - b[f]).ravel()) / np.linalg.norm(b[f].ravel()) for f in range(a.shape[0])])


@pytest.mark.parametrize("nx", LENGTHS)
@pytest.mark.parametrize("elastic", [True, False])
def test_fused_x_rhs_matches_oracle(pfg, params, nx, elastic):
    import torch
    p = params if elastic else synth.load_params(eps_c=0.0, eps_a=0.0)
    shape = (6, 10, nx)  # 30 row pairs: a ragged last CTA for every fused plan
    y = synth.random_state(shape, 60 + nx)
    m = oracle.Model(shape, p)
    yh = m.to_k(y)
    ref = m.rhs_explicit(yh)
    dev = torch.from_numpy(yh).to("cuda")
    with pfg.Simulation(shape, p, "ark4", "fp32bulk") as s:
        for off, stg, inpl in ((0, 0, 0), (0, 1, 0), (0, 0, 1), (0, 1, 1), (1, 0, 0)):
            cfg = s.tuning()
            cfg[39] = off
            cfg[41] = stg
            cfg[42] = inpl
            s.set_tuning(cfg)
            got = s.rhs_explicit(dev).cpu().numpy()
            err = relerr(got, ref)
            assert np.all(err <= 2e-5), (off, stg, inpl, err)


@pytest.mark.parametrize("nx", [96, 256, 640])
def test_fused_x_step_and_error_norm(pfg, params, nx):
    """One ARK4 step: the state to 1e-5 and the WRMS norm of the local error
    (formed by the fused C2R of the error and the compensated FP32 sums) to
    1e-3 of the oracle's."""
    shape = (4, 12, nx)
    y = synth.random_state(shape, 70 + nx, phi_scale=0.9)
    m = oracle.Model(shape, params)
    yh, e_ref, _ = oracle.ark_step(m, m.to_k(y), 0.5, oracle.ark436l2sa(), params["rtol"], params["atol"])
    for inpl in (0, 1):
        with pfg.Simulation(shape, params, "ark4", "fp32bulk") as s:
            cfg = s.tuning()
            cfg[42] = inpl
            s.set_tuning(cfg)
            s.set_state(y)
            e = s.step(0.5)
            got = s.state_hat().cpu().numpy()
        assert np.all(relerr(got, yh) <= 1e-5)
        assert abs(e - e_ref) <= 1e-3 * e_ref, (inpl, e, e_ref)
