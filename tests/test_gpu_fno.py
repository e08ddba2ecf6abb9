"""FNO surrogate kernels against the FP64 oracle (oracle/fno.py), through the
C ABI: forward outputs and every parameter gradient, in the FP32-weight
checking mode (tight) and with BF16 spectral weights (BF16-level), plus the
Adam training loop and the proposal/judge logic of pf_surrogate_step."""
import numpy as np
import pytest

import synth
from oracle import fno as ofno

pytestmark = pytest.mark.gpu

SHAPE = (16, 16, 16)
DIMS = dict(C=8, modes=4, H=16, L=2)


@pytest.fixture(scope="module")
def pfg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2609_36100_gb300 as m
    m.build()
    return m


def odims():
    return ofno.Dims(SHAPE, C=DIMS["C"], m=DIMS["modes"], H=DIMS["H"], L=DIMS["L"])


def data(seed=1):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((4,) + SHAPE)
    t = rng.standard_normal((4,) + SHAPE) * 0.1
    return x, t


def per_tensor(d, a, b):
    out = {}
    o = 0
    for name, s in ofno.layout(d):
        k = int(np.prod(s))
        da, db = a[o:o + k], b[o:o + k]
        out[name] = np.linalg.norm(da - db) / max(np.linalg.norm(db), 1e-30)
        o += k
    return out


@pytest.mark.parametrize("bf16,tol_out,tol_g", [(False, 1e-5, 1e-4), (True, 2e-2, 2e-2)])
def test_forward_and_gradients_vs_oracle(pfg, bf16, tol_out, tol_g):
    import torch
    d = odims()
    theta = ofno.init_params(d, 5)
    # spectral weights large enough that the spectral path matters
    P = ofno.unpack(d, theta)
    for l in range(d.L):
        P["W%d" % l][...] *= 20.0
    x, tgt = data()
    out_ref, acts = ofno.forward(d, theta, x, cache=True)
    g_ref = ofno.backward(d, theta, acts, out_ref, tgt)
    net = pfg.FNO(SHAPE, bf16=bf16, **DIMS)
    try:
        assert net.n == theta.size
        net.set_params(theta.astype(np.float32))
        xt = torch.from_numpy(x.astype(np.float32)).cuda()
        tt = torch.from_numpy(tgt.astype(np.float32)).cuda()
        out = net.forward(xt).cpu().numpy()
        rel = np.linalg.norm(out - out_ref) / np.linalg.norm(out_ref)
        assert rel <= tol_out, rel
        loss = net.backward(tt)
        assert loss == pytest.approx(ofno.loss(out_ref, tgt), rel=max(tol_out, 1e-6))
        errs = per_tensor(d, net.grads().astype(np.float64), g_ref)
        bad = {k: v for k, v in errs.items() if v > tol_g}
        assert not bad, bad
    finally:
        net.close()


def test_adam_training_reduces_loss(pfg):
    import torch
    d = odims()
    theta = ofno.init_params(d, 6)
    x, _ = data(2)
    tgt = 0.5 * x[::-1].copy()  # a learnable map: scaled channel permutation
    net = pfg.FNO(SHAPE, bf16=True, **DIMS)
    try:
        net.set_params(theta.astype(np.float32))
        xt = torch.from_numpy(x.astype(np.float32)).cuda()
        tt = torch.from_numpy(tgt.astype(np.float32)).cuda()
        first = net.train_step(xt, tt, 3e-3)
        for _ in range(100):
            last = net.train_step(xt, tt, 3e-3)
        assert last < 0.3 * first
        # one GPU Adam step equals the oracle's update from the same gradient
        net.set_params(theta.astype(np.float32))
        net.forward(xt)
        net.backward(tt)
        g = net.grads().astype(np.float64)
        lib = pfg.lib()
        assert lib.pf_fno_adam(net.f, 1e-3, 0.9, 0.999, 1e-8) == 0
        want = ofno.adam_step(theta.astype(np.float32).astype(np.float64), g, np.zeros_like(g), np.zeros_like(g), 1,
                              1e-3)
        assert np.max(np.abs(net.params() - want)) < 1e-6
    finally:
        net.close()


def test_surrogate_step_accept_and_restore(pfg, params):
    p = params
    y0 = synth.ic_spheres(16, 2, 3.0, 4.0, 3, p)
    net = pfg.FNO(SHAPE, bf16=True, **DIMS)
    sim = pfg.Simulation(SHAPE, p, "ark4", "fp64")
    try:
        net.set_norm([0.05, 0.0, 0.0, 0.0], [0.05, 1.0, 1.0, 1.0], [1e-3, 1e-2, 1e-2, 1e-2])
        # zero network: the proposal is y(t) itself, so the judge step is an
        # ordinary step and is accepted; the clock advances by tau + h
        net.set_params(np.zeros(net.n, dtype=np.float32))
        sim.set_state(y0)
        ok, e = net.surrogate_step(sim, 8.0, 0.5)
        assert ok and e <= 1.0
        t, _ = sim.time()
        assert t == pytest.approx(8.5)
        with pfg.Simulation(SHAPE, p, "ark4", "fp64") as ref:
            ref.set_state(y0)
            ref.step(0.5)
            a = ref.state_hat().cpu().numpy()
        b = sim.state_hat().cpu().numpy()
        assert np.max(np.abs(a - b)) <= 1e-14 * np.max(np.abs(a))
        # a noisy network: rejected, state and clock restored exactly
        rng = np.random.default_rng(3)
        net.set_params((rng.standard_normal(net.n) * 3.0).astype(np.float32))
        before = sim.state_hat().cpu().numpy()
        ok, e = net.surrogate_step(sim, 8.0, 0.5)
        assert not ok and not (e <= 1.0)  # large or non-finite error estimate
        assert sim.time()[0] == pytest.approx(8.5)
        assert np.array_equal(sim.state_hat().cpu().numpy(), before)
    finally:
        sim.close()
        net.close()
