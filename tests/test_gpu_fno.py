"""FNO surrogate kernels against the FP64 oracle (oracle/fno.py), through the
C ABI: forward outputs and every parameter gradient, in the FP32-weight
checking mode (tight) and with BF16 spectral weights (BF16-level), plus the
Adam training loop, the library-side normalisation and pair training, and
the judge of pf_surrogate_step."""
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


def test_fit_norm_and_train_pair(pfg, params):
    """The library's normalisation statistics equal numpy's over all
    consecutive snapshot pairs, and a training step on a raw pair equals a
    training step on the pair normalised by hand."""
    import torch
    rng = np.random.default_rng(9)
    snaps = rng.standard_normal((2, 3, 4) + SHAPE).astype(np.float32) * np.array([0.01, 0.3, 0.2, 0.1],
                                                                              dtype=np.float32)[None, None, :, None,
                                                                                                 None, None]
    snaps += np.array([0.05, 0.2, 0.1, 0.0], dtype=np.float32)[None, None, :, None, None, None]
    x = snaps[:, :-1].transpose(2, 0, 1, 3, 4, 5).reshape(4, -1).astype(np.float64)
    d = (snaps[:, 1:] - snaps[:, :-1]).transpose(2, 0, 1, 3, 4, 5).reshape(4, -1).astype(np.float64)
    mean, sd, dsd = x.mean(axis=1), x.std(axis=1), d.std(axis=1)
    dev = torch.from_numpy(snaps).to("cuda").contiguous()
    a = pfg.FNO(SHAPE, bf16=False, **DIMS)
    b = pfg.FNO(SHAPE, bf16=False, **DIMS)
    try:
        th = (np.random.default_rng(4).standard_normal(a.n) * 0.05).astype(np.float32)
        a.set_params(th)
        b.set_params(th)
        a.fit_norm(dev)
        la = a.train_pair(dev[0, 0], dev[0, 1], 1e-3)
        b.set_norm(mean, sd, dsd)
        xin = torch.from_numpy(((snaps[0, 0] - mean[:, None, None, None]) / sd[:, None, None, None])
                               .astype(np.float32)).to("cuda").contiguous()
        tgt = torch.from_numpy(((snaps[0, 1] - snaps[0, 0]) / dsd[:, None, None, None])
                               .astype(np.float32)).to("cuda").contiguous()
        lb = b.train_step(xin, tgt, 1e-3)
        assert la == pytest.approx(lb, rel=1e-4)
        assert np.max(np.abs(a.params() - b.params())) <= 1e-6
    finally:
        a.close()
        b.close()


def test_surrogate_step_judged_by_verified_integration(pfg, params):
    """The judge integrates the proposal's interval with the method itself:
    the call ends at the state and time of a plain adaptive integration of
    the same interval (bitwise), and reports the proposal's WRMS distance to
    it (weights from the verified state), accepting only within 1."""
    import torch  # noqa: F401
    p = params
    y0 = synth.ic_spheres(16, 2, 3.0, 4.0, 3, p)
    tau, h, rtol, atol = 8.0, 0.5, 1e-4, 1e-8
    with pfg.Simulation(SHAPE, p, "ark4", "fp64") as ref:
        ref.set_state(y0)
        ref.set_time(0.0, h)
        ref.advance(tau, rtol, atol)
        y_tau = ref.get_state()
        yh_tau = ref.state_hat().cpu().numpy()
    net = pfg.FNO(SHAPE, bf16=True, **DIMS)
    sim = pfg.Simulation(SHAPE, p, "ark4", "fp64")
    try:
        net.set_norm([0.05, 0.0, 0.0, 0.0], [0.05, 1.0, 1.0, 1.0], [1e-3, 1e-2, 1e-2, 1e-2])
        # zero network: the proposal is y(t) itself
        net.set_params(np.zeros(net.n, dtype=np.float32))
        sim.set_state(y0)
        ok, dist = net.surrogate_step(sim, tau, h, rtol, atol)
        want = np.sqrt(np.mean(((y0 - y_tau) / (rtol * np.abs(y_tau) + atol)) ** 2))
        assert dist == pytest.approx(want, rel=1e-9)
        assert ok == (want <= 1.0)
        assert sim.time()[0] == pytest.approx(tau, rel=1e-14)
        assert np.array_equal(sim.state_hat().cpu().numpy(), yh_tau)
        # a noisy network: far outside the tolerance, rejected; the state is
        # still the verified integration
        rng = np.random.default_rng(3)
        net.set_params((rng.standard_normal(net.n) * 3.0).astype(np.float32))
        sim.set_state(y0)
        sim.set_time(0.0, h)
        ok, dist = net.surrogate_step(sim, tau, h, rtol, atol)
        assert not ok and not (dist <= 1.0)
        assert np.array_equal(sim.state_hat().cpu().numpy(), yh_tau)
    finally:
        sim.close()
        net.close()
