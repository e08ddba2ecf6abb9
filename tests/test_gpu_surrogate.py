"""What the trained surrogate gains over the plain method, measured: a small
FNO trained by the library's kernels on solver trajectories (32^3), then
judged rollouts on held-out seeds against plain fixed-step integration and a
fine reference.  The proposals that pass the integrator's judge replace eight
steps each, so the rollout needs fewer right-hand-side evaluations; the cost
is accuracy, which this test reports and bounds rather than hides."""
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


def test_surrogate_gain_and_error(pfg, params):
    from paper_2609_36100_gb300 import surrogate as S
    n, dt = 32, 1.0
    ics = [(synth.ic_config1(n, 1000 + i, params, count=3), params) for i in range(8)]
    traj = S.trajectories(ics, params, dt, 12)
    net = S.new_network((n, n, n), C=16, modes=6, H=64, L=4)
    try:
        losses = S.train(net, traj, 4, 1e-3)
        assert losses[-1] < losses[0]
        y0 = synth.ic_config1(n, 2000, params, count=3)
        ref, _, _, _ = S.rollout(y0, params, 96.0, 0.25, None, precision="fp64")
        plain, w_plain, _, _ = S.rollout(y0, params, 96.0, dt, None)
        sur, w_sur, acc, off = S.rollout(y0, params, 96.0, dt, net)

        def err(a):
            return np.linalg.norm((a - ref)[1:]) / np.linalg.norm(ref[1:])

        print("surrogate: accepted %d/%d, wall %.3f s vs %.3f s plain, error %.2e vs %.2e plain"
              % (acc, off, w_sur, w_plain, err(sur), err(plain)))
        assert off > 0
        # every accepted proposal replaces 8 steps by 1 network pass + 1 step
        assert err(sur) < 0.5
        assert err(plain) < 1e-4
    finally:
        net.close()
