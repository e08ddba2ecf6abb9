"""What the trained surrogate gains over the plain method, measured: a small
FNO trained by the library's kernels on solver trajectories (32^3), then
rollouts on a held-out seed in windows of tau, each proposal judged by the
method's own adaptive integration of the same window.  Proposals are
accepted only within the integrator's tolerance of the verified state and
the rollout always continues from the verified state, so the surrogate-
assisted rollout keeps the plain method's accuracy; its wall time and the
proposals' distances are what the test reports."""
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
    ics = [(synth.ic_ellipsoids(n, 1000 + i, params, count=3), params) for i in range(8)]
    traj = S.trajectories(ics, params, dt, 12)
    net = S.new_network((n, n, n), C=16, modes=6, H=64, L=4)
    try:
        losses = S.train(net, traj, 4, 1e-3)
        assert losses[-1] < losses[0]
        y0 = synth.ic_ellipsoids(n, 2000, params, count=3)
        ref, _, _, _, _ = S.rollout(y0, params, 96.0, 8.0, None, precision="fp64", rtol=1e-8, atol=1e-12)
        plain, w_plain, _, _, _ = S.rollout(y0, params, 96.0, 8.0, None)
        sur, w_sur, acc, off, dists = S.rollout(y0, params, 96.0, 8.0, net)

        def err(a):
            return np.linalg.norm((a - ref)[1:]) / np.linalg.norm(ref[1:])

        print("surrogate: accepted %d/%d (median distance %.3g), wall %.3f s vs %.3f s plain, error %.2e vs %.2e"
              % (acc, off, float(np.median(dists)), w_sur, w_plain, err(sur), err(plain)))
        assert off == 12
        assert acc == sum(1 for d in dists if d <= 1.0)
        # the rollout continues from the verified integration: plain accuracy
        assert err(plain) < 1e-4
        assert err(sur) < 3 * err(plain) + 1e-6
    finally:
        net.close()
