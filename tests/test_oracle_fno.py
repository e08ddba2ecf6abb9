"""Pins of the FNO oracle (CPU): the truncated transform against numpy's FFT,
the reverse-mode gradient against central finite differences of the loss,
and Adam against its defining recursion on a scalar."""
import numpy as np
import pytest

from oracle import fno


@pytest.fixture(scope="module")
def small():
    d = fno.Dims((8, 8, 10), C=3, m=2, H=5, L=2)
    theta = fno.init_params(d, 3)
    rng = np.random.default_rng(1)
    x = rng.standard_normal((4,) + d.shape)
    tgt = rng.standard_normal((4,) + d.shape)
    return d, theta, x, tgt


def test_truncated_dft_matches_fft(small):
    d, _, x, _ = small
    a = x[:3]
    A = fno.fwd_dft(d, a)
    full = np.fft.fftn(a, axes=(1, 2, 3))
    ky = fno.mode_indices(d.shape[1], d.m, False)
    kz = fno.mode_indices(d.shape[0], d.m, False)
    ref = full[:, kz][:, :, ky][:, :, :, : d.m]
    assert np.max(np.abs(A - ref)) < 1e-12 * np.max(np.abs(ref))


def test_inverse_of_hermitian_truncation(small):
    """For a field band-limited to the retained modes (and no kx = nx/2
    content), Re F^-1 (F a) recovers a."""
    d, _, _, _ = small
    nz, ny, nx = d.shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    a = (np.cos(2 * np.pi * (x / nx + z / nz)) + 0.5 * np.sin(2 * np.pi * (y / ny - x / nx)) + 0.3)[None]
    back = fno.inv_re(d, fno.fwd_dft(d, a))
    assert np.max(np.abs(back - a)) < 1e-12


def test_gradient_matches_finite_differences(small):
    d, theta, x, tgt = small
    out, acts = fno.forward(d, theta, x, cache=True)
    g = fno.backward(d, theta, acts, out, tgt)
    rng = np.random.default_rng(7)
    idx = rng.choice(theta.size, size=40, replace=False)
    eps = 1e-4

    def L(i, h):
        tp = theta.copy()
        tp[i] += h
        return fno.loss(fno.forward(d, tp, x), tgt)

    for i in idx:
        # fourth-order central difference
        fd = (8 * (L(i, eps) - L(i, -eps)) - (L(i, 2 * eps) - L(i, -2 * eps))) / (12 * eps)
        assert g[i] == pytest.approx(fd, rel=1e-6, abs=1e-11)


def test_adam_definition():
    th = np.array([1.0])
    m = np.zeros(1)
    v = np.zeros(1)
    fno.adam_step(th, np.array([0.5]), m, v, 1, 0.1)
    # first step of Adam moves by lr * sign(g) (bias-corrected m/sqrt(v) = 1)
    assert th[0] == pytest.approx(1.0 - 0.1 * 0.5 / (0.5 + 1e-8), rel=1e-12)
