"""FP64 CPU oracle of the Fourier neural operator surrogate (forward and
backward).

TEST INFRASTRUCTURE ONLY (see oracle/model.py).  The surrogate is not in the
paper; its definition here is the plain one, written out with explicit DFT
matrices so that every step and its adjoint can be checked by eye:

  a_0 = P x + p                                    (lift, C x 4)
  for l = 0..L-1:
    A   = F_K(a_l)          truncated DFT: kx in [0, m), ky, kz in {0..m-1, n-m..n-1}
    O   = W_l A             per-mode complex C x C channel mix
    s   = Re F_K^-1(O)      s(r) = (1/N) Re sum_{k in K} w_kx O(k) e^{ik.r}, w = 1 (kx = 0) else 2
    z   = V_l a_l + v_l + s
    a_{l+1} = GELU(z)  (no activation after the last layer)
  h = GELU(Q1 a_L + q1);  out = Q2 h + q2         (projection C -> H -> 4)

GELU(z) = z/2 (1 + erf(z/sqrt 2)).  Loss = mean((out - target)^2).
Parameters live in one flat FP64 vector (layout in `layout`).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf


class Dims:
    def __init__(self, shape, C=32, m=12, H=128, L=4, cin=4):
        self.shape = tuple(int(s) for s in shape)  # (nz, ny, nx)
        self.C, self.m, self.H, self.L, self.cin = C, m, H, L, cin
        nz, ny, nx = self.shape
        assert nx // 2 >= m and ny >= 2 * m and nz >= 2 * m
        self.N = nz * ny * nx
        self.K = (2 * m) * (2 * m) * m


def layout(d: Dims):
    """Ordered (name, shape) of the flat parameter vector; spectral weights are
    stored as (re, im) pairs: shape (K, C, C, 2)."""
    C, H, L, cin, K = d.C, d.H, d.L, d.cin, d.K
    out = [("P", (C, cin)), ("p", (C,))]
    for l in range(L):
        out += [("W%d" % l, (K, C, C, 2)), ("V%d" % l, (C, C)), ("v%d" % l, (C,))]
    out += [("Q1", (H, C)), ("q1", (H,)), ("Q2", (cin, H)), ("q2", (cin,))]
    return out


def n_params(d: Dims) -> int:
    return sum(int(np.prod(s)) for _, s in layout(d))


def unpack(d: Dims, theta: np.ndarray) -> dict:
    out, o = {}, 0
    for name, s in layout(d):
        k = int(np.prod(s))
        out[name] = theta[o:o + k].reshape(s)
        o += k
    return out


def init_params(d: Dims, seed: int) -> np.ndarray:
    """Seeded initialisation (uniform, fan-in scaled)."""
    rng = np.random.default_rng(seed)
    parts = []
    for name, s in layout(d):
        if name.startswith("W"):
            scale = 1.0 / (d.C * d.C)
        elif len(s) == 2:
            scale = 1.0 / math.sqrt(s[1])
        else:
            scale = 0.0
        parts.append((rng.uniform(-1.0, 1.0, size=s) * scale).ravel())
    return np.concatenate(parts)


def mode_indices(n: int, m: int, half: bool):
    return list(range(m)) if half else list(range(m)) + list(range(n - m, n))


def dft_matrices(d: Dims):
    """Complex matrices of the truncated forward DFT along each axis:
    Mx[kx, x] = exp(-2 pi i kx x / nx) for kx < m, and My, Mz over the 2m
    retained y / z modes."""
    nz, ny, nx = d.shape
    m = d.m
    kx = np.array(mode_indices(nx, m, True))
    ky = np.array(mode_indices(ny, m, False))
    kz = np.array(mode_indices(nz, m, False))
    Mx = np.exp(-2j * np.pi * np.outer(kx, np.arange(nx)) / nx)
    My = np.exp(-2j * np.pi * np.outer(ky, np.arange(ny)) / ny)
    Mz = np.exp(-2j * np.pi * np.outer(kz, np.arange(nz)) / nz)
    w = np.where(kx == 0, 1.0, 2.0)
    return Mx, My, Mz, w


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def fwd_dft(d, a):
    """a[c, z, y, x] real -> A[c, kz, ky, kx] over the retained modes."""
    Mx, My, Mz, _ = dft_matrices(d)
    return np.einsum("az,by,cx,nzyx->nabc", Mz, My, Mx, a)


def inv_re(d, O, weighted=True, scale=True):
    """Re( sum_k c_k O(k) e^{ik.r} ), c_k = w_kx / N (weighted, scaled)."""
    Mx, My, Mz, w = dft_matrices(d)
    Ow = O * (w[None, None, None, :] if weighted else 1.0)
    r = np.einsum("az,by,cx,nabc->nzyx", np.conj(Mz), np.conj(My), np.conj(Mx), Ow).real
    return r / d.N if scale else r


def forward(d: Dims, theta: np.ndarray, x: np.ndarray, cache: bool = False):
    """x [cin, nz, ny, nx] -> out [cin, nz, ny, nx] (and the activations)."""
    P = unpack(d, theta)
    a = np.einsum("ci,i...->c...", P["P"], x) + P["p"][:, None, None, None]
    acts = {"x": x, "a": [a], "A": [], "z": []}
    for l in range(d.L):
        A = fwd_dft(d, a)
        W = P["W%d" % l][..., 0] + 1j * P["W%d" % l][..., 1]  # [K, C, C]
        Af = A.reshape(d.C, -1)                                # [C, K]
        O = np.einsum("kcd,dk->ck", W, Af).reshape(A.shape)
        s = inv_re(d, O)
        z = np.einsum("cd,d...->c...", P["V%d" % l], a) + P["v%d" % l][:, None, None, None] + s
        a = gelu(z) if l < d.L - 1 else z
        acts["A"].append(A)
        acts["z"].append(z)
        acts["a"].append(a)
    hpre = np.einsum("hc,c...->h...", P["Q1"], a) + P["q1"][:, None, None, None]
    h = gelu(hpre)
    out = np.einsum("oh,h...->o...", P["Q2"], h) + P["q2"][:, None, None, None]
    acts["hpre"], acts["h"] = hpre, h
    return (out, acts) if cache else out


def loss(out, target):
    return float(np.mean((out - target) ** 2))


def backward(d: Dims, theta: np.ndarray, acts: dict, out: np.ndarray, target: np.ndarray) -> np.ndarray:
    """Gradient of the MSE loss w.r.t. the flat parameter vector (manual
    reverse mode of `forward`)."""
    P = unpack(d, theta)
    G = {name: np.zeros(s) for name, s in layout(d)}
    n_el = out.size
    dout = 2.0 * (out - target) / n_el
    h, hpre = acts["h"], acts["hpre"]
    flat = lambda u: u.reshape(u.shape[0], -1)  # noqa: E731
    G["Q2"] = flat(dout) @ flat(h).T
    G["q2"] = dout.sum(axis=(1, 2, 3))
    dh = np.einsum("oh,o...->h...", P["Q2"], dout) * gelu_grad(hpre)
    aL = acts["a"][-1]
    G["Q1"] = flat(dh) @ flat(aL).T
    G["q1"] = dh.sum(axis=(1, 2, 3))
    da = np.einsum("hc,h...->c...", P["Q1"], dh)
    for l in reversed(range(d.L)):
        z, a_l, A = acts["z"][l], acts["a"][l], acts["A"][l]
        dz = da * gelu_grad(z) if l < d.L - 1 else da
        G["V%d" % l] = flat(dz) @ flat(a_l).T
        G["v%d" % l] = dz.sum(axis=(1, 2, 3))
        da = np.einsum("cd,c...->d...", P["V%d" % l], dz)
        # s = Re F^-1(O): dL/dO (as re + i im) = (w/N) F(dz)
        _, _, _, w = dft_matrices(d)
        GO = fwd_dft(d, dz) * (w[None, None, None, :] / d.N)
        W = P["W%d" % l][..., 0] + 1j * P["W%d" % l][..., 1]
        GOf = GO.reshape(d.C, -1)
        Af = A.reshape(d.C, -1)
        GW = np.einsum("ck,dk->kcd", GOf, np.conj(Af))
        G["W%d" % l] = np.stack([GW.real, GW.imag], axis=-1)
        GA = np.einsum("kcd,ck->dk", np.conj(W), GOf).reshape(A.shape)
        # A = F(a), a real: dL/da = Re sum_k GA(k) e^{ik.r}
        da = da + inv_re(d, GA, weighted=False, scale=False)
    x = acts["x"]
    G["P"] = flat(da) @ flat(x).T
    G["p"] = da.sum(axis=(1, 2, 3))
    return np.concatenate([G[name].ravel() for name, _ in layout(d)])


def adam_step(theta, g, mom, vel, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """Adam (Kingma & Ba) update in place; t counts from 1."""
    mom *= b1
    mom += (1 - b1) * g
    vel *= b2
    vel += (1 - b2) * g * g
    mh = mom / (1 - b1 ** t)
    vh = vel / (1 - b2 ** t)
    theta -= lr * mh / (np.sqrt(vh) + eps)
    return theta
