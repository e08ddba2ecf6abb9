"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the CPU oracle.

This module holds no arithmetic of the phase-field method itself: it reads the
parameter file and draws initial conditions (nuclei in a supersaturated matrix,
Sec. 2.1 and Sec. 2.3 of the paper) as plain FP64 arrays laid out
``[field][z][y][x]`` with field order (X, phi_1, phi_2, phi_3).

Nucleus recipe (the paper gives positions/sizes only for its two-particle test,
Sec. 2.3): a nucleus of variant v is an ellipsoid with semi-axes (a, a, c), c
along axis v; phi_v = 1/2 [1 - tanh(d / (sqrt(2) l))] with
d = (rho - 1) min(a, c) dx, rho the ellipsoidal radius and l = sqrt(kappa/omega_bar)
the equilibrium interface length of the double-well barrier. Nuclei never
overlap (rejection sampling on periodic center distance). PRNG: numpy PCG64.
"""
from __future__ import annotations

import json
import math
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_PARAMS = os.path.join(_HERE, "params_default.json")


def load_params(path: str | None = None, **overrides) -> dict:
    """Read the parameter JSON and expand the isotropic/default entries into the
    full per-variant form both implementations consume.

    kappa[v] and eps_star[v] are Voigt 6-vectors (xx, yy, zz, yz, xz, xy);
    variant v has its c-axis along spatial axis v (0 = x, 1 = y, 2 = z).
    omega_pair is (w12, w13, w23).
    """
    with open(path or DEFAULT_PARAMS) as f:
        p = {k: v for k, v in json.load(f).items() if not k.startswith("_")}
    p.update(overrides)
    if "kappa" not in p:
        k = p["kappa_iso"]
        p["kappa"] = [[k, k, k, 0.0, 0.0, 0.0] for _ in range(3)]
    if "eps_star" not in p:
        es = []
        for v in range(3):
            d = [p["eps_a"]] * 3
            d[v] = p["eps_c"]
            es.append(d + [0.0, 0.0, 0.0])
        p["eps_star"] = es
    if "omega_pair" not in p:
        p["omega_pair"] = [p["omega_vq"]] * 3
    return p


def interface_length(p: dict) -> float:
    """l = sqrt(kappa/omega_bar) for the isotropic default (nm)."""
    return math.sqrt(p["kappa_iso"] / p["omega_bar"])


def _periodic_disp(n: int, center: float) -> np.ndarray:
    i = np.arange(n, dtype=np.float64)
    return (i - center + n / 2.0) % n - n / 2.0


def _stamp(phi: np.ndarray, center, semi, dx: float, ell: float):
    """Max-combine one tanh-edged ellipsoid into phi (z, y, x). center/semi in
    cells, ordered (x, y, z)."""
    nz, ny, nx = phi.shape
    margin = int(math.ceil(20.0 * ell / dx)) + 2
    ax = []
    for dim, n in zip(range(3), (nx, ny, nz)):
        r = int(math.ceil(semi[dim])) + margin
        if 2 * r + 1 >= n:
            idx = np.arange(n)
        else:
            c0 = int(math.floor(center[dim]))
            idx = np.arange(c0 - r, c0 + r + 2) % n
        d = (idx - center[dim] + n / 2.0) % n - n / 2.0
        ax.append((idx, d))
    (ix, ddx), (iy, ddy), (iz, ddz) = ax
    rho = np.sqrt((ddz[:, None, None] / semi[2]) ** 2 + (ddy[None, :, None] / semi[1]) ** 2
                  + (ddx[None, None, :] / semi[0]) ** 2)
    dist = (rho - 1.0) * min(semi) * dx
    val = 0.5 * (1.0 - np.tanh(dist / (math.sqrt(2.0) * ell)))
    sub = phi[np.ix_(iz, iy, ix)]
    phi[np.ix_(iz, iy, ix)] = np.maximum(sub, val)


def nuclei_ic(shape, p: dict, nuclei, x_inside: float | None = None,
              x_matrix: float | None = None, noise: float = 0.0, rng=None) -> np.ndarray:
    """Build a [4][nz][ny][nx] FP64 state from a list of nuclei
    (variant, (cx, cy, cz) cells, (sx, sy, sz) semi-axes in cells)."""
    nz, ny, nx = shape
    dx = p["dx"]
    ell = interface_length(p)
    y = np.zeros((4, nz, ny, nx), dtype=np.float64)
    for v, c, s in nuclei:
        _stamp(y[1 + v], c, s, dx, ell)
    xm = p["X_matrix"] if x_matrix is None else x_matrix
    if x_inside is None:
        y[0] = xm
    else:
        tot = np.clip(y[1] + y[2] + y[3], 0.0, 1.0)
        y[0] = xm + tot * (x_inside - xm)
    if noise > 0.0:
        y[0] += rng.normal(0.0, noise, size=(nz, ny, nx))
    return y


def draw_nuclei(shape, count: int, rng, semi_fn, gap: float = 2.0, max_tries: int = 200000):
    """Rejection-sample `count` non-overlapping nuclei; semi_fn(rng, v) returns
    the (sx, sy, sz) semi-axes (cells) of a variant-v nucleus."""
    nz, ny, nx = shape
    out = []
    tries = 0
    while len(out) < count:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("could not place %d non-overlapping nuclei" % count)
        v = int(rng.integers(0, 3))
        s = semi_fn(rng, v)
        c = (rng.uniform(0, nx), rng.uniform(0, ny), rng.uniform(0, nz))
        r = max(s)
        ok = True
        for _, c2, s2 in out:
            d2 = 0.0
            for a, b, n in zip(c, c2, (nx, ny, nz)):
                d = abs(a - b) % n
                d = min(d, n - d)
                d2 += d * d
            if math.sqrt(d2) < r + max(s2) + gap:
                ok = False
                break
        if ok:
            out.append((v, c, s))
    return out


def _disc(a: float, c: float, v: int):
    s = [a, a, a]
    s[v] = c
    return tuple(s)


def ic_ellipsoids(n: int = 64, seed: int = 1, p: dict | None = None, count: int = 8) -> np.ndarray:
    """8 ellipsoidal nuclei (semi-axes 3-6 cells, c-axis along the variant
    axis), uniform matrix composition plus N(0, 1e-3) noise."""
    p = p or load_params()
    rng = np.random.default_rng(seed)

    def semi(rng, v):
        a = rng.uniform(3.0, 6.0)
        c = rng.uniform(3.0, a)
        return _disc(a, c, v)

    nuc = draw_nuclei((n, n, n), count, rng, semi)
    return nuclei_ic((n, n, n), p, nuc, noise=1e-3, rng=rng)


def ic_spheres(n: int, count: int, rmin: float, rmax: float, seed: int, p: dict | None = None,
               x_inside: bool = True) -> np.ndarray:
    """`count` spherical nuclei with radius U[rmin, rmax] cells, random
    variant; composition at the precipitate value B_v inside."""
    p = p or load_params()
    rng = np.random.default_rng(seed)

    def semi(rng, v):
        r = rng.uniform(rmin, rmax)
        return (r, r, r)

    nuc = draw_nuclei((n, n, n), count, rng, semi)
    return nuclei_ic((n, n, n), p, nuc, x_inside=p["B_v"] if x_inside else None)


def ic_spheres_32(n: int = 256, seed: int = 2, p: dict | None = None) -> np.ndarray:
    return ic_spheres(n, 32, 4.0, 10.0, seed, p)


def ensemble_member(index: int, p: dict | None = None, sides=(64, 96, 120, 128, 160)):
    """Member `index` (0..63) of the uneven-grid ensemble: seed 100+index, side
    drawn from `sides`, 4-24 nuclei of radius 3-6 cells, aging temperature
    uniform in +/-20 K around T0. Returns (state, params)."""
    p = dict(p or load_params())
    rng = np.random.default_rng(100 + index)
    n = int(sides[int(rng.integers(0, len(sides)))])
    count = int(rng.integers(4, 25))
    p["T"] = p["T0"] + float(rng.uniform(-20.0, 20.0))

    def semi(rng, v):
        r = rng.uniform(3.0, 6.0)
        return (r, r, r)

    nuc = draw_nuclei((n, n, n), count, rng, semi)
    return nuclei_ic((n, n, n), p, nuc, x_inside=p["B_v"]), p


def ic_spheres_300(n: int = 640, seed: int = 5, p: dict | None = None) -> np.ndarray:
    return ic_spheres(n, 300, 4.0, 12.0, seed, p)


def ic_two_particle(n: int = 64, p: dict | None = None) -> np.ndarray:
    """Sec. 2.3 two-particle geometry: variant 1, seeds of radius 2.5 nm at
    (10, 15.5, 15.5) nm and 3 nm at (20.5, 20.5, 20.5) nm."""
    p = p or load_params()
    dx = p["dx"]
    nuc = [(0, (10.0 / dx, 15.5 / dx, 15.5 / dx), (2.5 / dx,) * 3),
           (0, (20.5 / dx, 20.5 / dx, 20.5 / dx), (3.0 / dx,) * 3)]
    return nuclei_ic((n, n, n), p, nuc)


def ic_slab(nx: int, ny: int, nz: int, p: dict, x_lo: float, x_hi: float, x_of_phi=None) -> np.ndarray:
    """Planar slab of variant 1 between x_lo and x_hi (nm) with tanh edges of
    length l; composition X = x_of_phi(phi) (default: matrix value)."""
    dx = p["dx"]
    ell = interface_length(p)
    x = (np.arange(nx) + 0.0) * dx
    prof = 0.5 * (np.tanh((x - x_lo) / (math.sqrt(2.0) * ell)) - np.tanh((x - x_hi) / (math.sqrt(2.0) * ell)))
    y = np.zeros((4, nz, ny, nx))
    y[1] = prof[None, None, :]
    y[0] = p["X_matrix"] if x_of_phi is None else x_of_phi(y[1])
    return y


def ic_mode(shape, p: dict, field: int, mode, amp: float, base_x: float | None = None) -> np.ndarray:
    """Uniform state (X = base, phi = 0) plus a small cosine of integer wave
    numbers `mode` = (mx, my, mz) on one field."""
    nz, ny, nx = shape
    y = np.zeros((4, nz, ny, nx))
    y[0] = p["X_matrix"] if base_x is None else base_x
    z, yy, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    arg = 2 * np.pi * (mode[0] * x / nx + mode[1] * yy / ny + mode[2] * z / nz)
    y[field] += amp * np.cos(arg)
    return y


def random_state(shape, seed: int, phi_scale: float = 1.0) -> np.ndarray:
    """Smooth-ish random state for parity tests: X around the matrix value,
    phi in [0, 1] with random structure."""
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape
    y = np.empty((4, nz, ny, nx))
    y[0] = 0.05 + 0.02 * rng.standard_normal((nz, ny, nx))
    y[1:] = phi_scale * rng.uniform(0.0, 1.0, size=(3, nz, ny, nx))
    return y
