"""Values the paper prints, kept as text fixtures under tests/golden/ (each
file names its passage), checked against the oracle and the input
generators (no GPU)."""
import os

import numpy as np
import pytest

import oracle
import synth
from tests.order_conditions import max_violation

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    out = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].split()
            if line:
                out.append(line)
    return out


RHS = {r[0]: (int(r[1]), int(r[2])) for r in _rows("rhs_per_step.txt")}


@pytest.mark.parametrize("meth", sorted(RHS))
def test_rhs_evaluations_per_step(meth, params):
    """Sec. 2.3: the number of explicit RHS evaluations one step of each
    method takes, counted by the oracle's step on a small state."""
    order, nrhs = RHS[meth]
    tab = oracle.ark.TABLES[meth]()
    shape = (6, 6, 6)
    m = oracle.Model(shape, params)
    y0 = synth.ic_mode(shape, params, 1, (1, 0, 0), 0.05)
    y0[1] += 0.3
    _, _, st = oracle.ark.ark_step(m, m.to_k(y0), 0.25, tab)
    assert st["rhs"] == nrhs


@pytest.mark.parametrize("meth", sorted(RHS))
def test_method_order(meth):
    """Sec. 2.3 / Sec. 4.4: first- through fourth-order methods: the tables
    satisfy the coupled order conditions of their order and not of the next."""
    order, _ = RHS[meth]
    t = oracle.ark.TABLES[meth]()
    assert max_violation(t.AE, t.AI, t.bE, t.bI, order) < 1e-13
    assert max_violation(t.AE, t.AI, t.bE, t.bI, order + 1) > 1e-6


def test_two_particle_geometry(params):
    """Sec. 2.3 benchmark geometry: grid, spacing and the two seeds; the
    generator's variant-1 field is above 1/2 exactly inside the two seed
    spheres (periodic distance), every other field is the matrix state."""
    kv = {}
    seeds = []
    for r in _rows("two_particle.txt"):
        if r[0] == "seed":
            seeds.append(tuple(float(v) for v in r[1:]))
        else:
            kv[r[0]] = float(r[1])
    assert kv["dx_nm"] == params["dx"]
    n = int(kv["n"])
    assert n * kv["dx_nm"] == kv["domain_nm"]
    y = synth.ic_two_particle(n, params)
    assert y.shape == (4, n, n, n)
    idx = np.arange(n) * kv["dx_nm"]
    z, yy, x = np.meshgrid(idx, idx, idx, indexing="ij")
    L = kv["domain_nm"]
    margin = np.full(x.shape, np.inf)   # signed distance to the nearest seed surface (nm)
    for cx, cy, cz, r in seeds:
        d2 = 0.0
        for c, g in ((cx, x), (cy, yy), (cz, z)):
            d = np.abs(g - c)
            d = np.minimum(d, L - d)
            d2 = d2 + d * d
        margin = np.minimum(margin, np.sqrt(d2) - r)
    inside = margin < -1e-9
    outside = margin > 1e-9
    assert np.all(y[1][inside] > 0.5)
    assert np.all(y[1][outside] < 0.5)
    assert inside.sum() > 0.5 * (4 / 3) * np.pi * sum((s[3] / kv["dx_nm"]) ** 3 for s in seeds)
    assert np.all(y[2] == 0.0) and np.all(y[3] == 0.0)
    assert np.allclose(y[0], params["X_matrix"])
