"""Pins of the oracle's inhomogeneous-modulus elasticity (Hu-Chen iterations
for Eq. u_gov with the Reuss-mixed stiffness, Sec. 4.1/4.2) against what the
mechanics fixes, without a GPU."""
import numpy as np
import pytest

import oracle
import synth
from oracle.elastic import HuChen


def _voigt_cubic(C11, C12, C44):
    """6x6 Voigt stiffness (engineering shear strains) of a cubic crystal."""
    C = np.zeros((6, 6))
    C[:3, :3] = C12
    np.fill_diagonal(C[:3, :3], C11)
    C[3, 3] = C[4, 4] = C[5, 5] = C44
    return C


def test_homogeneous_modulus_reduces_to_the_green_kernel(params):
    """With equal phase moduli the iteration converges at once (the second
    pass changes nothing) and its driving force -sigma:eps*_v equals the
    closed-form Khachaturyan contraction IFFT[sum_q B_vq h^_q]: two
    independent formulations of the homogeneous solution.  Odd axis lengths:
    on the Nyquist planes of even axes the iteration admits no displacement
    mode, where the closed-form kernel relaxes them."""
    shape = (9, 11, 15)
    y = synth.random_state(shape, 21)
    m = oracle.Model(shape, params)
    h = oracle.h_interp(y[1:])
    ref = m.elastic_potential(h)
    p = dict(params, el_inhom=1, C11_v=params["C11"], C12_v=params["C12"], C44_v=params["C44"], el_tol=1e-14)
    mi = oracle.Model(shape, p)
    e, sig, el, ebar, it = mi.hc.solve(h)
    assert it == 2
    assert np.max(np.abs(e - ref)) <= 1e-12 * np.max(np.abs(ref))
    # stress-free mean: <sigma> = 0
    assert np.max(np.abs(sig.reshape(9, -1).mean(axis=1))) <= 1e-12 * np.max(np.abs(sig))


def test_laminate_with_phase_contrast_matches_closed_form(params):
    """A slab of variant 1 normal to x with tanh edges and a stiffer
    precipitate (C11, C12, C44 up 30, 10 and 20 %).  In a laminate the strains tangential to the layers are
    uniform and the tractions on the layer planes vanish, so with the
    stress-free mean: sigma_xx = sigma_xy = sigma_xz = 0 everywhere, and
    the uniform tangential strains solve the 2x2 system <sigma_yy> =
    <sigma_zz> = 0 with the point-wise Reuss-mixed constants (computed here
    from Voigt 6x6 compliances, independently of the oracle's Mandel
    algebra).  The converged iteration reproduces that stress field."""
    p = dict(params, el_inhom=1, C11_v=1.3 * params["C11"], C12_v=1.1 * params["C12"], C44_v=1.2 * params["C44"],
             el_tol=1e-12, el_max_iter=200)
    nx = 75  # odd lengths: no Nyquist plane, whose stress modes the discrete displacement cannot relax
    y = synth.ic_slab(nx, 3, 3, p, 8.0, 24.0)
    m = oracle.Model(y.shape[1:], p)
    h = oracle.h_interp(y[1:])
    e, sig, el, ebar, it = m.hc.solve(h)
    assert 2 < it < 200
    # closed form along x
    H = h[0][0, 0, :]
    Sm = np.linalg.inv(_voigt_cubic(p["C11"], p["C12"], p["C44"]))
    Sv = np.linalg.inv(_voigt_cubic(p["C11_v"], p["C12_v"], p["C44_v"]))
    C11 = np.empty(nx)
    C12 = np.empty(nx)
    for i in range(nx):
        Cl = np.linalg.inv((1 - H[i]) * Sm + H[i] * Sv)
        C11[i], C12[i] = Cl[0, 0], Cl[0, 1]
    es = p["eps_star"][0]  # variant 1: c-axis along x
    e0 = {"xx": H * es[0], "yy": H * es[1], "zz": H * es[2]}
    a = C11 - C12 ** 2 / C11
    b = C12 - C12 ** 2 / C11
    A = np.array([[a.mean(), b.mean()], [b.mean(), a.mean()]])
    rhs = np.array([(a * e0["yy"] + b * e0["zz"]).mean(), (b * e0["yy"] + a * e0["zz"]).mean()])
    Eyy, Ezz = np.linalg.solve(A, rhs)
    elyy, elzz = Eyy - e0["yy"], Ezz - e0["zz"]
    elxx = -C12 / C11 * (elyy + elzz)
    syy = C12 * elxx + C11 * elyy + C12 * elzz
    szz = C12 * elxx + C12 * elyy + C11 * elzz
    scale = np.max(np.abs(syy))
    got = sig[:, :, 0, 0, :]
    for (i, j) in [(0, 0), (0, 1), (0, 2), (1, 2)]:
        assert np.max(np.abs(got[i, j])) <= 1e-7 * scale, (i, j)
    assert np.max(np.abs(got[1, 1] - syy)) <= 1e-7 * scale
    assert np.max(np.abs(got[2, 2] - szz)) <= 1e-7 * scale
    # fields vary along x only
    assert np.max(np.abs(sig - sig[:, :, :1, :1, :])) <= 1e-9 * scale


def test_iterations_grow_with_contrast_and_stop_at_the_tolerance(params):
    shape = (12, 12, 12)
    y = synth.ic_spheres(12, 1, 3.0, 3.5, 5, params)
    h = oracle.h_interp(y[1:])
    its = []
    for c in (1.0, 1.15, 1.4):
        p = dict(params, el_inhom=1, C11_v=c * params["C11"], C12_v=params["C12"], C44_v=c * params["C44"],
                 el_tol=1e-10, el_max_iter=100)
        its.append(HuChen(oracle.Model(shape, p), p).solve(h)[4])
    assert its[0] == 2 and its[0] < its[1] < its[2] < 100
    p = dict(params, el_inhom=1, C11_v=1.4 * params["C11"], C12_v=params["C12"], C44_v=1.4 * params["C44"],
             el_tol=1e-2, el_max_iter=100)
    assert HuChen(oracle.Model(shape, p), p).solve(h)[4] < its[2]


def test_inhomogeneous_rhs_is_variational_derivative(params):
    """With a phase contrast the order-parameter right-hand side is still
    -L dF/dphi_v of the free energy that includes 1/2 eps_el:C(r):eps_el at
    mechanical equilibrium (fourth-order finite differences of F)."""
    p = dict(params, el_inhom=1, C11_v=1.25 * params["C11"], C12_v=1.1 * params["C12"], C44_v=1.2 * params["C44"],
             el_tol=1e-13, el_max_iter=200)
    shape = (8, 8, 8)
    rng = np.random.default_rng(6)
    y = np.empty((4,) + shape)
    y[0] = 0.06 + 0.01 * rng.standard_normal(shape)
    y[1:] = rng.uniform(0.05, 0.4, size=(3,) + shape)  # sum_v h(phi_v) < 1: a valid compliance mix
    m = oracle.Model(shape, p)
    yh = m.to_k(y)
    tot = m.to_r(m.rhs_explicit(yh) + m.rhs_implicit(yh))
    dV = p["dx"] ** 3
    eps = 2e-5

    def F_at(field, idx, d):
        yp = y.copy()
        yp[(field,) + idx] += d
        return m.free_energy(m.to_k(yp))

    for idx in [(0, 0, 0), (3, 5, 2)]:
        for v in range(3):
            d1 = F_at(1 + v, idx, eps) - F_at(1 + v, idx, -eps)
            d2 = F_at(1 + v, idx, 2 * eps) - F_at(1 + v, idx, -2 * eps)
            dF = (8 * d1 - d2) / (12 * eps * dV)
            assert tot[1 + v][idx] == pytest.approx(-p["L"] * dF, rel=1e-5, abs=1e-9)


def _contrast(params, tol, it=200):
    return dict(params, el_inhom=1, C11_v=1.3 * params["C11"], C12_v=1.1 * params["C12"], C44_v=1.2 * params["C44"],
                el_tol=tol, el_max_iter=it)


def test_warm_start_from_the_solution_stops_after_one_iteration(params):
    """Started from the converged eps(u) of the same fields, one iteration
    reproduces it (the fixed point of the iteration is the equilibrium), so
    the warm-started solve stops after one solve with the same force."""
    shape = (10, 12, 14)
    p = _contrast(params, 1e-12)
    y = synth.random_state(shape, 21)
    y[1:] *= 0.4
    h = oracle.h_interp(y[1:])
    hc = HuChen(oracle.Model(shape, p), p)
    e_cold, _, _, _, it_cold = hc.solve(h)
    e_warm, _, _, _, it_warm = hc.solve(h, hc.last_eps_u)
    assert it_cold > 5 and it_warm == 1
    assert np.max(np.abs(e_warm - e_cold)) <= 1e-9 * np.max(np.abs(e_cold))


def test_warm_start_after_a_small_change_meets_the_same_tolerance(params):
    """Fields moved a little since the previous solve (as between the stages
    of a step): the warm-started solve takes fewer iterations than the cold
    one at the loose tolerance, and both forces lie within the tolerance's
    reach of the converged one."""
    shape = (10, 12, 14)
    y0 = synth.random_state(shape, 22)
    y0[1:] *= 0.4
    rng = np.random.default_rng(3)
    y1 = y0.copy()
    y1[1:] += 1e-3 * rng.standard_normal(y0[1:].shape)
    h0, h1 = oracle.h_interp(y0[1:]), oracle.h_interp(y1[1:])
    tight = HuChen(oracle.Model(shape, _contrast(params, 1e-13)), _contrast(params, 1e-13))
    e_ref = tight.solve(h1)[0]
    p = _contrast(params, 1e-6)
    hc = HuChen(oracle.Model(shape, p), p)
    hc.solve(h0)
    prev = hc.last_eps_u
    e_warm, _, _, _, it_warm = hc.solve(h1, prev)
    e_cold, _, _, _, it_cold = hc.solve(h1)
    assert it_warm < it_cold
    scale = np.max(np.abs(e_ref))
    assert np.max(np.abs(e_warm - e_ref)) <= 1e-4 * scale
    assert np.max(np.abs(e_cold - e_ref)) <= 1e-4 * scale


def test_model_carries_the_warm_start_between_evaluations(params):
    """The model's solves continue one sequence (right-hand sides and free
    energy alike); el_warm = 0 restores independent cold solves."""
    shape = (8, 8, 8)
    y = synth.random_state(shape, 23)
    y[1:] *= 0.4
    p = _contrast(params, 1e-6)
    m = oracle.Model(shape, p)
    yh = m.to_k(y)
    m.rhs_explicit(yh)
    assert m.hc_prev is not None
    first = m.hc_prev
    m.rhs_explicit(yh)
    assert m.hc_prev is not first
    mc = oracle.Model(shape, dict(p, el_warm=0))
    mc.rhs_explicit(yh)
    assert mc.hc_prev is None
