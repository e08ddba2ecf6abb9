"""Inhomogeneous-modulus elasticity of the oracle: the iterative scheme of Hu
and Chen for mechanical equilibrium, Eq. u_gov (Sec. 4.1; Sec. 4.2 names the
method).

TEST INFRASTRUCTURE ONLY (see oracle/model.py).

Readings:
* local stiffness: the Reuss mix C(r) = [sum_v h_v S^v + (1 - H) S^m]^-1 of
  the phases' compliances S^p = (C^p)^-1 (the printed formula mixes the
  compliances and omits the outer inverse);
* eigenstrain field eps0(r) = sum_v h(phi_v) eps*_v (as in the homogeneous
  reading);
* stress-free mean strain: <sigma> = 0 fixes the uniform strain eps_bar;
* elastic energy f_el = 1/2 eps_el : C(r) : eps_el with
  eps_el = eps_bar + eps(u) - eps0, whose Euler-Lagrange equation is
  Eq. u_gov.  Its derivative with respect to h_v at fixed displacement is
  e_v = -sigma : eps*_v - 1/2 sigma : (S^v - S^m) : sigma (the Reuss
  derivative dC/dh_v = -C (S^v - S^m) C), the elastic term of the
  order-parameter driving force h'(phi_v) e_v.

Hu-Chen iteration with the homogeneous reference medium C0 = (C^m + C^v)/2
(the paper does not state one; the mean of the two phases keeps
|C(r) - C0| at most half the contrast, for which the iteration contracts
where a reference equal to one phase stalls beyond ~30 % contrast) and
C'(r) = C(r) - C0: each step solves the homogeneous problem
div C0 eps(u) = div tau with the eigenstress
tau = C0 eps0 - C'(eps_bar + eps(u_prev) - eps0) (iteration 0: tau = C0
eps0), in Fourier space eps^(u)(k) = Gamma(n) : tau^(k), Gamma_ijkl =
sym_ij sym_kl n_i Omega_jk(n) n_l with Omega = (n.C0.n)^-1, zero at k = 0
and on the Nyquist planes of even axes (no displacement mode there); eps_bar
follows from <C (eps_bar + eps(u) - eps0)> = 0.  The loop stops when the
largest change of eps(u) between iterations is <= el_tol times the largest
|eps0| (or after el_max_iter iterations).

Warm start (el_warm, the default): a solve starts from the strain field
eps(u) of the previous solve of the same trajectory instead of the cold
tau = C0 eps0, so its first iteration already measures a change; when the
fields moved little since that solve, one iteration meets the tolerance.
This is the reading of Sec. 2.3's remark that with the loose tolerance the
solver exits after one iteration for nearly all steps (a cold start needs
several iterations for any contrast, since the first one measures no
change).  The carried field is part of the trajectory, not of the state: a
solve without it starts cold.

Tensors are handled as full 3x3x3x3 arrays and 3x3 matrices with einsum
and numpy.linalg (Mandel 6x6 form only to invert fourth-order tensors).
"""
from __future__ import annotations

import numpy as np

from .model import cubic_stiffness, voigt_to_tensor

# Mandel basis: symmetric 3x3 <-> 6-vectors with sqrt(2) on the shears, so
# that fourth-order tensors with minor symmetries invert as 6x6 matrices
_IDX = [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]
_W = np.array([1.0, 1.0, 1.0, np.sqrt(2.0), np.sqrt(2.0), np.sqrt(2.0)])


def to_mandel(C):
    """3x3x3x3 (minor-symmetric) -> 6x6 Mandel matrix."""
    M = np.empty((6, 6))
    for a, (i, j) in enumerate(_IDX):
        for b, (k, l) in enumerate(_IDX):
            M[a, b] = C[i, j, k, l] * _W[a] * _W[b]
    return M


def from_mandel(M):
    """6x6 Mandel matrix -> 3x3x3x3 tensor with minor symmetries."""
    C = np.empty((3, 3, 3, 3))
    for a, (i, j) in enumerate(_IDX):
        for b, (k, l) in enumerate(_IDX):
            v = M[a, b] / (_W[a] * _W[b])
            for (p, q) in {(i, j), (j, i)}:
                for (r, s) in {(k, l), (l, k)}:
                    C[p, q, r, s] = v
    return C


def invert4(C):
    """Inverse of a fourth-order tensor on symmetric second-order tensors."""
    return from_mandel(np.linalg.inv(to_mandel(C)))


def from_mandel_stack(M):
    """[..., 6, 6] Mandel matrices -> [..., 3, 3, 3, 3] tensors."""
    C = np.empty(M.shape[:-2] + (3, 3, 3, 3))
    for a, (i, j) in enumerate(_IDX):
        for b, (k, l) in enumerate(_IDX):
            v = M[..., a, b] / (_W[a] * _W[b])
            for (p, q) in {(i, j), (j, i)}:
                for (r, s) in {(k, l), (l, k)}:
                    C[..., p, q, r, s] = v
    return C


class HuChen:
    """Mechanical equilibrium with a phase-dependent (Reuss-mixed) stiffness
    on one periodic grid; real-space fields are [..., nz, ny, nx]."""

    def __init__(self, model, p: dict):
        self.m = model
        self.Cm = cubic_stiffness(p["C11"], p["C12"], p["C44"])
        self.Cv = cubic_stiffness(p.get("C11_v", p["C11"]), p.get("C12_v", p["C12"]), p.get("C44_v", p["C44"]))
        self.Sm = invert4(self.Cm)
        self.Sv = invert4(self.Cv)
        self.dS = self.Sv - self.Sm
        self.C0 = 0.5 * (self.Cm + self.Cv)
        self.eps = np.array([voigt_to_tensor(e) for e in p["eps_star"]])  # [v][3][3]
        self.tol = float(p.get("el_tol", 1e-6))
        self.max_iter = int(p.get("el_max_iter", 20))
        KX, KY, KZ = model.kvec
        kn = np.sqrt(KX ** 2 + KY ** 2 + KZ ** 2)
        safe = np.where(kn > 0, kn, 1.0)
        n = np.stack([KX / safe, KY / safe, KZ / safe], axis=-1)  # [..., 3]
        self.zero = kn == 0
        # Nyquist planes of the even axes (x: half-spectrum index nx/2; y, z:
        # index n/2): a displacement mode there has no derivative on the grid
        # (its sampled gradient vanishes), so the displacement space excludes
        # them and eps(u) has no Nyquist content; with that restriction the
        # discrete energy 1/2 sum sigma:eps_el is exactly minimised over u and
        # the driving force below is its exact derivative
        nz_, ny_, nx_ = model.shape
        nyq = np.zeros(KX.shape, bool)
        if nx_ % 2 == 0:
            nyq[..., nx_ // 2] = True
        if ny_ % 2 == 0:
            nyq[:, ny_ // 2, :] = True
        if nz_ % 2 == 0:
            nyq[nz_ // 2, :, :] = True
        self.zero = (kn == 0) | nyq
        Kac = np.einsum("ijkl,...j,...l->...ik", self.C0, n, n)
        Kac[self.zero] = np.eye(3)
        self.Om = np.linalg.inv(Kac)  # Omega(n), [..., 3, 3]
        self.n = n

    def stiffness(self, h):
        """Per-point Reuss-mixed stiffness [..., 3,3,3,3] from h [3, ...]:
        the compliance sum_v h_v S^v + (1 - H) S^m inverted point by point."""
        H = h.sum(axis=0)[..., None, None]
        S = (1.0 - H) * to_mandel(self.Sm) + H * to_mandel(self.Sv)
        return from_mandel_stack(np.linalg.inv(S))

    def green(self, tau):
        """eps(u) of the homogeneous (C0) problem with eigenstress tau
        [3, 3, nz, ny, nx] (real space): eps^_ij = 1/2 (n_i w_j + n_j w_i),
        w = Omega (tau^ n), zero mean."""
        m = self.m
        th = np.empty((3, 3) + m.k2.shape, dtype=complex)
        for i in range(3):
            for j in range(3):
                th[i, j] = m.to_k(tau[i, j][None])[0]
        th = np.moveaxis(th, (0, 1), (-2, -1))  # [..., 3, 3]
        t_n = np.einsum("...ij,...j->...i", th, self.n)
        w = np.einsum("...ij,...j->...i", self.Om, t_n)
        ek = 0.5 * (self.n[..., :, None] * w[..., None, :] + self.n[..., None, :] * w[..., :, None])
        ek[self.zero] = 0.0
        ek = np.moveaxis(ek, (-2, -1), (0, 1))
        out = np.empty((3, 3) + m.shape)
        for i in range(3):
            for j in range(3):
                out[i, j] = m.to_r(ek[i, j][None])[0]
        return out

    def solve(self, h, eps_u0=None):
        """Returns (e [3, ...] driving-force terms, sigma [3,3,...], eps_el
        [3,3,...], eps_bar [3,3], iterations); the final eps(u) is kept in
        self.last_eps_u.  eps_u0: the eps(u) to start from (warm start), or
        None for the cold start."""
        C = self.stiffness(h)  # [..., 3,3,3,3]
        e0 = np.einsum("v...,vij->ij...", h, self.eps)  # eps0 [3,3,...]
        Cp = C - self.C0
        Cavg = C.reshape(-1, 3, 3, 3, 3).mean(axis=0)
        C0e0 = np.einsum("ijkl,kl...->ij...", self.C0, e0)
        scale = max(np.max(np.abs(e0)), 1e-300)

        def mean_strain(eu):
            rhs = np.einsum("...ijkl,kl...->ij...", C, e0 - eu).reshape(3, 3, -1).mean(axis=-1)
            Sinv = invert4(Cavg)
            return np.einsum("ijkl,kl->ij", Sinv, rhs)

        if eps_u0 is None:
            eps_u = self.green(C0e0)
            it = 1
        else:
            eps_u = eps_u0
            it = 0
        ebar = mean_strain(eps_u)
        while it < self.max_iter:
            tot = ebar[:, :, None, None, None] + eps_u - e0
            tau = C0e0 - np.einsum("...ijkl,kl...->ij...", Cp, tot)
            new = self.green(tau)
            change = np.max(np.abs(new - eps_u))
            eps_u = new
            ebar = mean_strain(eps_u)
            it += 1
            if change <= self.tol * scale:
                break
        self.last_eps_u = eps_u
        el = ebar[:, :, None, None, None] + eps_u - e0
        sig = np.einsum("...ijkl,kl...->ij...", C, el)
        e = np.empty((3,) + h.shape[1:])
        for v in range(3):
            e[v] = -np.einsum("ij...,ij->...", sig, self.eps[v]) \
                - 0.5 * np.einsum("ij...,ijkl,kl...->...", sig, self.dS, sig)
        return e, sig, el, ebar, it
