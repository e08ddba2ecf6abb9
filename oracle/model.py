"""FP64 CPU oracle of the pseudospectral KKS gamma'' phase-field model.

TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the bench's CPU
baseline may import this module; the library never routes through it. It
shares no code with the CUDA path: FFTs are scipy's pocketfft (a library
primitive), everything else is written out below in the paper's order.

State: k-space coefficients y = {X^, phi^_1..3}, y^(k) = (1/N) sum_r y(r) e^{-ik.r}
(half spectrum, kx = 0..nx/2), so the DC entry is the field mean
(the integration runs in reciprocal space, Sec. 4.2).

Model (Sec. 4.1, Eqs. f_b, f_ch, x_sum, equal_mu, x_gov, phi_gov, u_gov) with
the readings:
* linear terms of Eqs. composition/order are diffusive (negative sign);
* composition stiff part lambda_X = -2 A^m M k^2, the rest explicit;
* parabolic f^p = A0^p + A^p (X^p - B^p)^2 (Eq. f_ch_p read as squared);
* barrier: omega_bar sum_v phi_v^2 (1 - phi_v)^2 (double-well reading of Eq. f_b);
  with barrier = 1 the literal term of Eq. f_b instead, omega_bar S (1 - S)
  with S = sum_v phi_v (derivative omega_bar (1 - 2 S)), an obstacle-type
  potential that needs phi_v in [0, 1]: project() clamps the order parameters
  in real space, applied after every completed step (the paper does not say
  how the bound is kept);
* the |x| of the pairwise barrier omega_vq |phi_v phi_q| is Huber-regularised
  with width eps (A(x) = x^2/(2 eps) for |x| < eps, |x| - eps/2 beyond), so
  d/dphi_v = omega_vq clip(phi_v phi_q / eps, -1, 1) phi_q is continuous;
* one solute (Nb);
* homogeneous modulus (iteration 0 of the Hu-Chen scheme), stress-free mean
  strain so that B(k = 0) = 0; with el_inhom set, a phase-dependent
  (Reuss-mixed) stiffness solved by the Hu-Chen iterations of
  oracle/elastic.py;
* Nyquist wave numbers taken as +pi/dx.
"""
from __future__ import annotations

import math
import os

import numpy as np
import scipy.fft as sfft

R_GAS = 8.314462618  # J/(mol K)
_WORKERS = int(os.environ.get("PF_ORACLE_THREADS", os.cpu_count() or 1))


def voigt_to_tensor(v) -> np.ndarray:
    """Voigt (xx, yy, zz, yz, xz, xy) tensor components -> symmetric 3x3."""
    xx, yy, zz, yz, xz, xy = v
    return np.array([[xx, xy, xz], [xy, yy, yz], [xz, yz, zz]], dtype=np.float64)


def cubic_stiffness(C11: float, C12: float, C44: float) -> np.ndarray:
    """C_ijkl of a cubic crystal in its cube axes, written entry by entry."""
    C = np.zeros((3, 3, 3, 3))
    for i in range(3):
        for j in range(3):
            for k in range(3):
                for l in range(3):
                    if i == j and k == l:
                        C[i, j, k, l] = C11 if i == k else C12
                    elif (i == k and j == l) or (i == l and j == k):
                        C[i, j, k, l] = C44
    return C


def wavenumbers(n: int, d: float, half: bool) -> np.ndarray:
    """k_m = 2 pi m / (n d), m in {0..n/2} (half) or {0..n/2, -n/2+1..-1};
    the Nyquist index n/2 takes +pi/d."""
    if half:
        m = np.arange(n // 2 + 1, dtype=np.float64)
    else:
        m = np.arange(n, dtype=np.float64)
        m[m > n // 2] -= n
    return 2.0 * math.pi * m / (n * d)


def h_interp(phi):
    """h(phi) = phi^3 (6 phi^2 - 15 phi + 10) (Sec. 4.1)."""
    return phi ** 3 * (6.0 * phi ** 2 - 15.0 * phi + 10.0)


def h_prime(phi):
    """h'(phi) = 30 phi^2 (1 - phi)^2."""
    return 30.0 * phi ** 2 * (1.0 - phi) ** 2


class Model:
    """All derived constants and operators on one periodic grid."""

    def __init__(self, shape, p: dict, dx: float | None = None):
        self.shape = tuple(int(s) for s in shape)  # (nz, ny, nx)
        nz, ny, nx = self.shape
        self.N = nz * ny * nx
        self.p = p
        d = p["dx"] if dx is None else dx
        self.dx = d
        self.dV = d ** 3
        # temperature dependence (proposed: Arrhenius mobility, linear B^m)
        self.M = p["M0"] * math.exp(-p["Q_act"] / R_GAS * (1.0 / p["T"] - 1.0 / p["T0"]))
        self.Bm = p["B_m0"] + p["dBm_dT"] * (p["T"] - p["T0"])
        self.Bv = p["B_v"]
        self.Am, self.Av = p["A_m"], p["A_v"]
        self.A0m, self.A0v = p["A0_m"], p["A0_v"]
        self.L = p["L"]
        self.wbar = p["omega_bar"]
        self.obstacle = int(p.get("barrier", 0)) == 1
        self.pair_eps = p["pair_eps"]
        w12, w13, w23 = p["omega_pair"]
        self.omega = np.array([[0.0, w12, w13], [w12, 0.0, w23], [w13, w23, 0.0]])
        kx = wavenumbers(nx, d, True)
        ky = wavenumbers(ny, d, False)
        kz = wavenumbers(nz, d, False)
        KZ, KY, KX = np.meshgrid(kz, ky, kx, indexing="ij")
        self.kvec = (KX, KY, KZ)
        self.k2 = KX ** 2 + KY ** 2 + KZ ** 2
        # k . kappa_v . k for each variant
        self.kk = np.empty((3,) + self.k2.shape)
        for v in range(3):
            kap = voigt_to_tensor(p["kappa"][v])
            acc = np.zeros(self.k2.shape)
            kv = (KX, KY, KZ)
            for i in range(3):
                for j in range(3):
                    acc += kap[i, j] * kv[i] * kv[j]
            self.kk[v] = acc
        # implicit (stiff, linear) operator: lambda(k) per field
        self.lam = np.empty((4,) + self.k2.shape)
        self.lam[0] = -2.0 * self.Am * self.M * self.k2
        for v in range(3):
            self.lam[1 + v] = -self.L * self.kk[v]
        self.elastic_on = any(abs(x) > 0 for e in p["eps_star"] for x in e)
        self.B = elastic_B(self.kvec, p) if self.elastic_on else None
        # phase-dependent stiffness: Hu-Chen iterations (oracle/elastic.py)
        self.inhom = bool(p.get("el_inhom", 0)) and self.elastic_on
        if self.inhom:
            from .elastic import HuChen
            self.hc = HuChen(self, p)
            self.hc_warm = bool(p.get("el_warm", 1))
            self.hc_prev = None  # eps(u) of the last solve (warm start)

    # --- transforms -------------------------------------------------------
    def to_k(self, real: np.ndarray) -> np.ndarray:
        return sfft.rfftn(real, axes=(-3, -2, -1), workers=_WORKERS) / self.N

    def to_r(self, khat: np.ndarray) -> np.ndarray:
        return sfft.irfftn(khat * self.N, s=self.shape, axes=(-3, -2, -1), workers=_WORKERS)

    # --- local thermodynamics --------------------------------------------
    def kks(self, X, h):
        """Parabolic KKS: equal chemical potential mu in all phases (Eq.
        equal_mu) and the mixture rule (Eq. x_sum) solved in closed form."""
        H = h.sum(axis=0)
        denom = H / (2.0 * self.Av) + (1.0 - H) / (2.0 * self.Am)
        mu = (X - H * self.Bv - (1.0 - H) * self.Bm) / denom
        Xm = mu / (2.0 * self.Am) + self.Bm
        Xv = mu / (2.0 * self.Av) + self.Bv
        fm = self.A0m + self.Am * (Xm - self.Bm) ** 2
        fv = self.A0v + self.Av * (Xv - self.Bv) ** 2
        return H, mu, Xm, Xv, fm, fv

    def dfb_dphi(self, phi):
        """Derivative of the local part of f_b: double well plus the
        (regularised) pairwise |phi_v phi_q| barrier."""
        if self.obstacle:
            # d/dphi_v of omega_bar S (1 - S), S = sum_q phi_q
            out = np.broadcast_to(self.wbar * (1.0 - 2.0 * phi.sum(axis=0)), phi.shape).copy()
        else:
            out = 2.0 * self.wbar * phi * (1.0 - phi) * (1.0 - 2.0 * phi)
        for v in range(3):
            for q in range(3):
                if q != v:
                    slope = np.clip(phi[v] * phi[q] / self.pair_eps, -1.0, 1.0)
                    out[v] = out[v] + self.omega[v, q] * slope * phi[q]
        return out

    def pair_abs(self, x):
        """Huber-regularised |x| of the pairwise barrier."""
        e = self.pair_eps
        return np.where(np.abs(x) < e, x * x / (2.0 * e), np.abs(x) - 0.5 * e)

    def elastic_potential(self, h):
        """e_v(r) = IFFT[sum_q B_vq(n) h^_q(k)] (homogeneous-modulus solution
        of Eq. u_gov; functional derivative of the elastic energy w.r.t. h_v)."""
        if not self.elastic_on:
            return np.zeros_like(h)
        if self.inhom:
            return self.hc_solve(h)[0]
        hk = self.to_k(h)
        ek = np.einsum("vq...,q...->v...", self.B, hk)
        return self.to_r(ek)

    def hc_solve(self, h):
        """Hu-Chen solve at interpolated fields h, started from the previous
        solve's eps(u) when the warm start is on (every solve of the model,
        right-hand side or free energy, continues the same sequence)."""
        out = self.hc.solve(h, self.hc_prev if self.hc_warm else None)
        if self.hc_warm:
            self.hc_prev = self.hc.last_eps_u
        self.hc_last_iters = out[4]
        return out

    def project(self, yhat: np.ndarray) -> np.ndarray:
        """The obstacle barrier's bound: the order parameters clamped to
        [0, 1] in real space; the composition's coefficients are kept as
        they are (its mean stays exact).  The identity without the obstacle."""
        if not self.obstacle:
            return yhat
        real = self.to_r(yhat)
        real[1:] = np.clip(real[1:], 0.0, 1.0)
        out = self.to_k(real)
        out[0] = yhat[0]
        return out

    # --- right-hand sides -------------------------------------------------
    def rhs_explicit(self, yhat: np.ndarray) -> np.ndarray:
        """f^E(y): the non-stiff remainder of Eqs. composition and order."""
        real = self.to_r(yhat)
        X, phi = real[0], real[1:4]
        h = h_interp(phi)
        hp = h_prime(phi)
        H, mu, Xm, Xv, fm, fv = self.kks(X, h)
        e = self.elastic_potential(h)
        g = self.dfb_dphi(phi) + hp * (fv - fm - mu * (Xv - Xm)) + hp * e
        qfield = mu - 2.0 * self.Am * X
        fE = np.empty_like(yhat)
        fE[0] = -self.M * self.k2 * self.to_k(qfield)
        fE[1:4] = -self.L * self.to_k(g)
        return fE

    def rhs_implicit(self, yhat: np.ndarray) -> np.ndarray:
        """f^I(y) = lambda(k) y^(k)."""
        return self.lam * yhat

    def solve_implicit(self, gamma: float, rhat: np.ndarray) -> np.ndarray:
        """Solve (I - gamma lambda) z = r, diagonal in k (the stage linear
        solve of Sec. 4.4)."""
        return rhat / (1.0 - gamma * self.lam)

    # --- diagnostics --------------------------------------------------------
    def free_energy(self, yhat: np.ndarray) -> float:
        """F = int (f_b + f_el + f_ch) dV (Sec. 4.1) with the same readings."""
        real = self.to_r(yhat)
        X, phi = real[0], real[1:4]
        h = h_interp(phi)
        H, mu, Xm, Xv, fm, fv = self.kks(X, h)
        if self.obstacle:
            S = phi.sum(axis=0)
            local = self.wbar * S * (1.0 - S)
        else:
            local = self.wbar * (phi ** 2 * (1.0 - phi) ** 2).sum(axis=0)
        for v in range(3):
            for q in range(v + 1, 3):
                local = local + self.omega[v, q] * self.pair_abs(phi[v] * phi[q])
        local = local + H * fv + (1.0 - H) * fm
        F = local.sum() * self.dV
        nx = self.shape[2]
        w = np.full(self.k2.shape, 2.0)
        w[..., 0] = 1.0
        if nx % 2 == 0:
            w[..., nx // 2] = 1.0
        V = self.N * self.dV
        for v in range(3):
            F += 0.5 * V * np.sum(w * self.kk[v] * np.abs(yhat[1 + v]) ** 2)
        if self.inhom:
            _, sig, el, _, _ = self.hc_solve(h)
            F += 0.5 * float(np.sum(sig * el)) * self.dV
        elif self.elastic_on:
            hk = self.to_k(h)
            for v in range(3):
                for q in range(3):
                    F += 0.5 * V * np.sum(w * self.B[v, q] * (hk[v] * np.conj(hk[q])).real)
        return float(F)


def elastic_B(kvec, p: dict) -> np.ndarray:
    """Khachaturyan kernel B_vq(n) = eps*_v : C : eps*_q - n.sigma*_v.Omega(n).sigma*_q.n
    with Omega^{-1}_ik = C_ijkl n_j n_l and sigma* = C : eps* (homogeneous
    modulus), n = k/|k|, and B(0) = 0 (stress-free mean strain)."""
    KX, KY, KZ = kvec
    C = cubic_stiffness(p["C11"], p["C12"], p["C44"])
    eps = [voigt_to_tensor(e) for e in p["eps_star"]]
    sig = [np.einsum("ijkl,kl->ij", C, e) for e in eps]
    shape = KX.shape
    kn = np.sqrt(KX ** 2 + KY ** 2 + KZ ** 2)
    safe = np.where(kn > 0, kn, 1.0)
    n = np.stack([KX / safe, KY / safe, KZ / safe], axis=-1).reshape(-1, 3)
    Oinv = np.einsum("ijkl,mj,ml->mik", C, n, n)
    zero = (kn.reshape(-1) == 0)
    Oinv[zero] = np.eye(3)
    Om = np.linalg.inv(Oinv)
    B = np.empty((3, 3) + shape)
    sn = [n @ s.T for s in sig]  # (sigma*_v n)_i per k
    for v in range(3):
        for q in range(3):
            c = float(np.sum(eps[v] * sig[q]))
            val = c - np.einsum("mi,mik,mk->m", sn[v], Om, sn[q])
            val[zero] = 0.0
            B[v, q] = val.reshape(shape)
    return B
