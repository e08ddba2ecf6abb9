"""ImEx additive Runge-Kutta integrator of the oracle (Sec. 4.4).

TEST INFRASTRUCTURE ONLY (see oracle/model.py).

Stage equations (Eq. ARK_stage), step completion (Eq. ARK_method), embedded
solution (Eq. ARK_embedding), WRMS norm and weights (Eqs. wrms_norm,
wrms_weights). The WRMS norm is taken over the real-space values of all four
fields (N = 4 n^3 entries), with weights from the real-space previous
solution: the paper integrates in reciprocal space but applies the
tolerances pointwise to the field change (Sec. 2.3), so the error estimate
is transformed back to real space before it is normed.

Tables (Sec. 4.4 names the family: first to fourth order with 1, 3, 4 and 6
right-hand-side evaluations per step):
* ImEx (forward-backward) Euler written as a 2-stage ARK pair;
* ARK2 of Giraldo, Kelly & Constantinescu (2013): three stages, ESDIRK with
  gamma = 1 - 1/sqrt(2), first-order embedding;
* ARK3(2)4L[2]SA of Kennedy & Carpenter (2003): four stages, second-order
  embedding;
* ARK4(3)6L[2]SA of Kennedy & Carpenter (2003), the fourth-order method of
  Sec. 2.3, with its third-order embedding.
All coefficients are checked by the order-condition tests, not trusted as
typed.
"""
from __future__ import annotations

from fractions import Fraction as Fr

import numpy as np


def _f(rows):
    return np.array([[float(Fr(x)) for x in r] for r in rows])


def _v(xs):
    return np.array([float(Fr(x)) for x in xs])


class Tableau:
    def __init__(self, name, AE, AI, bE, bI, btE=None, btI=None, order=1, emb_order=0):
        self.name = name
        self.AE, self.AI = AE, AI
        self.bE, self.bI = bE, bI
        self.btE, self.btI = btE, btI
        self.s = AE.shape[0]
        self.order, self.emb_order = order, emb_order
        self.cE = AE.sum(axis=1)
        self.cI = AI.sum(axis=1)

    @property
    def adaptive(self):
        return self.btE is not None


def euler() -> Tableau:
    """First-order ImEx Euler: explicit forward Euler on f^E, backward Euler on
    f^I; one right-hand-side evaluation per step."""
    AE = _f([["0", "0"], ["1", "0"]])
    AI = _f([["0", "0"], ["0", "1"]])
    return Tableau("imex-euler", AE, AI, _v(["1", "0"]), _v(["0", "1"]), order=1)


def ark436l2sa() -> Tableau:
    """ARK4(3)6L[2]SA (Kennedy & Carpenter 2003): ESDIRK implicit part with
    gamma = 1/4, six stages, explicit first stage, stiffly accurate."""
    AE = _f([
        ["0", "0", "0", "0", "0", "0"],
        ["1/2", "0", "0", "0", "0", "0"],
        ["13861/62500", "6889/62500", "0", "0", "0", "0"],
        ["-116923316275/2393684061468", "-2731218467317/15368042101831",
         "9408046702089/11113171139209", "0", "0", "0"],
        ["-451086348788/2902428689909", "-2682348792572/7519795681897",
         "12662868775082/11960479115383", "3355817975965/11060851509271", "0", "0"],
        ["647845179188/3216320057751", "73281519250/8382639484533",
         "552539513391/3454668386233", "3354512671639/8306763924573", "4040/17871", "0"],
    ])
    AI = _f([
        ["0", "0", "0", "0", "0", "0"],
        ["1/4", "1/4", "0", "0", "0", "0"],
        ["8611/62500", "-1743/31250", "1/4", "0", "0", "0"],
        ["5012029/34652500", "-654441/2922500", "174375/388108", "1/4", "0", "0"],
        ["15267082809/155376265600", "-71443401/120774400", "730878875/902184768",
         "2285395/8070912", "1/4", "0"],
        ["82889/524892", "0", "15625/83664", "69875/102672", "-2260/8211", "1/4"],
    ])
    b = _v(["82889/524892", "0", "15625/83664", "69875/102672", "-2260/8211", "1/4"])
    bt = _v(["4586570599/29645900160", "0", "178811875/945068544", "814220225/1159782912",
             "-3700637/11593932", "61727/225920"])
    return Tableau("ark4(3)6l[2]sa", AE, AI, b.copy(), b.copy(), bt.copy(), bt.copy(), order=4, emb_order=3)


def ark2_giraldo() -> Tableau:
    """ARK2 of Giraldo, Kelly & Constantinescu (2013): explicit first stage,
    ESDIRK implicit part with gamma = 1 - 1/sqrt(2), stiffly accurate, shared
    weights b, first-order embedding; abscissae c = (0, 2 - sqrt(2), 1)."""
    r2 = np.sqrt(2.0)
    g = 1.0 - 1.0 / r2
    a = (3.0 + 2.0 * r2) / 6.0
    AE = np.array([[0.0, 0.0, 0.0], [2.0 - r2, 0.0, 0.0], [1.0 - a, a, 0.0]])
    AI = np.array([[0.0, 0.0, 0.0], [g, g, 0.0], [1.0 / (2.0 * r2), 1.0 / (2.0 * r2), g]])
    b = AI[2].copy()
    bt = np.array([(4.0 - r2) / 8.0, (4.0 - r2) / 8.0, 1.0 / (2.0 * r2)])
    return Tableau("ark2", AE, AI, b.copy(), b.copy(), bt.copy(), bt.copy(), order=2, emb_order=1)


def ark324l2sa() -> Tableau:
    """ARK3(2)4L[2]SA (Kennedy & Carpenter 2003): four stages, explicit first
    stage, ESDIRK implicit part with gamma = 1767732205903/4055673282236,
    stiffly accurate, shared weights b, second-order embedding."""
    g = "1767732205903/4055673282236"
    AE = _f([
        ["0", "0", "0", "0"],
        ["1767732205903/2027836641118", "0", "0", "0"],
        ["5535828885825/10492691773637", "788022342437/10882634858940", "0", "0"],
        ["6485989280629/16251701735622", "-4246266847089/9704473918619",
         "10755448449292/10357097424841", "0"],
    ])
    AI = _f([
        ["0", "0", "0", "0"],
        [g, g, "0", "0"],
        ["2746238789719/10658868560708", "-640167445237/6845629431997", g, "0"],
        ["1471266399579/7840856788654", "-4482444167858/7529755066697",
         "11266239266428/11593286722821", g],
    ])
    b = AI[3].copy()
    bt = _v(["2756255671327/12835298489170", "-10771552573575/22201958757719",
             "9247589265047/10645013368117", "2193209047091/5459859503100"])
    return Tableau("ark3(2)4l[2]sa", AE, AI, b.copy(), b.copy(), bt.copy(), bt.copy(), order=3, emb_order=2)


TABLES = {"euler": euler, "ark2": ark2_giraldo, "ark3": ark324l2sa, "ark4": ark436l2sa}


def stability_function(tab: Tableau, zI: complex, zE: complex) -> complex:
    """R(zI, zE) = 1 + (zI bI + zE bE)^T (I - zI AI - zE AE)^{-1} 1 for the
    scalar test equation y' = lambda_I y + lambda_E y."""
    s = tab.s
    M = np.eye(s) - zI * tab.AI - zE * tab.AE
    u = np.linalg.solve(M.astype(complex), np.ones(s, dtype=complex))
    return 1.0 + (zI * tab.bI + zE * tab.bE) @ u


def wrms(v: np.ndarray, yprev: np.ndarray, rtol: float, atol: float) -> float:
    """||v||_WRMS = sqrt(1/N sum (v_i w_i)^2), w_i = 1/(rtol |y_{n-1,i}| + atol)."""
    w = 1.0 / (rtol * np.abs(yprev) + atol)
    return float(np.sqrt(np.mean((v * w) ** 2)))


def ark_step(model, yhat: np.ndarray, dt: float, tab: Tableau, rtol: float = 1e-4,
             atol: float = 1e-8, want_lte: bool = True):
    """One ImEx-ARK step from y_{n-1} = yhat. Returns (y_n, ||LTE||_WRMS, stats)."""
    s = tab.s
    Z, FE = [], []
    need_fe = [bool(tab.bE[i] != 0.0 or np.any(tab.AE[i + 1:, i] != 0.0)
                    or (tab.btE is not None and tab.btE[i] != 0.0)) for i in range(s)]
    nrhs = 0
    for i in range(s):
        r = yhat.copy()
        for j in range(i):
            if tab.AI[i, j] != 0.0:
                r = r + dt * tab.AI[i, j] * model.rhs_implicit(Z[j])
            if tab.AE[i, j] != 0.0:
                r = r + dt * tab.AE[i, j] * FE[j]
        if tab.AI[i, i] != 0.0:
            z = model.solve_implicit(dt * tab.AI[i, i], r)
        else:
            z = r
        Z.append(z)
        if need_fe[i]:
            FE.append(model.rhs_explicit(z))
            nrhs += 1
        else:
            FE.append(None)
    ynew = yhat.copy()
    for i in range(s):
        if tab.bI[i] != 0.0:
            ynew = ynew + dt * tab.bI[i] * model.rhs_implicit(Z[i])
        if tab.bE[i] != 0.0:
            ynew = ynew + dt * tab.bE[i] * FE[i]
    err = 0.0
    if tab.adaptive and want_lte:
        lte = np.zeros_like(yhat)
        for i in range(s):
            dI = tab.bI[i] - tab.btI[i]
            dE = tab.bE[i] - tab.btE[i]
            if dI != 0.0:
                lte = lte + dt * dI * model.rhs_implicit(Z[i])
            if dE != 0.0:
                lte = lte + dt * dE * FE[i]
        err = wrms(model.to_r(lte), model.to_r(yhat), rtol, atol)
    return ynew, err, {"rhs": nrhs}


def chen_shen_euler(model, yhat: np.ndarray, dt: float) -> np.ndarray:
    """The hand-coded first-order semi-implicit step of Chen and Shen:
    y_n = (y_{n-1} + dt f^E(y_{n-1})) / (1 - dt lambda)."""
    return (yhat + dt * model.rhs_explicit(yhat)) / (1.0 - dt * model.lam)


class Controller:
    """Proposed PI step-size controller (the paper uses ARKODE's defaults and
    gives no constants): h_new = h min(eta_max, max(eta_min,
    safety e_n^{-k1/q} e_{n-1}^{k2/q})), q = embedded order + 1; after a
    rejection h *= max(eta_reject_min, safety e^{-1/q}) and growth is capped at 1
    for the next step."""

    def __init__(self, p: dict, q: int):
        self.safety = p["safety"]
        self.k1, self.k2 = p["k1"], p["k2"]
        self.eta_max, self.eta_min = p["eta_max"], p["eta_min"]
        self.eta_rej = p["eta_reject_min"]
        self.q = q
        self.e_prev = 1.0
        self.after_reject = False

    def accept(self, h: float, e: float) -> float:
        e = max(e, 1e-10)
        eta = self.safety * e ** (-self.k1 / self.q) * self.e_prev ** (self.k2 / self.q)
        cap = 1.0 if self.after_reject else self.eta_max
        eta = min(cap, max(self.eta_min, eta))
        self.e_prev = e
        self.after_reject = False
        return h * eta

    def reject(self, h: float, e: float) -> float:
        self.after_reject = True
        if not np.isfinite(e):
            return h * 0.25
        return h * max(self.eta_rej, self.safety * e ** (-1.0 / self.q))


def advance(model, yhat: np.ndarray, t0: float, t_final: float, tab: Tableau, p: dict,
            rtol: float, atol: float, h0: float | None = None, replay=None, max_steps: int = 100000):
    """Adaptive integration from t0 to t_final. With `replay` (a list of
    (h, accepted) attempts taken elsewhere) the step sizes and decisions are
    followed instead of computed, and the oracle's own errors are reported so
    that decisions can be compared. Returns (y, t, log) with log a list of
    (t, h, e, accepted)."""
    ctl = Controller(p, tab.emb_order + 1)
    h = p["h0"] if h0 is None else h0
    t = t0
    y = yhat
    log = []
    k = 0
    nrej = 0
    while t < t_final * (1 - 1e-14) and k < max_steps:
        if replay is not None:
            if k >= len(replay):
                break
            h, acc_given = replay[k]
        else:
            h = min(h, t_final - t)
        ynew, e, _ = ark_step(model, y, h, tab, rtol, atol)
        ok = np.isfinite(e) and e <= 1.0
        if replay is not None:
            ok = bool(acc_given)
        log.append((t, h, e, ok))
        k += 1
        if ok:
            y = model.project(ynew) if hasattr(model, "project") else ynew
            t = t + h
            nrej = 0
            hn = ctl.accept(h, e)
        else:
            nrej += 1
            if nrej > p["max_rejects"]:
                raise RuntimeError("step failed: too many rejections")
            hn = ctl.reject(h, e)
        h = min(max(hn, p["h_min"]), p["h_max"])
    return y, t, log
