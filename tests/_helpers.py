"""Oracle-side set-up for the parity tests: the oracle's own bath and initial
unique variables from a workload description (written independently of the
product package's problem set-up)."""
from __future__ import annotations

import math

import numpy as np

import oracle
import oracle.bath as OB


def oracle_bath(w):
    if w["scheme"] == "high_t":
        return OB.high_t(w["lam"], w["gam"], w["kT"], w["sigma"])
    if w["scheme"] == "matsubara":
        return OB.matsubara(w["lam"], w["gam"], w["kT"], w["poles"], w["sigma"])
    return OB.pade(w["lam"], w["gam"], w["kT"], w["poles"], w["sigma"])


def oracle_sa(w, cache=True):
    b = oracle_bath(w)
    N = int(w["N"])
    return oracle.SA(N, len(b["c"]), w["L"], b, w["detuning"], w["gsn"] / math.sqrt(N), w["kappa"], cache=cache)


def oracle_rho0(w, draws=None):
    """Eqs. cavity-initial-uvar, bright-initial-uvar, upper-/lower-polariton-
    initial; the random kind builds rho from the cavity-bright block and the
    dark eigenvalue."""
    N = int(w["N"])
    om = 2.0 * w["gsn"]                       # Omega_R = 2 g sqrt(N)
    th = 0.5 * math.atan2(om, -w["detuning"])  # tan 2theta = Omega_R / (omega_c - eps_x)
    kind = w["init"]
    if kind == "cavity":
        return (1.0, 0.0, 0.0, 0.0, 0.0)
    if kind == "bright":
        return (0.0, 0.0, 0.0, 1.0 / N, 1.0 / N)
    if kind == "up":
        c2, s2, sc = math.cos(th) ** 2, math.sin(th) ** 2, math.sin(th) * math.cos(th)
        return (c2, sc / math.sqrt(N), sc / math.sqrt(N), s2 / N, s2 / N)
    if kind == "lp":
        c2, s2, sc = math.cos(th) ** 2, math.sin(th) ** 2, math.sin(th) * math.cos(th)
        return (s2, -sc / math.sqrt(N), -sc / math.sqrt(N), c2 / N, c2 / N)
    if kind == "random":
        A = np.asarray(draws["A"])
        wd = float(draws["w_dark"])
        Wm = A @ np.conj(A.T)
        Wm = Wm * (1.0 - wd) / np.real(np.trace(Wm))
        # |B> block: [[Z, sqrt(N) Y0], [sqrt(N) X0, P_B]]; dark: P0 - T0 = wd/(N-1)
        Z = Wm[0, 0].real
        X0 = Wm[1, 0] / math.sqrt(N)
        Y0 = Wm[0, 1] / math.sqrt(N)
        PB = Wm[1, 1].real
        d = wd / (N - 1)
        T0 = (PB - d) / N
        P0 = T0 + d
        return (Z, X0, Y0, P0, T0)
    raise ValueError(kind)


def rel_err(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))
