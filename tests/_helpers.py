"""Oracle-side set-up for the parity tests: the oracle's own bath and initial
unique variables from a workload description (written independently of the
product package's problem set-up)."""
from __future__ import annotations

import math

import numpy as np

import oracle
import oracle.bath as OB


# hbar = 1 with energies as angular frequencies in rad/fs: E[cm^-1] * 2 pi c;
# k_B / (h c) in cm^-1 per K (CODATA 2018)
_CM_TO_RAD_FS = 2.0 * math.pi * 2.99792458e10 * 1e-15
_KB_CM = 1.380649e-23 / (6.62607015e-34 * 2.99792458e10)  # exact SI k / (h c), cm^-1 per K


def physical(w):
    """A description in cm^-1 / K / fs as the oracle's plain numbers."""
    if w.get("units") != "cm-1/fs":
        return w
    u = dict(w)
    u["lam"], u["gam"] = w["lam_cm"] * _CM_TO_RAD_FS, w["gam_cm"] * _CM_TO_RAD_FS
    u["kT"] = w["T_K"] * _KB_CM * _CM_TO_RAD_FS
    u["gsn"] = w["omega_R_cm"] / 2 * _CM_TO_RAD_FS        # g sqrt(N) = Omega_R / 2
    u["detuning"], u["kappa"] = w["detuning_cm"] * _CM_TO_RAD_FS, w["kappa_cm"] * _CM_TO_RAD_FS
    u["dt"] = w["dt_fs"]
    return u


def oracle_bath(w):
    w = physical(w)
    if w["scheme"] == "high_t":
        return OB.high_t(w["lam"], w["gam"], w["kT"], w["sigma"])
    if w["scheme"] == "matsubara":
        return OB.matsubara(w["lam"], w["gam"], w["kT"], w["poles"], w["sigma"])
    return OB.pade(w["lam"], w["gam"], w["kT"], w["poles"], w["sigma"])


def oracle_sa(w, cache=True):
    b = oracle_bath(w)
    w = physical(w)
    N = int(w["N"])
    term = float(OB.terminator(w["lam"], w["gam"], w["kT"], w["poles"])) if w.get("terminator") else 0.0
    return oracle.SA(N, len(b["c"]), w["L"], b, w["detuning"], w["gsn"] / math.sqrt(N), w["kappa"], cache=cache,
                     term=term, d=w.get("d", 0))


def oracle_initial(sa, w, draws=None):
    """The whole initial hierarchy for a description: permutation-invariant
    states through the five representative values, the Sec. V.F states of a
    d = 1 hierarchy from their dense rho_S entries."""
    kind = w["init"]
    if kind in ("localised", "superposed"):
        ix = sa.rho0_index()
        x = sa.zeros()
        if kind == "localised":
            x[ix["Pd"]] = 1.0
        else:
            x[ix["Z"]], x[ix["Pd"]] = 0.7, 0.3
            x[ix["Xd"]] = x[ix["Yd"]] = math.sqrt(0.7 * 0.3)
        return x
    Z, X0, Y0, P0, T0 = oracle_rho0(w, draws)
    if sa.d == 0:
        return sa.initial_state(Z, X0, Y0, P0, T0)
    ix = sa.rho0_index()
    x = sa.zeros()
    for k, v in ix.items():
        x[v] = {"Z": Z, "X": X0, "Y": Y0, "P": P0, "S": T0, "T": T0}[k[0]]
    return x


def oracle_rho0(w, draws=None):
    """Eqs. cavity-initial-uvar, bright-initial-uvar, upper-/lower-polariton-
    initial; the random kind builds rho from the cavity-bright block and the
    dark eigenvalue."""
    w = physical(w)
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
