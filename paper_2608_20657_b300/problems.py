"""Problem set-up on the product side: sa_params from a workload description
(bath through the library's sa_bath_drude_lorentz) and the factorised initial
unique variables of the physical representative.

Initial states (Sec. V.A): cavity |c><c| (Eq. cavity-initial-uvar), bright
|B><B| (Eq. bright-initial-uvar), upper / lower polariton (Eqs. upper-/lower-
polariton-initial) with tan(2 theta) = Omega_R / Delta, Delta = omega_cav -
eps_x, theta in [0, pi/2]; and a random permutation-invariant density matrix
built from seeded draws: dark-block eigenvalue P_0 - T_0 = w_dark / (N - 1),
cavity-bright block W = (1 - w_dark) A A^+ / tr(A A^+) with
W = [[Z, sqrt(N) Y_0], [sqrt(N) X_0, P_0 + (N-1) T_0]].
"""
from __future__ import annotations

import math

import numpy as np

from . import binding as B

_SCHEME = {"high_t": B.BATH_HIGH_T, "matsubara": B.BATH_MATSUBARA, "pade": B.BATH_PADE}


# the cm^-1 / K / fs unit set of the paper's Sec. V: with hbar = 1 an energy
# E in cm^-1 is the angular frequency 2 pi c E, in rad/fs
C_CM_PER_FS = 2.99792458e-5        # speed of light (exact SI value), cm/fs
KB_CM_PER_K = 0.695034800486127    # k_B / (h c) from the exact SI k, h, c: cm^-1 per K
RAD_PER_FS_PER_CM = 2.0 * math.pi * C_CM_PER_FS


def in_library_units(w: dict) -> dict:
    """A workload description in the library's units (hbar = 1).  For a
    "cm-1/fs" description the energies become angular frequencies in rad/fs,
    kT = k_B T, gsn = g sqrt(N) = Omega_R / 2, and dt is in fs; others are
    returned unchanged."""
    if w.get("units") != "cm-1/fs":
        return w
    f = RAD_PER_FS_PER_CM
    r = dict(w)
    r.update(lam=w["lam_cm"] * f, gam=w["gam_cm"] * f, kT=KB_CM_PER_K * w["T_K"] * f, gsn=0.5 * w["omega_R_cm"] * f,
             detuning=w["detuning_cm"] * f, kappa=w["kappa_cm"] * f, dt=w["dt_fs"])
    return r


def params_from(w: dict) -> B.Params:
    w = in_library_units(w)
    bath = B.bath_drude_lorentz(w["lam"], w["gam"], w["kT"], _SCHEME[w["scheme"]], w["poles"], w["sigma"])
    N = int(w["N"])
    term = B.bath_terminator(w["lam"], w["gam"], w["kT"], w["poles"]) if w.get("terminator") else 0.0
    return B.make_params(N, len(bath["c"]), w["L"], bath, detuning=w["detuning"], g=w["gsn"] / math.sqrt(N),
                         kappa=w["kappa"], term=term, d=w.get("d", 0))


def theta(N: int, g: float, detuning: float) -> float:
    return 0.5 * math.atan2(2.0 * g * math.sqrt(N), -detuning)


def rho0_vars(w: dict, draws: dict | None = None) -> np.ndarray:
    """(Z, X_0, Y_0, P_0, T_0) of the initial physical representative."""
    w = in_library_units(w)
    N = int(w["N"])
    g = w["gsn"] / math.sqrt(N)
    kind = w["init"]
    if kind == "cavity":
        return np.array([1, 0, 0, 0, 0], complex)
    if kind == "bright":
        return np.array([0, 0, 0, 1 / N, 1 / N], complex)
    if kind in ("up", "lp"):
        th = theta(N, g, w["detuning"])
        s, c = math.sin(th), math.cos(th)
        if kind == "up":
            return np.array([c * c, s * c / math.sqrt(N), s * c / math.sqrt(N), s * s / N, s * s / N], complex)
        return np.array([s * s, -s * c / math.sqrt(N), -s * c / math.sqrt(N), c * c / N, c * c / N], complex)
    if kind == "random":
        A = draws["A"]
        wd = draws["w_dark"] if N >= 2 else 0.0
        W = A @ A.conj().T
        W = (1.0 - wd) * W / np.trace(W).real
        Z = W[0, 0].real
        Y0 = W[0, 1] / math.sqrt(N)
        X0 = W[1, 0] / math.sqrt(N)
        bright = W[1, 1].real          # P_0 + (N-1) T_0
        dark = wd / (N - 1) if N >= 2 else 0.0   # P_0 - T_0
        P0 = (bright + (N - 1) * dark) / N
        T0 = P0 - dark
        return np.array([Z, X0, Y0, P0, T0], complex)
    raise ValueError(kind)


def phys_vars(w: dict, draws: dict | None = None) -> np.ndarray:
    """The physical representative's variables in the canonical layout, for
    sa_heom_init_physical.  d = 0: Z, X_0, Y_0, P_0, T_0.  d = 1 (categories
    1 = molecule 1, 2 = the other N - 1): Z, X_1, X_2, Y_1, Y_2, P_1, P_2,
    S_12, S_21, T_2, with the N = 1 and N = 2 layouts cut short.  States:
    the permutation-invariant ones of rho0_vars (their molecule-1 entries equal
    the others'), "localised" |e_1><e_1| and "superposed"
    sqrt(0.3)|e_1> + sqrt(0.7)|c> (Sec. V.F)."""
    N, d, kind = int(w["N"]), int(w.get("d", 0)), w["init"]
    if d == 0:
        v = rho0_vars(w, draws)
        return v if N >= 2 else v[:4]
    if d != 1:
        raise ValueError("phys_vars covers d = 0 and d = 1")
    if kind == "localised":
        Z, X1, Y1, P1, X2, Y2, P2, S, T = 0.0, 0, 0, 1.0, 0, 0, 0, 0, 0
    elif kind == "superposed":
        a = math.sqrt(0.21)
        Z, X1, Y1, P1, X2, Y2, P2, S, T = 0.7, a, a, 0.3, 0, 0, 0, 0, 0
    else:
        Z, X0, Y0, P0, T0 = rho0_vars(w, draws)
        X1 = X2 = X0
        Y1 = Y2 = Y0
        P1 = P2 = P0
        S = T = T0   # any two molecules: the off-diagonal entry of the permutation-invariant block
    if N == 1:
        return np.array([Z, X1, Y1, P1], complex)
    out = [Z, X1, X2, Y1, Y2, P1, P2, S, S]
    if N >= 3:
        out.append(T)
    return np.array(out, complex)
