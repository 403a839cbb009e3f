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


def in_library_units(w: dict) -> dict:
    """A workload description in the library's units (hbar = 1; the library's
    sa_unit_* conversions).  For a "cm-1/fs" description the energies become
    angular frequencies in rad/fs, kT = k_B T, gsn = g sqrt(N) = Omega_R / 2,
    and dt is in fs; others are returned unchanged."""
    if w.get("units") != "cm-1/fs":
        return w
    f = B.unit_cm_to_rad_fs
    r = dict(w)
    r.update(lam=f(w["lam_cm"]), gam=f(w["gam_cm"]), kT=B.unit_kT_rad_fs(w["T_K"]), gsn=f(0.5 * w["omega_R_cm"]),
             detuning=f(w["detuning_cm"]), kappa=f(w["kappa_cm"]), dt=w["dt_fs"])
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
    """(Z, X_0, Y_0, P_0, T_0) of the initial physical representative
    (sa_heom_initial_vars with d = 0; T_0 = 0 for N = 1)."""
    p = params_from(dict(w, d=0))
    v = B.initial_vars(p, w["init"], draws if w["init"] == "random" else None)
    return np.concatenate([v, np.zeros(5 - v.size, complex)])


def phys_vars(w: dict, draws: dict | None = None) -> np.ndarray:
    """The physical representative's variables in the canonical layout, for
    sa_heom_init_physical (sa_heom_initial_vars).  d = 0: Z, X_0, Y_0, P_0,
    T_0.  d = 1 (categories 1 = molecule 1, 2 = the other N - 1): Z, X_1, X_2,
    Y_1, Y_2, P_1, P_2, S_12, S_21, T_2, with the N = 1 and N = 2 layouts cut
    short.  States: the permutation-invariant ones of rho0_vars, "localised"
    |e_1><e_1| and "superposed" sqrt(0.3)|e_1> + sqrt(0.7)|c> (Sec. V.F)."""
    if int(w.get("d", 0)) not in (0, 1):
        raise ValueError("phys_vars covers d = 0 and d = 1")
    return B.initial_vars(params_from(w), w["init"], draws if w["init"] == "random" else None)
