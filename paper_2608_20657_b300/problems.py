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


def params_from(w: dict) -> B.Params:
    bath = B.bath_drude_lorentz(w["lam"], w["gam"], w["kT"], _SCHEME[w["scheme"]], w["poles"], w["sigma"])
    N = int(w["N"])
    return B.make_params(N, len(bath["c"]), w["L"], bath, detuning=w["detuning"], g=w["gsn"] / math.sqrt(N),
                         kappa=w["kappa"])


def theta(N: int, g: float, detuning: float) -> float:
    return 0.5 * math.atan2(2.0 * g * math.sqrt(N), -detuning)


def rho0_vars(w: dict, draws: dict | None = None) -> np.ndarray:
    """(Z, X_0, Y_0, P_0, T_0) of the initial physical representative."""
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
