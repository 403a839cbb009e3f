"""ORACLE -- test infrastructure only (tests, the package smoke check and the
benchmark's CPU legs may import it; the product never does).

Arbitrary initial system operators (Sec. IV, "General initial density
operators"): the reduced map G_t is linear (Eq. Gt-linearity) and commutes
with molecular relabelling (Eq. Gt-covariance), so rho_S(t) for any initial
operator in the single-excitation manifold (Eq. arbitrary-initial-expansion)
follows from the five representative propagations of Table
tab:representative-initial-operators:
    |c><c| (d = 0), |e_1><c|, |c><e_1|, |e_1><e_1| (d = 1), |e_1><e_2| (d = 2).

Plain and slow on purpose: every G_t[|a><b|] is formed as a dense
(N+1) x (N+1) matrix by relabelling a representative's dense response with an
explicit permutation matrix (Eqs. reconstruct-ec, reconstruct-ee), then the
responses are summed with the initial operator's entries as weights.  Dense
matrices use the basis {c, e_1 .. e_N} (index 0 = cavity, i = molecule i).
"""
from __future__ import annotations

import numpy as np

from . import SA

# representative name -> (distinguished molecules, (row, col) of its single nonzero entry)
REPRESENTATIVES = {"cc": (0, (0, 0)), "ec": (1, (1, 0)), "ce": (1, (0, 1)), "ee": (1, (1, 1)), "e1e2": (2, (1, 2))}


def physical_dense(sa: SA, x: np.ndarray) -> np.ndarray:
    """Dense rho_S from the physical representative of a state of a hierarchy
    with d distinguished molecules.  An entry (a, b) is the variable named by
    the categories of a and b: molecule i <= d is its own category, the others
    share the zero category; two different molecules of the zero category
    give T, the same molecule gives P."""
    N, d = sa.N, sa.d
    ix = sa.rho0_index()
    name = (lambda i: "d" if i == 1 else "0") if d == 1 else (lambda i: str(i) if i <= d else "0")
    rho = np.zeros((N + 1, N + 1), complex)
    for a in range(N + 1):
        for b in range(N + 1):
            if a == 0 and b == 0:
                k = "Z"
            elif b == 0:
                k = "X" + name(a)
            elif a == 0:
                k = "Y" + name(b)
            elif a == b:
                k = "P" + name(a)
            elif name(a) == name(b):
                k = "T0"
            else:
                k = "S" + name(a) + name(b)
            rho[a, b] = x[ix[k]]
    return rho


def representative_hierarchies(N, m, L, bath, detuning=0.0, g=0.0, kappa=0.0, term=0.0) -> dict:
    """The five reduced hierarchies with their unit initial operators as
    factorised initial states (hierarchy ADOs zero).  |e_1><e_2| needs N >= 2."""
    out = {}
    for key, (d, (a, b)) in REPRESENTATIVES.items():
        if max(a, b) > N:
            continue
        sa = SA(N, m, L, bath, detuning, g, kappa, term=term, d=d)
        unit = np.zeros((N + 1, N + 1), complex)
        unit[a, b] = 1.0
        out[key] = (sa, sa.initial_state_dense(unit))
    return out


def responses(hier: dict, dt: float, nsteps: int) -> dict:
    """G_t[representative] as dense matrices after nsteps RK4 steps."""
    return {k: physical_dense(sa, sa.rk4(x, dt, nsteps)) for k, (sa, x) in hier.items()}


def _perm(N, pairs) -> np.ndarray:
    """Permutation matrix of a relabelling that sends molecule s to t for each
    (s, t) in pairs (the cavity stays), completed by the remaining molecules
    in increasing order."""
    src = [s for s, _ in pairs]
    dst = [t for _, t in pairs]
    rest_s = [i for i in range(1, N + 1) if i not in src]
    rest_t = [i for i in range(1, N + 1) if i not in dst]
    pi = {0: 0}
    pi.update(dict(pairs))
    pi.update(dict(zip(rest_s, rest_t)))
    U = np.zeros((N + 1, N + 1))
    for s, t in pi.items():
        U[t, s] = 1.0
    return U


def reconstruct(resp: dict, rho0: np.ndarray) -> np.ndarray:
    """rho_S(t) = sum_ab rho0[a, b] G_t[|a><b|], each G_t[|a><b|] the
    relabelled response of its representative: U G_t[rep] U^T with U sending
    molecule 1 to the molecule of a (or b), and 2 to b for a molecular
    coherence."""
    n = rho0.shape[0]
    N = n - 1
    out = np.zeros((n, n), complex)
    for a in range(n):
        for b in range(n):
            w = rho0[a, b]
            if w == 0:
                continue
            if a == 0 and b == 0:
                R, U = resp["cc"], np.eye(n)
            elif b == 0:
                R, U = resp["ec"], _perm(N, [(1, a)])
            elif a == 0:
                R, U = resp["ce"], _perm(N, [(1, b)])
            elif a == b:
                R, U = resp["ee"], _perm(N, [(1, a)])
            else:
                R, U = resp["e1e2"], _perm(N, [(1, a), (2, b)])
            out += w * (U @ R @ U.T)
    return out
