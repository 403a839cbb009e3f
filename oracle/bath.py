"""ORACLE -- test infrastructure only.  Bath decompositions in extended precision.

The finite exponential bath correlation function of Eq. BCF-exp,
``C_m(t) = sum_k c_k exp(-nu_k t)`` with ``C_m^*(t) = sum_k cc_k exp(-nu_k t)``,
for the Drude-Lorentz spectral density of Eq. Drude_Lorentz,
``J(w) = 2 lambda gamma w / (w^2 + gamma^2)``, inserted in Eq. BCF-spectral.

Three schemes (the paper names Matsubara, Pade or a fit without formulas):

* ``high_t``: one exponential, the high-temperature limit
  ``cot(beta gamma / 2) -> 2 / (beta gamma)``.
* ``matsubara``: the gamma pole with the exact cotangent plus the first
  ``K`` Matsubara poles ``nu_j = 2 pi j / beta``.
* ``pade``: the [K-1/K] Pade approximant in ``z = x^2`` of
  ``(coth x - 1/x) / x``, built from its Taylor (Bernoulli) coefficients in
  exact rational arithmetic, written as ``coth x ~ 1/x + sum_j 2 eta_j x /
  (x^2 + xi_j^2)``.  Poles ``nu_j = 2 xi_j / beta``; the gamma-pole weight uses
  the approximant continued to imaginary argument,
  ``cot~(y) = 1/y - sum_j 2 eta_j y / (xi_j^2 - y^2)``.

Static Gaussian disorder (Eq. C_static) is one more channel with
``c = cc = sigma^2`` and ``nu = 0``.

Every channel here has a real rate, so ``cc_k = conj(c_k)`` (the rule stated
below Eq. BCF-exp for self-conjugate rates).
"""
from __future__ import annotations

from fractions import Fraction

import mpmath as mp
import numpy as np

mp.mp.dps = 50


def _bernoulli(n: int) -> Fraction:
    """B_n (B_1 = -1/2) from the recurrence sum_{j<=n} C(n+1, j) B_j = 0."""
    B = [Fraction(1)]
    for mm in range(1, n + 1):
        s = Fraction(0)
        for j in range(mm):
            s += Fraction(_binom(mm + 1, j)) * B[j]
        B.append(-s / (mm + 1))
    return B[n]


def _binom(n: int, k: int) -> int:
    from math import comb
    return comb(n, k)


def coth_series_coeffs(nterms: int) -> list[Fraction]:
    """a_n with (coth x - 1/x)/x = sum_{n>=1} a_n z^{n-1}, z = x^2;
    a_n = 2^{2n} B_{2n} / (2n)!."""
    from math import factorial
    return [Fraction(2 ** (2 * n)) * _bernoulli(2 * n) / factorial(2 * n) for n in range(1, nterms + 1)]


def pade_poles(K: int):
    """(eta_j, xi_j), j = 1..K, of the [K-1/K] Pade approximant of
    F(z) = (coth sqrt(z) - 1/sqrt(z))/sqrt(z) written as
    F(z) ~ sum_j 2 eta_j / (z + xi_j^2).  Returned as mpmath numbers."""
    a = coth_series_coeffs(2 * K)           # F(z) = sum_{i>=0} a[i] z^i
    # Q(z) = 1 + q_1 z + ... + q_K z^K with (F Q)_i = 0 for i = K .. 2K-1
    # (the numerator P has degree K-1).  Exact rational Gaussian elimination.
    A = [[a[i - j] if i - j >= 0 else Fraction(0) for j in range(1, K + 1)] for i in range(K, 2 * K)]
    rhs = [-a[i] for i in range(K, 2 * K)]
    q = _solve_exact(A, rhs)
    Q = [Fraction(1)] + q                   # ascending coefficients
    P = [sum((a[i - j] * Q[j] for j in range(0, i + 1)), Fraction(0)) for i in range(K)]
    # roots of Q in z: Q(z) = 0 -> z_j = -xi_j^2
    coeffs_desc = [mp.mpf(c.numerator) / c.denominator for c in reversed(Q)]
    roots = mp.polyroots(coeffs_desc, maxsteps=200, extraprec=200)
    dQ = [Q[j] * j for j in range(1, K + 1)]  # ascending, Q'(z)

    def ev(cs, z):
        return sum(mp.mpf(c.numerator) / c.denominator * z ** i for i, c in enumerate(cs))

    out = []
    for z in roots:
        z = mp.re(z) if abs(mp.im(z)) < mp.mpf(10) ** -30 else z
        res = ev(P, z) / ev(dQ, z)          # F ~ sum res / (z - z_j)
        xi = mp.sqrt(-z)
        eta = res / 2
        out.append((eta, xi))
    out.sort(key=lambda t: mp.re(t[1]))
    return out


def _solve_exact(A, b):
    n = len(b)
    M = [list(row) + [bi] for row, bi in zip(A, b)]
    for col in range(n):
        piv = next(r for r in range(col, n) if M[r][col] != 0)
        M[col], M[piv] = M[piv], M[col]
        for r in range(n):
            if r != col and M[r][col] != 0:
                f = M[r][col] / M[col][col]
                M[r] = [x - f * y for x, y in zip(M[r], M[col])]
    return [M[i][n] / M[i][i] for i in range(n)]


def _dl_pole_terms(lam, gam, kT, etas, xis, cot_gamma):
    beta = 1 / mp.mpf(kT)
    lam, gam = mp.mpf(lam), mp.mpf(gam)
    c = [lam * gam * (cot_gamma - 1j)]
    nu = [gam]
    for eta, xi in zip(etas, xis):
        nuj = 2 * xi / beta
        c.append(eta * (4 * lam * gam / beta) * nuj / (nuj ** 2 - gam ** 2))
        nu.append(nuj)
    return c, nu


def _pack(c, nu, sigma=0.0):
    c = [complex(x) for x in c]
    nu = [complex(x) for x in nu]
    if sigma and sigma > 0:
        c.append(complex(sigma * sigma))
        nu.append(0j)
    c = np.array(c, dtype=complex)
    return {"c": c, "cc": np.conj(c), "nu": np.array(nu, dtype=complex)}


def high_t(lam, gam, kT, sigma=0.0):
    """m = 1: c_0 = 2 lambda kT - i lambda gamma, nu_0 = gamma."""
    c = [2 * mp.mpf(lam) * mp.mpf(kT) - 1j * mp.mpf(lam) * mp.mpf(gam)]
    return _pack(c, [mp.mpf(gam)], sigma)


def matsubara(lam, gam, kT, K, sigma=0.0):
    """gamma pole (exact cot) + K Matsubara poles."""
    beta = 1 / mp.mpf(kT)
    cot = mp.cot(beta * mp.mpf(gam) / 2)
    etas = [mp.mpf(1)] * K
    xis = [mp.pi * j for j in range(1, K + 1)]
    c, nu = _dl_pole_terms(lam, gam, kT, etas, xis, cot)
    return _pack(c, nu, sigma)


def pade(lam, gam, kT, K, sigma=0.0):
    """gamma pole + K Pade poles ([K-1/K] in z = x^2)."""
    poles = pade_poles(K)
    etas = [mp.re(e) for e, _ in poles]
    xis = [mp.re(x) for _, x in poles]
    beta = 1 / mp.mpf(kT)
    y = beta * mp.mpf(gam) / 2
    cot_approx = 1 / y - sum(2 * e * y / (x ** 2 - y ** 2) for e, x in zip(etas, xis))
    c, nu = _dl_pole_terms(lam, gam, kT, etas, xis, cot_approx)
    return _pack(c, nu, sigma)


def terminator(lam, gam, kT, K):
    """Terminator strength Delta for a Drude-Lorentz bath kept to K Matsubara
    terms: the omitted terms j > K of the Matsubara expansion (Eq. BCF-exp with
    nu_j = 2 pi j kT, c_j = 4 lam gam kT nu_j / (nu_j^2 - gam^2)) taken as white
    noise, Delta = sum_{j > K} c_j / nu_j, summed directly in 50-digit
    arithmetic (the sum converges like 1/j^2)."""
    lam, gam, kT = mp.mpf(lam), mp.mpf(gam), mp.mpf(kT)

    def term(j):
        nuj = 2 * mp.pi * j * kT
        return 4 * lam * gam * kT / (nuj ** 2 - gam ** 2)

    return float(mp.nsum(term, [K + 1, mp.inf]))


def coth_approx(x, scheme: str, K: int):
    """coth x as represented by a scheme: 1/x + sum 2 eta x / (x^2 + xi^2)."""
    if scheme == "matsubara":
        poles = [(mp.mpf(1), mp.pi * j) for j in range(1, K + 1)]
    else:
        poles = pade_poles(K)
    x = mp.mpf(x)
    return 1 / x + sum(2 * e * x / (x ** 2 + xi ** 2) for e, xi in poles)


def bcf_exact(t, lam, gam, kT):
    """C(t) of Eq. BCF-spectral for the Drude-Lorentz J, by quadrature."""
    beta = 1 / mp.mpf(kT)
    lam, gam, t = mp.mpf(lam), mp.mpf(gam), mp.mpf(t)

    def J(w):
        return 2 * lam * gam * w / (w ** 2 + gam ** 2)

    re = mp.quadosc(lambda w: J(w) * mp.coth(beta * w / 2) * mp.cos(w * t), [0, mp.inf], omega=t) / mp.pi
    im = -mp.quadosc(lambda w: J(w) * mp.sin(w * t), [0, mp.inf], omega=t) / mp.pi
    return complex(re) + 1j * float(im)


def bcf_from(bath, t):
    return complex(np.sum(bath["c"] * np.exp(-bath["nu"] * t)))
