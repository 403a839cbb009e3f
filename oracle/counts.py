"""ORACLE -- test infrastructure only.  Closed-form hierarchy sizes.

* conventional ADO count C(Nm+L, L) (Eq. direct-ado-count) and dense
  variable count C(Nm+L, L)(N+1)^2 (Eq. direct-dimension);
* one-vector storage in decimal GB at 16 bytes per complex double
  (Eqs. resources-naive-memory, resources-uvar-memory) and the reduction
  factor R (Eq. resources-reduction-factor);
* restricted partition counts p_N(l) (Eq. canonical-count-one) and, for
  m > 1 with N >= L, the multiset-of-vectors count from the generating
  function prod_{k>=1} (1 - x^k)^(-C(k+m-1, m-1)).
"""
from __future__ import annotations

from math import comb


def n_ado_conventional(N: int, m: int, L: int) -> int:
    return comb(N * m + L, L)


def n_var_conventional(N: int, m: int, L: int) -> int:
    return n_ado_conventional(N, m, L) * (N + 1) ** 2


def partitions_restricted(l: int, maxparts: int) -> int:
    """Number of partitions of l into at most maxparts positive parts."""
    # p(n, k) = partitions of n into parts of size <= k (conjugate count)
    table = [[0] * (maxparts + 1) for _ in range(l + 1)]
    for k in range(maxparts + 1):
        table[0][k] = 1
    for n in range(1, l + 1):
        for k in range(1, maxparts + 1):
            table[n][k] = table[n][k - 1] + (table[n - k][k] if n >= k else 0)
    return table[l][maxparts] if maxparts >= 0 else 0


def canonical_count_m1(N: int, L: int) -> int:
    return sum(partitions_restricted(l, min(N, l)) if l > 0 else 1 for l in range(L + 1))


def multiset_vector_count(m: int, L: int) -> int:
    """Sum over tiers 0..L of the coefficients of
    prod_{k>=1} (1 - x^k)^(-C(k+m-1, m-1)): multisets of nonzero vectors in
    N0^m with total norm <= L, no length limit (the N >= L count)."""
    coeff = [1] + [0] * L
    for k in range(1, L + 1):
        kinds = comb(k + m - 1, m - 1)          # vectors of norm k
        for _ in range(kinds):                  # multiply by 1/(1-x^k)
            for n in range(k, L + 1):
                coeff[n] += coeff[n - k]
    return sum(coeff)


def table1_row(N: int, L: int, n_can: int, n_unq: int) -> dict:
    """Columns of the paper's resource table for m = 1 as exact integers /
    rationals: naive ADOs, naive GB, canonical ADOs, unique variables,
    unique GB, reduction factor."""
    from fractions import Fraction

    nado = n_ado_conventional(N, 1, L)
    mem_naive = Fraction(16 * (N + 1) ** 2 * nado, 10 ** 9)
    mem_unq = Fraction(16 * n_unq, 10 ** 9)
    R = Fraction(nado * (N + 1) ** 2, n_unq)
    return {"n_ado_naive": nado, "m_ado_naive_gb": mem_naive, "n_ado_can": n_can,
            "n_var_unq": n_unq, "m_var_unq_gb": mem_unq, "R": R}


def sig3(x) -> str:
    """x (int or Fraction, > 0) rounded to 3 significant figures, 'd.dde+X'."""
    from fractions import Fraction

    x = Fraction(x)
    e = 0
    while x >= 10:
        x /= 10
        e += 1
    while x < 1:
        x *= 10
        e -= 1
    mant = round(x * 100)
    if mant >= 1000:
        mant //= 10
        e += 1
    return f"{mant // 100}.{mant % 100:02d}e{e}"
