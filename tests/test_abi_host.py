"""C-ABI library: loads without a GPU, exports every symbol the header
declares, and its host-side bath decompositions agree with the oracle's
extended-precision ones (Eq. BCF-exp for Eq. Drude_Lorentz; Eq. C_static)."""
import ctypes
import os
import re

import math

import numpy as np
import pytest

import oracle.bath as OB
import paper_2608_20657_b300 as S
from paper_2608_20657_b300 import binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            names += re.findall(r"^\s*(?:int|void|const char\*)\s+(sa_\w+)\s*\(", src, re.M)
    return sorted(set(names))


def test_header_symbols_exported():
    names = _declared()
    assert len(names) >= 20
    L = ctypes.CDLL(binding.LIB_PATH)
    for n in names:
        assert hasattr(L, n), n
    assert sorted(binding.exported_symbols()) == names


def test_strerror():
    L = binding.lib()
    for code in range(0, -8, -1):
        assert L.sa_heom_strerror(code)
    assert L.sa_heom_strerror(-1) == b"invalid argument"


@pytest.mark.parametrize("scheme,K,sigma", [("high_t", 0, 0.0), ("matsubara", 1, 0.0), ("matsubara", 4, 0.02),
                                            ("pade", 1, 0.0), ("pade", 3, 0.0), ("pade", 5, 0.01)])
def test_bath_matches_oracle(scheme, K, sigma):
    lam, gam, kT = 0.03, 0.02, 0.01
    code = {"high_t": S.BATH_HIGH_T, "matsubara": S.BATH_MATSUBARA, "pade": S.BATH_PADE}[scheme]
    got = S.bath_drude_lorentz(lam, gam, kT, code, K, sigma)
    if scheme == "high_t":
        ref = OB.high_t(lam, gam, kT, sigma)
    elif scheme == "matsubara":
        ref = OB.matsubara(lam, gam, kT, K, sigma)
    else:
        ref = OB.pade(lam, gam, kT, K, sigma)
    for key in ("c", "cc", "nu"):
        assert got[key].shape == ref[key].shape
        assert np.allclose(got[key], ref[key], rtol=1e-13, atol=1e-18), (key, got[key], ref[key])


def test_bath_rejects_bad_input():
    with pytest.raises(S.SaHeomError):
        S.bath_drude_lorentz(-1.0, 0.05, 0.025, S.BATH_MATSUBARA, 1)
    with pytest.raises(S.SaHeomError):
        S.bath_drude_lorentz(0.01, 0.05, 0.025, S.BATH_MATSUBARA, 8)


@pytest.mark.parametrize("N,m,L", [(2, 1, 3), (10, 2, 6), (100, 2, 8), (1000, 4, 12), (2 ** 61 - 1, 8, 1),
                                   (2 ** 61, 8, 1), (40, 3, 17), (10 ** 12, 1, 2)])
def test_exact_conventional_ado_count(N, m, L):
    """sa_counts.conventional_ados is C(Nm+L, L) (Eq. direct-ado-count) whenever
    that fits in 64 bits and 0 otherwise; its log10 agrees either way."""
    rng = np.random.default_rng(m)
    bath = {"c": rng.uniform(0.1, 0.5, m) + 0j, "cc": rng.uniform(0.1, 0.5, m) + 0j,
            "nu": rng.uniform(0.2, 1.2, m) + 0j}
    c = S.counts(S.make_params(N, m, L, bath))
    exact = math.comb(N * m + L, L)
    assert c["conventional_ados"] == (exact if exact < 2 ** 64 else 0)
    assert abs(c["log10_conventional_ados"] - math.log10(exact)) < 1e-9 * max(1.0, math.log10(exact))


@pytest.mark.parametrize("K", [0, 1, 3, 6])
def test_terminator_strength_matches_oracle(K):
    """sa_bath_terminator (closed form less the kept poles) against the oracle's
    term-by-term sum of the omitted Matsubara c_j / nu_j."""
    for lam, gam, kT in [(0.01, 0.05, 0.025), (0.03, 0.02, 0.01), (0.02, 0.05, 0.025)]:
        got = S.bath_terminator(lam, gam, kT, K)
        ref = OB.terminator(lam, gam, kT, K)
        assert abs(got - ref) <= 1e-15 + 1e-12 * abs(ref)
    with pytest.raises(S.SaHeomError):
        S.bath_terminator(-0.01, 0.05, 0.025, K)


@pytest.mark.parametrize("kind", ["cavity", "bright", "up", "lp", "random"])
@pytest.mark.parametrize("N", [1, 2, 7, 1000])
def test_initial_vars_match_oracle(kind, N):
    """sa_heom_initial_vars against the oracle's initial unique variables
    (Eqs. cavity-/bright-initial-uvar, upper-/lower-polariton-initial, the
    random invariant state of its draws)."""
    import workloads as W
    from tests._helpers import oracle_rho0

    if kind == "random" and N == 1:
        pytest.skip("the oracle's random state needs a dark block (N >= 2)")
    w = dict(W.WORKLOADS["w3"], N=N, init=kind)
    draws = W.random_rho_draws()
    got = S.rho0_vars(w, draws)
    ref = np.array(oracle_rho0(w, draws), complex)
    n = 5 if N >= 2 else 4
    assert np.max(np.abs(got[:n] - ref[:n])) <= 1e-15
