"""Pins of the oracle's bath decompositions (Eq. BCF-exp for the Drude-Lorentz
spectral density of Eq. Drude_Lorentz, Eq. BCF-spectral, Eq. C_static)."""
import os
from fractions import Fraction

import mpmath as mp
import numpy as np
import pytest

import oracle.bath as B

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_pade_hand_worked():
    """[0/1] approximant worked by hand (golden file): eta = 5/2, xi^2 = 15."""
    line = [l for l in open(os.path.join(GOLD, "pade_hand.txt")) if l[0] != "#"][0].split()
    eta, xi2 = Fraction(line[3]), Fraction(line[5])
    (e, x), = B.pade_poles(1)
    assert abs(e - mp.mpf(eta.numerator) / eta.denominator) < mp.mpf(10) ** -40
    assert abs(x ** 2 - mp.mpf(xi2.numerator) / xi2.denominator) < mp.mpf(10) ** -40


def test_taylor_coefficients():
    """(coth x - 1/x)/x = 1/3 - x^2/45 + 2x^4/945 - x^6/4725 + ..."""
    a = B.coth_series_coeffs(4)
    assert a == [Fraction(1, 3), Fraction(-1, 45), Fraction(2, 945), Fraction(-1, 4725)]


@pytest.mark.parametrize("K", [1, 2, 3, 4, 5])
def test_pade_poles_real_positive(K):
    poles = B.pade_poles(K)
    xs = [x for _, x in poles]
    for e, x in poles:
        assert abs(mp.im(x)) < 1e-30 and mp.re(x) > 0
        assert abs(mp.im(e)) < 1e-30 and mp.re(e) > 0
    assert all(xs[i] < xs[i + 1] for i in range(K - 1))
    if K >= 3:
        assert abs(xs[0] - mp.pi) < 1e-3        # lowest pole ~ first Matsubara


@pytest.mark.parametrize("K", [1, 2, 3, 4])
def test_pade_beats_matsubara_on_coth(K):
    """Same number of poles: the Pade coth is closer to coth on the real
    axis than the truncated Matsubara (Mittag-Leffler) series."""
    xs = [0.2, 0.5, 1.0, 2.0, 3.0]
    ep = max(abs(B.coth_approx(x, "pade", K) - mp.coth(x)) for x in xs)
    em = max(abs(B.coth_approx(x, "matsubara", K) - mp.coth(x)) for x in xs)
    assert ep < em


def test_matsubara_series_converges():
    """Matsubara is the eta = 1, xi = j pi special case: the Mittag-Leffler
    expansion of coth converges as the pole count grows."""
    errs = [abs(B.coth_approx(1.3, "matsubara", K) - mp.coth(1.3)) for K in (5, 50, 500)]
    assert errs[0] > errs[1] > errs[2] and errs[2] < 1e-3


@pytest.mark.parametrize("t", [5.0, 20.0, 60.0])
def test_bcf_converges_to_quadrature(t):
    """C_m(t) of both schemes approaches the quadrature of Eq. BCF-spectral as
    the term count grows (t > 0; the Drude-Lorentz C(0) is divergent)."""
    lam, gam, kT = 0.03, 0.02, 0.01
    ref = B.bcf_exact(t, lam, gam, kT)
    em = [abs(B.bcf_from(B.matsubara(lam, gam, kT, K), t) - ref) for K in (1, 4, 40)]
    ep = [abs(B.bcf_from(B.pade(lam, gam, kT, K), t) - ref) for K in (1, 6, 12)]
    assert em[2] < em[0] and em[2] < 1e-3 * abs(ref)
    assert ep[0] > ep[1] > ep[2] and ep[2] < 1e-5 * abs(ref)
    assert abs(B.bcf_from(B.matsubara(lam, gam, kT, 1), t).imag - ref.imag) < 1e-12


def test_high_t_limit():
    """cot(beta gamma/2) -> 2/(beta gamma) at high temperature: the Matsubara
    gamma-pole weight tends to the high-T c_0 = 2 lambda kT - i lambda gamma."""
    lam, gam = 0.01, 0.05
    for kT in (1.0, 10.0):
        cm = B.matsubara(lam, gam, kT, 0)["c"][0]
        ch = B.high_t(lam, gam, kT)["c"][0]
        assert abs(cm - ch) < 0.01 * abs(ch) / kT


def test_static_channel_and_conjugates():
    """Eq. C_static adds c = sigma^2, nu = 0; real rates give cc = conj(c)."""
    b = B.matsubara(0.02, 0.05, 0.025, 1, sigma=0.02)
    assert len(b["c"]) == 3 and b["nu"][2] == 0 and b["c"][2] == pytest.approx(4e-4)
    assert np.all(b["cc"] == np.conj(b["c"]))
