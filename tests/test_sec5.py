"""The paper's production set (Sec. V) on the host: unit conversion, the
product's parameters against the oracle's (converted independently), the
hierarchy sizes the paper prints for L = 25, and the initial populations it
states for each initial state.  No GPU is used."""
import math

import numpy as np
import pytest

import paper_2608_20657_b300 as S
import workloads as W
from tests._helpers import oracle_initial, oracle_sa, physical


def test_unit_constants():
    """With hbar = 1, 1 cm^-1 is 2 pi c rad/fs: hbar = 5308.8 cm^-1 fs
    (textbook value); k_B T at 300 K is about 208 cm^-1 (Sec. V)."""
    f = S.binding.unit_cm_to_rad_fs(1.0)
    assert abs(1.0 / f - 5308.837) < 1e-3
    kT_cm = S.binding.unit_kT_rad_fs(300.0) / f
    assert abs(kT_cm - 208.0) < 1.0
    u = physical(W.sec5(10))
    assert abs(u["kT"] / f - kT_cm) < 1e-9
    assert abs(S.in_library_units(W.sec5(10))["kT"] - u["kT"]) <= 1e-15 * u["kT"]


@pytest.mark.parametrize("N", (1, 2, 3) + W.SEC5_N)
@pytest.mark.parametrize("init", ["up", "localised", "superposed"])
def test_params_agree_with_oracle(N, init):
    """The product's sa_params (bath through sa_bath_drude_lorentz, Delta
    through sa_bath_terminator, g = Omega_R / (2 sqrt N), Eq. g-fixed-Rabi)
    equal the oracle's to rounding, and so does the physical representative
    handed to sa_heom_init_physical."""
    w = W.sec5(N, init)
    p = S.params_from(w)
    sa = oracle_sa(w, cache=False)
    q = sa.params
    assert (p.N, p.m, p.L, p.d) == (q.N, q.m, q.L, q.d) == (N, 1, 25, 1 if init != "up" else 0)
    for f in ("detuning", "g", "kappa", "term"):
        a, b = getattr(p, f), getattr(q, f)
        assert abs(a - b) <= 1e-14 * max(abs(b), 1e-300), f
    for f in ("c_re", "c_im", "cc_re", "cc_im", "nu_re", "nu_im"):
        a, b = getattr(p, f)[0], getattr(q, f)[0]
        assert abs(a - b) <= 1e-14 * abs(b), f
    # Omega_R = 2 g sqrt(N) = 500 cm^-1 at every N
    assert abs(2 * p.g * math.sqrt(N) / S.binding.unit_cm_to_rad_fs(1.0) - 500.0) < 1e-9
    assert p.term > 0
    ph = S.phys_vars(w)
    x = oracle_initial(sa, w)
    np.testing.assert_allclose(ph, x[:ph.size], rtol=0, atol=1e-15)
    assert np.all(x[ph.size:] == 0)


def test_hierarchy_sizes_at_L25():
    """Sec. V.F text: at L = 25 with one exponential the symmetric hierarchy
    has 9296 patterns and 306751 variables (N >= 27), the d = 1 hierarchy
    41391 patterns and 1715600 variables (N >= 28)."""
    for N, init, npat, nvar in [(10 ** 12, "up", 9296, 306751), (1000, "up", 9296, 306751),
                                (100, "localised", 41391, 1715600), (10 ** 12, "localised", 41391, 1715600)]:
        c = S.counts(S.params_from(W.sec5(N, init)))
        assert (c["n_patterns"], c["n_vars"]) == (npat, nvar)


@pytest.mark.parametrize("N", W.SEC5_N)
def test_initial_populations(N):
    """Initial TC-basis populations the paper states: upper polariton
    P_+ = 1 with cavity and bright weights 1/2 (Sec. V.A); localised
    P_+ = P_- = 1/(2N), P_D = 1 - 1/N; cavity-site superposition
    P_D = 0.3 (1 - 1/N), P_+- = (sqrt 0.7 +- sqrt(0.3/N))^2 / 2 (Sec. V.F)."""
    for init in ("up", "localised", "superposed"):
        w = W.sec5(N, init)
        sa = oracle_sa(w, cache=False)
        o = sa.observables(oracle_initial(sa, w))
        assert abs(o[0] - 1) < 1e-14
        if init == "up":
            exp = {1: 0.5, 3: 0.5, 4: 0.0, 5: 1.0, 6: 0.0}
        elif init == "localised":
            exp = {1: 0.0, 4: 1 - 1 / N, 5: 1 / (2 * N), 6: 1 / (2 * N)}
        else:
            exp = {1: 0.7, 4: 0.3 * (1 - 1 / N), 5: 0.5 * (math.sqrt(0.7) + math.sqrt(0.3 / N)) ** 2,
                   6: 0.5 * (math.sqrt(0.7) - math.sqrt(0.3 / N)) ** 2}
        for k, v in exp.items():
            assert abs(o[k] - v) < 1e-12, (init, k)
