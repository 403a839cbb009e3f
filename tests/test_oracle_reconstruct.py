"""Pins of the oracle's reconstruction of arbitrary initial operators from the
five representative propagations (Sec. IV, Table tab:representative-initial-
operators): against the conventional hierarchy propagated from the same
dense initial operator, which knows nothing of symmetry or relabelling."""
import numpy as np
import pytest


def _bath(m, seed, conjugate=False):
    rng = np.random.default_rng(seed)
    c = rng.uniform(0.1, 0.5, m) + 1j * rng.uniform(-0.4, 0.4, m)
    if conjugate:
        # real decay rates and c-check = conj(c): the map preserves adjoints
        return {"c": c, "cc": np.conj(c), "nu": rng.uniform(0.2, 1.2, m) + 0j}
    return {"c": c, "cc": rng.uniform(0.1, 0.5, m) + 1j * rng.uniform(-0.4, 0.4, m),
            "nu": rng.uniform(0.2, 1.2, m) + 1j * rng.uniform(-0.3, 0.3, m)}


@pytest.mark.parametrize("N,m,L", [(1, 1, 3), (2, 1, 3), (3, 1, 3), (4, 2, 2), (5, 1, 2)])
def test_reconstruction_equals_conventional(orc, N, m, L):
    """Eqs. Gt-linearity, Gt-covariance, reconstruct-ec, reconstruct-ee: the
    weighted, relabelled representative responses equal rho_S(t) of the
    conventional hierarchy started from a random (non-Hermitian) operator."""
    from oracle import reconstruct as R

    bath = _bath(m, 10 * N + m + L)
    kw = dict(detuning=0.07, g=0.15, kappa=0.03, term=0.004)
    resp = R.responses(R.representative_hierarchies(N, m, L, bath, **kw), 0.05, 30)
    rng = np.random.default_rng(N)
    rho0 = rng.standard_normal((N + 1, N + 1)) + 1j * rng.standard_normal((N + 1, N + 1))
    cv = orc.Conventional(N, m, L, bath, **kw)
    x = cv.zeros()
    x[0] = rho0
    ref = cv.rk4(x, 0.05, 30)[0]
    got = R.reconstruct(resp, rho0)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
    assert orc.errors() == 0


def test_physical_dense_round_trip(orc):
    """physical_dense inverts initial_state_dense for operators invariant
    under the residual group (here d = 2, molecules 3..N interchangeable)."""
    from oracle import reconstruct as R

    N = 5
    sa = orc.SA(N, 1, 2, _bath(1, 1), d=2)
    rng = np.random.default_rng(3)
    rho = rng.standard_normal((N + 1, N + 1)) + 1j * rng.standard_normal((N + 1, N + 1))
    # make it invariant under permutations of molecules 3..5: average
    import itertools

    acc = np.zeros_like(rho)
    ps = list(itertools.permutations(range(3, N + 1)))
    for p in ps:
        idx = [0, 1, 2] + list(p)
        acc += rho[np.ix_(idx, idx)]
    acc /= len(ps)
    np.testing.assert_allclose(R.physical_dense(sa, sa.initial_state_dense(acc)), acc, rtol=0, atol=1e-15)


@pytest.mark.parametrize("conjugate", [True, False])
def test_adjoint_reduction(orc, conjugate):
    """Eq. adjoint-preservation: with real decay rates and c-check = conj(c)
    the response to |c><e_1| is the adjoint of the response to |e_1><c|, so
    four propagations suffice; with complex decay rates that are not paired
    it is not."""
    from oracle import reconstruct as R

    bath = _bath(2, 5, conjugate)
    resp = R.responses(R.representative_hierarchies(3, 2, 3, bath, detuning=0.05, g=0.2), 0.05, 40)
    diff = np.abs(resp["ce"] - resp["ec"].conj().T).max()
    if conjugate:
        assert diff <= 1e-14
    else:
        assert diff > 1e-6
