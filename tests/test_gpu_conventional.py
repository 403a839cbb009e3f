"""Conventional scaled HEOM on the GPU (Eq. scaled-HEOM, dense ADOs) against
the conventional oracle, and as a cross-check of the symmetry-adapted GPU
path on workload w2 (230,230 ADOs x 121 entries)."""
import math

import numpy as np
import pytest

import oracle
import paper_2608_20657_b300 as S
import workloads as W
from tests._helpers import oracle_bath, oracle_rho0, oracle_sa, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def _generic_bath(m, seed):
    rng = np.random.default_rng(seed)
    return {"c": rng.uniform(0.1, 0.5, m) + 1j * rng.uniform(-0.4, 0.4, m),
            "cc": rng.uniform(0.1, 0.5, m) + 1j * rng.uniform(-0.4, 0.4, m),
            "nu": rng.uniform(0.2, 1.2, m) + 1j * rng.uniform(-0.3, 0.3, m)}


def _to_dev(x):
    return torch.from_numpy(np.ascontiguousarray(x).view(np.float64).ravel()).cuda().view(torch.uint8)


@pytest.mark.parametrize("N,m,L", [(1, 2, 3), (2, 1, 4), (3, 2, 3), (4, 1, 4), (3, 3, 2)])
def test_conventional_rhs_and_steps(N, m, L):
    bath = _generic_bath(m, 3 * N + m)
    kw = dict(detuning=0.1, g=0.2, kappa=0.05, term=0.011 * (N % 2))  # terminator in the odd-N cases
    cv = oracle.Conventional(N, m, L, bath, **kw)
    gc = S.Conventional(S.make_params(N, m, L, bath, **kw))
    assert gc.nado == cv.nado
    assert np.array_equal(gc.labels(), cv.labels())
    rng = np.random.default_rng(1)
    x = rng.standard_normal(cv.zeros().shape) + 1j * rng.standard_normal(cv.zeros().shape)
    xd = _to_dev(x)
    dx = gc.new_state()
    gc.rhs(xd, dx)
    torch.cuda.synchronize()
    assert rel_err(gc.to_numpy(dx), cv.rhs(x)) <= 1e-13
    x0 = 0.1 * x
    st = _to_dev(x0)
    gc.step(st, 0.05, 30)
    torch.cuda.synchronize()
    assert rel_err(gc.to_numpy(st), cv.rk4(x0, 0.05, 30)) <= 1e-11


def test_w2_conventional_equals_symmetry_adapted():
    """Workload w2 (N = 10, m = 2, L = 6): the dense conventional hierarchy and
    the symmetry-adapted unique variables, both on the GPU, from the bright
    state for 500 RK4 steps; every conventional entry equals its unique
    variable (Eq. central-covariance)."""
    w = W.WORKLOADS["w2"]
    N = w["N"]
    p = S.params_from(w)
    gc = S.Conventional(p)
    assert gc.nado == math.comb(N * p.m + w["L"], w["L"]) == 230230
    h = S.Heom(p)
    sa_state = h.new_state()
    h.init_state(sa_state, S.rho0_vars(w))
    Z, X0, Y0, P0, T0 = S.rho0_vars(w)
    rho = np.zeros((N + 1, N + 1), complex)
    rho[0, 0], rho[1:, 0], rho[0, 1:] = Z, X0, Y0
    rho[1:, 1:] = T0
    np.fill_diagonal(rho[1:, 1:], P0)
    cst = gc.new_state()
    gc.set_rho0(cst, rho)
    gc.step(cst, w["dt"], 500)
    h.propagate(sa_state, w["dt"], 500, observe=False)
    torch.cuda.synchronize()
    xs = h.download(sa_state)
    xc = gc.to_numpy(cst)
    b = oracle_bath(w)
    mp = oracle.Conventional(N, len(b["c"]), w["L"], b).map_to(oracle_sa(w))
    assert rel_err(xc, xs[mp]) <= 1e-11
