"""GPU parity on the deep hierarchy w5 (N = 1000, Drude-Lorentz + 3 Pade poles
so m = 4, L = 12, kappa = 0.005; 4,058,820 patterns, 170,187,185 unique
variables), propagated rather than a single right-hand side.

* FP64 on the GPU against the FP64 oracle's RK4 (Eq. scaled-HEOM in unique
  variables, Secs. III-IV) over a short prefix from the workload's random
  permutation-invariant density matrix: three steps at dt = 0.01 reach every
  tier (each RK4 step couples four tiers further), compared over the whole
  state at <= 1e-11 relative.
* One FP64 step from a seeded random state of the whole hierarchy, so that
  the deepest tiers carry O(1) values, at the same tolerance.
* FP32 auxiliary variables (FP64 rho_0) against the FP64 GPU path over 2000
  steps (t = 20): every population within 1e-5 at every 100th step.  The FP64
  run also keeps rho_S Hermitian (real nu_k with c-check_k = conj(c_k)) and
  its trace within [Tr(0) e^(-kappa t), Tr(0)] (the loss only removes
  population: d Tr / dt = -kappa Z with 0 <= Z <= Tr).
"""
import math

import numpy as np
import pytest

import paper_2608_20657_b300 as S
import workloads as W
from tests._helpers import oracle_initial, oracle_sa, rel_err

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

W5 = W.WORKLOADS["w5"]
NVAR = 170187185


@pytest.fixture(scope="module")
def w5_fp64():
    h = S.Heom(S.params_from(W5), precision=S.SA_FP64)
    assert h.n_vars == NVAR
    yield h
    h.close()
    torch.cuda.empty_cache()


@pytest.fixture(scope="module")
def w5_oracle():
    return oracle_sa(W5, cache=False)


def _rho0():
    return S.rho0_vars(W5, W.random_rho_draws())


def test_w5_fp64_prefix_against_oracle(w5_fp64, w5_oracle):
    """Three RK4 steps from the random invariant rho_S: the whole GPU state
    against the oracle's."""
    h, sa = w5_fp64, w5_oracle
    st = h.new_state()
    h.init_state(st, _rho0())
    x0 = oracle_initial(sa, W5, W.random_rho_draws())
    assert rel_err(h.download(st), x0) <= 1e-15
    h.propagate(st, W5["dt"], 3, observe=False)
    torch.cuda.synchronize()
    got = h.download(st)
    del st
    ref = sa.rk4(x0, W5["dt"], 3)
    pt = h.dump_patterns(0)
    deep = pt["var_off"][np.searchsorted(pt["tier"], W5["L"])]
    assert np.count_nonzero(ref[deep:]) > 0  # the deepest tier is reached
    assert rel_err(got, ref) <= 1e-11


def test_w5_fp64_random_state_step(w5_fp64, w5_oracle):
    """One RK4 step from a seeded random state of the whole hierarchy."""
    h, sa = w5_fp64, w5_oracle
    x = W.random_state(NVAR, seed=2609)
    st = h.new_state()
    h.upload(st, x)
    h.step(st, W5["dt"])
    torch.cuda.synchronize()
    got = h.download(st)
    del st
    assert rel_err(got, sa.rk4(x, W5["dt"], 1)) <= 1e-11


def test_w5_fp32_populations_against_fp64(w5_fp64):
    """FP32-aux against FP64, 2000 steps at dt = 0.01, observed every 100."""
    nsteps, every, dt = 2000, 100, W5["dt"]
    st = w5_fp64.new_state()
    w5_fp64.init_state(st, _rho0())
    o64 = w5_fp64.propagate(st, dt, nsteps, every)[:, 0]
    del st
    h32 = S.Heom(S.params_from(W5), precision=S.SA_FP32_AUX)
    s32 = h32.new_state()
    h32.init_state(s32, _rho0())
    o32 = h32.propagate(s32, dt, nsteps, every)[:, 0]
    del s32
    h32.close()
    torch.cuda.empty_cache()
    err = float(np.max(np.abs(o64[:, 1:7] - o32[:, 1:7])))
    print(f"w5 FP32-aux max population error against FP64 over {nsteps} steps: {err:.3e}")
    assert err <= 1e-5
    # FP64 invariants of the lossy dynamics
    t = np.arange(o64.shape[0]) * every * dt
    tr0 = o64[0, 0]
    assert np.all(o64[:, 0] <= tr0 + 1e-12)
    assert np.all(o64[:, 0] >= tr0 * np.exp(-W5["kappa"] * t) - 1e-12)
    assert np.all(np.diff(o64[:, 0]) <= 1e-12)
    assert np.max(o64[:, 7]) <= 1e-12
    assert np.all(np.isfinite(o32))
    assert math.isclose(o32[0, 0], tr0, rel_tol=0, abs_tol=1e-12)
