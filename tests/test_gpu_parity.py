"""GPU parity: the sm_103a kernels (through the C ABI) against the FP64 oracle.

Tolerances (FP64 path): max |x_gpu - x_oracle| / max |x_oracle| <= 1e-11 over
the whole unique-variable vector.  FP32-aux path: the right-hand side of a
float-rounded input within 2e-6 of max |dx| (single-precision arithmetic over
at most ~4m+G terms), populations within 1e-5 of the FP64 oracle.
"""
import math

import numpy as np
import pytest

import oracle
import paper_2608_20657_b300 as S
import workloads as W
from tests._helpers import oracle_rho0, oracle_sa, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def _generic_bath(m, seed):
    rng = np.random.default_rng(seed)
    return {"c": rng.uniform(0.1, 0.5, m) + 1j * rng.uniform(-0.4, 0.4, m),
            "cc": rng.uniform(0.1, 0.5, m) + 1j * rng.uniform(-0.4, 0.4, m),
            "nu": rng.uniform(0.2, 1.2, m) + 1j * rng.uniform(-0.3, 0.3, m)}


SMALL = [(1, 1, 3), (2, 1, 3), (3, 1, 0), (3, 2, 3), (4, 1, 5), (5, 2, 4), (10, 2, 6), (12, 3, 4), (7, 4, 3),
         (30, 1, 12), (6, 5, 3), (2, 2, 6), (40, 2, 7)]


def _rhs_gpu(h, x):
    xs = h.new_state()
    dx = h.new_state()
    h.upload(xs, x)
    h.rhs(xs, dx)
    torch.cuda.synchronize()
    return h.download(dx)


KERNELS = [S.SA_KERNEL_RECORDS, S.SA_KERNEL_LISTS, S.SA_KERNEL_ELL]


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("N,m,L", SMALL)
def test_rhs_fp64(N, m, L, kernel):
    """Eq. uvar-propagator: one right-hand side on a seeded random vector (the
    terminator on in every other case)."""
    bath = _generic_bath(m, N + 7 * m + L)
    kw = dict(detuning=0.1, g=0.2, kappa=0.05, term=0.013 * ((N + L) % 2))
    sa = oracle.SA(N, m, L, bath, **kw)
    h = S.Heom(S.make_params(N, m, L, bath, **kw))
    h.set_kernel(kernel)
    x = W.random_state(sa.nvar, seed=N * 100 + L)
    assert rel_err(_rhs_gpu(h, x), sa.rhs(x)) <= 1e-13


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("N,m,L", SMALL[::2])
def test_rhs_fp32(N, m, L, kernel):
    bath = _generic_bath(m, N + 7 * m + L)
    kw = dict(detuning=0.1, g=0.2, kappa=0.05, term=0.013 * ((N + L) % 2))
    sa = oracle.SA(N, m, L, bath, **kw)
    h = S.Heom(S.make_params(N, m, L, bath, **kw), precision=S.SA_FP32_AUX)
    h.set_kernel(kernel)
    x = W.random_state(sa.nvar, seed=N * 100 + L).astype(np.complex64).astype(np.complex128)
    assert rel_err(_rhs_gpu(h, x), sa.rhs(x)) <= 2e-6


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("N,m,L", [(3, 2, 3), (10, 2, 6), (12, 3, 4), (40, 2, 7)])
def test_rk4_steps_fp64(N, m, L, kernel):
    """Classical RK4 fused into the stage kernels: 40 steps vs the oracle."""
    bath = _generic_bath(m, N + 7 * m + L)
    kw = dict(detuning=0.1, g=0.2, kappa=0.05, term=0.009)
    sa = oracle.SA(N, m, L, bath, **kw)
    h = S.Heom(S.make_params(N, m, L, bath, **kw))
    h.set_kernel(kernel)
    x = W.random_state(sa.nvar, seed=3, scale=0.1)
    st = h.new_state()
    h.upload(st, x)
    for _ in range(40):
        h.step(st, 0.05)
    torch.cuda.synchronize()
    assert rel_err(h.download(st), sa.rk4(x, 0.05, 40)) <= 1e-11


@pytest.mark.parametrize("key,steps", [("w1", 2000), ("w2", 5000), ("w3", 20000)])
def test_workload_fp64_full(key, steps):
    """Workloads w1-w3 in full: whole state at t_final within 1e-11 relative,
    observables every 100 steps within 1e-11."""
    w = W.WORKLOADS[key]
    sa = oracle_sa(w)
    x0 = sa.initial_state(*oracle_rho0(w))
    y_or, obs_or = sa.propagate(x0, w["dt"], steps, 100)
    h = S.Heom(S.params_from(w))
    st = h.new_state()
    h.init_state(st, S.rho0_vars(w))
    obs = h.propagate(st, w["dt"], steps, 100)
    torch.cuda.synchronize()
    assert rel_err(h.download(st), y_or) <= 1e-11
    assert np.max(np.abs(obs[:, 0, :7] - obs_or[:, :7])) <= 1e-11
    assert oracle.errors() == 0


def test_w3_fp32_population_error():
    """FP32 auxiliary variables with FP64 rho_0: every population of w3 over
    20000 steps within 1e-5 of the FP64 oracle (reported per run)."""
    w = W.WORKLOADS["w3"]
    sa = oracle_sa(w)
    _, obs_or = sa.propagate(sa.initial_state(*oracle_rho0(w)), w["dt"], w["steps"], 100)
    h = S.Heom(S.params_from(w), precision=S.SA_FP32_AUX)
    st = h.new_state()
    h.init_state(st, S.rho0_vars(w))
    obs = h.propagate(st, w["dt"], w["steps"], 100)
    err = np.max(np.abs(obs[:, 0, 1:7] - obs_or[:, 1:7]))
    print(f"w3 FP32-aux max population error vs FP64 oracle: {err:.3e}")
    assert err <= 1e-5


@pytest.mark.parametrize("kernel", KERNELS)
def test_batch_matches_single_instances(kernel):
    """A batch of uneven instances (w4 recipe) equals the oracle run of each
    instance: 30 RK4 steps from the upper-polariton start, FP64."""
    ws = W.batch_w4(24, seed=11)
    h = S.Heom([S.params_from(w) for w in ws])
    h.set_kernel(kernel)
    st = h.new_state()
    h.init_state(st, np.stack([S.rho0_vars(w) for w in ws]))
    for _ in range(30):
        h.step(st, 0.02)
    torch.cuda.synchronize()
    y = h.download(st)
    for i, w in enumerate(ws):
        sa = oracle_sa(w)
        ref = sa.rk4(sa.initial_state(*oracle_rho0(w)), 0.02, 30)
        a = h.var_offset(i)
        assert rel_err(y[a:a + sa.nvar], ref) <= 1e-11, i


@pytest.mark.parametrize("kernel", KERNELS)
def test_batch_fp32_population_error(kernel):
    """Batched FP32-aux vs the FP64 oracle for a few w4 instances over 2000
    steps: populations within 1e-5."""
    ws = W.batch_w4(8, seed=5)
    h = S.Heom([S.params_from(w) for w in ws], precision=S.SA_FP32_AUX)
    h.set_kernel(kernel)
    st = h.new_state()
    h.init_state(st, np.stack([S.rho0_vars(w) for w in ws]))
    obs = h.propagate(st, 0.02, 2000, 500)
    for i, w in enumerate(ws):
        sa = oracle_sa(w)
        _, ob = sa.propagate(sa.initial_state(*oracle_rho0(w)), 0.02, 2000, 500)
        assert np.max(np.abs(obs[:, i, 1:7] - ob[:, 1:7])) <= 1e-5, i


def test_prepare_builds_the_graphs_propagate_uses():
    """sa_heom_prepare runs nothing; a propagation after it equals one
    without it, bit for bit, with and without observables."""
    w = W.WORKLOADS["w2"]
    h = S.Heom(S.params_from(w))
    a, b = h.new_state(), h.new_state()
    h.init_state(a, S.rho0_vars(w))
    h.init_state(b, S.rho0_vars(w))
    h.prepare(a, 0.02, 150)
    h.prepare(a, 0.02, 150, 7)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    h.propagate(a, 0.02, 150, observe=False)
    oa = h.propagate(a, 0.02, 150, 7)
    h.propagate(b, 0.02, 150, observe=False)
    ob = h.propagate(b, 0.02, 150, 7)
    torch.cuda.synchronize()
    assert torch.equal(a, b) and np.array_equal(oa, ob)


@pytest.mark.parametrize("kernel", KERNELS)
def test_graph_equals_steps_and_tuning_invariance(kernel):
    """propagate (CUDA graph) is bit-identical to single steps, and every
    launch tuning gives bit-identical results (each variable's arithmetic
    does not depend on the chunking)."""
    w = W.WORKLOADS["w3"]
    h = S.Heom(S.params_from(w))
    h.set_kernel(kernel)
    a, b = h.new_state(), h.new_state()
    h.init_state(a, S.rho0_vars(w))
    h.init_state(b, S.rho0_vars(w))
    for _ in range(70):
        h.step(a, 0.02)
    h.propagate(b, 0.02, 70, observe=False)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    ref = h.download(a)
    for blk, chk, q in [(128, 128, 0), (256, 256, 1), (64, 160, 1), (128, 192, 0), (64, 1024, 1)]:
        try:
            h.set_tuning(blk, chk, q)
        except S.SaHeomError as e:  # a tuning whose shared-memory image does not fit
            assert e.code == -2
            continue
        c = h.new_state()
        h.init_state(c, S.rho0_vars(w))
        h.propagate(c, 0.02, 70, observe=False)
        torch.cuda.synchronize()
        assert np.array_equal(h.download(c), ref), (blk, chk, q)


def test_invariants_on_gpu():
    """kappa = 0: Tr rho_S conserved; Hermiticity defect of rho_S at rounding
    level (real nu, c-check = conj(c)); P_B + P_D = P_exc."""
    w = dict(W.WORKLOADS["w2"])
    h = S.Heom(S.params_from(w))
    st = h.new_state()
    h.init_state(st, S.rho0_vars(w))
    obs = h.propagate(st, w["dt"], 3000, 300)[:, 0]
    assert np.max(np.abs(obs[:, 0] - 1)) < 1e-12
    assert np.max(obs[:, 7]) < 1e-13
    assert np.max(np.abs(obs[:, 3] + obs[:, 4] - obs[:, 2])) < 1e-13


def test_edge_cases():
    """N = 1 (4 physical variables), L = 0 (the empty pattern only: Rabi
    closed form), and many more patterns than one work item's 16-pattern
    limit."""
    bath = {"c": np.array([0.1 + 0.05j]), "cc": np.array([0.1 - 0.05j]), "nu": np.array([0.3 + 0j])}
    for N, L in [(1, 4), (1, 0)]:
        sa = oracle.SA(N, 1, L, bath, 0.05, 0.1, 0.02)
        h = S.Heom(S.make_params(N, 1, L, bath, detuning=0.05, g=0.1, kappa=0.02))
        x = W.random_state(sa.nvar, 9)
        assert rel_err(_rhs_gpu(h, x), sa.rhs(x)) <= 1e-13
    N, gsn, det = 50, 0.1, 0.03
    h = S.Heom(S.make_params(N, 1, 0, bath, detuning=det, g=gsn / math.sqrt(N)))
    st = h.new_state()
    h.init_state(st, [1, 0, 0, 0, 0])
    obs = h.propagate(st, 0.05, 800, 100)[:, 0]
    t = np.arange(obs.shape[0]) * 5.0
    Om = math.hypot(2 * gsn, det)
    assert np.max(np.abs(obs[:, 1] - (1 - (2 * gsn / Om) ** 2 * np.sin(Om * t / 2) ** 2))) < 1e-9
    # many tiny patterns: N = 1, m = 6, L = 5 gives 462 four-variable patterns,
    # so work items hit the 16-pattern limit before the variable limit
    bath6 = _generic_bath(6, 2)
    sa = oracle.SA(1, 6, 5, bath6, 0.1, 0.2, 0.0)
    h = S.Heom(S.make_params(1, 6, 5, bath6, detuning=0.1, g=0.2))
    assert sa.npat > 256
    x = W.random_state(sa.nvar, 4)
    assert rel_err(_rhs_gpu(h, x), sa.rhs(x)) <= 1e-13


def test_fp32_rho0_is_fp64():
    """In SA_FP32_AUX mode the physical representative is stored and
    integrated in FP64: a pure Rabi run (L = 0) matches the FP64 closed form
    far below single precision."""
    bath = {"c": np.array([0.1 + 0j]), "cc": np.array([0.1 + 0j]), "nu": np.array([1.0 + 0j])}
    N, gsn = 10, 0.05
    h = S.Heom(S.make_params(N, 1, 0, bath, g=gsn / math.sqrt(N)), precision=S.SA_FP32_AUX)
    st = h.new_state()
    h.init_state(st, [0, 0, 0, 1 / N, 1 / N])
    obs = h.propagate(st, 0.05, 2000, 200)[:, 0]
    t = np.arange(obs.shape[0]) * 10.0
    assert np.max(np.abs(obs[:, 3] - np.cos(gsn * t) ** 2)) < 1e-10


@pytest.mark.slow
@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("precision,tol", [(S.SA_FP64, 1e-13), (S.SA_FP32_AUX, 2e-6)])
def test_w5_full_size_sampled(precision, tol, kernel):
    """Full-size w5 (4,058,820 patterns, 170,187,185 variables) in the launch
    configuration the benchmark uses: the right-hand side of a seeded random
    state at 20,000 sampled variables against the oracle evaluated one by one."""
    w = W.WORKLOADS["w5"]
    sa = oracle_sa(w, cache=False)
    h = S.Heom(S.params_from(w), precision=precision)
    h.set_kernel(kernel)
    assert h.n_vars == sa.nvar == 170187185
    x = W.random_state(sa.nvar, seed=2608)
    if precision == S.SA_FP32_AUX:
        x = x.astype(np.complex64).astype(np.complex128)
    xs, dx = h.new_state(), h.new_state()
    h.upload(xs, x)
    h.rhs(xs, dx)
    torch.cuda.synchronize()
    d = h.download(dx)
    idx = W.sample_indices(sa.nvar, 20000, seed=1)
    ref = sa.rhs_at(x, idx)
    assert rel_err(d[idx], ref) <= tol
    del xs, dx
    torch.cuda.empty_cache()


@pytest.mark.slow
@pytest.mark.parametrize("kernel", KERNELS)
def test_w4_full_batch_sampled(kernel):
    """Full w4 batch (512 instances, FP32-aux) in the benchmark's launch
    configuration: RHS of a seeded random float state at sampled variables."""
    ws = W.batch_w4()
    h = S.Heom([S.params_from(w) for w in ws], precision=S.SA_FP32_AUX)
    h.set_kernel(kernel)
    x = W.random_state(h.n_vars, seed=7).astype(np.complex64).astype(np.complex128)
    xs, dx = h.new_state(), h.new_state()
    h.upload(xs, x)
    h.rhs(xs, dx)
    torch.cuda.synchronize()
    d = h.download(dx)
    for i in [0, 100, 255, 511]:
        sa = oracle_sa(ws[i])
        a = h.var_offset(i)
        xi = x[a:a + sa.nvar]
        assert rel_err(d[a:a + sa.nvar], sa.rhs(xi)) <= 2e-6, i
