"""GPU parity with distinguished molecules (Sec. V.F, Eq. N-symmetric-pool):
molecules 1..d keep categories of their own in every pattern, so states that
are not permutation-invariant -- the localised |e_1><e_1| (Eq. localized_
initial_condition), the cavity-site superposition, (|e_1> + |e_2>)/sqrt 2 --
propagate in the reduced hierarchy.  The kernels are the d = 0 kernels on the
larger tables; the FP64 physical-representative kernel, the observables and
the initial state run over the physical pattern's d + 1 categories.

Tolerances as for d = 0: FP64 within 1e-11 relative of the FP64 oracle (1e-13
for one right-hand side), FP32-aux right-hand side within 2e-6, FP32-aux
populations within 1e-5.
"""
import numpy as np
import pytest

import oracle
import oracle.bath as OB
import paper_2608_20657_b300 as S
import workloads as W
from tests._helpers import rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

KERNELS = [S.SA_KERNEL_RECORDS, S.SA_KERNEL_LISTS, S.SA_KERNEL_ELL]
D_SMALL = [(1, 1, 3), (2, 1, 3), (3, 2, 3), (5, 2, 4), (10, 2, 6), (12, 3, 4), (7, 4, 3), (30, 1, 12), (2, 2, 6)]


def _generic_bath(m, seed):
    rng = np.random.default_rng(seed)
    return {"c": rng.uniform(0.1, 0.5, m) + 1j * rng.uniform(-0.4, 0.4, m),
            "cc": rng.uniform(0.1, 0.5, m) + 1j * rng.uniform(-0.4, 0.4, m),
            "nu": rng.uniform(0.2, 1.2, m) + 1j * rng.uniform(-0.3, 0.3, m)}


def _rhs_gpu(h, x):
    xs, dx = h.new_state(), h.new_state()
    h.upload(xs, x)
    h.rhs(xs, dx)
    torch.cuda.synchronize()
    return h.download(dx)


def _initial(sa, kind):
    """Physical representative of the localised state or of
    sqrt(0.3)|e_1> + sqrt(0.7)|c> (all hierarchy ADOs zero)."""
    ix = sa.rho0_index()
    e1 = "d" if sa.d == 1 else "1"  # molecule 1's category
    x = sa.zeros()
    if kind == "localised":
        x[ix["P" + e1]] = 1.0
    else:
        x[ix["P" + e1]], x[ix["Z"]] = 0.3, 0.7
        x[ix["X" + e1]] = x[ix["Y" + e1]] = np.sqrt(0.21)
    return x


D_MULTI = [(2, 1, 3, 2), (4, 2, 3, 2), (9, 1, 6, 2), (3, 1, 3, 3), (6, 2, 3, 3), (12, 1, 5, 3)]


def _nphys(sa):
    return int(sa.patterns()["var_off"][1])


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("N,m,L", D_SMALL)
def test_rhs_fp64_distinguished(N, m, L, kernel):
    bath = _generic_bath(m, N + 7 * m + L)
    kw = dict(detuning=0.1, g=0.2, kappa=0.05, term=0.013 * ((N + L) % 2), d=1)
    sa = oracle.SA(N, m, L, bath, **kw)
    h = S.Heom(S.make_params(N, m, L, bath, **kw))
    h.set_kernel(kernel)
    x = W.random_state(sa.nvar, seed=N * 100 + L)
    assert rel_err(_rhs_gpu(h, x), sa.rhs(x)) <= 1e-13


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("N,m,L", D_SMALL[::2])
def test_rhs_fp32_distinguished(N, m, L, kernel):
    bath = _generic_bath(m, N + 7 * m + L)
    kw = dict(detuning=0.1, g=0.2, kappa=0.05, term=0.013 * ((N + L) % 2), d=1)
    sa = oracle.SA(N, m, L, bath, **kw)
    h = S.Heom(S.make_params(N, m, L, bath, **kw), precision=S.SA_FP32_AUX)
    h.set_kernel(kernel)
    x = W.random_state(sa.nvar, seed=N * 100 + L).astype(np.complex64).astype(np.complex128)
    assert rel_err(_rhs_gpu(h, x), sa.rhs(x)) <= 2e-6


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("N,m,L,d", D_MULTI)
def test_rhs_several_distinguished(N, m, L, d, kernel):
    """d = 2, 3: one right-hand side, FP64 (1e-13) and FP32-aux (2e-6)."""
    bath = _generic_bath(m, N + 7 * m + L + d)
    kw = dict(detuning=0.1, g=0.2, kappa=0.05, term=0.011, d=d)
    sa = oracle.SA(N, m, L, bath, **kw)
    x = W.random_state(sa.nvar, seed=N * 100 + L + d)
    h = S.Heom(S.make_params(N, m, L, bath, **kw))
    h.set_kernel(kernel)
    assert rel_err(_rhs_gpu(h, x), sa.rhs(x)) <= 1e-13
    h = S.Heom(S.make_params(N, m, L, bath, **kw), precision=S.SA_FP32_AUX)
    h.set_kernel(kernel)
    xf = x.astype(np.complex64).astype(np.complex128)
    assert rel_err(_rhs_gpu(h, xf), sa.rhs(xf)) <= 2e-6


@pytest.mark.parametrize("precision", [S.SA_FP64, S.SA_FP32_AUX])
def test_two_distinguished_propagation(precision):
    """(|e_1> + |e_2>)/sqrt 2 with d = 2 (N = 8, two exponentials, L = 5):
    at t = 0 on resonance P_+ = P_- = 1/N, P_D = 1 - 2/N; 1000 RK4 steps
    against the oracle."""
    N, L = 8, 5
    bath = OB.matsubara(0.01, 0.05, 0.025, 1, 0.0)
    kw = dict(detuning=0.0, g=0.05 / np.sqrt(N), kappa=0.004, term=0.001, d=2)
    sa = oracle.SA(N, len(bath["c"]), L, bath, **kw)
    ix = sa.rho0_index()
    x0 = sa.zeros()
    x0[ix["P1"]] = x0[ix["P2"]] = x0[ix["S12"]] = x0[ix["S21"]] = 0.5
    y_or, obs_or = sa.propagate(x0, 0.02, 1000, 100)
    h = S.Heom(S.make_params(N, len(bath["c"]), L, bath, **kw), precision=precision)
    st = h.new_state()
    h.init_physical(st, x0[:_nphys(sa)])
    obs = h.propagate(st, 0.02, 1000, 100)
    torch.cuda.synchronize()
    assert abs(obs[0, 0, 5] - 1 / N) < 1e-14 and abs(obs[0, 0, 6] - 1 / N) < 1e-14
    assert abs(obs[0, 0, 4] - (1 - 2 / N)) < 1e-14
    if precision == S.SA_FP64:
        assert rel_err(h.download(st), y_or) <= 1e-11
        assert np.max(np.abs(obs[:, 0, :7] - obs_or[:, :7])) <= 1e-11
    else:
        assert np.max(np.abs(obs[:, 0, 1:7] - obs_or[:, 1:7])) <= 1e-5


@pytest.mark.parametrize("kind", ["localised", "superposed"])
@pytest.mark.parametrize("precision", [S.SA_FP64, S.SA_FP32_AUX])
def test_propagation_distinguished(precision, kind):
    """N = 10, a two-exponential Matsubara bath, L = 6, with loss and the
    terminator: 2000 RK4 steps through sa_heom_init_physical and
    sa_heom_propagate, observables every 100 steps."""
    N, L = 10, 6
    bath = OB.matsubara(0.01, 0.05, 0.025, 1, 0.0)
    kw = dict(detuning=0.0, g=0.05 / np.sqrt(N), kappa=0.005, term=0.002, d=1)
    sa = oracle.SA(N, len(bath["c"]), L, bath, **kw)
    x0 = _initial(sa, kind)
    y_or, obs_or = sa.propagate(x0, 0.02, 2000, 100)
    h = S.Heom(S.make_params(N, len(bath["c"]), L, bath, **kw), precision=precision)
    st = h.new_state()
    h.init_physical(st, x0[:_nphys(sa)])
    obs = h.propagate(st, 0.02, 2000, 100)
    torch.cuda.synchronize()
    if kind == "localised":
        # Sec. V.F on resonance: P_+ = P_- = 1/(2N), P_D = 1 - 1/N at t = 0
        assert abs(obs[0, 0, 5] - 1 / (2 * N)) < 1e-14 and abs(obs[0, 0, 6] - 1 / (2 * N)) < 1e-14
        assert abs(obs[0, 0, 4] - (1 - 1 / N)) < 1e-14
    if precision == S.SA_FP64:
        assert rel_err(h.download(st), y_or) <= 1e-11
        assert np.max(np.abs(obs[:, 0, :7] - obs_or[:, :7])) <= 1e-11
    else:
        err = np.max(np.abs(obs[:, 0, 1:7] - obs_or[:, 1:7]))
        print(f"d=1 {kind} FP32-aux max population error vs FP64 oracle: {err:.3e}")
        assert err <= 1e-5
    assert oracle.errors() == 0


@pytest.mark.parametrize("precision,tol", [(S.SA_FP64, 1e-11), (S.SA_FP32_AUX, 1e-5)])
def test_localised_paper_size(precision, tol):
    """The Sec. V.F hierarchy at its own size: one exponential, L = 25,
    N = 100 >= 28, so 1715600 unique variables; the localised state for 10
    RK4 steps against the oracle (whole state in FP64, populations in
    FP32-aux)."""
    N, L = 100, 25
    bath = OB.high_t(0.01, 0.05, 0.025, 0.0)
    kw = dict(detuning=0.0, g=0.05 / np.sqrt(N), kappa=0.0, d=1)
    sa = oracle.SA(N, 1, L, bath, **kw)
    assert sa.nvar == 1715600
    x0 = _initial(sa, "localised")
    y_or, obs_or = sa.propagate(x0, 0.05, 10, 5)
    h = S.Heom(S.make_params(N, 1, L, bath, **kw), precision=precision)
    assert h.n_vars == 1715600
    st = h.new_state()
    h.init_physical(st, x0[:_nphys(sa)])
    obs = h.propagate(st, 0.05, 10, 5)
    torch.cuda.synchronize()
    if precision == S.SA_FP64:
        assert rel_err(h.download(st), y_or) <= tol
    assert np.max(np.abs(obs[:, 0, 1:7] - obs_or[:, 1:7])) <= tol


@pytest.mark.parametrize("kernel", KERNELS)
def test_mixed_batch_matches_oracle(kernel):
    """A batch with d = 0 .. 3 instances, all started through
    sa_heom_init_physical: 40 RK4 steps of every instance against its oracle,
    FP64."""
    specs = [(5, 2, 4, 0), (9, 1, 5, 1), (3, 3, 3, 1), (1, 2, 4, 1), (6, 1, 4, 2), (7, 2, 3, 3)]
    sas, ps, xs = [], [], []
    for i, (N, m, L, d) in enumerate(specs):
        b = _generic_bath(m, 40 + i)
        kw = dict(detuning=0.02 * i, g=0.1, kappa=0.01, term=0.003 * i, d=d)
        sa = oracle.SA(N, m, L, b, **kw)
        sas.append(sa)
        ps.append(S.make_params(N, m, L, b, **kw))
        xs.append(_initial(sa, "superposed") if d else sa.initial_state(0.7, 0.2, 0.2, 0.3 / N, 0.0))
    h = S.Heom(ps)
    h.set_kernel(kernel)
    st = h.new_state()
    phys = np.zeros((len(sas), S.PHYS_SLOTS), complex)
    for i, (sa, x) in enumerate(zip(sas, xs)):
        phys[i, :_nphys(sa)] = x[:_nphys(sa)]
    h.init_physical(st, phys)
    for _ in range(40):
        h.step(st, 0.05)
    torch.cuda.synchronize()
    y = h.download(st)
    for i, (sa, x) in enumerate(zip(sas, xs)):
        off = h.var_offset(i)
        assert rel_err(y[off:off + sa.nvar], sa.rk4(x, 0.05, 40)) <= 1e-11
    assert oracle.errors() == 0


def test_init_state_rejects_distinguished():
    """The five-value symmetric initial state cannot describe a d = 1
    instance: sa_heom_init_state refuses it, sa_heom_init_physical takes it."""
    bath = OB.high_t(0.01, 0.05, 0.025, 0.0)
    h = S.Heom(S.make_params(4, 1, 3, bath, g=0.05, d=1))
    st = h.new_state()
    with pytest.raises(S.SaHeomError) as e:
        h.init_state(st, [1.0, 0, 0, 0, 0])
    assert e.value.code == -1
    sa = oracle.SA(4, 1, 3, bath, 0.0, 0.05, 0.0, d=1)
    h.init_physical(st, _initial(sa, "localised")[:_nphys(sa)])
    np.testing.assert_array_equal(h.download(st), _initial(sa, "localised"))
