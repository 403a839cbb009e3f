"""The packed device layout (SA_BUILD_PACK_INSTANCES) and the pack kernel on
the GPU: the right-hand side of a batch with packed templates and
singletons against the oracle in both precisions, RK4 propagation against
the unpacked handle and the oracle, state marshalling and the documented
element of every variable, observables, the bounded-wait failure path,
checkpoints, and the full w4 batch."""
import numpy as np
import pytest

import oracle
import paper_2608_20657_b300 as S
import workloads as W
from tests._helpers import oracle_sa, rel_err
from tests.test_packs import _batch

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def _setup(precision, pack=True):
    specs = _batch()
    ps = [S.make_params(N, m, L, b, d=d, **kw) for (N, m, L, d, b, kw) in specs]
    sas = [oracle.SA(N, m, L, b, d=d, **kw) for (N, m, L, d, b, kw) in specs]
    return S.Heom(ps, precision=precision, pack=pack), sas


def _rand(h, seed):
    return W.random_state(h.n_vars, seed=seed)


@pytest.mark.parametrize("precision", [S.SA_FP64, S.SA_FP32_AUX])
def test_packed_rhs_against_oracle(precision):
    h, sas = _setup(precision)
    assert h.launches_per_step() == 4 * (1 if precision == S.SA_FP64 else 2)  # pack kernel with list units (+ rho_0)
    x = _rand(h, 11)
    if precision == S.SA_FP32_AUX:
        x = x.astype(np.complex64).astype(np.complex128)
    xs, dx = h.new_state(), h.new_state()
    h.upload(xs, x)
    h.rhs(xs, dx)
    torch.cuda.synchronize()
    d = h.download(dx)
    tol = 1e-13 if precision == S.SA_FP64 else 2e-6
    for i, sa in enumerate(sas):
        a = h.var_offset(i)
        assert rel_err(d[a:a + sa.nvar], sa.rhs(x[a:a + sa.nvar])) <= tol, i


def test_packed_rk4_against_unpacked_and_oracle():
    hp, sas = _setup(S.SA_FP64)
    hu, _ = _setup(S.SA_FP64, pack=False)
    x = _rand(hp, 12)
    sp, su = hp.new_state(), hu.new_state()
    hp.upload(sp, x)
    hu.upload(su, x)
    hp.propagate(sp, 0.05, 20, observe=False)
    hu.propagate(su, 0.05, 20, observe=False)
    torch.cuda.synchronize()
    xp, xu = hp.download(sp), hu.download(su)
    assert rel_err(xp, xu) <= 1e-13
    for i in (0, 7, len(sas) - 1):
        a = hp.var_offset(i)
        n = sas[i].nvar
        assert rel_err(xp[a:a + n], sas[i].rk4(x[a:a + n], 0.05, 20)) <= 1e-11, i


@pytest.mark.parametrize("precision", [S.SA_FP64, S.SA_FP32_AUX])
def test_packed_tuning_invariance(precision):
    """The pack kernel takes the list units of the unpacked instances after its
    pack units, from the atomic counter or by static striding: every block
    size, item size and queue mode gives the same bits (no sum depends on
    which warp evaluates an item)."""
    h, _ = _setup(precision)
    x = _rand(h, 13)
    out = []
    for (b, c, q) in [(128, 192, 1), (128, 192, 0), (64, 160, 1), (256, 128, 0), (96, 96, 1)]:
        h.set_tuning(b, c, q)
        st = h.new_state()
        h.upload(st, x)
        h.propagate(st, 0.05, 6, observe=False)
        torch.cuda.synchronize()
        out.append(h.download(st))
    h.device_error()  # raises if a wait expired or an index was out of range
    for o in out[1:]:
        assert np.array_equal(o, out[0])


@pytest.mark.parametrize("precision", [S.SA_FP64, S.SA_FP32_AUX])
def test_packed_marshalling_and_element_index(precision):
    h, _ = _setup(precision)
    x = _rand(h, 13)
    st = h.new_state()
    h.upload(st, x)
    torch.cuda.synchronize()
    back = h.download(st)
    if precision == S.SA_FP64:
        assert np.array_equal(back, x)
        raw = st.view(torch.float64).cpu().numpy()[:2 * h.n_vars].view(np.complex128)
    else:
        rho = np.zeros(h.n_vars, bool)
        for i in range(h.count):  # physical representatives: from their FP64 side slots
            a = h.var_offset(i)
            rho[a:a + int(h.dump_patterns(i)["var_off"][1])] = True
        assert np.array_equal(back[rho], x[rho])
        x32 = x.astype(np.complex64).astype(np.complex128)
        assert np.array_equal(back[~rho], x32[~rho])
        raw = st.view(torch.float32).cpu().numpy()[:2 * h.n_vars].view(np.complex64).astype(np.complex128)
    for i in range(h.count):
        a = h.var_offset(i)
        nv = (h.var_offset(i + 1) if i + 1 < h.count else h.n_vars) - a
        e = np.array([h.state_index(i, v) for v in range(nv)])
        ref = x[a:a + nv] if precision == S.SA_FP64 else x[a:a + nv].astype(np.complex64).astype(np.complex128)
        assert np.array_equal(raw[e], ref), i


def test_packed_observables_match_unpacked():
    """FP32-aux from the same physical initial states: populations of the
    packed and unpacked handles agree to FP32 rounding over 300 steps."""
    hp, sas = _setup(S.SA_FP32_AUX)
    hu, _ = _setup(S.SA_FP32_AUX, pack=False)
    rng = np.random.default_rng(5)
    phys = []
    for sa in sas:
        v = np.zeros(sa.nvar, complex)
        v[0] = 0.6
        v[1:3] = 0.2 * (rng.standard_normal(2) + 1j * rng.standard_normal(2))
        phys.append(v[:int(sa.patterns()["var_off"][1])])
    width = max(p.size for p in phys)
    arr = np.zeros((len(phys), width), complex)
    for i, p in enumerate(phys):
        arr[i, :p.size] = p
    sp, su = hp.new_state(), hu.new_state()
    hp.init_physical(sp, arr)
    hu.init_physical(su, arr)
    op = hp.propagate(sp, 0.05, 300, 50)
    ou = hu.propagate(su, 0.05, 300, 50)
    assert np.max(np.abs(op[..., :7] - ou[..., :7])) <= 1e-6


def test_packed_expired_wait_reported_then_recovers():
    h, sas = _setup(S.SA_FP64)
    x = _rand(h, 14)
    st = h.new_state()
    h.upload(st, x)
    h.device_error()
    h.set_debug(S.SA_DEBUG_EXPIRE_WAIT)
    h.step(st, 0.05)
    with pytest.raises(S.SaHeomError) as e:
        h.device_error()
    assert e.value.code == -5
    h.set_debug(0)
    h.upload(st, x)
    h.step(st, 0.05)
    h.device_error()
    got = h.download(st)
    for i in (0, len(sas) - 1):
        a = h.var_offset(i)
        n = sas[i].nvar
        assert rel_err(got[a:a + n], sas[i].rk4(x[a:a + n], 0.05, 1)) <= 1e-13


def test_packed_checkpoint_resume_and_refusal():
    h, _ = _setup(S.SA_FP64)
    st = h.new_state()
    h.upload(st, _rand(h, 15))
    h.propagate(st, 0.05, 10, observe=False)
    ck = h.checkpoint(st, 10)
    h.propagate(st, 0.05, 10, observe=False)
    torch.cuda.synchronize()
    ref = st.clone()
    h2, _ = _setup(S.SA_FP64)
    st2 = h2.new_state()
    assert h2.resume(st2, ck) == 10
    h2.propagate(st2, 0.05, 10, observe=False)
    torch.cuda.synchronize()
    assert torch.equal(st2, ref)
    hu, _ = _setup(S.SA_FP64, pack=False)  # same parameters, other layout
    with pytest.raises(S.SaHeomError) as e:
        hu.resume(hu.new_state(), ck)
    assert e.value.code == -7


@pytest.mark.slow
def test_w4_packed_full_batch():
    """The full w4 batch packed (FP32-aux): the right-hand side of a seeded
    random float state against the oracle at four instances, and FP32-aux
    populations against the packed FP64 run over 500 steps."""
    ws = W.batch_w4()
    ps = [S.params_from(w) for w in ws]
    h = S.Heom(ps, precision=S.SA_FP32_AUX, pack=True)
    x = W.random_state(h.n_vars, seed=7).astype(np.complex64).astype(np.complex128)
    xs, dx = h.new_state(), h.new_state()
    h.upload(xs, x)
    h.rhs(xs, dx)
    torch.cuda.synchronize()
    d = h.download(dx)
    del xs, dx
    for i in [0, 100, 255, 511]:
        sa = oracle_sa(ws[i])
        a = h.var_offset(i)
        assert rel_err(d[a:a + sa.nvar], sa.rhs(x[a:a + sa.nvar])) <= 2e-6, i
    h64 = S.Heom(ps, precision=S.SA_FP64, pack=True)
    rho0 = np.stack([S.rho0_vars(w) for w in ws])
    s32, s64 = h.new_state(), h64.new_state()
    h.init_state(s32, rho0)
    h64.init_state(s64, rho0)
    o32 = h.propagate(s32, 0.02, 500, 100)
    o64 = h64.propagate(s64, 0.02, 500, 100)
    assert np.max(np.abs(o32[..., 1:7] - o64[..., 1:7])) <= 1e-5
    h64.close()
    h.close()
    torch.cuda.empty_cache()
