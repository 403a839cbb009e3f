"""Failure detection on the GPU, without a fault: the stage kernels' bounded
wait on their bulk copies is made to report expiry (SA_DEBUG_EXPIRE_WAIT: the
expiry path is taken without testing the barrier, and each warp still drains
its copies before leaving), which sa_heom_device_error must return as
SA_ERR_TIMEOUT; with the flag off again the same handle steps correctly.  A
NaN in the hierarchy surfaces as SA_ERR_NUMERIC at the first observable it
reaches.  With SA_DEBUG_CHECK_INDICES the list and pack kernels check every
table index they read: on correct tables the result is unchanged bit for bit,
and a target planted out of range (SA_DEBUG_CORRUPT_LIST, only ever together
with the check, which replaces it by index 0 before any access) is reported
as SA_ERR_STATE; with the flags off again the tables are rebuilt correct."""
import numpy as np
import pytest

import oracle
import paper_2608_20657_b300 as S
import workloads as W
from tests._helpers import rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

BATH = {"c": np.array([0.2 + 0.05j]), "cc": np.array([0.2 - 0.05j]), "nu": np.array([0.5 + 0j])}
KW = dict(detuning=0.05, g=0.1, kappa=0.01)


@pytest.mark.parametrize("kernel", [S.SA_KERNEL_LISTS])
def test_expired_wait_reported_then_recovers(kernel):
    N, m, L = 3, 1, 3
    sa = oracle.SA(N, m, L, BATH, **KW)
    h = S.Heom(S.make_params(N, m, L, BATH, **KW))
    h.set_kernel(kernel)
    x = W.random_state(sa.nvar, seed=77)
    st = h.new_state()
    h.upload(st, x)
    h.device_error()  # clean
    h.set_debug(S.SA_DEBUG_EXPIRE_WAIT)
    h.step(st, 0.05)
    with pytest.raises(S.SaHeomError) as e:
        h.device_error()
    assert e.value.code == -5
    h.device_error()  # reading cleared the word
    h.set_debug(0)
    h.upload(st, x)
    h.step(st, 0.05)
    h.device_error()
    assert rel_err(h.download(st), sa.rk4(x, 0.05, 1)) <= 1e-13


def test_expired_wait_fails_propagate_with_observables():
    h = S.Heom(S.make_params(3, 1, 3, BATH, **KW))
    st = h.new_state()
    h.init_state(st, [1, 0, 0, 0, 0])
    h.set_debug(S.SA_DEBUG_EXPIRE_WAIT)
    with pytest.raises(S.SaHeomError) as e:
        h.propagate(st, 0.05, 3, 1)
    assert e.value.code == -5


@pytest.mark.parametrize("precision", [S.SA_FP64, S.SA_FP32_AUX])
def test_nan_in_hierarchy_flagged_at_first_observable(precision):
    N, m, L = 4, 1, 3
    sa = oracle.SA(N, m, L, BATH, **KW)
    h = S.Heom(S.make_params(N, m, L, BATH, **KW), precision=precision)
    st = h.new_state()
    h.init_state(st, [1, 0, 0, 0, 0])
    x = h.download(st)
    pt = h.dump_patterns(0)
    x[pt["var_off"][1]] = np.nan  # Z of the first tier-1 pattern
    h.upload(st, x)
    assert np.all(np.isfinite(h.observables(st)))  # rho_S itself is still finite
    with pytest.raises(S.SaHeomError) as e:
        h.propagate(st, 0.05, 2, 1)  # tier 1 feeds rho_S in the first step
    assert e.value.code == -6


def _batch(pack=False):
    """A batch of w4-like instances, or (pack) one with templates large
    enough to form packs of 32, 20 and 17 lanes besides unpacked instances."""
    if pack:
        from tests.test_packs import _batch as packed_specs

        ps = [S.make_params(N, m, L, b, d=d, **kw) for (N, m, L, d, b, kw) in packed_specs()]
        h = S.Heom(ps, precision=S.SA_FP64, pack=True)
        assert len(h.dump_packs()["packs"]) == 3
    else:
        h = S.Heom([S.params_from(w) for w in W.batch_w4(40, seed=44)], precision=S.SA_FP64)
    return h, W.random_state(h.n_vars, seed=45)


@pytest.mark.parametrize("pack", [False, True])
def test_index_checks_leave_results_unchanged(pack):
    h, x = _batch(pack)
    a, b = h.new_state(), h.new_state()
    h.upload(a, x)
    h.upload(b, x)
    h.propagate(a, 0.02, 5, observe=False)
    h.set_debug(S.SA_DEBUG_CHECK_INDICES)
    h.propagate(b, 0.02, 5, observe=False)
    h.device_error()  # no index out of range
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    h.set_debug(0)


def test_planted_bad_index_reported_then_recovers():
    N, m, L = 4, 1, 3
    sa = oracle.SA(N, m, L, BATH, **KW)
    h = S.Heom(S.make_params(N, m, L, BATH, **KW))
    x = W.random_state(sa.nvar, seed=46)
    st = h.new_state()
    h.set_debug(S.SA_DEBUG_CHECK_INDICES | S.SA_DEBUG_CORRUPT_LIST)
    h.upload(st, x)
    h.step(st, 0.05)
    with pytest.raises(S.SaHeomError) as e:
        h.device_error()
    assert e.value.code == -7 and "index out of range" in str(e.value)
    h.device_error()  # reading cleared the word
    h.set_debug(0)  # the lists are rebuilt correct
    h.upload(st, x)
    h.step(st, 0.05)
    h.device_error()
    assert rel_err(h.download(st), sa.rk4(x, 0.05, 1)) <= 1e-13
