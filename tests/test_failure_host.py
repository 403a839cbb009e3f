"""Failure detection on the host (no GPU): the table validation accepts every
table the builder makes and rejects a connection record whose target has been
moved off its pattern; the debug flags are checked for their preconditions."""
import numpy as np
import pytest

import paper_2608_20657_b300 as S
import workloads as W


def _host(params):
    return S.Heom(params, host_only=True)


@pytest.mark.parametrize("N,m,L,d", [(1, 1, 3, 0), (3, 2, 3, 0), (10, 2, 6, 0), (40, 3, 5, 0), (8, 2, 4, 1),
                                     (6, 1, 5, 2), (5, 2, 3, 3)])
def test_validate_accepts_built_tables(N, m, L, d):
    bath = S.bath_drude_lorentz(0.01, 0.05, 0.025, S.BATH_MATSUBARA, m - 1)
    h = _host(S.make_params(N, len(bath["c"]), L, bath, g=0.02, d=d))
    h.validate()


def test_validate_accepts_w4_batch():
    ws = W.batch_w4(24, seed=5)
    _host([S.params_from(w) for w in ws]).validate()


def test_corrupted_record_rejected():
    bath = S.bath_drude_lorentz(0.01, 0.05, 0.025, S.BATH_MATSUBARA, 1)
    h = _host(S.make_params(6, len(bath["c"]), 4, bath, g=0.02))
    h.validate()
    h.set_debug(S.SA_DEBUG_CORRUPT_RECORD)
    with pytest.raises(S.SaHeomError) as e:
        h.validate()
    assert e.value.code == -7
    assert "target is not the first variable of a pattern" in str(e.value)


def test_debug_flags_preconditions():
    bath = S.bath_drude_lorentz(0.01, 0.05, 0.025, S.BATH_HIGH_T, 0)
    h = _host(S.make_params(3, 1, 0, bath, g=0.02))  # L = 0: no records at all
    with pytest.raises(S.SaHeomError) as e:
        h.set_debug(S.SA_DEBUG_CORRUPT_RECORD)
    assert e.value.code == -7
    with pytest.raises(S.SaHeomError) as e:
        h.set_debug(64)
    assert e.value.code == -1
    h.set_debug(S.SA_DEBUG_EXPIRE_WAIT)  # accepted; takes effect on a device handle
    h.set_debug(S.SA_DEBUG_CHECK_INDICES)
    h.set_debug(0)
    # a planted bad list index only ever comes with the kernels' index check,
    # and only on a device handle
    for flags in (S.SA_DEBUG_CORRUPT_LIST, S.SA_DEBUG_CORRUPT_LIST | S.SA_DEBUG_CHECK_INDICES):
        with pytest.raises(S.SaHeomError) as e:
            h.set_debug(flags)
        assert e.value.code == -1
