"""Checkpoint / resume on the GPU: a run stopped at step 60, saved, loaded into
a fresh handle and state and continued for 60 more steps lands bit for bit on
the uninterrupted 120-step run, in both precisions; a checkpoint of other
parameters, another precision or a truncated buffer is refused and leaves the
state untouched."""
import numpy as np
import pytest

import paper_2608_20657_b300 as S
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def _setup(precision, ws):
    h = S.Heom([S.params_from(w) for w in ws], precision=precision)
    st = h.new_state()
    h.init_state(st, np.stack([S.rho0_vars(w) for w in ws]))
    return h, st


@pytest.mark.parametrize("precision", [S.SA_FP64, S.SA_FP32_AUX])
def test_resume_is_bit_identical(precision):
    ws = W.batch_w4(6, seed=31)
    h, st = _setup(precision, ws)
    h.propagate(st, 0.02, 60, observe=False)
    ck = h.checkpoint(st, 60)
    h.propagate(st, 0.02, 60, observe=False)
    torch.cuda.synchronize()
    ref = st.clone()
    h2, st2 = _setup(precision, ws)
    assert h2.resume(st2, ck) == 60
    h2.propagate(st2, 0.02, 60, observe=False)
    torch.cuda.synchronize()
    assert torch.equal(st2, ref)


def test_resume_refuses_other_configurations():
    ws = W.batch_w4(4, seed=32)
    h, st = _setup(S.SA_FP64, ws)
    h.propagate(st, 0.02, 10, observe=False)
    ck = h.checkpoint(st, 10)
    other = [dict(w) for w in ws]
    other[1]["gsn"] *= 1.01
    h2, st2 = _setup(S.SA_FP64, other)
    before = st2.clone()
    with pytest.raises(S.SaHeomError) as e:
        h2.resume(st2, ck)
    assert e.value.code == -7 and "parameters" in str(e.value)
    h3, st3 = _setup(S.SA_FP32_AUX, ws)
    with pytest.raises(S.SaHeomError) as e:
        h3.resume(st3, ck)
    assert e.value.code == -7
    h4, st4 = _setup(S.SA_FP64, ws)
    before4 = st4.clone()
    with pytest.raises(S.SaHeomError) as e:
        h4.resume(st4, ck[:len(ck) // 2])
    assert e.value.code == -7 and "truncated" in str(e.value)
    torch.cuda.synchronize()
    assert torch.equal(st2, before) and torch.equal(st4, before4)
