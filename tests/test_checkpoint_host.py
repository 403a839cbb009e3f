"""The configuration hash a checkpoint carries (no GPU): equal for equal
handles, different as soon as any parameter, the precision or an instance of
the batch differs."""
import numpy as np

import paper_2608_20657_b300 as S
import workloads as W


def _hash(params, precision=S.SA_FP64):
    return S.Heom(params, precision=precision, host_only=True).config_hash()


def test_hash_stable_and_sensitive():
    ws = W.batch_w4(5, seed=9)
    ps = [S.params_from(w) for w in ws]
    h0 = _hash(ps)
    assert h0 == _hash([S.params_from(w) for w in ws])
    assert h0 != _hash(ps, S.SA_FP32_AUX)
    assert h0 != _hash(ps[:4])
    assert h0 != _hash(ps[::-1])
    for field, delta in [("g", 1e-12), ("detuning", 1e-9), ("kappa", 1e-6), ("term", 1e-3)]:
        q = [S.params_from(w) for w in ws]
        setattr(q[2], field, getattr(q[2], field) + delta)
        assert _hash(q) != h0, field
    q = [S.params_from(w) for w in ws]
    q[1].c_re[0] = np.nextafter(q[1].c_re[0], 1.0)
    assert _hash(q) != h0
    q = [S.params_from(w) for w in ws]
    q[3].N = q[3].N + 1
    assert _hash(q) != h0
