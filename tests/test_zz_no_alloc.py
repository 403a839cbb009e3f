"""sa_heom_observables_noalloc: the observables entry point that allocates no
device memory (its output buffer is a fixed array inside the library) must
return what sa_heom_observables returns.  Collected last on purpose."""
import numpy as np
import pytest

import paper_2608_20657_b300 as S
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


@pytest.mark.parametrize("precision", [S.SA_FP32_AUX, S.SA_FP64])
def test_noalloc_observables_match(precision):
    ws = W.batch_w4(6, seed=21)
    h = S.Heom([S.params_from(w) for w in ws], precision=precision)
    st = h.new_state()
    h.init_state(st, np.stack([S.rho0_vars(w) for w in ws]))
    for call in range(2):  # two calls in a row, the state advanced in between
        h.propagate(st, 0.02, 25, observe=False)
        torch.cuda.synchronize()
        ref = h.observables(st)
        got = h.observables_noalloc(st)
        assert got.shape == ref.shape == (6, 8)
        assert np.max(np.abs(got - ref)) <= 1e-14, call
        assert np.all(np.isfinite(got))


def test_noalloc_rejects_oversized_batch():
    bath = S.bath_drude_lorentz(0.01, 0.05, 0.025, S.BATH_HIGH_T, 0)
    p = S.make_params(2, len(bath["c"]), 0, bath, g=0.03)
    n = 4097
    h = S.Heom([p] * n, precision=S.SA_FP32_AUX)
    st = h.new_state()
    h.init_state(st, np.tile(np.array([1, 0, 0, 0, 0], complex), (n, 1)))
    with pytest.raises(S.SaHeomError) as e:
        h.observables_noalloc(st)
    assert e.value.code == -2
    assert np.allclose(h.observables(st)[:, 1], 1.0)
