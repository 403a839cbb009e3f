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


def test_noalloc_full_array_and_side_stream():
    """A batch of exactly SA_HEOM_NOALLOC_MAX_INSTANCES small instances fills
    the whole fixed array; calls on a stream of the caller's own, twice in a
    row with the state advanced in between, match sa_heom_observables."""
    bath = S.bath_drude_lorentz(0.01, 0.05, 0.025, S.BATH_HIGH_T, 0)
    n = S.NOALLOC_MAX_INSTANCES
    assert n == 4096
    rng = np.random.default_rng(11)
    ps = [S.make_params(2, len(bath["c"]), 0, bath, detuning=float(rng.uniform(-0.05, 0.05)),
                        g=float(rng.uniform(0.01, 0.1))) for _ in range(n)]
    h = S.Heom(ps, precision=S.SA_FP64)
    st = h.new_state()
    h.init_state(st, np.tile(np.array([1, 0, 0, 0, 0], complex), (n, 1)))
    side = torch.cuda.Stream()
    torch.cuda.synchronize()
    for call in range(2):
        with torch.cuda.stream(side):
            h.propagate(st, 0.05, 40, observe=False, stream=side)
            got = h.observables_noalloc(st, stream=side)
        ref = h.observables(st, stream=side)
        assert got.shape == ref.shape == (n, 8)
        assert np.max(np.abs(got - ref)) <= 1e-14, call
        assert np.all(np.abs(got[:, 1] - 1.0) > 1e-6), call  # the cavity population moved


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
