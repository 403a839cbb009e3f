"""The launch-tuning cache on the GPU: the first sa_heom_autotune times the
variants and stores the winner under the handle's key; a second handle of
the same shape gets it without timing (much faster, same tuning); a forced
call times afresh; a cache saved to a file and loaded into an emptied cache
serves the same tuning."""
import time

import numpy as np
import pytest

import paper_2608_20657_b300 as S
from paper_2608_20657_b300 import binding as B
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def _handle():
    ws = W.batch_w4(24, seed=41)
    h = S.Heom([S.params_from(w) for w in ws], precision=S.SA_FP32_AUX)
    st = h.new_state()
    h.init_state(st, np.stack([S.rho0_vars(w) for w in ws]))
    return h, st


def _timed(h, st, **kw):
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    best = h.autotune(st, **kw)
    torch.cuda.synchronize()
    return best, time.perf_counter() - t0


def test_autotune_cache_hit_force_and_file(tmp_path):
    B.tuning_cache_clear()
    h1, s1 = _handle()
    best1, t1 = _timed(h1, s1)
    assert B.tuning_cache_size() == 1
    h2, s2 = _handle()
    assert h2.tuning_key() == h1.tuning_key()
    best2, t2 = _timed(h2, s2)
    assert best2 == best1 and h2.tuning() == h1.tuning()
    assert t2 < 0.2 * t1, (t1, t2)
    _, t3 = _timed(h2, s2, force=True)
    assert t3 > 5 * t2
    f = tmp_path / "tune.txt"
    B.tuning_cache_save(str(f))
    B.tuning_cache_clear()
    B.tuning_cache_load(str(f))
    h3, s3 = _handle()
    best3, t4 = _timed(h3, s3)
    assert t4 < 0.2 * t1
    assert h3.tuning() == h2.tuning()
    # the cached tuning gives the same propagation as the handle it came from
    o2 = h2.propagate(s2, 0.02, 20, 20)
    o3 = h3.propagate(s3, 0.02, 20, 20)
    assert np.array_equal(o2, o3)
    B.tuning_cache_clear()
