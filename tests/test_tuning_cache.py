"""The launch-tuning cache on the host: the key of a handle depends on its
precision, layout and batch shape and not on N beyond the size bucket, and
the cache's text file round-trips and rejects malformed input.  (Hits and
misses of sa_heom_autotune: tests/test_gpu_tuning_cache.py.)"""
import os

import numpy as np
import pytest

import paper_2608_20657_b300 as S
from paper_2608_20657_b300 import binding as B

BATH = {"c": np.array([0.3 + 0.1j]), "cc": np.array([0.3 - 0.1j]), "nu": np.array([0.6 + 0j])}


def _key(specs, precision=S.SA_FP64, pack=False):
    ps = [S.make_params(N, 1, L, BATH, d=d, g=0.1) for N, L, d in specs]
    return S.Heom(ps, precision=precision, host_only=True, pack=pack).tuning_key()


def test_key_follows_shape_precision_layout():
    base = [(12, 3, 0), (20, 4, 1)]
    k = _key(base)
    assert _key(base) == k
    assert _key([(13, 3, 0), (21, 4, 1)]) == k          # saturated N: same shapes, same variable count
    assert _key(base, precision=S.SA_FP32_AUX) != k
    assert _key([(12, 3, 0), (20, 5, 1)]) != k          # another L
    assert _key([(12, 3, 0), (20, 4, 0)]) != k          # another d
    assert _key(base + [(12, 3, 0)]) != k               # another multiset
    specs = [(10 + i, 3, 0) for i in range(20)]
    assert _key(specs, pack=True) != _key(specs)


def test_cache_file_round_trip(tmp_path):
    B.tuning_cache_clear()
    assert B.tuning_cache_size() == 0
    src = tmp_path / "in.txt"
    src.write_text("00000000000000ab 128 192 1 1\n123456789abcdef0 256 64 0 0\n")
    B.tuning_cache_load(str(src))
    assert B.tuning_cache_size() == 2
    out = tmp_path / "out.txt"
    B.tuning_cache_save(str(out))
    assert sorted(out.read_text().split("\n")) == sorted(src.read_text().split("\n"))
    B.tuning_cache_clear()
    assert B.tuning_cache_size() == 0


@pytest.mark.parametrize("text", ["zz 128 192 1 1\n", "00000000000000ab 100 192 1 1\n",
                                  "00000000000000ab 128 192 2 1\n", "00000000000000ab 128 192 1\n",
                                  "00000000000000ab 128 4096 1 1\n"])
def test_cache_rejects_malformed_files(tmp_path, text):
    B.tuning_cache_clear()
    f = tmp_path / "bad.txt"
    f.write_text(text)
    with pytest.raises(S.SaHeomError) as e:
        B.tuning_cache_load(str(f))
    assert e.value.code == -1
    assert B.tuning_cache_size() == 0
    with pytest.raises(S.SaHeomError):
        B.tuning_cache_load(os.path.join(str(tmp_path), "missing.txt"))
