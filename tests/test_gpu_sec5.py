"""GPU parity at the paper's production set (Sec. V): L = 25, one exponential
plus the terminator, dt = 0.5 fs, in rad/fs units.  Short runs against the
FP64 oracle: the whole state in FP64 within 1e-11 relative, populations
within 1e-11 (FP64) and 1e-5 (FP32-aux)."""
import numpy as np
import pytest

import oracle
import paper_2608_20657_b300 as S
import workloads as W
from tests._helpers import oracle_initial, oracle_sa, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


@pytest.mark.parametrize("precision", [S.SA_FP64, S.SA_FP32_AUX])
@pytest.mark.parametrize("N,init,steps", [(5, "up", 40), (10 ** 12, "up", 20), (1000, "localised", 10),
                                          (25, "superposed", 20)])
def test_sec5_short_runs(N, init, steps, precision):
    w = W.sec5(N, init, steps=steps)
    sa = oracle_sa(w)
    x0 = oracle_initial(sa, w)
    y_or, obs_or = sa.propagate(x0, w["dt_fs"], steps, steps // 2)
    h = S.Heom(S.params_from(w), precision=precision)
    assert h.n_vars == sa.nvar
    st = h.new_state()
    h.init_physical(st, S.phys_vars(w))
    obs = h.propagate(st, w["dt_fs"], steps, steps // 2)
    torch.cuda.synchronize()
    if precision == S.SA_FP64:
        assert rel_err(h.download(st), y_or) <= 1e-11
        assert np.max(np.abs(obs[:, 0, :7] - obs_or[:, :7])) <= 1e-11
    else:
        assert np.max(np.abs(obs[:, 0, 1:7] - obs_or[:, 1:7])) <= 1e-5
    assert oracle.errors() == 0
