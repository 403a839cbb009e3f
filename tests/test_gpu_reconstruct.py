"""GPU parity of the reconstruction of arbitrary initial operators (Sec. IV,
Table tab:representative-initial-operators): the representatives propagated
as one batch (d = 0, 1, 1, 1, 2), then sa_heom_reconstruct_dense, against the
oracle's explicit relabelling of its own representative responses.

Tolerances: FP64 within 1e-11 of max |rho_S(t)|; FP32-aux within 1e-5 (its
hierarchy is single precision, its physical representative FP64)."""
import time

import numpy as np
import pytest

import oracle
import paper_2608_20657_b300 as S
from oracle import reconstruct as R

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def _bath(seed):
    rng = np.random.default_rng(seed)
    return {"c": rng.uniform(0.1, 0.5, 2) + 1j * rng.uniform(-0.4, 0.4, 2),
            "cc": rng.uniform(0.1, 0.5, 2) + 1j * rng.uniform(-0.4, 0.4, 2),
            "nu": rng.uniform(0.2, 1.2, 2) + 1j * rng.uniform(-0.3, 0.3, 2)}


def _gpu_reconstruct(p, A, dt, steps, precision=S.SA_FP64, times=1):
    h = S.Heom(p, precision=precision, representatives=True)
    st = h.new_state()
    h.init_representatives(st)
    if steps:
        h.propagate(st, dt, steps, observe=False)
    a = torch.from_numpy(np.ascontiguousarray(A)).to("cuda")
    outs = [h.reconstruct_dense(st, a).cpu().numpy() for _ in range(times)]
    torch.cuda.synchronize()
    return outs


@pytest.mark.parametrize("precision,tol", [(S.SA_FP64, 1e-11), (S.SA_FP32_AUX, 1e-5)])
@pytest.mark.parametrize("N,L", [(1, 3), (2, 3), (3, 3), (5, 3), (40, 2)])
def test_reconstruct_matches_oracle(N, L, precision, tol):
    bath = _bath(N + L)
    kw = dict(detuning=0.08, g=0.15, kappa=0.02, term=0.005)
    resp = R.responses(R.representative_hierarchies(N, 2, L, bath, **kw), 0.05, 30)
    rng = np.random.default_rng(7 + N)
    A = rng.standard_normal((N + 1, N + 1)) + 1j * rng.standard_normal((N + 1, N + 1))
    ref = R.reconstruct(resp, A)
    got, again = _gpu_reconstruct(S.make_params(N, 2, L, bath, **kw), A, 0.05, 30, precision, times=2)
    assert np.abs(got - ref).max() <= tol * np.abs(ref).max()
    assert np.array_equal(got, again)  # fixed summation order
    assert oracle.errors() == 0


def _conjugate_bath(seed):
    rng = np.random.default_rng(seed)
    c = rng.uniform(0.1, 0.5, 2) + 1j * rng.uniform(-0.4, 0.4, 2)
    return {"c": c, "cc": c.conj(), "nu": rng.uniform(0.2, 1.2, 2) + 0j}


@pytest.mark.parametrize("precision,tol", [(S.SA_FP64, 1e-11), (S.SA_FP32_AUX, 1e-5)])
@pytest.mark.parametrize("N,L", [(1, 3), (2, 3), (5, 3), (40, 2)])
def test_reconstruct_adjoint_shortcut(N, L, precision, tol):
    """Eq. adjoint-preservation: with real nu_k and c-check_k = conj(c_k) the
    |c><e_1| response is the adjoint of the |e_1><c| one, so four
    propagations (SA_BUILD_ADJOINT_REPS) give the same rho_S(t) as five, and
    the oracle's."""
    bath = _conjugate_bath(N + 3 * L)
    kw = dict(detuning=0.08, g=0.15, kappa=0.02, term=0.005)
    p = S.make_params(N, 2, L, bath, **kw)
    rng = np.random.default_rng(11 + N)
    A = rng.standard_normal((N + 1, N + 1)) + 1j * rng.standard_normal((N + 1, N + 1))
    ref = R.reconstruct(R.responses(R.representative_hierarchies(N, 2, L, bath, **kw), 0.05, 30), A)
    h5 = S.Heom(p, precision=precision, representatives=True)
    h4 = S.Heom(p, precision=precision, representatives=True, adjoint=True)
    assert h4.count == h5.count - 1 == (4 if N >= 2 else 3)
    assert h4.n_vars < h5.n_vars
    out = []
    for h in (h5, h4):
        st = h.new_state()
        h.init_representatives(st)
        h.propagate(st, 0.05, 30, observe=False)
        a = torch.from_numpy(np.ascontiguousarray(A)).to("cuda")
        out.append(h.reconstruct_dense(st, a).cpu().numpy())
    five, four = out
    scale = np.abs(ref).max()
    assert np.abs(four - ref).max() <= tol * scale
    assert np.abs(four - five).max() <= (1e-13 if precision == S.SA_FP64 else 1e-6) * scale


def test_reconstruct_large_symmetric_state():
    """N = 2000: for the permutation-invariant upper-polariton operator the
    reconstruction from the five representatives equals the symmetric
    (d = 0) propagation of that operator itself, entry by entry."""
    N, L, m = 2000, 3, 1
    bath = {"c": np.array([0.3 + 0.05j]), "cc": np.array([0.3 - 0.05j]), "nu": np.array([0.6 + 0j])}
    kw = dict(detuning=0.0, g=0.1 / np.sqrt(N), kappa=0.01)
    th = np.pi / 4
    ket = np.zeros(N + 1, complex)
    ket[0] = np.cos(th)
    ket[1:] = np.sin(th) / np.sqrt(N)
    A = np.outer(ket, ket.conj())
    sa = oracle.SA(N, m, L, bath, **kw)
    y = sa.rk4(sa.initial_state_dense(A), 0.05, 40)
    ref = R.physical_dense(sa, y)
    got = _gpu_reconstruct(S.make_params(N, m, L, bath, **kw), A, 0.05, 40)[0]
    assert np.abs(got - ref).max() <= 1e-11 * np.abs(ref).max()


def test_reconstruct_bandwidth():
    """Time the reconstruction at N + 1 = 8192 (1 GiB per dense operator)
    against its algorithmic 48 bytes per entry (A read twice, rho_S(t)
    written once); prints the achieved HBM bandwidth."""
    N = 8191
    bath = {"c": np.array([0.3 + 0.05j]), "cc": np.array([0.3 - 0.05j]), "nu": np.array([0.6 + 0j])}
    h = S.Heom(S.make_params(N, 1, 2, bath, g=0.01), representatives=True)
    st = h.new_state()
    h.init_representatives(st)
    n = N + 1
    a = torch.randn(n, n, dtype=torch.complex128, device="cuda")
    out = torch.empty_like(a)
    for _ in range(3):
        h.reconstruct_dense(st, a, out)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 10
    e0.record()
    for _ in range(reps):
        h.reconstruct_dense(st, a, out)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    gbs = 48.0 * n * n / (ms * 1e-3) / 1e9
    print(f"reconstruct n={n}: {ms:.3f} ms per call, {gbs:.0f} GB/s algorithmic (48 B per entry)")
    assert torch.isfinite(out).all()
