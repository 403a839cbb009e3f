"""The library's host-built tables against the oracle's, bit for bit.

Integer tables (local vectors, canonical patterns and their order, tiers,
categories, multiplicities M_q, variable offsets) must be identical, and the
hierarchy connections -- every (variable, source variable, channel, occupation,
raise/lower, row/column) term of Eqs. uvar-up and uvar-down -- must be the
same set.  The oracle lists the two raise terms of P_q, which cancel exactly
(both deltas of Eq. projector-commutator-element name the same molecule); the
library omits them.  No GPU is used: the handle is built host-only.
"""
import numpy as np
import pytest

import oracle
import oracle.bath as OB
import paper_2608_20657_b300 as S
import workloads as W


def _oracle_bath(w):
    if w["scheme"] == "high_t":
        return OB.high_t(w["lam"], w["gam"], w["kT"], w["sigma"])
    if w["scheme"] == "matsubara":
        return OB.matsubara(w["lam"], w["gam"], w["kT"], w["poles"], w["sigma"])
    return OB.pade(w["lam"], w["gam"], w["kT"], w["poles"], w["sigma"])


def _pair(N, m, L, bath, **kw):
    sa = oracle.SA(N, m, L, bath, **kw)
    lib = S.Heom(S.make_params(N, m, L, bath, **kw), host_only=True)
    return sa, lib


def _generic_bath(m, seed):
    rng = np.random.default_rng(seed)
    return {"c": rng.uniform(0.1, 0.5, m) + 1j * rng.uniform(-0.4, 0.4, m),
            "cc": rng.uniform(0.1, 0.5, m) + 1j * rng.uniform(-0.4, 0.4, m),
            "nu": rng.uniform(0.2, 1.2, m) + 1j * rng.uniform(-0.3, 0.3, m)}


CASES = [(1, 1, 3), (2, 1, 3), (3, 1, 0), (3, 2, 3), (4, 1, 5), (5, 2, 4), (10, 2, 6), (12, 3, 4), (7, 4, 3),
         (100, 2, 8), (30, 1, 12), (1000000, 1, 9), (6, 5, 3), (2, 2, 6)]


D_CASES = [(1, 1, 3), (2, 1, 3), (3, 1, 0), (3, 2, 3), (4, 1, 5), (5, 2, 4), (10, 2, 6), (12, 3, 4), (7, 4, 3),
           (100, 2, 8), (30, 1, 12), (1000000, 1, 9), (6, 5, 3), (2, 2, 6), (2, 1, 1), (1, 3, 4)]


@pytest.mark.parametrize("N,m,L", CASES)
def test_tables_bit_exact(N, m, L):
    _check_tables(N, m, L, 0)


@pytest.mark.parametrize("N,m,L", D_CASES)
def test_tables_bit_exact_distinguished(N, m, L):
    """One distinguished molecule (Sec. V.F): molecule 1's vector ids
    V .. 2V-1 close every pattern, with the same order, categories and
    connections as the oracle's."""
    _check_tables(N, m, L, 1)


@pytest.mark.parametrize("N,m,L,d", [(2, 1, 3, 2), (3, 2, 3, 2), (5, 2, 4, 2), (30, 1, 8, 2), (4, 3, 3, 2),
                                     (3, 1, 3, 3), (6, 2, 3, 3), (40, 1, 6, 3), (3, 4, 2, 3)])
def test_tables_bit_exact_several_distinguished(N, m, L, d):
    """d = 2, 3 (Eq. N-symmetric-pool): molecule j's ids j V .. j V + V - 1
    close every pattern in molecule order."""
    _check_tables(N, m, L, d)


def _check_tables(N, m, L, d):
    sa, lib = _pair(N, m, L, _generic_bath(m, N + 7 * m + L), detuning=0.1, g=0.2, kappa=0.05, d=d)
    assert lib.n_patterns == sa.npat and lib.n_vars == sa.nvar
    assert np.array_equal(lib.dump_vectors(0), sa.vectors())
    a, b = lib.dump_patterns(0), sa.patterns()
    for key in ("tier", "r", "G", "h", "var_off", "cat_off", "ids", "cat_id", "cat_M"):
        assert np.array_equal(a[key], b[key]), key
    lt, ot = lib.dump_terms(0), sa.terms()
    lab = sa.var_labels()
    # oracle: drop the cancelling raise pairs of P_q
    isP = lab["kind"][ot["var"]] == 3
    keep = ~(isP & (ot["dir"] == 1))
    pairs = ot["var"][isP & (ot["dir"] == 1)]
    # each dropped P raise term comes with its opposite-side twin
    if pairs.size:
        sub = {k: v[isP & (ot["dir"] == 1)] for k, v in ot.items()}
        key = np.stack([sub["var"], sub["src"], sub["k"], sub["n"]], 1)
        u, cnt = np.unique(key, axis=0, return_counts=True)
        assert np.all(cnt == 2)
        assert np.all(np.bincount(sub["side"]) == pairs.size // 2)
    o = np.stack([ot[k][keep] for k in ("var", "src", "k", "n", "dir", "side")], 1)
    l = np.stack([lt[k] for k in ("var", "src", "k", "n", "dir", "side")], 1)
    oi, li = np.lexsort(o.T[::-1]), np.lexsort(l.T[::-1])
    o, l = o[oi], l[li]
    assert o.shape == l.shape
    assert np.array_equal(o, l)
    # the FP64 coefficient of every term, exactly (IEEE equality) as the
    # oracle forms it per term
    row, col = lib.dump_coefficients(0)
    cid = (l[:, 2] * 32 + l[:, 3]) * 2 + (l[:, 4] > 0)
    lc = np.where(l[:, 5] == 0, row[cid], col[cid])
    oc = ot["coef"][keep][oi]
    assert np.all(lc.real == oc.real) and np.all(lc.imag == oc.imag)
    assert oracle.errors() == 0


@pytest.mark.parametrize("key", ["w1", "w2", "w3"])
def test_workload_tables_bit_exact(key):
    w = W.WORKLOADS[key]
    bath = _oracle_bath(w)
    N = w["N"]
    sa = oracle.SA(N, len(bath["c"]), w["L"], bath, w["detuning"], w["gsn"] / np.sqrt(N), w["kappa"])
    lib = S.Heom(S.params_from(w), host_only=True)
    a, b = lib.dump_patterns(0), sa.patterns()
    for k in ("tier", "r", "G", "h", "var_off", "cat_off", "ids", "cat_id", "cat_M"):
        assert np.array_equal(a[k], b[k]), k
    assert lib.info(0)["n_terms"] == sa.terms()["var"].size - int(
        ((sa.var_labels()["kind"][sa.terms()["var"]] == 3) & (sa.terms()["dir"] == 1)).sum())


def test_batch_offsets_and_counts():
    """A batch is the instances' tables concatenated; per-instance counts
    equal the stand-alone counts and offsets are prefix sums."""
    ws = W.batch_w4(12)
    ps = [S.params_from(w) for w in ws]
    h = S.Heom(ps, precision=S.SA_FP32_AUX, host_only=True)
    off = 0
    for i, p in enumerate(ps):
        c = S.counts(p)
        assert h.var_offset(i) == off
        assert h.info(i)["n_vars"] == c["n_vars"]
        off += c["n_vars"]
    assert h.n_vars == off
    side = (off * 8 + 255) // 256 * 256
    assert h.state_bytes == side + 12 * 32 * 16  # 32 FP64 slots per instance


def test_saturation_in_library():
    """Eqs. first-saturation / second-saturation hold for the library counts."""
    bath = _generic_bath(2, 1)
    L = 5
    npat = [S.counts(S.make_params(N, 2, L, bath))["n_patterns"] for N in range(1, L + 5)]
    nvar = [S.counts(S.make_params(N, 2, L, bath))["n_vars"] for N in range(1, L + 5)]
    assert npat[L - 2] < npat[L - 1] == npat[-1]          # index N-1
    assert nvar[L] < nvar[L + 1] == nvar[-1]


@pytest.mark.parametrize("bad", [dict(N=0), dict(m=0), dict(m=9), dict(L=-1), dict(L=31), dict(d=4), dict(d=-1),
                                 dict(N=2, d=3), dict(reserved=1)])
def test_invalid_arguments_rejected(bad):
    args = dict(N=3, m=1, L=2, d=0, reserved=0)
    args.update(bad)
    bath = {"c": np.ones(8) * 0.1, "cc": np.ones(8) * 0.1, "nu": np.ones(8)}
    p = S.make_params(args["N"], min(max(args["m"], 1), 8), args["L"], bath)
    p.m, p.d, p.reserved = args["m"], args["d"], args["reserved"]
    with pytest.raises(S.SaHeomError) as e:
        S.Heom(p, host_only=True)
    assert e.value.code == -1


def test_zero_coefficient_rejected():
    bath = {"c": np.array([0j]), "cc": np.array([0j]), "nu": np.array([1.0])}
    with pytest.raises(S.SaHeomError):
        S.Heom(S.make_params(3, 1, 2, bath), host_only=True)
    bath = {"c": np.array([np.nan + 0j]), "cc": np.array([0.1 + 0j]), "nu": np.array([1.0])}
    with pytest.raises(S.SaHeomError):
        S.Heom(S.make_params(3, 1, 2, bath), host_only=True)


def test_host_only_handle_refuses_device_calls():
    bath = {"c": np.array([0.1 + 0j]), "cc": np.array([0.1 + 0j]), "nu": np.array([1.0])}
    h = S.Heom(S.make_params(3, 1, 2, bath), host_only=True)
    with pytest.raises(S.SaHeomError) as e:
        h.step(0, 0.1, stream=0)
    assert e.value.code == -7


def test_representatives_handle_structure():
    """sa_heom_build_representatives: the five representative hierarchies of
    one parameter set (Table tab:representative-initial-operators) as a batch
    with d = 0, 1, 1, 1, 2 -- four for N = 1 -- each instance the same tables
    as a stand-alone build with that d; d != 0 in the input is refused."""
    bath = _generic_bath(2, 5)
    for N in (1, 2, 7):
        p = S.make_params(N, 2, 3, bath, detuning=0.1, g=0.2, kappa=0.01, term=0.002)
        h = S.Heom(p, host_only=True, representatives=True)
        ds = [0, 1, 1, 1, 2] if N >= 2 else [0, 1, 1, 1]
        assert h.count == len(ds) and [q.d for q in h.params] == ds
        for i, d in enumerate(ds):
            c = S.counts(S.make_params(N, 2, 3, bath, detuning=0.1, g=0.2, kappa=0.01, term=0.002, d=d))
            assert h.info(i)["n_vars"] == c["n_vars"] and h.info(i)["n_patterns"] == c["n_patterns"]
            a = h.dump_patterns(i)
            sa = oracle.SA(N, 2, 3, bath, 0.1, 0.2, 0.01, term=0.002, d=d)
            b = sa.patterns()
            assert np.array_equal(a["ids"], b["ids"]) and np.array_equal(a["var_off"], b["var_off"])
    with pytest.raises(S.SaHeomError) as e:
        S.Heom(S.make_params(3, 2, 3, bath, d=1), host_only=True, representatives=True)
    assert e.value.code == -1


def test_new_entry_points_refuse_host_only_handles():
    """sa_heom_init_physical, sa_heom_init_representatives and
    sa_heom_reconstruct_dense need a device handle (SA_ERR_STATE, -7);
    reconstruction also needs a representatives handle."""
    import ctypes

    bath = _generic_bath(1, 2)
    h = S.Heom(S.make_params(3, 1, 2, bath), host_only=True, representatives=True)
    L = S.lib()
    buf = np.zeros(2 * S.PHYS_SLOTS * h.count)
    assert L.sa_heom_init_physical(h._h, buf.ctypes.data_as(ctypes.c_void_p), ctypes.c_void_p(16), None) == -7
    assert L.sa_heom_init_representatives(h._h, ctypes.c_void_p(16), None) == -7
    assert L.sa_heom_reconstruct_dense(h._h, ctypes.c_void_p(16), ctypes.c_void_p(32), ctypes.c_void_p(48),
                                       None) == -7


def test_adjoint_shortcut_needs_a_conjugate_bath():
    """SA_BUILD_ADJOINT_REPS is refused unless every nu_k is real and
    c-check_k = conj(c_k) (Eq. adjoint-preservation); accepted, it leaves the
    |c><e_1| propagation out of the batch."""
    c = np.array([0.3 + 0.1j, 0.2 - 0.05j])
    good = {"c": c, "cc": c.conj(), "nu": np.array([0.5 + 0j, 0.9 + 0j])}
    h5 = S.Heom(S.make_params(4, 2, 3, good, g=0.1), host_only=True, representatives=True)
    h4 = S.Heom(S.make_params(4, 2, 3, good, g=0.1), host_only=True, representatives=True, adjoint=True)
    assert (h5.count, h4.count) == (5, 4)
    assert h4.n_vars == h5.n_vars - h5.info(2)["n_vars"]
    for bad in [dict(good, nu=np.array([0.5 + 0.1j, 0.9 + 0j])), dict(good, cc=c.conj() * 1.01)]:
        with pytest.raises(S.SaHeomError) as e:
            S.Heom(S.make_params(4, 2, 3, bad, g=0.1), host_only=True, representatives=True, adjoint=True)
        assert e.value.code == -1
