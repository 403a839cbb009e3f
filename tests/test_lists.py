"""The term tables of the SA_KERNEL_LISTS and SA_KERNEL_ELL stage kernels,
checked on the CPU.

A host-only handle builds the same lists the device kernel reads.  Here they
are evaluated in numpy the way the kernel does -- per work item an operand
area (the item's stage-input slice, the grouped row and column sums R_q and
C_q of Eqs. grouped-row-sum / grouped-column-sum, the Z sums of Eq. HZ, a
zero), then for every lane variable
    dv = diag * v - i g (op[a] - op[b]) + sum_t coef[slot_t] * x[idx_t]
-- with the coefficients of Eqs. uvar-up / uvar-down written out from the
bath, and compared with the oracle's right-hand side.  The structure of the
lists is checked too: every variable once, rounds padded to their longest
list and no further, padding only with the zero slot.
"""
import numpy as np
import pytest

import oracle
import oracle.bath as OB
import paper_2608_20657_b300 as S
import workloads as W

ZERO_SLOT = 0
PACK_UNIT = 0x80000000


def _generic_bath(m, seed):
    rng = np.random.default_rng(seed)
    return {"c": rng.uniform(0.1, 0.5, m) + 1j * rng.uniform(-0.4, 0.4, m),
            "cc": rng.uniform(0.1, 0.5, m) + 1j * rng.uniform(-0.4, 0.4, m),
            "nu": rng.uniform(0.2, 1.2, m) + 1j * rng.uniform(-0.3, 0.3, m)}


def _slot_coefficients(bath, L):
    """Coefficient of every list slot of one instance: slot 0 zero, then for
    each channel k, occupation n = 0..L before the move and direction (lower,
    raise) the row, column and row + column coefficients side by side."""
    c, cc = np.asarray(bath["c"]), np.asarray(bath["cc"])
    out = np.zeros(1 + 6 * c.size * (L + 1), complex)
    for k in range(c.size):
        ac = abs(c[k])
        for n in range(L + 1):
            for up in (0, 1):
                if up:
                    row, col = -1j * np.sqrt((n + 1) * ac), 1j * np.sqrt((n + 1) * ac)
                else:
                    row, col = -1j * np.sqrt(n / ac) * c[k], 1j * np.sqrt(n / ac) * cc[k]
                s0 = 1 + ((k * (L + 1) + n) * 2 + up) * 3
                out[s0], out[s0 + 1], out[s0 + 2] = row, col, row + col
    return out


def _layout(G, M):
    """Local indices of the canonical layout of a pattern with multiplicities M."""
    X = lambda q: q
    Y = lambda q: G + q
    P = lambda q: 2 * G + q
    Sv = lambda q, r: 3 * G + 1 + (q - 1) * (G - 1) + (r - 1) - (1 if r > q else 0)
    tr = np.cumsum([0] + [1 if m >= 2 else 0 for m in M])
    T = lambda q: (G + 1) ** 2 + tr[q - 1]
    return X, Y, P, Sv, T


def _eval_lists(lib, sas, baths, x, insts):
    """Right-hand side of the batch from the dumped lists, work unit by work
    unit (a template item evaluated for one instance); NaN where no lane
    writes (the physical representative in SA_FP32_AUX mode)."""
    L = lib.dump_lists()
    R0, C0, Z0, ZZ = (int(v) for v in L["opz"])
    out = np.full(x.size, np.nan, complex)
    pats = [lib.dump_patterns(i) for i in range(len(sas))]
    voff = [lib.var_offset(i) for i in range(len(sas))]
    gams = []
    for i, (P, sa) in enumerate(zip(pats, sas)):
        vec = sa.vectors().astype(float)
        nu = np.asarray(baths[i]["nu"])
        gams.append([sum(vec[v % len(vec)] @ nu for v in P["ids"][p] if v >= 0)  # molecule 1: ids V + v
                     for p in range(P["G"].size)])
    coefs = [_slot_coefficients(b, sa.L) for b, sa in zip(baths, sas)]
    covered = np.zeros(x.size, np.int64)
    for c, inst in L["units"]:
        if int(c) & PACK_UNIT:  # pack units: tests/test_packs.py
            continue
        p0, np_, v0, nv, c0, ncat, r0, nl = (int(v) for v in L["items"][c][:8])
        inst = int(inst)
        P, vb, cf = pats[inst], voff[inst], coefs[inst]
        op = np.zeros(ZZ + 1, complex)
        op[:nv] = x[vb + v0:vb + v0 + nv]
        for j in range(np_):
            p = p0 + j
            G, M = int(P["G"][p]), P["cat_M"][P["cat_off"][p]:P["cat_off"][p + 1]]
            X, Y, Pv, Sv, T = _layout(G, M)
            xp = x[vb + P["var_off"][p]:]
            cb = int(P["cat_off"][p]) - c0
            zs = 0
            for q in range(1, G + 1):
                base = xp[Pv(q)] + ((M[q - 1] - 1) * xp[T(q)] if M[q - 1] >= 2 else 0)
                op[R0 + cb + q - 1] = base + sum(M[b - 1] * xp[Sv(q, b)] for b in range(1, G + 1) if b != q)
                op[C0 + cb + q - 1] = base + sum(M[b - 1] * xp[Sv(b, q)] for b in range(1, G + 1) if b != q)
                zs += M[q - 1] * (xp[X(q)] - xp[Y(q)])
            op[Z0 + j] = zs
        seen = []
        for rho, i0 in enumerate(range(0, nl, 32)):
            ra, rb = int(L["rbase"][r0 + rho]), int(L["rbase"][r0 + rho + 1])
            rows = np.arange(ra, rb)
            counts = []
            for u in range(32):
                e = rows * 32 + u
                idx, slot = L["tidx"][e].astype(np.int64), L["tcid"][e].astype(np.int64)
                real = slot != ZERO_SLOT
                # padding only after the variable's own terms
                n = int(real.sum())
                assert np.all(real[:n]) and not np.any(real[n:])
                if i0 + u >= nl:
                    assert n == 0
                    continue
                counts.append(n)
                w0, w1 = int(L["lvd"][32 * r0 + i0 + u]), int(L["lvj"][32 * r0 + i0 + u])
                l, a, b = w0 & 1023, (w0 >> 10) & 2047, w0 >> 21
                j, cls = w1 & 31, w1 >> 5
                p = p0 + j
                vg = vb + v0 + l
                assert P["var_off"][p] <= v0 + l < P["var_off"][p + 1]
                sa_p = sas[inst].params
                g, det, kap = sa_p.g, sa_p.detuning, sa_p.kappa
                # classes: 0 S T, 1 X, 2 Y, 3 Z, 4 P
                lossf = [0.0, 0.5, 0.5, 1.0, 0.0][cls]
                dim = [0.0, -det, det, 0.0, 0.0][cls]
                wt = [2.0, 1.0, 1.0, 0.0, 0.0][cls]  # terminator weight
                gam = gams[inst][p]
                diag = -(gam.real + lossf * kap + wt * sa_p.term) + 1j * (dim - gam.imag)
                dv = diag * op[l] - 1j * g * (op[a] - op[b])
                dv += np.sum(cf[slot[:n]] * x[vb + idx[:n]])
                out[vg] = dv
                covered[vg] += 1
                seen.append(l)
            # a round is as long as its longest list, and lists are sorted
            assert counts and max(counts) == rb - ra and counts == sorted(counts, reverse=True)
        assert len(seen) == len(set(seen)) == nl
    # every variable of every instance is written by exactly one lane, except
    # the physical representatives the FP64 kernel integrates in SA_FP32_AUX
    assert covered.max() <= 1
    return out


def _case(params_list, baths, sas, precision, chunk=None):
    lib = S.Heom(params_list, precision=precision, host_only=True)
    if chunk:
        lib.set_tuning(chunk=chunk)
    lib.set_kernel(S.SA_KERNEL_LISTS)
    assert lib.tuning()["kernel"] == S.SA_KERNEL_LISTS
    rng = np.random.default_rng(11)
    xs = [rng.standard_normal(sa.nvar) + 1j * rng.standard_normal(sa.nvar) for sa in sas]
    x = np.concatenate(xs)
    got = _eval_lists(lib, sas, baths, x, range(len(sas)))
    off = 0
    for i, sa in enumerate(sas):
        ref = sa.rhs(xs[i])
        g = got[off:off + sa.nvar]
        n_rho0 = int(sa.patterns()["var_off"][1])  # the physical representative's variables
        if precision == S.SA_FP32_AUX:
            # the physical representative is integrated by the FP64 kernel
            assert np.all(np.isnan(g[:n_rho0]))
            g, ref = g[n_rho0:], ref[n_rho0:]
        assert not np.any(np.isnan(g))
        np.testing.assert_allclose(g, ref, rtol=0, atol=1e-12 * max(1.0, np.abs(ref).max()))
        off += sa.nvar
    assert oracle.errors() == 0


@pytest.mark.parametrize("precision", [S.SA_FP64, S.SA_FP32_AUX])
@pytest.mark.parametrize("N,m,L", [(1, 1, 3), (2, 1, 3), (3, 2, 3), (10, 2, 6), (12, 3, 4), (7, 4, 3), (2, 2, 6)])
@pytest.mark.parametrize("d", [0, 1, 2])
def test_lists_reproduce_oracle_rhs(N, m, L, precision, d):
    if d > N:
        pytest.skip("d <= N")
    bath = _generic_bath(m, N + 7 * m + L)
    kw = dict(detuning=0.1, g=0.2, kappa=0.05, term=0.013, d=d)
    sa = oracle.SA(N, m, L, bath, **kw)
    _case([S.make_params(N, m, L, bath, **kw)], [bath], [sa], precision)


def test_lists_batch_and_chunk():
    """A batch of unlike instances, with a larger work-item capacity; the
    second and third keep one and two molecules distinguished."""
    specs = [(3, 1, 4, 1), (9, 2, 3, 2), (5, 3, 3, 3)]
    sas, baths, ps = [], [], []
    for N, m, L, seed in specs:
        b = _generic_bath(m, seed)
        kw = dict(detuning=0.03 * seed, g=0.1 / seed, kappa=0.01 * seed, d=seed - 1)
        sas.append(oracle.SA(N, m, L, b, **kw))
        baths.append(b)
        ps.append(S.make_params(N, m, L, b, **kw))
    _case(ps, baths, sas, S.SA_FP32_AUX, chunk=256)
    _case(ps, baths, sas, S.SA_FP64, chunk=64)


def _eval_ell(lib, sas, baths, x):
    """Right-hand side of the batch from the dumped ELL tables."""
    E = lib.dump_ell()
    pats = [lib.dump_patterns(i) for i in range(len(sas))]
    voff = [lib.var_offset(i) for i in range(len(sas))]
    labs = [sa.var_labels() for sa in sas]
    gvar, ginst, gG, gM, ggam = [], [], [], [], []
    for i, (P, sa) in enumerate(zip(pats, sas)):
        vec = sa.vectors().astype(float)
        nu = np.asarray(baths[i]["nu"])
        for p in range(P["G"].size):
            gvar.append(voff[i] + P["var_off"][p])
            ginst.append(i)
            gG.append(P["G"][p])
            gM.append(P["cat_M"][P["cat_off"][p]:P["cat_off"][p + 1]])
            ggam.append(sum(vec[v % len(vec)] @ nu for v in P["ids"][p] if v >= 0))
    gvar.append(x.size)
    coefs = [_slot_coefficients(b, sa.L) for b, sa in zip(baths, sas)]
    out = np.zeros(x.size, complex)
    nw = E["wpat"].size
    assert nw == (x.size + 31) // 32
    for v in range(x.size):
        w, lane = v >> 5, v & 31
        e = int(E["vword"][v])
        p = int(E["wpat"][w]) + (e & 31)
        kind, q, r, trq = (e >> 5) & 7, (e >> 8) & 31, (e >> 13) & 31, (e >> 18) & 31
        assert gvar[p] <= v < gvar[p + 1]
        inst = ginst[p]
        lab = labs[inst]
        lv = v - voff[inst]
        assert (kind, q, r) == (lab["kind"][lv], lab["q"][lv], lab["r"][lv] if kind == 4 else 0)
        G, M = gG[p], gM[p]
        X, Y, P, Sv, T = _layout(G, M)
        assert trq == (T(q) - (G + 1) ** 2 if q and M[q - 1] >= 2 else 31)
        xp = x[gvar[p]:]
        if kind in (3, 4, 5):
            a, b = xp[Y(r if kind == 4 else q)], xp[X(q)]
        elif kind == 0:
            a, b = sum(M[c - 1] * (xp[X(c)] - xp[Y(c)]) for c in range(1, G + 1)), 0
        else:
            s = xp[P(q)] + ((M[q - 1] - 1) * xp[T(q)] if M[q - 1] >= 2 else 0)
            if kind == 1:
                a, b = xp[0], s + sum(M[c - 1] * xp[Sv(q, c)] for c in range(1, G + 1) if c != q)
            else:
                a, b = s + sum(M[c - 1] * xp[Sv(c, q)] for c in range(1, G + 1) if c != q), xp[0]
        sp = sas[inst].params
        lossf = {0: 1.0, 1: 0.5, 2: 0.5}.get(kind, 0.0)
        wt = {1: 1.0, 2: 1.0, 4: 2.0, 5: 2.0}.get(kind, 0.0)  # terminator weight
        dim = {1: -sp.detuning, 2: sp.detuning}.get(kind, 0.0)
        diag = -(ggam[p].real + lossf * sp.kappa + wt * sp.term) + 1j * (dim - ggam[p].imag)
        rows = np.arange(int(E["rbase"][w]), int(E["rbase"][w + 1]))
        idx, slot = E["tidx"][rows * 32 + lane].astype(np.int64), E["tcid"][rows * 32 + lane].astype(np.int64)
        real = slot != ZERO_SLOT
        n = int(real.sum())
        assert np.all(real[:n]) and not np.any(real[n:])
        out[v] = diag * x[v] - 1j * sp.g * (a - b) + np.sum(coefs[inst][slot[:n]] * x[idx[:n]])
    # every warp's rows are as many as its longest list
    for w in range(nw):
        rows = np.arange(int(E["rbase"][w]), int(E["rbase"][w + 1]))
        if rows.size:
            assert np.any(E["tcid"][rows[-1] * 32:(rows[-1] + 1) * 32] != ZERO_SLOT)
    return out


@pytest.mark.parametrize("precision", [S.SA_FP64, S.SA_FP32_AUX])
@pytest.mark.parametrize("N,m,L", [(1, 1, 3), (3, 2, 3), (10, 2, 6), (7, 4, 3)])
@pytest.mark.parametrize("d", [0, 1, 3])
def test_ell_reproduces_oracle_rhs(N, m, L, precision, d):
    if d > N:
        pytest.skip("d <= N")
    bath = _generic_bath(m, N + 7 * m + L)
    kw = dict(detuning=0.1, g=0.2, kappa=0.05, term=0.013, d=d)
    sa = oracle.SA(N, m, L, bath, **kw)
    lib = S.Heom(S.make_params(N, m, L, bath, **kw), precision=precision, host_only=True)
    lib.set_kernel(S.SA_KERNEL_ELL)
    x = W.random_state(sa.nvar, seed=5)
    got = _eval_ell(lib, [sa], [bath], x)
    ref = sa.rhs(x)
    n0 = int(sa.patterns()["var_off"][1]) if precision == S.SA_FP32_AUX else 0  # no lists for the FP64 rho_0
    if n0:
        # without its hierarchy terms, the physical representative differs
        assert np.max(np.abs(got[:n0] - ref[:n0])) > 1e-6
    np.testing.assert_allclose(got[n0:], ref[n0:], rtol=0, atol=1e-12 * max(1.0, np.abs(ref).max()))


def test_ell_batch():
    specs = [(3, 1, 4, 1), (9, 2, 3, 2), (5, 3, 3, 3)]
    sas, baths, ps = [], [], []
    for N, m, L, seed in specs:
        b = _generic_bath(m, seed)
        kw = dict(detuning=0.03 * seed, g=0.1 / seed, kappa=0.01 * seed)
        sas.append(oracle.SA(N, m, L, b, **kw))
        baths.append(b)
        ps.append(S.make_params(N, m, L, b, **kw))
    lib = S.Heom(ps, precision=S.SA_FP64, host_only=True)
    lib.set_kernel(S.SA_KERNEL_ELL)
    xs = [W.random_state(sa.nvar, seed=i) for i, sa in enumerate(sas)]
    got = _eval_ell(lib, sas, baths, np.concatenate(xs))
    off = 0
    for sa, x in zip(sas, xs):
        ref = sa.rhs(x)
        np.testing.assert_allclose(got[off:off + sa.nvar], ref, rtol=0, atol=1e-12 * np.abs(ref).max())
        off += sa.nvar


def test_lists_state_errors():
    """Dumps exist only for host-only handles whose tables were built by
    sa_heom_set_kernel; an unknown variant is rejected and changes nothing."""
    bath = _generic_bath(1, 3)
    lib = S.Heom(S.make_params(2, 1, 3, bath), host_only=True)
    assert lib.tuning()["kernel"] == S.SA_KERNEL_LISTS
    for dump in (lib.dump_lists, lib.dump_ell):
        with pytest.raises(S.SaHeomError) as e:
            dump()
        assert e.value.code == -7
    with pytest.raises(S.SaHeomError) as e:
        lib.set_kernel(7)
    assert e.value.code == -1
    assert lib.tuning()["kernel"] == S.SA_KERNEL_LISTS
    lib.set_kernel(S.SA_KERNEL_ELL)
    with pytest.raises(S.SaHeomError) as e:
        lib.dump_lists()
    assert e.value.code == -7
    assert lib.dump_ell()["wpat"].size == (lib.n_vars + 31) // 32


def test_lists_share_templates():
    """Instances with identical tables -- the same m, L, d and decay rates, and
    N >= L + d + 2 so that the hierarchy's structure no longer depends on N --
    share one template: its items and lists are built once, and each instance
    gets its own work units with its own N (zero-category multiplicity N - r),
    g, detuning, loss, terminator and coefficients.  Instances below
    saturation (N = 3 < L + 2 here) and other baths get templates of their
    own.  Every instance's right-hand side matches the oracle's."""
    specs = [(12, 0.10, 0.020), (30, 0.04, 0.000), (7, 0.15, 0.010), (3, 0.08, 0.030), (64, 0.02, 0.005)]
    m, L = 2, 4
    bath = _generic_bath(m, 99)
    sas, baths, ps = [], [], []
    for N, g, kap in specs:
        kw = dict(detuning=0.3 * g, g=g, kappa=kap, term=0.7 * kap)
        sas.append(oracle.SA(N, m, L, bath, **kw))
        baths.append(bath)
        ps.append(S.make_params(N, m, L, bath, **kw))
    other = _generic_bath(m, 5)  # another bath: a template of its own
    sas.append(oracle.SA(40, m, L, other, g=0.05))
    baths.append(other)
    ps.append(S.make_params(40, m, L, other, g=0.05))
    for precision in (S.SA_FP64, S.SA_FP32_AUX):
        lib = S.Heom(ps, precision=precision, host_only=True)
        lib.set_kernel(S.SA_KERNEL_LISTS)
        Ld = lib.dump_lists()
        units = Ld["units"]
        reps = {}
        for c, inst in units:
            reps.setdefault(int(inst), set()).add(int(c))
        # the four saturated instances of the first bath read the same items
        assert reps[0] == reps[1] == reps[2] == reps[4]
        assert reps[3].isdisjoint(reps[0]) and reps[5].isdisjoint(reps[0])
        assert len(Ld["items"]) == len(reps[0] | reps[3] | reps[5])
        _case(ps, baths, sas, precision)
