"""The packed device layout (SA_BUILD_PACK_INSTANCES) and the pack kernel's
tables, checked on the CPU.

A host-only handle builds the same packs, layout and pack-item blobs the
device uses.  The layout is checked to be a bijection of (instance, variable)
onto the state's elements with the documented interleaving; the right-hand
side is evaluated from the blobs in numpy the way the pack kernel does --
pattern by pattern, Z with the sum of Eq. HZ, the grouped sums R_q and C_q
(Eqs. grouped-row-sum, grouped-column-sum) for X_q and Y_q, two reads for
P_q, S_{q,r} and T_q, the diagonal, and the blob's hierarchy terms with the
lane instance's coefficient slots -- and compared with the oracle's.
"""
import numpy as np
import pytest

import oracle
import paper_2608_20657_b300 as S
from tests.test_lists import PACK_UNIT, _eval_lists, _generic_bath, _layout, _slot_coefficients

A16 = lambda b: (b + 15) // 16 * 16
PAT = np.dtype([("var_rel", "<u2"), ("cat_rel", "<u2"), ("G", "u1"), ("tier", "u1"), ("islot", "<u2")])


def _batch(seed=5):
    """Templates of 35 (a pack of 32, three members left unpacked), 20 and 17
    instances (one pack each), and two singletons.  Members of a template share m, L, d and the decay rates nu_k
    and are saturated (N > L + d + 1); their c_k, c-check_k, N, g, detuning,
    loss and terminator differ."""
    rng = np.random.default_rng(seed)
    specs = []
    for (m, L, d, K) in [(1, 3, 0, 35), (2, 4, 0, 20), (1, 4, 1, 17)]:
        nu = _generic_bath(m, 100 + m * 10 + L)["nu"]
        for _ in range(K):
            b = _generic_bath(m, int(rng.integers(1 << 30)))
            b["nu"] = nu
            N = int(rng.integers(L + d + 3, L + d + 40))
            specs.append((N, m, L, d, b, dict(detuning=float(rng.uniform(-0.1, 0.1)), g=float(rng.uniform(0.05, 0.3)),
                                              kappa=float(rng.uniform(0, 0.05)), term=float(rng.uniform(0, 0.02)))))
    specs.append((3, 2, 3, 0, _generic_bath(2, 77), dict(detuning=0.02, g=0.1, kappa=0.01, term=0.0)))
    specs.append((4, 1, 6, 1, _generic_bath(1, 78), dict(detuning=0.0, g=0.2, kappa=0.0, term=0.01)))
    order = rng.permutation(len(specs))  # members of a template interleaved with others
    return [specs[i] for i in order]


def _handle(specs, precision, pack=True):
    ps = [S.make_params(N, m, L, b, d=d, **kw) for (N, m, L, d, b, kw) in specs]
    return S.Heom(ps, precision=precision, host_only=True, pack=pack)


def test_pack_layout_is_an_interleaved_bijection():
    specs = _batch()
    h = _handle(specs, S.SA_FP64)
    P = h.dump_packs()
    assert len(P["packs"]) == 3  # 35 -> 32 (three left unpacked), 20, 17
    assert sorted(int(n) for n in P["packs"][:, 1]) == [17, 20, 32]
    seen = np.zeros(h.n_vars, np.int64)
    packed = set(int(i) for i in P["lanes"])
    for i in range(h.count):
        nv = (h.var_offset(i + 1) if i + 1 < h.count else h.n_vars) - h.var_offset(i)
        e = np.array([h.state_index(i, v) for v in range(nv)])
        seen[e] += 1
        if i not in packed:  # contiguous (though not at its canonical offset)
            assert np.array_equal(e, e[0] + np.arange(nv))
    assert np.all(seen == 1)
    for base, n, cbase, lane0 in P["packs"]:
        members = P["lanes"][lane0:lane0 + n]
        assert list(members) == sorted(members)  # lanes in instance order
        nv = h.info(int(members[0]))["n_vars"]
        for j, i in enumerate(members):
            assert h.info(int(i))["n_vars"] == nv
            assert h.state_index(int(i), 0) == base + j
            assert h.state_index(int(i), nv - 1) == base + (nv - 1) * n + j
    # the unpacked handle keeps the canonical layout; the hashes differ
    u = _handle(specs, S.SA_FP64, pack=False)
    assert len(u.dump_packs()["packs"]) == 0
    assert all(u.state_index(i, 0) == u.var_offset(i) for i in range(u.count))
    assert u.config_hash() != h.config_hash()


def _pack_layout(np_, ncat, nl, nterm, nw, sz):
    L = {"pat": 16}
    L["pd"] = L["pat"] + A16(np_ * 8)
    L["cM"] = L["pd"] + A16(np_ * 2 * sz)
    L["vrec"] = L["cM"] + A16(ncat * sz)
    L["tgt"] = L["vrec"] + nl * 16
    L["tsl"] = L["tgt"] + A16(nterm * 4)
    L["wab"] = L["tsl"] + A16(nterm * 2)
    L["bytes"] = L["wab"] + A16(nw * 8)
    return L


def _eval_packs(h, specs, sas, x, out, precision):
    """Pack units of the dumped tables, evaluated lane by lane as the pack
    kernel does -- records in their three phases, each variable first adding
    its weighted value to the grouped sums it enters, then its derivative
    from operands, diagonal and terms -- into `out` (canonical order).  The
    phase order is checked to make every sum complete before it is read."""
    L = h.dump_lists()
    P = h.dump_packs()
    items, blobs = L["items"], P["blobs"]
    sz, ft = (8, np.float64) if precision == S.SA_FP64 else (4, np.float32)
    voff = [h.var_offset(i) for i in range(h.count)]
    baths = [s[4] for s in specs]
    coefs = [_slot_coefficients(b, s[2]) for b, s in zip(baths, specs)]
    pats = {}
    covered = np.zeros(x.size, np.int64)
    n_units = 0
    for c, k in L["units"]:
        if not int(c) & PACK_UNIT:
            continue
        n_units += 1
        p0, np_, v0, nv, c0, ncat, r0, nl, b16, bb = (int(v) for v in items[int(c) & ~PACK_UNIT])
        assert r0 == 0xffffffff
        blob = blobs[16 * b16:16 * b16 + bb]
        nw = int(np.frombuffer(blob[:4].tobytes(), "<u4")[0])
        B0 = _pack_layout(np_, ncat, nl, 0, 0, sz)
        vrec = np.frombuffer(blob[B0["vrec"]:B0["vrec"] + 16 * nl].tobytes(), "<u4").astype(np.int64).reshape(-1, 4)
        cnts = vrec[:, 1] >> 26
        starts = (vrec[:, 1] >> 10) & 65535
        nterm = int(cnts.sum())
        assert np.array_equal(starts, np.concatenate([[0], np.cumsum(cnts)[:-1]]))  # terms one variable after another
        B = _pack_layout(np_, ncat, nl, nterm, nw, sz)
        assert B["bytes"] <= bb
        wab = np.frombuffer(blob[B["wab"]:B["wab"] + 8 * nw].tobytes(), "<i4").astype(np.int64).reshape(-1, 2)
        assert len({(int(a_), int(b_)) for a_, b_ in wab}) == nw  # distinct weights
        ph = np.frombuffer(blob[B["pat"]:B["pat"] + 8 * np_].tobytes(), PAT)
        pd = np.frombuffer(blob[B["pd"]:B["pd"] + 2 * sz * np_].tobytes(), ft).astype(float).view(complex)
        cM = np.frombuffer(blob[B["cM"]:B["cM"] + sz * ncat].tobytes(), ft).astype(float)
        tgt = np.frombuffer(blob[B["tgt"]:B["tgt"] + 4 * nterm].tobytes(), "<u4").astype(np.int64)
        tsl = np.frombuffer(blob[B["tsl"]:B["tsl"] + 2 * nterm].tobytes(), "<u2").astype(np.int64)
        nslot = 2 * ncat + np_
        # phase of every record from its class: 0 S T / 4 P, then 1 X / 2 Y, then 3 Z
        cls_all = (vrec[:, 0] >> 22) & 7
        phase = np.select([np.isin(cls_all, [0, 4]), np.isin(cls_all, [1, 2])], [0, 1], 2)
        assert np.all(np.diff(phase) >= 0)
        for q in range(3):
            ls = vrec[phase == q, 1] & 1023
            assert np.all(np.diff(ls) > 0)  # canonical order within a phase
        base, n, cbase, lane0 = (int(v) for v in P["packs"][int(k)])
        for lane in range(n):
            i = int(P["lanes"][lane0 + lane])
            if i not in pats:
                pats[i] = h.dump_patterns(i)
            pt, sa, (N, m, Lh, d, b, kw) = pats[i], sas[i], specs[i]
            cf, vb = coefs[i], voff[i]
            vec = sa.vectors().astype(float)
            nu = np.asarray(b["nu"])
            xi = x[vb + v0:vb + v0 + nv]  # the item's variables of this lane's instance
            Mall = np.where(cM > 0, cM, N + cM)
            gam = np.zeros(np_, complex)
            for jj in range(np_):
                e = ph[jj]
                G, cr = int(e["G"]), int(e["cat_rel"])
                p = p0 + jj
                assert G == int(pt["G"][p]) and int(pt["var_off"][p]) == v0 + int(e["var_rel"])
                gam[jj] = sum(vec[v % len(vec)] @ nu for v in pt["ids"][p] if v >= 0)
                np.testing.assert_allclose(pd[jj], -gam[jj], rtol=2e-7 if sz == 4 else 1e-15, atol=1e-300)
                catM = pt["cat_M"][pt["cat_off"][p]:pt["cat_off"][p + 1]]
                assert np.array_equal(Mall[cr:cr + G], catM.astype(float))
            sums = np.zeros(nslot + 1, complex)
            done = np.zeros(nslot + 1, np.int64)  # the phase that last wrote a slot
            for idx, (w, w1, wz, ww) in enumerate(vrec):
                w, l, u0, cnt = int(w), int(w1) & 1023, (int(w1) >> 10) & 65535, int(w1) >> 26
                a, bo, cls, jj = w & 2047, (w >> 11) & 2047, (w >> 22) & 7, (w >> 25) & 31
                ncon = (2, 1, 0)[phase[idx]]  # P, T, S enter two sums, X and Y one, Z none
                for con in (int(wz), int(ww))[:ncon]:
                    slot, kw_ = con & 2047, con >> 11
                    assert kw_ < nw
                    aa, bb = (int(v_) for v_ in wab[kw_])
                    sums[slot] += (aa + bb * N) * xi[l]
                    done[slot] = max(done[slot], phase[idx])
                for opc in (a, bo):
                    if opc >= nv:  # a sum read: written only in an earlier phase
                        assert done[opc - nv] < phase[idx] or opc - nv == nslot
                ops = np.concatenate([xi, sums])
                lossf = [0.0, 0.5, 0.5, 1.0, 0.0][cls]
                dim = [0.0, -kw["detuning"], kw["detuning"], 0.0, 0.0][cls]
                wt = [2.0, 1.0, 1.0, 0.0, 0.0][cls]
                g0 = gam[jj]
                diag = -(g0.real + lossf * kw["kappa"] + wt * kw["term"]) + 1j * (dim - g0.imag)
                u1 = u0 + cnt
                dv = diag * xi[l] - 1j * kw["g"] * (ops[a] - ops[bo]) + np.sum(cf[tsl[u0:u1]] * x[vb + tgt[u0:u1]])
                out[vb + v0 + l] = dv
                covered[vb + v0 + l] += 1
    assert covered.max() <= 1
    return n_units


@pytest.mark.parametrize("precision", [S.SA_FP64, S.SA_FP32_AUX])
def test_pack_tables_reproduce_oracle_rhs(precision):
    specs = _batch()
    sas = [oracle.SA(N, m, L, b, d=d, **kw) for (N, m, L, d, b, kw) in specs]
    h = _handle(specs, precision)
    h.set_kernel(S.SA_KERNEL_LISTS)
    rng = np.random.default_rng(3)
    xs = [rng.standard_normal(sa.nvar) + 1j * rng.standard_normal(sa.nvar) for sa in sas]
    x = np.concatenate(xs)
    out = _eval_lists(h, sas, [s[4] for s in specs], x, range(len(sas)))  # the list units
    n_pack_units = _eval_packs(h, specs, sas, x, out, precision)
    assert n_pack_units > 0
    off = 0
    for i, sa in enumerate(sas):
        ref = sa.rhs(xs[i])
        g = out[off:off + sa.nvar]
        if precision == S.SA_FP32_AUX:
            n0 = int(sa.patterns()["var_off"][1])
            assert np.all(np.isnan(g[:n0]))
            g, ref = g[n0:], ref[n0:]
        assert not np.any(np.isnan(g)), i
        np.testing.assert_allclose(g, ref, rtol=0, atol=1e-12 * max(1.0, np.abs(ref).max()))
        off += sa.nvar
    assert oracle.errors() == 0


def test_packed_handle_refuses_other_kernels():
    h = _handle(_batch(), S.SA_FP32_AUX)
    with pytest.raises(S.SaHeomError) as e:
        h.set_kernel(S.SA_KERNEL_RECORDS)
    assert e.value.code == -2
    h.set_kernel(S.SA_KERNEL_LISTS)  # still usable


@pytest.mark.parametrize("precision", [S.SA_FP32_AUX, S.SA_FP64])
def test_pack_items_respect_the_budget(precision):
    """Every pack item's blob, grouped sums and (FP64) per-lane weight and
    diagonal tables fit the per-warp budget -- 6 KB in FP32, 12 KB in FP64 -- or the item
    holds one pattern, with at most 16 patterns."""
    h = _handle(_batch(), precision)
    h.set_kernel(S.SA_KERNEL_LISTS)
    L = h.dump_lists()
    n = 0
    blobs = h.dump_packs()["blobs"]
    cs, budget, wtab = (8, 6144, 0) if precision == S.SA_FP32_AUX else (16, 12288, 8)
    for it in L["items"]:
        if int(it[6]) == 0xffffffff:
            n += 1
            sums = (2 * int(it[5]) + int(it[1]) + 1) * 32 * cs
            nw = int(np.frombuffer(blobs[16 * int(it[8]):16 * int(it[8]) + 4].tobytes(), "<u4")[0])
            assert nw >= 1
            dtab = int(it[1]) * 5 * 32 * 2 * wtab  # (FP64) per-lane diagonal per pattern and class
            assert int(it[9]) + sums + nw * 32 * wtab + dtab <= budget or int(it[1]) == 1
            assert int(it[1]) <= 16
    assert n > 0
