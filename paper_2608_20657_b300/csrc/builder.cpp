// builder.cpp -- host construction of the symmetry-adapted hierarchy tables.
//
// For one instance (N, m, L, bath, system parameters):
//  1. local hierarchy vectors alpha in N0^m, |alpha| <= L (last paragraph of
//     Sec. IV: a molecule carries a whole vector that moves as a unit);
//  2. canonical occupation patterns (Eq. pattern-one generalised to vectors):
//     multisets of nonzero vectors with total norm <= L and at most N
//     members, enumerated tier by tier directly in canonical order;
//  3. occupation categories, multiplicities M_q (Eqs. Mq, M0), T-ranks
//     (Eq. h-Lambda) and the variable layout (Eq. uvar-count);
//  4. damping rates Gamma_Lambda (Eq. tier-damping);
//  5. connection records: for every (pattern, category, channel, raise /
//     lower) the canonical target (Eqs. canonical-target-plus/minus) and the
//     integer data that resolve the aligned accessor (Eq. aligned-accessor)
//     for every variable of the source category -- "record the source, the
//     target, the alignment, the multiplicity and the coefficient" of the
//     precomputed matrix-free right-hand side (Sec. IV.B.4);
//  6. the coefficient table of the hierarchy terms of Eqs. uvar-up and
//     uvar-down generalised to channel k as in Eq. scaled-HEOM.
// Every record is checked against the target's actual category vectors.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <unordered_map>

#include "sa_internal.h"

#ifdef _OPENMP
#include <omp.h>
#endif

namespace sa {

namespace {

// ---- local vectors ---------------------------------------------------------
bool vec_before(const uint8_t* a, const uint8_t* b, int m) {
    int na = 0, nb = 0;
    for (int k = 0; k < m; ++k) {
        na += a[k];
        nb += b[k];
    }
    if (na != nb) return na > nb;
    for (int k = 0; k < m; ++k)
        if (a[k] != b[k]) return a[k] > b[k];
    return false;
}

int64_t vcode(const uint8_t* a, int m, int L) {
    int64_t c = 0;
    for (int k = 0; k < m; ++k) c = c * (L + 1) + a[k];
    return c;
}

void build_vectors(HostInstance& hi) {
    const int m = hi.m, L = hi.L;
    // all nonzero tuples with |alpha| <= L, generated by odometer
    std::vector<std::vector<uint8_t>> vecs;
    std::vector<uint8_t> t(m, 0);
    while (true) {
        int s = 0;
        for (int k = 0; k < m; ++k) s += t[k];
        if (s > 0 && s <= L) vecs.push_back(t);
        int k = m - 1;
        while (k >= 0) {
            if (t[k] < L) {
                ++t[k];
                break;
            }
            t[k] = 0;
            --k;
        }
        if (k < 0) break;
    }
    std::sort(vecs.begin(), vecs.end(),
              [m](const std::vector<uint8_t>& a, const std::vector<uint8_t>& b) { return vec_before(a.data(), b.data(), m); });
    hi.V = int(vecs.size()) + 1;
    hi.Vtot = (hi.d + 1) * hi.V;
    hi.comp.assign(size_t(hi.Vtot) * m, 0);
    hi.norm.assign(hi.Vtot, 0);
    for (int v = 1; v < hi.V; ++v) {
        for (int k = 0; k < m; ++k) {
            hi.comp[size_t(v) * m + k] = vecs[v - 1][k];
            hi.norm[v] += vecs[v - 1][k];
        }
    }
    // the distinguished molecules' copies, zero vector included
    for (int v = hi.V; v < hi.Vtot; ++v) {
        std::memcpy(&hi.comp[size_t(v) * m], &hi.comp[size_t(v % hi.V) * m], m);
        hi.norm[v] = hi.norm[v % hi.V];
    }
    int64_t total = 1;
    for (int k = 0; k < m; ++k) total *= (L + 1);
    hi.lut.assign(total, -1);
    for (int v = 0; v < hi.V; ++v) hi.lut[vcode(&hi.comp[size_t(v) * m], m, L)] = v;
}

// id of alpha +/- e_k, -1 outside the set; a distinguished molecule's
// vectors stay among its own ids
int shift_vec(const HostInstance& hi, int id, int k, int dir) {
    uint8_t t[SA_HEOM_MAXM];
    std::memcpy(t, &hi.comp[size_t(id) * hi.m], hi.m);
    int v = int(t[k]) + dir;
    if (v < 0 || v > hi.L) return -1;
    t[k] = uint8_t(v);
    const int w = hi.lut[vcode(t, hi.m, hi.L)];
    return w >= 0 ? (id / hi.V) * hi.V + w : w;
}

// ---- pattern enumeration ---------------------------------------------------
struct Enum {
    HostInstance& hi;
    std::vector<uint32_t> cur;
    int maxr;
    std::vector<int> first_with_norm_le;  // smallest id whose norm <= n
    void dfs(int start, int remaining, int tier) {
        if (remaining == 0) {
            hi.ids.insert(hi.ids.end(), cur.begin(), cur.end());
            hi.id_off.push_back(uint32_t(hi.ids.size()));
            hi.tier.push_back(uint8_t(tier));
            return;
        }
        if (int(cur.size()) >= maxr) return;
        int v0 = std::max(start, first_with_norm_le[remaining]);
        for (int v = v0; v < hi.V; ++v) {
            cur.push_back(uint32_t(v));
            dfs(v, remaining - hi.norm[v], tier);
            cur.pop_back();
        }
    }
};

// open-addressing map from an id sequence to its pattern index
struct PatMap {
    const HostInstance* hi;
    std::vector<uint32_t> slot;  // pattern + 1, 0 = empty
    uint64_t mask = 0;
    static uint64_t hash(const uint32_t* a, int r) {
        uint64_t h = 0x9e3779b97f4a7c15ull ^ uint64_t(r);
        for (int i = 0; i < r; ++i) {
            h ^= uint64_t(a[i]) + 0x9e3779b97f4a7c15ull + (h << 6) + (h >> 2);
            h *= 0xbf58476d1ce4e5b9ull;
        }
        return h ^ (h >> 31);
    }
    void build(const HostInstance& H) {
        hi = &H;
        uint64_t cap = 16;
        while (cap < uint64_t(H.P) * 2) cap <<= 1;
        slot.assign(cap, 0);
        mask = cap - 1;
        for (int64_t i = 0; i < H.P; ++i) {
            const uint32_t* a = &H.ids[H.id_off[i]];
            int r = int(H.id_off[i + 1] - H.id_off[i]);
            uint64_t s = hash(a, r) & mask;
            while (slot[s]) s = (s + 1) & mask;
            slot[s] = uint32_t(i + 1);
        }
    }
    int64_t find(const uint32_t* a, int r) const {
        uint64_t s = hash(a, r) & mask;
        while (slot[s]) {
            int64_t i = int64_t(slot[s]) - 1;
            int ri = int(hi->id_off[i + 1] - hi->id_off[i]);
            if (ri == r && std::equal(a, a + r, &hi->ids[hi->id_off[i]])) return i;
            s = (s + 1) & mask;
        }
        return -1;
    }
};

}  // namespace

int build_instance(const sa_params& p, HostInstance& hi, std::string& err) {
    if (p.N < 1 || p.m < 1 || p.m > SA_HEOM_MAXM || p.L < 0 || p.L > SA_HEOM_MAXL || p.d < 0 ||
        p.d > SA_HEOM_MAXD || p.d > p.N || p.reserved != 0) {
        err = "N >= 1, 1 <= m <= 8, 0 <= L <= 30, 0 <= d <= min(3, N), reserved = 0 required";
        return SA_ERR_INVALID_ARG;
    }
    const double scal[4] = {p.detuning, p.g, p.kappa, p.term};
    for (double v : scal)
        if (!std::isfinite(v)) {
            err = "non-finite system parameter";
            return SA_ERR_INVALID_ARG;
        }
    for (int k = 0; k < p.m; ++k) {
        const double v[6] = {p.c_re[k], p.c_im[k], p.cc_re[k], p.cc_im[k], p.nu_re[k], p.nu_im[k]};
        for (double x : v)
            if (!std::isfinite(x)) {
                err = "non-finite bath coefficient";
                return SA_ERR_INVALID_ARG;
            }
        if (!(std::sqrt(p.c_re[k] * p.c_re[k] + p.c_im[k] * p.c_im[k]) > 0.0)) {
            err = "|c_k| = 0 makes the scaled hierarchy singular (Eq. scaled-ADO)";
            return SA_ERR_INVALID_ARG;
        }
    }
    hi = HostInstance();
    hi.p = p;
    hi.m = p.m;
    hi.L = p.L;
    hi.N = p.N;
    hi.d = p.d;
    const int m = hi.m, L = hi.L;
    build_vectors(hi);

    // patterns, tier by tier, each tier in canonical (lexicographic) order:
    // at most N - d nonzero vectors of the symmetrised molecules
    Enum en{hi, {}, int(std::min<int64_t>(L, p.N - p.d)), {}};
    en.first_with_norm_le.assign(L + 1, hi.V);
    for (int n = 0; n <= L; ++n) {
        for (int v = 1; v < hi.V; ++v)
            if (hi.norm[v] <= n) {
                en.first_with_norm_le[n] = v;
                break;
            }
    }
    hi.id_off.push_back(0);
    if (!hi.d) {
        for (int t = 0; t <= L; ++t) en.dfs(1, t, t);
    } else {
        // distinguished molecule j's id (j V + v, above every id of molecule
        // j - 1) closes each list in molecule order; the lists of one tier
        // are then sorted lexicographically
        std::vector<uint32_t> all_ids, scratch_off{0};
        std::vector<uint8_t> all_tier;
        int dv[SA_HEOM_MAXD] = {0};
        for (int t = 0; t <= L; ++t) {
            const size_t first = all_tier.size();
            // odometer over the distinguished molecules' vectors
            std::fill(dv, dv + hi.d, 0);
            while (true) {
                int dn = 0;
                for (int j = 0; j < hi.d; ++j) dn += hi.norm[dv[j]];
                if (dn <= t) {
                    const size_t before = hi.tier.size();
                    en.dfs(1, t - dn, t);
                    // dfs appended to hi.ids / id_off / tier: move them out,
                    // with the distinguished ids
                    for (size_t j = before; j < hi.tier.size(); ++j) {
                        all_ids.insert(all_ids.end(), hi.ids.begin() + hi.id_off[j],
                                       hi.ids.begin() + hi.id_off[j + 1]);
                        for (int q = 0; q < hi.d; ++q) all_ids.push_back(uint32_t((q + 1) * hi.V + dv[q]));
                        scratch_off.push_back(uint32_t(all_ids.size()));
                        all_tier.push_back(uint8_t(t));
                    }
                    hi.ids.resize(hi.id_off[before]);
                    hi.id_off.resize(before + 1);
                    hi.tier.resize(before);
                }
                int j = hi.d - 1;
                while (j >= 0 && ++dv[j] == hi.V) dv[j--] = 0;
                if (j < 0) break;
            }
            std::vector<size_t> ord(all_tier.size() - first);
            for (size_t j = 0; j < ord.size(); ++j) ord[j] = first + j;
            std::sort(ord.begin(), ord.end(), [&](size_t a, size_t b) {
                return std::lexicographical_compare(all_ids.begin() + scratch_off[a], all_ids.begin() + scratch_off[a + 1],
                                                    all_ids.begin() + scratch_off[b], all_ids.begin() + scratch_off[b + 1]);
            });
            for (size_t j : ord) {
                hi.ids.insert(hi.ids.end(), all_ids.begin() + scratch_off[j], all_ids.begin() + scratch_off[j + 1]);
                hi.id_off.push_back(uint32_t(hi.ids.size()));
                hi.tier.push_back(uint8_t(t));
            }
        }
    }
    hi.P = int64_t(hi.tier.size());

    // categories, multiplicities, layout, damping
    hi.G.resize(hi.P);
    hi.h.resize(hi.P);
    hi.cat_off.assign(hi.P + 1, 0);
    hi.var_off.assign(hi.P + 1, 0);
    hi.gamma_re.resize(hi.P);
    hi.gamma_im.resize(hi.P);
    for (int64_t i = 0; i < hi.P; ++i) {
        const uint32_t* a = &hi.ids[hi.id_off[i]];
        int r = int(hi.id_off[i + 1] - hi.id_off[i]);
        int G = 0;
        hi.cat_off[i] = uint32_t(hi.cat_vec.size());
        for (int j = 0; j < r; ++j) {
            if (j == 0 || a[j] != a[j - 1]) {
                hi.cat_vec.push_back(a[j]);
                hi.cat_M.push_back(1);
                ++G;
            } else {
                hi.cat_M.back() += 1;
            }
        }
        if (p.N - r >= 1) {
            hi.cat_vec.push_back(0);
            hi.cat_M.push_back(p.N - r);
            ++G;
        }
        if (G > kMaxG) {
            err = "more than 31 occupation categories in a pattern";
            return SA_ERR_UNSUPPORTED;
        }
        int h = 0;
        double gre = 0, gim = 0;
        for (int q = 0; q < G; ++q) {
            int64_t M = hi.cat_M[hi.cat_off[i] + q];
            hi.cat_trank.push_back(int8_t(M >= 2 ? h++ : -1));
            uint32_t v = hi.cat_vec[hi.cat_off[i] + q];
            for (int k = 0; k < m; ++k) {
                double nk = double(hi.comp[size_t(v) * m + k]) * double(M);
                gre += nk * p.nu_re[k];
                gim += nk * p.nu_im[k];
            }
        }
        hi.G[i] = uint8_t(G);
        hi.h[i] = uint8_t(h);
        hi.gamma_re[i] = gre;
        hi.gamma_im[i] = gim;
        hi.var_off[i + 1] = hi.var_off[i] + uint64_t((G + 1) * (G + 1) + h);
    }
    hi.cat_off[hi.P] = uint32_t(hi.cat_vec.size());

    // coefficient table (Eqs. uvar-up, uvar-down with c_k, c-check_k of
    // Eq. scaled-HEOM): raise: row -i sqrt((n+1)|c|), column +i sqrt((n+1)|c|);
    // lower: row -i sqrt(n/|c|) c_k, column +i sqrt(n/|c|) c-check_k
    hi.coef_row.assign(2 * kCoefPerInst, 0.0);
    hi.coef_col.assign(2 * kCoefPerInst, 0.0);
    for (int k = 0; k < m; ++k) {
        double ac = std::sqrt(p.c_re[k] * p.c_re[k] + p.c_im[k] * p.c_im[k]);
        for (int n = 0; n <= L && n < kCoefN; ++n) {
            int up = coef_id(k, n, 1), dn = coef_id(k, n, 0);
            double su = std::sqrt(double(n + 1) * ac);
            hi.coef_row[2 * up] = 0.0;
            hi.coef_row[2 * up + 1] = -su;
            hi.coef_col[2 * up] = 0.0;
            hi.coef_col[2 * up + 1] = su;
            double sd = std::sqrt(double(n) / ac);
            // -i sd c = sd (c_im - i c_re)
            hi.coef_row[2 * dn] = sd * p.c_im[k];
            hi.coef_row[2 * dn + 1] = -sd * p.c_re[k];
            // +i sd cc = sd (-cc_im + i cc_re)
            hi.coef_col[2 * dn] = -sd * p.cc_im[k];
            hi.coef_col[2 * dn + 1] = sd * p.cc_re[k];
        }
    }

    // connection records
    PatMap pm;
    pm.build(hi);
    const int64_t P = hi.P;
    std::vector<std::vector<Record>> per(P);
    std::vector<std::vector<uint32_t>> words(P);
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 256) reduction(+ : bad)
    for (int64_t i = 0; i < P; ++i) {
        const uint32_t* a = &hi.ids[hi.id_off[i]];
        int r = int(hi.id_off[i + 1] - hi.id_off[i]);
        int G = hi.G[i];
        const uint32_t* cv = &hi.cat_vec[hi.cat_off[i]];
        const int64_t* cM = &hi.cat_M[hi.cat_off[i]];
        uint32_t key[SA_HEOM_MAXL + 2];
        std::vector<Record>& out = per[i];
        std::vector<uint32_t>& cw = words[i];
        for (int q = 1; q <= G; ++q) {
            int start = int(out.size());
            uint32_t vq = cv[q - 1];
            // raise records of every channel first, then the lower records
            // (the P_q variables only need the lower ones)
            for (int dir = +1; dir >= -1; dir -= 2) {
                for (int k = 0; k < m; ++k) {
                    int n = hi.comp[size_t(vq) * m + k];
                    if (dir > 0 && hi.tier[i] >= L) continue;   // Eq. hard-cutoff-factor
                    if (dir < 0 && n == 0) continue;            // only occupied channels lower
                    int w = shift_vec(hi, int(vq), k, dir);
                    if (w < 0) {
                        ++bad;
                        continue;
                    }
                    // raw target as a multiset: one v_q replaced by w
                    int nk = 0;
                    bool dropped = (vq == 0);
                    for (int j = 0; j < r; ++j) {
                        if (!dropped && a[j] == vq) {
                            dropped = true;
                            continue;
                        }
                        key[nk++] = a[j];
                    }
                    if (w != 0) {
                        int pos = nk;
                        while (pos > 0 && key[pos - 1] > uint32_t(w)) {
                            key[pos] = key[pos - 1];
                            --pos;
                        }
                        key[pos] = uint32_t(w);
                        ++nk;
                    }
                    int64_t t = pm.find(key, nk);
                    if (t < 0) {
                        ++bad;
                        continue;
                    }
                    int del = cM[q - 1] == 1 ? 1 : 0;
                    int s_merge = 0;
                    for (int s = 1; s <= G; ++s)
                        if (s != q && cv[s - 1] == uint32_t(w)) s_merge = s;
                    int ins = s_merge ? 0 : 1;
                    int ipos = G + 1;
                    if (ins) {
                        // first old category that sorts after w (zero vector sorts last)
                        for (int s = 1; s <= G; ++s) {
                            bool after = (cv[s - 1] == 0) ? (w != 0) : (w != 0 && cv[s - 1] > uint32_t(w));
                            if (after) {
                                ipos = s;
                                break;
                            }
                        }
                    }
                    auto tau = [&](int rr) { return rr - ((del && rr > q) ? 1 : 0) + ((ins && rr >= ipos) ? 1 : 0); };
                    int tstar = ins ? ipos - ((del && q < ipos) ? 1 : 0) : tau(s_merge);
                    int Gp = hi.G[t];
                    // verify the remap against the target's categories
                    const uint32_t* tv = &hi.cat_vec[hi.cat_off[t]];
                    if (Gp != G + ins - del || tstar < 1 || tstar > Gp || tv[tstar - 1] != uint32_t(w)) ++bad;
                    for (int rr = 1; rr <= G; ++rr) {
                        if (rr == q && del) continue;
                        int tr = tau(rr);
                        if (tr < 1 || tr > Gp || tv[tr - 1] != cv[rr - 1]) ++bad;
                    }
                    int trs = hi.cat_trank[hi.cat_off[t] + tstar - 1];
                    Record rec;
                    rec.target = uint32_t(hi.var_off[t]);
                    // a merge record (ins = 0) keeps the merged source category
                    // in the ipos field, which only inserts use
                    rec.packed = pack_record(tstar, Gp, trs < 0 ? 0 : trs, trs >= 0 ? 1 : 0, ins ? ipos : s_merge,
                                             ins, del, coef_id(k, n, dir > 0 ? 1 : 0));
                    out.push_back(rec);
                }
            }
            cw.push_back(pack_cat(start, int(out.size()) - start, hi.cat_trank[hi.cat_off[i] + q - 1],
                                  hi.tier[i] < L ? m : 0));
        }
    }
    if (bad) {
        err = "internal: inconsistent connection record";
        return SA_ERR_INVALID_ARG;
    }
    hi.rec_off.assign(P + 1, 0);
    for (int64_t i = 0; i < P; ++i) hi.rec_off[i + 1] = hi.rec_off[i] + uint32_t(per[i].size());
    hi.rec.resize(hi.rec_off[P]);
    hi.cat_word.resize(hi.cat_vec.size());
    for (int64_t i = 0; i < P; ++i) {
        std::copy(per[i].begin(), per[i].end(), hi.rec.begin() + hi.rec_off[i]);
        std::copy(words[i].begin(), words[i].end(), hi.cat_word.begin() + hi.cat_off[i]);
    }
    hi.n_terms = expand_terms(hi, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr);
    return SA_OK;
}

// Expand the records into per-variable hierarchy terms, with the same
// integer resolution the kernels use.  Returns the number of terms; writes
// them when the arrays are not NULL.
int64_t expand_terms(const HostInstance& hi, int64_t* var, int64_t* src, int32_t* kk, int32_t* nn, int32_t* dd,
                     int32_t* side) {
    int64_t cnt = 0;
    for (int64_t i = 0; i < hi.P; ++i) {
        const int64_t base = int64_t(hi.var_off[i]);
        for_each_term(hi, i, [&](int64_t loc, int kind, int64_t s, uint32_t packed, int sd) {
            (void)kind;
            if (var) {
                const int cid = int(packed >> 23);
                var[cnt] = base + loc;
                src[cnt] = s;
                kk[cnt] = (cid >> 1) / kCoefN;
                nn[cnt] = (cid >> 1) % kCoefN;
                dd[cnt] = (cid & 1) ? +1 : -1;
                side[cnt] = sd;
            }
            ++cnt;
        });
    }
    return cnt;
}

}  // namespace sa
