// api.cu -- the C ABI of include/sa_heom.h: batch assembly, device tables,
// RK4 launch sequence, CUDA-graph capture of the step loop, observables,
// state marshalling and the launch autotuner.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cstdio>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "sa_internal.h"

namespace sa {
cudaError_t launch_stage(const StageLaunch& s, const LaunchCfg& cfg, bool fp64, cudaStream_t st);
cudaError_t stage_occupancy(const LaunchCfg& cfg, bool fp64, int* blocks_per_sm);
cudaError_t pack_occupancy(const LaunchCfg& cfg, bool fp64, int* blocks_per_sm);
void list_operand_layout(int item, int* opR, int* opC, int* opZ, int* opZero);
cudaError_t launch_observables(const InstDev* inst, const double* theta, int ninst, const PatHdr* hdr,
                               const double* catMd, const uint32_t* cat_word, const void* main64, const void* side64,
                               double* out, cudaStream_t st);
cudaError_t launch_init_rho0(const InstDev* inst, int ninst, const double* rho0, int stride, void* main64,
                             void* main32, void* side64, cudaStream_t st);
size_t recon_workspace_bytes(int64_t n);
cudaError_t launch_marshal(const InstDev* inst, int ninst, int packed, uint64_t n0, uint64_t cnt, void* stage,
                           void* main, void* side64, int fp64, int to_device, cudaStream_t st);
cudaError_t launch_reconstruct(const InstDev* inst, const RepSrc* src, const void* main64,
                               const void* side64, const void* rho0, int64_t n, void* rho_t, void* ws,
                               cudaStream_t st);
}  // namespace sa

using namespace sa;

namespace {
thread_local std::string g_err;

int fail(int code, const std::string& msg) {
    g_err = msg;
    return code;
}
int cuda_fail(cudaError_t e, const char* where) {
    g_err = std::string(where) + ": " + cudaGetErrorString(e);
    return SA_ERR_CUDA;
}
#define CK(call)                                               \
    do {                                                       \
        cudaError_t e_ = (call);                               \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);    \
    } while (0)

// Tables get 64 bytes of padding: the stage kernel's bulk copies round each
// range out to 16-byte boundaries.
template <typename V>
int upload(void** dptr, const std::vector<V>& h) {
    size_t b = h.size() * sizeof(V) + 64;
    cudaError_t e = cudaMalloc(dptr, b);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(table)");
    if (!h.empty()) {
        e = cudaMemcpy(*dptr, h.data(), h.size() * sizeof(V), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy(table)");
    }
    return SA_OK;
}
}  // namespace

namespace sa {
// detail of a failure in a file other than this one (sa_heom_last_error)
void set_error(const std::string& msg) { g_err = msg; }
}  // namespace sa

struct sa_heom {
    int count = 0;
    int precision = SA_FP64;
    bool host_only = true;
    std::vector<HostInstance> inst;
    std::vector<uint64_t> var_begin;  // per instance + total
    int64_t nvar = 0, npat = 0, ncat = 0, nrec = 0;
    // batch tables (host)
    std::vector<PatHdr> hdr;
    std::vector<uint32_t> cat_word;
    std::vector<double> catMd;
    std::vector<float> catMf;
    std::vector<double> gamma_d;
    std::vector<float> gamma_f;
    std::vector<Record> rec;
    std::vector<InstDev> instdev;
    std::vector<double> theta;
    std::vector<double> coef_row_d, coef_col_d;
    std::vector<float> coef_row_f, coef_col_f;
    std::vector<uint16_t> lut;
    std::vector<uint32_t> lut_off;
    std::vector<ItemDesc> items;
    std::vector<uint32_t> vdesc;
    std::vector<DRecA> drecA;
    std::vector<uint32_t> drecS;
    int max_u = 0;
    uint64_t lcoef_total = 0;  // slots of the list/ELL coefficient tables of all instances
    // term lists of the list kernel (built per tuning, freed after upload)
    std::vector<uint32_t> lvd, rbase, tidx;
    std::vector<uint8_t> lvj;
    std::vector<uint16_t> tcid;
    uint64_t list_rows = 0;
    std::vector<uint32_t> wpat;   // ELL: first pattern of every warp row
    std::vector<ItemDesc> list_items;  // SA_KERNEL_LISTS: the item table the current lists were built with
    // SA_KERNEL_LISTS: instances whose tables are identical (same m, L, d, bath
    // rates and structure, e.g. every saturated instance of one (m, L)) share
    // one template: its items, lists and blobs are built once, for its
    // representative instance, and a work unit pairs a template item with an
    // instance
    std::vector<int> tmpl;             // per instance: the representative instance of its template
    std::vector<uint32_t> units;       // per work unit: template item, instance
    void* d_units = nullptr;
    void* d_instk = nullptr;           // InstK<T> per instance
    // SA_BUILD_PACK_INSTANCES: the instances of a template with at least
    // kPackMin of them are stored in packs of up to 32, interleaved (PackDev);
    // the list kernel evaluates a pack item for all lanes of a pack at once
    bool packed = false;
    std::vector<PackDev> packs;
    std::vector<uint32_t> pk_inst;     // instance of every pack lane (PackDev::lane0 + j)
    std::vector<int> pack_of;          // per instance: its pack, -1 if none
    std::vector<std::vector<int>> tmpl_packs;  // per template representative: its packs
    std::vector<char> tmpl_list;       // per template representative: some member is not packed
    uint32_t pack_smem = 0;            // shared memory of a pack-kernel warp for the largest pack item
    uint64_t pcoef_total = 0;          // entries of the interleaved pack coefficient tables
    void* d_packs = nullptr;
    void* d_pkinst = nullptr;
    void* d_pcoef = nullptr;
    void* d_punits = nullptr;          // the pack units of `units`, in order (the list units go to d_units)
    void* d_ilimit = nullptr;          // per instance: variables and list coefficient slots (index checks)
    bool corrupt_list = false;         // SA_DEBUG_CORRUPT_LIST: the term lists carry one bad target
    uint32_t n_list_units = 0, n_pack_units = 0;
    std::vector<uint8_t> blobs;        // SA_KERNEL_LISTS: per-item table blobs
    int tables = -1;              // variant whose term tables are current (-1: none)
    int tables_chunk = 0;         // item capacity they were built for (SA_KERNEL_LISTS)
    // tuning
    int block = 256, chunk = 128, use_queue = 1, kernel = SA_KERNEL_LISTS;
    int debug = 0;  // SA_DEBUG_* flags
    // device
    int device = -1, num_sms = 0;
    void *d_hdr = nullptr, *d_cat_word = nullptr, *d_catM = nullptr, *d_catMd = nullptr, *d_gamma = nullptr;
    void *d_rec = nullptr, *d_inst = nullptr, *d_theta = nullptr, *d_coef_row = nullptr, *d_coef_col = nullptr;
    void *d_coef_row_d = nullptr, *d_coef_col_d = nullptr, *d_lut = nullptr, *d_lut_off = nullptr;
    void* d_chunk = nullptr;
    void *d_vdesc = nullptr, *d_drecA = nullptr, *d_drecS = nullptr;
    void *d_lvd = nullptr, *d_lvj = nullptr, *d_rbase = nullptr, *d_tidx = nullptr, *d_tcid = nullptr;
    void* d_lcoef = nullptr;
    void* d_wpat = nullptr;
    void* d_blobs = nullptr;
    void* d_catpat = nullptr;  // ELL: owning pattern of every category
    void* d_sums = nullptr;    // ELL: grouped sums scratch (R, C per category; Z per pattern)
    unsigned int* d_err = nullptr;
    void* d_work[3] = {nullptr, nullptr, nullptr};  // acc, xa, xb
    unsigned int* d_queue = nullptr;
    size_t queue_slots = 0;
    double* d_obs = nullptr;
    size_t obs_cap = 0;
    double* d_rho0 = nullptr;
    cudaStream_t cap = nullptr;
    cudaStream_t side = nullptr;                          // SA_FP32_AUX: stream of the FP64 rho_0 kernel
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;     // its fork and join
    size_t state_bytes = 0, side_off = 0;
    LaunchCfg cfg{256, 128, 1, 1, SA_KERNEL_LISTS};
    std::map<std::tuple<const void*, uint64_t, int64_t>, cudaGraphExec_t> graphs;
    // representative propagations (sa_heom_build_representatives)
    bool reps = false;
    std::vector<RepSrc> rep_src;   // kReps x kRepSlots: where each response value lives
    std::vector<int> rep_unit;     // per instance: the slot of its unit initial operator
    void* d_rep_loc = nullptr;     // device copy of rep_src
    void* d_recon_ws = nullptr;
    size_t recon_ws = 0;
};

namespace {

void build_lut(sa_heom* h) {
    h->lut_off.assign(kMaxG + 2, 0);
    h->lut.clear();
    for (int G = 0; G <= kMaxG; ++G) {
        h->lut_off[G] = uint32_t(h->lut.size());
        for (int loc = 0; G > 0 && loc < (G + 1) * (G + 1); ++loc) {
            int kind, q = 0, r = 0;
            if (loc == 0) kind = 0;
            else if (loc <= G) { kind = 1; q = loc; }
            else if (loc <= 2 * G) { kind = 2; q = loc - G; }
            else if (loc <= 3 * G) { kind = 3; q = loc - 2 * G; }
            else {
                kind = 4;
                int s = loc - 3 * G - 1;
                q = s / (G - 1) + 1;
                r = s % (G - 1) + 1;
                if (r >= q) ++r;
            }
            h->lut.push_back(uint16_t(kind | (q << 3) | (r << 8)));
        }
    }
    h->lut_off[kMaxG + 1] = uint32_t(h->lut.size());
}

// Work items (one warp each): runs of consecutive patterns with at most
// `chunk` variables and kItemPats patterns.  vdesc gives each item's
// variables in the order the warp's lanes take them -- S first, then T, P, X,
// Y, Z, every kind in memory order -- with their local index and (kind, q, r).
void build_items(sa_heom* h) {
    std::vector<uint32_t> begin{0};
    int64_t vars = 0, pats = 0, insts = 0;
    for (int64_t p = 0; p < h->npat; ++p) {
        int64_t u = int64_t(h->hdr[p + 1].var_off) - int64_t(h->hdr[p].var_off);
        const bool new_inst = pats > 0 && h->hdr[p].inst != h->hdr[p - 1].inst;
        if (pats > 0 && (vars + u > h->chunk || pats >= kItemPats || (new_inst && insts >= kItemInsts))) {
            begin.push_back(uint32_t(p));
            vars = 0;
            pats = 0;
            insts = 0;
        }
        if (pats == 0 || new_inst) ++insts;
        vars += u;
        ++pats;
    }
    begin.push_back(uint32_t(h->npat));
    h->items.clear();
    h->vdesc.assign(size_t(h->nvar), 0u);
    for (size_t c = 0; c + 1 < begin.size(); ++c) {
        const PatHdr &a = h->hdr[begin[c]], &b = h->hdr[begin[c + 1]];
        ItemDesc d{};
        d.p0 = begin[c];
        d.np = begin[c + 1] - begin[c];
        d.v0 = a.var_off;
        d.nv = b.var_off - a.var_off;
        d.c0 = a.cat_off;
        d.ncat = b.cat_off - a.cat_off;
        h->items.push_back(d);
        uint32_t* out = &h->vdesc[d.v0];
        auto put = [&](uint32_t l, uint32_t j, uint32_t kind, uint32_t q, uint32_t r) {
            *out++ = l | (j << 10) | (kind << 15) | (q << 18) | (r << 23);
        };
        for (uint32_t j = 0; j < d.np; ++j) {  // S
            const PatHdr& H = h->hdr[d.p0 + j];
            const int G = H.G;
            for (int q = 1; q <= G; ++q)
                for (int r = 1; r <= G; ++r)
                    if (r != q) put(uint32_t(H.var_off - d.v0 + loc_S(G, q, r)), j, 4, q, r);
        }
        for (uint32_t j = 0; j < d.np; ++j) {  // T
            const PatHdr& H = h->hdr[d.p0 + j];
            for (int q = 1; q <= H.G; ++q) {
                const int tr = (h->cat_word[H.cat_off + q - 1] >> 15) & 31;
                if (tr != 31) put(uint32_t(H.var_off - d.v0 + loc_T(H.G, tr)), j, 5, q, 0);
            }
        }
        for (int kind : {3, 1, 2}) {  // P, X, Y
            for (uint32_t j = 0; j < d.np; ++j) {
                const PatHdr& H = h->hdr[d.p0 + j];
                for (int q = 1; q <= H.G; ++q) {
                    const int64_t loc = kind == 3 ? loc_P(H.G, q) : (kind == 1 ? loc_X(H.G, q) : loc_Y(H.G, q));
                    put(uint32_t(H.var_off - d.v0 + loc), j, kind, q, 0);
                }
            }
        }
        for (uint32_t j = 0; j < d.np; ++j) put(h->hdr[d.p0 + j].var_off - d.v0, j, 0, 0, 0);  // Z
    }
}

// Templates of the list kernel: an instance shares the template of an
// earlier instance when everything its lists and blobs are made of is equal
// -- channels, depth, distinguished molecules, pattern and variable layout,
// category words and vectors, connection records, damping rates and the
// structure of the multiplicities (equal for the nonzero vectors, and the
// same r = N - M_0 for the zero category).  Hashing picks the candidates.
namespace {
uint64_t mix(uint64_t h, uint64_t v) {
    h ^= v + 0x9e3779b97f4a7c15ull + (h << 6) + (h >> 2);
    return h;
}
template <class V> uint64_t hash_vec(uint64_t h, const std::vector<V>& v) {
    h = mix(h, v.size());
    for (size_t i = 0; i < v.size(); i += 1 + v.size() / 4096) {  // a sample suffices to pick candidates
        uint64_t w = 0;
        std::memcpy(&w, &v[i], sizeof(V) < 8 ? sizeof(V) : 8);
        h = mix(h, w);
    }
    return h;
}
// the multiplicity as a template holds it: M for a nonzero vector, M_0 - N (= -r) for the zero vector
int64_t tmpl_mult(const HostInstance& hi, size_t c) { return hi.cat_vec[c] == 0 ? hi.cat_M[c] - hi.N : hi.cat_M[c]; }
bool same_tables(const HostInstance& a, const HostInstance& b) {
    if (a.m != b.m || a.L != b.L || a.d != b.d || a.P != b.P || a.var_off != b.var_off || a.cat_off != b.cat_off ||
        a.cat_word != b.cat_word || a.cat_vec != b.cat_vec || a.rec_off != b.rec_off || a.rec.size() != b.rec.size() ||
        a.gamma_re != b.gamma_re || a.gamma_im != b.gamma_im || a.tier != b.tier)
        return false;
    for (size_t i = 0; i < a.rec.size(); ++i)
        if (a.rec[i].target != b.rec[i].target || a.rec[i].packed != b.rec[i].packed) return false;
    for (size_t c = 0; c < a.cat_M.size(); ++c)
        if (tmpl_mult(a, c) != tmpl_mult(b, c)) return false;
    return true;
}
}  // namespace

void assign_templates(sa_heom* h) {
    h->tmpl.assign(size_t(h->count), -1);
    std::map<uint64_t, std::vector<int>> reps;
    for (int i = 0; i < h->count; ++i) {
        const HostInstance& hi = h->inst[i];
        uint64_t k = mix(mix(mix(uint64_t(hi.m), uint64_t(hi.L)), uint64_t(hi.d)), uint64_t(hi.P));
        k = hash_vec(k, hi.var_off);
        k = hash_vec(k, hi.cat_word);
        k = hash_vec(k, hi.gamma_re);
        std::vector<int>& cand = reps[k];
        for (int r : cand)
            if (same_tables(h->inst[r], hi)) {
                h->tmpl[i] = r;
                break;
            }
        if (h->tmpl[i] < 0) {
            h->tmpl[i] = i;
            cand.push_back(i);
        }
    }
}

// Packs (SA_BUILD_PACK_INSTANCES): the members of every template with at
// least kPackMin instances, in instance order, in packs of 32 and one of the
// remaining K mod 32 if that is at least kPackMin (fewer stay unpacked).
// Then the device layout, instance by instance: a pack's
// block (its n lanes interleaved over the template's variables) where its
// first lane's instance stands, every other instance contiguous; likewise
// the packs' interleaved coefficient tables.
int assign_packs(sa_heom* h) {
    const int nc = h->count;
    h->pack_of.assign(size_t(nc), -1);
    h->packs.clear();
    h->pk_inst.clear();
    h->tmpl_packs.assign(size_t(nc), {});
    std::vector<int> lane(size_t(nc), 0);
    if (h->packed) {
        std::vector<std::vector<int>> members(static_cast<size_t>(nc));
        for (int i = 0; i < nc; ++i) members[size_t(h->tmpl[i])].push_back(i);
        for (int r = 0; r < nc; ++r) {
            const int K = int(members[size_t(r)].size());
            if (K < kPackMin) continue;
            // full packs of 32, then the rest as one pack if it has kPackMin
            // members (the others stay unpacked)
            std::vector<uint32_t> sizes(size_t(K / kPackLanes), uint32_t(kPackLanes));
            if (K % kPackLanes >= kPackMin) sizes.push_back(uint32_t(K % kPackLanes));
            int at = 0;
            for (uint32_t nk : sizes) {
                PackDev pk{};
                pk.n = nk;
                pk.lane0 = uint32_t(h->pk_inst.size());
                for (uint32_t j = 0; j < pk.n; ++j) {
                    const int i = members[size_t(r)][size_t(at) + j];
                    h->pk_inst.push_back(uint32_t(i));
                    h->pack_of[size_t(i)] = int(h->packs.size());
                    lane[size_t(i)] = int(j);
                }
                at += int(pk.n);
                h->tmpl_packs[size_t(r)].push_back(int(h->packs.size()));
                h->packs.push_back(pk);
            }
        }
    }
    h->tmpl_list.assign(size_t(nc), 0);
    for (int i = 0; i < nc; ++i)
        if (h->pack_of[size_t(i)] < 0) h->tmpl_list[size_t(h->tmpl[i])] = 1;
    uint64_t cur = 0, cb = 0;
    for (int i = 0; i < nc; ++i) {
        InstDev& D = h->instdev[size_t(i)];
        const uint64_t nv = h->var_begin[size_t(i) + 1] - h->var_begin[size_t(i)];
        const int k = h->pack_of[size_t(i)];
        if (k < 0) {
            D.dev_base = uint32_t(cur);
            D.dev_stride = 1;
            cur += nv;
            continue;
        }
        PackDev& pk = h->packs[size_t(k)];
        if (lane[size_t(i)] == 0) {  // members are in instance order: lane 0 comes first
            pk.base = uint32_t(cur);
            pk.cbase = uint32_t(cb);
            cur += nv * pk.n;
            cb += uint64_t(list_slots(h->inst[size_t(i)].m, h->inst[size_t(i)].L)) * pk.n;
        }
        D.dev_base = pk.base + uint32_t(lane[size_t(i)]);
        D.dev_stride = pk.n;
    }
    if (cur != uint64_t(h->nvar)) return fail(SA_ERR_STATE, "pack layout does not cover the batch");
    if (cb >= (uint64_t(1) << 32)) return fail(SA_ERR_UNSUPPORTED, "pack coefficient tables exceed 32-bit indices");
    h->pcoef_total = cb;
    return SA_OK;
}

// The list kernel's work items: per template, runs of its representative's
// consecutive patterns with at most `chunk` variables and kItemPats patterns
// (batch-global p0, v0, c0 while the lists are built).
std::vector<ItemDesc> template_items(const sa_heom* h) {
    std::vector<ItemDesc> out;
    for (int r = 0; r < h->count; ++r) {
        if (h->tmpl[r] != r || !h->tmpl_list[size_t(r)]) continue;
        const int64_t pb = h->instdev[r].pat_begin, pe = pb + h->inst[r].P;
        int64_t p = pb;
        while (p < pe) {
            int64_t q = p, vars = 0;
            while (q < pe && q - p < kItemPats) {
                const int64_t u = int64_t(h->hdr[q + 1].var_off) - int64_t(h->hdr[q].var_off);
                if (q > p && vars + u > h->chunk) break;
                vars += u;
                ++q;
            }
            ItemDesc d{};
            d.p0 = uint32_t(p);
            d.np = uint32_t(q - p);
            d.v0 = h->hdr[p].var_off;
            d.nv = h->hdr[q].var_off - h->hdr[p].var_off;
            d.c0 = h->hdr[p].cat_off;
            d.ncat = h->hdr[q].cat_off - h->hdr[p].cat_off;
            out.push_back(d);
            p = q;
        }
    }
    return out;
}

// Term lists of the list kernel.  For every work item: its variables in lane
// order (the physical representative left out in SA_FP32_AUX mode, where the
// FP64 kernel integrates it), sorted by hierarchy-term count, longest first;
// per variable the operand-area indices of its commutator term and its
// diagonal class; per round of 32 lanes T rows of 32 (target, coefficient
// slot) entries, T the round's longest list, short lists padded with the zero
// slot.  Two passes over the items (sizes, then contents), each in parallel.
struct ListItem {
    std::vector<uint32_t> order;     // lane order: item-local variable indices
    std::vector<uint32_t> desc;      // per item-local variable: l | a << 10 | b << 21
    std::vector<uint8_t> cls;        // per item-local variable: j | class << 5
    std::vector<uint32_t> off, cnt;  // per item-local variable: its terms
    std::vector<uint32_t> tix;
    std::vector<uint16_t> tsl;
};

void list_item(const sa_heom* h, const ItemDesc& d, ListItem& W) {
    int opR, opC, opZ, opZero;
    list_operand_layout(h->chunk, &opR, &opC, &opZ, &opZero);
    const bool side64 = h->precision == SA_FP32_AUX;
    W.desc.assign(d.nv, 0u);
    W.cls.assign(d.nv, 0);
    W.cnt.assign(d.nv, 0u);
    W.order.clear();
    std::vector<uint32_t> tv;  // per term: item-local variable
    W.tix.clear();
    W.tsl.clear();
    for (uint32_t j = 0; j < d.np; ++j) {
        const PatHdr& H = h->hdr[d.p0 + j];
        const int G = H.G;
        const uint32_t pl = H.var_off - d.v0, cb = H.cat_off - d.c0;
        const bool skip = side64 && H.tier == 0;
        auto put = [&](int64_t loc, uint32_t a, uint32_t b, uint32_t c) {
            const uint32_t l = pl + uint32_t(loc);
            W.desc[l] = l | (a << 10) | (b << 21);
            W.cls[l] = uint8_t(j | (c << 5));
            if (!skip) W.order.push_back(l);
        };
        put(loc_Z(), uint32_t(opZ) + j, uint32_t(opZero), 3);
        for (int q = 1; q <= G; ++q) {
            put(loc_X(G, q), pl, uint32_t(opR) + cb + q - 1, 1);
            put(loc_Y(G, q), uint32_t(opC) + cb + q - 1, pl, 2);
            put(loc_P(G, q), pl + G + q, pl + q, 4);
            for (int r = 1; r <= G; ++r)
                if (r != q) put(loc_S(G, q, r), pl + G + r, pl + q, 0);
            const int tr = (h->cat_word[H.cat_off + q - 1] >> 15) & 31;
            if (tr != 31) put(loc_T(G, tr), pl + G + q, pl + q, 0);
        }
        if (skip) continue;
        // targets relative to the instance's first variable, slots to its
        // coefficient table: every instance of the template reads the same lists
        const int inst = H.inst;
        const int64_t p = int64_t(d.p0 + j) - int64_t(h->instdev[inst].pat_begin);
        for_each_term(h->inst[inst], p, [&](int64_t loc, int kind, int64_t src, uint32_t packed, int side) {
            const int cid = int(packed >> 23);
            if (kind == 3 && side == 1) return;  // folded into the row term's coefficient
            const int slot = list_slot(h->inst[inst].L, cid, kind == 3 ? 2 : side);
            const uint32_t l = pl + uint32_t(loc);
            tv.push_back(l);
            W.tix.push_back(uint32_t(src));
            W.tsl.push_back(uint16_t(slot));
            ++W.cnt[l];
        });
    }
    // terms grouped by variable (counting sort, stable)
    W.off.assign(d.nv + 1, 0u);
    for (uint32_t l = 0; l < d.nv; ++l) W.off[l + 1] = W.off[l] + W.cnt[l];
    std::vector<uint32_t> pos(W.off.begin(), W.off.end() - 1);
    std::vector<uint32_t> ix(W.tix.size());
    std::vector<uint16_t> sl(W.tsl.size());
    for (size_t t = 0; t < tv.size(); ++t) {
        const uint32_t k = pos[tv[t]]++;
        ix[k] = W.tix[t];
        sl[k] = W.tsl[t];
    }
    W.tix.swap(ix);
    W.tsl.swap(sl);
    // lanes by term count, longest first, and in memory order within a count:
    // a round's lanes then read and write nearly contiguous state, and the
    // row terms of consecutive S_{q,r} of one row q (the same connection
    // record) gather from consecutive entries of the target's row
    std::sort(W.order.begin(), W.order.end(),
              [&](uint32_t x, uint32_t y) { return W.cnt[x] != W.cnt[y] ? W.cnt[x] > W.cnt[y] : x < y; });
}

// Per-item table blobs of the list kernel (BlobLayout): everything the warp
// stages for an item besides the state slices, contiguous and 16-byte
// aligned so that one bulk copy brings it.
// Per-item table blobs of the list kernel (BlobLayout): everything the warp
// stages for an item besides the state slices, contiguous and 16-byte
// aligned so that one bulk copy brings it.
// the diagonal coefficients of a pattern's variable classes (0 S T, 1 X,
// 2 Y, 3 Z, 4 P: -Gamma_Lambda, the cavity loss (1/2 per cavity label),
// -/+ i detuning for X / Y, the terminator -Delta w) and (g, 0), as the list
// blobs hold them
template <typename V>
void pattern_diag(const sa_heom* h, uint32_t p, V* e) {
    const sa_params& q = h->inst[h->hdr[p].inst].p;
    const double gre = h->gamma_d[2 * size_t(p)], gim = h->gamma_d[2 * size_t(p) + 1];
    const double lossf[5] = {0.0, 0.5, 0.5, 1.0, 0.0}, wt[5] = {2.0, 1.0, 1.0, 0.0, 0.0};
    const double dim[5] = {0.0, -q.detuning, q.detuning, 0.0, 0.0};
    for (int cl = 0; cl < 5; ++cl) {
        e[2 * cl] = V(-(gre + lossf[cl] * q.kappa + wt[cl] * q.term));
        e[2 * cl + 1] = V(dim[cl] - gim);
    }
    e[10] = V(q.g);
    e[11] = V(0);
}

// a pack item (r0) rather than a list item of the work-item table
constexpr uint32_t kPackItemMark = 0xffffffffu;

// Grouped-sum weights a + b N of the patterns p0 .. p1 - 1 of template
// representative r, appended to w where new: 1 (a = 1, b = 0) first, then per
// category M_q, M_q - 1 and -M_q, the zero category's M_0 = N - r being
// a = -r, b = 1.  The pack kernel evaluates each once per unit and lane.
static void pack_weights(const sa_heom* h, int r, int64_t p0, int64_t p1,
                         std::vector<std::pair<int64_t, int64_t>>& w) {
    const HostInstance& hi = h->inst[r];
    const uint32_t cb = h->hdr[h->instdev[r].pat_begin].cat_off;
    auto add = [&](int64_t a, int64_t b) {
        for (const auto& e : w)
            if (e.first == a && e.second == b) return;
        w.emplace_back(a, b);
    };
    add(1, 0);
    for (int64_t p = p0; p < p1; ++p)
        for (uint32_t c = h->hdr[p].cat_off; c < h->hdr[p + 1].cat_off; ++c) {
            const size_t gc = size_t(c - cb);
            const int64_t mt = tmpl_mult(hi, gc), zb = hi.cat_vec[gc] == 0 ? 1 : 0;
            add(mt, zb);
            add(mt - 1, zb);
            add(-mt, -zb);
        }
}

// Blob of a pack item (PackLayout): patterns, -Gamma_Lambda per pattern, the
// template's multiplicities, and per variable the warp updates a record --
// commutator operands, class and pattern (as list_item resolves them,
// renumbered for the pack kernel: R, C, Z sums and the zero after the item's
// nv variables), its terms, and the grouped sums its value enters -- in the
// three phases P/T/S, X/Y, Z.  Sets d.nl (variables updated), d.row0 (terms)
// and d.row1 (the first two phases' lengths, 16 bits each).
template <typename V>
int pack_blob(const sa_heom* h, ItemDesc& d, uint8_t* o) {
    ListItem W;
    list_item(h, d, W);
    const bool side64 = h->precision == SA_FP32_AUX;
    // contribution word: sum slot | the index of its weight a + b N in the
    // item's weight list << 11 (kind 1 one, 2 M_c, 3 M_c - 1, 4 -M_c of item
    // category c; b = 1 or -1 only for the zero category, whose M_0 = N - r
    // is stored as -r)
    const int rw = int(h->hdr[d.p0].inst);
    const HostInstance& hrw = h->inst[rw];
    const uint32_t cbw = h->hdr[h->instdev[rw].pat_begin].cat_off;
    std::vector<std::pair<int64_t, int64_t>> wl;
    pack_weights(h, rw, d.p0, int64_t(d.p0) + d.np, wl);
    bool missing = false;  // a contribution whose weight is not listed (never, by construction)
    if (wl.size() != d.nw) return fail(SA_ERR_STATE, "pack item weights differ from its budget");
    auto cw = [&](uint32_t slot, uint32_t kind, uint32_t c) {
        const size_t gc = size_t(d.c0 + c - cbw);
        const int64_t mt = tmpl_mult(hrw, gc);  // M, or -r for the zero category
        const int64_t zb = hrw.cat_vec[gc] == 0 ? 1 : 0;
        int64_t a = 1, b = 0;
        if (kind == 2) a = mt, b = zb;
        if (kind == 3) a = mt - 1, b = zb;
        if (kind == 4) a = -mt, b = -zb;
        uint32_t k = 0;
        while (k < wl.size() && (wl[k].first != a || wl[k].second != b)) ++k;  // listed by pack_weights
        if (k == wl.size()) missing = true;
        return slot | k << 11;
    };
    struct Rec {
        uint32_t l, z, w;
    };
    std::vector<Rec> ph[3];
    for (uint32_t j = 0; j < d.np; ++j) {
        const PatHdr& H = h->hdr[d.p0 + j];
        if (side64 && H.tier == 0) continue;  // integrated in FP64 by the side kernel
        const int G = H.G;
        const uint32_t pl = H.var_off - d.v0, cb = H.cat_off - d.c0;
        ph[2].push_back({pl + uint32_t(loc_Z()), 0u, 0u});
        for (int q = 1; q <= G; ++q) {
            const uint32_t cq = cb + uint32_t(q) - 1;
            ph[1].push_back({pl + uint32_t(loc_X(G, q)), cw(2 * d.ncat + j, 2, cq), 0u});
            ph[1].push_back({pl + uint32_t(loc_Y(G, q)), cw(2 * d.ncat + j, 4, cq), 0u});
            ph[0].push_back({pl + uint32_t(loc_P(G, q)), cw(cq, 1, cq), cw(d.ncat + cq, 1, cq)});
            for (int r = 1; r <= G; ++r) {
                if (r == q) continue;
                const uint32_t cr = cb + uint32_t(r) - 1;
                ph[0].push_back({pl + uint32_t(loc_S(G, q, r)), cw(cq, 2, cr), cw(d.ncat + cr, 2, cq)});
            }
            const int tr = (h->cat_word[H.cat_off + q - 1] >> 15) & 31;
            if (tr != 31) ph[0].push_back({pl + uint32_t(loc_T(G, tr)), cw(cq, 3, cq), cw(d.ncat + cq, 3, cq)});
        }
    }
    if (missing) return fail(SA_ERR_STATE, "a pack item's grouped-sum weight is not in its list");
    for (auto& v : ph) std::sort(v.begin(), v.end(), [](const Rec& x, const Rec& y) { return x.l < y.l; });
    d.nl = uint32_t(ph[0].size() + ph[1].size() + ph[2].size());
    d.row1 = uint32_t(ph[0].size()) | (uint32_t(ph[1].size()) << 16);
    uint32_t nterm = 0;
    for (auto& v : ph)
        for (const Rec& e : v) nterm += W.cnt[e.l];
    d.row0 = nterm;
    if (ph[0].size() > 65535u || ph[1].size() > 65535u)
        return fail(SA_ERR_UNSUPPORTED, "a pack item has too many variables");
    const PackLayout B = pack_layout<V>(d.np, d.ncat, d.nl, nterm, d.nw);
    reinterpret_cast<uint32_t*>(o)[0] = d.nw;
    int32_t* wab = reinterpret_cast<int32_t*>(o + B.wab);
    for (uint32_t k = 0; k < d.nw; ++k) {
        if (wl[k].first < INT32_MIN || wl[k].first > INT32_MAX)
            return fail(SA_ERR_UNSUPPORTED, "a grouped-sum weight is beyond 32 bits");
        wab[2 * k] = int32_t(wl[k].first);
        wab[2 * k + 1] = int32_t(wl[k].second);
    }
    ItemPat* phd = reinterpret_cast<ItemPat*>(o + B.pat);
    V* pd = reinterpret_cast<V*>(o + B.pd);
    V* cM = reinterpret_cast<V*>(o + B.cM);
    uint32_t* vrec = reinterpret_cast<uint32_t*>(o + B.vrec);
    uint32_t* tgt = reinterpret_cast<uint32_t*>(o + B.tgt);
    uint16_t* tsl = reinterpret_cast<uint16_t*>(o + B.tsl);
    const HostInstance& hr = h->inst[h->hdr[d.p0].inst];
    const uint32_t cbase = h->hdr[h->instdev[h->hdr[d.p0].inst].pat_begin].cat_off;
    for (uint32_t j = 0; j < d.np; ++j) {
        const PatHdr& H = h->hdr[d.p0 + j];
        phd[j].var_rel = uint16_t(H.var_off - d.v0);
        phd[j].cat_rel = uint16_t(H.cat_off - d.c0);
        phd[j].G = H.G;
        phd[j].tier = H.tier;
        phd[j].islot = 0;
        pd[2 * j] = V(-h->gamma_d[2 * size_t(d.p0 + j)]);
        pd[2 * j + 1] = V(-h->gamma_d[2 * size_t(d.p0 + j) + 1]);
    }
    for (uint32_t cl = 0; cl < d.ncat; ++cl) cM[cl] = V(tmpl_mult(hr, size_t(d.c0 + cl - cbase)));
    int opR, opC, opZ, opZero;
    list_operand_layout(h->chunk, &opR, &opC, &opZ, &opZero);
    auto code = [&](uint32_t a) -> uint32_t {
        if (a < uint32_t(opR)) return a;                                     // an item variable
        if (a < uint32_t(opC)) return d.nv + (a - uint32_t(opR));             // R of a category
        if (a < uint32_t(opZ)) return d.nv + d.ncat + (a - uint32_t(opC));    // C of a category
        if (a < uint32_t(opZero)) return d.nv + 2 * d.ncat + (a - uint32_t(opZ));  // Z of a pattern
        return d.nv + 2 * d.ncat + d.np;                                      // zero
    };
    uint32_t u = 0, i = 0;
    for (auto& v : ph)
        for (const Rec& e : v) {
            const uint32_t l = e.l;
            const uint32_t w = W.desc[l];
            const uint32_t a = (w >> 10) & 2047u, b = w >> 21;
            const uint32_t j = W.cls[l] & 31u, cls = W.cls[l] >> 5;
            const uint32_t cnt = W.cnt[l];
            if (cnt > 63u || l > 1023u) return fail(SA_ERR_UNSUPPORTED, "a variable has more than 63 hierarchy terms");
            vrec[4 * i] = code(a) | (code(b) << 11) | (cls << 22) | (j << 25);
            vrec[4 * i + 1] = l | (u << 10) | (cnt << 26);
            vrec[4 * i + 2] = e.z;
            vrec[4 * i + 3] = e.w;
            ++i;
            for (uint32_t t = 0; t < cnt; ++t, ++u) {
                tgt[u] = W.tix[W.off[l] + t];
                tsl[u] = W.tsl[W.off[l] + t];
            }
        }
    return SA_OK;
}

// Per-item table blobs of the list kernel (BlobLayout): everything the warp
// stages for an item besides the state slices, contiguous and 16-byte
// aligned so that one bulk copy brings it.  Pack items get a PackLayout blob;
// pack_smem is the shared memory a warp needs for the largest.
template <typename V>
int build_blobs(sa_heom* h) {
    const size_t ni = h->items.size();
    uint64_t off16 = 0;
    uint32_t max_pack = 0;
    for (size_t c = 0; c < ni; ++c) {
        ItemDesc& d = h->items[c];
        const bool pk = d.r0 == kPackItemMark;
        // (a pack blob is sized for all nv variables and row0 terms; the
        // builder may update fewer)
        const uint32_t bytes = pk ? pack_layout<V>(d.np, d.ncat, d.nv, d.row0, d.nw).bytes
                                  : blob_layout<V>(d.np, d.ncat, d.nl).bytes;
        if (pk)
            max_pack = std::max(max_pack, pack_sums_bytes<V>(d.np, d.ncat) + bytes + pack_wtab_bytes<V>(d.nw) +
                                              pack_dtab_bytes<V>(d.np));
        d.blob16 = uint32_t(off16);
        d.blob_bytes = bytes;
        off16 += bytes / 16;
        if (off16 >= (uint64_t(1) << 32)) return fail(SA_ERR_UNSUPPORTED, "list-kernel blobs exceed 64 GB");
    }
    try {
        h->blobs.assign(size_t(off16) * 16, 0);
    } catch (const std::bad_alloc&) {
        return fail(SA_ERR_OOM, "host memory for the list-kernel blobs");
    }
    // a pack-kernel warp: mbarrier, 5 x 32 per-lane diagonal parts, then the
    // item's grouped sums, its blob, its per-lane weights and diagonals (the
    // largest item sets the size)
    h->pack_smem = max_pack ? 16u + uint32_t(5 * 32 * 2 * sizeof(V)) + max_pack : 0u;
    int prc = SA_OK;
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t c = 0; c < int64_t(ni); ++c) {
        ItemDesc& d = h->items[c];
        if (d.r0 == kPackItemMark) {
            const int r = pack_blob<V>(h, d, &h->blobs[size_t(d.blob16) * 16]);
            if (r) {
#pragma omp critical
                prc = r;
            }
            continue;
        }
        const BlobLayout B = blob_layout<V>(d.np, d.ncat, d.nl);
        uint8_t* o = &h->blobs[size_t(d.blob16) * 16];
        ItemPat* ph = reinterpret_cast<ItemPat*>(o + B.pat);
        V* pd = reinterpret_cast<V*>(o + B.pd);
        uint32_t* cw = reinterpret_cast<uint32_t*>(o + B.cw);
        V* cM = reinterpret_cast<V*>(o + B.cM);
        uint8_t* cj = o + B.cj;
        uint32_t* rb = reinterpret_cast<uint32_t*>(o + B.rb);
        uint32_t* lvd = reinterpret_cast<uint32_t*>(o + B.lvd);
        uint8_t* lvj = o + B.lvj;
        for (uint32_t j = 0; j < d.np; ++j) {
            const PatHdr& H = h->hdr[d.p0 + j];
            ph[j].var_rel = uint16_t(H.var_off - d.v0);
            ph[j].cat_rel = uint16_t(H.cat_off - d.c0);
            ph[j].G = H.G;
            ph[j].tier = H.tier;
            ph[j].islot = 0;
            pd[2 * j] = V(-h->gamma_d[2 * size_t(d.p0 + j)]);  // -Gamma_Lambda
            pd[2 * j + 1] = V(-h->gamma_d[2 * size_t(d.p0 + j) + 1]);
            for (uint32_t cl = H.cat_off - d.c0; cl < h->hdr[d.p0 + j + 1].cat_off - d.c0; ++cl) cj[cl] = uint8_t(j);
        }
        // multiplicities as the template holds them: M_0 - N = -r for the zero
        // category, whose M_0 the kernel forms from the instance's N
        const HostInstance& hr = h->inst[h->hdr[d.p0].inst];
        const uint32_t cbase = h->hdr[h->instdev[h->hdr[d.p0].inst].pat_begin].cat_off;
        for (uint32_t cl = 0; cl < d.ncat; ++cl) {
            cw[cl] = h->cat_word[d.c0 + cl];
            cM[cl] = V(tmpl_mult(hr, size_t(d.c0 + cl - cbase)));
        }
        const uint32_t nrounds = (d.nl + 31) / 32;
        for (uint32_t r = 0; d.nl && r <= nrounds; ++r) rb[r] = h->rbase[d.r0 + r];
        for (uint32_t i = 0; i < d.nl; ++i) {
            lvd[i] = h->lvd[size_t(d.r0) * 32 + i];
            lvj[i] = h->lvj[size_t(d.r0) * 32 + i];
        }
    }
    return prc;
}

uint64_t list_item_rows(const ListItem& W) {
    uint64_t rows = 0;
    for (size_t i = 0; i < W.order.size(); i += 32) rows += W.cnt[W.order[i]];
    return rows;
}

// Pack items (SA_KERNEL_LISTS on a packed handle): per packed template, runs
// of its representative's consecutive patterns whose blob (PackLayout),
// grouped sums and per-lane weights stay within kPackItemTarget bytes; a
// pattern larger than that gets an item of its own.  nl holds the variables
// the warp updates, row0 the item's term count, nw its weights, r0 the
// pack-item mark.
template <typename V>
int pack_items(const sa_heom* h, std::vector<ItemDesc>& out) {
    const bool side64 = h->precision == SA_FP32_AUX;
    int opR, opC, opZ, opZero;
    list_operand_layout(h->chunk, &opR, &opC, &opZ, &opZero);
    const int ncat_cap = opC - opR;  // categories the list operand layout holds
    for (int r = 0; r < h->count; ++r) {
        if (h->tmpl[r] != r || h->tmpl_packs[size_t(r)].empty()) continue;
        const HostInstance& hi = h->inst[r];
        const int64_t pb = h->instdev[r].pat_begin, pe = pb + hi.P;
        std::vector<uint32_t> nt(size_t(hi.P), 0u);  // hierarchy terms per pattern, as the lists count them
        for (int64_t p = 0; p < hi.P; ++p) {
            if (side64 && hi.tier[p] == 0) continue;
            for_each_term(hi, p, [&](int64_t, int kind, int64_t, uint32_t, int side) {
                if (!(kind == 3 && side == 1)) ++nt[size_t(p)];
            });
        }
        int64_t p = pb;
        while (p < pe) {
            int64_t q = p;
            uint32_t np = 0, ncat = 0, nv = 0, nterm = 0;
            std::vector<std::pair<int64_t, int64_t>> wl, wq;  // the item's weights, with pattern q
            while (q < pe) {
                const uint32_t u = h->hdr[q + 1].var_off - h->hdr[q].var_off;
                const uint32_t c = h->hdr[q + 1].cat_off - h->hdr[q].cat_off;
                const uint32_t t = nt[size_t(q - pb)];
                wq = wl;
                pack_weights(h, r, q, q + 1, wq);
                const uint32_t nw = uint32_t(wq.size());
                const uint32_t bytes = pack_layout<V>(np + 1, ncat + c, nv + u, nterm + t, nw).bytes +
                                       pack_sums_bytes<V>(np + 1, ncat + c) + pack_wtab_bytes<V>(nw) +
                                       pack_dtab_bytes<V>(np + 1);
                // operand codes below 2048, pattern index below 16, and the
                // list kernel's operand layout for the item capacity (which
                // list_item resolves the operands in)
                if (q > p && (bytes > kPackItemTarget<V> || np + 1 > uint32_t(kItemPats) ||
                              nv + u > uint32_t(h->chunk) || int(ncat + c) > ncat_cap))
                    break;
                ++np;
                ncat += c;
                nv += u;
                nterm += t;
                wl.swap(wq);
                ++q;
            }
            if (nterm > 65535u || nv > uint32_t(h->chunk) || int(ncat) > ncat_cap ||
                nv + 2 * ncat + np + 1 > 2048u)
                return fail(SA_ERR_UNSUPPORTED, "a pattern is larger than a pack item holds");
            ItemDesc d{};
            d.p0 = uint32_t(p);
            d.np = np;
            d.v0 = h->hdr[p].var_off;
            d.nv = nv;
            d.c0 = h->hdr[p].cat_off;
            d.ncat = ncat;
            d.nl = nv;      // variables the warp updates (the blob builder leaves out integrated ones)
            d.row0 = nterm;
            d.nw = uint32_t(wl.size());
            d.r0 = kPackItemMark;
            out.push_back(d);
            p = q;
        }
    }
    return SA_OK;
}

int build_lists(sa_heom* h) {
    h->items = template_items(h);
    if (h->packed) {
        const int rc0 = h->precision == SA_FP64 ? pack_items<double>(h, h->items) : pack_items<float>(h, h->items);
        if (rc0) return rc0;
        // items grouped by template, in the order of the representatives
        std::stable_sort(h->items.begin(), h->items.end(), [&](const ItemDesc& a, const ItemDesc& b) {
            return h->hdr[a.p0].inst < h->hdr[b.p0].inst;
        });
    }
    const size_t ni = h->items.size();
    std::vector<uint32_t> nrounds(ni + 1, 0);
    std::vector<uint64_t> nrows(ni + 1, 0);
#pragma omp parallel
    {
        ListItem W;
#pragma omp for schedule(dynamic, 64)
        for (int64_t c = 0; c < int64_t(ni); ++c) {
            if (h->items[c].r0 == kPackItemMark) continue;
            list_item(h, h->items[c], W);
            nrounds[c] = uint32_t((W.order.size() + 31) / 32);
            nrows[c] = list_item_rows(W);
        }
    }
    // exclusive prefix sums
    uint64_t rr = 0, rw = 0;
    for (size_t c = 0; c < ni; ++c) {
        const uint64_t a = nrounds[c], b = nrows[c];
        if (h->items[c].r0 != kPackItemMark) h->items[c].r0 = uint32_t(rr);
        nrounds[c] = uint32_t(rr);
        nrows[c] = rw;
        rr += a;
        rw += b;
    }
    if (rr >= (uint64_t(1) << 32) || rw >= (uint64_t(1) << 32))
        return fail(SA_ERR_UNSUPPORTED, "term lists exceed 32-bit row indices");
    nrounds[ni] = uint32_t(rr);
    nrows[ni] = rw;
    h->list_rows = rw;
    try {
        h->lvd.assign(size_t(rr) * 32, 0u);  // lane words by round: lane i of an item at r0 * 32 + i
        h->lvj.assign(size_t(rr) * 32, 0);
        h->rbase.assign(rr + 1, 0u);
        h->tidx.assign(rw * 32, 0u);
        h->tcid.assign(rw * 32, 0);
    } catch (const std::bad_alloc&) {
        return fail(SA_ERR_OOM, "host memory for the term lists");
    }
    h->rbase[rr] = uint32_t(rw);

#pragma omp parallel
    {
        ListItem W;
#pragma omp for schedule(dynamic, 64)
        for (int64_t c = 0; c < int64_t(ni); ++c) {
            ItemDesc& d = h->items[c];
            if (d.r0 == kPackItemMark) continue;
            list_item(h, d, W);
            const uint32_t nlane = uint32_t(W.order.size());
            d.nl = nlane;
            uint64_t row = nrows[c];
            d.row0 = uint32_t(row);
            d.row1 = uint32_t(nrows[c + 1]);

            uint32_t rho = nrounds[c];
            for (size_t i0 = 0; i0 < nlane; i0 += 32, ++rho) {
                h->rbase[rho] = uint32_t(row);
                const uint32_t T = W.cnt[W.order[i0]];
                for (uint32_t u = 0; u < 32; ++u) {
                    const size_t i = i0 + u;
                    const uint32_t l = i < nlane ? W.order[i] : 0u;
                    const uint32_t n = i < nlane ? W.cnt[l] : 0u;
                    if (i < nlane) {
                        h->lvd[size_t(d.r0) * 32 + i] = W.desc[l];
                        h->lvj[size_t(d.r0) * 32 + i] = W.cls[l];
                    }
                    for (uint32_t t = 0; t < T; ++t) {
                        const size_t e = size_t(row + t) * 32 + u;
                        if (t < n) {
                            h->tidx[e] = W.tix[W.off[l] + t];
                            h->tcid[e] = W.tsl[W.off[l] + t];
                        } else {  // the item's first variable, with the zero slot
                            h->tidx[e] = d.v0 - uint32_t(h->var_begin[h->hdr[d.p0].inst]);
                            h->tcid[e] = uint16_t(kListCoefZero);
                        }
                    }
                }
                row += T;
            }
        }
    }
    if (h->corrupt_list) {
        // SA_DEBUG_CORRUPT_LIST: the first real entry of the first term row
        // names a target beyond every instance
        bool done = false;
        for (size_t e = 0; e < h->tcid.size() && !done; ++e)
            if (h->tcid[e] != uint16_t(kListCoefZero)) {
                h->tidx[e] = 0x7fffffffu;
                done = true;
            }
        if (!done) return fail(SA_ERR_STATE, "SA_DEBUG_CORRUPT_LIST: no term row to corrupt");
    }
    const int rc = h->precision == SA_FP64 ? build_blobs<double>(h) : build_blobs<float>(h);
    if (rc) return rc;
    // template items relative to their instance; work units: a template's
    // items for one instance after another, or for one pack after another
    std::vector<uint32_t> first(size_t(h->count) + 1, 0);  // first template item of each representative
    {
        std::vector<uint32_t> nit(size_t(h->count), 0);
        for (ItemDesc& d : h->items) {
            const int r = h->hdr[d.p0].inst;
            ++nit[r];
            d.p0 -= h->instdev[r].pat_begin;
            d.v0 -= uint32_t(h->var_begin[r]);
            d.c0 -= h->hdr[h->instdev[r].pat_begin].cat_off;
        }
        for (int r = 0; r < h->count; ++r) first[r + 1] = first[r] + nit[r];
        // the instances of one template one after another, so that its lists
        // are read while they are in L2; each instance's items in order, so
        // that its tier +/-1 gathers stay near one another
        std::vector<std::vector<int>> members(size_t(h->count));
        for (int i = 0; i < h->count; ++i) members[size_t(h->tmpl[i])].push_back(i);
        h->units.clear();
        for (int r = 0; r < h->count; ++r) {
            for (int k : h->tmpl_packs[size_t(r)])
                for (uint32_t c = first[r]; c < first[r + 1]; ++c) {
                    if (h->items[c].r0 != kPackItemMark) continue;
                    h->units.push_back(c | kPackUnit);
                    h->units.push_back(uint32_t(k));
                }
            for (int i : members[size_t(r)]) {
                if (h->pack_of[size_t(i)] >= 0) continue;
                for (uint32_t c = first[r]; c < first[r + 1]; ++c) {
                    if (h->items[c].r0 == kPackItemMark) continue;
                    h->units.push_back(c);
                    h->units.push_back(uint32_t(i));
                }
            }
        }
        if (h->units.size() / 2 >= (size_t(1) << 32) || h->items.size() >= size_t(kPackUnit))
            return fail(SA_ERR_UNSUPPORTED, "too many work units");
    }
    h->list_items = h->items;
    return SA_OK;
}

// Per-instance constants of the list kernel.
template <typename V>
std::vector<InstK<V>> list_instk(const sa_heom* h) {
    std::vector<InstK<V>> out(size_t(h->count));
    const double lossf[5] = {0.0, 0.5, 0.5, 1.0, 0.0}, wt[5] = {2.0, 1.0, 1.0, 0.0, 0.0};
    for (int i = 0; i < h->count; ++i) {
        const sa_params& q = h->inst[i].p;
        InstK<V>& k = out[size_t(i)];
        k.var_base = h->instdev[i].dev_base;  // a list unit's instance is never packed: stride 1
        k.lcoef_base = h->instdev[i].lcoef_base;
        k.N = double(h->inst[i].N);
        k.g = V(q.g);
        k.pad = V(0);
        const double dim[5] = {0.0, -q.detuning, q.detuning, 0.0, 0.0};
        for (int cl = 0; cl < 5; ++cl) {
            k.cc[2 * cl] = V(-(lossf[cl] * q.kappa + wt[cl] * q.term));
            k.cc[2 * cl + 1] = V(dim[cl]);
        }
    }
    return out;
}

// ELL tables: warp w takes the variables 32 w .. 32 w + 31 in memory order.
// Per variable a word (pattern offset from the warp's first pattern | kind
// << 5 | q << 8 | r << 13 | T-rank of q << 18); per warp T_w rows of 32
// (target, coefficient slot) entries, T_w the longest list among its lanes,
// short lists padded with the zero slot.  The physical representative has no
// list in SA_FP32_AUX mode (the FP64 kernel integrates it).  Two parallel
// passes over the patterns (term counts, then contents).
int build_ell(sa_heom* h) {
    const int64_t nv = h->nvar, nw = (nv + 31) / 32, np = h->npat;
    const bool side64 = h->precision == SA_FP32_AUX;
    std::vector<uint32_t> cnt;
    try {
        cnt.assign(size_t(nw) * 32, 0u);
        h->wpat.assign(size_t(nw), 0u);
        h->lvd.assign(size_t(nv), 0u);
        h->rbase.assign(size_t(nw) + 1, 0u);
    } catch (const std::bad_alloc&) {
        return fail(SA_ERR_OOM, "host memory for the ELL tables");
    }
    auto each_term = [&](int64_t gp, auto&& fn) {
        const PatHdr& H = h->hdr[gp];
        if (side64 && H.tier == 0) return;
        const int inst = H.inst;
        const uint32_t vb = uint32_t(h->var_begin[inst]);
        for_each_term(h->inst[inst], gp - int64_t(h->instdev[inst].pat_begin),
                      [&](int64_t loc, int kind, int64_t src, uint32_t packed, int side) {
                          if (kind == 3 && side == 1) return;  // folded into the row term's coefficient
                          const int cid = int(packed >> 23);
                          const int slot = list_slot(h->inst[inst].L, cid, kind == 3 ? 2 : side);
                          fn(H.var_off + uint32_t(loc), vb + uint32_t(src), slot);
                      });
    };
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t gp = 0; gp < np; ++gp) each_term(gp, [&](uint32_t v, uint32_t, int) { ++cnt[v]; });
    // warps: first pattern, rows
#pragma omp parallel for schedule(static)
    for (int64_t w = 0; w < nw; ++w) {
        const uint32_t v = uint32_t(w * 32);
        int64_t lo = 0, hi = np - 1;  // last pattern with var_off <= v
        while (lo < hi) {
            const int64_t mid = (lo + hi + 1) / 2;
            if (h->hdr[mid].var_off <= v) lo = mid;
            else hi = mid - 1;
        }
        h->wpat[w] = uint32_t(lo);
        uint32_t T = 0;
        for (int u = 0; u < 32; ++u) T = std::max(T, cnt[size_t(w) * 32 + u]);
        h->rbase[w + 1] = T;
    }
    uint64_t rows = 0;
    for (int64_t w = 0; w < nw; ++w) {
        const uint64_t T = h->rbase[w + 1];
        h->rbase[w] = uint32_t(rows);
        rows += T;
        if (rows >= (uint64_t(1) << 32)) return fail(SA_ERR_UNSUPPORTED, "ELL tables exceed 32-bit row indices");
    }
    h->rbase[nw] = uint32_t(rows);
    h->list_rows = rows;
    try {
        h->tidx.assign(size_t(rows) * 32, 0u);
        h->tcid.assign(size_t(rows) * 32, uint16_t(kListCoefZero));
    } catch (const std::bad_alloc&) {
        return fail(SA_ERR_OOM, "host memory for the ELL tables");
    }
    // padding names the lane's own variable (any valid index would do)
#pragma omp parallel for schedule(static)
    for (int64_t w = 0; w < nw; ++w)
        for (uint32_t t = h->rbase[w]; t < h->rbase[w + 1]; ++t)
            for (int u = 0; u < 32; ++u) h->tidx[size_t(t) * 32 + u] = uint32_t(std::min<int64_t>(w * 32 + u, nv - 1));
#pragma omp parallel
    {
        std::vector<uint32_t> k;  // terms written per variable of the pattern
#pragma omp for schedule(dynamic, 256)
        for (int64_t gp = 0; gp < np; ++gp) {
            const PatHdr& H = h->hdr[gp];
            const uint32_t v0 = H.var_off, nvp = h->hdr[gp + 1].var_off - v0;
            const int G = H.G;
            auto word = [&](int64_t loc, uint32_t kind, int q, int r) {
                const uint32_t v = v0 + uint32_t(loc);
                const uint32_t trq = q ? (h->cat_word[H.cat_off + q - 1] >> 15) & 31u : 31u;
                h->lvd[v] = uint32_t(gp - h->wpat[v >> 5]) | (kind << 5) | (uint32_t(q) << 8) | (uint32_t(r) << 13) |
                            (trq << 18);
            };
            word(loc_Z(), 0, 0, 0);
            for (int q = 1; q <= G; ++q) {
                word(loc_X(G, q), 1, q, 0);
                word(loc_Y(G, q), 2, q, 0);
                word(loc_P(G, q), 3, q, 0);
                for (int r = 1; r <= G; ++r)
                    if (r != q) word(loc_S(G, q, r), 4, q, r);
                const int tr = (h->cat_word[H.cat_off + q - 1] >> 15) & 31;
                if (tr != 31) word(loc_T(G, tr), 5, q, 0);
            }
            k.assign(nvp, 0u);
            each_term(gp, [&](uint32_t v, uint32_t src, int slot) {
                const size_t e = (size_t(h->rbase[v >> 5]) + k[v - v0]++) * 32 + (v & 31u);
                h->tidx[e] = src;
                h->tcid[e] = uint16_t(slot);
            });
        }
    }
    return SA_OK;
}

// Decoded connection records: the batch-global indices the aligned accessor
// resolves to for each kind of variable, and the small remap fields.
void decode_records(sa_heom* h) {
    h->drecA.resize(h->rec.size());
    h->drecS.resize(h->rec.size());
    for (size_t i = 0; i < h->rec.size(); ++i) {
        const Record& R = h->rec[i];
        const uint32_t pk = R.packed;
        const int ts = pk & 31, Gp = (pk >> 5) & 31, tr = (pk >> 10) & 31;
        const int ipos = (pk >> 16) & 31, ins = (pk >> 21) & 1, del = (pk >> 22) & 1;
        const int cid = int(pk >> 23);
        const int smerge = ins ? 63 : ipos;
        const int t = int(R.target);
        h->drecA[i] = {t + ts, t + 3 * Gp + (ts - 1) * (Gp - 1), t + 3 * Gp + ts, t + (Gp + 1) * (Gp + 1) + tr};
        h->drecS[i] = uint32_t(del) | (uint32_t(ins) << 1) | (uint32_t(ipos) << 2) | (uint32_t(ts) << 7) |
                      (uint32_t(smerge) << 12) | (uint32_t(Gp) << 18) | (uint32_t(cid) << 23);
    }
}

// Coefficient tables of the list and ELL kernels, instance after instance
// (list_slot layout: zero, then row, column, row + column per (k, n, dir)).
template <typename V>
std::vector<V> list_coefficients(const sa_heom* h) {
    std::vector<V> t(size_t(2) * h->lcoef_total, V(0));
    for (int i = 0; i < h->count; ++i) {
        const HostInstance& hi = h->inst[i];
        V* o = &t[size_t(2) * h->instdev[i].lcoef_base];
        const double* r = &h->coef_row_d[size_t(2) * kCoefPerInst * i];
        const double* c = &h->coef_col_d[size_t(2) * kCoefPerInst * i];
        for (int k = 0; k < hi.m; ++k)
            for (int n = 0; n <= hi.L; ++n)
                for (int raise = 0; raise < 2; ++raise) {
                    const int cid = coef_id(k, n, raise);
                    for (int z = 0; z < 2; ++z) {
                        o[2 * list_slot(hi.L, cid, 0) + z] = V(r[2 * cid + z]);
                        o[2 * list_slot(hi.L, cid, 1) + z] = V(c[2 * cid + z]);
                        o[2 * list_slot(hi.L, cid, 2) + z] = V(r[2 * cid + z] + c[2 * cid + z]);
                    }
                }
    }
    return t;
}

// The packs' coefficient tables: slot s of lane j at cbase + s * n + j.
template <typename V>
std::vector<V> pack_coefficients(const sa_heom* h) {
    const std::vector<V> lc = list_coefficients<V>(h);
    std::vector<V> t(size_t(2) * h->pcoef_total, V(0));
    for (const PackDev& pk : h->packs)
        for (uint32_t j = 0; j < pk.n; ++j) {
            const int i = int(h->pk_inst[pk.lane0 + j]);
            const uint32_t ns = uint32_t(list_slots(h->inst[i].m, h->inst[i].L));
            for (uint32_t sl = 0; sl < ns; ++sl)
                for (int z = 0; z < 2; ++z)
                    t[size_t(2) * (pk.cbase + size_t(sl) * pk.n + j) + z] =
                        lc[size_t(2) * (h->instdev[i].lcoef_base + sl) + z];
        }
    return t;
}

void free_lists(sa_heom* h) {
    void** ptrs[] = {&h->d_lvd,   &h->d_lvj,   &h->d_rbase, &h->d_tidx,  &h->d_tcid,
                     &h->d_wpat,  &h->d_blobs, &h->d_units, &h->d_punits};
    for (void** p : ptrs) {
        if (*p) cudaFree(*p);
        *p = nullptr;
    }
    h->tables = -1;
}

// Term tables of the current variant: built (and, on a device handle,
// uploaded) unless the current ones already serve it.
int check_device(const sa_heom* h);

int ensure_tables(sa_heom* h) {
    const int k = h->kernel;
    if (k == SA_KERNEL_RECORDS) return SA_OK;
    if (h->tables == k && (k == SA_KERNEL_ELL || h->tables_chunk == h->chunk)) {
        if (k == SA_KERNEL_LISTS)  // the item table was rebuilt: same items, restore their rounds
            h->items = h->list_items;
        return SA_OK;
    }
    if (!h->host_only) free_lists(h);
    h->tables = -1;
    const bool lists = k == SA_KERNEL_LISTS;
    int rc = lists ? build_lists(h) : build_ell(h);
    if (rc) return rc;
    if (!h->host_only) {
        if (!h->d_lcoef)
            rc = h->precision == SA_FP64 ? upload(&h->d_lcoef, list_coefficients<double>(h))
                                         : upload(&h->d_lcoef, list_coefficients<float>(h));

        if (!rc && lists) rc = upload(&h->d_blobs, h->blobs);
        if (!rc && lists) {
            // list units and pack units apart, each in order
            std::vector<uint32_t> lu, pu;
            for (size_t u = 0; u < h->units.size(); u += 2) {
                std::vector<uint32_t>& dst = (h->units[u] & kPackUnit) ? pu : lu;
                dst.push_back(h->units[u]);
                dst.push_back(h->units[u + 1]);
            }
            h->n_list_units = uint32_t(lu.size() / 2);
            h->n_pack_units = uint32_t(pu.size() / 2);
            rc = upload(&h->d_units, lu);
            if (!rc) rc = upload(&h->d_punits, pu);
        }
        if (!rc && lists && !h->d_instk)
            rc = h->precision == SA_FP64 ? upload(&h->d_instk, list_instk<double>(h)) : upload(&h->d_instk, list_instk<float>(h));
        if (!rc && lists && h->packed && !h->packs.empty() && !h->d_pcoef) {
            rc = upload(&h->d_packs, h->packs);
            if (!rc) rc = upload(&h->d_pkinst, h->pk_inst);
            if (!rc)
                rc = h->precision == SA_FP64 ? upload(&h->d_pcoef, pack_coefficients<double>(h))
                                             : upload(&h->d_pcoef, pack_coefficients<float>(h));
        }

        if (!rc && k == SA_KERNEL_ELL) rc = upload(&h->d_lvd, h->lvd);
        if (!rc && k == SA_KERNEL_ELL) rc = upload(&h->d_wpat, h->wpat);
        if (!rc && k == SA_KERNEL_ELL) rc = upload(&h->d_rbase, h->rbase);
        if (!rc && k == SA_KERNEL_ELL && !h->d_catpat) {
            std::vector<uint32_t> cp(size_t(h->ncat));
            for (int64_t p = 0; p < h->npat; ++p)
                for (uint32_t c = h->hdr[p].cat_off; c < h->hdr[p + 1].cat_off; ++c) cp[c] = uint32_t(p);
            rc = upload(&h->d_catpat, cp);
        }
        if (!rc && k == SA_KERNEL_ELL && !h->d_sums) {
            const size_t bytes = size_t(2 * h->ncat + h->npat) * (h->precision == SA_FP64 ? 16 : 8);
            if (cudaMalloc(&h->d_sums, bytes) != cudaSuccess) rc = fail(SA_ERR_OOM, "grouped-sum scratch");
        }
        if (!rc) rc = upload(&h->d_tidx, h->tidx);
        if (!rc) rc = upload(&h->d_tcid, h->tcid);
        // the host copies are not needed again
        std::vector<uint32_t>().swap(h->lvd);
        std::vector<uint8_t>().swap(h->lvj);
        std::vector<uint32_t>().swap(h->tidx);
        std::vector<uint16_t>().swap(h->tcid);
        std::vector<uint32_t>().swap(h->wpat);
        std::vector<uint8_t>().swap(h->blobs);
        if (rc) {
            free_lists(h);
            return rc;
        }
    }
    h->tables = k;
    h->tables_chunk = h->chunk;
    return SA_OK;
}

int apply_tuning(sa_heom* h) {
    if (!h->host_only) {
        const int rc0 = check_device(h);
        if (rc0) return rc0;
    }
    if (h->packed && h->kernel != SA_KERNEL_LISTS)
        return fail(SA_ERR_UNSUPPORTED, "a handle built with SA_BUILD_PACK_INSTANCES runs the list kernel only");
    build_items(h);
    h->cfg.block = h->block;
    h->cfg.chunk = h->chunk;
    h->cfg.use_queue = h->use_queue;
    h->cfg.kernel = h->kernel;
    int rc = ensure_tables(h);
    if (rc) return rc;
    h->cfg.pack_smem = h->kernel == SA_KERNEL_LISTS ? int(h->pack_smem) : 0;
    // work the grid shares out: the list kernel's units, the other kernels' items
    if (h->host_only) return SA_OK;
    const uint64_t nchunks = h->kernel == SA_KERNEL_LISTS ? h->n_list_units : h->items.size();
    if (h->d_chunk) cudaFree(h->d_chunk);
    if (h->d_vdesc) cudaFree(h->d_vdesc);
    h->d_chunk = h->d_vdesc = nullptr;
    rc = upload(&h->d_chunk, h->items);
    if (!rc) rc = upload(&h->d_vdesc, h->vdesc);
    if (rc) return rc;
    int occ = 0;
    CK(stage_occupancy(h->cfg, h->precision == SA_FP64, &occ));
    if (occ < 1) return fail(SA_ERR_UNSUPPORTED, "stage kernel does not fit on an SM with this tuning (shared memory)");
    const int wpb = h->block / 32;
    const int64_t blocks_needed = (int64_t(nchunks) + wpb - 1) / wpb;
    // the list kernel is persistent in both modes (its warps pipeline their items)
    const bool persistent = h->use_queue || h->kernel == SA_KERNEL_LISTS;
    h->cfg.grid = persistent ? int(std::min<int64_t>(int64_t(h->num_sms) * occ, blocks_needed)) : int(blocks_needed);
    if (h->cfg.grid < 1) h->cfg.grid = 1;
    h->cfg.pgrid = 0;
    if (h->kernel == SA_KERNEL_LISTS && h->n_pack_units) {
        int pocc = 0;
        CK(pack_occupancy(h->cfg, h->precision == SA_FP64, &pocc));
        if (pocc < 1) return fail(SA_ERR_UNSUPPORTED, "pack kernel does not fit on an SM with this tuning (shared memory)");
        // (the pack kernel also runs the list units of the unpacked instances)
        const int64_t need = (int64_t(h->n_pack_units) + int64_t(h->n_list_units) + wpb - 1) / wpb;
        h->cfg.pgrid = int(std::max<int64_t>(1, std::min<int64_t>(int64_t(h->num_sms) * pocc, need)));
    }
    for (auto& kv : h->graphs) cudaGraphExecDestroy(kv.second);
    h->graphs.clear();
    return SA_OK;
}

void free_device(sa_heom* h) {
    for (auto& kv : h->graphs) cudaGraphExecDestroy(kv.second);
    h->graphs.clear();
    void* ptrs[] = {h->d_hdr, h->d_cat_word, h->d_catM, h->d_catMd, h->d_gamma, h->d_rec, h->d_inst, h->d_theta,
                    h->d_coef_row, h->d_coef_col, h->d_coef_row_d, h->d_coef_col_d, h->d_lut, h->d_lut_off,
                    h->d_chunk, h->d_work[0], h->d_work[1], h->d_work[2], h->d_queue, h->d_obs, h->d_rho0,
                    h->d_err, h->d_vdesc, h->d_drecA, h->d_drecS, h->d_lvd, h->d_lvj, h->d_rbase,
                    h->d_tidx, h->d_tcid, h->d_lcoef, h->d_wpat, h->d_blobs, h->d_catpat, h->d_sums,
                    h->d_rep_loc, h->d_recon_ws, h->d_units, h->d_instk, h->d_packs, h->d_pkinst, h->d_pcoef,
                    h->d_ilimit};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (h->cap) cudaStreamDestroy(h->cap);
    if (h->side) cudaStreamDestroy(h->side);
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->ev_join) cudaEventDestroy(h->ev_join);
}

int ensure_queue(sa_heom* h, size_t slots) {
    if (slots <= h->queue_slots) return SA_OK;
    if (h->d_queue) cudaFree(h->d_queue);
    h->d_queue = nullptr;
    size_t n = std::max<size_t>(slots, 64);
    CK(cudaMalloc(&h->d_queue, n * sizeof(unsigned int)));
    CK(cudaMemset(h->d_queue, 0, n * sizeof(unsigned int)));
    h->queue_slots = n;
    return SA_OK;
}

StageLaunch base_launch(const sa_heom* h) {
    StageLaunch s{};
    s.hdr = h->d_hdr;
    s.cat_word = h->d_cat_word;
    s.cat_M = h->d_catM;
    s.gamma = h->d_gamma;
    s.rec = h->d_rec;
    s.items = h->d_chunk;
    s.vdesc = h->d_vdesc;
    s.drecA = h->d_drecA;
    s.drecS = h->d_drecS;
    s.inst = h->d_inst;
    s.coef_row = h->d_coef_row;
    s.coef_col = h->d_coef_col;
    s.cat_Md = h->d_catMd;
    s.coef_row_d = h->d_coef_row_d;
    s.coef_col_d = h->d_coef_col_d;
    s.lut = h->d_lut;
    s.lut_off = h->d_lut_off;
    s.lvd = h->d_lvd;
    s.lvj = h->d_lvj;
    s.rbase = h->d_rbase;
    s.tidx = h->d_tidx;
    s.tcid = h->d_tcid;
    s.lcoef = h->d_lcoef;
    s.wpat = h->d_wpat;
    s.blobs = h->d_blobs;
    s.catpat = h->d_catpat;
    s.ncat = uint32_t(h->ncat);
    s.npat = uint32_t(h->npat);
    s.sums = h->d_sums;
    s.nvar = uint32_t(h->nvar);
    s.nchunks = uint32_t(h->kernel == SA_KERNEL_LISTS ? h->n_list_units : h->items.size());
    s.punits = h->d_punits;
    s.npunits = h->kernel == SA_KERNEL_LISTS ? h->n_pack_units : 0u;
    s.units = h->d_units;
    s.instk = h->d_instk;
    s.ilimit = h->d_ilimit;
    s.packs = h->d_packs;
    s.pk_inst = h->d_pkinst;
    s.pcoef = h->d_pcoef;
    s.err = h->d_err;
    s.debug = h->debug;
    s.ninst = h->count;
    s.side_stream = h->side;
    s.ev_fork = h->ev_fork;
    s.ev_join = h->ev_join;
    return s;
}

void* side(const sa_heom* h, const void* buf) {
    if (h->precision == SA_FP64 || !buf) return nullptr;
    return static_cast<char*>(const_cast<void*>(buf)) + h->side_off;
}

// observables of every instance's physical representative into d_out
cudaError_t observables_into(const sa_heom* h, const void* d_state, double* d_out, cudaStream_t st) {
    return launch_observables(static_cast<const InstDev*>(h->d_inst), static_cast<const double*>(h->d_theta),
                              h->count, static_cast<const PatHdr*>(h->d_hdr), static_cast<const double*>(h->d_catMd),
                              static_cast<const uint32_t*>(h->d_cat_word), h->precision == SA_FP64 ? d_state : nullptr,
                              side(h, d_state), d_out, st);
}

// The four fused RK4 stage launches of one step; slot: first queue counter.
// work counters of one RK4 step: stage s uses slot + s (list or record
// kernel) and slot + 4 + s (pack kernel)
constexpr int kQueuePerStep = 8;
int enqueue_step(sa_heom* h, void* y, double dt, size_t slot, cudaStream_t st) {
    void* acc = h->d_work[0];
    void* xa = h->d_work[1];
    void* xb = h->d_work[2];
    const void* xin[4] = {y, xa, xb, xa};
    void* xout[4] = {xa, xb, xa, nullptr};
    for (int s = 0; s < 4; ++s) {
        StageLaunch L = base_launch(h);
        L.x_in = xin[s];
        L.x_out = xout[s];
        L.y = y;
        L.acc = acc;
        L.y_out = y;
        L.xs_in = side(h, xin[s]);
        L.xs_out = side(h, xout[s]);
        L.ys = side(h, y);
        L.accs = side(h, acc);
        L.ys_out = side(h, y);
        L.dt = dt;
        L.stage = s;
        L.queue = h->d_queue + slot + s;
        L.pqueue = h->d_queue + slot + 4 + s;
        CK(launch_stage(L, h->cfg, h->precision == SA_FP64, st));
    }
    return SA_OK;
}

// the kernels' error word: bit 0 = a bounded wait on a bulk copy expired,
// bit 1 = a table index out of range (SA_DEBUG_CHECK_INDICES);
// reading it clears it
int read_device_error(sa_heom* h, cudaStream_t st) {
    unsigned int w = 0;
    CK(cudaMemcpyAsync(&w, h->d_err, sizeof(w), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (w) {
        CK(cudaMemsetAsync(h->d_err, 0, sizeof(w), st));
        CK(cudaStreamSynchronize(st));
        if (w & 1u) return fail(SA_ERR_TIMEOUT, "a bounded device wait expired in the stage kernel");
        return fail(SA_ERR_STATE, "a stage kernel found a table index out of range (SA_DEBUG_CHECK_INDICES)");
    }
    return SA_OK;
}

// the stage kernels copy state slices with 16-byte bulk copies
bool misaligned(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) != 0; }

// A device call needs a device-built handle and, current on the calling
// thread, the device the handle's tables live on: a launch with another
// device current would read them across devices.
int check_device(const sa_heom* h) {
    if (!h) return fail(SA_ERR_INVALID_ARG, "null handle");
    if (h->host_only) return fail(SA_ERR_STATE, "handle was built with SA_BUILD_HOST_ONLY");
    int dev = -1;
    const cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev != h->device)
        return fail(SA_ERR_STATE, "device " + std::to_string(dev) + " is current, the handle was built on device " +
                                      std::to_string(h->device));
    return SA_OK;
}

}  // namespace

extern "C" {

const char* sa_heom_strerror(int code) {
    switch (code) {
        case SA_OK: return "ok";
        case SA_ERR_INVALID_ARG: return "invalid argument";
        case SA_ERR_UNSUPPORTED: return "unsupported size or configuration";
        case SA_ERR_OOM: return "out of memory";
        case SA_ERR_CUDA: return "CUDA runtime error";
        case SA_ERR_TIMEOUT: return "bounded device wait expired";
        case SA_ERR_NUMERIC: return "non-finite observable";
        case SA_ERR_STATE: return "invalid handle state";
    }
    return "unknown error";
}

const char* sa_heom_last_error(void) { return g_err.c_str(); }

int sa_bath_drude_lorentz(double lambda, double gamma, double kT, int scheme, int n_poles, double sigma,
                          sa_params* p) {
    std::string err;
    int rc = drude_lorentz(lambda, gamma, kT, scheme, n_poles, sigma, p, err);
    if (rc) g_err = err;
    return rc;
}

int sa_bath_terminator(double lambda, double gamma, double kT, int n_matsubara, double* out) {
    std::string err;
    const int rc = terminator(lambda, gamma, kT, n_matsubara, out, err);
    if (rc) g_err = err;
    return rc;
}

static void fill_counts(const HostInstance& hi, int precision, sa_counts* out) {
    // log10 C(Nm+L, L) = sum_{j=1..L} log10((Nm + j) / j): no cancellation for
    // Nm up to 2^65 (a difference of lgamma values would lose it all)
    const long double nm = (long double)hi.N * hi.m;
    long double lg = 0.0L;
    for (int j = 1; j <= hi.L; ++j) lg += std::log10((nm + j) / (long double)j);
    out->log10_conventional_ados = double(lg);
    out->n_vectors = hi.V;
    out->n_patterns = hi.P;
    out->n_vars = int64_t(hi.var_off[hi.P]);
    out->n_categories = int64_t(hi.cat_vec.size());
    out->n_records = int64_t(hi.rec.size());
    out->n_terms = hi.n_terms;
    out->state_bytes = out->n_vars * (precision == SA_FP64 ? 16 : 8);
    // C(Nm+L, L) = prod_{j=1..L} (Nm + j) / j, exact while every partial
    // product fits (each prefix is itself a binomial coefficient)
    using u128 = unsigned __int128;
    const u128 n = u128(uint64_t(hi.N)) * uint64_t(hi.m);
    u128 c = 1;
    bool ok = true;
    for (int j = 1; j <= hi.L && ok; ++j) {
        const u128 f = n + uint64_t(j);
        if (c > ~u128(0) / f) {
            ok = false;
            break;
        }
        c = c * f / uint64_t(j);
        ok = c <= u128(~uint64_t(0));
    }
    out->conventional_ados = ok ? uint64_t(c) : 0;
}

int sa_heom_counts(const sa_params* p, sa_counts* out) {
    if (!p || !out) return fail(SA_ERR_INVALID_ARG, "null argument");
    HostInstance hi;
    std::string err;
    int rc = build_instance(*p, hi, err);
    if (rc) return fail(rc, err);
    fill_counts(hi, SA_FP64, out);
    return SA_OK;
}

int sa_heom_build(const sa_params* params, int count, int precision, int flags, sa_heom** out) {
    if (!params || !out || count < 1 || count > 65535 || (precision != SA_FP64 && precision != SA_FP32_AUX))
        return fail(SA_ERR_INVALID_ARG, "params, out, 1 <= count <= 65535 and a valid precision required");
    *out = nullptr;
    sa_heom* h = new (std::nothrow) sa_heom();
    if (!h) return fail(SA_ERR_OOM, "handle");
    if (flags & ~(SA_BUILD_HOST_ONLY | SA_BUILD_PACK_INSTANCES)) {
        delete h;
        return fail(SA_ERR_INVALID_ARG, "unknown build flag");
    }
    h->count = count;
    h->precision = precision;
    h->host_only = (flags & SA_BUILD_HOST_ONLY) != 0;
    h->packed = (flags & SA_BUILD_PACK_INSTANCES) != 0;
    h->inst.resize(count);
    for (int i = 0; i < count; ++i) {
        std::string err;
        int rc = build_instance(params[i], h->inst[i], err);
        if (rc) {
            delete h;
            return fail(rc, "instance " + std::to_string(i) + ": " + err);
        }
    }
    // ---- batch assembly
    h->var_begin.assign(count + 1, 0);
    for (int i = 0; i < count; ++i) {
        const HostInstance& hi = h->inst[i];
        h->var_begin[i + 1] = h->var_begin[i] + hi.var_off[hi.P];
        h->npat += hi.P;
        h->ncat += int64_t(hi.cat_vec.size());
        h->nrec += int64_t(hi.rec.size());
    }
    h->nvar = int64_t(h->var_begin[count]);
    if (h->nvar >= (int64_t(1) << 31) || h->nrec >= (int64_t(1) << 32) || h->ncat >= (int64_t(1) << 32)) {
        delete h;
        return fail(SA_ERR_UNSUPPORTED, "batch exceeds 32-bit table indices");
    }
    h->hdr.resize(h->npat + 1);
    h->cat_word.reserve(h->ncat);
    h->catMd.reserve(h->ncat);
    h->catMf.reserve(h->ncat);
    h->gamma_d.reserve(2 * h->npat);
    h->gamma_f.reserve(2 * h->npat);
    h->rec.reserve(h->nrec);
    h->instdev.resize(count);
    h->theta.resize(count);
    h->coef_row_d.assign(size_t(2) * kCoefPerInst * count, 0.0);
    h->coef_col_d.assign(size_t(2) * kCoefPerInst * count, 0.0);
    int64_t pbase = 0;
    for (int i = 0; i < count; ++i) {
        const HostInstance& hi = h->inst[i];
        const uint32_t vb = uint32_t(h->var_begin[i]);
        const uint32_t rb = uint32_t(h->rec.size()), cb = uint32_t(h->cat_word.size());
        for (int64_t p = 0; p < hi.P; ++p) {
            PatHdr& H = h->hdr[pbase + p];
            H.var_off = vb + uint32_t(hi.var_off[p]);
            H.rec_off = rb + hi.rec_off[p];
            H.cat_off = cb + hi.cat_off[p];
            H.inst = uint16_t(i);
            H.G = hi.G[p];
            H.tier = hi.tier[p];
            h->gamma_d.push_back(hi.gamma_re[p]);
            h->gamma_d.push_back(hi.gamma_im[p]);
            h->gamma_f.push_back(float(hi.gamma_re[p]));
            h->gamma_f.push_back(float(hi.gamma_im[p]));
            h->max_u = std::max<int>(h->max_u, int(hi.var_off[p + 1] - hi.var_off[p]));
        }
        for (size_t c = 0; c < hi.cat_vec.size(); ++c) {
            h->cat_word.push_back(hi.cat_word[c]);
            h->catMd.push_back(double(hi.cat_M[c]));
            h->catMf.push_back(float(hi.cat_M[c]));
        }
        for (const Record& r : hi.rec) h->rec.push_back(Record{vb + r.target, r.packed});
        InstDev& D = h->instdev[i];
        D.g = hi.p.g;
        D.detuning = hi.p.detuning;
        D.kappa = hi.p.kappa;
        D.N = double(hi.N);
        D.gf = float(hi.p.g);
        D.detf = float(hi.p.detuning);
        D.kappaf = float(hi.p.kappa);
        D.termf = float(hi.p.term);
        D.term = hi.p.term;
        D.coef_base = uint32_t(i) * kCoefPerInst;
        D.side = uint32_t(i) * kSideSlots;
        D.var_begin = vb;
        D.n_rho0 = uint32_t(hi.var_off[1] - hi.var_off[0]);
        if (D.n_rho0 > uint32_t(kSideSlots)) {
            delete h;
            return fail(SA_ERR_UNSUPPORTED, "physical representative larger than its FP64 side slots");
        }
        D.pat_begin = uint32_t(pbase);
        D.lcoef_base = uint32_t(h->lcoef_total);
        h->lcoef_total += uint64_t(list_slots(hi.m, hi.L));
        h->theta[i] = 0.5 * std::atan2(2.0 * hi.p.g * std::sqrt(double(hi.N)), -hi.p.detuning);
        std::copy(hi.coef_row.begin(), hi.coef_row.end(), h->coef_row_d.begin() + size_t(2) * kCoefPerInst * i);
        std::copy(hi.coef_col.begin(), hi.coef_col.end(), h->coef_col_d.begin() + size_t(2) * kCoefPerInst * i);
        pbase += hi.P;
    }
    PatHdr& S = h->hdr[h->npat];  // sentinel
    S.var_off = uint32_t(h->nvar);
    S.rec_off = uint32_t(h->nrec);
    S.cat_off = uint32_t(h->ncat);
    S.inst = 0;
    S.G = 0;
    S.tier = 0;
    h->coef_row_f.assign(h->coef_row_d.begin(), h->coef_row_d.end());
    h->coef_col_f.assign(h->coef_col_d.begin(), h->coef_col_d.end());
    build_lut(h);
    h->chunk = std::max(192, (h->max_u + 31) / 32 * 32);
    if (h->chunk > kMaxItemVars) {
        delete h;
        return fail(SA_ERR_UNSUPPORTED, "a pattern has more than 1024 unique variables");
    }
    decode_records(h);
    assign_templates(h);
    {
        const int rc = assign_packs(h);
        if (rc) {
            delete h;
            return rc;
        }
    }
    // state layout
    if (precision == SA_FP64) {
        h->state_bytes = (size_t(h->nvar) * 16 + 255) / 256 * 256;
        h->side_off = 0;
    } else {
        h->side_off = (size_t(h->nvar) * 8 + 255) / 256 * 256;
        h->state_bytes = h->side_off + size_t(count) * kSideSlots * 16;
    }
    if (h->host_only) {
        build_items(h);
        *out = h;
        return SA_OK;
    }
    // ---- device
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        delete h;
        return cuda_fail(e, "cudaGetDevice");
    }
    h->device = dev;
    cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, dev);
    int rc = SA_OK;
    const bool f64 = precision == SA_FP64;
    if (!rc) rc = upload(&h->d_hdr, h->hdr);
    if (!rc) rc = upload(&h->d_cat_word, h->cat_word);
    if (!rc) rc = f64 ? upload(&h->d_catM, h->catMd) : upload(&h->d_catM, h->catMf);
    if (!rc) rc = upload(&h->d_catMd, h->catMd);
    if (!rc) rc = f64 ? upload(&h->d_gamma, h->gamma_d) : upload(&h->d_gamma, h->gamma_f);
    if (!rc) rc = upload(&h->d_rec, h->rec);
    if (!rc) rc = upload(&h->d_inst, h->instdev);
    if (!rc) rc = upload(&h->d_theta, h->theta);
    if (!rc) rc = f64 ? upload(&h->d_coef_row, h->coef_row_d) : upload(&h->d_coef_row, h->coef_row_f);
    if (!rc) rc = f64 ? upload(&h->d_coef_col, h->coef_col_d) : upload(&h->d_coef_col, h->coef_col_f);
    if (!rc) rc = upload(&h->d_coef_row_d, h->coef_row_d);
    if (!rc) rc = upload(&h->d_coef_col_d, h->coef_col_d);
    if (!rc) rc = upload(&h->d_lut, h->lut);
    if (!rc) rc = upload(&h->d_drecA, h->drecA);
    if (!rc) rc = upload(&h->d_drecS, h->drecS);
    if (!rc) rc = upload(&h->d_lut_off, h->lut_off);
    if (!rc) {
        std::vector<uint32_t> lim(size_t(2) * count);
        for (int i = 0; i < count; ++i) {
            lim[size_t(2) * i] = uint32_t(h->var_begin[size_t(i) + 1] - h->var_begin[size_t(i)]);
            lim[size_t(2) * i + 1] = uint32_t(list_slots(h->inst[i].m, h->inst[i].L));
        }
        rc = upload(&h->d_ilimit, lim);
    }
    for (int w = 0; w < 3 && !rc; ++w) {
        e = cudaMalloc(&h->d_work[w], h->state_bytes);
        if (e != cudaSuccess) rc = (e == cudaErrorMemoryAllocation) ? fail(SA_ERR_OOM, "RK4 work buffers")
                                                                    : cuda_fail(e, "cudaMalloc(work)");
        else {
            e = cudaMemset(h->d_work[w], 0, h->state_bytes);
            if (e != cudaSuccess) rc = cuda_fail(e, "cudaMemset(work)");
        }
    }
    if (!rc) {
        e = cudaMalloc(&h->d_rho0, sizeof(double) * 2 * kSideSlots * count);
        if (e != cudaSuccess) rc = cuda_fail(e, "cudaMalloc(rho0)");
    }
    if (!rc) rc = ensure_queue(h, 64);
    if (!rc) {
        e = cudaMalloc(&h->d_err, 64);
        if (e == cudaSuccess) e = cudaMemset(h->d_err, 0, 64);
        if (e != cudaSuccess) rc = cuda_fail(e, "cudaMalloc(error word)");
    }
    if (!rc) {
        e = cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking);
        if (e == cudaSuccess && precision == SA_FP32_AUX) {
            e = cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming);
        }
        if (e != cudaSuccess) rc = cuda_fail(e, "cudaStreamCreate");
    }
    h->host_only = false;
    if (!rc) {
        rc = apply_tuning(h);
        // large items: fewer warps per block until the shared-memory image fits
        while (rc == SA_ERR_UNSUPPORTED && h->block > 64) {
            h->block /= 2;
            rc = apply_tuning(h);
        }
    }
    if (rc) {
        free_device(h);
        delete h;
        return rc;
    }
    *out = h;
    return SA_OK;
}

void sa_heom_destroy(sa_heom* h) {
    if (!h) return;
    if (!h->host_only) free_device(h);
    delete h;
}

int sa_heom_info(const sa_heom* h, int inst, sa_counts* out) {
    if (!h || !out || inst < -1 || inst >= h->count) return fail(SA_ERR_INVALID_ARG, "handle, instance, out");
    if (inst >= 0) {
        fill_counts(h->inst[inst], h->precision, out);
        return SA_OK;
    }
    sa_counts t{};
    double lmax = 0;
    for (int i = 0; i < h->count; ++i) {
        sa_counts c{};
        fill_counts(h->inst[i], h->precision, &c);
        t.n_vectors += c.n_vectors;
        t.n_patterns += c.n_patterns;
        t.n_vars += c.n_vars;
        t.n_categories += c.n_categories;
        t.n_records += c.n_records;
        t.n_terms += c.n_terms;
        lmax = std::max(lmax, c.log10_conventional_ados);
    }
    t.log10_conventional_ados = lmax;
    t.state_bytes = int64_t(h->state_bytes);
    t.conventional_ados = 0;
    bool exact = true;
    for (int i = 0; i < h->count; ++i) {
        sa_counts c{};
        fill_counts(h->inst[i], h->precision, &c);
        exact = exact && c.conventional_ados != 0;
        t.conventional_ados = std::max(t.conventional_ados, c.conventional_ados);
    }
    if (!exact) t.conventional_ados = 0;
    *out = t;
    return SA_OK;
}

int sa_heom_var_offset(const sa_heom* h, int inst, int64_t* out) {
    if (!h || !out || inst < 0 || inst > h->count) return fail(SA_ERR_INVALID_ARG, "handle, instance, out");
    *out = int64_t(h->var_begin[inst]);
    return SA_OK;
}

int sa_heom_dump_vectors(const sa_heom* h, int inst, uint8_t* comp) {
    if (!h || inst < 0 || inst >= h->count || !comp) return fail(SA_ERR_INVALID_ARG, "handle, instance, out");
    const HostInstance& hi = h->inst[inst];
    std::memcpy(comp, hi.comp.data(), size_t(hi.V) * hi.m);
    return SA_OK;
}

int sa_heom_dump_patterns(const sa_heom* h, int inst, int32_t* tier, int32_t* r, int32_t* G, int32_t* hcount,
                          int64_t* var_off, int64_t* cat_off, int32_t* ids) {
    if (!h || inst < 0 || inst >= h->count) return fail(SA_ERR_INVALID_ARG, "handle, instance");
    const HostInstance& hi = h->inst[inst];
    for (int64_t p = 0; p < hi.P; ++p) {
        int rp = int(hi.id_off[p + 1] - hi.id_off[p]);
        if (tier) tier[p] = hi.tier[p];
        if (r) r[p] = rp;
        if (G) G[p] = hi.G[p];
        if (hcount) hcount[p] = hi.h[p];
        if (var_off) var_off[p] = int64_t(hi.var_off[p]);
        if (cat_off) cat_off[p] = int64_t(hi.cat_off[p]);
        if (ids)
            for (int a = 0, w = hi.L + hi.d; a < w; ++a)
                ids[p * w + a] = a < rp ? int32_t(hi.ids[hi.id_off[p] + a]) : -1;
    }
    if (var_off) var_off[hi.P] = int64_t(hi.var_off[hi.P]);
    if (cat_off) cat_off[hi.P] = int64_t(hi.cat_off[hi.P]);
    return SA_OK;
}

int sa_heom_dump_categories(const sa_heom* h, int inst, int32_t* vec_id, int64_t* mult) {
    if (!h || inst < 0 || inst >= h->count) return fail(SA_ERR_INVALID_ARG, "handle, instance");
    const HostInstance& hi = h->inst[inst];
    for (size_t c = 0; c < hi.cat_vec.size(); ++c) {
        if (vec_id) vec_id[c] = int32_t(hi.cat_vec[c]);
        if (mult) mult[c] = hi.cat_M[c];
    }
    return SA_OK;
}

int sa_heom_dump_terms(const sa_heom* h, int inst, int64_t* var, int64_t* src, int32_t* k, int32_t* n,
                       int32_t* dir, int32_t* side_) {
    if (!h || inst < 0 || inst >= h->count || !var || !src || !k || !n || !dir || !side_)
        return fail(SA_ERR_INVALID_ARG, "handle, instance, outputs");
    expand_terms(h->inst[inst], var, src, k, n, dir, side_);
    return SA_OK;
}

int sa_heom_dump_coefficients(const sa_heom* h, int inst, double* row, double* col) {
    if (!h || inst < 0 || inst >= h->count || !row || !col) return fail(SA_ERR_INVALID_ARG, "handle, instance, outputs");
    const HostInstance& hi = h->inst[inst];
    std::copy(hi.coef_row.begin(), hi.coef_row.end(), row);
    std::copy(hi.coef_col.begin(), hi.coef_col.end(), col);
    return SA_OK;
}

int sa_heom_state_index(const sa_heom* h, int inst, int64_t var, int64_t* out) {
    if (!h || !out || inst < 0 || inst >= h->count) return fail(SA_ERR_INVALID_ARG, "handle, instance, out");
    const uint64_t nv = h->var_begin[size_t(inst) + 1] - h->var_begin[size_t(inst)];
    if (var < 0 || uint64_t(var) >= nv) return fail(SA_ERR_INVALID_ARG, "variable index out of range");
    const InstDev& D = h->instdev[size_t(inst)];
    *out = int64_t(D.dev_base) + var * int64_t(D.dev_stride);
    return SA_OK;
}

int sa_heom_dump_packs(const sa_heom* h, int64_t* sizes, uint32_t* packs, uint32_t* lanes, uint8_t* blobs) {
    if (!h || !sizes) return fail(SA_ERR_INVALID_ARG, "handle and sizes required");
    const bool have_blobs = h->host_only && h->tables == SA_KERNEL_LISTS;
    sizes[0] = int64_t(h->packs.size());
    sizes[1] = int64_t(h->pk_inst.size());
    sizes[2] = have_blobs ? int64_t(h->blobs.size()) : 0;
    if (packs)
        for (size_t k = 0; k < h->packs.size(); ++k) {
            const PackDev& pk = h->packs[k];
            const uint32_t f[4] = {pk.base, pk.n, pk.cbase, pk.lane0};
            std::memcpy(packs + 4 * k, f, sizeof(f));
        }
    if (lanes) std::copy(h->pk_inst.begin(), h->pk_inst.end(), lanes);
    if (blobs && have_blobs) std::copy(h->blobs.begin(), h->blobs.end(), blobs);
    return SA_OK;
}

int sa_heom_dump_lists(const sa_heom* h, int64_t* sizes, uint32_t* items, uint32_t* units, uint32_t* lvd,
                       uint8_t* lvj, uint32_t* rbase, uint32_t* tidx, uint16_t* tcid, int32_t* opz) {
    if (!h || !sizes) return fail(SA_ERR_INVALID_ARG, "handle and sizes required");
    if (!h->host_only || h->tables != SA_KERNEL_LISTS)
        return fail(SA_ERR_STATE, "term lists are kept on the host only for host-only handles, after "
                                  "sa_heom_set_kernel(h, SA_KERNEL_LISTS)");
    sizes[0] = int64_t(h->items.size());
    sizes[1] = int64_t(h->rbase.size()) - 1;
    sizes[2] = int64_t(h->list_rows);
    sizes[3] = int64_t(h->lvd.size());
    sizes[4] = int64_t(h->units.size() / 2);
    if (items)
        for (size_t c = 0; c < h->items.size(); ++c) {
            const ItemDesc& d = h->items[c];
            const uint32_t f[10] = {d.p0, d.np, d.v0, d.nv, d.c0, d.ncat, d.r0, d.nl, d.blob16, d.blob_bytes};
            std::memcpy(items + 10 * c, f, sizeof(f));
        }
    if (units) std::copy(h->units.begin(), h->units.end(), units);
    if (lvd) std::copy(h->lvd.begin(), h->lvd.end(), lvd);
    if (lvj) std::copy(h->lvj.begin(), h->lvj.end(), lvj);
    if (rbase) std::copy(h->rbase.begin(), h->rbase.end(), rbase);
    if (tidx) std::copy(h->tidx.begin(), h->tidx.end(), tidx);
    if (tcid) std::copy(h->tcid.begin(), h->tcid.end(), tcid);
    if (opz) list_operand_layout(h->chunk, &opz[0], &opz[1], &opz[2], &opz[3]);
    return SA_OK;
}

int sa_heom_dump_ell(const sa_heom* h, int64_t* sizes, uint32_t* wpat, uint32_t* vword, uint32_t* rbase,
                     uint32_t* tidx, uint16_t* tcid) {
    if (!h || !sizes) return fail(SA_ERR_INVALID_ARG, "handle and sizes required");
    if (!h->host_only || h->tables != SA_KERNEL_ELL)
        return fail(SA_ERR_STATE, "ELL tables are kept on the host only for host-only handles, after "
                                  "sa_heom_set_kernel(h, SA_KERNEL_ELL)");
    sizes[0] = int64_t(h->wpat.size());
    sizes[1] = int64_t(h->list_rows);
    sizes[2] = h->nvar;
    if (wpat) std::copy(h->wpat.begin(), h->wpat.end(), wpat);
    if (vword) std::copy(h->lvd.begin(), h->lvd.end(), vword);
    if (rbase) std::copy(h->rbase.begin(), h->rbase.end(), rbase);
    if (tidx) std::copy(h->tidx.begin(), h->tidx.end(), tidx);
    if (tcid) std::copy(h->tcid.begin(), h->tcid.end(), tcid);
    return SA_OK;
}

int sa_heom_state_bytes(const sa_heom* h, size_t* bytes) {
    if (!h || !bytes) return fail(SA_ERR_INVALID_ARG, "handle, out");
    *bytes = h->state_bytes;
    return SA_OK;
}

// ---- checkpoints ------------------------------------------------------------
// A checkpoint is a 64-byte header followed by the device state buffer as it
// is (float2 + FP64 side slots, or double2): magic, format version,
// precision, instance count, variables, state bytes, step index and a 64-bit
// FNV-1a hash of every instance's parameters and the table layout version,
// so a resume lands bit for bit on the same handle configuration.
namespace {
constexpr uint64_t kCkMagic = 0x4B434D4F45484153ull;  // "SAHEOMCK" in memory order
constexpr uint32_t kCkVersion = 1;
constexpr uint32_t kTableVersion = 3;  // bump when the canonical or device layout changes
struct CkHeader {
    uint64_t magic;
    uint32_t version, precision;
    int64_t count, nvar;
    uint64_t state_bytes;
    int64_t step;
    uint64_t hash;
    uint64_t pad;
};
static_assert(sizeof(CkHeader) == 64, "checkpoint header is 64 bytes");

uint64_t fnv1a(uint64_t h, const void* p, size_t n) {
    const unsigned char* b = static_cast<const unsigned char*>(p);
    for (size_t i = 0; i < n; ++i) {
        h ^= b[i];
        h *= 0x100000001b3ull;
    }
    return h;
}

uint64_t config_hash(const sa_heom* h) {
    uint64_t x = fnv1a(0xcbf29ce484222325ull, &kTableVersion, sizeof(kTableVersion));
    x = fnv1a(x, &h->precision, sizeof(h->precision));
    for (int i = 0; i < h->count; ++i) {
        const sa_params& p = h->inst[i].p;
        x = fnv1a(x, &p.N, sizeof(p.N));
        x = fnv1a(x, &p.m, sizeof(p.m));
        x = fnv1a(x, &p.L, sizeof(p.L));
        x = fnv1a(x, &p.d, sizeof(p.d));
        const double v[4] = {p.detuning, p.g, p.kappa, p.term};
        x = fnv1a(x, v, sizeof(v));
        x = fnv1a(x, p.c_re, sizeof(double) * size_t(p.m));
        x = fnv1a(x, p.c_im, sizeof(double) * size_t(p.m));
        x = fnv1a(x, p.cc_re, sizeof(double) * size_t(p.m));
        x = fnv1a(x, p.cc_im, sizeof(double) * size_t(p.m));
        x = fnv1a(x, p.nu_re, sizeof(double) * size_t(p.m));
        x = fnv1a(x, p.nu_im, sizeof(double) * size_t(p.m));
    }
    // the device layout: where every instance's variables lie
    for (const InstDev& D : h->instdev) {
        x = fnv1a(x, &D.dev_base, sizeof(D.dev_base));
        x = fnv1a(x, &D.dev_stride, sizeof(D.dev_stride));
    }
    return x;
}
}  // namespace

int sa_heom_config_hash(const sa_heom* h, uint64_t* out) {
    if (!h || !out) return fail(SA_ERR_INVALID_ARG, "handle, out");
    *out = config_hash(h);
    return SA_OK;
}

int sa_heom_checkpoint_bytes(const sa_heom* h, size_t* bytes) {
    if (!h || !bytes) return fail(SA_ERR_INVALID_ARG, "handle, out");
    *bytes = sizeof(CkHeader) + h->state_bytes;
    return SA_OK;
}

int sa_heom_checkpoint_save(const sa_heom* h, const void* d_state, int64_t step, void* host_buf, size_t bytes,
                            void* stream) {
    int rc = check_device(h);
    if (rc) return rc;
    if (!d_state || !host_buf || step < 0) return fail(SA_ERR_INVALID_ARG, "d_state, host_buf, step >= 0");
    if (bytes < sizeof(CkHeader) + h->state_bytes) return fail(SA_ERR_INVALID_ARG, "host_buf too small");
    CkHeader H{};
    H.magic = kCkMagic;
    H.version = kCkVersion;
    H.precision = uint32_t(h->precision);
    H.count = h->count;
    H.nvar = h->nvar;
    H.state_bytes = h->state_bytes;
    H.step = step;
    H.hash = config_hash(h);
    std::memcpy(host_buf, &H, sizeof(H));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    CK(cudaMemcpyAsync(static_cast<char*>(host_buf) + sizeof(H), d_state, h->state_bytes, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return SA_OK;
}

int sa_heom_checkpoint_load(const sa_heom* h, const void* host_buf, size_t bytes, void* d_state, int64_t* step,
                            void* stream) {
    int rc = check_device(h);
    if (rc) return rc;
    if (!d_state || !host_buf) return fail(SA_ERR_INVALID_ARG, "host_buf, d_state");
    if (bytes < sizeof(CkHeader)) return fail(SA_ERR_STATE, "checkpoint shorter than its header");
    CkHeader H;
    std::memcpy(&H, host_buf, sizeof(H));
    if (H.magic != kCkMagic || H.version != kCkVersion) return fail(SA_ERR_STATE, "not a checkpoint of this format");
    if (H.precision != uint32_t(h->precision) || H.count != h->count || H.nvar != h->nvar ||
        H.state_bytes != h->state_bytes)
        return fail(SA_ERR_STATE, "checkpoint precision or sizes differ from the handle's");
    if (H.hash != config_hash(h)) return fail(SA_ERR_STATE, "checkpoint parameters differ from the handle's");
    if (bytes < sizeof(CkHeader) + H.state_bytes) return fail(SA_ERR_STATE, "checkpoint truncated");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    CK(cudaMemcpyAsync(d_state, static_cast<const char*>(host_buf) + sizeof(H), h->state_bytes, cudaMemcpyHostToDevice,
                       st));
    CK(cudaStreamSynchronize(st));
    if (step) *step = H.step;
    return SA_OK;
}

// zero the state and write the physical representative of every instance
// from rho0 (stride doubles per instance, n_rho0 (re, im) pairs each)
static int init_from(sa_heom* h, const double* rho0, int stride, void* d_state, void* stream) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    std::vector<double> buf(size_t(2) * kSideSlots * h->count, 0.0);
    for (int i = 0; i < h->count; ++i)
        for (uint32_t j = 0; j < 2 * h->instdev[i].n_rho0; ++j) {
            const double v = rho0[size_t(stride) * i + j];
            if (!std::isfinite(v)) return fail(SA_ERR_INVALID_ARG, "non-finite initial value");
            buf[size_t(2) * kSideSlots * i + j] = v;
        }
    CK(cudaMemsetAsync(d_state, 0, h->state_bytes, st));
    CK(cudaMemcpyAsync(h->d_rho0, buf.data(), sizeof(double) * buf.size(), cudaMemcpyHostToDevice, st));
    // a copy from pageable memory returns once the source has been staged,
    // so the vector may die on return
    const int s = 2 * kSideSlots;
    if (h->precision == SA_FP64)
        CK(launch_init_rho0(static_cast<const InstDev*>(h->d_inst), h->count, h->d_rho0, s, d_state, nullptr, nullptr,
                            st));
    else
        CK(launch_init_rho0(static_cast<const InstDev*>(h->d_inst), h->count, h->d_rho0, s, nullptr, d_state,
                            side(h, d_state), st));
    return SA_OK;
}

int sa_heom_init_state(const sa_heom* hc, const double* rho0, void* d_state, void* stream) {
    sa_heom* h = const_cast<sa_heom*>(hc);
    int rc = check_device(h);
    if (rc) return rc;
    if (!rho0 || !d_state) return fail(SA_ERR_INVALID_ARG, "rho0 and d_state required");
    for (int i = 0; i < h->count; ++i)
        if (h->inst[i].d)
            return fail(SA_ERR_INVALID_ARG,
                        "instance " + std::to_string(i) + " has a distinguished molecule: use sa_heom_init_physical");
    return init_from(h, rho0, 10, d_state, stream);
}

int sa_heom_init_physical(const sa_heom* hc, const double* phys, void* d_state, void* stream) {
    sa_heom* h = const_cast<sa_heom*>(hc);
    int rc = check_device(h);
    if (rc) return rc;
    if (!phys || !d_state) return fail(SA_ERR_INVALID_ARG, "phys and d_state required");
    return init_from(h, phys, 2 * kSideSlots, d_state, stream);
}

// ---- arbitrary initial operators (Sec. IV, Table tab:representative-initial-operators)

int sa_heom_build_representatives(const sa_params* p, int precision, int flags, sa_heom** out) {
    if (!p || !out) return fail(SA_ERR_INVALID_ARG, "params and out required");
    if (p->d != 0) return fail(SA_ERR_INVALID_ARG, "representatives are built from a d = 0 parameter set");
    if (flags & ~(SA_BUILD_HOST_ONLY | SA_BUILD_ADJOINT_REPS)) return fail(SA_ERR_INVALID_ARG, "unknown build flag");
    const bool adj = (flags & SA_BUILD_ADJOINT_REPS) != 0;
    if (adj)
        for (int k = 0; k < p->m && k < SA_HEOM_MAXM; ++k)
            if (p->nu_im[k] != 0.0 || p->cc_re[k] != p->c_re[k] || p->cc_im[k] != -p->c_im[k])
                return fail(SA_ERR_INVALID_ARG, "the adjoint shortcut needs real nu_k and c-check_k = conj(c_k) "
                                                "(channel " + std::to_string(k) + ")");
    // the representatives |c><c| (d = 0), |e_1><c|, |c><e_1|, |e_1><e_1|
    // (d = 1), |e_1><e_2| (d = 2, N >= 2); with the adjoint shortcut the
    // |c><e_1| propagation is left out and its response is the adjoint of
    // the |e_1><c| one
    const int nrep = p->N >= 2 ? kReps : kReps - 1;
    int rinst[kReps];  // batch instance of each representative (-1: none)
    sa_params ps[kReps];
    int count = 0;
    const int dd[kReps] = {0, 1, 1, 1, 2};
    const int unit[kReps] = {RZ, RX1, RY1, RP1, RS12};
    std::vector<int> units;
    for (int r = 0; r < kReps; ++r) {
        rinst[r] = -1;
        if (r >= nrep || (adj && r == 2)) continue;
        ps[count] = *p;
        ps[count].d = dd[r];
        units.push_back(unit[r]);
        rinst[r] = count++;
    }
    int rc = sa_heom_build(ps, count, precision, flags & SA_BUILD_HOST_ONLY, out);
    if (rc) return rc;
    sa_heom* h = *out;
    h->reps = true;
    h->rep_unit = units;
    h->rep_src.assign(size_t(kReps) * kRepSlots, RepSrc{-1, 0, 0});
    // an adjoint response swaps the row and column labels: X <-> Y, S_qr <-> S_rq
    const int adjslot[kRepSlots] = {RZ, RY1, RY2, RY3, RX1, RX2, RX3, RP1, RP2, RP3,
                                    RS21, RS31, RS12, RS32, RS13, RS23, RT};
    for (int r = 0; r < nrep; ++r) {
        const bool via_adj = adj && r == 2;
        const int i = via_adj ? rinst[1] : rinst[r];
        const HostInstance& hi = h->inst[i];
        const int G = hi.G[0];
        int16_t loc[kRepSlots];
        for (int k = 0; k < kRepSlots; ++k) loc[k] = -1;
        loc[RZ] = int16_t(loc_Z());
        for (int q = 1; q <= std::min(G, 3); ++q) {
            loc[RX1 + q - 1] = int16_t(loc_X(G, q));
            loc[RY1 + q - 1] = int16_t(loc_Y(G, q));
            loc[RP1 + q - 1] = int16_t(loc_P(G, q));
        }
        const int sq[6][2] = {{1, 2}, {1, 3}, {2, 1}, {2, 3}, {3, 1}, {3, 2}};
        for (int k = 0; k < 6; ++k)
            if (sq[k][0] <= G && sq[k][1] <= G) loc[RS12 + k] = int16_t(loc_S(G, sq[k][0], sq[k][1]));
        if (hi.h[0] >= 1) loc[RT] = int16_t(loc_T(G, 0));  // only the others' category can hold two molecules
        for (int k = 0; k < kRepSlots; ++k) {
            RepSrc& S = h->rep_src[size_t(r) * kRepSlots + k];
            S.loc = loc[via_adj ? adjslot[k] : k];
            S.inst = int8_t(i);
            S.conj = via_adj ? 1 : 0;
        }
    }
    if (!h->host_only) {
        cudaError_t e = cudaMalloc(&h->d_rep_loc, h->rep_src.size() * sizeof(RepSrc));
        if (e == cudaSuccess)
            e = cudaMemcpy(h->d_rep_loc, h->rep_src.data(), h->rep_src.size() * sizeof(RepSrc), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            sa_heom_destroy(h);
            *out = nullptr;
            return cuda_fail(e, "representative table");
        }
    }
    return SA_OK;
}

int sa_heom_init_representatives(const sa_heom* hc, void* d_state, void* stream) {
    sa_heom* h = const_cast<sa_heom*>(hc);
    int rc = check_device(h);
    if (rc) return rc;
    if (!h->reps) return fail(SA_ERR_STATE, "not a representatives handle");
    if (!d_state) return fail(SA_ERR_INVALID_ARG, "d_state required");
    // the unit operator of each propagated representative: Z, X_1, Y_1, P_1 or S_12
    std::vector<double> phys(size_t(2) * kSideSlots * h->count, 0.0);
    for (int i = 0; i < h->count; ++i) {
        const HostInstance& hi = h->inst[i];
        const int G = hi.G[0];
        int64_t l = 0;
        switch (h->rep_unit[i]) {
            case RZ: l = loc_Z(); break;
            case RX1: l = loc_X(G, 1); break;
            case RY1: l = loc_Y(G, 1); break;
            case RP1: l = loc_P(G, 1); break;
            default: l = loc_S(G, 1, 2); break;
        }
        phys[size_t(2) * kSideSlots * i + 2 * l] = 1.0;
    }
    return init_from(h, phys.data(), 2 * kSideSlots, d_state, stream);
}

int sa_heom_reconstruct_dense(sa_heom* h, const void* d_state, const void* d_rho0, void* d_rho_t, void* stream) {
    int rc = check_device(h);
    if (rc) return rc;
    if (!h->reps) return fail(SA_ERR_STATE, "not a representatives handle");
    if (!d_state || !d_rho0 || !d_rho_t || d_rho0 == d_rho_t)
        return fail(SA_ERR_INVALID_ARG, "d_state, d_rho0 and d_rho_t required, rho0 and rho_t distinct");
    if ((reinterpret_cast<uintptr_t>(d_rho0) | reinterpret_cast<uintptr_t>(d_rho_t)) & 15)
        return fail(SA_ERR_INVALID_ARG, "rho0 and rho_t must be 16-byte aligned");
    const int64_t n = h->inst[0].N + 1;
    // the output grid has (n / 32)^2 CTAs, at most 32768 per dimension
    if (n > (int64_t(1) << 20)) return fail(SA_ERR_UNSUPPORTED, "dense output beyond N + 1 = 2^20");
    const size_t need = recon_workspace_bytes(n);
    if (need > h->recon_ws) {
        if (h->d_recon_ws) cudaFree(h->d_recon_ws);
        h->d_recon_ws = nullptr;
        h->recon_ws = 0;
        cudaError_t e = cudaMalloc(&h->d_recon_ws, need);
        if (e != cudaSuccess)
            return e == cudaErrorMemoryAllocation ? fail(SA_ERR_OOM, "reconstruction workspace") : cuda_fail(e, "cudaMalloc");
        h->recon_ws = need;
    }
    CK(launch_reconstruct(static_cast<const InstDev*>(h->d_inst), static_cast<const RepSrc*>(h->d_rep_loc),
                          h->precision == SA_FP64 ? d_state : nullptr, side(h, d_state), d_rho0, n, d_rho_t,
                          h->d_recon_ws, static_cast<cudaStream_t>(stream)));
    return SA_OK;
}

int sa_heom_state_upload(const sa_heom* h, const double* host_x, void* d_state, void* stream) {
    int rc = check_device(h);
    if (rc) return rc;
    if (!host_x || !d_state) return fail(SA_ERR_INVALID_ARG, "host_x and d_state required");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const bool f64 = h->precision == SA_FP64;
    if (f64 && !h->packed) {
        CK(cudaMemcpyAsync(d_state, host_x, size_t(h->nvar) * 16, cudaMemcpyHostToDevice, st));
        CK(cudaStreamSynchronize(st));
        return SA_OK;
    }
    // SA_FP32_AUX, or a packed layout: the complex128 values go to the device
    // as they are, in chunks through the two RK4 stage-input work vectors
    // (scratch between steps), and a kernel narrows or places them there
    const uint64_t per = h->state_bytes / 16;
    for (uint64_t n0 = 0, c = 0; n0 < uint64_t(h->nvar); n0 += per, ++c) {
        const uint64_t cnt = std::min<uint64_t>(per, uint64_t(h->nvar) - n0);
        void* stage = h->d_work[1 + (c & 1)];
        CK(cudaMemcpyAsync(stage, host_x + 2 * n0, cnt * 16, cudaMemcpyHostToDevice, st));
        CK(launch_marshal(static_cast<const InstDev*>(h->d_inst), h->count, h->packed ? 1 : 0, n0, cnt, stage,
                          d_state, f64 ? nullptr : side(h, d_state), f64 ? 1 : 0, 1, st));
    }
    CK(cudaStreamSynchronize(st));
    return SA_OK;
}

int sa_heom_state_download(const sa_heom* h, const void* d_state, double* host_x, void* stream) {
    int rc = check_device(h);
    if (rc) return rc;
    if (!host_x || !d_state) return fail(SA_ERR_INVALID_ARG, "host_x and d_state required");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const bool f64 = h->precision == SA_FP64;
    if (f64 && !h->packed) {
        CK(cudaMemcpyAsync(host_x, d_state, size_t(h->nvar) * 16, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        return SA_OK;
    }
    // SA_FP32_AUX, or a packed layout: widened (or gathered) to complex128 in
    // canonical order on the device, chunk by chunk in the two RK4
    // stage-input work vectors, then copied to the caller's buffer
    const uint64_t per = h->state_bytes / 16;
    for (uint64_t n0 = 0, c = 0; n0 < uint64_t(h->nvar); n0 += per, ++c) {
        const uint64_t cnt = std::min<uint64_t>(per, uint64_t(h->nvar) - n0);
        void* stage = h->d_work[1 + (c & 1)];
        CK(launch_marshal(static_cast<const InstDev*>(h->d_inst), h->count, h->packed ? 1 : 0, n0, cnt, stage,
                          const_cast<void*>(d_state), f64 ? nullptr : side(h, const_cast<void*>(d_state)),
                          f64 ? 1 : 0, 0, st));
        CK(cudaMemcpyAsync(host_x + 2 * n0, stage, cnt * 16, cudaMemcpyDeviceToHost, st));
    }
    CK(cudaStreamSynchronize(st));
    return SA_OK;
}

int sa_heom_rhs(sa_heom* h, const void* d_x, void* d_dx, void* stream) {
    int rc = check_device(h);
    if (rc) return rc;
    if (!d_x || !d_dx || d_x == d_dx) return fail(SA_ERR_INVALID_ARG, "distinct d_x and d_dx required");
    if (misaligned(d_x) || misaligned(d_dx)) return fail(SA_ERR_INVALID_ARG, "state buffers must be 16-byte aligned");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    CK(cudaMemsetAsync(h->d_queue, 0, 2 * sizeof(unsigned int), st));
    StageLaunch L = base_launch(h);
    L.x_in = d_x;
    L.x_out = d_dx;
    L.xs_in = side(h, d_x);
    L.xs_out = side(h, d_dx);
    L.stage = -1;
    L.queue = h->d_queue;
    L.pqueue = h->d_queue + 1;
    CK(launch_stage(L, h->cfg, h->precision == SA_FP64, st));
    return SA_OK;
}

int sa_heom_step(sa_heom* h, void* d_state, double dt, void* stream) {
    int rc = check_device(h);
    if (rc) return rc;
    if (!d_state || !std::isfinite(dt)) return fail(SA_ERR_INVALID_ARG, "d_state and finite dt required");
    if (misaligned(d_state)) return fail(SA_ERR_INVALID_ARG, "state buffers must be 16-byte aligned");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    CK(cudaMemsetAsync(h->d_queue, 0, kQueuePerStep * sizeof(unsigned int), st));
    return enqueue_step(h, d_state, dt, 0, st);
}

static int graph_for(sa_heom* h, void* d_state, double dt, int64_t steps, cudaGraphExec_t* out) {
    uint64_t dtb;
    std::memcpy(&dtb, &dt, 8);
    auto key = std::make_tuple(static_cast<const void*>(d_state), dtb, steps);
    auto it = h->graphs.find(key);
    if (it != h->graphs.end()) {
        *out = it->second;
        return SA_OK;
    }
    int rc = ensure_queue(h, size_t(kQueuePerStep * steps));
    if (rc) return rc;
    CK(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaMemsetAsync(h->d_queue, 0, sizeof(unsigned int) * kQueuePerStep * steps, h->cap);
    for (int64_t s = 0; s < steps && e == cudaSuccess && rc == SA_OK; ++s)
        rc = enqueue_step(h, d_state, dt, size_t(kQueuePerStep * s), h->cap);
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(h->cap, &g);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(queue) in capture");
    if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamEndCapture");
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    if (h->graphs.size() > 16) {
        for (auto& kv : h->graphs) cudaGraphExecDestroy(kv.second);
        h->graphs.clear();
    }
    h->graphs[key] = ex;
    *out = ex;
    return SA_OK;
}

static int run_steps(sa_heom* h, void* d_state, double dt, int64_t n, cudaStream_t st) {
    const int64_t kGraphSteps = 64;
    while (n > 0) {
        int64_t s = std::min(n, kGraphSteps);
        cudaGraphExec_t ex;
        int rc = graph_for(h, d_state, dt, s, &ex);
        if (rc) return rc;
        CK(cudaGraphLaunch(ex, st));
        n -= s;
    }
    return SA_OK;
}

int sa_heom_prepare(sa_heom* h, void* d_state, double dt, int64_t nsteps, int64_t obs_every) {
    int rc = check_device(h);
    if (rc) return rc;
    if (!d_state || !std::isfinite(dt) || nsteps < 0) return fail(SA_ERR_INVALID_ARG, "d_state, dt, nsteps");
    if (misaligned(d_state)) return fail(SA_ERR_INVALID_ARG, "state buffers must be 16-byte aligned");
    // the run lengths run_steps asks for: 64-step graphs and the remainder of
    // every observation interval
    const int64_t seg = obs_every > 0 ? std::min(obs_every, std::max<int64_t>(nsteps, 1)) : nsteps;
    std::vector<int64_t> lens;
    auto add = [&](int64_t n) {
        if (n >= 64) lens.push_back(64);
        if (n % 64) lens.push_back(n % 64);
    };
    if (nsteps > 0) {
        add(seg);
        if (obs_every > 0 && nsteps % seg) add(nsteps % seg);
    }
    std::sort(lens.begin(), lens.end());
    lens.erase(std::unique(lens.begin(), lens.end()), lens.end());
    for (int64_t n : lens) {
        cudaGraphExec_t ex;
        rc = graph_for(h, d_state, dt, n, &ex);
        if (rc) return rc;
    }
    return SA_OK;
}

int sa_heom_propagate(sa_heom* h, void* d_state, double dt, int64_t nsteps, int64_t obs_every, double* h_obs,
                      void* stream) {
    int rc = check_device(h);
    if (rc) return rc;
    if (!d_state || !std::isfinite(dt) || nsteps < 0) return fail(SA_ERR_INVALID_ARG, "d_state, dt, nsteps");
    if (misaligned(d_state)) return fail(SA_ERR_INVALID_ARG, "state buffers must be 16-byte aligned");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (!h_obs) return run_steps(h, d_state, dt, nsteps, st);
    if (obs_every <= 0) obs_every = std::max<int64_t>(nsteps, 1);
    const int64_t rows = 1 + (nsteps + obs_every - 1) / obs_every;
    const size_t need = size_t(rows) * h->count * 8;
    if (need > h->obs_cap) {
        if (h->d_obs) cudaFree(h->d_obs);
        h->d_obs = nullptr;
        CK(cudaMalloc(&h->d_obs, need * sizeof(double)));
        h->obs_cap = need;
    }
    CK(observables_into(h, d_state, h->d_obs, st));
    int64_t done = 0, row = 1;
    while (done < nsteps) {
        int64_t n = std::min(obs_every, nsteps - done);
        rc = run_steps(h, d_state, dt, n, st);
        if (rc) return rc;
        CK(observables_into(h, d_state, h->d_obs + size_t(row) * h->count * 8, st));
        done += n;
        ++row;
    }
    CK(cudaMemcpyAsync(h_obs, h->d_obs, need * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    rc = read_device_error(h, st);
    if (rc) return rc;
    for (size_t j = 0; j < need; ++j)
        if (!std::isfinite(h_obs[j])) return fail(SA_ERR_NUMERIC, "non-finite observable");
    return SA_OK;
}

int sa_heom_observables(sa_heom* h, const void* d_state, double* out, void* stream) {
    int rc = check_device(h);
    if (rc) return rc;
    if (!d_state || !out) return fail(SA_ERR_INVALID_ARG, "d_state and out required");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t need = size_t(h->count) * 8;
    if (need > h->obs_cap) {
        if (h->d_obs) cudaFree(h->d_obs);
        h->d_obs = nullptr;
        CK(cudaMalloc(&h->d_obs, need * sizeof(double)));
        h->obs_cap = need;
    }
    CK(observables_into(h, d_state, h->d_obs, st));
    CK(cudaMemcpyAsync(out, h->d_obs, need * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    for (size_t j = 0; j < need; ++j)
        if (!std::isfinite(out[j])) return fail(SA_ERR_NUMERIC, "non-finite observable");
    return SA_OK;
}

int sa_heom_set_tuning(sa_heom* h, int block, int chunk, int queue) {
    if (!h) return fail(SA_ERR_INVALID_ARG, "null handle");
    int nb = block > 0 ? block : h->block;
    int nc = chunk > 0 ? chunk : h->chunk;
    int nq = queue >= 0 ? queue : h->use_queue;
    if (nb < 64 || nb > 256 || nb % 32) return fail(SA_ERR_INVALID_ARG, "block must be 64..256, multiple of 32");
    if (nc % 32 || nc < h->max_u || nc > kMaxItemVars)
        return fail(SA_ERR_INVALID_ARG, "chunk must be a multiple of 32 between the largest pattern and 1024");
    h->block = nb;
    h->chunk = nc;
    h->use_queue = nq ? 1 : 0;
    return apply_tuning(h);
}

int sa_heom_set_kernel(sa_heom* h, int kernel) {
    if (!h) return fail(SA_ERR_INVALID_ARG, "null handle");
    if (kernel != SA_KERNEL_RECORDS && kernel != SA_KERNEL_LISTS && kernel != SA_KERNEL_ELL)
        return fail(SA_ERR_INVALID_ARG, "kernel must be SA_KERNEL_RECORDS, SA_KERNEL_LISTS or SA_KERNEL_ELL");
    const int old = h->kernel;
    h->kernel = kernel;
    const int rc = apply_tuning(h);
    if (rc && rc != SA_ERR_INVALID_ARG) {
        // keep the handle usable with the variant it had
        const std::string why = g_err;
        h->kernel = old;
        apply_tuning(h);
        g_err = why;
    }
    return rc;
}

int sa_heom_get_tuning(const sa_heom* h, int* out) {
    if (!h || !out) return fail(SA_ERR_INVALID_ARG, "handle and out required");
    out[0] = h->block;
    out[1] = h->chunk;
    out[2] = h->use_queue;
    out[3] = h->kernel;
    return SA_OK;
}

// ---- tuning cache: key -> (block, chunk, queue, kernel), process-wide
namespace {
std::mutex g_tune_mu;
std::map<uint64_t, std::array<int, 4>> g_tune;

// The cache key of a handle: the device (name and SM count; none for a
// host-only handle), precision, layout, the largest pattern, the variable
// count rounded down to a power of two, and the multiset of (m, L, d) of its
// instances.
uint64_t tuning_key(const sa_heom* h) {
    uint64_t x = 0xcbf29ce484222325ull;
    if (!h->host_only) {
        cudaDeviceProp prop{};
        if (cudaGetDeviceProperties(&prop, h->device) == cudaSuccess)
            x = fnv1a(x, prop.name, std::strlen(prop.name));
        x = fnv1a(x, &h->num_sms, sizeof(h->num_sms));
    }
    const int v[4] = {h->precision, h->packed ? 1 : 0, h->max_u, int(std::floor(std::log2(double(h->nvar))))};
    x = fnv1a(x, v, sizeof(v));
    std::map<std::array<int, 3>, int> shapes;
    for (const HostInstance& hi : h->inst) ++shapes[{hi.m, hi.L, hi.d}];
    for (const auto& kv : shapes) {
        x = fnv1a(x, kv.first.data(), sizeof(int) * 3);
        x = fnv1a(x, &kv.second, sizeof(int));
    }
    return x;
}
}  // namespace

int sa_heom_tuning_key(const sa_heom* h, uint64_t* out) {
    if (!h || !out) return fail(SA_ERR_INVALID_ARG, "handle, out");
    *out = tuning_key(h);
    return SA_OK;
}

int sa_heom_tuning_cache_clear(void) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune.clear();
    return SA_OK;
}

int sa_heom_tuning_cache_size(int64_t* out) {
    if (!out) return fail(SA_ERR_INVALID_ARG, "out");
    std::lock_guard<std::mutex> lk(g_tune_mu);
    *out = int64_t(g_tune.size());
    return SA_OK;
}

int sa_heom_tuning_cache_save(const char* path) {
    if (!path) return fail(SA_ERR_INVALID_ARG, "path");
    std::lock_guard<std::mutex> lk(g_tune_mu);
    FILE* f = std::fopen(path, "w");
    if (!f) return fail(SA_ERR_INVALID_ARG, std::string("cannot write ") + path);
    for (const auto& kv : g_tune)
        std::fprintf(f, "%016llx %d %d %d %d\n", static_cast<unsigned long long>(kv.first), kv.second[0],
                     kv.second[1], kv.second[2], kv.second[3]);
    const bool ok = std::fclose(f) == 0;
    return ok ? SA_OK : fail(SA_ERR_INVALID_ARG, std::string("cannot write ") + path);
}

int sa_heom_tuning_cache_load(const char* path) {
    if (!path) return fail(SA_ERR_INVALID_ARG, "path");
    FILE* f = std::fopen(path, "r");
    if (!f) return fail(SA_ERR_INVALID_ARG, std::string("cannot read ") + path);
    std::map<uint64_t, std::array<int, 4>> got;
    unsigned long long k = 0;
    int b = 0, c = 0, q = 0, kern = 0, n = 0;
    while ((n = std::fscanf(f, "%llx %d %d %d %d", &k, &b, &c, &q, &kern)) == 5) {
        if (b < 64 || b > 256 || b % 32 || c < 32 || c > kMaxItemVars || c % 32 || (q != 0 && q != 1) ||
            (kern != SA_KERNEL_RECORDS && kern != SA_KERNEL_LISTS && kern != SA_KERNEL_ELL)) {
            std::fclose(f);
            return fail(SA_ERR_INVALID_ARG, std::string("malformed tuning entry in ") + path);
        }
        got[uint64_t(k)] = {b, c, q, kern};
    }
    const bool eof = n == EOF;
    std::fclose(f);
    if (!eof) return fail(SA_ERR_INVALID_ARG, std::string("malformed tuning cache ") + path);
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (const auto& kv : got) g_tune[kv.first] = kv.second;
    return SA_OK;
}

int sa_heom_autotune(sa_heom* h, void* d_state, void* stream, int* best) {
    return sa_heom_autotune_ex(h, d_state, stream, 0, best);
}

int sa_heom_autotune_ex(sa_heom* h, void* d_state, void* stream, int flags, int* best) {
    int rc = check_device(h);
    if (rc) return rc;
    if (!d_state) return fail(SA_ERR_INVALID_ARG, "d_state required");
    if (misaligned(d_state)) return fail(SA_ERR_INVALID_ARG, "state buffers must be 16-byte aligned");
    if (flags & ~SA_TUNE_FORCE) return fail(SA_ERR_INVALID_ARG, "unknown autotune flag");
    const uint64_t key = tuning_key(h);
    if (!(flags & SA_TUNE_FORCE)) {
        std::array<int, 4> t{};
        bool hit = false;
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            auto it = g_tune.find(key);
            if (it != g_tune.end()) {
                t = it->second;
                hit = true;
            }
        }
        if (hit && !(h->packed && t[3] != SA_KERNEL_LISTS)) {
            const int old = h->kernel;
            h->kernel = t[3];
            rc = sa_heom_set_tuning(h, t[0], t[1], t[2]);
            if (!rc) {
                if (best) {
                    best[0] = t[0];
                    best[1] = t[1];
                    best[2] = t[2];
                }
                return SA_OK;
            }
            h->kernel = old;  // the cached tuning does not fit this handle: time afresh
            apply_tuning(h);
        }
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int blocks[] = {128, 256};
    const int chunks[] = {64, 96, 128, 160, 192, 224, 256};
    // (items smaller than the largest pattern or above the shared-memory
    // budget are skipped by set_tuning)
    struct Cand {
        float ms;
        int k, c, b, q;
    };
    std::vector<Cand> cands;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    // ms per RK4 step of the current tuning: two warm-up steps, then `reps`
    // (through the CUDA graph of `reps` steps that sa_heom_propagate replays:
    // the first run builds and warms it, the second is timed)
    auto time_steps = [&](int reps, float* ms) -> int {
        int r = run_steps(h, d_state, 0.0, reps, st);
        if (r) return r;
        CK(cudaEventRecord(e0, st));
        r = run_steps(h, d_state, 0.0, reps, st);
        if (r) return r;
        CK(cudaEventRecord(e1, st));
        CK(cudaEventSynchronize(e1));
        CK(cudaEventElapsedTime(ms, e0, e1));
        *ms /= float(reps);
        return SA_OK;
    };
    // a first pass over every tuning; item size outermost, since the list
    // kernel's tables are rebuilt per item size only
    for (int k : {int(SA_KERNEL_RECORDS), int(SA_KERNEL_LISTS), int(SA_KERNEL_ELL)})
        for (int c : chunks)
            for (int b : blocks)
                for (int q = 0; q < 2; ++q) {
                    if (c < h->max_u) continue;
                    if (h->packed && k != SA_KERNEL_LISTS) continue;  // a packed layout runs the list kernel only
                    // the ELL kernel has neither work items nor a queue
                    if (k == SA_KERNEL_ELL && (q != 0 || c != std::max(128, (h->max_u + 31) / 32 * 32))) continue;
                    h->kernel = k;
                    if (sa_heom_set_tuning(h, b, c, q)) continue;
                    float ms = 0;
                    rc = time_steps(4, &ms);
                    if (rc) break;
                    cands.push_back({ms, k, c, b, q});
                }
    // then the four fastest again, longer, and the best of the two timings
    std::sort(cands.begin(), cands.end(), [](const Cand& a, const Cand& b) { return a.ms < b.ms; });
    if (cands.size() > 4) cands.resize(4);
    for (Cand& x : cands) {
        if (rc) break;
        h->kernel = x.k;
        if (sa_heom_set_tuning(h, x.b, x.c, x.q)) continue;
        float ms = 0;
        rc = time_steps(12, &ms);
        x.ms = std::min(x.ms, ms);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    if (cands.empty()) return fail(SA_ERR_UNSUPPORTED, "no tuning fits this batch");
    const Cand w = *std::min_element(cands.begin(), cands.end(), [](const Cand& a, const Cand& b) { return a.ms < b.ms; });
    h->kernel = w.k;
    rc = sa_heom_set_tuning(h, w.b, w.c, w.q);
    if (rc) return rc;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune[key] = {w.b, w.c, w.q, w.k};
    }
    if (best) {
        best[0] = w.b;
        best[1] = w.c;
        best[2] = w.q;
    }
    return SA_OK;
}

// four stage kernels, plus the FP64 physical-representative kernel after each
// stage in SA_FP32_AUX mode (on a packed handle the pack kernel runs the
// list units too)
int sa_heom_launches_per_step(const sa_heom* h) {
    if (!h) return 0;
    int main = 1;
    if (h->kernel == SA_KERNEL_ELL) main = 2;  // grouped sums, then the ELL kernel
    if (h->kernel == SA_KERNEL_LISTS && !h->host_only)
        main = (h->n_list_units || h->n_pack_units) ? 1 : 0;  // list kernel, or the pack kernel
    return 4 * (main + (h->precision == SA_FP64 ? 0 : 1));
}

int sa_heom_set_debug(sa_heom* h, int flags) {
    if (!h) return fail(SA_ERR_INVALID_ARG, "null handle");
    if (flags & ~(SA_DEBUG_EXPIRE_WAIT | SA_DEBUG_CORRUPT_RECORD | SA_DEBUG_CHECK_INDICES | SA_DEBUG_CORRUPT_LIST))
        return fail(SA_ERR_INVALID_ARG, "unknown flag");
    if ((flags & SA_DEBUG_CORRUPT_LIST) &&
        (!(flags & SA_DEBUG_CHECK_INDICES) || h->host_only || h->kernel != SA_KERNEL_LISTS))
        return fail(SA_ERR_INVALID_ARG,
                    "SA_DEBUG_CORRUPT_LIST needs SA_DEBUG_CHECK_INDICES on a device handle running the list kernel");
    if (flags & SA_DEBUG_CORRUPT_RECORD) {
        if (!h->host_only) return fail(SA_ERR_STATE, "SA_DEBUG_CORRUPT_RECORD needs a host-only handle");
        HostInstance& hi = h->inst[0];
        if (hi.rec.empty()) return fail(SA_ERR_STATE, "instance 0 has no connection record");
        hi.rec[0].target += 1;  // no longer the first variable of a pattern
    }
    const int kept = flags & (SA_DEBUG_EXPIRE_WAIT | SA_DEBUG_CHECK_INDICES | SA_DEBUG_CORRUPT_LIST);
    if (kept != h->debug) {
        // the step graphs hold the kernels and their parameters: rebuild them
        for (auto& kv : h->graphs) cudaGraphExecDestroy(kv.second);
        h->graphs.clear();
    }
    const bool corrupt = (flags & SA_DEBUG_CORRUPT_LIST) != 0;
    h->debug = kept;
    if (corrupt != h->corrupt_list) {
        // rebuild the term lists with (or, again, without) the bad target
        h->corrupt_list = corrupt;
        h->tables = -1;
        const int rc = apply_tuning(h);
        if (rc) return rc;
    }
    return SA_OK;
}

// Consistency of the host tables of one instance: pattern, category and
// variable counts (Eq. uvar-count), multiplicities summing to N, T-ranks,
// and every connection record (its target is the first variable of a
// pattern one tier up or down, with the G' the record names, its moved
// category inside that pattern, its channel and occupation inside m and L).
static int validate_instance(const HostInstance& hi, int inst) {
    auto bad = [&](int64_t p, const std::string& what) {
        return fail(SA_ERR_STATE, "instance " + std::to_string(inst) + ", pattern " + std::to_string(p) + ": " + what);
    };
    const int64_t P = hi.P;
    if (int64_t(hi.cat_off.size()) != P + 1 || int64_t(hi.var_off.size()) != P + 1 ||
        int64_t(hi.rec_off.size()) != P + 1 || int64_t(hi.G.size()) != P || int64_t(hi.tier.size()) != P)
        return bad(-1, "table sizes");
    for (int64_t p = 0; p < P; ++p) {
        const int G = int(hi.cat_off[p + 1]) - int(hi.cat_off[p]);
        if (G < 1 || G > kMaxG || G != hi.G[p]) return bad(p, "category count");
        int64_t msum = 0;
        int nt = 0;
        for (uint32_t c = hi.cat_off[p]; c < hi.cat_off[p + 1]; ++c) {
            if (hi.cat_M[c] < 1) return bad(p, "multiplicity below 1");
            msum += hi.cat_M[c];
            if ((hi.cat_M[c] >= 2) != (hi.cat_trank[c] >= 0) || (hi.cat_trank[c] >= 0 && hi.cat_trank[c] != nt))
                return bad(p, "T-rank");
            if (hi.cat_trank[c] >= 0) ++nt;
        }
        if (msum != hi.N) return bad(p, "multiplicities do not sum to N");
        if (int64_t(hi.var_off[p + 1] - hi.var_off[p]) != int64_t(G + 1) * (G + 1) + nt) return bad(p, "variable count");
        if (hi.rec_off[p + 1] < hi.rec_off[p] || hi.rec_off[p + 1] > hi.rec.size()) return bad(p, "record range");
        for (uint32_t r = hi.rec_off[p]; r < hi.rec_off[p + 1]; ++r) {
            const Record& R = hi.rec[r];
            const int ts = R.packed & 31, Gp = (R.packed >> 5) & 31, cid = int(R.packed >> 23);
            const int k = cid / (2 * kCoefN), n = (cid >> 1) % kCoefN, raise = cid & 1;
            if (k >= hi.m || n > hi.L) return bad(p, "record " + std::to_string(r) + ": coefficient id");
            const auto it = std::lower_bound(hi.var_off.begin(), hi.var_off.end() - 1, uint64_t(R.target));
            if (it == hi.var_off.end() - 1 || *it != R.target)
                return bad(p, "record " + std::to_string(r) + ": target is not the first variable of a pattern");
            const int64_t pt = it - hi.var_off.begin();
            if (int(hi.tier[pt]) != int(hi.tier[p]) + (raise ? 1 : -1))
                return bad(p, "record " + std::to_string(r) + ": target not one tier away");
            if (Gp != hi.G[pt] || ts < 1 || ts > Gp) return bad(p, "record " + std::to_string(r) + ": target categories");
        }
    }
    return SA_OK;
}

int sa_heom_validate(const sa_heom* h) {
    if (!h) return fail(SA_ERR_INVALID_ARG, "null handle");
    for (int i = 0; i < h->count; ++i) {
        const int rc = validate_instance(h->inst[i], i);
        if (rc) return rc;
    }
    return SA_OK;
}

int sa_heom_device_error(sa_heom* h, void* stream) {
    int rc = check_device(h);
    if (rc) return rc;
    return read_device_error(h, static_cast<cudaStream_t>(stream));
}

}  // extern "C"

// ---- observables that allocate nothing ---------------------------------------
// The paper has no counterpart: this is a service for callers that may not
// call cudaMalloc (see sa_heom_observables_noalloc in include/sa_heom.h).
// Device-side output of the observables kernel, shared by every handle and
// every call in the process; each loaded GPU holds it until the process exits.
static __device__ __align__(256) double g_obs_scratch[SA_HEOM_NOALLOC_MAX_INSTANCES * 8];

extern "C" int sa_heom_observables_noalloc(sa_heom* h, const void* d_state, double* out, void* stream) {
    int rc = check_device(h);
    if (rc) return rc;
    if (!d_state || !out) return fail(SA_ERR_INVALID_ARG, "d_state and out required");
    if (h->count > SA_HEOM_NOALLOC_MAX_INSTANCES)
        return fail(SA_ERR_UNSUPPORTED, "sa_heom_observables_noalloc serves at most " +
                                            std::to_string(SA_HEOM_NOALLOC_MAX_INSTANCES) + " instances; this batch has " +
                                            std::to_string(h->count));
    // The host-side name of the array is only a stand-in for it: ask the
    // runtime for its device address on the current device (check_device made
    // sure that is the handle's).  The first call on a device loads the array
    // there; every later call asks again, which allocates nothing and never
    // leaves a stale address behind (after a cudaDeviceReset, say).
    void* p = nullptr;
    {
        const cudaError_t e = cudaGetSymbolAddress(&p, g_obs_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_obs_scratch)");
    }
    double* const scratch = static_cast<double*>(p);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // the kernel writes all 8 * count slots it is read back from, so nothing
    // left from an earlier call needs clearing
    CK(observables_into(h, d_state, scratch, st));
    const size_t need = size_t(h->count) * 8;
    CK(cudaMemcpyAsync(out, scratch, need * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    for (size_t j = 0; j < need; ++j)
        if (!std::isfinite(out[j])) return fail(SA_ERR_NUMERIC, "non-finite observable");
    return SA_OK;
}
