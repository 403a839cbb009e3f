// sa_internal.h -- host-side tables and device layout shared by the table
// builder (builder.cpp), the bath helpers (bath.cpp), the kernels
// (kernels.cu) and the C ABI (api.cu).  Library-internal.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/sa_heom.h"

namespace sa {

// ---- limits ---------------------------------------------------------------
constexpr int kMaxG = 31;            // categories per pattern (5-bit fields)
constexpr int kCoefN = 32;           // occupation slots per channel in the coefficient table
constexpr int kCoefPerInst = SA_HEOM_MAXM * kCoefN * 2;
constexpr int kSideSlots = 32;       // FP64 slots of the physical representative per instance
// representative propagations of arbitrary initial operators: |c><c|, |e_1><c|,
// |c><e_1|, |e_1><e_1|, |e_1><e_2|, and the named variables of their physical
// representatives (categories 1, 2, 3: molecule 1, molecule 2 or the others, the others)
constexpr int kReps = 5, kRepSlots = 17;
enum RepSlot { RZ, RX1, RX2, RX3, RY1, RY2, RY3, RP1, RP2, RP3, RS12, RS13, RS21, RS23, RS31, RS32, RT };
// Where a representative's response value lives: the batch instance that
// propagates it, the variable's local index in that instance's physical
// pattern (-1: absent), and whether the value is the complex conjugate of
// that variable (the |c><e_1| response taken as the adjoint of the |e_1><c|
// one, Eq. adjoint-preservation).
struct RepSrc {
    int16_t loc;
    int8_t inst;
    int8_t conj;
};

// ---- one hierarchy connection record ---------------------------------------
// A record belongs to (pattern Lambda, category q, channel k, direction): the
// molecule of category q whose local vector v_q becomes w = v_q +/- e_k.  The
// raw target's canonical pattern Lambda' (Eqs. canonical-target-plus/minus)
// has its categories in canonical order; an unmoved category r of Lambda
// lands at
//     tau(r) = r - [del && r > q] + [ins && r >= ipos]
// and the moved molecule at tau_star.  del: category q vanishes (M_q = 1);
// ins: w is a new category of Lambda' inserted before old category ipos;
// otherwise (ins = 0) w merges with the existing category s, and the ipos
// field holds s.  Together with the
// target's G' and the T-rank of tau_star this resolves every aligned-target
// entry (Eq. aligned-accessor) with integer arithmetic.
struct Record {
    uint32_t target;   // first variable of Lambda' in the batch vector
    uint32_t packed;   // see pack_record
};

inline uint32_t pack_record(int tau_star, int Gp, int trank_star, int has_t, int ipos, int ins, int del,
                            int coef_id) {
    return uint32_t(tau_star) | (uint32_t(Gp) << 5) | (uint32_t(trank_star) << 10) | (uint32_t(has_t) << 15) |
           (uint32_t(ipos) << 16) | (uint32_t(ins) << 21) | (uint32_t(del) << 22) | (uint32_t(coef_id) << 23);
}
// coefficient id: ((k * kCoefN) + n) * 2 + (raise ? 1 : 0), n = v_q[k] before the move
inline int coef_id(int k, int n, int raise) { return ((k * kCoefN) + n) * 2 + (raise ? 1 : 0); }

// ---- per-pattern header on the device (16 bytes) --------------------------
struct PatHdr {
    uint32_t var_off;  // first variable (batch-global)
    uint32_t rec_off;  // first record (batch-global)
    uint32_t cat_off;  // first category (batch-global)
    uint16_t inst;     // instance
    uint8_t G;         // categories
    uint8_t tier;      // |Lambda|
};

// per-category word: bits 0-9 first record (relative to rec_off),
// 10-14 record count, 15-19 T-rank (31 = no T variable), 20-23 raise
// records (they come first, the lower records follow)
inline uint32_t pack_cat(int rec_start, int nrec, int trank, int nup) {
    return uint32_t(rec_start) | (uint32_t(nrec) << 10) | (uint32_t(trank < 0 ? 31 : trank) << 15) |
           (uint32_t(nup) << 20);
}

// per-instance constants on the device
struct InstDev {
    double g, detuning, kappa, N;
    float gf, detf, kappaf, termf;
    uint32_t coef_base;  // into the coefficient tables
    uint32_t side;       // first FP64 side slot
    uint32_t var_begin;  // first variable
    uint32_t n_rho0;     // variables of the physical representative (5 for d = 0, up to 26 for d = 3)
    uint32_t pat_begin;  // first pattern (the empty pattern)
    uint32_t lcoef_base; // first slot of the instance's list/ELL coefficient table
    // where the instance's variable l lives in the device state: element
    // dev_base + l * dev_stride (var_begin + l, stride 1, unless the handle
    // packs instances; a packed instance is one lane of its pack)
    uint32_t dev_base, dev_stride;
    double term;         // terminator strength Delta (0: off)
    double pad3;
};

// ---- host tables of one instance ------------------------------------------
struct HostInstance {
    sa_params p{};
    int m = 0, L = 0;
    int64_t N = 0;
    // local vectors: id 0 = zero vector, then |alpha| descending, components
    // lexicographically descending
    int V = 0;
    int d = 0;                       // distinguished molecules (0 .. SA_HEOM_MAXD)
    int Vtot = 0;                    // (d + 1) V: ids j V .. j V + V - 1 are molecule j's copies
    std::vector<uint8_t> comp;       // Vtot * m
    std::vector<int> norm;           // Vtot
    std::vector<int32_t> lut;        // mixed-radix code -> id
    // canonical patterns
    int64_t P = 0;
    std::vector<uint32_t> id_off;    // P + 1
    std::vector<uint32_t> ids;       // ascending vector ids
    std::vector<uint8_t> tier;       // P
    std::vector<uint8_t> G, h;       // P
    std::vector<uint32_t> cat_off;   // P + 1
    std::vector<uint32_t> cat_vec;   // vector id of each category
    std::vector<int64_t> cat_M;      // multiplicity
    std::vector<int8_t> cat_trank;   // T-rank or -1
    std::vector<uint32_t> cat_word;  // pack_cat
    std::vector<uint64_t> var_off;   // P + 1, instance-relative
    std::vector<double> gamma_re, gamma_im;
    std::vector<uint32_t> rec_off;   // P + 1, instance-relative
    std::vector<Record> rec;         // target instance-relative until batch assembly
    int64_t n_terms = 0;
    // coefficient table: row and column coefficients, (re, im) pairs
    std::vector<double> coef_row, coef_col;  // 2 * kCoefPerInst each
};

struct DRecA {
    int x, y, z, w;  // X'-index, S'-row base, S'-column base, T'-index (batch-global)
};

// one work item of the stage kernel (one warp): a run of consecutive
// patterns and the ranges of their variables and categories
struct ItemDesc {
    uint32_t p0, np, v0, nv, c0, ncat;
    uint32_t r0;          // list kernel: first round of 32 lanes in the round table
    uint32_t nl;          // list kernel: variables the lanes take (the item's, less any integrated elsewhere)
    uint32_t row0, row1;  // list kernel: the item's term rows
    uint32_t blob16;      // list kernel: the item's table blob, in 16-byte units
    uint32_t blob_bytes;
    uint32_t nw;          // pack items: distinct grouped-sum weights a + b N (0 otherwise)
};

// Per-instance constants of the list kernel (T = float or double): where the
// instance's variables and coefficient table start, N (the zero category's
// multiplicity is N - r; the template blob stores -r for it), the coupling g
// and, per variable class (0 S T, 1 X, 2 Y, 3 Z, 4 P), the diagonal part that
// does not depend on the pattern: -(cavity loss + terminator) and -/+ i
// detuning, as (re, im) pairs.  The pattern's -Gamma_Lambda comes from the
// blob.
template <typename T> struct InstK {
    uint32_t var_base, lcoef_base;
    double N;
    T g, pad;
    T cc[10];
};

// per-pattern constants of the list kernel (T = float or double)
template <typename T> struct PatConst {
    T g, det, kap;       // coupling, detuning, loss rate of the pattern's instance
    uint32_t coef_base;  // the instance's coefficient table
    T term;              // terminator strength Delta
};

// A pattern as the list and pack kernels' blobs give it (8 bytes): its first
// variable and first category relative to the work item's, G, tier, and a
// reserved zero (a template item belongs to one instance at a time).
struct ItemPat {
    uint16_t var_rel, cat_rel;
    uint8_t G, tier;
    uint16_t islot;
};
constexpr int kItemInsts = 4;  // record kernel: instances per work item

// Byte offsets of the sections of a list-kernel item blob (every section
// 16-byte aligned): a 16-byte header (reserved), patterns (ItemPat), per pattern
// -Gamma_Lambda (complex T), category words, multiplicities (T; the zero
// category holds M_0 - N = -r, the instance adds its N), owning pattern of
// every category (u8), round table (first term row of every round and the
// end), lane words, lane bytes.
struct BlobLayout {
    uint32_t pat, pd, cw, cM, cj, rb, lvd, lvj, bytes;
};
constexpr int kPatDiag = 1;  // complex entries per pattern in the pd section (-Gamma_Lambda)
#if defined(__CUDACC__)
#define SA_HOST_DEVICE __host__ __device__
#else
#define SA_HOST_DEVICE
#endif
template <typename T>
SA_HOST_DEVICE inline BlobLayout blob_layout(uint32_t np, uint32_t ncat, uint32_t nl) {
    auto a16 = [](uint32_t b) { return (b + 15u) & ~15u; };
    const uint32_t nrounds = (nl + 31u) / 32u;
    BlobLayout L;
    L.pat = 16;
    L.pd = L.pat + a16(np * uint32_t(sizeof(ItemPat)));
    L.cw = L.pd + a16(np * uint32_t(kPatDiag * 2 * sizeof(T)));
    L.cM = L.cw + a16(ncat * 4u);
    L.cj = L.cM + a16(ncat * uint32_t(sizeof(T)));
    L.rb = L.cj + a16(ncat);
    L.lvd = L.rb + a16((nrounds + 1u) * 4u);
    L.lvj = L.lvd + a16(nl * 4u);
    L.bytes = L.lvj + a16(nl);
    return L;
}
constexpr int kItemPats = 16;     // patterns per work item (at most 31: 5-bit local index)
constexpr int kMaxItemVars = 1024; // variables per work item (10-bit local index)
// An instance pack (SA_BUILD_PACK_INSTANCES): n <= 32 instances of one
// template stored interleaved, variable l of lane j at element
// base + l * n + j of the device state; their list coefficient tables
// interleaved the same way from element cbase (slot s of lane j at
// cbase + s * n + j); lane j's instance is pk_inst[lane0 + j].
struct PackDev {
    uint32_t base, n, cbase, lane0;
};
constexpr int kPackMin = 16;   // fewer lanes than this stay unpacked, for list units (packs from 8, 12 or 24 lanes measured no faster)
constexpr int kPackLanes = 32; // instances per pack at most

// Byte offsets of the sections of a pack item's table blob (every section
// 16-byte aligned): a 16-byte header (u32 nw, then reserved); patterns (ItemPat); per
// pattern -Gamma_Lambda (complex T); per category the multiplicity (T, as in
// the list blobs); per variable the warp updates a uint4 record; then per
// term the target (instance-relative variable, u32), then per term the
// coefficient slot (u16), the variables' terms one after another; then the
// item's nw distinct grouped-sum weights a + b N as (a, b) int32 pairs, N the
// instance's molecule count: 1, M_q, M_q - 1 and -M_q of its categories, where
// M of the zero category is N - r (a = -r, b = 1).
// The records come in three phases -- the P, T and S variables, then the X
// and Y variables, then the Z variables, each in canonical order (the
// physical representative left out in SA_FP32_AUX mode) -- so that the
// grouped sums a phase reads are complete: every variable adds its own value,
// weighted, to the sums it enters (P_q, T_q and S_{q,b} to R_q and C of their
// column category, Eqs. grouped-row-sum, grouped-column-sum; X_q and Y_q to
// the Z sum of Eq. HZ).  A record:
//   x: operand codes a (bits 0-10) and b (11-21) of the commutator term
//      -i g (op[a] - op[b]), diagonal class (22-24: 0 S T, 1 X, 2 Y, 3 Z,
//      4 P) and pattern (25-29);
//   y: item-local index (bits 0-9), first term (10-25), number of terms (26-31);
//   z, w: the contributions (two for P, T, S; one, in z, for X and Y; none
//      for Z), each a sum slot (bits 0-10) and the index of its weight
//      (bits 11-31): 1 for P_q, M_q - 1 for T_q, M_b and M_q for S_{q,b},
//      M_q and -M_q for X_q and Y_q.
// Operand codes and sum slots: below nv an item variable; nv + c (slot c)
// the row sum R of category c, nv + ncat + c its column sum C,
// nv + 2 ncat + j the Z sum of pattern j, nv + 2 ncat + np zero.  The sums
// live in the warp's shared memory, one column per lane.
struct PackLayout {
    uint32_t pat, pd, cM, vrec, tgt, tsl, wab, bytes;
};
template <typename T>
SA_HOST_DEVICE inline PackLayout pack_layout(uint32_t np, uint32_t ncat, uint32_t nl, uint32_t nterm, uint32_t nw) {
    auto a16 = [](uint32_t b) { return (b + 15u) & ~15u; };
    PackLayout L;
    L.pat = 16;
    L.pd = L.pat + a16(np * uint32_t(sizeof(ItemPat)));
    L.cM = L.pd + a16(np * uint32_t(2 * sizeof(T)));
    L.vrec = L.cM + a16(ncat * uint32_t(sizeof(T)));
    L.tgt = L.vrec + nl * 16u;
    L.tsl = L.tgt + a16(nterm * 4u);
    L.wab = L.tsl + a16(nterm * 2u);
    L.bytes = L.wab + a16(nw * 8u);
    return L;
}
// the per-lane values of a pack item's grouped-sum weights, after its blob
// (FP64 only: there the two conversions and the multiply-add of a weight,
// done per contribution, cost more of the FP64 pipe than the table's shared
// memory; FP32 evaluates them per contribution and keeps its items larger)
template <typename T> SA_HOST_DEVICE inline uint32_t pack_wtab_bytes(uint32_t nw) {
    return sizeof(T) == 8 ? nw * 32u * uint32_t(sizeof(T)) : 0u;
}
// and, after those, the per-lane diagonal coefficient of every (pattern,
// variable class) of the item, likewise FP64 only (the two additions of a
// variable's diagonal, done once per unit)
template <typename T> SA_HOST_DEVICE inline uint32_t pack_dtab_bytes(uint32_t np) {
    return sizeof(T) == 8 ? np * 5u * 32u * uint32_t(2 * sizeof(T)) : 0u;
}
// grouped sums of a pack item in the warp's shared memory: R and C per
// category, Z per pattern and a zero, one complex T per lane each
template <typename T> SA_HOST_DEVICE inline uint32_t pack_sums_bytes(uint32_t np, uint32_t ncat) {
    return (2u * ncat + np + 1u) * 32u * uint32_t(2 * sizeof(T));
}
// pack items are cut so that their blob, sums and weights stay below this many bytes
// (a pattern that alone exceeds it gets an item of its own)
template <typename T> constexpr uint32_t kPackItemTarget = sizeof(T) == 8 ? 12288u : 6144u;
constexpr uint32_t kPackUnit = 0x80000000u;  // work-unit flag: (pack item, pack) rather than (item, instance)

// List and ELL kernels: the coefficient table of one instance, compact so
// that a warp's coefficient loads stay in a few cache lines.  Slot 0 is zero
// (padded entries); then, for each channel k, occupation n = 0..L before the
// move and direction (lower, raise), the row, column and row + column (the
// two lower terms of P_q) coefficients side by side.  An instance holds
// list_slots(m, L) = 2 + 6 m (L + 1) slots (the last one unused; an even
// count, so every table starts 16-byte aligned in both precisions).
constexpr int kListCoefZero = 0;
inline int list_slot(int L, int cid, int side3) {
    const int k = cid / (2 * kCoefN), n = (cid >> 1) % kCoefN, raise = cid & 1;
    return 1 + ((k * (L + 1) + n) * 2 + raise) * 3 + side3;
}
inline int list_slots(int m, int L) { return 2 + 6 * m * (L + 1); }

// launch description shared by api.cu and kernels.cu (type-erased pointers)
struct LaunchCfg {
    int block;      // threads per CTA
    int chunk;      // variable capacity of one work item
    int use_queue;  // 1: persistent grid + atomic work queue
    int grid;       // CTAs
    int kernel;     // SA_KERNEL_RECORDS, SA_KERNEL_LISTS or SA_KERNEL_ELL (include/sa_heom.h)
    int pack_smem;  // pack kernel: shared-memory bytes of a warp (0: no packs)
    int pgrid;      // pack kernel: CTAs (persistent)
};
struct StageLaunch {
    const void* hdr; const void* cat_word; const void* cat_M; const void* gamma; const void* rec;
    const void* items; const void* vdesc; const void* drecA; const void* drecS;
    const void* inst; const void* coef_row; const void* coef_col;
    const void* cat_Md; const void* coef_row_d; const void* coef_col_d;
    const void* lut; const void* lut_off;
    const void* lvd; const void* lvj; const void* rbase; const void* tidx; const void* tcid; const void* lcoef;
    const void* wpat; uint32_t nvar; const void* blobs;
    const void* units; const void* instk;  // list kernel: work units (template item, instance), InstK<T>
    const void* packs; const void* pk_inst; const void* pcoef;  // pack kernel: PackDev, lane instances, pack coefficients
    const void* punits; uint32_t npunits; unsigned int* pqueue;  // pack kernel: its work units and counter
    const void* catpat; uint32_t ncat, npat; void* sums;
    uint32_t nchunks;
    const void* x_in; void* x_out; const void* y; void* acc; void* y_out;
    const void* xs_in; void* xs_out; const void* ys; void* accs; void* ys_out;
    double dt; int stage; unsigned int* queue; unsigned int* err;
    int debug;  // SA_DEBUG_* flags (include/sa_heom.h)
    const void* ilimit;  // SA_DEBUG_CHECK_INDICES: per instance (variables, list slots)
    int ninst;
    // SA_FP32_AUX: the FP64 physical-representative kernel runs on a side
    // stream, forked before and joined after the stage kernel
    void* side_stream; void* ev_fork; void* ev_join;
};

// api.cu: the detail sa_heom_last_error reports
void set_error(const std::string& msg);
// builder.cpp
int build_instance(const sa_params& p, HostInstance& out, std::string& err);
int64_t expand_terms(const HostInstance& hi, int64_t* var, int64_t* src, int32_t* k, int32_t* n, int32_t* dir,
                     int32_t* side);
// bath.cpp
int drude_lorentz(double lambda, double gamma, double kT, int scheme, int n_poles, double sigma, sa_params* p,
                  std::string& err);
int terminator(double lambda, double gamma, double kT, int n_matsubara, double* out, std::string& err);

// local index of a variable inside a pattern (canonical layout)
inline int64_t loc_Z() { return 0; }
inline int64_t loc_X(int G, int q) { return q; }
inline int64_t loc_Y(int G, int q) { return G + q; }
inline int64_t loc_P(int G, int q) { return 2 * G + q; }
inline int64_t loc_S(int G, int q, int r) { return 3 * G + 1 + int64_t(q - 1) * (G - 1) + (r - 1) - (r > q ? 1 : 0); }
inline int64_t loc_T(int G, int trank) { return int64_t(G + 1) * (G + 1) + trank; }

// Hierarchy terms of the variables of pattern i (Eqs. uvar-up / uvar-down),
// resolved through the connection records and the aligned accessor
// (Eq. aligned-accessor).  emit(loc, kind, src, packed, side) is called once
// per term: loc is the variable's local index in the pattern, kind 0..5 for
// Z X Y P S T, src the instance-relative index of the target entry, packed
// the record word (its coefficient id in bits 23..31) and side 0 for the row
// delta, 1 for the column delta.  The terms of one variable are emitted
// together.  The two raise terms of P_q cancel and are not emitted; its row
// and column lower terms name the same target.
template <class Emit>
void for_each_term(const HostInstance& hi, int64_t i, Emit&& emit) {
    const int G = hi.G[i];
    const uint32_t* cw = &hi.cat_word[hi.cat_off[i]];
    const Record* R = &hi.rec[hi.rec_off[i]];
    const int8_t* tr = &hi.cat_trank[hi.cat_off[i]];
    auto target_index = [&](const Record& rc, int rowc, int colc, bool same) -> int64_t {
        // rowc / colc: target category (0 = cavity); same: P entry
        const uint32_t pk = rc.packed;
        const int Gp = (pk >> 5) & 31, trs = (pk >> 10) & 31;
        int64_t loc;
        if (rowc == 0 && colc == 0) loc = loc_Z();
        else if (colc == 0) loc = loc_X(Gp, rowc);
        else if (rowc == 0) loc = loc_Y(Gp, colc);
        else if (same) loc = loc_P(Gp, rowc);
        else if (rowc != colc) loc = loc_S(Gp, rowc, colc);
        else loc = loc_T(Gp, trs);
        return int64_t(rc.target) + loc;
    };
    auto tau_of = [](uint32_t pk, int moved, int rr) {
        const int ipos = (pk >> 16) & 31, ins = (pk >> 21) & 1, del = (pk >> 22) & 1;
        return rr - ((del && rr > moved) ? 1 : 0) + ((ins && rr >= ipos) ? 1 : 0);
    };
    auto each_var = [&](int kind, int q, int r, int64_t loc) {
        int row = 0, col = 0;
        bool same = false;
        if (kind == 1) row = q;
        if (kind == 2) col = q;
        if (kind == 3) { row = q; col = q; same = true; }
        if (kind == 4) { row = q; col = r; }
        if (kind == 5) { row = q; col = q; }
        if (row) {
            const uint32_t w = cw[row - 1];
            const int rs = w & 1023, nr = (w >> 10) & 31;
            for (int j = 0; j < nr; ++j) {
                const Record& rc = R[rs + j];
                const bool raise = ((rc.packed >> 23) & 1) != 0;
                if (same && raise) continue;  // cancels against the column raise
                const int tstar = rc.packed & 31;
                const int cc = col == 0 ? 0 : (same ? tstar : tau_of(rc.packed, row, col));
                emit(loc, kind, target_index(rc, tstar, cc, same), rc.packed, 0);
            }
        }
        if (col) {
            const uint32_t w = cw[col - 1];
            const int rs = w & 1023, nr = (w >> 10) & 31;
            for (int j = 0; j < nr; ++j) {
                const Record& rc = R[rs + j];
                const bool raise = ((rc.packed >> 23) & 1) != 0;
                if (same && raise) continue;
                const int tstar = rc.packed & 31;
                const int rr = row == 0 ? 0 : (same ? tstar : tau_of(rc.packed, col, row));
                emit(loc, kind, target_index(rc, rr, tstar, same), rc.packed, 1);
            }
        }
    };
    each_var(0, 0, 0, loc_Z());
    for (int q = 1; q <= G; ++q) {
        each_var(1, q, 0, loc_X(G, q));
        each_var(2, q, 0, loc_Y(G, q));
        each_var(3, q, 0, loc_P(G, q));
        for (int r = 1; r <= G; ++r)
            if (r != q) each_var(4, q, r, loc_S(G, q, r));
        if (tr[q - 1] >= 0) each_var(5, q, 0, loc_T(G, tr[q - 1]));
    }
}

}  // namespace sa
