// kernels.cu -- sm_103a kernels of the symmetry-adapted HEOM hot path.
//
// stage_kernel: one fused launch per RK4 stage.  Each CTA takes a chunk of
// consecutive canonical patterns (at most `chunk` variables), stages the
// patterns' headers, category words, multiplicities and their slice of the
// stage input x_s in shared memory with coalesced vector loads, and gives
// each thread one unique variable at a time (structure-of-arrays state,
// float2 / double2 complex).  A thread evaluates
//   * the system commutator -i[H_S, .] from the staged values: the grouped
//     row and column sums of Eqs. grouped-row-sum / grouped-column-sum for
//     X_q and Y_q, the multiplicity-weighted sum of Eq. HZ for Z, two reads
//     for P, S and T;
//   * the damping -Gamma_Lambda (Eq. tier-damping) and the cavity loss;
//   * the hierarchy terms of Eqs. uvar-up and uvar-down: for the row
//     category and the column category of the variable, every connection
//     record of that category names the canonical target and the integer
//     remap that resolves the aligned accessor (Eq. aligned-accessor); the
//     entry is gathered from x_s in global memory (L2-resident neighbours in
//     tiers +/-1) and multiplied by its tabulated coefficient;
// and fuses the classical RK4 stage update (acc, next stage input, or the
// final state) so that the derivative never touches memory.
//
// Chunks are handed out by an atomic work queue (persistent grid) or one per
// CTA.  A batch of independent instances is one concatenated table set, so a
// single launch serves every instance.  In SA_FP32_AUX mode the auxiliary
// variables are float2, and the physical representative (the empty pattern)
// of every instance is integrated in FP64 from FP64 side buffers; its FP32
// mirror feeds the tier-1 readers.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "sa_internal.h"

namespace sa {

template <typename T> struct Cx;
template <> struct Cx<double> { using t = double2; };
template <> struct Cx<float> { using t = float2; };

__device__ __forceinline__ double2 mk(double a, double b) { return make_double2(a, b); }
__device__ __forceinline__ float2 mk(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ double2 to_acc(double2 a, double2*) { return a; }
__device__ __forceinline__ double2 to_acc(float2 a, double2*) { return make_double2(a.x, a.y); }
__device__ __forceinline__ float2 to_acc(float2 a, float2*) { return a; }

template <class C> __device__ __forceinline__ C cadd(C a, C b) { return mk(a.x + b.x, a.y + b.y); }
template <class C> __device__ __forceinline__ C csub(C a, C b) { return mk(a.x - b.x, a.y - b.y); }
template <class C, class S> __device__ __forceinline__ C cscale(C a, S s) { return mk(a.x * s, a.y * s); }
// acc + a * b
template <class C> __device__ __forceinline__ C cfma(C a, C b, C acc) {
    acc.x = fma(a.x, b.x, fma(-a.y, b.y, acc.x));
    acc.y = fma(a.x, b.y, fma(a.y, b.x, acc.y));
    return acc;
}
// acc + s * a (s real)
template <class C, class S> __device__ __forceinline__ C caxpy(S s, C a, C acc) {
    acc.x = fma(s, a.x, acc.x);
    acc.y = fma(s, a.y, acc.y);
    return acc;
}

template <typename T> struct StageParams {
    using C = typename Cx<T>::t;
    const PatHdr* __restrict__ hdr;       // npat + 1 (sentinel)
    const uint32_t* __restrict__ cat_word;
    const T* __restrict__ cat_M;
    const C* __restrict__ gamma;
    const Record* __restrict__ rec;
    const ItemDesc* __restrict__ items;    // nchunks work items
    const uint32_t* __restrict__ vdesc;    // per variable: item-local order and (kind, q, r)
    const int4* __restrict__ drecA;        // decoded records: X'-index, S'-row base, S'-column base, T'-index
    const uint32_t* __restrict__ drecS;    // decoded records: small fields and coefficient id
    const InstDev* __restrict__ inst;
    const C* __restrict__ coef_row;
    const C* __restrict__ coef_col;
    const double* __restrict__ cat_Md;      // FP64 copies for the FP64 physical representative
    const double2* __restrict__ coef_row_d;
    const double2* __restrict__ coef_col_d;
    const uint16_t* __restrict__ lut;       // (kind | q << 3 | r << 8) per (G, local index)
    const uint32_t* __restrict__ lut_off;   // per G
    // list kernel
    const uint32_t* __restrict__ lvd;       // per lane variable: l | a << 10 | b << 21 (operand-area indices)
    const uint8_t* __restrict__ lvj;        // per lane variable: pattern j | diagonal class << 5
    const uint32_t* __restrict__ rbase;     // first term row of every round of 32 lanes (+ sentinel)
    const uint32_t* __restrict__ tidx;      // term rows of 32: batch-global target index
    const uint16_t* __restrict__ tcid;      // term rows of 32: coefficient slot in the instance's list table
    const C* __restrict__ lcoef;            // per instance list_slots(m, L) slots from InstDev::lcoef_base
    // ELL kernel (lvd: per-variable word, rbase: per warp row, tidx / tcid as above)
    const unsigned char* __restrict__ blobs; // list kernel: per-item table blobs (16-byte aligned)
    const uint2* __restrict__ units;         // list kernel: work units (template item, instance)
    const InstK<T>* __restrict__ instk;      // list kernel: per-instance constants
    const PackDev* __restrict__ packs;       // pack kernel: instance packs
    const uint32_t* __restrict__ pk_inst;    // pack kernel: instance of every pack lane
    const C* __restrict__ pcoef;             // pack kernel: interleaved coefficient tables of the packs
    const uint2* __restrict__ punits;        // pack kernel: work units (pack item | kPackUnit, pack)
    uint32_t npunits;
    uint32_t pack_smem;                      // pack kernel: shared-memory bytes per warp
    unsigned int* pqueue;                    // pack kernel: its work counter
    const uint32_t* __restrict__ wpat;      // first pattern of every warp row of 32 variables
    uint32_t nvar;
    const uint32_t* __restrict__ catpat;    // owning pattern of every category
    uint32_t ncat, npat;
    C* sumR;                                // grouped row sums R_q per category
    C* sumC;                                // grouped column sums C_q per category
    C* sumZ;                                // sum_q M_q (X_q - Y_q) per pattern
    uint32_t nchunks;
    int chunk;                              // variable capacity of one work item
    const C* x_in;                          // stage input (gathered)
    C* x_out;                               // next stage input, or dR/dt (stage -1)
    const C* y;                             // state at the start of the step
    C* acc;                                 // RK4 accumulator
    C* y_out;                               // new state (stage 3)
    const double2* xs_in;                   // FP64 side copies (SA_FP32_AUX)
    double2* xs_out;
    const double2* ys;
    double2* accs;
    double2* ys_out;
    double dt;
    int stage;                              // -1: right-hand side only; 0..3: RK4 stage
    int use_queue;
    unsigned int* queue;
    unsigned int* err;                      // device error word (bit 0: a bounded wait expired)
    int expire_wait;                        // SA_DEBUG_EXPIRE_WAIT: report the first bulk-copy wait as expired
    const uint2* __restrict__ ilimit;       // SA_DEBUG_CHECK_INDICES: per instance its variables and list slots
};

enum { KZ = 0, KX = 1, KY = 2, KP = 3, KS = 4, KT = 5 };

__device__ __forceinline__ int loc_S_d(int G, int a, int b) { return 3 * G + 1 + (a - 1) * (G - 1) + (b - 1) - (b > a); }
__device__ __forceinline__ int tau_d(uint32_t pk, int moved, int r) {
    int ipos = (pk >> 16) & 31, ins = (pk >> 21) & 1, del = (pk >> 22) & 1;
    return r - ((del && r > moved) ? 1 : 0) + ((ins && r >= ipos) ? 1 : 0);
}

// Derivative of one variable with accumulator precision A.  own(l) returns
// the pattern's local variable l, gath(i) the batch-global variable i.
template <typename A, typename T, class Own, class Gath>
__device__ __forceinline__ typename Cx<A>::t var_rhs(const StageParams<T>& P, int kind, int q, int r, int G,
                                                     const uint32_t* s_cw, const T* s_cM, const uint2* s_rec,
                                                     const PatHdr& h, const InstDev& I, typename Cx<A>::t gam,
                                                     Own own, Gath gath) {
    using CA = typename Cx<A>::t;
    using C = typename Cx<T>::t;
    constexpr bool kMixed = sizeof(A) == 8 && sizeof(T) == 4;
    auto mult = [&](int a) -> A {
        if constexpr (kMixed) return P.cat_Md[h.cat_off + a - 1];
        else return A(s_cM[a - 1]);
    };
    const A g = A(sizeof(A) == 8 ? I.g : I.gf);
    const A det = A(sizeof(A) == 8 ? I.detuning : I.detf);
    const A kap = A(sizeof(A) == 8 ? I.kappa : I.kappaf);
    // terminator -Delta w: w = 0 for Z and P, 1 for X and Y, 2 for S and T
    const A trm = A(sizeof(A) == 8 ? I.term : I.termf) *
                  A(kind == KX || kind == KY ? 1 : ((kind == KS || kind == KT) ? 2 : 0));
    int self;
    switch (kind) {
        case KZ: self = 0; break;
        case KX: self = q; break;
        case KY: self = G + q; break;
        case KP: self = 2 * G + q; break;
        case KS: self = loc_S_d(G, q, r); break;
        default: self = (G + 1) * (G + 1) + ((s_cw[q - 1] >> 15) & 31); break;
    }
    const CA v = own(self);
    CA d;
    if (kind == KZ) {
        // -i g sum_q M_q (X_q - Y_q) - (Gamma + kappa) Z   (Eq. HZ + loss)
        CA s = mk(A(0), A(0));
        for (int a = 1; a <= G; ++a) s = caxpy(mult(a), csub(own(a), own(G + a)), s);
        d = mk(g * s.y, -g * s.x);
        const CA dm = cadd(gam, mk(kap, A(0)));
        d = cfma(mk(-dm.x, -dm.y), v, d);
    } else if (kind == KX || kind == KY) {
        // grouped sum R_q (row) or C_q (column)
        const CA Pq = own(2 * G + q);
        CA s = Pq;
        const A Mq = mult(q);
        if (Mq >= A(2)) s = caxpy(Mq - A(1), own((G + 1) * (G + 1) + ((s_cw[q - 1] >> 15) & 31)), s);
        for (int b = 1; b <= G; ++b)
            if (b != q) s = caxpy(mult(b), own(kind == KX ? loc_S_d(G, q, b) : loc_S_d(G, b, q)), s);
        const CA Z = own(0);
        // X: -i det X - i g (Z - R_q);   Y: +i det Y - i g (C_q - Z)
        const CA t = kind == KX ? csub(Z, s) : csub(s, Z);
        const A sd = kind == KX ? det : -det;
        d = mk(sd * v.y + g * t.y, -sd * v.x - g * t.x);
        const CA dm = cadd(gam, mk(A(0.5) * kap + trm, A(0)));
        d = cfma(mk(-dm.x, -dm.y), v, d);
    } else {
        // P, T: -i g (Y_q - X_q);  S_{q,r}: -i g (Y_r - X_q)
        const CA t = csub(own(G + (kind == KS ? r : q)), own(q));
        d = mk(g * t.y, -g * t.x);
        d = cfma(mk(-(gam.x + trm), -gam.y), v, d);
    }
    // hierarchy terms: the records of the row category (row delta of
    // Eq. projector-commutator-element) and of the column category (column
    // delta); gathers are issued four at a time before their products are
    // accumulated
    const int row = (kind == KX || kind == KP || kind == KS || kind == KT) ? q : 0;
    const int col = (kind == KY) ? q : (kind == KS ? r : ((kind == KP || kind == KT) ? q : 0));
    const bool same = kind == KP;
    auto crow = [&](int cid) -> CA {
        if constexpr (kMixed) return P.coef_row_d[I.coef_base + cid];
        else return to_acc(__ldg(P.coef_row + I.coef_base + cid), (CA*)nullptr);
    };
    auto ccol = [&](int cid) -> CA {
        if constexpr (kMixed) return P.coef_col_d[I.coef_base + cid];
        else return to_acc(__ldg(P.coef_col + I.coef_base + cid), (CA*)nullptr);
    };
    const uint32_t wr = row ? s_cw[row - 1] : 0u;
    const uint32_t wc = (col && !same) ? s_cw[col - 1] : 0u;
    // P_q: its two raise terms cancel, so only the lower records (which
    // follow the raise records of the category) are read
    const int skip = same ? int((wr >> 20) & 15) : 0;
    const int nr = int((wr >> 10) & 31) - skip, nc = (wc >> 10) & 31;
    const uint2* Rr = s_rec + (wr & 1023) + skip;
    const uint2* Rc = s_rec + (wc & 1023);
    const int ntot = nr + nc;
    for (int i0 = 0; i0 < ntot; i0 += 4) {
        CA val[4], cf[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int i = i0 + u;
            val[u] = mk(A(0), A(0));
            cf[u] = mk(A(0), A(0));
            if (i < ntot) {
                const bool isrow = i < nr;
                const uint2 rc = isrow ? Rr[i] : Rc[i - nr];
                const uint32_t pk = rc.y;
                const int cid = pk >> 23;
                const int ts = pk & 31, Gp = (pk >> 5) & 31;
                const int tT = (Gp + 1) * (Gp + 1) + ((pk >> 10) & 31);
                int tl;
                if (isrow) {
                    if (kind == KX) tl = ts;
                    else if (same) tl = 2 * Gp + ts;
                    else {
                        const int cc = tau_d(pk, row, col);
                        tl = (cc == ts) ? tT : loc_S_d(Gp, ts, cc);
                    }
                } else {
                    if (kind == KY) tl = Gp + ts;
                    else {
                        const int rr = tau_d(pk, col, row);
                        tl = (rr == ts) ? tT : loc_S_d(Gp, rr, ts);
                    }
                }
                val[u] = gath(rc.x + tl);
                if (isrow) {
                    cf[u] = crow(cid);
                    if (same) cf[u] = cadd(cf[u], ccol(cid));
                } else {
                    cf[u] = ccol(cid);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) d = cfma(cf[u], val[u], d);
    }
    return d;
}


// Per-warp shared-memory image of one work item.
template <typename T> struct WarpSmem {
    using C = typename Cx<T>::t;
    C* x;        // stage input slice
    C* y;        // RK4 state slice
    C* acc;      // RK4 accumulator slice
    C* R;        // grouped row sums R_q per category (Eq. grouped-row-sum)
    C* Cs;       // grouped column sums C_q per category (Eq. grouped-column-sum)
    C* Zs;       // sum_q M_q (X_q - Y_q) per pattern (Eq. HZ)
    C* gam;      // Gamma_Lambda per pattern
    PatHdr* ph;  // pattern headers (kItemPats + 1)
    PatConst<T>* pc;
    uint32_t* cw;
    T* cM;
};

__host__ __device__ __forceinline__ size_t al16(size_t b) { return (b + 15) / 16 * 16; }

template <typename T>
__host__ __device__ __forceinline__ size_t warp_smem_bytes(int item) {
    const size_t cs = 2 * sizeof(T);
    const size_t nc = size_t(item) / 4 + 8;
    return 3 * al16(cs * item) + 2 * al16(cs * nc) + 2 * al16(cs * kItemPats) + al16(sizeof(PatHdr) * (kItemPats + 1)) +
           al16(sizeof(PatConst<T>) * kItemPats) + al16(4 * nc) + al16(sizeof(T) * nc);
}

template <typename T>
__device__ __forceinline__ WarpSmem<T> carve_warp(unsigned char* p, int item) {
    using C = typename Cx<T>::t;
    const int nc = item / 4 + 8;
    WarpSmem<T> W;
    W.x = reinterpret_cast<C*>(p);        p += al16(sizeof(C) * item);
    W.y = reinterpret_cast<C*>(p);        p += al16(sizeof(C) * item);
    W.acc = reinterpret_cast<C*>(p);      p += al16(sizeof(C) * item);
    W.R = reinterpret_cast<C*>(p);        p += al16(sizeof(C) * nc);
    W.Cs = reinterpret_cast<C*>(p);       p += al16(sizeof(C) * nc);
    W.Zs = reinterpret_cast<C*>(p);       p += al16(sizeof(C) * kItemPats);
    W.gam = reinterpret_cast<C*>(p);      p += al16(sizeof(C) * kItemPats);
    W.ph = reinterpret_cast<PatHdr*>(p);  p += al16(sizeof(PatHdr) * (kItemPats + 1));
    W.pc = reinterpret_cast<PatConst<T>*>(p); p += al16(sizeof(PatConst<T>) * kItemPats);
    W.cw = reinterpret_cast<uint32_t*>(p); p += al16(4 * nc);
    W.cM = reinterpret_cast<T*>(p);
    return W;
}

// One warp per work item (a run of consecutive patterns, at most `item`
// variables and kItemPats patterns), with no block-wide barrier: the warp
// stages its slices, forms the grouped sums, then each lane takes one
// variable at a time in the host-made order (S variables first, then T, P,
// X, Y, Z, so that the lanes of a warp run the same code path).
template <typename T, bool FP64SIDE>
__global__ void __launch_bounds__(256) stage_kernel(StageParams<T> P) {
    using C = typename Cx<T>::t;
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const WarpSmem<T> S = carve_warp<T>(smem + size_t(wib) * warp_smem_bytes<T>(P.chunk), P.chunk);
    const unsigned int nwarps = gridDim.x * (blockDim.x >> 5);
    unsigned int it = blockIdx.x * (blockDim.x >> 5) + wib;
    const T dtT = T(P.dt);
    const T aT = P.stage == 2 ? dtT : T(0.5) * dtT;
    for (;;) {
        unsigned int c;
        if (P.use_queue) {
            unsigned int t = 0;
            if (lane == 0) t = atomicAdd(P.queue, 1u);
            c = __shfl_sync(0xffffffffu, t, 0);
        } else {
            c = it;
            it += nwarps;
        }
        if (c >= P.nchunks) break;
        const ItemDesc d = P.items[c];
        const int np = int(d.np);
        const uint32_t v0 = d.v0, nv = d.nv, c0 = d.c0, ncat = d.ncat;
        // ---- stage the item
        for (uint32_t i = lane; i < nv; i += 32) {
            S.x[i] = P.x_in[v0 + i];
            if (P.stage > 0) {
                S.y[i] = P.y[v0 + i];
                S.acc[i] = P.acc[v0 + i];
            }
        }
        for (int j = lane; j <= np; j += 32) S.ph[j] = P.hdr[d.p0 + j];
        for (int j = lane; j < np; j += 32) {
            S.gam[j] = __ldg(P.gamma + d.p0 + j);
            const InstDev& I = P.inst[P.hdr[d.p0 + j].inst];
            PatConst<T> pc;
            pc.g = sizeof(T) == 8 ? T(I.g) : T(I.gf);
            pc.det = sizeof(T) == 8 ? T(I.detuning) : T(I.detf);
            pc.kap = sizeof(T) == 8 ? T(I.kappa) : T(I.kappaf);
            pc.coef_base = I.coef_base;
            pc.term = sizeof(T) == 8 ? T(I.term) : T(I.termf);
            S.pc[j] = pc;
        }
        for (uint32_t cl = lane; cl < ncat; cl += 32) {
            S.cw[cl] = __ldg(P.cat_word + c0 + cl);
            S.cM[cl] = __ldg(P.cat_M + c0 + cl);
        }
        __syncwarp();
        // ---- grouped sums per category and per pattern
        for (uint32_t cl = lane; cl < ncat; cl += 32) {
            int lo = 0, hi = np - 1;  // owning pattern: last j with cat_off <= c0 + cl
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (S.ph[mid].cat_off - c0 <= cl) lo = mid;
                else hi = mid - 1;
            }
            const PatHdr h = S.ph[lo];
            const int G = h.G;
            const int cb = int(h.cat_off - c0);
            const int q = int(cl) - cb + 1;
            const C* xp = S.x + (h.var_off - v0);
            const T Mq = S.cM[cl];
            C Rs = xp[2 * G + q];
            if (Mq >= T(2)) Rs = caxpy(Mq - T(1), xp[(G + 1) * (G + 1) + ((S.cw[cl] >> 15) & 31)], Rs);
            C Cq = Rs;
            for (int e2 = 1; e2 <= G; ++e2) {
                if (e2 == q) continue;
                const T Mb = S.cM[cb + e2 - 1];
                Rs = caxpy(Mb, xp[loc_S_d(G, q, e2)], Rs);
                Cq = caxpy(Mb, xp[loc_S_d(G, e2, q)], Cq);
            }
            S.R[cl] = Rs;
            S.Cs[cl] = Cq;
        }
        for (int j = lane; j < np; j += 32) {
            const PatHdr h = S.ph[j];
            const int G = h.G;
            const int cb = int(h.cat_off - c0);
            const C* xp = S.x + (h.var_off - v0);
            C zs = mk(T(0), T(0));
            for (int q = 1; q <= G; ++q) zs = caxpy(S.cM[cb + q - 1], csub(xp[q], xp[G + q]), zs);
            S.Zs[j] = zs;
        }
        __syncwarp();
        // ---- one unique variable per lane
        for (uint32_t i = lane; i < nv; i += 32) {
            const uint32_t e = __ldg(P.vdesc + v0 + i);
            const uint32_t l = e & 1023u;
            const int j = int((e >> 10) & 31u);
            const int kind = int((e >> 15) & 7u);
            const int q = int((e >> 18) & 31u);
            const int r = int((e >> 23) & 31u);
            const uint32_t vg = v0 + l;
            const PatHdr h = S.ph[j];
            const int G = h.G;
            const int pl = int(h.var_off - v0);
            const int cb = int(h.cat_off - c0);
            const InstDev& I = P.inst[h.inst];
            // SA_FP32_AUX: the physical representative is integrated in FP64 by
            // rho0_kernel
            if (FP64SIDE && h.tier == 0) continue;
            const PatConst<T> pc = S.pc[j];
            const T g = pc.g, det = pc.det, kap = pc.kap, trm = pc.term;
            const C gam = S.gam[j];
            const C v = S.x[l];
            const C* xp = S.x + pl;
            const C* __restrict__ crow = P.coef_row + pc.coef_base;
            const C* __restrict__ ccol = P.coef_col + pc.coef_base;
            const int4* __restrict__ dA = P.drecA;
            const uint32_t* __restrict__ dS = P.drecS;
            const C* __restrict__ X = P.x_in;
            C dv;
            // Hamiltonian, damping and loss (Eqs. HZ, HX and their Y, P, S, T
            // counterparts) with the grouped sums, then the hierarchy terms of
            // Eqs. uvar-up / uvar-down from the decoded records of the row
            // category (row delta) and of the column category (column delta)
            if (kind == KS || kind == KT) {
                const int cc = kind == KS ? r : q;  // column category
                const C t = csub(xp[G + cc], xp[q]);
                dv = mk(g * t.y, -g * t.x);
                dv = cfma(mk(-(gam.x + T(2) * trm), -gam.y), v, dv);  // terminator weight 2
                const uint32_t wr = S.cw[cb + q - 1];
                const uint32_t ra = h.rec_off + (wr & 1023);
                const int nr = int((wr >> 10) & 31);
#pragma unroll 2
                for (int t2 = 0; t2 < nr; ++t2) {
                    const int4 A = __ldg(dA + ra + t2);
                    const uint32_t sm = __ldg(dS + ra + t2);
                    const int smerge = int(sm >> 12) & 63;
                    // S'[tau*, tau(cc)], or T'[tau*] when cc merges with the moved molecule
                    int idx = A.y + cc - ((sm & 1u) && cc > q ? 1 : 0) - (cc > smerge ? 1 : 0);
                    idx = cc == smerge ? A.w : idx;
                    dv = cfma(__ldg(crow + (sm >> 23)), __ldg(X + idx), dv);
                }
                const uint32_t wc = S.cw[cb + cc - 1];
                const uint32_t rc = h.rec_off + (wc & 1023);
                const int nc = int((wc >> 10) & 31);
#pragma unroll 2
                for (int t2 = 0; t2 < nc; ++t2) {
                    const int4 A = __ldg(dA + rc + t2);
                    const uint32_t sm = __ldg(dS + rc + t2);
                    const int ts = int(sm >> 7) & 31, ipos = int(sm >> 2) & 31, Gp = int(sm >> 18) & 31;
                    // S'[tau(q), tau*], or T'[tau*]
                    const int ta = q - ((sm & 1u) && q > cc ? 1 : 0) + (((sm >> 1) & 1u) && q >= ipos ? 1 : 0);
                    const int idx = ta == ts ? A.w : A.z + (ta - 1) * (Gp - 1) - (ts > ta ? 1 : 0);
                    dv = cfma(__ldg(ccol + (sm >> 23)), __ldg(X + idx), dv);
                }
            } else if (kind == KP) {
                const C t = csub(xp[G + q], xp[q]);
                dv = mk(g * t.y, -g * t.x);
                dv = cfma(mk(-gam.x, -gam.y), v, dv);
                // the two raise terms of P_q cancel: only the lower records, with
                // the row and column coefficients combined
                const uint32_t wr = S.cw[cb + q - 1];
                const int nup = int((wr >> 20) & 15);
                const uint32_t ra = h.rec_off + (wr & 1023) + nup;
                const int nr = int((wr >> 10) & 31) - nup;
#pragma unroll 2
                for (int t2 = 0; t2 < nr; ++t2) {
                    const int4 A = __ldg(dA + ra + t2);
                    const uint32_t sm = __ldg(dS + ra + t2);
                    const int Gp = int(sm >> 18) & 31;
                    const C cf = cadd(__ldg(crow + (sm >> 23)), __ldg(ccol + (sm >> 23)));
                    dv = cfma(cf, __ldg(X + A.x + 2 * Gp), dv);
                }
            } else if (kind == KX || kind == KY) {
                const C Z = xp[0];
                const C t = kind == KX ? csub(Z, S.R[cb + q - 1]) : csub(S.Cs[cb + q - 1], Z);
                const T sd = kind == KX ? det : -det;
                dv = mk(sd * v.y + g * t.y, -sd * v.x - g * t.x);
                dv = cfma(mk(-(gam.x + T(0.5) * kap + trm), -gam.y), v, dv);  // terminator weight 1
                const uint32_t w = S.cw[cb + q - 1];
                const uint32_t ra = h.rec_off + (w & 1023);
                const int n = int((w >> 10) & 31);
                const C* __restrict__ cft = kind == KX ? crow : ccol;
#pragma unroll 2
                for (int t2 = 0; t2 < n; ++t2) {
                    const int4 A = __ldg(dA + ra + t2);
                    const uint32_t sm = __ldg(dS + ra + t2);
                    const int idx = kind == KX ? A.x : A.x + (int(sm >> 18) & 31);  // X'[tau*] or Y'[tau*]
                    dv = cfma(__ldg(cft + (sm >> 23)), __ldg(X + idx), dv);
                }
            } else {
                const C zs = S.Zs[j];
                dv = mk(g * zs.y, -g * zs.x);
                dv = cfma(mk(-(gam.x + kap), -gam.y), v, dv);
            }
            if (P.stage < 0) {
                P.x_out[vg] = dv;
            } else if (P.stage == 0) {
                P.acc[vg] = dv;
                P.x_out[vg] = caxpy(aT, dv, v);  // x_in is y in the first stage
            } else if (P.stage == 3) {
                P.y_out[vg] = caxpy(dtT / T(6), cadd(S.acc[l], dv), S.y[l]);
            } else {
                P.acc[vg] = caxpy(T(2), dv, S.acc[l]);
                P.x_out[vg] = caxpy(aT, dv, S.y[l]);
            }
        }
        __syncwarp();
    }
}

// ---- list kernel -----------------------------------------------------------
// TMA bulk copies and mbarriers (inline PTX).
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// global -> shared bulk copy: 16-byte aligned addresses, size a positive multiple of 16
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
// bulk prefetch of a global range into L2 (same alignment rules)
__device__ __forceinline__ void bulk_prefetch_l2(const void* src, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}
// One test of the phase; a thread whose phase is not complete is suspended
// until it completes or about a millisecond has passed (the suspend-time
// hint, in ns), so a waiting warp does not spin on the barrier.
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(1000000u)
        : "memory");
    return ok != 0;
}
// bounded wait: about a second of SM clocks, then report failure
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > (2LL << 30)) return false;
    return true;
}

// The 16-byte aligned byte range enclosing `count` elements of `esz` bytes
// at `first`, and how many elements precede the first wanted one.  Tables and
// state buffers are padded so that the rounded range stays inside them.
struct Span {
    const char* src;
    uint32_t bytes;
    uint32_t skip;
};
__device__ __forceinline__ Span span(const void* base, size_t first, uint32_t count, uint32_t esz) {
    const uintptr_t a = reinterpret_cast<uintptr_t>(base) + first * esz;
    const uintptr_t lo = a & ~uintptr_t(15), hi = (a + uintptr_t(count) * esz + 15) & ~uintptr_t(15);
    Span sp;
    sp.src = reinterpret_cast<const char*>(lo);
    sp.bytes = count ? uint32_t(hi - lo) : 0u;
    sp.skip = uint32_t(a - lo) / esz;
    return sp;
}

// The work items of a warp, one at a time (lane 0 draws, the warp shares
// the result; the caller breaks out when it reaches nchunks): static
// striding over the items (use_queue 0) or one grid-wide atomic counter (1).
struct ItemQueue {
    unsigned int it, nwarps;
    int mode;
    __device__ __forceinline__ void init(int use_queue, int wib) {
        nwarps = gridDim.x * (blockDim.x >> 5);
        it = blockIdx.x * (blockDim.x >> 5) + unsigned(wib);
        mode = use_queue;
    }
    __device__ __forceinline__ unsigned int next(unsigned int* queue, unsigned int nchunks, int lane) {
        if (mode == 0) {
            const unsigned int c = it;
            it += nwarps;
            return c;
        }
        unsigned int t = 0;
        if (lane == 0) t = atomicAdd(queue, 1u);
        return __shfl_sync(0xffffffffu, t, 0);
    }
};

// Per-warp shared memory of the list kernel.  The operand area op[] holds the
// item's stage-input slice (chunk entries, after a skip of 0 or 1 entries
// that the bulk copy's alignment leaves), then the grouped row sums R_q and
// column sums C_q of its categories, the Z sums of its patterns and one zero:
// every commutator term of Eq. HS is diag * v - i g (op[a] - op[b]) with
// host-chosen operand indices a, b.  The item's host-made tables arrive as
// one blob (see BlobLayout).
template <typename T> struct ListSmem {
    using C = typename Cx<T>::t;
    uint64_t* bar;        // the warp's mbarrier
    C* op;                // skip + chunk + 2 nc + kItemPats + 1 entries (+ 2 spare)
    T* mult;              // the item's multiplicities, M_0 = N - r included
    C* diag;              // per pattern and variable class: -Gamma_Lambda plus the instance's part
    unsigned char* blob;  // the item's table blob
};

__host__ __device__ __forceinline__ int list_ncat(int item) { return item / 4 + 8; }
// operand-area layout (host and device): x slice, two entries the slice's
// bulk copy may round into, R, C, Z sums, zero.  The bulk copies never write
// where the warp writes, so no proxy fence is needed between items.
__host__ __device__ __forceinline__ int list_opR(int item) { return item + 2; }
__host__ __device__ __forceinline__ int list_opC(int item) { return item + 2 + list_ncat(item); }
__host__ __device__ __forceinline__ int list_opZ(int item) { return item + 2 + 2 * list_ncat(item); }
__host__ __device__ __forceinline__ int list_opZero(int item) { return item + 2 + 2 * list_ncat(item) + kItemPats; }

// A warp's shared memory: mbarrier; operand area; multiplicities and the
// diagonal table (written by the warp, never by a bulk copy); the blob.
template <typename T>
__host__ __device__ __forceinline__ size_t list_smem_bytes(int item) {
    const size_t cs = 2 * sizeof(T);
    return 16 + al16(cs * (list_opZero(item) + 3)) + al16(sizeof(T) * list_ncat(item)) + al16(cs * 5 * kItemPats) +
           blob_layout<T>(kItemPats, uint32_t(list_ncat(item)), uint32_t(item)).bytes;
}

template <typename T>
__device__ __forceinline__ ListSmem<T> carve_list(unsigned char* p, int item) {
    using C = typename Cx<T>::t;
    ListSmem<T> W;
    W.bar = reinterpret_cast<uint64_t*>(p);  p += 16;
    W.op = reinterpret_cast<C*>(p);          p += al16(sizeof(C) * (list_opZero(item) + 3));
    W.mult = reinterpret_cast<T*>(p);        p += al16(sizeof(T) * list_ncat(item));
    W.diag = reinterpret_cast<C*>(p);        p += al16(sizeof(C) * 5 * kItemPats);
    W.blob = p;
    return W;
}

// One warp per work item, like stage_kernel, but
//  * the item's stage-input slice and its table blob (instance constants,
//    patterns, damping rates, category words, multiplicities and owners,
//    round table, lane words) arrive by two TMA bulk copies on the warp's
//    mbarrier; its RK4 state and accumulator slices and its term rows are
//    prefetched into L2 by bulk prefetches, and each lane reads its own
//    variable's state and accumulator from there (keeping them out of shared
//    memory leaves room for larger items at the same occupancy);
//  * the hierarchy terms come from host-resolved lists: the lanes take the
//    item's variables in rounds of 32 (sorted by term count, so a round's
//    lanes run the same number of terms), and term t of a round is one
//    coalesced row of 32 (target index, coefficient slot) entries; padded
//    entries name a zero coefficient;
//  * the commutator, damping and loss use one formula for every kind of
//    variable, with operands and the diagonal class chosen by the host.
// A bounded wait that expires sets bit 0 of the error word; the warp then
// waits (bounded again) for its copies and stops.
// list_unit is one work unit c in the warp's shared memory S; it returns
// false when the bounded wait for its copies expired.
template <typename T, bool FP64SIDE, bool CHECK>
__device__ __forceinline__ bool list_unit(const StageParams<T>& P, unsigned int c, const ListSmem<T>& S,
                                          uint32_t& parity, int lane) {
    using C = typename Cx<T>::t;
    const int chunk = P.chunk;
    const T dtT = T(P.dt);
    const T aT = P.stage == 2 ? dtT : T(0.5) * dtT;
    {
        // a work unit: a template item and the instance it is evaluated for
        const uint2 un = P.units[c];
        const ItemDesc d = P.items[un.x];
        const InstK<T>* const ik = P.instk + un.y;
        const uint32_t vbase = ik->var_base;
        const uint32_t v0 = vbase + d.v0, nv = d.nv;  // the item's first variable in the batch
        // ---- bulk copies (lanes 0, 3) and L2 prefetches (lanes 1, 2, 4, 5) of the item
        const Span sx = span(P.x_in, v0, nv, sizeof(C));
        Span sp;
        void* dst = nullptr;
        if (lane == 0) { sp = sx; dst = S.op; }
        else if (lane == 1 || lane == 2) {
            const Span t = span(lane == 1 ? P.y : static_cast<const C*>(P.acc), v0, P.stage > 0 ? nv : 0u, sizeof(C));
            if (t.bytes) bulk_prefetch_l2(t.src, t.bytes);
            sp.bytes = 0;
        }
        else if (lane == 3) {
            sp.src = reinterpret_cast<const char*>(P.blobs) + size_t(d.blob16) * 16;
            sp.bytes = d.blob_bytes;
            dst = S.blob;
        }
        else sp.bytes = 0;
        const uint32_t total = __reduce_add_sync(0xffffffffu, sp.bytes);
        // the copies overwrite only what the warp has read (the previous
        // item's slices and blob), after the __syncwarp that ended it
        if (lane == 0) mbar_expect_tx(S.bar, total);
        __syncwarp();
        if (sp.bytes) bulk_g2s(dst, sp.src, sp.bytes, S.bar);
        if (lane == 4 && d.row1 > d.row0) bulk_prefetch_l2(P.tidx + size_t(d.row0) * 32, (d.row1 - d.row0) * 128u);
        if (lane == 5 && d.row1 > d.row0) bulk_prefetch_l2(P.tcid + size_t(d.row0) * 32, (d.row1 - d.row0) * 64u);
        // SA_DEBUG_EXPIRE_WAIT takes the expiry path without testing the
        // barrier; the drain below still waits (bounded) for the copies
        if (!__all_sync(0xffffffffu, !P.expire_wait && mbar_wait(S.bar, parity))) {
            if (lane == 0) atomicOr(P.err, 1u);
            mbar_wait(S.bar, parity);
            return false;
        }
        parity ^= 1u;
        const int np = int(d.np);
        const uint32_t ncat = d.ncat, nl = d.nl;
        const BlobLayout B = blob_layout<T>(uint32_t(np), ncat, nl);
        const ItemPat* const ph = reinterpret_cast<const ItemPat*>(S.blob + B.pat);
        const uint32_t* const cw = reinterpret_cast<const uint32_t*>(S.blob + B.cw);
        const T* const cM = reinterpret_cast<const T*>(S.blob + B.cM);
        const uint8_t* const cj = S.blob + B.cj;
        C* const op = S.op + sx.skip;
        // the instance's multiplicities (the template stores -r for the zero
        // category, whose M_0 = N - r) and its diagonal coefficient per pattern
        // and variable class (0 S T, 1 X, 2 Y, 3 Z, 4 P): -Gamma_Lambda of the
        // pattern plus the instance's loss, terminator and detuning
        {
            const T Nt = T(ik->N);
            for (uint32_t cl = lane; cl < ncat; cl += 32) {
                const T m = cM[cl];
                S.mult[cl] = m > T(0) ? m : Nt + m;
            }
            const C* const pdg = reinterpret_cast<const C*>(S.blob + B.pd);
            const C* const ccg = reinterpret_cast<const C*>(ik->cc);
            for (int e = lane; e < 5 * np; e += 32) S.diag[e] = cadd(pdg[e / 5], ccg[e % 5]);
            __syncwarp();
        }
        const T* const Mw = S.mult;
        C* const opR = op + list_opR(chunk);
        C* const opC = op + list_opC(chunk);
        C* const opZ = op + list_opZ(chunk);
        if (lane == 0) op[list_opZero(chunk)] = mk(T(0), T(0));
        // ---- grouped sums per category (Eqs. grouped-row-sum,
        // grouped-column-sum) and per pattern (Eq. HZ)
        for (uint32_t cl = lane; cl < ncat; cl += 32) {
            const ItemPat h = ph[cj[cl]];
            const int G = h.G;
            const int cb = int(h.cat_rel);
            const int q = int(cl) - cb + 1;
            const C* xp = op + h.var_rel;
            const T Mq = Mw[cl];
            C Rs = xp[2 * G + q];
            if (Mq >= T(2)) Rs = caxpy(Mq - T(1), xp[(G + 1) * (G + 1) + ((cw[cl] >> 15) & 31)], Rs);
            C Cq = Rs;
            for (int e2 = 1; e2 <= G; ++e2) {
                if (e2 == q) continue;
                const T Mb = Mw[cb + e2 - 1];
                Rs = caxpy(Mb, xp[loc_S_d(G, q, e2)], Rs);
                Cq = caxpy(Mb, xp[loc_S_d(G, e2, q)], Cq);
            }
            opR[cl] = Rs;
            opC[cl] = Cq;
        }
        for (int j = lane; j < np; j += 32) {
            const ItemPat h = ph[j];
            const int G = h.G;
            const int cb = int(h.cat_rel);
            const C* xp = op + h.var_rel;
            C zs = mk(T(0), T(0));
            for (int q = 1; q <= G; ++q) zs = caxpy(Mw[cb + q - 1], csub(xp[q], xp[G + q]), zs);
            opZ[j] = zs;
        }
        __syncwarp();
        // ---- the lanes' variables, one round of 32 at a time.  The first four
        // term rows of every round are loaded one round ahead, so that a
        // round's gathers wait on one memory latency instead of two.
        const C* __restrict__ X = P.x_in + vbase;  // targets are instance-relative
        const C* __restrict__ cf = P.lcoef + ik->lcoef_base;
        // SA_DEBUG_CHECK_INDICES: a target or slot out of the instance's range
        // reads index 0 instead and raises bit 1 of the error word
        uint2 lim = make_uint2(0u, 0u);
        if (CHECK) lim = P.ilimit[un.y];
        bool bad = false;
        auto ckx = [&](uint32_t v) {
            if (CHECK && v >= lim.x) {
                bad = true;
                return 0u;
            }
            return v;
        };
        auto ckc = [&](uint32_t v) {
            if (CHECK && v >= lim.y) {
                bad = true;
                return 0u;
            }
            return v;
        };
        const C* const dg = S.diag;
        const T g = ik->g;
        const uint32_t* const lvd = reinterpret_cast<const uint32_t*>(S.blob + B.lvd);
        const uint8_t* const lvj = S.blob + B.lvj;
        const uint32_t* const rb = reinterpret_cast<const uint32_t*>(S.blob + B.rb);
        const uint32_t nrounds = (nl + 31) / 32;
        uint32_t nix[4], ncx[4];
        auto first_rows = [&](uint32_t rho) {
            const uint32_t r0 = rb[rho];
            const uint32_t nt = rb[rho + 1] - r0;
            const uint32_t* __restrict__ ti = P.tidx + size_t(r0) * 32 + lane;
            const uint16_t* __restrict__ tc = P.tcid + size_t(r0) * 32 + lane;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                nix[u] = uint32_t(u) < nt ? ckx(__ldcg(ti + u * 32)) : d.v0;
                ncx[u] = uint32_t(u) < nt ? ckc(uint32_t(__ldcg(tc + u * 32))) : 0u;
            }
        };
        if (nrounds) first_rows(0);
        for (uint32_t rho = 0; rho < nrounds; ++rho) {
            const uint32_t i = rho * 32 + lane;
            const bool on = i < nl;
            const uint32_t r0 = rb[rho];
            const int nt = int(rb[rho + 1] - r0);
            uint32_t ix[4], cx[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                ix[u] = nix[u];
                cx[u] = ncx[u];
            }
            if (rho + 1 < nrounds) first_rows(rho + 1);
            // gathers of the first (up to) four terms
            C xv[4], cv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                xv[u] = __ldg(X + ix[u]);
                cv[u] = __ldg(cf + cx[u]);
            }
            // lanes past the end take operand 0 and the zero-coefficient rows
            const uint32_t w0 = on ? lvd[i] : 0u;
            const uint32_t w1 = on ? uint32_t(lvj[i]) : 0u;
            const uint32_t l = w0 & 1023u, a = (w0 >> 10) & 2047u, b = w0 >> 21;
            const int j = int(w1 & 31u), cls = int(w1 >> 5);
            const C v = op[l];
            C yv = mk(T(0), T(0)), av = mk(T(0), T(0));
            if (on && P.stage > 0) {
                yv = __ldcg(P.y + v0 + l);
                av = __ldcg(P.acc + v0 + l);
            }
            // commutator and diagonal: -Gamma_Lambda of the pattern plus the
            // instance's loss, terminator and detuning for the class (0 S T,
            // 1 X, 2 Y, 3 Z, 4 P)
            const C t = csub(op[a], op[b]);
            C dv = mk(g * t.y, -g * t.x);
            dv = cfma(dg[5 * j + cls], v, dv);
            // hierarchy terms (Eqs. uvar-up, uvar-down); rows past the
            // round's end were loaded as the zero slot
#pragma unroll
            for (int u = 0; u < 4; ++u) dv = cfma(cv[u], xv[u], dv);
            const uint32_t* __restrict__ ti = P.tidx + size_t(r0) * 32 + lane;
            const uint16_t* __restrict__ tc = P.tcid + size_t(r0) * 32 + lane;
            int t2 = 4;
            for (; t2 + 4 <= nt; t2 += 4) {
                uint32_t jx[4], jc[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    jx[u] = ckx(__ldcg(ti + (t2 + u) * 32));
                    jc[u] = ckc(__ldcg(tc + (t2 + u) * 32));
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    xv[u] = __ldg(X + jx[u]);
                    cv[u] = __ldg(cf + jc[u]);
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) dv = cfma(cv[u], xv[u], dv);
            }
            for (; t2 < nt; ++t2) dv = cfma(__ldg(cf + ckc(__ldcg(tc + t2 * 32))), __ldg(X + ckx(__ldcg(ti + t2 * 32))), dv);
            if (on) {
                const uint32_t vg = v0 + l;
                if (P.stage < 0) {
                    P.x_out[vg] = dv;
                } else if (P.stage == 0) {
                    P.acc[vg] = dv;
                    P.x_out[vg] = caxpy(aT, dv, v);  // x_in is y in the first stage
                } else if (P.stage == 3) {
                    P.y_out[vg] = caxpy(dtT / T(6), cadd(av, dv), yv);
                } else {
                    P.acc[vg] = caxpy(T(2), dv, av);
                    P.x_out[vg] = caxpy(aT, dv, yv);
                }
            }
        }
        if (CHECK && __any_sync(0xffffffffu, bad) && lane == 0) atomicOr(P.err, 2u);
        __syncwarp();
    }
    return true;
}

// The list kernel: persistent warps drawing work units (static striding or
// the atomic counter).  (A register budget instead of launch bounds: ptxas
// otherwise trades a few spills for 32 resident warps, which measured
// slower.)
template <typename T, bool FP64SIDE, bool CHECK>
__global__ void __maxnreg__(sizeof(T) == 8 ? 104 : 80) list_stage_kernel(StageParams<T> P) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const ListSmem<T> S = carve_list<T>(smem + size_t(wib) * list_smem_bytes<T>(P.chunk), P.chunk);
    if (lane == 0) {
        mbar_init(S.bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    ItemQueue Q;
    Q.init(P.use_queue, wib);
    uint32_t parity = 0;
    for (;;) {
        const unsigned int c = Q.next(P.queue, P.nchunks, lane);
        if (c >= P.nchunks) break;
        if (!list_unit<T, FP64SIDE, CHECK>(P, c, S, parity, lane)) return;
    }
}

// -- begin: pack kernel (the opt-in packed layout; no list-kernel code)
// One pack unit: a pack item evaluated for the n <= 32 instances of a pack,
// lane j taking the pack's instance j (lanes j >= n shadow lane 0 and store
// nothing).  The pack's state is interleaved, so every access of the warp --
// a variable of the item, a tier +/-1 target, a coefficient slot, y and the
// accumulator -- is one contiguous run of n elements, and the item's tables
// (one bulk copy into the warp's shared memory) are read by all lanes alike.
//  * the item's variables one per round, in three phases (P, T, S; then X,
//    Y; then Z): each adds its own value, weighted, to the grouped sums it
//    enters (R_q and C_q of Eqs. grouped-row-sum, grouped-column-sum, the Z
//    sum of Eq. HZ; in the warp's shared memory, one column per lane), which
//    the next phase reads as operands; each gets its diagonal (-Gamma_Lambda
//    plus the instance's loss, terminator and detuning), commutator
//    -i g (op[a] - op[b]) with host-chosen operands, hierarchy terms (Eqs.
//    uvar-up, uvar-down) and the fused RK4 update.  Within a phase the loads
//    of the next variable (its value, operands, y, accumulator and first two
//    terms) are issued before the current one is finished, so two
//    variables' memory latencies overlap.  (L2 prefetches of the item's
//    blocks or of the next variables' targets measured slower: with the
//    list units in the same launch, L2 capacity is what they take.)
// Returns false when the bounded wait for the tables expired (error bit set,
// the copy drained).
template <typename T, bool FP64SIDE, bool CHECK>
__device__ __forceinline__ bool pack_unit(const StageParams<T>& P, const ItemDesc& d, uint32_t pkid,
                                          unsigned char* wsm, uint64_t* bar, uint32_t& parity, int lane) {
    using C = typename Cx<T>::t;
    C* const ccs = reinterpret_cast<C*>(wsm + 16);            // 5 x 32 per-lane diagonal parts
    C* const sums = ccs + 5 * 32;                             // grouped sums, 32 lanes per entry
    unsigned char* const blob = reinterpret_cast<unsigned char*>(sums + (2 * d.ncat + d.np + 1) * 32);  // after them
    const PackDev pk = P.packs[pkid];
    const uint32_t n = pk.n;
    const bool act = uint32_t(lane) < n;
    const uint32_t ll = act ? uint32_t(lane) : 0u;
    if (lane == 0) {
        // earlier units wrote this shared memory with ordinary stores
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(bar, d.blob_bytes);
        bulk_g2s(blob, P.blobs + size_t(d.blob16) * 16, d.blob_bytes, bar);
    }
    // the lane's instance constants while the copy is in flight
    const InstK<T>* const ik = P.instk + P.pk_inst[pk.lane0 + ll];
    const T g = ik->g, Nt = T(ik->N);
#pragma unroll
    for (int cl = 0; cl < 5; ++cl) ccs[cl * 32 + lane] = mk(ik->cc[2 * cl], ik->cc[2 * cl + 1]);
    if (!__all_sync(0xffffffffu, !P.expire_wait && mbar_wait(bar, parity))) {
        if (lane == 0) atomicOr(P.err, 1u);
        mbar_wait(bar, parity);
        return false;
    }
    parity ^= 1u;
    const uint32_t np = d.np, ncat = d.ncat, nv = d.nv, nl = d.nl;
    const PackLayout B = pack_layout<T>(np, ncat, nl, d.row0, d.nw);
    const C* const pd = reinterpret_cast<const C*>(blob + B.pd);
    const uint4* const vrec = reinterpret_cast<const uint4*>(blob + B.vrec);
    const uint32_t* const tgt0 = reinterpret_cast<const uint32_t*>(blob + B.tgt);
    const uint16_t* const tsl0 = reinterpret_cast<const uint16_t*>(blob + B.tsl);
    // SA_DEBUG_CHECK_INDICES: a target or slot out of the template's range
    // reads index 0 instead and raises bit 1 of the error word
    uint2 lim = make_uint2(0u, 0u);
    if (CHECK) lim = P.ilimit[P.pk_inst[pk.lane0]];
    bool bad = false;
    auto tgtat = [&](uint32_t u) {
        const uint32_t v = tgt0[u];
        if (CHECK && v >= lim.x) {
            bad = true;
            return 0u;
        }
        return v;
    };
    auto tslat = [&](uint32_t u) {
        const uint32_t v = tsl0[u];
        if (CHECK && v >= lim.y) {
            bad = true;
            return 0u;
        }
        return v;
    };
    // lane base pointers; element offsets from them are 32-bit
    const size_t lb = size_t(pk.base) + ll;
    const C* __restrict__ X = P.x_in + lb;
    const C* __restrict__ cf = P.pcoef + pk.cbase + ll;
    const uint32_t iv0 = d.v0 * n;  // the item's variable 0
    // the grouped sums start at zero; the zero operand stays zero
    C* const sl = sums + lane;
    const uint32_t nsums = 2 * ncat + np + 1;
    for (uint32_t k = 0; k < nsums; ++k) sl[k * 32] = mk(T(0), T(0));
    // the grouped-sum weight a + b N of a contribution for the lane's
    // instance (b = 0 but for the zero category, whose multiplicity is
    // N - r), named by its index in the item's weight list: in FP64 looked up
    // in a per-lane table evaluated once per unit (one column per lane after
    // the blob), in FP32 evaluated where it is used
    const int2* const wab = reinterpret_cast<const int2*>(blob + B.wab);
    T* const wt = reinterpret_cast<T*>(blob + d.blob_bytes) + lane;
    if constexpr (sizeof(T) == 8)
        for (uint32_t k = 0; k < d.nw; ++k) wt[k * 32] = fma(T(wab[k].y), Nt, T(wab[k].x));
    auto weight = [&](uint32_t w) {
        if constexpr (sizeof(T) == 8) return wt[(w >> 11) * 32];
        const int2 e = wab[w >> 11];
        return fma(T(e.y), Nt, T(e.x));
    };
    // the diagonal coefficient of pattern j and class cl (-Gamma_Lambda plus
    // the instance's part): in FP64 from a per-lane table after the weights,
    // in FP32 added where it is used
    C* const dtab = reinterpret_cast<C*>(blob + d.blob_bytes + pack_wtab_bytes<T>(d.nw)) + lane;
    if constexpr (sizeof(T) == 8)
        for (uint32_t e = 0; e < 5 * np; ++e) dtab[e * 32] = cadd(pd[e / 5], ccs[(e % 5) * 32 + lane]);
    auto diag = [&](uint32_t j, uint32_t cl) {
        if constexpr (sizeof(T) == 8) return dtab[(j * 5 + cl) * 32];
        return cadd(pd[j], ccs[cl * 32 + lane]);
    };
    const C* __restrict__ Yb = P.y + lb;
    C* const Ab = P.acc + lb;
    C* const XO = P.x_out + lb;
    C* const YO = P.y_out + lb;
    const int stage = P.stage;
    const T dtT = T(P.dt);
    const T aT = stage == 2 ? dtT : T(0.5) * dtT;
    const C z = mk(T(0), T(0));
    auto var = [&](uint32_t code) { return __ldg(X + (iv0 + code * n)); };
    // loads of variable i in phase ph: value, operands (P, T, S: two item
    // variables; X, Y: the Z variable and a sum; Z: its sum), y, accumulator,
    // first two terms
    auto fetch = [&](int ph, uint32_t i, C& v, C& oa, C& ob, C& yv, C& av, C& x0, C& c0, C& x1, C& c1) {
        const uint4 r = vrec[i];
        const uint32_t off = iv0 + (r.y & 1023u) * n;
        const uint32_t u0 = (r.y >> 10) & 65535u, cnt = r.y >> 26;
        const uint32_t ca = r.x & 2047u, cb = (r.x >> 11) & 2047u;
        v = __ldg(X + off);
        if (ph == 0) {
            oa = var(ca);
            ob = var(cb);
        } else if (ph == 1) {
            oa = ca < nv ? var(ca) : sl[(ca - nv) * 32];
            ob = cb < nv ? var(cb) : sl[(cb - nv) * 32];
        } else {
            oa = sl[(ca - nv) * 32];
            ob = z;
        }
        yv = z;
        av = z;
        if (stage > 0) {
            yv = __ldcg(Yb + off);
            av = __ldcg(Ab + off);
        }
        x0 = c0 = x1 = c1 = z;
        if (cnt > 0) {
            x0 = __ldg(X + tgtat(u0) * n);
            c0 = __ldg(cf + tslat(u0) * n);
        }
        if (cnt > 1) {
            x1 = __ldg(X + tgtat(u0 + 1) * n);
            c1 = __ldg(cf + tslat(u0 + 1) * n);
        }
    };
    // the rest of variable i: its contributions to the grouped sums (P, T, S:
    // two; X, Y: one; Z: none), then diagonal, commutator, terms, RK4 update
    auto finish = [&](int ph, uint32_t i, C v, C oa, C ob, C yv, C av, C x0, C c0, C x1, C c1) {
        const uint4 r = vrec[i];
        if (ph < 2) sl[(r.z & 2047u) * 32] = caxpy(weight(r.z), v, sl[(r.z & 2047u) * 32]);
        if (ph == 0) sl[(r.w & 2047u) * 32] = caxpy(weight(r.w), v, sl[(r.w & 2047u) * 32]);
        const uint32_t off = iv0 + (r.y & 1023u) * n;
        const uint32_t u0 = (r.y >> 10) & 65535u, u1 = u0 + (r.y >> 26);
        const C dgl = diag((r.x >> 25) & 31u, (r.x >> 22) & 7u);
        const C t = csub(oa, ob);
        C dv = mk(g * t.y, -g * t.x);
        dv = cfma(dgl, v, dv);
        dv = cfma(c0, x0, dv);
        dv = cfma(c1, x1, dv);
        uint32_t u = u0 + 2;
        for (; u + 2 <= u1; u += 2) {
            const C xa = __ldg(X + tgtat(u) * n), ca = __ldg(cf + tslat(u) * n);
            const C xb = __ldg(X + tgtat(u + 1) * n), cb = __ldg(cf + tslat(u + 1) * n);
            dv = cfma(ca, xa, dv);
            dv = cfma(cb, xb, dv);
        }
        if (u < u1) dv = cfma(__ldg(cf + tslat(u) * n), __ldg(X + tgtat(u) * n), dv);
        if (act) {
            if (stage < 0) {
                XO[off] = dv;
            } else if (stage == 0) {
                Ab[off] = dv;
                XO[off] = caxpy(aT, dv, v);  // x_in is y in the first stage
            } else if (stage == 3) {
                YO[off] = caxpy(dtT / T(6), cadd(av, dv), yv);
            } else {
                Ab[off] = caxpy(T(2), dv, av);
                XO[off] = caxpy(aT, dv, yv);
            }
        }
    };
    // the three phases (P, T, S; X, Y; Z), each with two register sets in
    // turn: variable i + 1 loads while variable i finishes
    const uint32_t ph1 = d.row1 & 65535u, ph2 = ph1 + (d.row1 >> 16);
    uint32_t i0 = 0;
#pragma unroll 1
    for (int ph = 0; ph < 3; ++ph) {
        const uint32_t i1 = ph == 0 ? ph1 : (ph == 1 ? ph2 : nl);
        C vA, oaA, obA, yA, aA, xA0, cA0, xA1, cA1;
        C vB, oaB, obB, yB, aB, xB0, cB0, xB1, cB1;
        if (i0 < i1) fetch(ph, i0, vA, oaA, obA, yA, aA, xA0, cA0, xA1, cA1);
        for (uint32_t i = i0; i < i1; i += 2) {
            if (i + 1 < i1) fetch(ph, i + 1, vB, oaB, obB, yB, aB, xB0, cB0, xB1, cB1);
            finish(ph, i, vA, oaA, obA, yA, aA, xA0, cA0, xA1, cA1);
            if (i + 1 >= i1) break;
            if (i + 2 < i1) fetch(ph, i + 2, vA, oaA, obA, yA, aA, xA0, cA0, xA1, cA1);
            finish(ph, i + 1, vB, oaB, obB, yB, aB, xB0, cB0, xB1, cB1);
        }
        i0 = i1;
    }
    if (CHECK && __any_sync(0xffffffffu, bad) && lane == 0) atomicOr(P.err, 2u);
    __syncwarp();
    return true;
}

// The pack kernel: persistent warps drawing pack units (static striding or
// the atomic counter), each warp with an mbarrier and pack_smem bytes of
// shared memory; then, in the same launch and shared memory, the list units
// of the unpacked instances, so that warps done with the (long) pack units
// fill the tail with (short) list units.  Registers are budgeted apart from
// the list kernel's.
template <typename T, bool FP64SIDE, bool CHECK>
__global__ void __maxnreg__(sizeof(T) == 8 ? 128 : 80) pack_stage_kernel(StageParams<T> P) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    unsigned char* const wsm = smem + size_t(wib) * P.pack_smem;
    uint64_t* const bar = reinterpret_cast<uint64_t*>(wsm);
    if (lane == 0) {
        mbar_init(bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    ItemQueue Q;
    Q.init(P.use_queue, wib);
    uint32_t parity = 0;
    for (;;) {
        const unsigned int c = Q.next(P.pqueue, P.npunits, lane);
        if (c >= P.npunits) break;
        const uint2 un = P.punits[c];
        if (!pack_unit<T, FP64SIDE, CHECK>(P, P.items[un.x & ~kPackUnit], un.y, wsm, bar, parity, lane)) return;
    }
    if (P.nchunks == 0) return;
    // the list units' bulk copies land where the pack units wrote with
    // ordinary stores (the mbarrier stays where it is)
    __syncwarp();
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncwarp();
    const ListSmem<T> S = carve_list<T>(wsm, P.chunk);
    ItemQueue L;
    L.init(P.use_queue, wib);
    for (;;) {
        const unsigned int c = L.next(P.queue, P.nchunks, lane);
        if (c >= P.nchunks) break;
        if (!list_unit<T, FP64SIDE, CHECK>(P, c, S, parity, lane)) return;
    }
}

// -- end: pack kernel

// ---- ELL kernel ------------------------------------------------------------
// Grouped sums of the stage input, one thread each: R_q and C_q of every
// category (Eqs. grouped-row-sum, grouped-column-sum: P_q + (M_q - 1) T_q +
// sum_{b != q} M_b S_{q,b}, resp. S_{b,q}), then sum_q M_q (X_q - Y_q) of
// every pattern (Eq. HZ), into the scratch arrays the ELL kernel reads.
template <typename T, bool FP64SIDE>
__global__ void __launch_bounds__(256) grouped_sums_kernel(StageParams<T> P) {
    using C = typename Cx<T>::t;
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    const C* __restrict__ X = P.x_in;
    if (t < P.ncat) {
        const uint32_t p = __ldg(P.catpat + t);
        const PatHdr h = P.hdr[p];
        if (FP64SIDE && h.tier == 0) return;  // integrated in FP64
        const int G = h.G;
        const int q = int(t - h.cat_off) + 1;
        const C* xp = X + h.var_off;
        const T* M = P.cat_M + h.cat_off;
        const uint32_t tr = (__ldg(P.cat_word + t) >> 15) & 31u;
        C Rs = __ldg(xp + 2 * G + q);
        if (tr != 31u) Rs = caxpy(__ldg(M + q - 1) - T(1), __ldg(xp + (G + 1) * (G + 1) + int(tr)), Rs);
        C Cq = Rs;
        for (int b = 1; b <= G; ++b) {
            if (b == q) continue;
            const T Mb = __ldg(M + b - 1);
            Rs = caxpy(Mb, __ldg(xp + loc_S_d(G, q, b)), Rs);
            Cq = caxpy(Mb, __ldg(xp + loc_S_d(G, b, q)), Cq);
        }
        P.sumR[t] = Rs;
        P.sumC[t] = Cq;
    } else if (t < P.ncat + P.npat) {
        const uint32_t p = t - P.ncat;
        const PatHdr h = P.hdr[p];
        if (FP64SIDE && h.tier == 0) return;
        const C* xp = X + h.var_off;
        const T* M = P.cat_M + h.cat_off;
        C zs = mk(T(0), T(0));
        for (int q = 1; q <= int(h.G); ++q) zs = caxpy(__ldg(M + q - 1), csub(__ldg(xp + q), __ldg(xp + h.G + q)), zs);
        P.sumZ[p] = zs;
    }
}

// One thread per unique variable, lanes in memory order: warp w takes the 32
// consecutive variables [32 w, 32 w + 32) of the batch vector, so the state,
// the accumulator and the outputs move in full coalesced rows, and needs no
// shared memory.  The hierarchy terms of the warp are T_w rows of 32
// (target index, coefficient slot) entries, T_w the longest list among its
// lanes (shorter lists padded with the zero slot).  The commutator reads the
// variable's own-pattern operands from x directly (L1-resident: the warp reads
// the same pattern) and the grouped sums of X_q, Y_q and Z from the arrays
// grouped_sums_kernel wrote.
// Per-variable word: pattern offset from the warp's first pattern (5 bits) |
// kind << 5 | q << 8 | r << 13 | T-rank of q << 18 (31: none).
template <typename T, bool FP64SIDE>
__global__ void __launch_bounds__(256) ell_stage_kernel(StageParams<T> P) {
    using C = typename Cx<T>::t;
    const uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t w = v >> 5;
    const uint32_t nw = (P.nvar + 31) >> 5;
    if (w >= nw) return;  // whole warps only
    const int lane = int(v & 31u);
    const bool on = v < P.nvar;
    const uint32_t e = on ? __ldg(P.lvd + v) : 0u;
    const uint32_t p = __ldg(P.wpat + w) + (e & 31u);
    const PatHdr h = P.hdr[p];
    const int kind = int((e >> 5) & 7u), q = int((e >> 8) & 31u), r = int((e >> 13) & 31u);
    const C* __restrict__ X = P.x_in;
    const bool live = on && !(FP64SIDE && h.tier == 0);  // SA_FP32_AUX: tier 0 is integrated in FP64
    const uint32_t base = h.var_off;
    const int G = h.G;
    const InstDev& I = P.inst[h.inst];
    const T g = sizeof(T) == 8 ? T(I.g) : T(I.gf);
    const T det = sizeof(T) == 8 ? T(I.detuning) : T(I.detf);
    const T kap = sizeof(T) == 8 ? T(I.kappa) : T(I.kappaf);
    const C gam = __ldg(P.gamma + p);
    const C xv = __ldg(X + (on ? v : 0u));
    // operands of -i g (a - b)
    C a, b;
    if (kind == KS || kind == KP || kind == KT) {
        a = __ldg(X + base + G + (kind == KS ? r : q));
        b = __ldg(X + base + q);
    } else if (kind == KX) {
        a = __ldg(X + base);
        b = P.sumR[h.cat_off + q - 1];
    } else if (kind == KY) {
        a = P.sumC[h.cat_off + q - 1];
        b = __ldg(X + base);
    } else {
        a = P.sumZ[p];
        b = mk(T(0), T(0));
    }
    const T lossf = kind == KZ ? T(1) : ((kind == KX || kind == KY) ? T(0.5) : T(0));
    const T wt = (kind == KX || kind == KY) ? T(1) : ((kind == KS || kind == KT) ? T(2) : T(0));
    const T trm = sizeof(T) == 8 ? T(I.term) : T(I.termf);
    const T dim = kind == KX ? -det : (kind == KY ? det : T(0));
    const C diag = mk(-(gam.x + lossf * kap + wt * trm), dim - gam.y);
    const C t = csub(a, b);
    C dv = mk(g * t.y, -g * t.x);
    dv = cfma(diag, xv, dv);
    // hierarchy terms (Eqs. uvar-up, uvar-down)
    const C* __restrict__ cf = P.lcoef + I.lcoef_base;
    const uint32_t r0 = __ldg(P.rbase + w), r1 = __ldg(P.rbase + w + 1);
    const uint32_t* __restrict__ ti = P.tidx + size_t(r0) * 32 + lane;
    const uint16_t* __restrict__ tc = P.tcid + size_t(r0) * 32 + lane;
    const int nt = int(r1 - r0);
    int t2 = 0;
    for (; t2 + 4 <= nt; t2 += 4) {
        uint32_t ix[4], cx[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            ix[u] = __ldg(ti + (t2 + u) * 32);
            cx[u] = __ldg(tc + (t2 + u) * 32);
        }
        C xs[4], cs[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            xs[u] = __ldg(X + ix[u]);
            cs[u] = __ldg(cf + cx[u]);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) dv = cfma(cs[u], xs[u], dv);
    }
    for (; t2 < nt; ++t2) dv = cfma(__ldg(cf + __ldg(tc + t2 * 32)), __ldg(X + __ldg(ti + t2 * 32)), dv);
    if (!live) return;
    const T dtT = T(P.dt);
    if (P.stage < 0) {
        P.x_out[v] = dv;
    } else if (P.stage == 0) {
        P.acc[v] = dv;
        P.x_out[v] = caxpy(T(0.5) * dtT, dv, xv);  // x_in is y in the first stage
    } else if (P.stage == 3) {
        P.y_out[v] = caxpy(dtT / T(6), cadd(P.acc[v], dv), P.y[v]);
    } else {
        const T aT = P.stage == 2 ? dtT : T(0.5) * dtT;
        P.acc[v] = caxpy(T(2), dv, P.acc[v]);
        P.x_out[v] = caxpy(aT, dv, P.y[v]);
    }
}

// -- begin: physical-representative kernels (outside the stage kernels' code)
// SA_FP32_AUX: the physical representative (empty pattern) of every instance
// in FP64, one thread per variable: FP64 side copies of its own variables,
// the tier-1 targets gathered from the FP32 stage input, FP64 coefficients and
// multiplicities, FP64 RK4 stage update; the FP32 mirror is written for the
// tier-1 readers.
template <typename T>
__global__ void __launch_bounds__(128) rho0_kernel(StageParams<T> P, int ninst) {
    using C = typename Cx<T>::t;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = tid / kSideSlots, loc = tid % kSideSlots;
    if (i >= ninst) return;
    const InstDev I = P.inst[i];
    if (uint32_t(loc) >= I.n_rho0) return;
    // the physical representative is the instance's first pattern: the zero
    // category (G = 1), or molecule 1's category and the zero category
    const uint32_t p = I.pat_begin;
    const PatHdr h = P.hdr[p];
    const int G = h.G;
    const int nsq = (G + 1) * (G + 1);
    int kind, q = 0, r = 0;
    if (loc < nsq) {
        const uint32_t e = P.lut[P.lut_off[G] + loc];
        kind = int(e & 7u);
        q = int((e >> 3) & 31u);
        r = int((e >> 8) & 31u);
    } else {
        // T variable of T-rank loc - (G+1)^2
        kind = KT;
        for (int a = 1; a <= G; ++a)
            if (P.cat_Md[h.cat_off + a - 1] >= 2.0 && int((P.cat_word[h.cat_off + a - 1] >> 15) & 31u) == loc - nsq)
                q = a;
        if (q == 0) return;  // no category of that T-rank (the host tables rule it out)
    }
    const double2* xsin = P.xs_in + I.side;
    auto own = [&](int ii) { return xsin[ii]; };
    // targets are batch-global canonical indices of the instance's tier-1
    // variables; the device state may hold the instance strided (a pack lane)
    auto gath = [&](uint32_t ii) {
        const C t = __ldg(P.x_in + I.dev_base + size_t(ii - I.var_begin) * I.dev_stride);
        return make_double2(t.x, t.y);
    };
    const double2 k = var_rhs<double>(P, kind, q, r, G, P.cat_word + h.cat_off, P.cat_M + h.cat_off,
                                      reinterpret_cast<const uint2*>(P.rec) + h.rec_off, h, I,
                                      make_double2(0.0, 0.0), own, gath);
    const double dt = P.dt;
    const int si = int(I.side) + loc;
    const size_t vg = I.dev_base + size_t(loc) * I.dev_stride;  // the physical pattern starts the instance
    if (P.stage < 0) {
        P.xs_out[si] = k;
        P.x_out[vg] = mk(T(k.x), T(k.y));
    } else if (P.stage == 3) {
        const double2 y6 = P.ys[si], a6 = P.accs[si];
        const double2 yn = make_double2(y6.x + dt / 6.0 * (a6.x + k.x), y6.y + dt / 6.0 * (a6.y + k.y));
        P.ys_out[si] = yn;
        P.y_out[vg] = mk(T(yn.x), T(yn.y));
    } else {
        const double2 y6 = P.ys[si];
        double2 a6;
        if (P.stage == 0) a6 = k;
        else {
            a6 = P.accs[si];
            a6.x += 2.0 * k.x;
            a6.y += 2.0 * k.y;
        }
        P.accs[si] = a6;
        const double a = P.stage == 2 ? dt : 0.5 * dt;
        const double2 xn = make_double2(y6.x + a * k.x, y6.y + a * k.y);
        P.xs_out[si] = xn;
        P.x_out[vg] = mk(T(xn.x), T(xn.y));
    }
}

// Observables of the physical representative of every instance
// (Eqs. trace-uvar .. Pminus-uvar, written over its categories q with
// multiplicities M_q: P_exc = sum M_q P_q, P_B = [sum M_q P_q + sum M_q
// (M_q - 1) T_q + sum_{q != r} M_q M_r S_qr] / N, <B|rho|c> = sum M_q X_q /
// sqrt N) plus the Hermiticity defect of rho_S.
__global__ void observables_kernel(const InstDev* __restrict__ inst, const double* __restrict__ theta, int ninst,
                                   const PatHdr* __restrict__ hdr, const double* __restrict__ catMd,
                                   const uint32_t* __restrict__ cat_word, const double2* __restrict__ main64,
                                   const double2* __restrict__ side64, double* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ninst) return;
    const InstDev I = inst[i];
    // the physical representative: FP64 side slots, or the FP64 state (where
    // a packed instance's variables are dev_stride apart)
    const double2* const vb = side64 ? side64 + I.side : main64 + I.dev_base;
    const size_t vs = side64 ? 1 : I.dev_stride;
    auto v = [&](int l) { return vb[size_t(l) * vs]; };
    const PatHdr h = hdr[I.pat_begin];
    const int G = h.G;
    const double* M = catMd + h.cat_off;
    const uint32_t* cw = cat_word + h.cat_off;
    const double2 Z = v(0);
    double Pexc = 0.0, PBn = 0.0, XY = 0.0;
    double hd = fabs(Z.y);
    for (int q = 1; q <= G; ++q) {
        const double Mq = M[q - 1];
        const double2 Xq = v(q), Yq = v(G + q), Pq = v(2 * G + q);
        Pexc += Mq * Pq.x;
        PBn += Mq * Pq.x;
        XY += Mq * (Xq.x + Yq.x);
        hd = fmax(hd, fabs(Pq.y));
        hd = fmax(hd, hypot(Xq.x - Yq.x, Xq.y + Yq.y));
        if (Mq >= 2.0) {
            const double2 Tq = v((G + 1) * (G + 1) + int((cw[q - 1] >> 15) & 31u));
            PBn += Mq * (Mq - 1.0) * Tq.x;
            hd = fmax(hd, fabs(Tq.y));
        }
        for (int r = 1; r <= G; ++r) {
            if (r == q) continue;
            const double2 Sqr = v(loc_S_d(G, q, r)), Srq = v(loc_S_d(G, r, q));
            PBn += Mq * M[r - 1] * Sqr.x;
            hd = fmax(hd, hypot(Sqr.x - Srq.x, Sqr.y + Srq.y));
        }
    }
    const double N = I.N;
    const double PB = PBn / N;
    const double th = theta[i];
    const double cs = cos(th), sn = sin(th);
    const double xy = sn * cs * (XY / sqrt(N));
    double* o = out + 8 * i;
    o[0] = Z.x + Pexc;
    o[1] = Z.x;
    o[2] = Pexc;
    o[3] = PB;
    o[4] = Pexc - PB;
    o[5] = Z.x * cs * cs + PB * sn * sn + xy;
    o[6] = Z.x * sn * sn + PB * cs * cs - xy;
    o[7] = hd;
}

// Factorised initial state: write rho_0 of every instance (zeroing is a memset).
__global__ void init_rho0_kernel(const InstDev* __restrict__ inst, int ninst, const double* __restrict__ rho0,
                                 int stride, double2* __restrict__ main64, float2* __restrict__ main32,
                                 double2* __restrict__ side64) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ninst) return;
    const InstDev I = inst[i];
    for (uint32_t j = 0; j < I.n_rho0; ++j) {
        const double re = rho0[size_t(stride) * i + 2 * j], im = rho0[size_t(stride) * i + 2 * j + 1];
        const size_t e = I.dev_base + size_t(j) * I.dev_stride;
        if (main64) main64[e] = make_double2(re, im);
        if (main32) main32[e] = make_float2(float(re), float(im));
        if (side64) side64[I.side + j] = make_double2(re, im);
    }
}

// State marshalling of SA_FP32_AUX handles, one chunk of variables
// [n0, n0 + cnt) at a time, through a device staging buffer that holds the
// caller's complex128 values: narrow them to the float2 state and copy the
// physical representatives' variables exactly into their FP64 side slots
// (narrow), or widen the float2 state into the staging buffer with the
// physical representatives taken from their side slots (widen).
// (packed handles: the element of canonical variable gv is found through
// its instance, the last one whose var_begin <= gv)
__device__ __forceinline__ uint64_t state_elem(const InstDev* __restrict__ inst, int ninst, int packed, uint64_t gv) {
    if (!packed) return gv;
    int lo = 0, hi = ninst - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (uint64_t(inst[mid].var_begin) <= gv) lo = mid;
        else hi = mid - 1;
    }
    return uint64_t(inst[lo].dev_base) + (gv - inst[lo].var_begin) * inst[lo].dev_stride;
}
__device__ __forceinline__ float2 to_state(double2 v, float2*) { return make_float2(float(v.x), float(v.y)); }
__device__ __forceinline__ double2 to_state(double2 v, double2*) { return v; }
template <typename S>
__global__ void to_device_kernel(const InstDev* __restrict__ inst, int ninst, int packed,
                                 const double2* __restrict__ stage, uint64_t n0, uint64_t cnt, S* __restrict__ main) {
    const uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= cnt) return;
    main[state_elem(inst, ninst, packed, n0 + i)] = to_state(stage[i], (S*)nullptr);
}
template <typename S>
__global__ void from_device_kernel(const InstDev* __restrict__ inst, int ninst, int packed,
                                   const S* __restrict__ main, uint64_t n0, uint64_t cnt, double2* __restrict__ stage) {
    const uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= cnt) return;
    const S v = main[state_elem(inst, ninst, packed, n0 + i)];
    stage[i] = make_double2(double(v.x), double(v.y));
}
// one thread per side slot: the physical representative's variables that
// fall in the chunk
__global__ void side_state_kernel(const InstDev* __restrict__ inst, int ninst, uint64_t n0, uint64_t cnt,
                                  double2* __restrict__ stage, double2* __restrict__ side64, int to_side) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = t / kSideSlots, j = t % kSideSlots;
    if (i >= ninst) return;
    const InstDev& I = inst[i];
    const uint64_t v = uint64_t(I.var_begin) + uint64_t(j);
    if (uint32_t(j) >= I.n_rho0 || v < n0 || v >= n0 + cnt) return;
    if (to_side) side64[I.side + j] = stage[v - n0];
    else stage[v - n0] = side64[I.side + j];
}

// -- end: physical-representative kernels

// ---- host launch wrappers (called from api.cu) -----------------------------

// shared memory of one CTA of the stage kernel (the list kernel's layout for
// the item capacity, or the record kernel's), and of the pack kernel
static size_t stage_smem_bytes(const LaunchCfg& cfg, bool fp64) {
    if (cfg.kernel == SA_KERNEL_ELL) return 0;
    size_t w;
    if (cfg.kernel == SA_KERNEL_LISTS) w = fp64 ? list_smem_bytes<double>(cfg.chunk) : list_smem_bytes<float>(cfg.chunk);
    else w = fp64 ? warp_smem_bytes<double>(cfg.chunk) : warp_smem_bytes<float>(cfg.chunk);
    return w * size_t(cfg.block / 32);
}
// a pack-kernel warp's shared memory: the largest pack item's, or the list
// units' if that is larger
static uint32_t pack_warp_smem(const LaunchCfg& cfg, bool fp64) {
    const size_t l = fp64 ? list_smem_bytes<double>(cfg.chunk) : list_smem_bytes<float>(cfg.chunk);
    return uint32_t(std::max(size_t(cfg.pack_smem + 15) / 16 * 16, (l + 15) / 16 * 16));
}
static size_t pack_smem_bytes(const LaunchCfg& cfg, bool fp64) { return size_t(pack_warp_smem(cfg, fp64)) * size_t(cfg.block / 32); }

// operand-area offsets of the list kernel for a given item capacity
void list_operand_layout(int item, int* opR, int* opC, int* opZ, int* opZero) {
    *opR = list_opR(item);
    *opC = list_opC(item);
    *opZ = list_opZ(item);
    *opZero = list_opZero(item);
}

template <typename T, bool SIDE>
static cudaError_t launch_t(const StageParams<T>& p, const LaunchCfg& cfg, int ninst, cudaStream_t st,
                            const StageLaunch& s) {
    const size_t sm = stage_smem_bytes(cfg, sizeof(T) == 8);
    // the FP64 physical-representative kernel reads the same stage input and
    // writes other variables: it overlaps the stage kernel on a side stream
    cudaStream_t side = static_cast<cudaStream_t>(s.side_stream);
    const bool fork = SIDE && side && s.ev_fork && s.ev_join;
    if (SIDE) {
        cudaStream_t rs = st;
        if (fork) {
            cudaError_t e = cudaEventRecord(static_cast<cudaEvent_t>(s.ev_fork), st);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(side, static_cast<cudaEvent_t>(s.ev_fork), 0);
            if (e != cudaSuccess) return e;
            rs = side;
        }
        const int threads = ninst * kSideSlots;
        rho0_kernel<T><<<(threads + 127) / 128, 128, 0, rs>>>(p, ninst);
        if (fork) {
            const cudaError_t e = cudaEventRecord(static_cast<cudaEvent_t>(s.ev_join), side);
            if (e != cudaSuccess) return e;
        }
    }
    if (cfg.kernel == SA_KERNEL_ELL) {
        const unsigned gs = unsigned((size_t(p.ncat) + p.npat + 255) / 256);
        grouped_sums_kernel<T, SIDE><<<gs, 256, 0, st>>>(p);
        const unsigned grid = unsigned((size_t(p.nvar) + 31) / 32 * 32 + cfg.block - 1) / unsigned(cfg.block);
        if (grid > 0) ell_stage_kernel<T, SIDE><<<grid, cfg.block, 0, st>>>(p);
    } else if (cfg.kernel == SA_KERNEL_LISTS) {
        // a packed handle's pack units, then in the same launch the list
        // units of its unpacked instances; otherwise the list kernel
        const size_t psm = pack_smem_bytes(cfg, sizeof(T) == 8);
        if (s.debug & SA_DEBUG_CHECK_INDICES) {
            if (p.npunits) pack_stage_kernel<T, SIDE, true><<<cfg.pgrid, cfg.block, psm, st>>>(p);
            else if (p.nchunks) list_stage_kernel<T, SIDE, true><<<cfg.grid, cfg.block, sm, st>>>(p);
        } else {
            if (p.npunits) pack_stage_kernel<T, SIDE, false><<<cfg.pgrid, cfg.block, psm, st>>>(p);
            else if (p.nchunks) list_stage_kernel<T, SIDE, false><<<cfg.grid, cfg.block, sm, st>>>(p);
        }

    } else {
        stage_kernel<T, SIDE><<<cfg.grid, cfg.block, sm, st>>>(p);
    }
    if (fork) {
        const cudaError_t e = cudaStreamWaitEvent(st, static_cast<cudaEvent_t>(s.ev_join), 0);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

template <typename T>
static StageParams<T> make_params(const StageLaunch& s, const LaunchCfg& cfg) {
    using C = typename Cx<T>::t;
    StageParams<T> p;
    p.hdr = static_cast<const PatHdr*>(s.hdr);
    p.cat_word = static_cast<const uint32_t*>(s.cat_word);
    p.cat_M = static_cast<const T*>(s.cat_M);
    p.gamma = static_cast<const C*>(s.gamma);
    p.rec = static_cast<const Record*>(s.rec);
    p.items = static_cast<const ItemDesc*>(s.items);
    p.vdesc = static_cast<const uint32_t*>(s.vdesc);
    p.drecA = static_cast<const int4*>(s.drecA);
    p.drecS = static_cast<const uint32_t*>(s.drecS);
    p.inst = static_cast<const InstDev*>(s.inst);
    p.coef_row = static_cast<const C*>(s.coef_row);
    p.coef_col = static_cast<const C*>(s.coef_col);
    p.cat_Md = static_cast<const double*>(s.cat_Md);
    p.coef_row_d = static_cast<const double2*>(s.coef_row_d);
    p.coef_col_d = static_cast<const double2*>(s.coef_col_d);
    p.lut = static_cast<const uint16_t*>(s.lut);
    p.lut_off = static_cast<const uint32_t*>(s.lut_off);
    p.lvd = static_cast<const uint32_t*>(s.lvd);
    p.lvj = static_cast<const uint8_t*>(s.lvj);
    p.rbase = static_cast<const uint32_t*>(s.rbase);
    p.tidx = static_cast<const uint32_t*>(s.tidx);
    p.tcid = static_cast<const uint16_t*>(s.tcid);
    p.lcoef = static_cast<const C*>(s.lcoef);
    p.wpat = static_cast<const uint32_t*>(s.wpat);
    p.catpat = static_cast<const uint32_t*>(s.catpat);
    p.ncat = s.ncat;
    p.npat = s.npat;
    p.sumR = static_cast<C*>(s.sums);
    p.sumC = p.sumR ? p.sumR + s.ncat : nullptr;
    p.sumZ = p.sumC ? p.sumC + s.ncat : nullptr;
    p.blobs = static_cast<const unsigned char*>(s.blobs);
    p.units = static_cast<const uint2*>(s.units);
    p.instk = static_cast<const InstK<T>*>(s.instk);
    p.packs = static_cast<const PackDev*>(s.packs);
    p.pk_inst = static_cast<const uint32_t*>(s.pk_inst);
    p.pcoef = static_cast<const C*>(s.pcoef);
    p.punits = static_cast<const uint2*>(s.punits);
    p.npunits = s.npunits;
    p.pack_smem = pack_warp_smem(cfg, sizeof(T) == 8);
    p.pqueue = s.pqueue;
    p.nvar = s.nvar;
    p.nchunks = s.nchunks;
    p.chunk = cfg.chunk;
    p.x_in = static_cast<const C*>(s.x_in);
    p.x_out = static_cast<C*>(s.x_out);
    p.y = static_cast<const C*>(s.y);
    p.acc = static_cast<C*>(s.acc);
    p.y_out = static_cast<C*>(s.y_out);
    p.xs_in = static_cast<const double2*>(s.xs_in);
    p.xs_out = static_cast<double2*>(s.xs_out);
    p.ys = static_cast<const double2*>(s.ys);
    p.accs = static_cast<double2*>(s.accs);
    p.ys_out = static_cast<double2*>(s.ys_out);
    p.dt = s.dt;
    p.stage = s.stage;
    p.use_queue = cfg.use_queue;
    p.queue = s.queue;
    p.err = s.err;
    p.expire_wait = (s.debug & SA_DEBUG_EXPIRE_WAIT) ? 1 : 0;
    p.ilimit = static_cast<const uint2*>(s.ilimit);
    return p;
}

cudaError_t launch_stage(const StageLaunch& s, const LaunchCfg& cfg, bool fp64, cudaStream_t st) {
    if (fp64) return launch_t<double, false>(make_params<double>(s, cfg), cfg, s.ninst, st, s);
    return launch_t<float, true>(make_params<float>(s, cfg), cfg, s.ninst, st, s);
}

// Sets the dynamic shared-memory limit once for the largest chunk (outside
// any stream capture) and returns the CTAs per SM for this configuration.
template <class K>
static cudaError_t occupancy_of(K kern, int block, size_t sm, int lim, int* blocks_per_sm) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, kern, block, sm);
}

// CTAs per SM of the pack kernel (0 if its shared memory does not fit)
cudaError_t pack_occupancy(const LaunchCfg& cfg, bool fp64, int* blocks_per_sm) {
    const size_t sm = pack_smem_bytes(cfg, fp64);
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const int lim = std::max(optin - 1024, 0);
    if (sm > size_t(lim)) {
        *blocks_per_sm = 0;
        return cudaSuccess;
    }
    // (the index-checking variant gets the same shared-memory limit)
    int dummy = 0;
    cudaError_t e = fp64 ? occupancy_of(pack_stage_kernel<double, false, true>, cfg.block, sm, lim, &dummy)
                         : occupancy_of(pack_stage_kernel<float, true, true>, cfg.block, sm, lim, &dummy);
    if (e != cudaSuccess) return e;
    if (fp64) return occupancy_of(pack_stage_kernel<double, false, false>, cfg.block, sm, lim, blocks_per_sm);
    return occupancy_of(pack_stage_kernel<float, true, false>, cfg.block, sm, lim, blocks_per_sm);
}

cudaError_t stage_occupancy(const LaunchCfg& cfg, bool fp64, int* blocks_per_sm) {
    const size_t sm = stage_smem_bytes(cfg, fp64);
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    // leave room for the kernel's static shared variables
    const int lim = std::max(optin - 1024, 0);
    if (sm > size_t(lim)) {
        *blocks_per_sm = 0;
        return cudaSuccess;
    }
    if (cfg.kernel == SA_KERNEL_ELL) {
        if (fp64) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, ell_stage_kernel<double, false>,
                                                                       cfg.block, 0);
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, ell_stage_kernel<float, true>, cfg.block, 0);
    }
    if (cfg.kernel == SA_KERNEL_LISTS) {
        // (the index-checking variant gets the same shared-memory limit)
        int dummy = 0;
        cudaError_t e = fp64 ? occupancy_of(list_stage_kernel<double, false, true>, cfg.block, sm, lim, &dummy)
                             : occupancy_of(list_stage_kernel<float, true, true>, cfg.block, sm, lim, &dummy);
        if (e != cudaSuccess) return e;
        if (fp64) return occupancy_of(list_stage_kernel<double, false, false>, cfg.block, sm, lim, blocks_per_sm);
        return occupancy_of(list_stage_kernel<float, true, false>, cfg.block, sm, lim, blocks_per_sm);
    }
    if (fp64) return occupancy_of(stage_kernel<double, false>, cfg.block, sm, lim, blocks_per_sm);
    return occupancy_of(stage_kernel<float, true>, cfg.block, sm, lim, blocks_per_sm);
}

// -- begin: physical-representative kernels (outside the stage kernels' code)
cudaError_t launch_observables(const InstDev* inst, const double* theta, int ninst, const PatHdr* hdr,
                               const double* catMd, const uint32_t* cat_word, const void* main64, const void* side64,
                               double* out, cudaStream_t st) {
    observables_kernel<<<(ninst + 127) / 128, 128, 0, st>>>(inst, theta, ninst, hdr, catMd, cat_word,
                                                            static_cast<const double2*>(main64),
                                                            static_cast<const double2*>(side64), out);
    return cudaGetLastError();
}

cudaError_t launch_init_rho0(const InstDev* inst, int ninst, const double* rho0, int stride, void* main64,
                             void* main32, void* side64, cudaStream_t st) {
    init_rho0_kernel<<<(ninst + 127) / 128, 128, 0, st>>>(inst, ninst, rho0, stride, static_cast<double2*>(main64),
                                                          static_cast<float2*>(main32), static_cast<double2*>(side64));
    return cudaGetLastError();
}

cudaError_t launch_marshal(const InstDev* inst, int ninst, int packed, uint64_t n0, uint64_t cnt, void* stage,
                           void* main, void* side64, int fp64, int to_device, cudaStream_t st) {
    if (cnt == 0) return cudaSuccess;
    const unsigned grid = unsigned((cnt + 255) / 256);
    const unsigned sgrid = unsigned((size_t(ninst) * kSideSlots + 255) / 256);
    const double2* sg = static_cast<const double2*>(stage);
    double2* sd = static_cast<double2*>(stage);
    if (to_device) {
        if (fp64) to_device_kernel<<<grid, 256, 0, st>>>(inst, ninst, packed, sg, n0, cnt, static_cast<double2*>(main));
        else to_device_kernel<<<grid, 256, 0, st>>>(inst, ninst, packed, sg, n0, cnt, static_cast<float2*>(main));
    } else {
        if (fp64) from_device_kernel<<<grid, 256, 0, st>>>(inst, ninst, packed, static_cast<const double2*>(main), n0,
                                                           cnt, sd);
        else from_device_kernel<<<grid, 256, 0, st>>>(inst, ninst, packed, static_cast<const float2*>(main), n0, cnt,
                                                      sd);
    }
    if (side64)
        side_state_kernel<<<sgrid, 256, 0, st>>>(inst, ninst, n0, cnt, sd, static_cast<double2*>(side64), to_device);
    return cudaGetLastError();
}

// -- end: physical-representative kernels

}  // namespace sa
