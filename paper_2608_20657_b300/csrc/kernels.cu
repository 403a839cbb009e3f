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
    const uint32_t* __restrict__ chunk_begin;  // nchunks + 1
    const InstDev* __restrict__ inst;
    const C* __restrict__ coef_row;
    const C* __restrict__ coef_col;
    const double* __restrict__ cat_Md;      // FP64 copies for the FP64 physical representative
    const double2* __restrict__ coef_row_d;
    const double2* __restrict__ coef_col_d;
    const uint16_t* __restrict__ lut;       // (kind | q << 3 | r << 8) per (G, local index)
    const uint32_t* __restrict__ lut_off;   // per G
    uint32_t nchunks;
    int chunk;                              // variable capacity of the staged slice
    int rec_cap;                            // record capacity of the staged slice
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
        const CA dm = cadd(gam, mk(A(0.5) * kap, A(0)));
        d = cfma(mk(-dm.x, -dm.y), v, d);
    } else {
        // P, T: -i g (Y_q - X_q);  S_{q,r}: -i g (Y_r - X_q)
        const CA t = csub(own(G + (kind == KS ? r : q)), own(q));
        d = mk(g * t.y, -g * t.x);
        d = cfma(mk(-gam.x, -gam.y), v, d);
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

// Shared-memory image of one work item (a chunk of consecutive patterns).
template <typename T> struct ChunkSmem {
    using C = typename Cx<T>::t;
    C* x;            // stage input slice
    C* R;            // grouped row sums R_q per category
    C* Cs;           // grouped column sums C_q per category
    C* Zs;           // sum_q M_q (X_q - Y_q) per pattern
    C* crow;         // decoded record: row coefficient
    C* ccol;         // decoded record: column coefficient
    int4* dA;        // decoded record: X'-index, S'-row base, S'-column base, T'-index
    uint32_t* dS;    // decoded record: small fields
    uint2* rec;      // raw records (the FP64 physical-representative path)
    PatHdr* hdr;
    uint32_t* cw;
    T* cM;
    uint32_t* perm;  // work order: l | j << 11 | kind << 19 | q << 22 | r << 27
    uint16_t* sb;
    uint16_t* ob;
};

template <typename T>
__device__ __forceinline__ ChunkSmem<T> carve(unsigned char* base, int chunk, int rec_cap) {
    using C = typename Cx<T>::t;
    ChunkSmem<T> S;
    const int ncat = chunk / 4 + 8;
    unsigned char* p = base;
    S.x = reinterpret_cast<C*>(p);       p += sizeof(C) * chunk;
    S.R = reinterpret_cast<C*>(p);       p += sizeof(C) * ncat;
    S.Cs = reinterpret_cast<C*>(p);      p += sizeof(C) * ncat;
    S.Zs = reinterpret_cast<C*>(p);      p += sizeof(C) * kMaxPatPerChunk;
    S.crow = reinterpret_cast<C*>(p);    p += sizeof(C) * rec_cap;
    S.ccol = reinterpret_cast<C*>(p);    p += sizeof(C) * rec_cap;
    S.dA = reinterpret_cast<int4*>(p);   p += sizeof(int4) * rec_cap;
    S.rec = reinterpret_cast<uint2*>(p); p += sizeof(uint2) * rec_cap;
    S.dS = reinterpret_cast<uint32_t*>(p); p += sizeof(uint32_t) * rec_cap;
    S.hdr = reinterpret_cast<PatHdr*>(p);  p += sizeof(PatHdr) * (kMaxPatPerChunk + 1);
    S.cw = reinterpret_cast<uint32_t*>(p); p += sizeof(uint32_t) * ncat;
    S.perm = reinterpret_cast<uint32_t*>(p); p += sizeof(uint32_t) * chunk;
    S.cM = reinterpret_cast<T*>(p);      p += sizeof(T) * ncat;
    S.sb = reinterpret_cast<uint16_t*>(p); p += sizeof(uint16_t) * kMaxPatPerChunk;
    S.ob = reinterpret_cast<uint16_t*>(p);
    return S;
}

template <typename T, bool FP64SIDE>
__global__ void __launch_bounds__(256) stage_kernel(StageParams<T> P) {
    using C = typename Cx<T>::t;
    extern __shared__ __align__(16) unsigned char smem[];
    const ChunkSmem<T> S = carve<T>(smem, P.chunk, P.rec_cap);
    __shared__ unsigned int s_c, s_nS;

    const T dtT = T(P.dt);
    const T aT = P.stage == 2 ? dtT : T(0.5) * dtT;
    unsigned int iter = 0;
    for (;;) {
        unsigned int c;
        if (P.use_queue) {
            if (threadIdx.x == 0) s_c = atomicAdd(P.queue, 1u);
            __syncthreads();
            c = s_c;
        } else {
            c = blockIdx.x + iter * gridDim.x;
            ++iter;
        }
        if (c >= P.nchunks) break;
        const uint32_t p0 = __ldg(P.chunk_begin + c), p1 = __ldg(P.chunk_begin + c + 1);
        const int np = int(p1 - p0);
        // ---- phase 1: stage the chunk (every thread reads the ranges itself)
        const PatHdr h0 = P.hdr[p0], h1 = P.hdr[p1];
        const uint32_t v0 = h0.var_off, nv = h1.var_off - v0;
        const uint32_t c0 = h0.cat_off, ncat = h1.cat_off - c0;
        const uint32_t r0 = h0.rec_off, nrec = h1.rec_off - r0;
        for (int j = threadIdx.x; j <= np; j += blockDim.x) S.hdr[j] = P.hdr[p0 + j];
        for (uint32_t l = threadIdx.x; l < nv; l += blockDim.x) S.x[l] = P.x_in[v0 + l];
        for (uint32_t l = threadIdx.x; l < nrec; l += blockDim.x)
            S.rec[l] = __ldg(reinterpret_cast<const uint2*>(P.rec) + r0 + l);
        for (uint32_t l = threadIdx.x; l < ncat; l += blockDim.x) {
            S.cw[l] = __ldg(P.cat_word + c0 + l);
            S.cM[l] = __ldg(P.cat_M + c0 + l);
        }
        __syncthreads();
        // ---- phase 2: warp 0 scans the work-order counts; the other threads
        // take the categories: grouped sums R_q, C_q (Eqs. grouped-row-sum,
        // grouped-column-sum) and the decoding of the category's records
        if (threadIdx.x < 32) {
            const int lane = threadIdx.x;
            const int per = (np + 31) / 32;
            const int a = lane * per, b = min(np, a + per);
            int ss = 0, so = 0;
            for (int j = a; j < b; ++j) {
                const int G = S.hdr[j].G;
                const int u = int(S.hdr[j + 1].var_off - S.hdr[j].var_off);
                ss += G * (G - 1);
                so += u - G * (G - 1);
            }
            int is = ss, io = so;
            for (int off = 1; off < 32; off <<= 1) {
                const int ts = __shfl_up_sync(0xffffffffu, is, off);
                const int to = __shfl_up_sync(0xffffffffu, io, off);
                if (lane >= off) {
                    is += ts;
                    io += to;
                }
            }
            int bs = is - ss, bo = io - so;
            for (int j = a; j < b; ++j) {
                const int G = S.hdr[j].G;
                const int u = int(S.hdr[j + 1].var_off - S.hdr[j].var_off);
                S.sb[j] = uint16_t(bs);
                S.ob[j] = uint16_t(bo);
                bs += G * (G - 1);
                bo += u - G * (G - 1);
            }
            if (lane == 31) s_nS = uint32_t(is);
        } else {
            for (uint32_t cl = threadIdx.x - 32; cl < ncat; cl += blockDim.x - 32) {
                // owning pattern: last j with cat_off <= c0 + cl
                int lo = 0, hi = np - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (S.hdr[mid].cat_off - c0 <= cl) lo = mid;
                    else hi = mid - 1;
                }
                const PatHdr& h = S.hdr[lo];
                const int G = h.G;
                const int cb = int(h.cat_off - c0);
                const int q = int(cl) - cb + 1;
                const C* xp = S.x + (h.var_off - v0);
                const uint32_t w = S.cw[cl];
                const T Mq = S.cM[cl];
                C Rs = xp[2 * G + q];
                if (Mq >= T(2)) Rs = caxpy(Mq - T(1), xp[(G + 1) * (G + 1) + ((w >> 15) & 31)], Rs);
                C Cq = Rs;
                for (int b = 1; b <= G; ++b) {
                    if (b == q) continue;
                    const T Mb = S.cM[cb + b - 1];
                    Rs = caxpy(Mb, xp[loc_S_d(G, q, b)], Rs);
                    Cq = caxpy(Mb, xp[loc_S_d(G, b, q)], Cq);
                }
                S.R[cl] = Rs;
                S.Cs[cl] = Cq;
                const InstDev& I = P.inst[h.inst];
                const int nr = (w >> 10) & 31;
                const int rl = int(h.rec_off - r0) + int(w & 1023);
                for (int t = 0; t < nr; ++t) {
                    const uint2 raw = S.rec[rl + t];
                    const uint32_t pk = raw.y;
                    const int ts = pk & 31, Gp = (pk >> 5) & 31, tr = (pk >> 10) & 31;
                    const int ipos = (pk >> 16) & 31, ins = (pk >> 21) & 1, del = (pk >> 22) & 1;
                    const int cid = pk >> 23;
                    const int smerge = ins ? 63 : ipos;
                    int4 A;
                    A.x = int(raw.x) + ts;                                   // X'[tau*]
                    A.y = int(raw.x) + 3 * Gp + (ts - 1) * (Gp - 1);         // S' row tau*
                    A.z = int(raw.x) + 3 * Gp + ts;                          // S' column tau*
                    A.w = int(raw.x) + (Gp + 1) * (Gp + 1) + tr;             // T'[tau*]
                    S.dA[rl + t] = A;
                    S.dS[rl + t] = uint32_t(del) | (uint32_t(ins) << 1) | (uint32_t(ipos) << 2) |
                                   (uint32_t(ts) << 7) | (uint32_t(smerge) << 12) | (uint32_t(Gp) << 18);
                    S.crow[rl + t] = __ldg(P.coef_row + I.coef_base + cid);
                    S.ccol[rl + t] = __ldg(P.coef_col + I.coef_base + cid);
                }
            }
        }
        __syncthreads();
        // ---- phase 3: pattern threads: work order (S variables first, then
        // the rest, each in memory order) and the Z sums of Eq. HZ
        {
            const uint32_t nS = s_nS;
            for (int j = threadIdx.x; j < np; j += blockDim.x) {
                const PatHdr& h = S.hdr[j];
                const int G = h.G;
                const uint32_t a = h.var_off - v0;
                const uint32_t ej = a | (uint32_t(j) << 11);
                uint32_t* ps = S.perm + S.sb[j];
                uint32_t* po = S.perm + nS + S.ob[j];
                const int cb = int(h.cat_off - c0);
                C zs = mk(T(0), T(0));
                *po++ = ej | (uint32_t(KZ) << 19);
                for (int q = 1; q <= G; ++q) {
                    *po++ = (ej + q) | (uint32_t(KX) << 19) | (uint32_t(q) << 22);
                    zs = caxpy(S.cM[cb + q - 1], csub(S.x[a + q], S.x[a + G + q]), zs);
                }
                for (int q = 1; q <= G; ++q) *po++ = (ej + G + q) | (uint32_t(KY) << 19) | (uint32_t(q) << 22);
                for (int q = 1; q <= G; ++q) *po++ = (ej + 2 * G + q) | (uint32_t(KP) << 19) | (uint32_t(q) << 22);
                uint32_t l = ej + 3 * G + 1;
                for (int q = 1; q <= G; ++q)
                    for (int r = 1; r <= G; ++r)
                        if (r != q) *ps++ = (l++) | (uint32_t(KS) << 19) | (uint32_t(q) << 22) | (uint32_t(r) << 27);
                for (int q = 1; q <= G; ++q) {
                    const int tr = (S.cw[cb + q - 1] >> 15) & 31;
                    if (tr != 31)
                        *po++ = (ej + (G + 1) * (G + 1) + tr) | (uint32_t(KT) << 19) | (uint32_t(q) << 22);
                }
                S.Zs[j] = zs;
            }
        }
        __syncthreads();
        // ---- phase 4: one unique variable per thread
        for (uint32_t i = threadIdx.x; i < nv; i += blockDim.x) {
            const uint32_t e = S.perm[i];
            const uint32_t l = e & 2047u;
            const int j = int((e >> 11) & 255u);
            const int kind = int((e >> 19) & 7u);
            const int q = int((e >> 22) & 31u);
            const int r = int(e >> 27);
            const uint32_t vg = v0 + l;
            const PatHdr h = S.hdr[j];
            const int G = h.G;
            const int pl = int(h.var_off - v0);
            const int cb = int(h.cat_off - c0);
            const InstDev& I = P.inst[h.inst];
            if (FP64SIDE && h.tier == 0) {
                // physical representative: FP64 arithmetic and FP64 storage
                const double2* xsin = P.xs_in + I.side;
                auto own = [&](int ii) { return xsin[ii]; };
                auto gath = [&](uint32_t ii) { const C t = __ldg(P.x_in + ii); return make_double2(t.x, t.y); };
                const double2 gam = make_double2(P.gamma[p0 + j].x, P.gamma[p0 + j].y);
                const int loc = int(l) - pl;
                const double2 k = var_rhs<double>(P, kind, q, r, G, S.cw + cb, S.cM + cb,
                                                  S.rec + (h.rec_off - r0), h, I, gam, own, gath);
                const double dt = P.dt;
                const int si = int(I.side) + loc;
                if (P.stage < 0) {
                    P.xs_out[si] = k;
                    P.x_out[vg] = mk(T(k.x), T(k.y));
                } else if (P.stage == 3) {
                    const double2 ys = P.ys[si], as = P.accs[si];
                    const double2 yn = make_double2(ys.x + dt / 6.0 * (as.x + k.x), ys.y + dt / 6.0 * (as.y + k.y));
                    P.ys_out[si] = yn;
                    P.y_out[vg] = mk(T(yn.x), T(yn.y));
                } else {
                    const double2 ys = P.ys[si];
                    double2 as;
                    if (P.stage == 0) as = k;
                    else {
                        as = P.accs[si];
                        as.x += 2.0 * k.x;
                        as.y += 2.0 * k.y;
                    }
                    P.accs[si] = as;
                    const double a = P.stage == 2 ? dt : 0.5 * dt;
                    const double2 xn = make_double2(ys.x + a * k.x, ys.y + a * k.y);
                    P.xs_out[si] = xn;
                    P.x_out[vg] = mk(T(xn.x), T(xn.y));
                }
                continue;
            }
            // stream operands of the RK4 stage, issued before the derivative
            C yv, av;
            if (P.stage == 0) {
                yv = S.x[l];
            } else if (P.stage > 0) {
                yv = P.y[vg];
                av = P.acc[vg];
            }
            const T g = sizeof(T) == 8 ? T(I.g) : T(I.gf);
            const T det = sizeof(T) == 8 ? T(I.detuning) : T(I.detf);
            const T kap = sizeof(T) == 8 ? T(I.kappa) : T(I.kappaf);
            const C gam = __ldg(P.gamma + p0 + j);
            const C v = S.x[l];
            const C* xp = S.x + pl;
            // Hamiltonian, damping and loss (Eqs. HZ, HX and their Y, P, S, T
            // counterparts), with the grouped sums of phases 2 and 3
            C d;
            if (kind == KZ) {
                const C zs = S.Zs[j];
                d = mk(g * zs.y, -g * zs.x);
                d = cfma(mk(-(gam.x + kap), -gam.y), v, d);
            } else if (kind == KX || kind == KY) {
                const C Z = xp[0];
                const C t = kind == KX ? csub(Z, S.R[cb + q - 1]) : csub(S.Cs[cb + q - 1], Z);
                const T sd = kind == KX ? det : -det;
                d = mk(sd * v.y + g * t.y, -sd * v.x - g * t.x);
                d = cfma(mk(-(gam.x + T(0.5) * kap), -gam.y), v, d);
            } else {
                const C t = csub(xp[G + (kind == KS ? r : q)], xp[q]);
                d = mk(g * t.y, -g * t.x);
                d = cfma(mk(-gam.x, -gam.y), v, d);
            }
            // hierarchy terms (Eqs. uvar-up, uvar-down) from the decoded records
            // of the row category and of the column category
            const bool rowside = kind == KX || kind == KP || kind == KS || kind == KT;
            const bool colside = kind == KY || kind == KS || kind == KT;
            const int rcat = q;                       // row category (moved on the row side)
            const int ccat = kind == KS ? r : q;      // column category (moved on the column side)
            const uint32_t wr = rowside ? S.cw[cb + rcat - 1] : 0u;
            const uint32_t wc = colside ? S.cw[cb + ccat - 1] : 0u;
            const int skip = kind == KP ? int((wr >> 20) & 15) : 0;  // P_q: lower records only
            const int nr = int((wr >> 10) & 31) - skip, nc = int((wc >> 10) & 31);
            const int rb = int(h.rec_off - r0);
            const int rr0 = rb + int(wr & 1023) + skip, rc0 = rb + int(wc & 1023);
            const int colrow = q;                     // row category seen from the column side
            const int rowcol = kind == KS ? r : q;    // column category seen from the row side
            const int ntot = nr + nc;
            for (int i0 = 0; i0 < ntot; i0 += 4) {
                C val[4], cf[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int ii = i0 + u;
                    val[u] = mk(T(0), T(0));
                    cf[u] = mk(T(0), T(0));
                    if (ii < ntot) {
                        const bool isrow = ii < nr;
                        const int rx = isrow ? rr0 + ii : rc0 + ii - nr;
                        const int4 A = S.dA[rx];
                        const uint32_t sm = S.dS[rx];
                        const int Gp = int(sm >> 18) & 31;
                        int idx;
                        if (isrow) {
                            if (kind == KX) idx = A.x;
                            else if (kind == KP) idx = A.x + 2 * Gp;
                            else {
                                // S'[tau*, tau(b)] or T'[tau*], b = rowcol
                                const int smerge = int(sm >> 12) & 63;
                                const int b = rowcol;
                                idx = A.y + b - (int(sm & 1u) && b > rcat ? 1 : 0) - (b > smerge ? 1 : 0);
                                if (b == smerge) idx = A.w;
                            }
                            cf[u] = S.crow[rx];
                            if (kind == KP) cf[u] = cadd(cf[u], S.ccol[rx]);
                        } else {
                            if (kind == KY) idx = A.x + Gp;
                            else {
                                // S'[tau(a), tau*] or T'[tau*], a = colrow
                                const int a = colrow;
                                const int ts = int(sm >> 7) & 31;
                                const int ipos = int(sm >> 2) & 31;
                                const int ta = a - ((sm & 1u) && a > ccat ? 1 : 0) + (((sm >> 1) & 1u) && a >= ipos ? 1 : 0);
                                idx = (ta == ts) ? A.w : A.z + (ta - 1) * (Gp - 1) - (ts > ta ? 1 : 0);
                            }
                            cf[u] = S.ccol[rx];
                        }
                        val[u] = __ldg(P.x_in + idx);
                    }
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) d = cfma(cf[u], val[u], d);
            }
            const C k = d;
            if (P.stage < 0) {
                P.x_out[vg] = k;
            } else if (P.stage == 0) {
                P.acc[vg] = k;
                P.x_out[vg] = caxpy(aT, k, yv);
            } else if (P.stage == 3) {
                P.y_out[vg] = caxpy(dtT / T(6), cadd(av, k), yv);
            } else {
                P.acc[vg] = caxpy(T(2), k, av);
                P.x_out[vg] = caxpy(aT, k, yv);
            }
        }
        __syncthreads();
    }
}

// Observables of the physical representative of every instance
// (Eqs. trace-uvar .. Pminus-uvar) plus the Hermiticity defect of rho_S.
__global__ void observables_kernel(const InstDev* __restrict__ inst, const double* __restrict__ theta, int ninst,
                                   const double2* __restrict__ main64, const double2* __restrict__ side64,
                                   double* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ninst) return;
    const InstDev I = inst[i];
    const double2* v = side64 ? side64 + I.side : main64 + I.var_begin;
    const double2 Z = v[0], X0 = v[1], Y0 = v[2], P0 = v[3];
    const double2 T0 = I.n_rho0 > 4 ? v[4] : make_double2(0.0, 0.0);
    const double N = I.N;
    const double th = theta[i];
    const double cs = cos(th), sn = sin(th);
    const double PBr = P0.x + (N - 1.0) * T0.x;
    const double sq = sqrt(N) * sn * cs;
    double* o = out + 8 * i;
    o[0] = Z.x + N * P0.x;
    o[1] = Z.x;
    o[2] = N * P0.x;
    o[3] = PBr;
    o[4] = (N - 1.0) * (P0.x - T0.x);
    o[5] = Z.x * cs * cs + PBr * sn * sn + sq * (X0.x + Y0.x);
    o[6] = Z.x * sn * sn + PBr * cs * cs - sq * (X0.x + Y0.x);
    double hd = fabs(Z.y);
    hd = fmax(hd, fabs(P0.y));
    hd = fmax(hd, fabs(T0.y));
    hd = fmax(hd, hypot(X0.x - Y0.x, X0.y + Y0.y));
    o[7] = hd;
}

// Factorised initial state: write rho_0 of every instance (zeroing is a memset).
__global__ void init_rho0_kernel(const InstDev* __restrict__ inst, int ninst, const double* __restrict__ rho0,
                                 double2* __restrict__ main64, float2* __restrict__ main32,
                                 double2* __restrict__ side64) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ninst) return;
    const InstDev I = inst[i];
    for (uint32_t j = 0; j < I.n_rho0; ++j) {
        const double re = rho0[10 * i + 2 * j], im = rho0[10 * i + 2 * j + 1];
        if (main64) main64[I.var_begin + j] = make_double2(re, im);
        if (main32) main32[I.var_begin + j] = make_float2(float(re), float(im));
        if (side64) side64[I.side + j] = make_double2(re, im);
    }
}

// ---- host launch wrappers (called from api.cu) -----------------------------

size_t stage_smem_bytes(int chunk, int rec_cap, bool fp64) {
    const size_t cs = fp64 ? 16 : 8, ts = fp64 ? 8 : 4;
    const size_t ncat = size_t(chunk) / 4 + 8;
    size_t b = cs * (size_t(chunk) + 2 * ncat + kMaxPatPerChunk + 2 * size_t(rec_cap));
    b += (sizeof(int4) + sizeof(uint2) + sizeof(uint32_t)) * size_t(rec_cap);
    b += sizeof(PatHdr) * (kMaxPatPerChunk + 1);
    b += sizeof(uint32_t) * (ncat + size_t(chunk));
    b += ts * ncat;
    b += 2 * sizeof(uint16_t) * kMaxPatPerChunk;
    return (b + 15) / 16 * 16 + 16;
}

template <typename T, bool SIDE>
static cudaError_t launch_t(const StageParams<T>& p, const LaunchCfg& cfg, cudaStream_t st) {
    const size_t sm = stage_smem_bytes(cfg.chunk, cfg.rec_cap, sizeof(T) == 8);
    stage_kernel<T, SIDE><<<cfg.grid, cfg.block, sm, st>>>(p);
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
    p.chunk_begin = static_cast<const uint32_t*>(s.chunk_begin);
    p.inst = static_cast<const InstDev*>(s.inst);
    p.coef_row = static_cast<const C*>(s.coef_row);
    p.coef_col = static_cast<const C*>(s.coef_col);
    p.cat_Md = static_cast<const double*>(s.cat_Md);
    p.coef_row_d = static_cast<const double2*>(s.coef_row_d);
    p.coef_col_d = static_cast<const double2*>(s.coef_col_d);
    p.lut = static_cast<const uint16_t*>(s.lut);
    p.lut_off = static_cast<const uint32_t*>(s.lut_off);
    p.nchunks = s.nchunks;
    p.chunk = cfg.chunk;
    p.rec_cap = cfg.rec_cap;
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
    return p;
}

cudaError_t launch_stage(const StageLaunch& s, const LaunchCfg& cfg, bool fp64, cudaStream_t st) {
    if (fp64) return launch_t<double, false>(make_params<double>(s, cfg), cfg, st);
    return launch_t<float, true>(make_params<float>(s, cfg), cfg, st);
}

// Sets the dynamic shared-memory limit once for the largest chunk (outside
// any stream capture) and returns the CTAs per SM for this configuration.
cudaError_t stage_occupancy(const LaunchCfg& cfg, bool fp64, int* blocks_per_sm) {
    const size_t sm = stage_smem_bytes(cfg.chunk, cfg.rec_cap, fp64);
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    // leave room for the kernel's static shared variables
    const int lim = int(std::min<size_t>(stage_smem_bytes(kMaxChunkVars, kMaxChunkVars * 4, fp64),
                                         size_t(std::max(optin - 1024, 0))));
    if (sm > size_t(lim)) {
        *blocks_per_sm = 0;
        return cudaSuccess;
    }
    cudaError_t e;
    if (fp64) {
        e = cudaFuncSetAttribute(stage_kernel<double, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
        if (e != cudaSuccess) return e;
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, stage_kernel<double, false>, cfg.block, sm);
    }
    e = cudaFuncSetAttribute(stage_kernel<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, stage_kernel<float, true>, cfg.block, sm);
}

cudaError_t launch_observables(const InstDev* inst, const double* theta, int ninst, const void* main64,
                               const void* side64, double* out, cudaStream_t st) {
    observables_kernel<<<(ninst + 127) / 128, 128, 0, st>>>(inst, theta, ninst, static_cast<const double2*>(main64),
                                                            static_cast<const double2*>(side64), out);
    return cudaGetLastError();
}

cudaError_t launch_init_rho0(const InstDev* inst, int ninst, const double* rho0, void* main64, void* main32,
                             void* side64, cudaStream_t st) {
    init_rho0_kernel<<<(ninst + 127) / 128, 128, 0, st>>>(inst, ninst, rho0, static_cast<double2*>(main64),
                                                          static_cast<float2*>(main32), static_cast<double2*>(side64));
    return cudaGetLastError();
}

}  // namespace sa
