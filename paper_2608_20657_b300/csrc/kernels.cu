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
    const ChunkDesc* __restrict__ desc;    // nchunks work items
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
    int cat_cap;                            // category capacity of the staged slice
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

// ---- TMA bulk copies and mbarriers (inline PTX) ----------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// global -> shared bulk copy (16-byte aligned addresses, size a multiple of 16)
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
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

// A bulk copy must start on a 16-byte boundary and cover a multiple of 16
// bytes: copy the enclosing aligned element range and remember how many
// elements precede the first wanted one.  Tables and state buffers are
// padded so that the rounded range stays inside the allocation.
struct Span {
    const char* src;
    uint32_t bytes;
    uint32_t skip;
};
__device__ __forceinline__ Span span(const void* base, uint32_t start, uint32_t count, uint32_t esz) {
    const uint32_t per = esz >= 16 ? 1u : 16u / esz;
    const uint32_t a = start - start % per;
    const uint32_t e = (start + count + per - 1) / per * per;
    Span sp;
    sp.src = static_cast<const char*>(base) + size_t(a) * esz;
    sp.bytes = count ? (e - a) * esz : 0u;
    sp.skip = start - a;
    return sp;
}

// Shared-memory image of one work item (double-buffered staging area plus
// the per-item work arrays).
template <typename T> struct StageBuf {
    using C = typename Cx<T>::t;
    PatHdr* hdr;
    C* x;
    C* y;
    C* acc;
    uint2* rec;
    uint32_t* cw;
    T* cM;
};
template <typename T> struct StageWork {
    using C = typename Cx<T>::t;
    C* R;            // grouped row sums R_q per category
    C* Cs;           // grouped column sums C_q per category
    C* Zs;           // sum_q M_q (X_q - Y_q) per pattern
    C* crow;         // decoded record: row coefficient
    C* ccol;         // decoded record: column coefficient
    int4* dA;        // decoded record: X'-index, S'-row base, S'-column base, T'-index
    uint32_t* dS;    // decoded record: small fields
    uint32_t* perm;  // work order: l | j << 11 | kind << 19 | q << 22 | r << 27
    uint16_t* sb;
    uint16_t* ob;
};

__host__ __device__ __forceinline__ size_t al16(size_t b) { return (b + 15) / 16 * 16; }

template <typename T>
__host__ __device__ __forceinline__ size_t buf_bytes(int chunk, int rec_cap, int cat_cap) {
    const size_t cs = 2 * sizeof(T);
    return al16(sizeof(PatHdr) * (kMaxPatPerChunk + 1)) + 3 * al16(cs * (chunk + 4)) + al16(8 * (rec_cap + 4)) +
           al16(4 * (cat_cap + 8)) + al16(sizeof(T) * (cat_cap + 8));
}
template <typename T>
__host__ __device__ __forceinline__ size_t work_bytes(int chunk, int rec_cap, int cat_cap) {
    const size_t cs = 2 * sizeof(T);
    return 2 * al16(cs * cat_cap) + al16(cs * kMaxPatPerChunk) + 2 * al16(cs * rec_cap) + al16(16 * rec_cap) +
           al16(4 * rec_cap) + al16(4 * chunk) + 2 * al16(2 * kMaxPatPerChunk);
}

template <typename T>
__device__ __forceinline__ StageBuf<T> carve_buf(unsigned char* p, int chunk, int rec_cap, int cat_cap) {
    using C = typename Cx<T>::t;
    StageBuf<T> B;
    B.hdr = reinterpret_cast<PatHdr*>(p); p += al16(sizeof(PatHdr) * (kMaxPatPerChunk + 1));
    B.x = reinterpret_cast<C*>(p);        p += al16(sizeof(C) * (chunk + 4));
    B.y = reinterpret_cast<C*>(p);        p += al16(sizeof(C) * (chunk + 4));
    B.acc = reinterpret_cast<C*>(p);      p += al16(sizeof(C) * (chunk + 4));
    B.rec = reinterpret_cast<uint2*>(p);  p += al16(8 * (rec_cap + 4));
    B.cw = reinterpret_cast<uint32_t*>(p); p += al16(4 * (cat_cap + 8));
    B.cM = reinterpret_cast<T*>(p);
    return B;
}
template <typename T>
__device__ __forceinline__ StageWork<T> carve_work(unsigned char* p, int chunk, int rec_cap, int cat_cap) {
    using C = typename Cx<T>::t;
    StageWork<T> W;
    W.R = reinterpret_cast<C*>(p);       p += al16(sizeof(C) * cat_cap);
    W.Cs = reinterpret_cast<C*>(p);      p += al16(sizeof(C) * cat_cap);
    W.Zs = reinterpret_cast<C*>(p);      p += al16(sizeof(C) * kMaxPatPerChunk);
    W.crow = reinterpret_cast<C*>(p);    p += al16(sizeof(C) * rec_cap);
    W.ccol = reinterpret_cast<C*>(p);    p += al16(sizeof(C) * rec_cap);
    W.dA = reinterpret_cast<int4*>(p);   p += al16(16 * rec_cap);
    W.dS = reinterpret_cast<uint32_t*>(p); p += al16(4 * rec_cap);
    W.perm = reinterpret_cast<uint32_t*>(p); p += al16(4 * chunk);
    W.sb = reinterpret_cast<uint16_t*>(p); p += al16(2 * kMaxPatPerChunk);
    W.ob = reinterpret_cast<uint16_t*>(p);
    return W;
}

// element offsets of the staged slices inside a buffer (the "skip" of each span)
struct Skips {
    uint32_t x, y, acc, rec, cw, cM;
};

// Issue the bulk copies of work item d into buffer B (one thread).
template <typename T>
__device__ __forceinline__ Skips issue_item(const StageParams<T>& P, const ChunkDesc& d, const StageBuf<T>& B,
                                            uint64_t* bar) {
    using C = typename Cx<T>::t;
    const uint32_t cs = sizeof(C);
    const Span sh = span(P.hdr, d.p0, d.np + 1, sizeof(PatHdr));
    const Span sx = span(P.x_in, d.v0, d.nv, cs);
    const bool want_y = P.stage > 0, want_acc = P.stage > 0;
    const Span sy = span(P.y, d.v0, want_y ? d.nv : 0u, cs);
    const Span sa = span(P.acc, d.v0, want_acc ? d.nv : 0u, cs);
    const Span sr = span(P.rec, d.r0, d.nrec, 8);
    const Span sw = span(P.cat_word, d.c0, d.ncat, 4);
    const Span sm = span(P.cat_M, d.c0, d.ncat, sizeof(T));
    mbar_expect_tx(bar, sh.bytes + sx.bytes + sy.bytes + sa.bytes + sr.bytes + sw.bytes + sm.bytes);
    bulk_g2s(B.hdr, sh.src, sh.bytes, bar);
    if (sx.bytes) bulk_g2s(B.x, sx.src, sx.bytes, bar);
    if (sy.bytes) bulk_g2s(B.y, sy.src, sy.bytes, bar);
    if (sa.bytes) bulk_g2s(B.acc, sa.src, sa.bytes, bar);
    if (sr.bytes) bulk_g2s(B.rec, sr.src, sr.bytes, bar);
    if (sw.bytes) bulk_g2s(B.cw, sw.src, sw.bytes, bar);
    if (sm.bytes) bulk_g2s(B.cM, sm.src, sm.bytes, bar);
    return Skips{sx.skip, sy.skip, sa.skip, sr.skip, sw.skip, sm.skip};
}

template <typename T, bool FP64SIDE>
__global__ void __launch_bounds__(256) stage_kernel(StageParams<T> P) {
    using C = typename Cx<T>::t;
    extern __shared__ __align__(16) unsigned char smem[];
    const size_t bb = buf_bytes<T>(P.chunk, P.rec_cap, P.cat_cap);
    auto buf = [&](int which) { return carve_buf<T>(smem + (which ? bb : 0), P.chunk, P.rec_cap, P.cat_cap); };
    const StageWork<T> W = carve_work<T>(smem + 2 * bb, P.chunk, P.rec_cap, P.cat_cap);
    __shared__ __align__(8) uint64_t s_bar[2];
    __shared__ ChunkDesc s_desc[2];
    __shared__ Skips s_skip[2];
    __shared__ unsigned int s_item[2], s_nS;

    const int tid = threadIdx.x;
    const int producer = blockDim.x - 32;  // lane 0 of the last warp issues the copies
    unsigned int iter = 0;
    auto next_item = [&]() -> unsigned int {
        if (P.use_queue) return atomicAdd(P.queue, 1u);
        return blockIdx.x + (iter++) * gridDim.x;
    };
    if (tid == producer) {
        mbar_init(&s_bar[0], 1);
        mbar_init(&s_bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        const unsigned int c = next_item();
        s_item[0] = c;
        if (c < P.nchunks) {
            const ChunkDesc d = P.desc[c];
            s_desc[0] = d;
            s_skip[0] = issue_item(P, d, buf(0), &s_bar[0]);
        }
    }
    __syncthreads();

    const T dtT = T(P.dt);
    const T aT = P.stage == 2 ? dtT : T(0.5) * dtT;
    uint32_t parity0 = 0, parity1 = 0;
    int b = 0;
    for (;;) {
        const unsigned int c = s_item[b];
        if (c >= P.nchunks) break;
        // prefetch the next work item into the other buffer
        if (tid == producer) {
            const unsigned int c2 = next_item();
            s_item[b ^ 1] = c2;
            if (c2 < P.nchunks) {
                const ChunkDesc d2 = P.desc[c2];
                s_desc[b ^ 1] = d2;
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                s_skip[b ^ 1] = issue_item(P, d2, buf(b ^ 1), &s_bar[b ^ 1]);
            }
        }
        const uint32_t par = b ? parity1 : parity0;
        if (!mbar_wait(&s_bar[b], par)) {
            // report, let a prefetch already in flight land (bounded), leave
            atomicOr(P.err, 1u);
            if (s_item[b ^ 1] < P.nchunks) mbar_wait(&s_bar[b ^ 1], b ? parity0 : parity1);
            return;
        }
        if (b) parity1 ^= 1u;
        else parity0 ^= 1u;

        const StageBuf<T> B = buf(b);
        const ChunkDesc d = s_desc[b];
        const Skips sk = s_skip[b];
        const int np = int(d.np);
        const uint32_t v0 = d.v0, nv = d.nv, c0 = d.c0, ncat = d.ncat, r0 = d.r0;
        const PatHdr* hdr = B.hdr;
        const C* xs = B.x + sk.x;
        const uint2* recs = B.rec + sk.rec;
        const uint32_t* cwa = B.cw + sk.cw;
        const T* cMa = B.cM + sk.cM;
        // ---- phase 2: warp 0 scans the work-order counts; the other threads
        // take the categories: grouped sums R_q, C_q (Eqs. grouped-row-sum,
        // grouped-column-sum) and the decoding of the category's records
        if (tid < 32) {
            const int lane = tid;
            const int per = (np + 31) / 32;
            const int a = lane * per, e = min(np, a + per);
            int ss = 0, so = 0;
            for (int j = a; j < e; ++j) {
                const int G = hdr[j].G;
                const int u = int(hdr[j + 1].var_off - hdr[j].var_off);
                ss += G * (G - 1);
                so += u - G * (G - 1);
            }
            int is = ss, io = so;
            for (int off = 1; off < 32; off <<= 1) {
                const int t1 = __shfl_up_sync(0xffffffffu, is, off);
                const int t2 = __shfl_up_sync(0xffffffffu, io, off);
                if (lane >= off) {
                    is += t1;
                    io += t2;
                }
            }
            int bs = is - ss, bo = io - so;
            for (int j = a; j < e; ++j) {
                const int G = hdr[j].G;
                const int u = int(hdr[j + 1].var_off - hdr[j].var_off);
                W.sb[j] = uint16_t(bs);
                W.ob[j] = uint16_t(bo);
                bs += G * (G - 1);
                bo += u - G * (G - 1);
            }
            if (lane == 31) s_nS = uint32_t(is);
        } else {
            for (uint32_t cl = tid - 32; cl < ncat; cl += blockDim.x - 32) {
                int lo = 0, hi = np - 1;  // owning pattern: last j with cat_off <= c0 + cl
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (hdr[mid].cat_off - c0 <= cl) lo = mid;
                    else hi = mid - 1;
                }
                const PatHdr h = hdr[lo];
                const int G = h.G;
                const int cb = int(h.cat_off - c0);
                const int q = int(cl) - cb + 1;
                const C* xp = xs + (h.var_off - v0);
                const uint32_t w = cwa[cl];
                const T Mq = cMa[cl];
                C Rs = xp[2 * G + q];
                if (Mq >= T(2)) Rs = caxpy(Mq - T(1), xp[(G + 1) * (G + 1) + ((w >> 15) & 31)], Rs);
                C Cq = Rs;
                for (int e2 = 1; e2 <= G; ++e2) {
                    if (e2 == q) continue;
                    const T Mb = cMa[cb + e2 - 1];
                    Rs = caxpy(Mb, xp[loc_S_d(G, q, e2)], Rs);
                    Cq = caxpy(Mb, xp[loc_S_d(G, e2, q)], Cq);
                }
                W.R[cl] = Rs;
                W.Cs[cl] = Cq;
                const InstDev& I = P.inst[h.inst];
                const int nr = (w >> 10) & 31;
                const int rl = int(h.rec_off - r0) + int(w & 1023);
                for (int t = 0; t < nr; ++t) {
                    const uint2 raw = recs[rl + t];
                    const uint32_t pk = raw.y;
                    const int ts = pk & 31, Gp = (pk >> 5) & 31, tr = (pk >> 10) & 31;
                    const int ipos = (pk >> 16) & 31, ins = (pk >> 21) & 1, del = (pk >> 22) & 1;
                    const int cid = pk >> 23;
                    const int smerge = ins ? 63 : ipos;
                    int4 A;
                    A.x = int(raw.x) + ts;                            // X'[tau*]
                    A.y = int(raw.x) + 3 * Gp + (ts - 1) * (Gp - 1);  // S' row tau*
                    A.z = int(raw.x) + 3 * Gp + ts;                   // S' column tau*
                    A.w = int(raw.x) + (Gp + 1) * (Gp + 1) + tr;      // T'[tau*]
                    W.dA[rl + t] = A;
                    W.dS[rl + t] = uint32_t(del) | (uint32_t(ins) << 1) | (uint32_t(ipos) << 2) | (uint32_t(ts) << 7) |
                                   (uint32_t(smerge) << 12) | (uint32_t(Gp) << 18);
                    W.crow[rl + t] = __ldg(P.coef_row + I.coef_base + cid);
                    W.ccol[rl + t] = __ldg(P.coef_col + I.coef_base + cid);
                }
            }
        }
        __syncthreads();
        // ---- phase 3: pattern threads: work order (S variables first, then
        // the rest, each in memory order) and the Z sums of Eq. HZ
        {
            const uint32_t nS = s_nS;
            for (int j = tid; j < np; j += blockDim.x) {
                const PatHdr h = hdr[j];
                const int G = h.G;
                const uint32_t a = h.var_off - v0;
                const uint32_t ej = a | (uint32_t(j) << 11);
                uint32_t* ps = W.perm + W.sb[j];
                uint32_t* po = W.perm + nS + W.ob[j];
                const int cb = int(h.cat_off - c0);
                C zs = mk(T(0), T(0));
                *po++ = ej | (uint32_t(KZ) << 19);
                for (int q = 1; q <= G; ++q) {
                    *po++ = (ej + q) | (uint32_t(KX) << 19) | (uint32_t(q) << 22);
                    zs = caxpy(cMa[cb + q - 1], csub(xs[a + q], xs[a + G + q]), zs);
                }
                for (int q = 1; q <= G; ++q) *po++ = (ej + G + q) | (uint32_t(KY) << 19) | (uint32_t(q) << 22);
                for (int q = 1; q <= G; ++q) *po++ = (ej + 2 * G + q) | (uint32_t(KP) << 19) | (uint32_t(q) << 22);
                uint32_t l = ej + 3 * G + 1;
                for (int q = 1; q <= G; ++q)
                    for (int r = 1; r <= G; ++r)
                        if (r != q) *ps++ = (l++) | (uint32_t(KS) << 19) | (uint32_t(q) << 22) | (uint32_t(r) << 27);
                for (int q = 1; q <= G; ++q) {
                    const int tr = (cwa[cb + q - 1] >> 15) & 31;
                    if (tr != 31)
                        *po++ = (ej + (G + 1) * (G + 1) + tr) | (uint32_t(KT) << 19) | (uint32_t(q) << 22);
                }
                W.Zs[j] = zs;
            }
        }
        __syncthreads();
        // ---- phase 4: one unique variable per thread
        const C* ys = B.y + sk.y;
        const C* as = B.acc + sk.acc;
        for (uint32_t i = tid; i < nv; i += blockDim.x) {
            const uint32_t e = W.perm[i];
            const uint32_t l = e & 2047u;
            const int j = int((e >> 11) & 255u);
            const int kind = int((e >> 19) & 7u);
            const int q = int((e >> 22) & 31u);
            const int r = int(e >> 27);
            const uint32_t vg = v0 + l;
            const PatHdr h = hdr[j];
            const int G = h.G;
            const int pl = int(h.var_off - v0);
            const int cb = int(h.cat_off - c0);
            const InstDev& I = P.inst[h.inst];
            if (FP64SIDE && h.tier == 0) {
                // physical representative: FP64 arithmetic and FP64 storage
                const double2* xsin = P.xs_in + I.side;
                auto own = [&](int ii) { return xsin[ii]; };
                auto gath = [&](uint32_t ii) { const C t = __ldg(P.x_in + ii); return make_double2(t.x, t.y); };
                const double2 gam = make_double2(P.gamma[d.p0 + j].x, P.gamma[d.p0 + j].y);
                const int loc = int(l) - pl;
                const double2 k = var_rhs<double>(P, kind, q, r, G, cwa + cb, cMa + cb, recs + (h.rec_off - r0), h, I,
                                                  gam, own, gath);
                const double dt = P.dt;
                const int si = int(I.side) + loc;
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
                continue;
            }
            const T g = sizeof(T) == 8 ? T(I.g) : T(I.gf);
            const T det = sizeof(T) == 8 ? T(I.detuning) : T(I.detf);
            const T kap = sizeof(T) == 8 ? T(I.kappa) : T(I.kappaf);
            const C gam = __ldg(P.gamma + d.p0 + j);
            const C v = xs[l];
            const C* xp = xs + pl;
            // Hamiltonian, damping and loss (Eqs. HZ, HX and their Y, P, S, T
            // counterparts), with the grouped sums of phases 2 and 3
            C dv;
            if (kind == KZ) {
                const C zs = W.Zs[j];
                dv = mk(g * zs.y, -g * zs.x);
                dv = cfma(mk(-(gam.x + kap), -gam.y), v, dv);
            } else if (kind == KX || kind == KY) {
                const C Z = xp[0];
                const C t = kind == KX ? csub(Z, W.R[cb + q - 1]) : csub(W.Cs[cb + q - 1], Z);
                const T sd = kind == KX ? det : -det;
                dv = mk(sd * v.y + g * t.y, -sd * v.x - g * t.x);
                dv = cfma(mk(-(gam.x + T(0.5) * kap), -gam.y), v, dv);
            } else {
                const C t = csub(xp[G + (kind == KS ? r : q)], xp[q]);
                dv = mk(g * t.y, -g * t.x);
                dv = cfma(mk(-gam.x, -gam.y), v, dv);
            }
            // hierarchy terms (Eqs. uvar-up, uvar-down) from the decoded records
            // of the row category and of the column category
            const bool rowside = kind == KX || kind == KP || kind == KS || kind == KT;
            const bool colside = kind == KY || kind == KS || kind == KT;
            const int rcat = q;                     // row category (moved on the row side)
            const int ccat = kind == KS ? r : q;    // column category (moved on the column side)
            const uint32_t wr = rowside ? cwa[cb + rcat - 1] : 0u;
            const uint32_t wc = colside ? cwa[cb + ccat - 1] : 0u;
            const int skip = kind == KP ? int((wr >> 20) & 15) : 0;  // P_q: lower records only
            const int nr = int((wr >> 10) & 31) - skip, nc = int((wc >> 10) & 31);
            const int rb = int(h.rec_off - r0);
            const int rr0 = rb + int(wr & 1023) + skip, rc0 = rb + int(wc & 1023);
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
                        const int4 A = W.dA[rx];
                        const uint32_t sm = W.dS[rx];
                        const int Gp = int(sm >> 18) & 31;
                        int idx;
                        if (isrow) {
                            if (kind == KX) idx = A.x;
                            else if (kind == KP) idx = A.x + 2 * Gp;
                            else {
                                // S'[tau*, tau(c)] or T'[tau*]; c = r (S) or q (T)
                                const int smerge = int(sm >> 12) & 63;
                                const int cc = kind == KS ? r : q;
                                idx = A.y + cc - ((sm & 1u) && cc > rcat ? 1 : 0) - (cc > smerge ? 1 : 0);
                                if (cc == smerge) idx = A.w;
                            }
                            cf[u] = W.crow[rx];
                            if (kind == KP) cf[u] = cadd(cf[u], W.ccol[rx]);
                        } else {
                            if (kind == KY) idx = A.x + Gp;
                            else {
                                // S'[tau(q), tau*] or T'[tau*]
                                const int ts = int(sm >> 7) & 31;
                                const int ipos = int(sm >> 2) & 31;
                                const int ta = q - ((sm & 1u) && q > ccat ? 1 : 0) +
                                               (((sm >> 1) & 1u) && q >= ipos ? 1 : 0);
                                idx = (ta == ts) ? A.w : A.z + (ta - 1) * (Gp - 1) - (ts > ta ? 1 : 0);
                            }
                            cf[u] = W.ccol[rx];
                        }
                        val[u] = __ldg(P.x_in + idx);
                    }
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) dv = cfma(cf[u], val[u], dv);
            }
            if (P.stage < 0) {
                P.x_out[vg] = dv;
            } else if (P.stage == 0) {
                P.acc[vg] = dv;
                P.x_out[vg] = caxpy(aT, dv, v);  // x_in is y in the first stage
            } else if (P.stage == 3) {
                P.y_out[vg] = caxpy(dtT / T(6), cadd(as[l], dv), ys[l]);
            } else {
                P.acc[vg] = caxpy(T(2), dv, as[l]);
                P.x_out[vg] = caxpy(aT, dv, ys[l]);
            }
        }
        __syncthreads();
        b ^= 1;
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

size_t stage_smem_bytes(int chunk, int rec_cap, int cat_cap, bool fp64) {
    if (fp64) return 2 * buf_bytes<double>(chunk, rec_cap, cat_cap) + work_bytes<double>(chunk, rec_cap, cat_cap);
    return 2 * buf_bytes<float>(chunk, rec_cap, cat_cap) + work_bytes<float>(chunk, rec_cap, cat_cap);
}

template <typename T, bool SIDE>
static cudaError_t launch_t(const StageParams<T>& p, const LaunchCfg& cfg, cudaStream_t st) {
    const size_t sm = stage_smem_bytes(cfg.chunk, cfg.rec_cap, cfg.cat_cap, sizeof(T) == 8);
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
    p.desc = static_cast<const ChunkDesc*>(s.desc);
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
    p.cat_cap = cfg.cat_cap;
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
    return p;
}

cudaError_t launch_stage(const StageLaunch& s, const LaunchCfg& cfg, bool fp64, cudaStream_t st) {
    if (fp64) return launch_t<double, false>(make_params<double>(s, cfg), cfg, st);
    return launch_t<float, true>(make_params<float>(s, cfg), cfg, st);
}

// Sets the dynamic shared-memory limit once for the largest chunk (outside
// any stream capture) and returns the CTAs per SM for this configuration.
cudaError_t stage_occupancy(const LaunchCfg& cfg, bool fp64, int* blocks_per_sm) {
    const size_t sm = stage_smem_bytes(cfg.chunk, cfg.rec_cap, cfg.cat_cap, fp64);
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    // leave room for the kernel's static shared variables
    const int lim = std::max(optin - 1024, 0);
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
