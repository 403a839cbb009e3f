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
                                                     const uint32_t* s_cw, const T* s_cM, const PatHdr& h,
                                                     const InstDev& I, typename Cx<A>::t gam, Own own,
                                                     Gath gath) {
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
    // hierarchy terms
    const int row = (kind == KX || kind == KP || kind == KS || kind == KT) ? q : 0;
    const int col = (kind == KY) ? q : (kind == KS ? r : ((kind == KP || kind == KT) ? q : 0));
    const bool same = kind == KP;
    const Record* R = P.rec + h.rec_off;
    auto crow = [&](int cid) -> CA {
        if constexpr (kMixed) return P.coef_row_d[I.coef_base + cid];
        else return to_acc(P.coef_row[I.coef_base + cid], (CA*)nullptr);
    };
    auto ccol = [&](int cid) -> CA {
        if constexpr (kMixed) return P.coef_col_d[I.coef_base + cid];
        else return to_acc(P.coef_col[I.coef_base + cid], (CA*)nullptr);
    };
    if (row) {
        const uint32_t w = s_cw[row - 1];
        const int rs = w & 1023, nr = (w >> 10) & 31;
        for (int j = 0; j < nr; ++j) {
            const uint2 rc = __ldg(reinterpret_cast<const uint2*>(R + rs + j));
            const uint32_t pk = rc.y;
            const int cid = pk >> 23;
            if (same && (cid & 1)) continue;  // the two raise terms of P_q cancel
            const int ts = pk & 31, Gp = (pk >> 5) & 31;
            int tl;
            if (kind == KX) tl = ts;
            else if (same) tl = 2 * Gp + ts;
            else {
                const int cc = tau_d(pk, row, col);
                tl = (cc == ts) ? (Gp + 1) * (Gp + 1) + ((pk >> 10) & 31) : loc_S_d(Gp, ts, cc);
            }
            CA cf = crow(cid);
            if (same) cf = cadd(cf, ccol(cid));
            d = cfma(cf, gath(rc.x + tl), d);
        }
    }
    if (col && !same) {
        const uint32_t w = s_cw[col - 1];
        const int rs = w & 1023, nr = (w >> 10) & 31;
        for (int j = 0; j < nr; ++j) {
            const uint2 rc = __ldg(reinterpret_cast<const uint2*>(R + rs + j));
            const uint32_t pk = rc.y;
            const int cid = pk >> 23;
            const int ts = pk & 31, Gp = (pk >> 5) & 31;
            int tl;
            if (kind == KY) tl = Gp + ts;
            else {
                const int rr = tau_d(pk, col, row);
                tl = (rr == ts) ? (Gp + 1) * (Gp + 1) + ((pk >> 10) & 31) : loc_S_d(Gp, rr, ts);
            }
            d = cfma(ccol(cid), gath(rc.x + tl), d);
        }
    }
    return d;
}

template <typename T, bool FP64SIDE>
__global__ void __launch_bounds__(256) stage_kernel(StageParams<T> P) {
    using C = typename Cx<T>::t;
    extern __shared__ __align__(16) unsigned char smem[];
    // shared layout: x slice | headers | category words | multiplicities | local pattern ids
    C* s_x = reinterpret_cast<C*>(smem);
    PatHdr* s_hdr = reinterpret_cast<PatHdr*>(s_x + P.chunk);
    uint32_t* s_cw = reinterpret_cast<uint32_t*>(s_hdr + kMaxPatPerChunk + 1);
    T* s_cM = reinterpret_cast<T*>(s_cw + P.chunk / 4 + 8);
    uint8_t* s_lp = reinterpret_cast<uint8_t*>(s_cM + P.chunk / 4 + 8);
    __shared__ unsigned int s_c;

    const T dtT = T(P.dt);
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
        for (int j = threadIdx.x; j <= np; j += blockDim.x) s_hdr[j] = P.hdr[p0 + j];
        __syncthreads();
        const uint32_t v0 = s_hdr[0].var_off, nv = s_hdr[np].var_off - v0;
        const uint32_t c0 = s_hdr[0].cat_off, ncat = s_hdr[np].cat_off - c0;
        for (uint32_t l = threadIdx.x; l < nv; l += blockDim.x) s_x[l] = P.x_in[v0 + l];
        for (uint32_t l = threadIdx.x; l < ncat; l += blockDim.x) {
            s_cw[l] = __ldg(P.cat_word + c0 + l);
            s_cM[l] = __ldg(P.cat_M + c0 + l);
        }
        for (int j = threadIdx.x; j < np; j += blockDim.x) {
            const uint32_t a = s_hdr[j].var_off - v0, b = s_hdr[j + 1].var_off - v0;
            for (uint32_t l = a; l < b; ++l) s_lp[l] = uint8_t(j);
        }
        __syncthreads();
        for (uint32_t l = threadIdx.x; l < nv; l += blockDim.x) {
            const int j = s_lp[l];
            const PatHdr h = s_hdr[j];
            const int G = h.G;
            const int pl = int(h.var_off - v0);
            const int loc = int(l) - pl;
            int kind, q, r = 0;
            if (loc < (G + 1) * (G + 1)) {
                const uint32_t code = __ldg(P.lut + __ldg(P.lut_off + G) + loc);
                kind = code & 7;
                q = (code >> 3) & 31;
                r = (code >> 8) & 31;
            } else {
                kind = KT;
                const int t = loc - (G + 1) * (G + 1);
                q = 1;
                for (int a = 1; a <= G; ++a)
                    if (((s_cw[h.cat_off - c0 + a - 1] >> 15) & 31) == uint32_t(t)) q = a;
            }
            const InstDev& I = P.inst[h.inst];
            const uint32_t* cw = s_cw + (h.cat_off - c0);
            const T* cM = s_cM + (h.cat_off - c0);
            const uint32_t vg = v0 + l;
            if (FP64SIDE && h.tier == 0) {
                // physical representative: FP64 arithmetic and FP64 storage
                const double2* xsin = P.xs_in + I.side;
                auto own = [&](int i) { return xsin[i]; };
                auto gath = [&](uint32_t i) { const C t = P.x_in[i]; return make_double2(t.x, t.y); };
                const double2 gam = make_double2(P.gamma[p0 + j].x, P.gamma[p0 + j].y);
                const double2 k = var_rhs<double>(P, kind, q, r, G, cw, cM, h, I, gam, own, gath);
                const double dt = P.dt;
                const int si = int(I.side) + loc;
                if (P.stage < 0) {
                    P.xs_out[si] = k;
                    P.x_out[vg] = mk(T(k.x), T(k.y));
                } else if (P.stage == 3) {
                    const double2 yv = P.ys[si], av = P.accs[si];
                    const double2 yn = make_double2(yv.x + dt / 6.0 * (av.x + k.x), yv.y + dt / 6.0 * (av.y + k.y));
                    P.ys_out[si] = yn;
                    P.y_out[vg] = mk(T(yn.x), T(yn.y));
                } else {
                    const double2 yv = P.ys[si];
                    double2 av;
                    if (P.stage == 0) av = k;
                    else {
                        av = P.accs[si];
                        av.x += 2.0 * k.x;
                        av.y += 2.0 * k.y;
                    }
                    P.accs[si] = av;
                    const double a = P.stage == 2 ? dt : 0.5 * dt;
                    const double2 xn = make_double2(yv.x + a * k.x, yv.y + a * k.y);
                    P.xs_out[si] = xn;
                    P.x_out[vg] = mk(T(xn.x), T(xn.y));
                }
                continue;
            }
            auto own = [&](int i) { return s_x[pl + i]; };
            auto gath = [&](uint32_t i) { return P.x_in[i]; };
            const C k = var_rhs<T>(P, kind, q, r, G, cw, cM, h, I, __ldg(P.gamma + p0 + j), own, gath);
            if (P.stage < 0) {
                P.x_out[vg] = k;
            } else if (P.stage == 0) {
                // x_in is y in the first stage
                const C yv = s_x[l];
                P.acc[vg] = k;
                P.x_out[vg] = caxpy(T(0.5) * dtT, k, yv);
            } else if (P.stage == 3) {
                const C yv = P.y[vg], av = P.acc[vg];
                P.y_out[vg] = caxpy(dtT / T(6), cadd(av, k), yv);
            } else {
                const C yv = P.y[vg];
                const C av = P.acc[vg];
                P.acc[vg] = caxpy(T(2), k, av);
                P.x_out[vg] = caxpy(P.stage == 2 ? dtT : T(0.5) * dtT, k, yv);
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

size_t stage_smem_bytes(int chunk, bool fp64) {
    const size_t cs = fp64 ? 16 : 8, ts = fp64 ? 8 : 4;
    size_t b = size_t(chunk) * cs;
    b += sizeof(PatHdr) * (kMaxPatPerChunk + 1);
    b += sizeof(uint32_t) * (chunk / 4 + 8);
    b += ts * (chunk / 4 + 8);
    b += size_t(chunk);
    return (b + 15) / 16 * 16;
}

template <typename T, bool SIDE>
static cudaError_t launch_t(const StageParams<T>& p, const LaunchCfg& cfg, cudaStream_t st) {
    const size_t sm = stage_smem_bytes(cfg.chunk, sizeof(T) == 8);
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
    const size_t sm = stage_smem_bytes(cfg.chunk, fp64);
    const int lim = int(stage_smem_bytes(kMaxChunkVars, fp64));
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
