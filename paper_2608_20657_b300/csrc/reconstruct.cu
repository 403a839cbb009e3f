// reconstruct.cu -- rho_S(t) of an arbitrary initial operator from the five
// representative propagations (Sec. IV, general initial density operators;
// Table tab:representative-initial-operators).
//
// The reduced map is linear (Eq. Gt-linearity) and commutes with molecular
// relabelling (Eq. Gt-covariance), so with A = rho_S(0) (basis {c, e_1..e_N},
// row-major, n = N + 1)
//     rho_S(t) = A_cc G[|c><c|] + sum_i A_ic G[|e_i><c|] + sum_i A_ci G[|c><e_i|]
//              + sum_i A_ii G[|e_i><e_i|] + sum_{i != j} A_ij G[|e_i><e_j|],
// and every G[.] is a relabelled response of a representative.  A response
// is constant on the classes of its distinguished molecules, so each output
// entry needs only A_ab, A_ba and O(1) aggregates of A:
//     u_i = A_ic, v_i = A_ci, p_i = A_ii (and their totals U, V, P),
//     r_i = sum_{j != i} A_ij, s_j = sum_{i != j} A_ij over the molecular
//     block (and its total O).
// E.g. the |e_i><e_j| responses give entry (a, b), a != b molecules,
//     A_ab S12 + A_ba S21 + (r_a - A_ab) S13 + (s_a - A_ba) S23
//     + (r_b - A_ba) S31 + (s_b - A_ab) S32 + (O - r_a - s_a - r_b - s_b + A_ab + A_ba) T
// with S_qr, T the d = 2 response's variables (category 3 = the others).
//
// For molecules a != b the entry separates as
//     rho_ab(t) = alpha_a + beta_b + c1 A_ab + c2 A_ba
// (alpha_a from a's aggregates and the constant terms, beta_b from b's), so
// the bulk of the output costs two complex FMAs per entry: on B300, whose
// FP64 rate is about 2 operations per clock per SM, a general form of ~100
// FP64 operations per entry would bound the kernel by the FP64 pipe, not by
// HBM.
//
// Kernels (FP64): a tile pass of row / column partial sums (a butterfly
// reduce-scatter gives each lane one row's sum, about one add per element and
// component), two small passes finishing the per-index vectors and the four
// totals (fixed summation order: the result is bitwise repeatable), a
// per-index pass for alpha, beta and the cavity row, cavity column and
// diagonal (general form), and the bulk pass, one CTA per symmetric pair of
// 32 x 32 tiles so that A is read once there and rho_S(t) written once.
#include "sa_internal.h"

namespace sa {

namespace {

__device__ __forceinline__ double2 d2(double a, double b) { return make_double2(a, b); }
__device__ __forceinline__ double2 add(double2 a, double2 b) { return d2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 sub(double2 a, double2 b) { return d2(a.x - b.x, a.y - b.y); }
// acc + a * b (complex)
__device__ __forceinline__ double2 fma2(double2 a, double2 b, double2 acc) {
    acc.x = fma(a.x, b.x, fma(-a.y, b.y, acc.x));
    acc.y = fma(a.x, b.y, fma(a.y, b.x, acc.y));
    return acc;
}

constexpr int kRB = 128;  // partial-sum tile: rows
constexpr int kCB = 256;  // partial-sum tile: columns (one per thread)
constexpr int kT = 32;    // output tile

// response value of representative r, slot k (zero where the
// representative or the variable does not exist)
__global__ void gather_responses_kernel(const InstDev* __restrict__ inst, const RepSrc* __restrict__ src,
                                        const double2* __restrict__ main64, const double2* __restrict__ side64,
                                        double2* __restrict__ resp) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= kReps * kRepSlots) return;
    const RepSrc S = src[t];
    double2 v = d2(0.0, 0.0);
    if (S.loc >= 0) {
        const InstDev I = inst[S.inst];
        v = side64 ? side64[I.side + S.loc] : main64[I.dev_base + size_t(S.loc) * I.dev_stride];
        if (S.conj) v.y = -v.y;
    }
    resp[t] = v;
}

// per tile (kRB rows x kCB columns): row partial sums rowpart[tile col][row]
// and column partial sums colpart[tile row][col] of the molecular block
// without its diagonal.  Each warp owns 32 columns and takes 32 rows at a
// time: every lane sums its column, then a butterfly reduce-scatter leaves
// in lane l the sum of row l over the warp's columns.
__global__ void __launch_bounds__(kCB) recon_partials_kernel(const double2* __restrict__ A, int64_t n,
                                                             double2* __restrict__ rowpart,
                                                             double2* __restrict__ colpart) {
    __shared__ double2 red[kRB][kCB / 32];
    const int64_t j = int64_t(blockIdx.x) * kCB + threadIdx.x;
    const int64_t i0 = int64_t(blockIdx.y) * kRB;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double2 cs = d2(0.0, 0.0);
    for (int c = 0; c < kRB / 32; ++c) {
        double2 v[32];
#pragma unroll
        for (int k = 0; k < 32; ++k) {
            const int64_t i = i0 + c * 32 + k;
            v[k] = (i < n && j < n && i >= 1 && j >= 1 && i != j) ? __ldg(A + i * n + j) : d2(0.0, 0.0);
        }
#pragma unroll
        for (int k = 0; k < 32; ++k) cs = add(cs, v[k]);
        // reduce-scatter: at width w a lane keeps the upper half of its rows
        // when bit w of its lane index is set, and adds its partner's copy
#pragma unroll
        for (int w = 16; w >= 1; w >>= 1) {
            const bool up = (lane & w) != 0;
#pragma unroll
            for (int k = 0; k < w; ++k) {
                const double2 send = up ? v[k] : v[k + w];
                const double2 keep = up ? v[k + w] : v[k];
                const double rx = __shfl_xor_sync(0xffffffffu, send.x, w);
                const double ry = __shfl_xor_sync(0xffffffffu, send.y, w);
                v[k] = d2(keep.x + rx, keep.y + ry);
            }
        }
        red[c * 32 + lane][warp] = v[0];
    }
    __syncthreads();
    if (threadIdx.x < kRB) {
        const int k = threadIdx.x;
        double2 s = d2(0.0, 0.0);
#pragma unroll
        for (int w = 0; w < kCB / 32; ++w) s = add(s, red[k][w]);
        const int64_t i = i0 + k;
        if (i < n) rowpart[int64_t(blockIdx.x) * n + i] = s;
    }
    if (j < n) colpart[int64_t(blockIdx.y) * n + j] = cs;
}

// r_i, s_i from the partials; per-block totals of u, v, p, r over molecules
__global__ void __launch_bounds__(256) recon_vectors_kernel(const double2* __restrict__ A, int64_t n,
                                                            const double2* __restrict__ rowpart, int ncb,
                                                            const double2* __restrict__ colpart, int nrb,
                                                            double2* __restrict__ r, double2* __restrict__ s,
                                                            double2* __restrict__ blocktot) {
    __shared__ double2 red[4][256];
    const int64_t i = int64_t(blockIdx.x) * 256 + threadIdx.x;
    double2 ri = d2(0.0, 0.0), si = d2(0.0, 0.0), ui = d2(0.0, 0.0), vi = d2(0.0, 0.0), pi = d2(0.0, 0.0);
    if (i < n) {
        for (int c = 0; c < ncb; ++c) ri = add(ri, rowpart[int64_t(c) * n + i]);
        for (int c = 0; c < nrb; ++c) si = add(si, colpart[int64_t(c) * n + i]);
        r[i] = ri;
        s[i] = si;
        if (i >= 1) {
            ui = __ldg(A + i * n);
            vi = __ldg(A + i);
            pi = __ldg(A + i * n + i);
        } else {
            ri = d2(0.0, 0.0);
        }
    }
    red[0][threadIdx.x] = ui;
    red[1][threadIdx.x] = vi;
    red[2][threadIdx.x] = pi;
    red[3][threadIdx.x] = ri;
    __syncthreads();
    for (int w = 128; w; w >>= 1) {
        if (threadIdx.x < w)
            for (int q = 0; q < 4; ++q) red[q][threadIdx.x] = add(red[q][threadIdx.x], red[q][threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x < 4) blocktot[int64_t(blockIdx.x) * 4 + threadIdx.x] = red[threadIdx.x][0];
}

// tot[0..3] = U, V, P, O from the per-block totals (one block, fixed order)
__global__ void __launch_bounds__(256) recon_totals_kernel(const double2* __restrict__ blocktot, int nblk,
                                                           double2* __restrict__ tot) {
    __shared__ double2 red[4][256];
    double2 a[4] = {d2(0.0, 0.0), d2(0.0, 0.0), d2(0.0, 0.0), d2(0.0, 0.0)};
    for (int b = threadIdx.x; b < nblk; b += 256)
        for (int q = 0; q < 4; ++q) a[q] = add(a[q], blocktot[int64_t(b) * 4 + q]);
    for (int q = 0; q < 4; ++q) red[q][threadIdx.x] = a[q];
    __syncthreads();
    for (int w = 128; w; w >>= 1) {
        if (threadIdx.x < w)
            for (int q = 0; q < 4; ++q) red[q][threadIdx.x] = add(red[q][threadIdx.x], red[q][threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x < 4) tot[threadIdx.x] = red[threadIdx.x][0];
}

struct Agg {
    double2 u, v, p, r, s;  // of one molecule
};

// one output entry (a, b); R: the 5 x 17 responses (rep-major), tot: U V P O,
// Acc = A_cc
__device__ __forceinline__ double2 recon_entry(int64_t a, int64_t b, double2 Aab, double2 Aba, const Agg& ga,
                                               const Agg& gb, const double2* R, const double2* tot, double2 Acc) {
    const double2* Rc = R;                    // |c><c| (d = 0): slots Z X1 Y1 P1 T
    const double2* Rw = R + 4 * kRepSlots;    // |e_1><e_2| (d = 2)
    const double2 U = tot[0], V = tot[1], P = tot[2], O = tot[3];
    // the three d = 1 representatives with their weights
    const double2* R1[3] = {R + 1 * kRepSlots, R + 2 * kRepSlots, R + 3 * kRepSlots};
    double2 out;
    if (a == 0 && b == 0) {
        out = fma2(Acc, Rc[RZ], d2(0.0, 0.0));
        out = fma2(U, R1[0][RZ], out);
        out = fma2(V, R1[1][RZ], out);
        out = fma2(P, R1[2][RZ], out);
        out = fma2(O, Rw[RZ], out);
        return out;
    }
    if (b == 0 || a == 0) {
        // X (column 0) or Y (row 0) of molecule m
        const bool X = (b == 0);
        const Agg& g = X ? ga : gb;
        const int s1 = X ? RX1 : RY1, s2 = X ? RX2 : RY2, s3 = X ? RX3 : RY3;
        out = fma2(Acc, Rc[s1], d2(0.0, 0.0));
        const double2 w[3] = {g.u, g.v, g.p}, W[3] = {U, V, P};
        for (int q = 0; q < 3; ++q) {
            out = fma2(w[q], R1[q][s1], out);
            out = fma2(sub(W[q], w[q]), R1[q][s2], out);
        }
        out = fma2(g.r, Rw[s1], out);
        out = fma2(g.s, Rw[s2], out);
        out = fma2(sub(sub(O, g.r), g.s), Rw[s3], out);
        return out;
    }
    if (a == b) {
        out = fma2(Acc, Rc[RP1], d2(0.0, 0.0));
        const double2 w[3] = {ga.u, ga.v, ga.p}, W[3] = {U, V, P};
        for (int q = 0; q < 3; ++q) {
            out = fma2(w[q], R1[q][RP1], out);
            out = fma2(sub(W[q], w[q]), R1[q][RP2], out);
        }
        out = fma2(ga.r, Rw[RP1], out);
        out = fma2(ga.s, Rw[RP2], out);
        out = fma2(sub(sub(O, ga.r), ga.s), Rw[RP3], out);
        return out;
    }
    out = fma2(Acc, Rc[RT], d2(0.0, 0.0));
    const double2 wa[3] = {ga.u, ga.v, ga.p}, wb[3] = {gb.u, gb.v, gb.p}, W[3] = {U, V, P};
    for (int q = 0; q < 3; ++q) {
        out = fma2(wa[q], R1[q][RS12], out);
        out = fma2(wb[q], R1[q][RS21], out);
        out = fma2(sub(sub(W[q], wa[q]), wb[q]), R1[q][RT], out);
    }
    out = fma2(Aab, Rw[RS12], out);
    out = fma2(Aba, Rw[RS21], out);
    out = fma2(sub(ga.r, Aab), Rw[RS13], out);
    out = fma2(sub(ga.s, Aba), Rw[RS23], out);
    out = fma2(sub(gb.r, Aba), Rw[RS31], out);
    out = fma2(sub(gb.s, Aab), Rw[RS32], out);
    const double2 rest = add(sub(sub(sub(sub(O, ga.r), ga.s), gb.r), gb.s), add(Aab, Aba));
    out = fma2(rest, Rw[RT], out);
    return out;
}

// c1, c2 of the separated form: the |e_1><e_2| response's weights of A_ab, A_ba
__device__ __forceinline__ void sep_consts(const double2* Rw, double2& c1, double2& c2) {
    c1 = add(sub(sub(Rw[RS12], Rw[RS13]), Rw[RS32]), Rw[RT]);
    c2 = add(sub(sub(Rw[RS21], Rw[RS23]), Rw[RS31]), Rw[RT]);
}

// per index k: alpha_k and beta_k of the separated form, and the entries
// (0, k), (k, 0), (k, k) in the general form
__global__ void __launch_bounds__(256) recon_edges_kernel(const double2* __restrict__ A, int64_t n,
                                                          const double2* __restrict__ resp,
                                                          const double2* __restrict__ tot,
                                                          const double2* __restrict__ rv,
                                                          const double2* __restrict__ sv,
                                                          double2* __restrict__ alpha, double2* __restrict__ beta,
                                                          double2* __restrict__ B) {
    __shared__ double2 R[kReps * kRepSlots];
    __shared__ double2 T4[4];
    for (int t = threadIdx.x; t < kReps * kRepSlots; t += blockDim.x) R[t] = resp[t];
    if (threadIdx.x < 4) T4[threadIdx.x] = tot[threadIdx.x];
    __syncthreads();
    const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const double2 Acc = __ldg(A);
    const Agg z{d2(0.0, 0.0), d2(0.0, 0.0), d2(0.0, 0.0), d2(0.0, 0.0), d2(0.0, 0.0)};
    if (k == 0) {
        B[0] = recon_entry(0, 0, Acc, Acc, z, z, R, T4, Acc);
        alpha[0] = beta[0] = d2(0.0, 0.0);
        return;
    }
    Agg g;
    g.u = __ldg(A + k * n);
    g.v = __ldg(A + k);
    g.p = __ldg(A + k * n + k);
    g.r = rv[k];
    g.s = sv[k];
    B[k] = recon_entry(0, k, g.v, g.u, z, g, R, T4, Acc);          // (c, e_k)
    B[k * n] = recon_entry(k, 0, g.u, g.v, g, z, R, T4, Acc);      // (e_k, c)
    B[k * n + k] = recon_entry(k, k, g.p, g.p, g, g, R, T4, Acc);  // (e_k, e_k)
    const double2* Rc = R;
    const double2* Rw = R + 4 * kRepSlots;
    const double2 U = T4[0], V = T4[1], P = T4[2], O = T4[3];
    const double2 w[3] = {g.u, g.v, g.p}, W[3] = {U, V, P};
    // the constant terms go into alpha
    double2 a = fma2(Acc, Rc[RT], d2(0.0, 0.0));
    a = fma2(O, Rw[RT], a);
    double2 b = d2(0.0, 0.0);
    for (int q = 0; q < 3; ++q) {
        const double2* R1 = R + (1 + q) * kRepSlots;
        a = fma2(W[q], R1[RT], a);
        a = fma2(w[q], sub(R1[RS12], R1[RT]), a);
        b = fma2(w[q], sub(R1[RS21], R1[RT]), b);
    }
    a = fma2(g.r, sub(Rw[RS13], Rw[RT]), a);
    a = fma2(g.s, sub(Rw[RS23], Rw[RT]), a);
    b = fma2(g.r, sub(Rw[RS31], Rw[RT]), b);
    b = fma2(g.s, sub(Rw[RS32], Rw[RT]), b);
    alpha[k] = a;
    beta[k] = b;
}

// entries (a, b), a != b molecules: one CTA per tile pair {(I, J), (J, I)},
// I <= J, both tiles of A staged in shared memory, both output tiles written
// with coalesced rows
__global__ void __launch_bounds__(kT * 8) recon_output_kernel(const double2* __restrict__ A, int64_t n,
                                                             const double2* __restrict__ resp,
                                                             const double2* __restrict__ alpha,
                                                             const double2* __restrict__ beta,
                                                             double2* __restrict__ B) {
    const int64_t I = blockIdx.y, J = blockIdx.x;
    if (I > J) return;
    __shared__ double2 sA[kT][kT + 1];  // A(I-tile rows, J-tile cols)
    __shared__ double2 sB[kT][kT + 1];  // A(J-tile rows, I-tile cols)
    __shared__ double2 aI[kT], bI[kT], aJ[kT], bJ[kT];
    const int tx = threadIdx.x % kT, ty = threadIdx.x / kT;  // 32 x 8
    const int64_t i0 = I * kT, j0 = J * kT;
    if (threadIdx.x < 4 * kT) {
        const int q = threadIdx.x / kT, t = threadIdx.x % kT;
        const int64_t m = (q < 2 ? i0 : j0) + t;
        const double2 val = m < n ? ((q & 1) ? beta[m] : alpha[m]) : d2(0.0, 0.0);
        (q == 0 ? aI : q == 1 ? bI : q == 2 ? aJ : bJ)[t] = val;
    }
    for (int yy = ty; yy < kT; yy += 8) {
        const int64_t ra = i0 + yy, ca = j0 + tx;
        sA[yy][tx] = (ra < n && ca < n) ? __ldg(A + ra * n + ca) : d2(0.0, 0.0);
        if (I != J) {
            const int64_t rb = j0 + yy, cb = i0 + tx;
            sB[yy][tx] = (rb < n && cb < n) ? __ldg(A + rb * n + cb) : d2(0.0, 0.0);
        }
    }
    double2 c1, c2;
    sep_consts(resp + 4 * kRepSlots, c1, c2);
    __syncthreads();
    // tile (I, J): entry (a, b) = (i0 + yy, j0 + tx); A_ba lies in sB (or sA when I == J)
    for (int yy = ty; yy < kT; yy += 8) {
        const int64_t a = i0 + yy, b = j0 + tx;
        if (a >= 1 && b >= 1 && a != b && a < n && b < n) {
            const double2 Aba = (I == J) ? sA[tx][yy] : sB[tx][yy];
            double2 o = add(aI[yy], bJ[tx]);
            o = fma2(c1, sA[yy][tx], o);
            o = fma2(c2, Aba, o);
            B[a * n + b] = o;
        }
    }
    if (I == J) return;
    // tile (J, I): entry (a, b) = (j0 + yy, i0 + tx)
    for (int yy = ty; yy < kT; yy += 8) {
        const int64_t a = j0 + yy, b = i0 + tx;
        if (a >= 1 && b >= 1 && a != b && a < n && b < n) {
            double2 o = add(aJ[yy], bI[tx]);
            o = fma2(c1, sB[yy][tx], o);
            o = fma2(c2, sA[tx][yy], o);
            B[a * n + b] = o;
        }
    }
}

}  // namespace

size_t recon_workspace_bytes(int64_t n) {
    const int64_t ncb = (n + kCB - 1) / kCB, nrb = (n + kRB - 1) / kRB, nblk = (n + 255) / 256;
    // rowpart, colpart, r, s, alpha, beta, block totals, totals, responses
    return size_t(16) * size_t(ncb * n + nrb * n + 4 * n + 4 * nblk + 4 + kReps * kRepSlots);
}

cudaError_t launch_reconstruct(const InstDev* inst, const RepSrc* src, const void* main64,
                               const void* side64, const void* rho0, int64_t n, void* rho_t, void* ws,
                               cudaStream_t st) {
    const int64_t ncb = (n + kCB - 1) / kCB, nrb = (n + kRB - 1) / kRB, nblk = (n + 255) / 256;
    double2* w = static_cast<double2*>(ws);
    double2* rowpart = w;
    double2* colpart = rowpart + ncb * n;
    double2* r = colpart + nrb * n;
    double2* s = r + n;
    double2* alpha = s + n;
    double2* beta = alpha + n;
    double2* blocktot = beta + n;
    double2* tot = blocktot + 4 * nblk;
    double2* resp = tot + 4;
    const double2* A = static_cast<const double2*>(rho0);
    gather_responses_kernel<<<1, 128, 0, st>>>(inst, src, static_cast<const double2*>(main64),
                                              static_cast<const double2*>(side64), resp);
    recon_partials_kernel<<<dim3(unsigned(ncb), unsigned(nrb)), kCB, 0, st>>>(A, n, rowpart, colpart);
    recon_vectors_kernel<<<unsigned(nblk), 256, 0, st>>>(A, n, rowpart, int(ncb), colpart, int(nrb), r, s, blocktot);
    recon_totals_kernel<<<1, 256, 0, st>>>(blocktot, int(nblk), tot);
    double2* Bt = static_cast<double2*>(rho_t);
    recon_edges_kernel<<<unsigned(nblk), 256, 0, st>>>(A, n, resp, tot, r, s, alpha, beta, Bt);
    const unsigned nt = unsigned((n + kT - 1) / kT);
    recon_output_kernel<<<dim3(nt, nt), kT * 8, 0, st>>>(A, n, resp, alpha, beta, Bt);
    return cudaGetLastError();
}

}  // namespace sa
