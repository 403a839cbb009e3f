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
// Kernels (FP64, HBM-bound): a tile pass of row / column partial sums, two
// small passes finishing the per-index vectors and the four totals (fixed
// summation order: the result is bitwise repeatable), and the output pass,
// one CTA per symmetric pair of 32 x 32 tiles so that A is read once and
// rho_S(t) written once.
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

// response value of representative r, slot k
__global__ void gather_responses_kernel(const InstDev* __restrict__ inst, const int16_t* __restrict__ loc, int nrep,
                                        const double2* __restrict__ main64, const double2* __restrict__ side64,
                                        double2* __restrict__ resp) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= kReps * kRepSlots) return;
    const int r = t / kRepSlots;
    double2 v = d2(0.0, 0.0);
    if (r < nrep) {
        const int l = loc[t];
        if (l >= 0) {
            const InstDev I = inst[r];
            v = side64 ? side64[I.side + l] : main64[I.var_begin + l];
        }
    }
    resp[t] = v;
}

// per tile (kRB rows x kCB columns): row partial sums rowpart[tile col][row]
// and column partial sums colpart[tile row][col] of the molecular block
// without its diagonal
__global__ void __launch_bounds__(kCB) recon_partials_kernel(const double2* __restrict__ A, int64_t n,
                                                             double2* __restrict__ rowpart,
                                                             double2* __restrict__ colpart) {
    __shared__ double2 red[kRB][kCB / 32];
    const int64_t j = int64_t(blockIdx.x) * kCB + threadIdx.x;
    const int64_t i0 = int64_t(blockIdx.y) * kRB;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double2 cs = d2(0.0, 0.0);
    for (int k = 0; k < kRB; ++k) {
        const int64_t i = i0 + k;
        double2 a = d2(0.0, 0.0);
        if (i < n && j < n && i >= 1 && j >= 1 && i != j) a = __ldg(A + i * n + j);
        cs = add(cs, a);
        double rx = a.x, ry = a.y;
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            rx += __shfl_xor_sync(0xffffffffu, rx, o);
            ry += __shfl_xor_sync(0xffffffffu, ry, o);
        }
        if (lane == 0) red[k][warp] = d2(rx, ry);
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

// one CTA per tile pair {(I, J), (J, I)}, I <= J: both tiles of A staged in
// shared memory, both output tiles written with coalesced rows
__global__ void __launch_bounds__(kT * 8, 2) recon_output_kernel(const double2* __restrict__ A, int64_t n,
                                                             const double2* __restrict__ resp,
                                                             const double2* __restrict__ tot,
                                                             const double2* __restrict__ rv,
                                                             const double2* __restrict__ sv,
                                                             double2* __restrict__ B) {
    const int64_t I = blockIdx.y, J = blockIdx.x;
    if (I > J) return;
    __shared__ double2 sA[kT][kT + 1];  // A(I-tile rows, J-tile cols)
    __shared__ double2 sB[kT][kT + 1];  // A(J-tile rows, I-tile cols)
    __shared__ double2 R[kReps * kRepSlots];
    __shared__ double2 T4[4];
    __shared__ Agg gI[kT], gJ[kT];
    const int tx = threadIdx.x % kT, ty = threadIdx.x / kT;  // 32 x 8
    const int64_t i0 = I * kT, j0 = J * kT;
    for (int t = threadIdx.x; t < kReps * kRepSlots; t += blockDim.x) R[t] = resp[t];
    if (threadIdx.x < 4) T4[threadIdx.x] = tot[threadIdx.x];
    for (int k = threadIdx.x; k < 2 * kT; k += blockDim.x) {
        const int64_t m = (k < kT ? i0 : j0) + (k % kT);
        Agg g{d2(0.0, 0.0), d2(0.0, 0.0), d2(0.0, 0.0), d2(0.0, 0.0), d2(0.0, 0.0)};
        if (m >= 1 && m < n) {
            g.u = __ldg(A + m * n);
            g.v = __ldg(A + m);
            g.p = __ldg(A + m * n + m);
            g.r = rv[m];
            g.s = sv[m];
        }
        (k < kT ? gI : gJ)[k % kT] = g;
    }
    for (int yy = ty; yy < kT; yy += 8) {
        const int64_t ra = i0 + yy, ca = j0 + tx;
        sA[yy][tx] = (ra < n && ca < n) ? __ldg(A + ra * n + ca) : d2(0.0, 0.0);
        if (I != J) {
            const int64_t rb = j0 + yy, cb = i0 + tx;
            sB[yy][tx] = (rb < n && cb < n) ? __ldg(A + rb * n + cb) : d2(0.0, 0.0);
        }
    }
    __syncthreads();
    const double2 Acc = __ldg(A);
    // tile (I, J): entry (a, b) = (i0 + yy, j0 + tx); A_ba lies in sB (or sA when I == J)
    for (int yy = ty; yy < kT; yy += 8) {
        const int64_t a = i0 + yy, b = j0 + tx;
        if (a < n && b < n) {
            const double2 Aab = sA[yy][tx];
            const double2 Aba = (I == J) ? sA[tx][yy] : sB[tx][yy];
            B[a * n + b] = recon_entry(a, b, Aab, Aba, gI[yy], gJ[tx], R, T4, Acc);
        }
    }
    if (I == J) return;
    // tile (J, I): entry (a, b) = (j0 + yy, i0 + tx)
    for (int yy = ty; yy < kT; yy += 8) {
        const int64_t a = j0 + yy, b = i0 + tx;
        if (a < n && b < n) {
            const double2 Aab = sB[yy][tx];
            const double2 Aba = sA[tx][yy];
            B[a * n + b] = recon_entry(a, b, Aab, Aba, gJ[yy], gI[tx], R, T4, Acc);
        }
    }
}

}  // namespace

size_t recon_workspace_bytes(int64_t n) {
    const int64_t ncb = (n + kCB - 1) / kCB, nrb = (n + kRB - 1) / kRB, nblk = (n + 255) / 256;
    // rowpart, colpart, r, s, block totals, totals, responses
    return size_t(16) * size_t(ncb * n + nrb * n + 2 * n + 4 * nblk + 4 + kReps * kRepSlots);
}

cudaError_t launch_reconstruct(const InstDev* inst, const int16_t* loc, int nrep, const void* main64,
                               const void* side64, const void* rho0, int64_t n, void* rho_t, void* ws,
                               cudaStream_t st) {
    const int64_t ncb = (n + kCB - 1) / kCB, nrb = (n + kRB - 1) / kRB, nblk = (n + 255) / 256;
    double2* w = static_cast<double2*>(ws);
    double2* rowpart = w;
    double2* colpart = rowpart + ncb * n;
    double2* r = colpart + nrb * n;
    double2* s = r + n;
    double2* blocktot = s + n;
    double2* tot = blocktot + 4 * nblk;
    double2* resp = tot + 4;
    const double2* A = static_cast<const double2*>(rho0);
    gather_responses_kernel<<<1, 128, 0, st>>>(inst, loc, nrep, static_cast<const double2*>(main64),
                                              static_cast<const double2*>(side64), resp);
    recon_partials_kernel<<<dim3(unsigned(ncb), unsigned(nrb)), kCB, 0, st>>>(A, n, rowpart, colpart);
    recon_vectors_kernel<<<unsigned(nblk), 256, 0, st>>>(A, n, rowpart, int(ncb), colpart, int(nrb), r, s, blocktot);
    recon_totals_kernel<<<1, 256, 0, st>>>(blocktot, int(nblk), tot);
    const unsigned nt = unsigned((n + kT - 1) / kT);
    recon_output_kernel<<<dim3(nt, nt), kT * 8, 0, st>>>(A, n, resp, tot, r, s, static_cast<double2*>(rho_t));
    return cudaGetLastError();
}

}  // namespace sa
