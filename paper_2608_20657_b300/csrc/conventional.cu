// conventional.cu -- the conventional scaled HEOM (Eq. scaled-HEOM) on the
// GPU, as a cross-check of the symmetry-adapted path on small ensembles.
//
// Every ADO label n in N0^{N m} with |n| <= L is kept (Eq. direct-ado-count)
// and every ADO is a dense (N+1) x (N+1) complex matrix in the basis
// {c, e_1..e_N} (Eq. basis).  Because Q_i = |e_i><e_i|, the entry (a, b) of
// [Q_i, A] and of c Q_i A - c-check A Q_i involves only the entry (a, b) of A,
// for i = a or i = b (Eq. projector-commutator-element).  So one thread owns
// one matrix entry of one ADO and gathers the same entry of the neighbouring
// ADOs n +/- e_ik named by a precomputed table; threads of one ADO share the
// table row and read neighbouring entries contiguously.  The system
// commutator needs the cavity row / column sums for the entries of row 0 and
// column 0.  The RK4 stage update is fused as in the symmetry-adapted kernel.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "sa_internal.h"

namespace sa {

struct ConvDev {
    const int32_t* nbr;     // per ADO: 2 N m neighbours (raise of (i,k), lower of (i,k)), -1 = none
    const uint8_t* lab;     // per ADO: N m occupations
    const double2* gamma;   // per ADO: Gamma_n
    const double2* coef;    // per k: [0] sqrt|c_k|, [1] c_k / sqrt|c_k|, [2] cc_k / sqrt|c_k| (complex)
    int N, D, m, L;
    double g, det, kappa, term;
    long long nado;
};

__global__ void __launch_bounds__(256) conv_stage_kernel(ConvDev P, const double2* __restrict__ x,
                                                         double2* __restrict__ xout, const double2* __restrict__ y,
                                                         double2* __restrict__ acc, double2* __restrict__ yout,
                                                         double dt, int stage) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int D = P.D, D2 = D * D, N = P.N, m = P.m;
    if (e >= P.nado * D2) return;
    const long long t = e / D2;
    const int ab = int(e - t * D2);
    const int a = ab / D, b = ab - a * D;
    const double2* rho = x + t * D2;
    const double2 v = rho[ab];
    // -i [H, rho]_{ab} with H = det sum_i |e_i><e_i| + g sum_i (|c><e_i| + |e_i><c|)
    const double hr = (a > 0 ? P.det : 0.0);
    double2 Hr;  // (H rho)_{ab} - (rho H)_{ab}
    {
        double sx = 0, sy = 0;
        if (a == 0) {
            for (int i = 1; i <= N; ++i) { sx += rho[i * D + b].x; sy += rho[i * D + b].y; }
        } else {
            sx = rho[b].x;
            sy = rho[b].y;
        }
        double tx = 0, ty = 0;
        if (b == 0) {
            for (int j = 1; j <= N; ++j) { tx += rho[a * D + j].x; ty += rho[a * D + j].y; }
        } else {
            tx = rho[a * D].x;
            ty = rho[a * D].y;
        }
        const double hb = (b > 0 ? P.det : 0.0);
        Hr.x = (hr - hb) * v.x + P.g * (sx - tx);
        Hr.y = (hr - hb) * v.y + P.g * (sy - ty);
    }
    const double2 gam = P.gamma[t];
    // cavity loss and the terminator: sum_i [Q_i, [Q_i, rho]]_{ab} counts the
    // molecules i for which exactly one of a, b is e_i
    const double lk = 0.5 * P.kappa * ((a == 0 ? 1.0 : 0.0) + (b == 0 ? 1.0 : 0.0)) +
                      P.term * (a != b ? double((a > 0) + (b > 0)) : 0.0);
    // -i Hr - Gamma v - loss v
    double dx = Hr.y - (gam.x + lk) * v.x + gam.y * v.y;
    double dy = -Hr.x - (gam.x + lk) * v.y - gam.y * v.x;
    // hierarchy terms for molecule i = a (row delta) and i = b (column delta)
    const int32_t* nb = P.nbr + t * (2LL * N * m);
    const uint8_t* n = P.lab + t * (long long)(N * m);
    for (int side = 0; side < 2; ++side) {
        const int i = side == 0 ? a : b;  // molecule 1..N
        if (i == 0) continue;
        if (side == 1 && a == b) {
            // a = b = e_i: the raise terms cancel; the lower terms give (c - cc)
            for (int k = 0; k < m; ++k) {
                const int nik = n[(i - 1) * m + k];
                const int dn = nb[N * m + (i - 1) * m + k];
                if (nik > 0 && dn >= 0) {
                    const double s = sqrt(double(nik));
                    const double2 c = P.coef[3 * k + 1], cc = P.coef[3 * k + 2];
                    const double2 w = x[(long long)dn * D2 + ab];
                    // -i s (c - cc) w
                    const double fx = s * (c.x - cc.x), fy = s * (c.y - cc.y);
                    dx += fx * w.y + fy * w.x;
                    dy += -(fx * w.x - fy * w.y);
                }
            }
            continue;
        }
        if (side == 0 && a == b) continue;  // handled on the column pass
        const double sg = side == 0 ? -1.0 : 1.0;  // -i for the row delta, +i for the column delta
        for (int k = 0; k < m; ++k) {
            const int nik = n[(i - 1) * m + k];
            const int up = nb[(i - 1) * m + k];
            const int dn = nb[N * m + (i - 1) * m + k];
            if (up >= 0) {
                const double s = sqrt(double(nik + 1)) * P.coef[3 * k].x;
                const double2 w = x[(long long)up * D2 + ab];
                // sg i s w
                dx += -sg * s * w.y;
                dy += sg * s * w.x;
            }
            if (nik > 0 && dn >= 0) {
                const double s = sqrt(double(nik));
                const double2 c = side == 0 ? P.coef[3 * k + 1] : P.coef[3 * k + 2];
                const double2 w = x[(long long)dn * D2 + ab];
                const double px = c.x * w.x - c.y * w.y, py = c.x * w.y + c.y * w.x;
                // sg i s c w
                dx += -sg * s * py;
                dy += sg * s * px;
            }
        }
    }
    const double2 k2 = make_double2(dx, dy);
    if (stage < 0) {
        xout[e] = k2;
    } else if (stage == 0) {
        acc[e] = k2;
        xout[e] = make_double2(v.x + 0.5 * dt * dx, v.y + 0.5 * dt * dy);
    } else if (stage == 3) {
        const double2 yv = y[e], av = acc[e];
        yout[e] = make_double2(yv.x + dt / 6.0 * (av.x + dx), yv.y + dt / 6.0 * (av.y + dy));
    } else {
        const double2 yv = y[e], av = acc[e];
        acc[e] = make_double2(av.x + 2.0 * dx, av.y + 2.0 * dy);
        const double s = stage == 2 ? dt : 0.5 * dt;
        xout[e] = make_double2(yv.x + s * dx, yv.y + s * dy);
    }
}

cudaError_t conv_launch(const ConvDev& P, const void* x, void* xout, const void* y, void* acc, void* yout,
                        double dt, int stage, cudaStream_t st) {
    const long long n = P.nado * P.D * P.D;
    const int block = 256;
    const long long grid = (n + block - 1) / block;
    conv_stage_kernel<<<unsigned(grid), block, 0, st>>>(
        P, static_cast<const double2*>(x), static_cast<double2*>(xout), static_cast<const double2*>(y),
        static_cast<double2*>(acc), static_cast<double2*>(yout), dt, stage);
    return cudaGetLastError();
}

}  // namespace sa
