// initial.cpp -- the factorised initial states of the physical representative
// (Sec. V.A and V.F) and the cm^-1 / K / fs unit set of Sec. V, behind the C
// ABI so that C callers and the Python binding get the same numbers.
#include <cmath>
#include <complex>
#include <string>

#include "sa_internal.h"

namespace {
using cplx = std::complex<double>;

int bad(const char* msg) {
    sa::set_error(msg);
    return SA_ERR_INVALID_ARG;
}

// (Z, X_0, Y_0, P_0, T_0) of a permutation-invariant state
int invariant_vars(const sa_params& p, int kind, const double* draws, cplx v[5]) {
    const double N = double(p.N);
    const double rn = std::sqrt(N);
    for (int j = 0; j < 5; ++j) v[j] = 0.0;
    switch (kind) {
        case SA_INIT_CAVITY:  // Eq. cavity-initial-uvar
            v[0] = 1.0;
            return SA_OK;
        case SA_INIT_BRIGHT:  // Eq. bright-initial-uvar: every entry of the molecular block 1/N
            v[3] = v[4] = 1.0 / N;
            return SA_OK;
        case SA_INIT_UP:
        case SA_INIT_LP: {
            // Eqs. upper-/lower-polariton-initial: tan 2 theta = Omega_R / Delta,
            // Omega_R = 2 g sqrt(N), Delta = omega_cav - eps_x, theta in [0, pi / 2]
            const double th = 0.5 * std::atan2(2.0 * p.g * rn, -p.detuning);
            const double s = std::sin(th), c = std::cos(th);
            const double a = kind == SA_INIT_UP ? c : s, b = kind == SA_INIT_UP ? s : -c;
            // |psi> = a |c> + b |B>: Z = a^2, X_0 = Y_0 = a b / sqrt N, P_0 = T_0 = b^2 / N
            v[0] = a * a;
            v[1] = v[2] = a * b / rn;
            v[3] = v[4] = b * b / N;
            return SA_OK;
        }
        case SA_INIT_RANDOM: {
            // draws: A (2 x 2 complex, row-major (re, im) pairs) and the dark
            // weight w: W = (1 - w) A A^+ / tr(A A^+) is the cavity-bright block
            // [[Z, sqrt N Y_0], [sqrt N X_0, P_0 + (N - 1) T_0]], and the dark
            // block has the single eigenvalue P_0 - T_0 = w / (N - 1)
            if (!draws) return bad("SA_INIT_RANDOM needs its draws");
            const cplx A[2][2] = {{cplx(draws[0], draws[1]), cplx(draws[2], draws[3])},
                                  {cplx(draws[4], draws[5]), cplx(draws[6], draws[7])}};
            const double wd = p.N >= 2 ? draws[8] : 0.0;
            if (!(wd >= 0.0 && wd < 1.0)) return bad("dark weight outside [0, 1)");
            cplx W[2][2];
            for (int i = 0; i < 2; ++i)
                for (int j = 0; j < 2; ++j) W[i][j] = A[i][0] * std::conj(A[j][0]) + A[i][1] * std::conj(A[j][1]);
            const double tr = W[0][0].real() + W[1][1].real();
            if (!(tr > 0.0)) return bad("draws give a zero cavity-bright block");
            for (int i = 0; i < 2; ++i)
                for (int j = 0; j < 2; ++j) W[i][j] *= (1.0 - wd) / tr;
            const double dark = p.N >= 2 ? wd / (N - 1.0) : 0.0;
            const double P0 = (W[1][1].real() + (N - 1.0) * dark) / N;
            v[0] = W[0][0].real();
            v[1] = W[1][0] / rn;
            v[2] = W[0][1] / rn;
            v[3] = P0;
            v[4] = P0 - dark;
            return SA_OK;
        }
        default:
            return bad("unknown initial-state kind");
    }
}
}  // namespace

extern "C" {

int sa_heom_initial_vars(const sa_params* p, int kind, const double* draws, double* out, int* count) {
    if (!p || !out || !count) return bad("params, out and count required");
    if (p->N < 1 || p->d < 0 || p->d > 1 || p->d > p->N) return bad("N >= 1 and d in {0, 1} (d <= N)");
    if (!std::isfinite(p->g) || !std::isfinite(p->detuning)) return bad("non-finite g or detuning");
    const int64_t N = p->N;
    cplx o[10];
    int n = 0;
    if (p->d == 0) {
        if (kind == SA_INIT_LOCALISED || kind == SA_INIT_SUPERPOSED) return bad("localised states need d = 1");
        cplx v[5];
        const int rc = invariant_vars(*p, kind, draws, v);
        if (rc) return rc;
        n = N >= 2 ? 5 : 4;
        for (int j = 0; j < n; ++j) o[j] = v[j];
    } else {
        // d = 1 (Sec. V.F): categories 1 = molecule 1, 2 = the other N - 1;
        // layout Z, X_1, X_2, Y_1, Y_2, P_1, P_2, S_12, S_21, T_2, cut short
        // for N = 1 (Z, X_1, Y_1, P_1) and N = 2 (no T_2)
        cplx Z, X1, X2, Y1, Y2, P1, P2, S, T;
        if (kind == SA_INIT_LOCALISED) {  // |e_1><e_1|
            Z = X1 = X2 = Y1 = Y2 = P2 = S = T = 0.0;
            P1 = 1.0;
        } else if (kind == SA_INIT_SUPERPOSED) {  // sqrt(0.3) |e_1> + sqrt(0.7) |c>
            const double a = std::sqrt(0.7 * 0.3);
            Z = 0.7;
            X1 = Y1 = a;
            P1 = 0.3;
            X2 = Y2 = P2 = S = T = 0.0;
        } else {  // a permutation-invariant state: molecule 1 like the others
            cplx v[5];
            const int rc = invariant_vars(*p, kind, draws, v);
            if (rc) return rc;
            Z = v[0];
            X1 = X2 = v[1];
            Y1 = Y2 = v[2];
            P1 = P2 = v[3];
            S = T = v[4];
        }
        if (N == 1) {
            o[0] = Z; o[1] = X1; o[2] = Y1; o[3] = P1;
            n = 4;
        } else {
            const cplx w[10] = {Z, X1, X2, Y1, Y2, P1, P2, S, S, T};
            n = N >= 3 ? 10 : 9;
            for (int j = 0; j < n; ++j) o[j] = w[j];
        }
    }
    for (int j = 0; j < n; ++j) {
        out[2 * j] = o[j].real();
        out[2 * j + 1] = o[j].imag();
    }
    *count = n;
    return SA_OK;
}

// Sec. V units with hbar = 1: an energy E in cm^-1 is the angular frequency
// 2 pi c E in rad/fs (c exact SI); k_B T in cm^-1 from the exact SI k_B, h, c
int sa_unit_cm_to_rad_fs(double e_cm, double* out) {
    if (!out || !std::isfinite(e_cm)) return bad("finite energy and out required");
    *out = e_cm * (2.0 * M_PI * 2.99792458e-5);
    return SA_OK;
}

int sa_unit_kT_rad_fs(double T_K, double* out) {
    if (!out || !(T_K >= 0.0) || !std::isfinite(T_K)) return bad("temperature >= 0 and out required");
    const double kB_cm = 1.380649e-23 / (6.62607015e-34 * 2.99792458e10);  // cm^-1 per K
    *out = T_K * kB_cm * (2.0 * M_PI * 2.99792458e-5);
    return SA_OK;
}

}  // extern "C"
