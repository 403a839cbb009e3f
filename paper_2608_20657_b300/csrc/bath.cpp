// bath.cpp -- exponential decompositions of the Drude-Lorentz bath
// correlation function (Eq. Drude_Lorentz inserted in Eq. BCF-spectral,
// written as Eq. BCF-exp), plus the static-disorder channel of Eq. C_static.
//
// coth x = 1/x + sum_j 2 eta_j x / (x^2 + xi_j^2) gives the poles
// nu_j = 2 xi_j kT with weights c_j = eta_j (4 lambda gamma kT) nu_j /
// (nu_j^2 - gamma^2), and the gamma pole c_0 = lambda gamma (cot~(beta gamma/2)
// - i), cot~(y) = 1/y - sum_j 2 eta_j y / (xi_j^2 - y^2).
//   Matsubara: eta_j = 1, xi_j = j pi, and the exact cotangent for c_0.
//   Pade:      [K-1/K] approximant in z = x^2 of F(z) = (coth x - 1/x)/x,
//              from the continued fraction of F (see pade_poles).  Extended
//              (long double) precision throughout.
#include <algorithm>
#include <cmath>
#include <complex>
#include <string>
#include <vector>

#include "sa_internal.h"

namespace sa {

namespace {

using ld = long double;

// [K-1/K] Pade poles of F(z) = (coth x - 1/x)/x, z = x^2.  F is the
// continued fraction 1/(3 + z/(5 + z/(7 + ...))) (Lambert's fraction for
// tanh), whose convergent of depth 2K is the [K-1/K] approximant.  With the
// convergent denominators P_j = b_j P_{j-1} + z P_{j-2} (b_j = 2j + 3,
// P_{-1} = 1, P_{-2} = 0), z = -xi^2 and s = 1/xi, the values v_j = P_j s^{j+1}
// obey s v_{j-1} = (v_j + v_{j-2}) / b_j, so the zeros of P_{2K-1} are the
// eigenvalues s of the symmetric tridiagonal 2K x 2K matrix with zero diagonal
// and off-diagonals 1/sqrt(b_k b_{k+1}); its K positive eigenvalues give xi.
// Eigenvalues by Sturm-sequence bisection, residues 2 eta_j = Q(z_j)/P'(z_j)
// by the same recurrences -- all well conditioned.
bool pade_poles(int K, std::vector<ld>& eta, std::vector<ld>& xi) {
    const int n = 2 * K;
    std::vector<ld> e(n > 1 ? n - 1 : 1);
    for (int k = 0; k + 1 < n; ++k) e[k] = 1.0L / std::sqrt(ld(2 * k + 3) * ld(2 * k + 5));
    // number of eigenvalues below lam
    auto below = [&](ld lam) {
        int cnt = 0;
        ld d = -lam;
        if (d < 0) ++cnt;
        for (int k = 1; k < n; ++k) {
            if (d == 0) d = 1e-4000L;
            d = -lam - e[k - 1] * e[k - 1] / d;
            if (d < 0) ++cnt;
        }
        return cnt;
    };
    ld hi = 0;
    for (int k = 0; k + 1 < n; ++k) hi = std::max(hi, e[k]);
    hi = 2.0L * hi + 1.0L;
    eta.clear();
    xi.clear();
    for (int j = 0; j < K; ++j) {
        // the (K + j)-th smallest eigenvalue (0-based) is the j-th positive one
        const int idx = K + j;
        ld lo = 0.0L, up = hi;
        for (int it = 0; it < 200; ++it) {
            ld mid = 0.5L * (lo + up);
            if (mid == lo || mid == up) break;
            if (below(mid) > idx) up = mid;
            else lo = mid;
        }
        const ld s = 0.5L * (lo + up);
        if (!(s > 0)) return false;
        const ld x = 1.0L / s;
        const ld z = -x * x;
        // P_{n-1}(z), P'_{n-1}(z) from P_{-2} = 0, P_{-1} = 1 and the numerator
        // Q_{n-1}(z) from Q_{-1} = 0, Q_0 = 1, all by the same recurrence
        ld Pm2 = 0, Pm1 = 1, dPm2 = 0, dPm1 = 0;
        for (int k = 0; k < n; ++k) {
            const ld b = ld(2 * k + 3);
            const ld P = b * Pm1 + z * Pm2;
            const ld dP = b * dPm1 + Pm2 + z * dPm2;
            Pm2 = Pm1; Pm1 = P;
            dPm2 = dPm1; dPm1 = dP;
        }
        ld Qm2 = 0, Qm1 = 1;
        for (int k = 1; k < n; ++k) {
            const ld Q = ld(2 * k + 3) * Qm1 + z * Qm2;
            Qm2 = Qm1; Qm1 = Q;
        }
        if (dPm1 == 0) return false;
        xi.push_back(x);
        eta.push_back(Qm1 / dPm1 / 2.0L);
    }
    // ascending xi
    std::vector<std::pair<ld, ld>> pr;
    for (int j = 0; j < K; ++j) pr.push_back({xi[j], eta[j]});
    std::sort(pr.begin(), pr.end());
    for (int j = 0; j < K; ++j) {
        xi[j] = pr[j].first;
        eta[j] = pr[j].second;
    }
    return true;
}

}  // namespace

// Terminator strength of the Matsubara scheme: the omitted poles' c_j / nu_j.
// With nu_j = 2 pi j kT and c_j = 4 lambda gamma kT nu_j / (nu_j^2 - gamma^2),
// c_j / nu_j = 4 lambda gamma kT / (nu_j^2 - gamma^2), whose sum over all j
// is lambda (2 kT / gamma - cot(gamma / 2 kT)) (partial fractions of cot).
int terminator(double lambda, double gamma, double kT, int n_matsubara, double* out, std::string& err) {
    if (!out || !(lambda > 0) || !(gamma > 0) || !(kT > 0) || !std::isfinite(lambda) || !std::isfinite(gamma) ||
        !std::isfinite(kT) || n_matsubara < 0) {
        err = "lambda, gamma, kT > 0 and n_matsubara >= 0 required";
        return SA_ERR_INVALID_ARG;
    }
    const long double x = (long double)gamma / (2.0L * kT);
    const long double pi = 3.141592653589793238462643383279502884L;
    if (std::fabs(std::sin(x)) < 1e-300L) {
        err = "gamma / (2 kT) is a multiple of pi";
        return SA_ERR_INVALID_ARG;
    }
    long double d = (long double)lambda * (1.0L / x - std::cos(x) / std::sin(x));
    for (int j = 1; j <= n_matsubara; ++j) {
        const long double nuj = 2.0L * pi * j * kT;
        const long double den = nuj * nuj - (long double)gamma * gamma;
        if (den == 0.0L) {
            err = "a Matsubara pole coincides with gamma";
            return SA_ERR_INVALID_ARG;
        }
        d -= 4.0L * lambda * gamma * kT / den;
    }
    *out = double(d);
    return SA_OK;
}

int drude_lorentz(double lambda, double gamma, double kT, int scheme, int n_poles, double sigma, sa_params* p,
                  std::string& err) {
    if (!p || !(lambda > 0) || !(gamma > 0) || !(kT > 0) || !(sigma >= 0) || !std::isfinite(lambda) ||
        !std::isfinite(gamma) || !std::isfinite(kT) || !std::isfinite(sigma) || n_poles < 0) {
        err = "lambda, gamma, kT > 0 and sigma >= 0 required";
        return SA_ERR_INVALID_ARG;
    }
    int K = scheme == SA_BATH_HIGH_T ? 0 : n_poles;
    int m = 1 + K + (sigma > 0 ? 1 : 0);
    if (m > SA_HEOM_MAXM || (scheme == SA_BATH_PADE && K > 12) || scheme < 0 || scheme > 2) {
        err = "too many bath terms";
        return SA_ERR_INVALID_ARG;
    }
    std::vector<ld> eta, xi;
    const ld L = lambda, g = gamma, T = kT;
    const ld beta = 1.0L / T;
    const ld y = beta * g / 2.0L;
    ld cot0;
    if (scheme == SA_BATH_HIGH_T) {
        cot0 = 1.0L / y;  // cot(y) -> 1/y: c_0 = 2 lambda kT - i lambda gamma
    } else if (scheme == SA_BATH_MATSUBARA) {
        for (int j = 1; j <= K; ++j) {
            eta.push_back(1.0L);
            xi.push_back(ld(j) * 3.141592653589793238462643383279502884L);
        }
        cot0 = std::cos(y) / std::sin(y);
    } else {
        if (K > 0 && !pade_poles(K, eta, xi)) {
            err = "Pade pole construction failed";
            return SA_ERR_INVALID_ARG;
        }
        cot0 = 1.0L / y;
        for (int j = 0; j < K; ++j) cot0 -= 2.0L * eta[j] * y / (xi[j] * xi[j] - y * y);
    }
    p->m = m;
    for (int k = 0; k < SA_HEOM_MAXM; ++k) {
        p->c_re[k] = p->c_im[k] = p->cc_re[k] = p->cc_im[k] = p->nu_re[k] = p->nu_im[k] = 0.0;
    }
    p->c_re[0] = double(L * g * cot0);
    p->c_im[0] = double(-L * g);
    p->nu_re[0] = double(g);
    for (int j = 0; j < K; ++j) {
        ld nu = 2.0L * xi[j] / beta;
        p->c_re[1 + j] = double(eta[j] * (4.0L * L * g / beta) * nu / (nu * nu - g * g));
        p->nu_re[1 + j] = double(nu);
    }
    if (sigma > 0) {
        p->c_re[m - 1] = sigma * sigma;
        p->nu_re[m - 1] = 0.0;
    }
    for (int k = 0; k < m; ++k) {  // real rates: c-check_k = conj(c_k)
        p->cc_re[k] = p->c_re[k];
        p->cc_im[k] = -p->c_im[k];
    }
    return SA_OK;
}

}  // namespace sa
