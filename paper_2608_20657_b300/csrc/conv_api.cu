// conv_api.cu -- C ABI of the conventional-HEOM cross-check path
// (sa_conv_* in include/sa_heom.h): host enumeration of every label with its
// neighbour table, device upload, RK4 steps, dense state transfers.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <unordered_map>
#include <vector>

#include "sa_internal.h"

namespace sa {
struct ConvDev {
    const int32_t* nbr;
    const uint8_t* lab;
    const double2* gamma;
    const double2* coef;
    int N, D, m, L;
    double g, det, kappa, term;
    long long nado;
};
cudaError_t conv_launch(const ConvDev& P, const void* x, void* xout, const void* y, void* acc, void* yout,
                        double dt, int stage, cudaStream_t st);
}  // namespace sa

using namespace sa;

namespace {
thread_local std::string g_conv_err;
int cfail(int code, const std::string& m) {
    g_conv_err = m;
    return code;
}
#define CCK(call)                                                                      \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess) return cfail(SA_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)
}  // namespace

struct sa_conv {
    sa_params p{};
    int N = 0, D = 0, m = 0, L = 0;
    long long nado = 0;
    std::vector<uint8_t> lab;
    std::vector<int32_t> nbr;
    std::vector<double> gamma, coef;
    void *d_lab = nullptr, *d_nbr = nullptr, *d_gamma = nullptr, *d_coef = nullptr;
    void* d_work[3] = {nullptr, nullptr, nullptr};
    size_t state_bytes = 0;
};

namespace {

// labels with |n| <= L over N m components, lexicographic order (odometer
// with a running total)
void enumerate(sa_conv* c) {
    const int nm = c->N * c->m;
    std::vector<uint8_t> cur(nm, 0);
    int tot = 0;
    while (true) {
        c->lab.insert(c->lab.end(), cur.begin(), cur.end());
        int pos = nm - 1;
        while (pos >= 0) {
            if (tot < c->L) {
                ++cur[pos];
                ++tot;
                break;
            }
            tot -= cur[pos];
            cur[pos] = 0;
            --pos;
        }
        if (pos < 0) break;
    }
    c->nado = (long long)(c->lab.size() / nm);
}

void free_conv(sa_conv* c) {
    void* ptrs[] = {c->d_lab, c->d_nbr, c->d_gamma, c->d_coef, c->d_work[0], c->d_work[1], c->d_work[2]};
    for (void* p : ptrs)
        if (p) cudaFree(p);
}

ConvDev devview(const sa_conv* c) {
    ConvDev P;
    P.nbr = static_cast<const int32_t*>(c->d_nbr);
    P.lab = static_cast<const uint8_t*>(c->d_lab);
    P.gamma = static_cast<const double2*>(c->d_gamma);
    P.coef = static_cast<const double2*>(c->d_coef);
    P.N = c->N;
    P.D = c->D;
    P.m = c->m;
    P.L = c->L;
    P.g = c->p.g;
    P.det = c->p.detuning;
    P.kappa = c->p.kappa;
    P.term = c->p.term;
    P.nado = c->nado;
    return P;
}

}  // namespace

extern "C" {

int sa_conv_build(const sa_params* p, sa_conv** out) {
    if (!p || !out) return cfail(SA_ERR_INVALID_ARG, "params and out required");
    *out = nullptr;
    if (p->N < 1 || p->N > 64 || p->m < 1 || p->m > SA_HEOM_MAXM || p->L < 0 || p->L > SA_HEOM_MAXL)
        return cfail(SA_ERR_INVALID_ARG, "1 <= N <= 64, 1 <= m <= 8, 0 <= L <= 30 required");
    for (int k = 0; k < p->m; ++k)
        if (!(std::sqrt(p->c_re[k] * p->c_re[k] + p->c_im[k] * p->c_im[k]) > 0.0))
            return cfail(SA_ERR_INVALID_ARG, "|c_k| = 0");
    // the label count C(Nm + L, L) must stay modest: four state vectors (the
    // caller's and three RK4 work vectors) of at most 16 GB each
    const double lg = std::lgamma(double(p->N * p->m + p->L) + 1) - std::lgamma(double(p->L) + 1) -
                      std::lgamma(double(p->N * p->m) + 1);
    const double D = double(p->N + 1);
    if (lg > std::log(5.0e8) || std::exp(lg) * D * D * 16.0 > 16.0e9)
        return cfail(SA_ERR_UNSUPPORTED, "conventional hierarchy too large (more than 16 GB per state vector)");
    sa_conv* c = new sa_conv();
    c->p = *p;
    c->N = int(p->N);
    c->D = c->N + 1;
    c->m = p->m;
    c->L = p->L;
    enumerate(c);
    const int nm = c->N * c->m;
    // neighbour table: raise / lower of every (i, k)
    std::unordered_map<std::string, int32_t> index;
    index.reserve(size_t(c->nado) * 2);
    for (long long t = 0; t < c->nado; ++t)
        index.emplace(std::string(reinterpret_cast<const char*>(&c->lab[size_t(t) * nm]), nm), int32_t(t));
    c->nbr.assign(size_t(c->nado) * 2 * nm, -1);
    c->gamma.assign(size_t(c->nado) * 2, 0.0);
    std::string key(nm, '\0');
    for (long long t = 0; t < c->nado; ++t) {
        const uint8_t* n = &c->lab[size_t(t) * nm];
        int tier = 0;
        double gr = 0, gi = 0;
        for (int j = 0; j < nm; ++j) {
            tier += n[j];
            gr += n[j] * p->nu_re[j % c->m];
            gi += n[j] * p->nu_im[j % c->m];
        }
        c->gamma[2 * t] = gr;
        c->gamma[2 * t + 1] = gi;
        for (int j = 0; j < nm; ++j) {
            std::memcpy(&key[0], n, nm);
            if (tier < c->L) {
                key[j] = char(n[j] + 1);
                auto it = index.find(key);
                if (it != index.end()) c->nbr[size_t(t) * 2 * nm + j] = it->second;
                key[j] = char(n[j]);
            }
            if (n[j] > 0) {
                key[j] = char(n[j] - 1);
                auto it = index.find(key);
                if (it != index.end()) c->nbr[size_t(t) * 2 * nm + nm + j] = it->second;
            }
        }
    }
    // coefficients per channel: sqrt|c_k|, c_k / sqrt|c_k|, cc_k / sqrt|c_k|
    c->coef.assign(size_t(c->m) * 6, 0.0);
    for (int k = 0; k < c->m; ++k) {
        const double ac = std::sqrt(p->c_re[k] * p->c_re[k] + p->c_im[k] * p->c_im[k]);
        const double s = std::sqrt(ac);
        c->coef[6 * k + 0] = s;
        c->coef[6 * k + 2] = p->c_re[k] / s;
        c->coef[6 * k + 3] = p->c_im[k] / s;
        c->coef[6 * k + 4] = p->cc_re[k] / s;
        c->coef[6 * k + 5] = p->cc_im[k] / s;
    }
    c->state_bytes = size_t(c->nado) * c->D * c->D * 16;
    auto up = [&](void** d, const void* h, size_t bytes) -> int {
        cudaError_t e = cudaMalloc(d, bytes + 64);
        if (e != cudaSuccess) return cfail(SA_ERR_OOM, "cudaMalloc (conventional tables)");
        e = cudaMemcpy(*d, h, bytes, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cfail(SA_ERR_CUDA, cudaGetErrorString(e));
        return SA_OK;
    };
    int rc = up(&c->d_lab, c->lab.data(), c->lab.size());
    if (!rc) rc = up(&c->d_nbr, c->nbr.data(), c->nbr.size() * 4);
    if (!rc) rc = up(&c->d_gamma, c->gamma.data(), c->gamma.size() * 8);
    if (!rc) rc = up(&c->d_coef, c->coef.data(), c->coef.size() * 8);
    for (int w = 0; w < 3 && !rc; ++w) {
        if (cudaMalloc(&c->d_work[w], c->state_bytes) != cudaSuccess) rc = cfail(SA_ERR_OOM, "cudaMalloc (work)");
    }
    if (rc) {
        free_conv(c);
        delete c;
        return rc;
    }
    *out = c;
    return SA_OK;
}

void sa_conv_destroy(sa_conv* c) {
    if (!c) return;
    free_conv(c);
    delete c;
}

int sa_conv_info(const sa_conv* c, int64_t* n_ados, size_t* state_bytes) {
    if (!c) return cfail(SA_ERR_INVALID_ARG, "null handle");
    if (n_ados) *n_ados = c->nado;
    if (state_bytes) *state_bytes = c->state_bytes;
    return SA_OK;
}

int sa_conv_labels(const sa_conv* c, uint8_t* out) {
    if (!c || !out) return cfail(SA_ERR_INVALID_ARG, "handle and out required");
    std::copy(c->lab.begin(), c->lab.end(), out);
    return SA_OK;
}

int sa_conv_set_rho0(const sa_conv* c, const double* rho0, void* d_state, void* stream) {
    if (!c || !rho0 || !d_state) return cfail(SA_ERR_INVALID_ARG, "handle, rho0, d_state required");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    CCK(cudaMemsetAsync(d_state, 0, c->state_bytes, st));
    // the zero label is the first one: the physical density operator
    CCK(cudaMemcpyAsync(d_state, rho0, size_t(c->D) * c->D * 16, cudaMemcpyHostToDevice, st));
    CCK(cudaStreamSynchronize(st));
    return SA_OK;
}

int sa_conv_rhs(sa_conv* c, const void* d_x, void* d_dx, void* stream) {
    if (!c || !d_x || !d_dx || d_x == d_dx) return cfail(SA_ERR_INVALID_ARG, "distinct d_x, d_dx required");
    CCK(conv_launch(devview(c), d_x, d_dx, nullptr, nullptr, nullptr, 0.0, -1, static_cast<cudaStream_t>(stream)));
    return SA_OK;
}

int sa_conv_step(sa_conv* c, void* d_state, double dt, int64_t nsteps, void* stream) {
    if (!c || !d_state || nsteps < 0) return cfail(SA_ERR_INVALID_ARG, "handle, d_state, nsteps");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const ConvDev P = devview(c);
    void *acc = c->d_work[0], *xa = c->d_work[1], *xb = c->d_work[2];
    for (int64_t s = 0; s < nsteps; ++s) {
        CCK(conv_launch(P, d_state, xa, d_state, acc, nullptr, dt, 0, st));
        CCK(conv_launch(P, xa, xb, d_state, acc, nullptr, dt, 1, st));
        CCK(conv_launch(P, xb, xa, d_state, acc, nullptr, dt, 2, st));
        CCK(conv_launch(P, xa, nullptr, d_state, acc, d_state, dt, 3, st));
    }
    return SA_OK;
}

const char* sa_conv_last_error(void) { return g_conv_err.c_str(); }

}  // extern "C"
