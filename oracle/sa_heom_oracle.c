/*
 * sa_heom_oracle.c -- ORACLE: test infrastructure only.
 *
 * Plain, slow, FP64 CPU reference for Mondal & Huo, "Symmetry Adapted
 * Hierarchical Equations of Motion for Exact Simulations of Large Polariton
 * Systems" (arXiv 2608.20657).  Only the test suite, the package smoke check
 * and the CPU-baseline leg of the benchmark load this file's library.  The
 * product library shares no code, header, table or helper with it.
 *
 * Two independent parts:
 *
 *  O-1  Conventional scaled HEOM (Sec. II.C, Eq. scaled-HEOM): every label
 *       n in N0^{N m} with |n| <= L (Eq. direct-ado-count), every ADO a dense
 *       (N+1)x(N+1) matrix in the basis {c, e_1..e_N} (Eq. basis), the system
 *       Hamiltonian of Eq. HS, hard cutoff at tier L.  Matrix products are
 *       written out with explicit Q_i = |e_i><e_i| matrices.
 *
 *  O-2  Symmetry-adapted HEOM (Secs. III-IV): canonical occupation patterns
 *       (Eq. pattern-one; local hierarchy vectors for m > 1 per the last
 *       paragraph of Sec. IV), categories and multiplicities (Eqs. Mq, M0),
 *       unique variables Z, X_q, Y_q, P_q, S_{q,r}, T_q (Eqs. Z-variable ..
 *       T-variable, counted by Eq. uvar-count), grouped row and column sums
 *       (Eqs. grouped-row-sum, grouped-column-sum), Hamiltonian + damping
 *       terms (Eqs. HZ, HX and the same derivation for Y, P, S, T), hierarchy
 *       terms through the aligned-target accessor (Eqs. aligned-accessor,
 *       projector-commutator-element, uvar-up, uvar-down).
 *
 * Readings where the paper is silent (its Supporting Information is absent):
 *  - m > 1: a local vector alpha in N0^m moves as a unit; vectors are ordered
 *    by |alpha| descending, then components lexicographically descending;
 *    a pattern is the multiset of nonzero vectors, listed in that order.
 *  - Aligned accessor: an entry (x, y) of the aligned target is the variable
 *    of the canonical target selected by the local vectors the molecules
 *    named by x and y carry in the raw target (Eq. aligned-target without an
 *    explicit permutation).
 *  - Cavity loss: Lindblad kappa (a rho a^+ - 1/2 {a^+ a, rho}); the jump part
 *    leaves the single-excitation manifold, so -kappa/2 {|c><c|, .} acts on
 *    every ADO.
 *  - Terminator (Sec. V names the Ishizaki-Tanimura treatment of the omitted
 *    Matsubara terms without a formula): the residual correlation is taken as
 *    white noise of weight Delta = sum over omitted terms of c_k / nu_k, which
 *    adds -Delta sum_i [Q_i, [Q_i, rho_n]] to every ADO (off when Delta = 0).
 *  - Distinguished molecules (Sec. IV, Eq. N-symmetric-pool; Sec. V.F): with
 *    d of them, molecule j <= d carries its vector v as id j V + v, so its
 *    vector is a category of its own (M = 1) in every pattern, and the lists
 *    end with molecules 1..d in order; the other N - d molecules fill at most
 *    min(L, N - d) nonzero slots and the zero category holds N - r of them
 *    (r counting the distinguished entries).
 *  - Pattern order (the global vector of Eq. global-R): tier ascending, then
 *    the vector lists compared lexicographically with larger vectors first.
 *    Variable order inside a pattern: Z; X_1..X_G; Y_1..Y_G; P_1..P_G;
 *    S_{q,r} for q = 1..G, r = 1..G, r != q (row major); T_q for each q with
 *    M_q >= 2 in category order.  Categories: distinct nonzero vectors in
 *    pattern order, then the zero category when M_0 = N - r >= 1.
 *
 * Complex numbers are stored interleaved (re, im) in double arrays.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

#define ORC_MAXM 8
#define ORC_MAXD 3   /* distinguished molecules */

/* count of internal inconsistencies (a missing target or category); a
 * correct oracle leaves it at zero and the tests assert that */
static long long g_orc_errors = 0;
long long orc_errors(void) { return g_orc_errors; }

typedef struct {
    long long N;    /* number of molecules, >= 1 */
    int m;          /* exponentials per local bath */
    int L;          /* hierarchy depth */
    double detuning;/* eps_x - omega_cav (omega_cav = 0 in the rotating frame) */
    double g;       /* single-molecule light-matter coupling */
    double kappa;   /* photon population decay rate */
    double c_re[ORC_MAXM], c_im[ORC_MAXM];   /* c_k  (Eq. BCF-exp) */
    double cc_re[ORC_MAXM], cc_im[ORC_MAXM]; /* c-check_k */
    double nu_re[ORC_MAXM], nu_im[ORC_MAXM]; /* nu_k */
    double term;    /* terminator strength Delta (0: off) */
    int d;          /* distinguished molecules 0..ORC_MAXD: molecules 1..d keep their labels */
} orc_params;

static cplx ck(const orc_params* p, int k) { return p->c_re[k] + I * p->c_im[k]; }
static cplx cck(const orc_params* p, int k) { return p->cc_re[k] + I * p->cc_im[k]; }
static cplx nuk(const orc_params* p, int k) { return p->nu_re[k] + I * p->nu_im[k]; }
/* |c_k|, written as the modulus definition. */
static double absck(const orc_params* p, int k) {
    return sqrt(p->c_re[k] * p->c_re[k] + p->c_im[k] * p->c_im[k]);
}

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ====================================================================== */
/*  Local hierarchy vectors alpha in N0^m, |alpha| <= L                    */
/* ====================================================================== */

typedef struct {
    int m, L;
    int V;                 /* vectors including the zero vector (id 0) */
    int Vtot;              /* (d + 1) V: ids j V .. j V + V - 1 are distinguished
                              molecule j's vectors (id - j V), j = 1..d */
    unsigned char* comp;   /* Vtot * m components */
    int* norm;             /* |alpha| */
    int* lut;              /* mixed-radix (L+1)^m code -> id, -1 if |alpha| > L */
    long long lut_size;
} vecset;

static int g_sort_m; /* qsort comparator context */

/* Vector order: |alpha| descending, then components lexicographically
 * descending.  Returns <0 if a comes first. */
static int vec_cmp_raw(const unsigned char* a, const unsigned char* b, int m) {
    int na = 0, nb = 0;
    for (int k = 0; k < m; ++k) { na += a[k]; nb += b[k]; }
    if (na != nb) return na > nb ? -1 : 1;
    for (int k = 0; k < m; ++k)
        if (a[k] != b[k]) return a[k] > b[k] ? -1 : 1;
    return 0;
}
static int vec_qsort_cmp(const void* a, const void* b) {
    return vec_cmp_raw((const unsigned char*)a, (const unsigned char*)b, g_sort_m);
}

static long long vec_code(const unsigned char* a, int m, int L) {
    long long c = 0;
    for (int k = 0; k < m; ++k) c = c * (L + 1) + a[k];
    return c;
}

static void vecset_build(vecset* vs, int m, int L, int d) {
    vs->m = m; vs->L = L;
    long long total = 1;
    for (int k = 0; k < m; ++k) total *= (L + 1);
    vs->lut_size = total;
    /* every tuple with components <= L; keep those with |alpha| <= L */
    unsigned char* all = (unsigned char*)malloc((size_t)total * m);
    int cnt = 0;
    unsigned char t[ORC_MAXM];
    for (long long code = 0; code < total; ++code) {
        long long c = code; int s = 0;
        for (int k = m - 1; k >= 0; --k) { t[k] = (unsigned char)(c % (L + 1)); c /= (L + 1); s += t[k]; }
        if (s <= L) { memcpy(all + (size_t)cnt * m, t, m); ++cnt; }
    }
    g_sort_m = m;
    qsort(all, cnt, m, vec_qsort_cmp);
    /* after sorting, the zero vector is last; move it to id 0 */
    vs->V = cnt;   /* >= 1: the zero vector is always in the set */
    vs->Vtot = (d + 1) * cnt;
    vs->comp = (unsigned char*)calloc((size_t)vs->Vtot + 1, m);
    for (int v = 1; v < cnt; ++v)
        for (int k = 0; k < m; ++k) vs->comp[(size_t)v * m + k] = all[(size_t)(v - 1) * m + k];
    free(all);
    vs->norm = (int*)malloc(sizeof(int) * vs->Vtot);
    vs->lut = (int*)malloc(sizeof(int) * total);
    for (long long c = 0; c < total; ++c) vs->lut[c] = -1;
    for (int v = 0; v < cnt; ++v) {
        int s = 0;
        for (int k = 0; k < m; ++k) s += vs->comp[v * m + k];
        vs->norm[v] = s;
        vs->lut[vec_code(vs->comp + (size_t)v * m, m, L)] = v;
    }
    for (int v = cnt; v < vs->Vtot; ++v) { /* the distinguished molecules' copies */
        memcpy(vs->comp + (size_t)v * m, vs->comp + (size_t)(v % cnt) * m, m);
        vs->norm[v] = vs->norm[v % cnt];
    }
}

static void vecset_free(vecset* vs) { free(vs->comp); free(vs->norm); free(vs->lut); }

/* id of alpha +/- e_k; -1 if it leaves the set (negative or |alpha| > L).
 * A distinguished molecule's vector stays among its own ids. */
static int vec_shift(const vecset* vs, int id, int k, int dir) {
    unsigned char t[ORC_MAXM];
    memcpy(t, vs->comp + (size_t)id * vs->m, vs->m);
    int v = (int)t[k] + dir;
    if (v < 0 || v > vs->L) return -1;
    t[k] = (unsigned char)v;
    int w = vs->lut[vec_code(t, vs->m, vs->L)];
    if (w < 0) return -1;
    return (id / vs->V) * vs->V + w;
}

/* ====================================================================== */
/*  O-2: symmetry-adapted HEOM                                             */
/* ====================================================================== */

enum { K_Z = 0, K_X = 1, K_Y = 2, K_P = 3, K_S = 4, K_T = 5 };

typedef struct {
    orc_params p;
    vecset vs;
    long long P;            /* number of canonical patterns */
    long long* id_off;      /* P+1 offsets into ids */
    int* ids;               /* nonzero vector ids of each pattern, ascending id */
    int* tier;
    int* G;                 /* categories per pattern */
    int* h;                 /* categories with M_q >= 2 */
    long long* cat_off;     /* P+1 offsets into cat_id / cat_M */
    int* cat_id;            /* vector id of each category (0 = zero category) */
    long long* cat_M;       /* multiplicity of each category */
    int* trank;             /* rank of a category among those with M >= 2, -1 otherwise */
    long long* var_off;     /* P+1 offsets of each pattern's variables */
    cplx* gamma;            /* Gamma_Lambda */
    long long nvar;
    int* tcache;            /* optional: per (pattern, category, k, dir) target pattern, -2 = unset */
} orc_sa;


/* pattern comparator: tier ascending, then ids ascending (larger vectors
 * first), shorter list first on a common prefix (never happens within a
 * tier, kept for completeness). */
static int pat_cmp_lists(int tiera, const int* a, int ra, int tierb, const int* b, int rb) {
    if (tiera != tierb) return tiera < tierb ? -1 : 1;
    int r = ra < rb ? ra : rb;
    for (int i = 0; i < r; ++i)
        if (a[i] != b[i]) return a[i] < b[i] ? -1 : 1;
    if (ra != rb) return ra < rb ? -1 : 1;
    return 0;
}

typedef struct { int tier; int r; long long off; } patref;
static const int* g_sort_ids;
static int patref_cmp(const void* x, const void* y) {
    const patref* a = (const patref*)x;
    const patref* b = (const patref*)y;
    return pat_cmp_lists(a->tier, g_sort_ids + a->off, a->r, b->tier, g_sort_ids + b->off, b->r);
}

/* recursive enumeration of multisets: ids non-decreasing, sum of norms <= L,
 * length <= maxr */
typedef struct {
    int* buf; long long len, cap;    /* flat ids */
    patref* refs; long long n, ncap;
} patgen;

static void patgen_push(patgen* pg, const int* cur, int r, int tier) {
    if (pg->len + r > pg->cap) {
        pg->cap = (pg->cap + r) * 2;
        pg->buf = (int*)realloc(pg->buf, sizeof(int) * pg->cap);
    }
    if (pg->n + 1 > pg->ncap) {
        pg->ncap = (pg->ncap + 1) * 2;
        pg->refs = (patref*)realloc(pg->refs, sizeof(patref) * pg->ncap);
    }
    memcpy(pg->buf + pg->len, cur, sizeof(int) * r);
    pg->refs[pg->n].tier = tier;
    pg->refs[pg->n].r = r;
    pg->refs[pg->n].off = pg->len;
    pg->len += r;
    pg->n += 1;
}

/* extra[0..nextra-1]: the distinguished molecules' ids, appended to every
 * multiset (they are the largest ids, in molecule order, so the list stays
 * ascending); their norms are already in tier */
static void patgen_rec(patgen* pg, const vecset* vs, int* cur, int r, int tier, int start, int maxr,
                       const int* extra, int nextra) {
    for (int j = 0; j < nextra; ++j) cur[r + j] = extra[j];
    patgen_push(pg, cur, r + nextra, tier);
    if (r >= maxr) return;
    for (int v = start; v < vs->V; ++v) {
        if (tier + vs->norm[v] > vs->L) continue;
        cur[r] = v;
        patgen_rec(pg, vs, cur, r + 1, tier + vs->norm[v], v, maxr, extra, nextra);
    }
}

/* every choice of the d distinguished molecules' vectors (zero vector
 * included) with total norm <= L, then the multisets of the others */
static void patgen_dist(patgen* pg, const vecset* vs, int* cur, int* extra, int j, int d, int tier, int maxr) {
    if (j == d) {
        patgen_rec(pg, vs, cur, 0, tier, 1, maxr, extra, d);
        return;
    }
    for (int dv = 0; dv < vs->V; ++dv) {
        if (tier + vs->norm[dv] > vs->L) continue;
        extra[j] = (j + 1) * vs->V + dv;
        patgen_dist(pg, vs, cur, extra, j + 1, d, tier + vs->norm[dv], maxr);
    }
}

static void fill_cache(orc_sa* s);

static long long pat_find(const orc_sa* s, const int* key, int r, int tier) {
    long long lo = 0, hi = s->P - 1;
    while (lo <= hi) {
        long long mid = (lo + hi) / 2;
        int c = pat_cmp_lists(s->tier[mid], s->ids + s->id_off[mid], (int)(s->id_off[mid + 1] - s->id_off[mid]),
                              tier, key, r);
        if (c == 0) return mid;
        if (c < 0) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

/* index of variable (kind, q, r) inside a pattern; categories 1..G */
static long long var_local(int G, int kind, int q, int r, int trank_q) {
    switch (kind) {
    case K_Z: return 0;
    case K_X: return q;
    case K_Y: return G + q;
    case K_P: return 2 * G + q;
    case K_S: return 3 * G + 1 + (long long)(q - 1) * (G - 1) + (r - 1) - (r > q ? 1 : 0);
    case K_T: return (long long)(G + 1) * (G + 1) + trank_q;
    }
    return -1;
}

orc_sa* orc_sa_create(const orc_params* p, int use_cache) {
    if (p->N < 1 || p->m < 1 || p->m > ORC_MAXM || p->L < 0 || p->d < 0 || p->d > ORC_MAXD || p->d > p->N)
        return NULL;
    for (int k = 0; k < p->m; ++k)
        if (!(absck(p, k) > 0.0)) return NULL;
    orc_sa* s = (orc_sa*)calloc(1, sizeof(orc_sa));
    s->p = *p;
    vecset_build(&s->vs, p->m, p->L, p->d);
    /* patterns: at most N - d nonzero vectors of the undistinguished
     * molecules, never more than L; each distinguished molecule's vector
     * (zero included) is one more entry of every pattern */
    int maxr = p->L;
    if ((long long)maxr > p->N - p->d) maxr = (int)(p->N - p->d);
    patgen pg; memset(&pg, 0, sizeof(pg));
    int cur[256], extra[ORC_MAXD + 1];
    patgen_dist(&pg, &s->vs, cur, extra, 0, p->d, 0, maxr);
    g_sort_ids = pg.buf;
    qsort(pg.refs, pg.n, sizeof(patref), patref_cmp);
    s->P = pg.n;
    s->id_off = (long long*)malloc(sizeof(long long) * (s->P + 1));
    s->ids = (int*)malloc(sizeof(int) * (pg.len > 0 ? pg.len : 1));
    s->tier = (int*)malloc(sizeof(int) * s->P);
    long long o = 0;
    for (long long i = 0; i < s->P; ++i) {
        s->id_off[i] = o;
        memcpy(s->ids + o, pg.buf + pg.refs[i].off, sizeof(int) * pg.refs[i].r);
        s->tier[i] = pg.refs[i].tier;
        o += pg.refs[i].r;
    }
    s->id_off[s->P] = o;
    free(pg.buf); free(pg.refs);

    /* categories (Eq. Mq, Eq. M0), variable counts (Eq. uvar-count) */
    s->G = (int*)malloc(sizeof(int) * s->P);
    s->h = (int*)malloc(sizeof(int) * s->P);
    s->cat_off = (long long*)malloc(sizeof(long long) * (s->P + 1));
    s->var_off = (long long*)malloc(sizeof(long long) * (s->P + 1));
    s->gamma = (cplx*)malloc(sizeof(cplx) * s->P);
    long long ncat = 0;
    for (long long i = 0; i < s->P; ++i) {
        int r = (int)(s->id_off[i + 1] - s->id_off[i]);
        int distinct = 0;
        for (int a = 0; a < r; ++a)
            if (a == 0 || s->ids[s->id_off[i] + a] != s->ids[s->id_off[i] + a - 1]) ++distinct;
        ncat += distinct + ((p->N - r) >= 1 ? 1 : 0);
    }
    s->cat_id = (int*)malloc(sizeof(int) * (ncat > 0 ? ncat : 1));
    s->cat_M = (long long*)malloc(sizeof(long long) * (ncat > 0 ? ncat : 1));
    s->trank = (int*)malloc(sizeof(int) * (ncat > 0 ? ncat : 1));
    long long co = 0, vo = 0;
    for (long long i = 0; i < s->P; ++i) {
        int r = (int)(s->id_off[i + 1] - s->id_off[i]);
        const int* ids = s->ids + s->id_off[i];
        s->cat_off[i] = co;
        int G = 0;
        for (int a = 0; a < r; ++a) {
            if (a == 0 || ids[a] != ids[a - 1]) {
                s->cat_id[co + G] = ids[a];
                s->cat_M[co + G] = 1;
                ++G;
            } else {
                s->cat_M[co + G - 1] += 1;
            }
        }
        long long M0 = p->N - r;
        if (M0 >= 1) { s->cat_id[co + G] = 0; s->cat_M[co + G] = M0; ++G; }
        int h = 0;
        for (int q = 0; q < G; ++q) {
            if (s->cat_M[co + q] >= 2) s->trank[co + q] = h++;
            else s->trank[co + q] = -1;
        }
        s->G[i] = G; s->h[i] = h;
        s->var_off[i] = vo;
        vo += (long long)(G + 1) * (G + 1) + h;
        /* Gamma_Lambda = sum_i sum_k n_ik nu_k (Eq. tier-damping) */
        cplx gam = 0;
        for (int q = 0; q < G; ++q) {
            int v = s->cat_id[co + q];
            for (int k = 0; k < p->m; ++k)
                gam += (double)s->cat_M[co + q] * (double)s->vs.comp[(size_t)v * p->m + k] * nuk(p, k);
        }
        s->gamma[i] = gam;
        co += G;
    }
    s->cat_off[s->P] = co;
    s->var_off[s->P] = vo;
    s->nvar = vo;
    if (use_cache) {
        s->tcache = (int*)malloc(sizeof(int) * (size_t)(co > 0 ? co : 1) * p->m * 2);
        fill_cache(s);
    }
    return s;
}

void orc_sa_destroy(orc_sa* s) {
    if (!s) return;
    vecset_free(&s->vs);
    free(s->id_off); free(s->ids); free(s->tier); free(s->G); free(s->h);
    free(s->cat_off); free(s->cat_id); free(s->cat_M); free(s->trank);
    free(s->var_off); free(s->gamma); free(s->tcache);
    free(s);
}

long long orc_sa_num_patterns(const orc_sa* s) { return s->P; }
long long orc_sa_num_vars(const orc_sa* s) { return s->nvar; }
int orc_sa_num_vectors(const orc_sa* s) { return s->vs.V; }
long long orc_sa_num_categories(const orc_sa* s) { return s->cat_off[s->P]; }

void orc_sa_vectors(const orc_sa* s, unsigned char* out) { memcpy(out, s->vs.comp, (size_t)s->vs.V * s->vs.m); }

/* per pattern: tier, r, G, h, var_off, cat_off; ids padded with -1 to width
 * L + d (a pattern lists at most L nonzero vectors of the symmetric molecules
 * and one entry per distinguished molecule) */
void orc_sa_patterns(const orc_sa* s, int* tier, int* r, int* G, int* h, long long* var_off,
                     long long* cat_off, int* ids_padded) {
    int L = s->p.L + s->p.d;
    for (long long i = 0; i < s->P; ++i) {
        int ri = (int)(s->id_off[i + 1] - s->id_off[i]);
        if (tier) tier[i] = s->tier[i];
        if (r) r[i] = ri;
        if (G) G[i] = s->G[i];
        if (h) h[i] = s->h[i];
        if (var_off) var_off[i] = s->var_off[i];
        if (cat_off) cat_off[i] = s->cat_off[i];
        if (ids_padded)
            for (int a = 0; a < L; ++a)
                ids_padded[(size_t)i * L + a] = a < ri ? s->ids[s->id_off[i] + a] : -1;
    }
    if (var_off) var_off[s->P] = s->var_off[s->P];
    if (cat_off) cat_off[s->P] = s->cat_off[s->P];
}

void orc_sa_categories(const orc_sa* s, int* cat_id, long long* cat_M) {
    long long n = s->cat_off[s->P];
    if (cat_id) memcpy(cat_id, s->cat_id, sizeof(int) * n);
    if (cat_M) memcpy(cat_M, s->cat_M, sizeof(long long) * n);
}

/* label of every variable: pattern, kind, q, r (categories 1..G, 0 = unused) */
void orc_sa_var_labels(const orc_sa* s, long long* pat, int* kind, int* q, int* r) {
    for (long long i = 0; i < s->P; ++i) {
        int G = s->G[i];
        long long base = s->var_off[i];
        const int* tr = s->trank + s->cat_off[i];
        long long j;
#define SETL(idx, pp, kk, qq, rr) do { j = (idx); pat[j] = (pp); kind[j] = (kk); q[j] = (qq); r[j] = (rr); } while (0)
        SETL(base + var_local(G, K_Z, 0, 0, 0), i, K_Z, 0, 0);
        for (int a = 1; a <= G; ++a) {
            SETL(base + var_local(G, K_X, a, 0, 0), i, K_X, a, 0);
            SETL(base + var_local(G, K_Y, a, 0, 0), i, K_Y, a, 0);
            SETL(base + var_local(G, K_P, a, 0, 0), i, K_P, a, 0);
            for (int b = 1; b <= G; ++b)
                if (b != a) SETL(base + var_local(G, K_S, a, b, 0), i, K_S, a, b);
            if (tr[a - 1] >= 0) SETL(base + var_local(G, K_T, a, 0, tr[a - 1]), i, K_T, a, 0);
        }
#undef SETL
    }
}

/* ---- targets and the aligned accessor ------------------------------- */

/* Canonical target of pattern i when one molecule of category q (1..G)
 * changes its vector by dir*e_k (Eqs. raw-target-plus/minus and
 * canonical-target-plus/minus).  Returns the target pattern or -1. */
static long long target_pattern(const orc_sa* s, long long i, int q, int k, int dir) {
    int m = s->p.m;
    if (s->tcache) return s->tcache[((size_t)(s->cat_off[i] + q - 1) * m + k) * 2 + (dir > 0 ? 1 : 0)];
    int vq = s->cat_id[s->cat_off[i] + q - 1];
    int w = vec_shift(&s->vs, vq, k, dir);
    long long res = -1;
    if (w >= 0) {
        /* raw target as a multiset: drop one copy of vq (if nonzero), add w (if nonzero) */
        int r = (int)(s->id_off[i + 1] - s->id_off[i]);
        const int* ids = s->ids + s->id_off[i];
        int key[256]; int nk = 0; int dropped = (vq == 0);
        for (int a = 0; a < r; ++a) {
            if (!dropped && ids[a] == vq) { dropped = 1; continue; }
            key[nk++] = ids[a];
        }
        if (w != 0) {
            /* insert w keeping ids ascending */
            int pos = nk;
            while (pos > 0 && key[pos - 1] > w) { key[pos] = key[pos - 1]; --pos; }
            key[pos] = w; ++nk;
        }
        int tier = 0;
        for (int a = 0; a < nk; ++a) tier += s->vs.norm[key[a]];
        if (tier <= s->p.L && nk <= s->p.N) res = pat_find(s, key, nk, tier);
    }
    return res;
}

/* fill the optional target cache (serial; afterwards it is only read) */
static void fill_cache(orc_sa* s) {
    int m = s->p.m;
    long long co = s->cat_off[s->P];
    int* cache = s->tcache;
    s->tcache = NULL;               /* compute without reading the cache */
    for (long long i = 0; i < s->P; ++i)
        for (int q = 1; q <= s->G[i]; ++q)
            for (int k = 0; k < m; ++k)
                for (int d = 0; d < 2; ++d)
                    cache[((size_t)(s->cat_off[i] + q - 1) * m + k) * 2 + d] =
                        (int)target_pattern(s, i, q, k, d ? +1 : -1);
    (void)co;
    s->tcache = cache;
}

/* category (1..G) of pattern t whose vector is id v; 0 if absent */
static int cat_of_vector(const orc_sa* s, long long t, int v) {
    for (int q = 0; q < s->G[t]; ++q)
        if (s->cat_id[s->cat_off[t] + q] == v) return q + 1;
    return 0;
}

/*
 * Aligned accessor (Eq. aligned-accessor): entry <x|R^{[m]}_{Lambda'}|y> of
 * the raw target obtained from pattern i by moving one molecule of category
 * qm by dir*e_k.  The row and column are described by the categories of the
 * molecules they name in the SOURCE pattern:
 *   xr = 0 for the cavity, else the source category of the row molecule;
 *   yc likewise for the column;
 *   xmoved / ymoved: the row / column molecule is the moved molecule;
 *   same: row and column name the same molecule.
 * In the raw target the moved molecule carries w = v_qm + dir e_k and every
 * other molecule keeps its vector; the entry is the variable of Lambda'
 * selected by those vectors.  Returns the global variable index.
 */
static long long accessor(const orc_sa* s, long long i, int qm, int k, int dir,
                          int xr, int xmoved, int yc, int ymoved, int same) {
    long long t = target_pattern(s, i, qm, k, dir);
    if (t < 0) return -1;
    int vq = s->cat_id[s->cat_off[i] + qm - 1];
    int w = vec_shift(&s->vs, vq, k, dir);
    int a = 0, b = 0; /* categories in the target, 0 = cavity */
    if (xr > 0) a = cat_of_vector(s, t, xmoved ? w : s->cat_id[s->cat_off[i] + xr - 1]);
    if (yc > 0) b = cat_of_vector(s, t, ymoved ? w : s->cat_id[s->cat_off[i] + yc - 1]);
    if ((xr > 0 && a == 0) || (yc > 0 && b == 0)) {
#pragma omp atomic
        g_orc_errors++;
        return -1;
    }
    int G = s->G[t];
    const int* tr = s->trank + s->cat_off[t];
    long long loc;
    if (a == 0 && b == 0) loc = var_local(G, K_Z, 0, 0, 0);
    else if (b == 0) loc = var_local(G, K_X, a, 0, 0);
    else if (a == 0) loc = var_local(G, K_Y, b, 0, 0);
    else if (same) loc = var_local(G, K_P, a, 0, 0);
    else if (a != b) loc = var_local(G, K_S, a, b, 0);
    else loc = var_local(G, K_T, a, 0, tr[a - 1]);
    return s->var_off[t] + loc;
}

/* one hierarchy term of the derivative of a variable */
typedef struct { long long src; int k, n, dir, side; cplx coef; } hterm;

/*
 * All hierarchy terms of variable (kind, q, r) of pattern i, Eqs. uvar-up and
 * uvar-down generalised to channel k with c_k and c-check_k as in
 * Eq. scaled-HEOM.  side = 0: the row delta (molecule of the row category is
 * moved); side = 1: the column delta.  For P_q both deltas name the same
 * molecule, so both appear (their up terms cancel numerically).
 * Returns the number of terms written to out (at most 4 m).
 */
static int var_hterms(const orc_sa* s, long long i, int kind, int q, int r, hterm* out) {
    const orc_params* p = &s->p;
    int m = p->m, L = p->L;
    int chi = s->tier[i] < L ? 1 : 0;           /* Eq. hard-cutoff-factor */
    int row = 0, col = 0, same = 0;
    switch (kind) {
    case K_Z: return 0;                          /* no molecular row or column */
    case K_X: row = q; break;
    case K_Y: col = q; break;
    case K_P: row = q; col = q; same = 1; break;
    case K_S: row = q; col = r; break;
    case K_T: row = q; col = q; break;           /* two different molecules */
    }
    int nt = 0;
    for (int k = 0; k < m; ++k) {
        double ac = absck(p, k);
        if (row > 0) {
            int n = s->vs.comp[(size_t)s->cat_id[s->cat_off[i] + row - 1] * m + k];
            if (chi) {   /* -i sqrt((n+1)|c_k|) A+(e_i, b) */
                long long src = accessor(s, i, row, k, +1, row, 1, col, same, same);
                if (src >= 0) {
                    out[nt].src = src; out[nt].k = k; out[nt].n = n; out[nt].dir = +1; out[nt].side = 0;
                    out[nt].coef = -I * sqrt((double)(n + 1) * ac);
                    ++nt;
                }
            }
            if (n > 0) { /* -i sqrt(n/|c_k|) c_k A-(e_i, b) */
                long long src = accessor(s, i, row, k, -1, row, 1, col, same, same);
                if (src < 0) {
#pragma omp atomic
                    g_orc_errors++;
                    continue;
                }
                out[nt].src = src; out[nt].k = k; out[nt].n = n; out[nt].dir = -1; out[nt].side = 0;
                out[nt].coef = -I * sqrt((double)n / ac) * ck(p, k);
                ++nt;
            }
        }
        if (col > 0) {
            int n = s->vs.comp[(size_t)s->cat_id[s->cat_off[i] + col - 1] * m + k];
            if (chi) {   /* +i sqrt((n+1)|c_k|) A+(a, e_j) */
                long long src = accessor(s, i, col, k, +1, row, same, col, 1, same);
                if (src >= 0) {
                    out[nt].src = src; out[nt].k = k; out[nt].n = n; out[nt].dir = +1; out[nt].side = 1;
                    out[nt].coef = I * sqrt((double)(n + 1) * ac);
                    ++nt;
                }
            }
            if (n > 0) { /* +i sqrt(n/|c_k|) c-check_k A-(a, e_j) */
                long long src = accessor(s, i, col, k, -1, row, same, col, 1, same);
                if (src < 0) {
#pragma omp atomic
                    g_orc_errors++;
                    continue;
                }
                out[nt].src = src; out[nt].k = k; out[nt].n = n; out[nt].dir = -1; out[nt].side = 1;
                out[nt].coef = I * sqrt((double)n / ac) * cck(p, k);
                ++nt;
            }
        }
    }
    return nt;
}

static cplx ld(const double* x, long long j) { return x[2 * j] + I * x[2 * j + 1]; }

/* Grouped row sum R_q (Eq. grouped-row-sum) and column sum C_q
 * (Eq. grouped-column-sum) of pattern i. */
static cplx row_sum(const orc_sa* s, const double* x, long long i, int q) {
    int G = s->G[i];
    long long base = s->var_off[i];
    const long long* M = s->cat_M + s->cat_off[i];
    const int* tr = s->trank + s->cat_off[i];
    cplx acc = ld(x, base + var_local(G, K_P, q, 0, 0));
    if (M[q - 1] >= 2) acc += (double)(M[q - 1] - 1) * ld(x, base + var_local(G, K_T, q, 0, tr[q - 1]));
    for (int r = 1; r <= G; ++r)
        if (r != q) acc += (double)M[r - 1] * ld(x, base + var_local(G, K_S, q, r, 0));
    return acc;
}
static cplx col_sum(const orc_sa* s, const double* x, long long i, int q) {
    int G = s->G[i];
    long long base = s->var_off[i];
    const long long* M = s->cat_M + s->cat_off[i];
    const int* tr = s->trank + s->cat_off[i];
    cplx acc = ld(x, base + var_local(G, K_P, q, 0, 0));
    if (M[q - 1] >= 2) acc += (double)(M[q - 1] - 1) * ld(x, base + var_local(G, K_T, q, 0, tr[q - 1]));
    for (int r = 1; r <= G; ++r)
        if (r != q) acc += (double)M[r - 1] * ld(x, base + var_local(G, K_S, r, q, 0));
    return acc;
}

/* derivative of one variable of pattern i */
static cplx var_rhs(const orc_sa* s, const double* x, long long i, int kind, int q, int r) {
    const orc_params* p = &s->p;
    int G = s->G[i];
    long long base = s->var_off[i];
    const long long* M = s->cat_M + s->cat_off[i];
    const int* tr = s->trank + s->cat_off[i];
    double g = p->g, dlt = p->detuning, kap = p->kappa;
    cplx gam = s->gamma[i];
    long long self;
    switch (kind) {
    case K_Z: self = base + var_local(G, K_Z, 0, 0, 0); break;
    case K_X: self = base + var_local(G, K_X, q, 0, 0); break;
    case K_Y: self = base + var_local(G, K_Y, q, 0, 0); break;
    case K_P: self = base + var_local(G, K_P, q, 0, 0); break;
    case K_S: self = base + var_local(G, K_S, q, r, 0); break;
    default:  self = base + var_local(G, K_T, q, 0, tr[q - 1]); break;
    }
    cplx v = ld(x, self);
    cplx Z = ld(x, base + var_local(G, K_Z, 0, 0, 0));
    cplx d = 0;
    /* Hamiltonian + damping + loss.  Z and X are Eqs. HZ and HX; Y, P, S, T
     * follow from <a|H R - R H|b> with the same grouped sums. */
    switch (kind) {
    case K_Z: {
        cplx sum = 0;
        for (int a = 1; a <= G; ++a)
            sum += (double)M[a - 1] * (ld(x, base + var_local(G, K_X, a, 0, 0)) - ld(x, base + var_local(G, K_Y, a, 0, 0)));
        d = -I * g * sum - gam * v - kap * v;
        break;
    }
    case K_X:
        d = -I * dlt * v - I * g * (Z - row_sum(s, x, i, q)) - gam * v - 0.5 * kap * v;
        break;
    case K_Y:
        d = I * dlt * v - I * g * (col_sum(s, x, i, q) - Z) - gam * v - 0.5 * kap * v;
        break;
    case K_P:
    case K_T:
        d = -I * g * (ld(x, base + var_local(G, K_Y, q, 0, 0)) - ld(x, base + var_local(G, K_X, q, 0, 0))) - gam * v;
        break;
    case K_S:
        d = -I * g * (ld(x, base + var_local(G, K_Y, r, 0, 0)) - ld(x, base + var_local(G, K_X, q, 0, 0))) - gam * v;
        break;
    }
    (void)M;
    /* terminator: -Delta sum_i [Q_i, [Q_i, rho]] multiplies entry (a, b) by the
     * number of molecules i for which exactly one of a, b is e_i: 0 for Z and
     * P, 1 for X and Y, 2 for S and T */
    {
        int w = (kind == K_X || kind == K_Y) ? 1 : ((kind == K_S || kind == K_T) ? 2 : 0);
        d += -p->term * (double)w * v;
    }
    hterm ht[4 * ORC_MAXM];
    int nt = var_hterms(s, i, kind, q, r, ht);
    for (int t = 0; t < nt; ++t) d += ht[t].coef * ld(x, ht[t].src);
    return d;
}

/* pattern of a variable (binary search on var_off) */
static long long pat_of_var(const orc_sa* s, long long j) {
    long long lo = 0, hi = s->P - 1;
    while (lo < hi) {
        long long mid = (lo + hi + 1) / 2;
        if (s->var_off[mid] <= j) lo = mid; else hi = mid - 1;
    }
    return lo;
}

/* decode a local index into (kind, q, r) */
static void decode_local(const orc_sa* s, long long i, long long loc, int* kind, int* q, int* r) {
    int G = s->G[i];
    const int* tr = s->trank + s->cat_off[i];
    *q = 0; *r = 0;
    if (loc == 0) { *kind = K_Z; return; }
    if (loc <= G) { *kind = K_X; *q = (int)loc; return; }
    if (loc <= 2 * G) { *kind = K_Y; *q = (int)(loc - G); return; }
    if (loc <= 3 * G) { *kind = K_P; *q = (int)(loc - 2 * G); return; }
    if (loc < (long long)(G + 1) * (G + 1)) {
        long long sidx = loc - (3 * G + 1);
        int a = (int)(sidx / (G - 1)) + 1;
        int b = (int)(sidx % (G - 1)) + 1;
        if (b >= a) b += 1;
        *kind = K_S; *q = a; *r = b; return;
    }
    int t = (int)(loc - (long long)(G + 1) * (G + 1));
    for (int a = 1; a <= G; ++a)
        if (tr[a - 1] == t) { *kind = K_T; *q = a; return; }
    *kind = -1;
}

/* full right-hand side dx = M_u x (Eq. uvar-propagator) */
void orc_sa_rhs(const orc_sa* s, const double* x, double* dx) {
#pragma omp parallel for schedule(dynamic, 64)
    for (long long i = 0; i < s->P; ++i) {
        long long u = s->var_off[i + 1] - s->var_off[i];
        for (long long loc = 0; loc < u; ++loc) {
            int kind, q, r;
            decode_local(s, i, loc, &kind, &q, &r);
            cplx d = var_rhs(s, x, i, kind, q, r);
            dx[2 * (s->var_off[i] + loc)] = creal(d);
            dx[2 * (s->var_off[i] + loc) + 1] = cimag(d);
        }
    }
}

/* derivative at selected variables only (for sampled checks on large cases) */
void orc_sa_rhs_at(const orc_sa* s, const double* x, const long long* idx, long long n, double* out) {
#pragma omp parallel for schedule(dynamic, 16)
    for (long long t = 0; t < n; ++t) {
        long long j = idx[t];
        long long i = pat_of_var(s, j);
        int kind, q, r;
        decode_local(s, i, j - s->var_off[i], &kind, &q, &r);
        cplx d = var_rhs(s, x, i, kind, q, r);
        out[2 * t] = creal(d);
        out[2 * t + 1] = cimag(d);
    }
}

/* number of hierarchy terms over all variables (P up pairs included) */
long long orc_sa_num_terms(const orc_sa* s) {
    long long total = 0;
    for (long long i = 0; i < s->P; ++i) {
        long long u = s->var_off[i + 1] - s->var_off[i];
        for (long long loc = 0; loc < u; ++loc) {
            int kind, q, r;
            decode_local(s, i, loc, &kind, &q, &r);
            hterm ht[4 * ORC_MAXM];
            total += var_hterms(s, i, kind, q, r, ht);
        }
    }
    return total;
}

/* dump of all hierarchy terms: variable, source variable, channel k,
 * occupation n of the moved molecule before the move, dir (+1 raise,
 * -1 lower), side (0 row, 1 column) */
void orc_sa_terms(const orc_sa* s, long long* var, long long* src, int* k, int* n, int* dir, int* side) {
    long long t = 0;
    for (long long i = 0; i < s->P; ++i) {
        long long u = s->var_off[i + 1] - s->var_off[i];
        for (long long loc = 0; loc < u; ++loc) {
            int kind, q, r;
            decode_local(s, i, loc, &kind, &q, &r);
            hterm ht[4 * ORC_MAXM];
            int nt = var_hterms(s, i, kind, q, r, ht);
            for (int a = 0; a < nt; ++a, ++t) {
                var[t] = s->var_off[i] + loc; src[t] = ht[a].src; k[t] = ht[a].k;
                n[t] = ht[a].n; dir[t] = ht[a].dir; side[t] = ht[a].side;
            }
        }
    }
}

/* the coefficient of every hierarchy term, in the order of orc_sa_terms */
void orc_sa_term_coefs(const orc_sa* s, double* re, double* im) {
    long long t = 0;
    for (long long i = 0; i < s->P; ++i) {
        long long u = s->var_off[i + 1] - s->var_off[i];
        for (long long loc = 0; loc < u; ++loc) {
            int kind, q, r;
            decode_local(s, i, loc, &kind, &q, &r);
            hterm ht[4 * ORC_MAXM];
            int nt = var_hterms(s, i, kind, q, r, ht);
            for (int a = 0; a < nt; ++a, ++t) {
                re[t] = creal(ht[a].coef);
                im[t] = cimag(ht[a].coef);
            }
        }
    }
}

/* classical RK4 (the integrator named in Sec. V), in place */
void orc_sa_rk4(const orc_sa* s, double* x, double dt, long long nsteps) {
    long long n2 = 2 * s->nvar;
    double* k1 = (double*)malloc(sizeof(double) * n2);
    double* k2 = (double*)malloc(sizeof(double) * n2);
    double* k3 = (double*)malloc(sizeof(double) * n2);
    double* k4 = (double*)malloc(sizeof(double) * n2);
    double* t = (double*)malloc(sizeof(double) * n2);
    for (long long step = 0; step < nsteps; ++step) {
        orc_sa_rhs(s, x, k1);
        for (long long j = 0; j < n2; ++j) t[j] = x[j] + 0.5 * dt * k1[j];
        orc_sa_rhs(s, t, k2);
        for (long long j = 0; j < n2; ++j) t[j] = x[j] + 0.5 * dt * k2[j];
        orc_sa_rhs(s, t, k3);
        for (long long j = 0; j < n2; ++j) t[j] = x[j] + dt * k3[j];
        orc_sa_rhs(s, t, k4);
        for (long long j = 0; j < n2; ++j)
            x[j] = x[j] + dt / 6.0 * (k1[j] + 2.0 * k2[j] + 2.0 * k3[j] + k4[j]);
    }
    free(k1); free(k2); free(k3); free(k4); free(t);
}

/*
 * Observables from the physical representative (Eqs. trace-uvar, Pcav-uvar,
 * Pexc-uvar, PB-uvar, PD-uvar, Pplus-uvar, Pminus-uvar).  theta follows
 * tan(2 theta) = Omega_R / Delta with Delta = omega_cav - eps_x and
 * theta in [0, pi/2] (Eq. polariton-states).
 * out: Tr, P_cav, P_exc, P_B, P_D, P_+, P_-, Hermiticity defect of rho_S.
 */
void orc_sa_observables(const orc_sa* s, const double* x, double* out) {
    /* the physical density operator is the empty pattern (pattern 0): its
     * categories are the zero category, and with d = 1 also the
     * distinguished molecule's; rho_S entries follow from the variables and
     * the multiplicities (Eqs. trace-uvar .. Pminus-uvar, written over the
     * categories) */
    const orc_params* p = &s->p;
    int G = s->G[0];
    const long long* M = s->cat_M + s->cat_off[0];
    const int* tr = s->trank + s->cat_off[0];
    double N = (double)p->N;
    cplx Z = ld(x, var_local(G, K_Z, 0, 0, 0));
    cplx Pexc = 0, PBn = 0, XB = 0, YB = 0;
    double hd = fabs(cimag(Z));
    for (int q = 1; q <= G; ++q) {
        double Mq = (double)M[q - 1];
        cplx Xq = ld(x, var_local(G, K_X, q, 0, 0)), Yq = ld(x, var_local(G, K_Y, q, 0, 0));
        cplx Pq = ld(x, var_local(G, K_P, q, 0, 0));
        Pexc += Mq * Pq;
        PBn += Mq * Pq;
        XB += Mq * Xq;
        YB += Mq * Yq;
        if (fabs(cimag(Pq)) > hd) hd = fabs(cimag(Pq));
        if (cabs(Xq - conj(Yq)) > hd) hd = cabs(Xq - conj(Yq));
        if (M[q - 1] >= 2) {
            cplx Tq = ld(x, var_local(G, K_T, q, 0, tr[q - 1]));
            PBn += Mq * (Mq - 1.0) * Tq;
            if (fabs(cimag(Tq)) > hd) hd = fabs(cimag(Tq));
        }
        for (int r = 1; r <= G; ++r) {
            if (r == q) continue;
            cplx Sqr = ld(x, var_local(G, K_S, q, r, 0)), Srq = ld(x, var_local(G, K_S, r, q, 0));
            PBn += Mq * (double)M[r - 1] * Sqr;
            if (cabs(Sqr - conj(Srq)) > hd) hd = cabs(Sqr - conj(Srq));
        }
    }
    cplx PB = PBn / N;
    XB /= sqrt(N);
    YB /= sqrt(N);
    double omr = 2.0 * p->g * sqrt(N);
    double theta = 0.5 * atan2(omr, -p->detuning);
    double cs = cos(theta), sn = sin(theta);
    out[0] = creal(Z + Pexc);
    out[1] = creal(Z);
    out[2] = creal(Pexc);
    out[3] = creal(PB);
    out[4] = creal(Pexc - PB);
    out[5] = creal(Z * cs * cs + PB * sn * sn + sn * cs * (XB + YB));
    out[6] = creal(Z * sn * sn + PB * cs * cs - sn * cs * (XB + YB));
    out[7] = hd;
}

/* RK4 with observables every obs_every steps (row 0 = initial state) */
void orc_sa_propagate(const orc_sa* s, double* x, double dt, long long nsteps, long long obs_every, double* obs) {
    long long row = 0;
    if (obs) orc_sa_observables(s, x, obs + 8 * row++);
    for (long long done = 0; done < nsteps;) {
        long long chunk = obs_every > 0 ? obs_every : nsteps;
        if (chunk > nsteps - done) chunk = nsteps - done;
        orc_sa_rk4(s, x, dt, chunk);
        done += chunk;
        if (obs) orc_sa_observables(s, x, obs + 8 * row++);
    }
}

/* ====================================================================== */
/*  O-1: conventional scaled HEOM                                          */
/* ====================================================================== */

typedef struct {
    orc_params p;
    int N, D, nm;          /* molecules, D = N+1, label length N*m */
    long long nado;
    unsigned char* lab;    /* nado * nm, lexicographic order */
} orc_conv;

static int g_conv_nm;
static int conv_lab_cmp(const void* a, const void* b) { return memcmp(a, b, g_conv_nm); }

static void conv_gen(unsigned char* cur, int pos, int left, int nm, unsigned char** out, long long* n, long long* cap) {
    if (pos == nm) {
        if (*n >= *cap) { *cap = (*cap + 1) * 2; *out = (unsigned char*)realloc(*out, (size_t)*cap * nm); }
        memcpy(*out + (size_t)(*n) * nm, cur, nm);
        ++*n;
        return;
    }
    for (int v = 0; v <= left; ++v) {
        cur[pos] = (unsigned char)v;
        conv_gen(cur, pos + 1, left - v, nm, out, n, cap);
    }
}

orc_conv* orc_conv_create(const orc_params* p) {
    if (p->N < 1 || p->N > 16 || p->m < 1 || p->m > ORC_MAXM || p->L < 0) return NULL;
    for (int k = 0; k < p->m; ++k)
        if (!(absck(p, k) > 0.0)) return NULL;
    orc_conv* c = (orc_conv*)calloc(1, sizeof(orc_conv));
    c->p = *p;
    c->N = (int)p->N; c->D = c->N + 1; c->nm = c->N * p->m;
    unsigned char cur[256];
    long long cap = 0;
    conv_gen(cur, 0, p->L, c->nm, &c->lab, &c->nado, &cap);
    g_conv_nm = c->nm;
    qsort(c->lab, c->nado, c->nm, conv_lab_cmp);
    return c;
}

void orc_conv_destroy(orc_conv* c) { if (c) { free(c->lab); free(c); } }
long long orc_conv_num_ados(const orc_conv* c) { return c->nado; }
void orc_conv_labels(const orc_conv* c, unsigned char* out) { memcpy(out, c->lab, (size_t)c->nado * c->nm); }

static long long conv_find(const orc_conv* c, const unsigned char* lab) {
    g_conv_nm = c->nm;
    const unsigned char* f = (const unsigned char*)bsearch(lab, c->lab, c->nado, c->nm, conv_lab_cmp);
    return f ? (long long)((f - c->lab) / c->nm) : -1;
}

/* dense D x D products written out */
static void matmul(int D, const cplx* A, const cplx* B, cplx* C) {
    for (int a = 0; a < D; ++a)
        for (int b = 0; b < D; ++b) {
            cplx s = 0;
            for (int t = 0; t < D; ++t) s += A[a * D + t] * B[t * D + b];
            C[a * D + b] = s;
        }
}

/* Eq. scaled-HEOM plus the cavity-loss term, for every ADO */
void orc_conv_rhs(const orc_conv* c, const double* xin, double* dxout) {
    const orc_params* p = &c->p;
    int D = c->D, N = c->N, m = p->m, nm = c->nm;
    cplx* H = (cplx*)calloc((size_t)D * D, sizeof(cplx));
    cplx* Pc = (cplx*)calloc((size_t)D * D, sizeof(cplx));
    cplx* Q = (cplx*)calloc((size_t)N * D * D, sizeof(cplx));
    /* Eq. HS with omega_cav = 0 and eps_x = detuning */
    H[0] = 0.0;
    for (int i = 1; i <= N; ++i) {
        H[i * D + i] = p->detuning;
        H[0 * D + i] = p->g;
        H[i * D + 0] = p->g;
        Q[(size_t)(i - 1) * D * D + i * D + i] = 1.0;
    }
    Pc[0] = 1.0;
    const cplx* x = (const cplx*)xin;
    cplx* dx = (cplx*)dxout;
    cplx* t1 = (cplx*)malloc(sizeof(cplx) * D * D);
    cplx* t2 = (cplx*)malloc(sizeof(cplx) * D * D);
    unsigned char lab[256];
    for (long long a = 0; a < c->nado; ++a) {
        const unsigned char* n = c->lab + (size_t)a * nm;
        const cplx* rho = x + (size_t)a * D * D;
        cplx* d = dx + (size_t)a * D * D;
        int tier = 0;
        cplx gam = 0;
        for (int i = 0; i < N; ++i)
            for (int k = 0; k < m; ++k) { tier += n[i * m + k]; gam += (double)n[i * m + k] * nuk(p, k); }
        matmul(D, H, rho, t1);
        matmul(D, rho, H, t2);
        for (int e = 0; e < D * D; ++e) d[e] = -I * (t1[e] - t2[e]) - gam * rho[e];
        matmul(D, Pc, rho, t1);
        matmul(D, rho, Pc, t2);
        for (int e = 0; e < D * D; ++e) d[e] += -0.5 * p->kappa * (t1[e] + t2[e]);
        /* terminator: -Delta sum_i [Q_i, [Q_i, rho]], with the matrices */
        if (p->term != 0.0) {
            cplx* t3 = (cplx*)malloc(sizeof(cplx) * D * D);
            for (int i = 0; i < N; ++i) {
                const cplx* Qi = Q + (size_t)i * D * D;
                matmul(D, Qi, rho, t1);
                matmul(D, rho, Qi, t2);
                for (int e = 0; e < D * D; ++e) t3[e] = t1[e] - t2[e];
                matmul(D, Qi, t3, t1);
                matmul(D, t3, Qi, t2);
                for (int e = 0; e < D * D; ++e) d[e] += -p->term * (t1[e] - t2[e]);
            }
            free(t3);
        }
        for (int i = 0; i < N; ++i) {
            const cplx* Qi = Q + (size_t)i * D * D;
            for (int k = 0; k < m; ++k) {
                int nik = n[i * m + k];
                double ac = absck(p, k);
                if (tier < p->L) {
                    memcpy(lab, n, nm); lab[i * m + k] += 1;
                    long long b = conv_find(c, lab);
                    const cplx* rb = x + (size_t)b * D * D;
                    matmul(D, Qi, rb, t1);
                    matmul(D, rb, Qi, t2);
                    double cf = sqrt((double)(nik + 1) * ac);
                    for (int e = 0; e < D * D; ++e) d[e] += -I * cf * (t1[e] - t2[e]);
                }
                if (nik > 0) {
                    memcpy(lab, n, nm); lab[i * m + k] -= 1;
                    long long b = conv_find(c, lab);
                    const cplx* rb = x + (size_t)b * D * D;
                    matmul(D, Qi, rb, t1);
                    matmul(D, rb, Qi, t2);
                    double cf = sqrt((double)nik / ac);
                    for (int e = 0; e < D * D; ++e) d[e] += -I * cf * (ck(p, k) * t1[e] - cck(p, k) * t2[e]);
                }
            }
        }
    }
    free(H); free(Pc); free(Q); free(t1); free(t2);
}

void orc_conv_rk4(const orc_conv* c, double* x, double dt, long long nsteps) {
    long long n2 = 2 * c->nado * c->D * c->D;
    double* k1 = (double*)malloc(sizeof(double) * n2);
    double* k2 = (double*)malloc(sizeof(double) * n2);
    double* k3 = (double*)malloc(sizeof(double) * n2);
    double* k4 = (double*)malloc(sizeof(double) * n2);
    double* t = (double*)malloc(sizeof(double) * n2);
    for (long long step = 0; step < nsteps; ++step) {
        orc_conv_rhs(c, x, k1);
        for (long long j = 0; j < n2; ++j) t[j] = x[j] + 0.5 * dt * k1[j];
        orc_conv_rhs(c, t, k2);
        for (long long j = 0; j < n2; ++j) t[j] = x[j] + 0.5 * dt * k2[j];
        orc_conv_rhs(c, t, k3);
        for (long long j = 0; j < n2; ++j) t[j] = x[j] + dt * k3[j];
        orc_conv_rhs(c, t, k4);
        for (long long j = 0; j < n2; ++j)
            x[j] = x[j] + dt / 6.0 * (k1[j] + 2.0 * k2[j] + 2.0 * k3[j] + k4[j]);
    }
    free(k1); free(k2); free(k3); free(k4); free(t);
}

/*
 * For every entry (a, b) of every conventional ADO, the symmetry-adapted
 * variable that holds it: canonicalise the label (sort the molecules' local
 * vectors, Eq. pattern-one; with d = 1 molecule 1 keeps its own category),
 * then name the entry by the categories of the molecules in its row and
 * column (Eqs. Z-variable .. T-variable).
 * map has nado * (N+1)^2 entries; -1 if the canonical pattern is missing.
 */
void orc_conv_to_sa(const orc_conv* c, const orc_sa* s, long long* map) {
    int N = c->N, D = c->D, m = c->p.m, nm = c->nm;
    int vid[64], key[64];
    for (long long a = 0; a < c->nado; ++a) {
        const unsigned char* n = c->lab + (size_t)a * nm;
        int nk = 0, tier = 0;
        for (int i = 0; i < N; ++i) {
            vid[i] = s->vs.lut[vec_code(n + i * m, m, s->p.L)];
            /* molecules 1..d are the distinguished ones: their own ids */
            if (i < s->p.d) vid[i] += (i + 1) * s->vs.V;
            if (vid[i] > 0) { key[nk++] = vid[i]; tier += s->vs.norm[vid[i]]; }
        }
        /* insertion sort: ascending id = vectors in canonical order */
        for (int x = 1; x < nk; ++x) {
            int v = key[x], y = x;
            while (y > 0 && key[y - 1] > v) { key[y] = key[y - 1]; --y; }
            key[y] = v;
        }
        long long t = pat_find(s, key, nk, tier);
        for (int ra = 0; ra < D; ++ra)
            for (int cb = 0; cb < D; ++cb) {
                long long* out = map + (size_t)a * D * D + ra * D + cb;
                if (t < 0) { *out = -1; continue; }
                int qa = ra == 0 ? 0 : cat_of_vector(s, t, vid[ra - 1]);
                int qb = cb == 0 ? 0 : cat_of_vector(s, t, vid[cb - 1]);
                int G = s->G[t];
                const int* tr = s->trank + s->cat_off[t];
                long long loc;
                if (qa == 0 && qb == 0) loc = var_local(G, K_Z, 0, 0, 0);
                else if (qb == 0) loc = var_local(G, K_X, qa, 0, 0);
                else if (qa == 0) loc = var_local(G, K_Y, qb, 0, 0);
                else if (ra == cb) loc = var_local(G, K_P, qa, 0, 0);
                else if (qa != qb) loc = var_local(G, K_S, qa, qb, 0);
                else loc = var_local(G, K_T, qa, 0, tr[qa - 1]);
                *out = s->var_off[t] + loc;
            }
    }
}
