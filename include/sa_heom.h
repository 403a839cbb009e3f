/*
 * sa_heom.h -- C ABI of the B300 (sm_103a) symmetry-adapted HEOM library.
 *
 * The library propagates the symmetry-adapted hierarchical equations of
 * motion of Mondal & Huo (arXiv 2608.20657) for the Holstein-Tavis-Cummings
 * model (N identical two-level molecules, one cavity mode, single-excitation
 * manifold, Eq. HS), with independent identical local baths decomposed into
 * m exponentials (Eq. BCF-exp) and hierarchy depth L (Eq. scaled-HEOM with a
 * hard cutoff).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Return value: 0 (SA_OK) on success, a negative SA_ERR_* code otherwise.
 *    No exception, abort or exit crosses this boundary.  sa_heom_strerror()
 *    names a code; sa_heom_last_error() gives a one-line detail of the most
 *    recent failure on the calling thread.
 *  - Handles are not thread-safe: one thread uses a handle at a time.
 *  - A device-built handle belongs to the device that was current when it
 *    was built; every entry point that touches the device returns
 *    SA_ERR_STATE, before any launch, when another device is current.
 *  - "stream" arguments are cudaStream_t values passed as void*; NULL is the
 *    legacy default stream.  Device pointers are plain CUDA device addresses
 *    (for instance a torch tensor's data_ptr()); the library never frees
 *    memory it did not allocate.
 *  - Complex numbers are interleaved (re, im) pairs: double2 for SA_FP64,
 *    float2 for the auxiliary variables of SA_FP32_AUX.
 *  - State layout ("canonical layout"): instances one after another; inside
 *    an instance the canonical patterns in the order tier ascending, then
 *    their local-vector lists compared lexicographically with larger vectors
 *    first (vectors ordered by |alpha| descending, then components
 *    lexicographically descending).  Inside a pattern with G occupation
 *    categories (distinct nonzero vectors in pattern order, then the zero
 *    category when M_0 = N - r >= 1) the (G+1)^2 + h unique variables of
 *    Eq. uvar-count are stored as
 *        Z; X_1..X_G; Y_1..Y_G; P_1..P_G; S_{q,r} (q = 1..G, r != q,
 *        row major); T_q for the categories with M_q >= 2, in order.
 *    The physical density operator is the first pattern of each instance
 *    (Z, X_0, Y_0, P_0[, T_0], Sec. IV.C).
 *  - State buffers (d_state, d_x, d_dx) must be 16-byte aligned (cudaMalloc
 *    and torch allocations are); the entry points that run the stage
 *    kernels return INVALID_ARG otherwise.
 *  - SA_FP64 state buffers hold double2[n_vars_total] padded to 256 bytes.
 *    SA_FP32_AUX state buffers hold float2[n_vars_total], padded to 256
 *    bytes, followed by double2[32 * n_instances]: slot 32*i + j holds
 *    variable j of instance i's physical representative in FP64; the float2
 *    copy of those variables mirrors it for readers in FP32.
 *  - Device state layout: the canonical layout, unless the handle was built
 *    with SA_BUILD_PACK_INSTANCES.  Such a handle stores the instances of
 *    every template (instances whose tables are identical: same m, L, d,
 *    decay rates and hierarchy structure) that has at least 16 members in
 *    packs of up to 32 instances (a remainder under 16 stays unpacked),
 *    interleaved: variable l of the pack's lane j lies at element
 *    base + l * n + j (n the pack's lanes); other instances are contiguous.  sa_heom_state_index gives every variable's
 *    element.  The host arrays of sa_heom_state_upload / _download and the
 *    observables stay canonical; a packed device state is meant to be
 *    written and read through them (and sa_heom_init_*), and a checkpoint
 *    records the layout in its hash.
 */
#ifndef SA_HEOM_H
#define SA_HEOM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SA_HEOM_MAXM 8  /* exponentials per local bath (static channel included) */
#define SA_HEOM_MAXD 3  /* distinguished molecules */
#define SA_HEOM_PHYS_SLOTS 32 /* complex values per instance in sa_heom_init_physical */
#define SA_HEOM_MAXL 30 /* hierarchy depth */

enum {
    SA_OK = 0,
    SA_ERR_INVALID_ARG = -1, /* N < 1, m outside 1..8, L outside 0..30, d outside 0..min(3, N), |c_k| = 0,
                                non-finite input */
    SA_ERR_UNSUPPORTED = -2, /* size beyond the 32-bit table indices, missing device */
    SA_ERR_OOM = -3,         /* host or device allocation failed */
    SA_ERR_CUDA = -4,        /* a CUDA runtime call failed; see sa_heom_last_error() */
    SA_ERR_TIMEOUT = -5,     /* a bounded device wait expired (sa_heom_device_error says what is
                                then undefined) */
    SA_ERR_NUMERIC = -6,     /* NaN or Inf in the observables */
    SA_ERR_STATE = -7        /* handle built host-only, another device current, or wrong call order */
};

enum { SA_FP64 = 0, SA_FP32_AUX = 1 };                  /* precision */
enum { SA_BUILD_DEVICE = 0, SA_BUILD_HOST_ONLY = 1 };   /* build flags */
enum { SA_BUILD_PACK_INSTANCES = 4 };  /* build flag: interleave the instances of repeated templates (see above) */
enum { SA_BUILD_ADJOINT_REPS = 2 };  /* sa_heom_build_representatives: the adjoint shortcut */
enum { SA_BATH_HIGH_T = 0, SA_BATH_MATSUBARA = 1, SA_BATH_PADE = 2 };

/*
 * One HTC + bath instance.  Units: any energy unit with hbar = 1.
 *   N          molecules (1 .. 2^62); only multiplicities depend on it.
 *   m, L       exponentials per local bath, hierarchy depth (Eq. n-label).
 *   detuning   eps_x - omega_cav (the propagated frame has omega_cav = 0).
 *   g          single-molecule coupling of Eq. HS (collective g*sqrt(N)).
 *   kappa      photon population decay rate: -kappa/2 {|c><c|, .} on every
 *              ADO (Lindblad on the cavity mode restricted to the manifold).
 *   c, cc, nu  c_k, c-check_k, nu_k of Eq. BCF-exp, k < m.
 *   term       terminator strength Delta (0: off): the bath terms left out of
 *              the expansion taken as white noise (the Ishizaki-Tanimura
 *              treatment Sec. V names), -Delta sum_i [Q_i, [Q_i, .]] on every
 *              ADO, i.e. -Delta w V per unique variable with w = 0 for Z and
 *              P, 1 for X and Y, 2 for S and T.  sa_bath_terminator gives
 *              Delta for the Matsubara scheme.
 *   d          distinguished molecules, 0 .. min(SA_HEOM_MAXD, N)
 *              (Eq. N-symmetric-pool).  Molecules 1..d are kept out of the
 *              permutation symmetry (Sec. V.F: the localised state
 *              |e_1><e_1| and cavity-site superpositions need d = 1): the
 *              local vector v of molecule j is stored with the pattern as
 *              vector id j V + v (V = n_vectors), so each forms a category of
 *              its own with M = 1, listed after the other nonzero vectors in
 *              molecule order and before the zero category (M = N - r, r
 *              counting the distinguished entries).  The other N - d
 *              molecules are symmetrised as with d = 0.  Set the initial
 *              state with sa_heom_init_physical.
 *   reserved   must be 0.
 */
typedef struct sa_params {
    int64_t N;
    int32_t m;
    int32_t L;
    double detuning;
    double g;
    double kappa;
    double c_re[SA_HEOM_MAXM], c_im[SA_HEOM_MAXM];
    double cc_re[SA_HEOM_MAXM], cc_im[SA_HEOM_MAXM];
    double nu_re[SA_HEOM_MAXM], nu_im[SA_HEOM_MAXM];
    double term;
    int32_t d;
    int32_t reserved;
} sa_params;

/* Sizes of one instance or of a whole batch. */
typedef struct sa_counts {
    double log10_conventional_ados; /* log10 C(Nm+L, L), Eq. direct-ado-count */
    int64_t n_vectors;              /* local vectors incl. the zero vector */
    int64_t n_patterns;             /* canonical representatives, Eq. canonical-count-one */
    int64_t n_vars;                 /* unique complex variables, Eq. Du-one */
    int64_t n_categories;           /* sum over patterns of G */
    int64_t n_records;              /* hierarchy connection records (pattern, category, k, +/-) */
    int64_t n_terms;                /* per-variable hierarchy terms the records expand to */
    int64_t state_bytes;            /* one state vector at the handle's precision */
    uint64_t conventional_ados;     /* C(Nm+L, L) exactly when it is below 2^64, else 0
                                       (batch: the largest instance's, 0 if any overflows) */
} sa_counts;

typedef struct sa_heom sa_heom;

/*
 * sa_bath_drude_lorentz -- fill m, c, cc, nu of *p for the Drude-Lorentz
 * density J(w) = 2 lambda gamma w / (w^2 + gamma^2) (Eq. Drude_Lorentz) in
 * Eq. BCF-spectral, decomposed as Eq. BCF-exp:
 *   SA_BATH_HIGH_T:    one term, c_0 = 2 lambda kT - i lambda gamma, nu_0 = gamma
 *                      (n_poles ignored);
 *   SA_BATH_MATSUBARA: gamma pole with cot(beta gamma/2) plus n_poles
 *                      Matsubara poles nu_j = 2 pi j kT;
 *   SA_BATH_PADE:      gamma pole plus n_poles poles of the [K-1/K] Pade
 *                      approximant in x^2 of (coth x - 1/x)/x (K = n_poles);
 *   sigma > 0 appends the static-disorder channel c = cc = sigma^2, nu = 0
 *   (Eq. C_static).  Real rates give cc_k = conj(c_k) (text below Eq. BCF-exp).
 * Other fields of *p are left untouched.  Errors: INVALID_ARG (non-positive
 * lambda, gamma or kT, negative sigma, too many terms, n_poles > 12 for Pade).
 */
/*
 * sa_bath_terminator -- *out = Delta for a Drude-Lorentz bath kept to
 * n_matsubara Matsubara poles (SA_BATH_MATSUBARA): the sum over the omitted
 * poles j > n_matsubara of c_j / nu_j, from the closed form of the full sum,
 * lambda (2 kT / gamma - cot(gamma / (2 kT))), less the kept ones.  Errors:
 * INVALID_ARG (non-positive lambda, gamma or kT, n_matsubara < 0, a pole on
 * gamma).
 */
int sa_bath_terminator(double lambda, double gamma, double kT, int n_matsubara, double* out);

int sa_bath_drude_lorentz(double lambda, double gamma, double kT, int scheme, int n_poles,
                          double sigma, sa_params* p);

/*
 * sa_heom_counts -- sizes of one instance without touching a device
 * (canonical patterns of Eq. pattern-one, unique variables of Eq. uvar-count,
 * connection records).  Pure host; builds the tables and drops them.
 */
int sa_heom_counts(const sa_params* p, sa_counts* out);

/*
 * sa_heom_build -- build the canonical patterns, categories, multiplicities
 * (Eqs. Mq, M0), variable layout and the precomputed hierarchy connections
 * (raw -> canonical targets with the aligned-target accessor resolved,
 * Eqs. canonical-target-plus/minus, aligned-accessor, uvar-up, uvar-down) of
 * `count` instances and, unless flags = SA_BUILD_HOST_ONLY, upload them to the
 * current CUDA device and allocate the RK4 work buffers (two stage vectors
 * and one accumulator, library-owned).  precision: SA_FP64 or SA_FP32_AUX.
 * The handle owns everything it allocates until sa_heom_destroy.
 * flags: SA_BUILD_HOST_ONLY (tables on the host only, for the dumps), and
 * SA_BUILD_PACK_INSTANCES (the packed device layout described at the top;
 * the list kernel's launch then evaluates one template item for all lanes
 * of a pack at once, followed in the same launch by the list units of the
 * unpacked instances, and sa_heom_set_kernel accepts SA_KERNEL_LISTS only).
 * Errors: INVALID_ARG (unknown flag too), UNSUPPORTED (more than 2^32 - 1
 * variables or records), OOM, CUDA.
 */
int sa_heom_build(const sa_params* params, int count, int precision, int flags, sa_heom** out);

/* sa_heom_destroy -- free the handle and everything it owns; NULL is a no-op. */
void sa_heom_destroy(sa_heom* h);

/* sa_heom_info -- totals of the batch (inst = -1) or of instance inst. */
int sa_heom_info(const sa_heom* h, int inst, sa_counts* out);

/* sa_heom_var_offset -- first variable of instance inst in the batch vector
 * (canonical layout: the host arrays of upload, download and the dumps). */
int sa_heom_var_offset(const sa_heom* h, int inst, int64_t* out);

/*
 * sa_heom_state_index -- the element of a device state buffer (index into
 * its double2 or float2 array) that holds variable `var` (canonical,
 * instance-relative) of instance `inst`: var_offset + var unless the handle
 * packs instances.  Pure host.  INVALID_ARG for an index out of range.
 */
int sa_heom_state_index(const sa_heom* h, int inst, int64_t var, int64_t* out);

/*
 * sa_heom_dump_packs -- the packs of a handle built with
 * SA_BUILD_PACK_INSTANCES (none otherwise) and, after
 * sa_heom_set_kernel(h, SA_KERNEL_LISTS) on a host-only handle, the table
 * blobs of the pack items.  sizes[0..2] <- packs, pack lanes, blob bytes.
 *   packs  uint32[4 * packs]: base element, lanes n, first element of the
 *          interleaved coefficient tables (slot s of lane j at
 *          cbase + s * n + j, slots as in sa_heom_dump_lists), first lane;
 *   lanes  uint32[pack lanes]: the instance of every lane (first lane + j);
 *   blobs  uint8[blob bytes]: every work item's table blob, at 16 times
 *          its blob field (sa_heom_dump_lists items).  A pack item's blob
 *          holds, each section starting on a 16-byte boundary after a
 *          16-byte header (u32 nw, the number of weights; the rest
 *          reserved): per pattern (var_rel u16, cat_rel u16, G u8, tier u8,
 *          0 u16); per pattern -Gamma_Lambda (re, im) in the handle's
 *          auxiliary precision; per category the multiplicity in that
 *          precision (-r for the zero category, whose M_0 = N - r); per
 *          variable the pack kernel updates a 16-byte record, in three
 *          phases (P, T, S; X, Y; Z): x = operand codes a | b << 11 of
 *          -i g (op[a] - op[b]) | diagonal class << 22 | pattern << 25,
 *          y = item-local variable | first term << 10 | term count << 26,
 *          z, w = grouped-sum contributions, each sum slot | weight index
 *          << 11 (operand codes and slots: below nv an item variable, then
 *          R and C per category, Z per pattern, zero); per term the
 *          instance-relative target (u32), then per term the coefficient
 *          slot (u16); then the nw distinct weights a + b N as int32 pairs
 *          (a, b), N the lane's molecule count.
 */
int sa_heom_dump_packs(const sa_heom* h, int64_t* sizes, uint32_t* packs, uint32_t* lanes, uint8_t* blobs);

/*
 * Table dumps of instance inst (host copies, canonical order), for checking
 * the builder against an independent implementation:
 *   sa_heom_dump_vectors:   comp[n_vectors * m] local vectors (id 0 = zero).
 *   sa_heom_dump_patterns:  per pattern tier, r (entries of its id list:
 *                           nonzero vectors of the symmetric molecules plus
 *                           one per distinguished molecule), G, h,
 *                           var_off (n_patterns + 1, instance-relative),
 *                           cat_off (n_patterns + 1), ids[n_patterns * (L + d)]
 *                           (vector ids padded with -1).
 *   sa_heom_dump_categories: vector id and multiplicity M_q of each category.
 *   sa_heom_dump_terms:     the per-variable hierarchy terms the records
 *                           expand to: variable, source variable (both
 *                           instance-relative), channel k, occupation n of
 *                           the moved molecule before the move, dir (+1
 *                           raise, -1 lower), side (0: row delta, 1: column
 *                           delta of Eq. projector-commutator-element).  The
 *                           exactly cancelling raise pair of P_q is omitted.
 * Array sizes come from sa_heom_info.  Pointers may be NULL to skip a field.
 */
int sa_heom_dump_vectors(const sa_heom* h, int inst, uint8_t* comp);
int sa_heom_dump_patterns(const sa_heom* h, int inst, int32_t* tier, int32_t* r, int32_t* G, int32_t* hcount,
                          int64_t* var_off, int64_t* cat_off, int32_t* ids);
int sa_heom_dump_categories(const sa_heom* h, int inst, int32_t* vec_id, int64_t* mult);
int sa_heom_dump_terms(const sa_heom* h, int inst, int64_t* var, int64_t* src, int32_t* k, int32_t* n,
                       int32_t* dir, int32_t* side);

/*
 * sa_heom_dump_coefficients -- the FP64 coefficients of the hierarchy terms
 * of instance `inst` (Eqs. uvar-up, uvar-down with c_k, c-check_k of Eq.
 * scaled-HEOM), as the host tables hold them.  row and col receive
 * 2 * SA_HEOM_MAXM * 32 * 2 doubles each: the (re, im) pair of coefficient
 * id ((k * 32) + n) * 2 + raise, n the moved molecule's occupation in
 * channel k before the move (0 .. L; 32 slots per channel), raise 1 for
 * n -> n + 1 and 0 for n -> n - 1:
 *   raise:  row -i sqrt((n + 1) |c_k|),  column +i sqrt((n + 1) |c_k|);
 *   lower:  row -i sqrt(n / |c_k|) c_k,  column +i sqrt(n / |c_k|) c-check_k;
 * with |c_k| = sqrt(Re c_k^2 + Im c_k^2); unused ids are zero.  Pure host.
 */
int sa_heom_dump_coefficients(const sa_heom* h, int inst, double* row, double* col);

/*
 * sa_heom_dump_lists -- the host copy of the SA_KERNEL_LISTS tables for the
 * current tuning (handles built with SA_BUILD_HOST_ONLY after
 * sa_heom_set_kernel(h, SA_KERNEL_LISTS); device handles keep them on the
 * device only and get STATE).  Instances whose tables are identical (same
 * m, L, d, decay rates and hierarchy structure -- e.g. every instance with
 * N >= L + d + 2 of one (m, L)) share one template: its work items and lists
 * are built once, for the first such instance, with targets and coefficient
 * slots relative to the instance, and a work unit pairs a template item with
 * an instance.  sizes[0..4] <- template items, rounds of 32 lanes, term rows,
 * lane slots (32 per round), work units.  Each non-NULL array receives:
 *   items  uint32[10 * items]: first pattern, patterns, first variable v0,
 *          variables, first category (relative to the template's
 *          representative instance), categories, first round r0, lane
 *          variables nl, blob offset (16-byte units) and blob bytes of
 *          every template item; a pack item (packed handles) has
 *          r0 = 0xffffffff and its hierarchy-term count in nl;
 *   units  uint32[2 * units]: template item, instance; the instances of a
 *          template one after another, each instance's items in order.  A
 *          pack unit has bit 31 set on the item and a pack in place of the
 *          instance;
 *   lvd    uint32[lane slots]: at 32 r0 + i, lane position i < nl of the
 *          item, l | a << 10 | b << 21 (item-local variable l; operand-area
 *          indices a, b of the term -i g (op[a] - op[b]));
 *   lvj    uint8[lane slots]: at 32 r0 + i, j | class << 5 (pattern j of the
 *          item; diagonal class 0: S T, 1: X, 2: Y, 3: Z, 4: P);
 *   rbase  uint32[rounds + 1]: first term row of every round;
 *   tidx   uint32[32 * rows], tcid uint16[32 * rows]: entry 32 * row + lane
 *          = target variable relative to the instance's first variable and
 *          coefficient slot in the instance's coefficient table.  Every
 *          instance holds 2 + 6 m (L + 1) slots (the last unused), the
 *          instances' tables one after another: slot 0 is zero (padding),
 *          then for channel k, occupation n = 0..L before the move and
 *          direction (lower, raise) the row, column and row + column (the
 *          P_q lower terms) coefficients at 1 + 3 ((k (L + 1) + n) 2 + raise)
 *          + side;
 *   opz    int32[4]: operand-area offsets of R_q, C_q, the Z sums, the zero
 *          (the item's stage-input slice occupies [0, chunk)).
 */
int sa_heom_dump_lists(const sa_heom* h, int64_t* sizes, uint32_t* items, uint32_t* units, uint32_t* lvd,
                       uint8_t* lvj, uint32_t* rbase, uint32_t* tidx, uint16_t* tcid, int32_t* opz);

/*
 * sa_heom_dump_ell -- the host copy of the SA_KERNEL_ELL tables (host-only
 * handles after sa_heom_set_kernel(h, SA_KERNEL_ELL); STATE otherwise).
 * sizes[0..2] <- warps W = ceil(variables / 32), term rows, variables.
 *   wpat   uint32[W]: first pattern (batch index) of warp w's variables
 *          32 w .. 32 w + 31;
 *   vword  uint32[variables]: pattern offset from wpat (5 bits) | kind << 5
 *          (0..5: Z X Y P S T) | q << 8 | r << 13 | T-rank of q << 18
 *          (31: none);
 *   rbase  uint32[W + 1]: first term row of every warp;
 *   tidx   uint32[32 * rows], tcid uint16[32 * rows]: entry 32 * row + lane
 *          = batch-global target variable and coefficient slot in the
 *          variable's own instance's table (layout as in sa_heom_dump_lists;
 *          0 = zero slot, padding).
 */
int sa_heom_dump_ell(const sa_heom* h, int64_t* sizes, uint32_t* wpat, uint32_t* vword, uint32_t* rbase,
                     uint32_t* tidx, uint16_t* tcid);

/* sa_heom_state_bytes -- bytes of one state vector of the whole batch. */
int sa_heom_state_bytes(const sa_heom* h, size_t* bytes);

/*
 * sa_heom_initial_vars -- the physical representative's variables of a
 * factorised initial state, in the canonical layout sa_heom_init_physical
 * takes (for d = 0 the first 10 doubles are also the rho0 of
 * sa_heom_init_state).  Uses p->N, p->g, p->detuning and p->d (0 or 1).
 *   SA_INIT_CAVITY      |c><c|                      (Eq. cavity-initial-uvar)
 *   SA_INIT_BRIGHT      |B><B|, B = sum_i e_i / sqrt N (Eq. bright-initial-uvar)
 *   SA_INIT_UP, _LP     upper / lower polariton cos(theta)|c> +/- ... with
 *                       tan 2 theta = Omega_R / Delta, Omega_R = 2 g sqrt N,
 *                       Delta = omega_cav - eps_x, theta in [0, pi/2]
 *                       (Eqs. upper-/lower-polariton-initial)
 *   SA_INIT_RANDOM      a random permutation-invariant density matrix from
 *                       draws[0..8]: a 2 x 2 complex matrix A (row-major
 *                       (re, im) pairs) and a dark weight w in [0, 1): the
 *                       cavity-bright block is (1 - w) A A^+ / tr(A A^+), the
 *                       dark block the eigenvalue w / (N - 1) (w ignored at
 *                       N = 1)
 *   SA_INIT_LOCALISED   |e_1><e_1| (d = 1 only; Sec. V.F)
 *   SA_INIT_SUPERPOSED  sqrt(0.3)|e_1> + sqrt(0.7)|c> (d = 1 only; Sec. V.F)
 * out receives *count (re, im) pairs: d = 0: Z, X_0, Y_0, P_0, T_0 (4 for
 * N = 1); d = 1 (categories 1 = molecule 1, 2 = the others): Z, X_1, X_2,
 * Y_1, Y_2, P_1, P_2, S_12, S_21, T_2 (9 for N = 2; Z, X_1, Y_1, P_1 for
 * N = 1).  out needs room for 20 doubles.  Pure host.
 *
 * sa_unit_cm_to_rad_fs, sa_unit_kT_rad_fs -- the unit set of Sec. V with
 * hbar = 1: an energy E in cm^-1 is the angular frequency 2 pi c E in
 * rad/fs, and k_B T (T in K) likewise, from the exact SI c, h and k_B.
 */
enum { SA_INIT_CAVITY = 0, SA_INIT_BRIGHT = 1, SA_INIT_UP = 2, SA_INIT_LP = 3, SA_INIT_RANDOM = 4,
       SA_INIT_LOCALISED = 5, SA_INIT_SUPERPOSED = 6 };
int sa_heom_initial_vars(const sa_params* p, int kind, const double* draws, double* out, int* count);
int sa_unit_cm_to_rad_fs(double e_cm, double* out);
int sa_unit_kT_rad_fs(double T_K, double* out);

/*
 * sa_heom_init_state -- factorised initial hierarchy/*
 * sa_heom_init_state -- factorised initial hierarchy (Eqs. factorized-
 * initial-zero/higher): every ADO zero except the physical representative,
 * set per instance from rho0[10 * i ..]: Z, X_0, Y_0, P_0, T_0 as (re, im)
 * pairs (T_0 ignored for N = 1).  d_state: caller-owned device buffer of
 * sa_heom_state_bytes bytes.  SA_ERR_INVALID_ARG for a batch with a d >= 1
 * instance.  Asynchronous on `stream`.
 */
int sa_heom_init_state(const sa_heom* h, const double* rho0, void* d_state, void* stream);

/*
 * sa_heom_init_physical -- the same factorised initial hierarchy with the
 * physical representative (the tier-0 pattern, whose variables are rho_S
 * written over its categories) given variable by variable in the canonical
 * layout: Z, X_1..X_G, Y_1..Y_G, P_1..P_G, S_{q,r} row-major (r != q), then
 * T.  phys[2 * SA_HEOM_PHYS_SLOTS * i ..] holds instance i's values as
 * (re, im) pairs; only the first n of them are read, n = the pattern's
 * variable count: (G + 1)^2 + h with G = d + 1 categories for N > d
 * (molecules 1..d, then the other N - d), h = 1 for N - d >= 2 -- 5 for
 * d = 0, 10 for d = 1, 17 for d = 2, 26 for d = 3.  Needed for d >= 1
 * (sa_heom_init_state returns SA_ERR_INVALID_ARG for such instances); valid
 * for every instance.
 * The values are not checked for Hermiticity.  Asynchronous on `stream`.
 */
int sa_heom_init_physical(const sa_heom* h, const double* phys, void* d_state, void* stream);

/*
 * Arbitrary initial operators (Sec. IV, Eqs. Gt-linearity, Gt-covariance,
 * reconstruct-ec, reconstruct-ee; Table tab:representative-initial-
 * operators).  rho_S(t) of any initial operator A in the single-excitation
 * manifold is a weighted sum of relabelled responses to five representative
 * operators, each propagated in its own reduced hierarchy.
 *
 *   sa_heom_build_representatives: a batch handle of the representatives of
 *     one d = 0 parameter set *p (d must be 0): instance 0 |c><c| (d = 0),
 *     1 |e_1><c|, 2 |c><e_1|, 3 |e_1><e_1| (d = 1), 4 |e_1><e_2| (d = 2,
 *     only for N >= 2).  Same precision and flags as sa_heom_build; the
 *     handle takes every sa_heom_* call.  With flags | SA_BUILD_ADJOINT_REPS
 *     the |c><e_1| propagation is left out (instances 0 |c><c|, 1 |e_1><c|,
 *     2 |e_1><e_1|, 3 |e_1><e_2|: a fifth fewer variables) and its response
 *     is taken as the adjoint of the |e_1><c| response (Eq. adjoint-
 *     preservation).  That holds when the propagator maps adjoints to
 *     adjoints, which needs every nu_k real and c-check_k = conj(c_k)
 *     exactly; other baths get SA_ERR_INVALID_ARG.
 *   sa_heom_init_representatives: the factorised initial state of each
 *     instance with its unit operator.  Asynchronous on `stream`.
 *   sa_heom_reconstruct_dense: after any propagation of that state, writes
 *     rho_S(t) = sum_ab A_ab G_t[|a><b|] for the dense initial operator
 *     A = d_rho0 to d_rho_t.  Both are caller-owned device arrays of
 *     (N+1)^2 complex128 (row-major, basis {c, e_1..e_N}, 16-byte aligned,
 *     distinct); N + 1 <= 2^20.  A need not be Hermitian.  The handle keeps a
 *     device workspace of about (3/256)(N+1)^2 complex values (allocated on
 *     first use).  Reads A once in a partial-sum pass and once more with the
 *     write of rho_S(t); repeatable bit for bit.  Asynchronous on `stream`.
 *     SA_ERR_STATE if the handle is not a representatives handle.
 */
int sa_heom_build_representatives(const sa_params* p, int precision, int flags, sa_heom** out);
int sa_heom_init_representatives(const sa_heom* h, void* d_state, void* stream);
int sa_heom_reconstruct_dense(sa_heom* h, const void* d_state, const void* d_rho0, void* d_rho_t, void* stream);

/*
 * sa_heom_state_upload / sa_heom_state_download -- copy a full state between
 * a host complex128 array in the canonical layout (n_vars_total complex
 * values) and a device state buffer, converting to / from the handle's
 * precision (the FP64 copies of the physical representative are exact).
 * The complex128 values cross the bus as they are (16 bytes per variable;
 * from page-locked host memory at full DMA speed) and an SA_FP32_AUX handle
 * narrows or widens them on the device, staging them in its own RK4 work
 * vectors (scratch between steps, so a call must not overlap a propagation
 * of the same handle).  Synchronous with respect to the host.
 */
int sa_heom_state_upload(const sa_heom* h, const double* host_x, void* d_state, void* stream);
int sa_heom_state_download(const sa_heom* h, const void* d_state, double* host_x, void* stream);

/*
 * sa_heom_rhs -- one evaluation of the matrix-free right-hand side
 * dR/dt = M_u R (Eq. uvar-propagator; Hamiltonian terms from grouped sums,
 * Eqs. grouped-row-sum, grouped-column-sum, HZ, HX and their Y, P, S, T
 * counterparts; damping Gamma_Lambda; cavity loss; hierarchy terms of
 * Eqs. uvar-up, uvar-down).  d_x, d_dx: device buffers of state layout
 * (may not alias).  Asynchronous on `stream`.
 */
int sa_heom_rhs(sa_heom* h, const void* d_x, void* d_dx, void* stream);

/*
 * sa_heom_step -- one classical RK4 step of size dt (the integrator of
 * Sec. V) on d_state, in place, as four fused right-hand-side + stage
 * kernels.  Asynchronous on `stream`.
 */
int sa_heom_step(sa_heom* h, void* d_state, double dt, void* stream);

/*
 * sa_heom_propagate -- nsteps RK4 steps.  The steps run as a CUDA graph of
 * obs_every steps (captured on first use for this state pointer, dt and
 * obs_every, then replayed).  If h_obs is not NULL, the observables of
 * sa_heom_observables are recorded for every instance before the first step
 * and after every obs_every steps (and after the last step): h_obs receives
 * rows * count * 8 doubles with rows = 1 + ceil(nsteps / obs_every).
 * Returns when the work is done when h_obs is not NULL; otherwise
 * asynchronous on `stream`.
 */
int sa_heom_propagate(sa_heom* h, void* d_state, double dt, int64_t nsteps, int64_t obs_every, double* h_obs,
                      void* stream);

/*
 * sa_heom_prepare -- capture and instantiate now every CUDA graph that
 * sa_heom_propagate(h, d_state, dt, nsteps, obs_every, ...) will replay
 * (runs of at most 64 steps, keyed by state pointer, dt and run length), so
 * that the propagation itself builds none.  Runs no kernel; synchronous.
 * obs_every <= 0: no observables (one run of nsteps).  The handle keeps up to
 * 16 graphs; a call needing more than that prepares only the last ones.
 */
int sa_heom_prepare(sa_heom* h, void* d_state, double dt, int64_t nsteps, int64_t obs_every);

/*
 * sa_heom_observables -- Eqs. trace-uvar, Pcav-uvar, Pexc-uvar, PB-uvar,
 * PD-uvar, Pplus-uvar, Pminus-uvar from the FP64 physical representative of
 * every instance: out[8 * i ..] = Tr, P_cav, P_exc, P_B, P_D, P_+, P_-,
 * max Hermiticity defect of rho_S.  theta from tan(2 theta) =
 * Omega_R / Delta, Delta = omega_cav - eps_x, theta in [0, pi/2]
 * (Eq. polariton-states).  Synchronous; returns NUMERIC if a value is not
 * finite.
 */
int sa_heom_observables(sa_heom* h, const void* d_state, double* out, void* stream);

/*
 * Launch tuning.  block: threads per CTA (64..256, multiple of 32);
 * chunk: variables per warp work item (>= largest pattern, <= 1024, multiple
 * of 32); queue: 1 for the dynamic work queue over a persistent grid, 0 for
 * one work item per warp.  Any argument
 * <= 0 keeps its current value.  sa_heom_autotune times every variant
 * (the list kernel only on a packed handle), block size (128, 256), item
 * size (64 .. 256) and queue mode on d_state (which it leaves changed) over
 * four RK4 steps replayed as the CUDA graph sa_heom_propagate uses, times
 * the four fastest again over twelve and keeps the best; best[3] receives
 * block, chunk, queue (sa_heom_get_tuning also reports the kernel variant it
 * chose).
 */
int sa_heom_set_tuning(sa_heom* h, int block, int chunk, int queue);
int sa_heom_autotune(sa_heom* h, void* d_state, void* stream, int* best);

/*
 * Tuning cache.  sa_heom_autotune first looks its answer up in a process-wide
 * cache keyed by sa_heom_tuning_key -- the device (name and SM count), the
 * precision, the layout (packed or not), the largest pattern, the variable
 * count rounded down to a power of two and the multiset of (m, L, d) of the
 * instances -- and a hit applies the cached tuning without timing anything;
 * after timing, the winner is stored under the key.
 *   sa_heom_autotune_ex      as sa_heom_autotune; flags SA_TUNE_FORCE times
 *                            afresh and replaces the entry.
 *   sa_heom_tuning_key       the handle's key (pure host; without the device
 *                            part for a host-only handle).
 *   sa_heom_tuning_cache_save / _load   the cache as a text file, one entry
 *                            per line: key (16 hex digits), block, chunk,
 *                            queue, kernel.  Loading adds to the cache;
 *                            INVALID_ARG, and nothing added, for a missing or
 *                            malformed file.
 *   sa_heom_tuning_cache_clear, _size   empty it, count its entries.
 * The cache is shared by the threads of a process (guarded by a mutex).
 */
enum { SA_TUNE_FORCE = 1 };
int sa_heom_autotune_ex(sa_heom* h, void* d_state, void* stream, int flags, int* best);
int sa_heom_tuning_key(const sa_heom* h, uint64_t* out);
int sa_heom_tuning_cache_save(const char* path);
int sa_heom_tuning_cache_load(const char* path);
int sa_heom_tuning_cache_clear(void);
int sa_heom_tuning_cache_size(int64_t* out);

/*
 * Stage-kernel variant.  Both evaluate the same right-hand side (Eqs.
 * uvar-up, uvar-down and the commutator of Eq. HS) and fuse the RK4 stage.
 *   SA_KERNEL_RECORDS  each lane walks the connection records of its
 *                      variable's row and column categories and resolves
 *                      the aligned accessor (Eq. aligned-accessor) on the
 *                      fly; device tables ~ 24 B per record.
 *   SA_KERNEL_LISTS    the host resolves every hierarchy term once; the
 *                      device holds, per work item, the variables in lane
 *                      order (sorted by term count) and per round of 32
 *                      lanes a term-major list of (target index, coefficient
 *                      slot) entries: 6 B per term plus padding to the
 *                      round's longest list, 5 B per variable.
 *   SA_KERNEL_ELL      the same host-resolved terms, one thread per variable
 *                      in memory order (warp w takes variables 32 w ..
 *                      32 w + 31): T_w rows of 32 entries per warp, T_w its
 *                      longest list; 4 B per variable; no shared memory.
 *                      A grouped-sum kernel forms R_q, C_q and the Z sums
 *                      first (scratch: 2 per category + 1 per pattern).
 *                      The item capacity (chunk) does not apply to it.
 * A new handle uses SA_KERNEL_LISTS.
 * sa_heom_set_kernel rebuilds the launch tables (synchronous; INVALID_ARG for
 * an unknown variant, OOM if the lists do not fit).  sa_heom_get_tuning
 * writes block, chunk, queue, kernel to out[0..3].
 */
enum { SA_KERNEL_RECORDS = 0, SA_KERNEL_LISTS = 1, SA_KERNEL_ELL = 2 };
int sa_heom_set_kernel(sa_heom* h, int kernel);
int sa_heom_get_tuning(const sa_heom* h, int* out);

/* Kernel launches one RK4 step issues: 4 stage kernels (SA_FP64), or 4 stage
 * kernels each with the FP64 physical-representative kernel (SA_FP32_AUX);
 * SA_KERNEL_ELL adds a grouped-sum kernel before each stage kernel; a
 * packed handle's stage kernel is the pack kernel, which also runs the list
 * units of the instances left unpacked. */
int sa_heom_launches_per_step(const sa_heom* h);

/*
 * sa_heom_device_error -- read the kernels' device error word (synchronises
 * `stream`).  Returns SA_ERR_TIMEOUT if a stage kernel gave up a bounded
 * wait on its bulk copies, SA_ERR_STATE if a stage kernel checking its table
 * indices (SA_DEBUG_CHECK_INDICES) found one out of range, SA_OK otherwise.
 * sa_heom_propagate with observables checks it too.  Reading the word clears
 * it.  After
 * SA_ERR_TIMEOUT the outputs of the affected launches, and so the caller's
 * state buffer, are undefined, and unless the expiry was injected
 * (SA_DEBUG_EXPIRE_WAIT) a copy the kernel gave up on may still land in
 * shared memory of the exited block: discard the state and the handle
 * (sa_heom_destroy) and build anew.
 */
int sa_heom_device_error(sa_heom* h, void* stream);

/*
 * Checkpoint / resume (no counterpart in the paper).  A checkpoint is a
 * host buffer of sa_heom_checkpoint_bytes bytes: a 64-byte header (format,
 * precision, instance count, variables, state bytes, the caller's step index
 * and sa_heom_config_hash) followed by the device state exactly as stored
 * (float2 auxiliaries plus the FP64 copies of rho_S, or double2), so a resume
 * continues bit for bit: the kernels compute every variable in a fixed
 * order whatever the scheduling.
 *   sa_heom_config_hash      64-bit FNV-1a hash of the precision, every
 *                            instance's sa_params, the table layout version
 *                            and the device layout (where every instance's
 *                            variables lie).  Pure host.
 *   sa_heom_checkpoint_save  d_state -> host_buf (caller-owned, at least
 *                            sa_heom_checkpoint_bytes); synchronous.
 *   sa_heom_checkpoint_load  host_buf -> d_state, *step (nullable) <- the
 *                            saved step index; SA_ERR_STATE, and d_state
 *                            untouched, if the format, precision, sizes or
 *                            parameter hash differ or the buffer is short.
 *                            Synchronous.
 */
int sa_heom_config_hash(const sa_heom* h, uint64_t* out);
int sa_heom_checkpoint_bytes(const sa_heom* h, size_t* bytes);
int sa_heom_checkpoint_save(const sa_heom* h, const void* d_state, int64_t step, void* host_buf, size_t bytes,
                            void* stream);
int sa_heom_checkpoint_load(const sa_heom* h, const void* host_buf, size_t bytes, void* d_state, int64_t* step,
                            void* stream);

/*
 * Failure detection (no counterpart in the paper).
 *   sa_heom_validate   checks the host tables of every instance: pattern,
 *                      category and variable counts (Eq. uvar-count),
 *                      multiplicities summing to N, T-ranks, and every
 *                      connection record -- its target must be the first
 *                      variable of a pattern one tier up (raise) or down
 *                      (lower) with the G' the record names, its moved
 *                      category inside that pattern, its channel below m and
 *                      occupation at most L.  SA_ERR_STATE names the first
 *                      inconsistency (sa_heom_last_error).  Pure host; about
 *                      a second at 10^8 records.
 *   sa_heom_set_debug  SA_DEBUG_EXPIRE_WAIT: the list stage kernel
 *                      takes the expiry path of their bounded wait on
 *                      an item's bulk copies without testing it (each warp
 *                      still waits, bounded, for its copies before it
 *                      leaves), so sa_heom_device_error reports
 *                      SA_ERR_TIMEOUT; the launch's outputs are incomplete.
 *                      0 turns it off again.  SA_DEBUG_CORRUPT_RECORD
 *                      (host-only handles; STATE otherwise) moves the target
 *                      of instance 0's first connection record off its
 *                      pattern, for which sa_heom_validate must fail; it
 *                      cannot be undone.  SA_DEBUG_CHECK_INDICES: the list
 *                      and pack kernels check every hierarchy-term target
 *                      and coefficient slot they read from their tables
 *                      against the instance's variable and slot counts; an
 *                      index out of range is replaced by 0 (no access outside
 *                      the buffers) and sets the device error word, which
 *                      sa_heom_device_error reports as SA_ERR_STATE; the
 *                      launch's outputs are then wrong.  SA_DEBUG_CORRUPT_LIST
 *                      (device handles running the list kernel, and only
 *                      together with SA_DEBUG_CHECK_INDICES; INVALID_ARG
 *                      otherwise) rebuilds the term lists with one target of
 *                      the first term row out of range, for that check to
 *                      find; turning it off rebuilds them correct.  Other
 *                      bits: INVALID_ARG.
 */
enum { SA_DEBUG_EXPIRE_WAIT = 1, SA_DEBUG_CORRUPT_RECORD = 2, SA_DEBUG_CHECK_INDICES = 4, SA_DEBUG_CORRUPT_LIST = 8 };
int sa_heom_validate(const sa_heom* h);
int sa_heom_set_debug(sa_heom* h, int flags);

/*
 * sa_heom_observables_noalloc -- the same observables as sa_heom_observables
 * (same kernel, same out[8 * i ..] layout), for callers that may not call
 * cudaMalloc.  The paper has no counterpart to this entry point.
 *
 * sa_heom_observables keeps its device output buffer in the handle and
 * allocates or grows it with cudaMalloc on first use, and cudaMalloc /
 * cudaFree can synchronise the whole device.  That is not acceptable for an
 * application that reserves the device's memory up front for its own pool
 * allocator and forbids any further driver allocation, nor inside a timing-
 * critical loop that must not stall other streams.  This entry point calls
 * no cudaMalloc, cudaFree or other allocating routine: its device output
 * lives in a fixed array of SA_HEOM_NOALLOC_MAX_INSTANCES * 8 doubles
 * (256 KiB) compiled into the library, which every GPU that loads the library
 * holds until the process exits.
 *   - Batches with more than SA_HEOM_NOALLOC_MAX_INSTANCES instances are
 *     rejected with SA_ERR_UNSUPPORTED.
 *   - Every call looks up the array's device address (cudaGetSymbolAddress,
 *     which allocates nothing) with the handle's device current; the first
 *     call on a device also loads the array there, so make that first call
 *     before any stream capture.  No address is cached across calls, so a
 *     cudaDeviceReset between calls leaves nothing stale.
 *   - Every call and every handle shares the one array, which keeps the last
 *     call's contents; calls whose work overlaps on the GPU (different streams
 *     or host threads) race on it.  Each call overwrites every slot it reads
 *     back, so no clearing is needed between calls.
 * Synchronous on `stream`; returns SA_ERR_NUMERIC if a value is not finite.
 */
#define SA_HEOM_NOALLOC_MAX_INSTANCES 4096
int sa_heom_observables_noalloc(sa_heom* h, const void* d_state, double* out, void* stream);

/*
 * Conventional scaled HEOM on the GPU (cross-check of the symmetry-adapted
 * path on small ensembles): every label n in N0^{N m} with |n| <= L
 * (Eq. direct-ado-count, lexicographic order, the zero label first), every
 * ADO a dense (N+1) x (N+1) complex matrix (Eq. basis), right-hand side
 * Eq. scaled-HEOM with the same cavity loss, classical RK4.
 *   sa_conv_build:   tables for one instance (N <= 64, at most 16 GB per
 *                    state vector); allocates three RK4 work vectors.  The
 *                    host build hashes every label once per channel and
 *                    direction: seconds at a million ADOs.
 *   sa_conv_info:    number of ADOs and bytes of one state vector
 *                    (double2[n_ados * (N+1)^2], ADO-major, row-major).
 *   sa_conv_labels:  n_ados * N * m occupations (molecule-major).
 *   sa_conv_set_rho0: zero the state and copy rho0 ((N+1)^2 complex,
 *                    row-major, host) into the zero-label ADO; synchronous.
 *   sa_conv_rhs:     one right-hand side, d_x -> d_dx (distinct).
 *   sa_conv_step:    nsteps RK4 steps of size dt in place; asynchronous.
 * Errors as for sa_heom_*; sa_conv_last_error gives the detail.
 */
typedef struct sa_conv sa_conv;
int sa_conv_build(const sa_params* p, sa_conv** out);
void sa_conv_destroy(sa_conv* c);
int sa_conv_info(const sa_conv* c, int64_t* n_ados, size_t* state_bytes);
int sa_conv_labels(const sa_conv* c, uint8_t* out);
int sa_conv_set_rho0(const sa_conv* c, const double* rho0, void* d_state, void* stream);
int sa_conv_rhs(sa_conv* c, const void* d_x, void* d_dx, void* stream);
int sa_conv_step(sa_conv* c, void* d_state, double dt, int64_t nsteps, void* stream);
const char* sa_conv_last_error(void);

const char* sa_heom_strerror(int code);
const char* sa_heom_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SA_HEOM_H */
