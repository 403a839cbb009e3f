"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Nothing here uses the CUDA path.  Each test names the passage it follows.
"""
import itertools
import os
from math import comb, factorial

import numpy as np
import pytest

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _bath_generic(m, seed=0):
    """A generic complex bath: complex c_k, c-check_k not conj(c_k), complex
    nu_k.  Exercises every coefficient path of Eq. scaled-HEOM."""
    rng = np.random.default_rng(seed)
    c = rng.uniform(0.1, 0.5, m) + 1j * rng.uniform(-0.4, 0.4, m)
    cc = rng.uniform(0.1, 0.5, m) + 1j * rng.uniform(-0.4, 0.4, m)
    nu = rng.uniform(0.2, 1.2, m) + 1j * rng.uniform(-0.3, 0.3, m)
    return {"c": c, "cc": cc, "nu": nu}


# ---------------------------------------------------------------- counts ---

def test_table1_counts(orc):
    """Table 1 (Sec. V.F): all six rows, six columns, 3 significant figures."""
    from oracle.counts import sig3, table1_row

    bath = {"c": np.array([0.1 + 0.0j]), "cc": np.array([0.1 + 0.0j]), "nu": np.array([1.0])}
    rows = [l.split() for l in open(os.path.join(GOLD, "table1_L25_m1.txt")) if l.strip() and l[0] != "#"]
    assert len(rows) == 6
    for row in rows:
        N = int(float(row[0]))
        sa = orc.SA(N, 1, 25, bath, cache=False)
        got = table1_row(N, 25, sa.npat, sa.nvar)
        want = row[1:]
        cols = ["n_ado_naive", "m_ado_naive_gb", "n_ado_can", "n_var_unq", "m_var_unq_gb", "R"]
        for c, w in zip(cols, want):
            mant, exp = w.split("e")
            assert sig3(got[c]) == f"{float(mant):.2f}e{int(exp)}", (N, c, sig3(got[c]), w)


def test_exact_counts_text(orc):
    """Sec. V.F text: 9296 patterns; 306743 / 306750 / 306751 variables;
    4.91 MB saturated storage."""
    bath = {"c": np.array([0.1 + 0.0j]), "cc": np.array([0.1 + 0.0j]), "nu": np.array([1.0])}
    for line in open(os.path.join(GOLD, "exact_counts.txt")):
        if not line.strip() or line[0] == "#":
            continue
        kind, m, L, d, N, val = line.split()
        if int(d) != 0:
            continue  # distinguished molecules are pinned in their own test
        sa = orc.SA(int(N), int(m), int(L), bath, cache=False)
        if kind == "patterns":
            assert sa.npat == int(val)
        elif kind == "variables":
            assert sa.nvar == int(val)
        elif kind == "megabytes":
            assert f"{16 * sa.nvar / 1e6:.2f}" == val


@pytest.mark.parametrize("N,m,L", [(1, 1, 3), (2, 1, 3), (3, 2, 2), (2, 3, 3), (4, 1, 4), (3, 3, 2)])
def test_conventional_ado_count(orc, N, m, L):
    """Eq. direct-ado-count: C(Nm+L, L) labels, each a dense (N+1)^2 matrix;
    checked against brute-force enumeration of N0^{Nm} with |n| <= L."""
    bath = _bath_generic(m)
    cv = orc.Conventional(N, m, L, bath)
    assert cv.nado == comb(N * m + L, L)
    brute = sum(1 for n in itertools.product(range(L + 1), repeat=N * m) if sum(n) <= L)
    assert cv.nado == brute
    labs = cv.labels()
    assert len({tuple(r) for r in labs}) == cv.nado
    assert labs.sum(axis=1).max() <= L


@pytest.mark.parametrize("L", [3, 6, 10, 14])
def test_canonical_count_partitions(orc, L):
    """Eqs. canonical-count-one, first-saturation: sum_l p_N(l) patterns for
    m = 1, constant for N >= L (textbook partition counts)."""
    from oracle.counts import canonical_count_m1

    bath = {"c": np.array([0.1 + 0.0j]), "cc": np.array([0.1 + 0.0j]), "nu": np.array([1.0])}
    for N in list(range(1, L + 3)) + [10 * L]:
        sa = orc.SA(N, 1, L, bath, cache=False)
        assert sa.npat == canonical_count_m1(N, L)
    sat = orc.SA(L, 1, L, bath, cache=False).npat
    assert orc.SA(L - 1, 1, L, bath, cache=False).npat < sat
    assert orc.SA(5 * L, 1, L, bath, cache=False).npat == sat


@pytest.mark.parametrize("m,L", [(2, 4), (2, 6), (3, 4), (4, 3), (2, 8)])
def test_pattern_count_generating_function(orc, m, L):
    """m > 1 (last paragraph of Sec. IV): patterns are multisets of nonzero
    local vectors; for N >= L their number is the generating-function count
    prod_k (1-x^k)^(-C(k+m-1, m-1)) summed to tier L."""
    from oracle.counts import multiset_vector_count

    bath = _bath_generic(m)
    assert orc.SA(L, m, L, bath, cache=False).npat == multiset_vector_count(m, L)
    assert orc.SA(3 * L, m, L, bath, cache=False).npat == multiset_vector_count(m, L)


@pytest.mark.parametrize("m,L", [(1, 5), (1, 9), (2, 4), (3, 3)])
def test_unique_variable_saturation(orc, m, L):
    """Eq. second-saturation: the unique-variable count is constant for
    N >= L+2 and still grows at N = L+1; the pattern count is constant for
    N >= L (Eq. first-saturation)."""
    bath = _bath_generic(m)
    nv = {N: orc.SA(N, m, L, bath, cache=False).nvar for N in range(1, L + 6)}
    npt = {N: orc.SA(N, m, L, bath, cache=False).npat for N in range(1, L + 6)}
    assert nv[L + 1] < nv[L + 2] == nv[L + 3] == nv[L + 5]
    assert npt[L - 1] < npt[L] == npt[L + 5]


def test_uvar_count_formula(orc):
    """Eq. uvar-count: u = (G+1)^2 + h per pattern, h = #{q: M_q >= 2}
    (Eq. h-Lambda), with sum_q M_q = N and sum_q q M_q = |Lambda|
    (Eqs. multiplicity-molecule-sum, multiplicity-tier-sum)."""
    bath = _bath_generic(2)
    N, m, L = 7, 2, 5
    sa = orc.SA(N, m, L, bath)
    pt = sa.patterns()
    vec = sa.vectors()
    norms = vec.sum(axis=1)
    for i in range(sa.npat):
        a, b = pt["cat_off"][i], pt["cat_off"][i + 1]
        ids, M = pt["cat_id"][a:b], pt["cat_M"][a:b]
        G = b - a
        h = int((M >= 2).sum())
        assert pt["G"][i] == G and pt["h"][i] == h
        assert pt["var_off"][i + 1] - pt["var_off"][i] == (G + 1) ** 2 + h
        assert M.sum() == N
        assert int((M * norms[ids]).sum()) == pt["tier"][i]


def test_ordering_count_example(orc):
    """Eq. ordering-count worked example: N_ord([2,1]; 4) = 4!/(1!1!2!) = 12,
    equal to the number of distinct arrangements of (2,1,0,0)."""
    bath = {"c": np.array([0.1 + 0.0j]), "cc": np.array([0.1 + 0.0j]), "nu": np.array([1.0])}
    sa = orc.SA(4, 1, 3, bath)
    pt = sa.patterns()
    vec = sa.vectors()[:, 0]
    i = [j for j in range(sa.npat) if list(vec[pt["ids"][j][: pt["r"][j]]]) == [2, 1]][0]
    M = pt["cat_M"][pt["cat_off"][i]:pt["cat_off"][i + 1]]
    nord = factorial(4) // int(np.prod([factorial(int(x)) for x in M]))
    assert nord == 12
    assert len(set(itertools.permutations((2, 1, 0, 0)))) == 12


def test_canonicalisation_example(orc):
    """Eq. pattern-example: (2,1,0,0), (0,2,1,0), (1,0,0,2) all map to [2,1]."""
    bath = {"c": np.array([0.1 + 0.0j]), "cc": np.array([0.1 + 0.0j]), "nu": np.array([1.0])}
    sa = orc.SA(4, 1, 3, bath)
    cv = orc.Conventional(4, 1, 3, bath)
    mp = cv.map_to(sa)
    labs = cv.labels()
    pt = sa.patterns()
    vec = sa.vectors()[:, 0]
    lab = sa.var_labels()
    for target in [(2, 1, 0, 0), (0, 2, 1, 0), (1, 0, 0, 2)]:
        a = [j for j in range(cv.nado) if tuple(labs[j]) == target][0]
        p = lab["pat"][mp[a, 0, 0]]
        assert list(vec[pt["ids"][p][: pt["r"][p]]]) == [2, 1]


def test_matrix_example_layout(orc):
    """Eq. matrix-example: the 5x5 representative of [2,1] at N = 4 has the
    printed structure, 17 distinct entries; the same 17 at N = 10."""
    bath = {"c": np.array([0.1 + 0.0j]), "cc": np.array([0.1 + 0.0j]), "nu": np.array([1.0])}
    gold = [l.split() for l in open(os.path.join(GOLD, "matrix_example_21_N4.txt")) if l.strip() and l[0] != "#"]
    sa = orc.SA(4, 1, 3, bath)
    cv = orc.Conventional(4, 1, 3, bath)
    mp = cv.map_to(sa)
    labs = cv.labels()
    a = [j for j in range(cv.nado) if tuple(labs[j]) == (2, 1, 0, 0)][0]
    lab = sa.var_labels()
    pt = sa.patterns()
    vec = sa.vectors()[:, 0]
    p = lab["pat"][mp[a, 0, 0]]
    cats = pt["cat_id"][pt["cat_off"][p]:pt["cat_off"][p + 1]]
    occ = {q + 1: int(vec[c]) for q, c in enumerate(cats)}   # category -> occupation
    names = {0: "Z", 1: "X", 2: "Y", 3: "P", 4: "S", 5: "T"}
    for ra in range(5):
        for cb in range(5):
            v = mp[a, ra, cb]
            k = names[int(lab["kind"][v])]
            q, r = int(lab["q"][v]), int(lab["r"][v])
            s = k if k == "Z" else (k + str(occ[q]) + (str(occ[r]) if k == "S" else ""))
            assert s == gold[ra][cb], (ra, cb, s, gold[ra][cb])
    assert len(set(mp[a].ravel())) == 17
    assert pt["var_off"][p + 1] - pt["var_off"][p] == 17
    sa10 = orc.SA(10, 1, 3, bath)
    pt10 = sa10.patterns()
    vec10 = sa10.vectors()[:, 0]
    p10 = [j for j in range(sa10.npat) if list(vec10[pt10["ids"][j][: pt10["r"][j]]]) == [2, 1]][0]
    assert pt10["var_off"][p10 + 1] - pt10["var_off"][p10] == 17


def test_row_sum_example(orc):
    """Eq. row-sum-example: R_0^{[2,1]} = P_0 + T_0 + S_{0,2} + S_{0,1} at
    N = 4.  With nu = 0, L = 3 ([2,1] at the top tier, no raising), Z = 0 and
    g = 1, Eq. HX reduces to dX_0/dt = i R_0."""
    bath = {"c": np.array([0.3 + 0.0j]), "cc": np.array([0.3 + 0.0j]), "nu": np.array([0.0])}
    sa = orc.SA(4, 1, 3, bath, g=1.0)
    lab = sa.var_labels()
    pt = sa.patterns()
    vec = sa.vectors()[:, 0]
    p = [j for j in range(sa.npat) if list(vec[pt["ids"][j][: pt["r"][j]]]) == [2, 1]][0]
    cats = pt["cat_id"][pt["cat_off"][p]:pt["cat_off"][p + 1]]
    qof = {int(vec[c]): q + 1 for q, c in enumerate(cats)}  # occupation -> category
    rng = np.random.default_rng(3)
    x = np.zeros(sa.nvar, complex)
    sel = lab["pat"] == p
    x[sel] = rng.standard_normal(sel.sum()) + 1j * rng.standard_normal(sel.sum())
    x[pt["var_off"][p]] = 0.0  # Z = 0

    def var(kind, q, r=0):
        hit = np.nonzero(sel & (lab["kind"] == kind) & (lab["q"] == q) & (lab["r"] == r))[0]
        assert len(hit) == 1
        return hit[0]

    q0, q1, q2 = qof[0], qof[1], qof[2]
    printed = x[var(3, q0)] + x[var(5, q0)] + x[var(4, q0, q2)] + x[var(4, q0, q1)]
    dx = sa.rhs(x)
    assert abs(dx[var(1, q0)] - 1j * printed) < 1e-14


def test_swap_example(orc):
    """Sec. III.B example: for [2,2] at N = 4, lowering molecule 1 gives the
    raw target (1,2,0,0) whose canonical pattern [2,1] stores molecule 1 and 2
    swapped.  The row-lowering term of T_2 = <e1|R|e2> must read the [2,1]
    entry S_{1,2} (row: occupation 1, column: occupation 2), which is also
    what the conventional ADO (1,2,0,0) holds at (e1, e2)."""
    bath = {"c": np.array([0.3 + 0.1j]), "cc": np.array([0.3 - 0.1j]), "nu": np.array([1.0])}
    sa = orc.SA(4, 1, 4, bath)
    cv = orc.Conventional(4, 1, 4, bath)
    lab = sa.var_labels()
    pt = sa.patterns()
    vec = sa.vectors()[:, 0]

    def pat(occ):
        return [j for j in range(sa.npat) if list(vec[pt["ids"][j][: pt["r"][j]]]) == occ][0]

    p22, p21 = pat([2, 2]), pat([2, 1])
    cats22 = pt["cat_id"][pt["cat_off"][p22]:pt["cat_off"][p22 + 1]]
    cats21 = pt["cat_id"][pt["cat_off"][p21]:pt["cat_off"][p21 + 1]]
    q2 = [q + 1 for q, c in enumerate(cats22) if vec[c] == 2][0]
    T2 = np.nonzero((lab["pat"] == p22) & (lab["kind"] == 5) & (lab["q"] == q2))[0][0]
    tm = sa.terms()
    hit = np.nonzero((tm["var"] == T2) & (tm["dir"] == -1) & (tm["side"] == 0))[0]
    assert len(hit) == 1
    src = tm["src"][hit[0]]
    occ21 = {q + 1: int(vec[c]) for q, c in enumerate(cats21)}
    assert lab["pat"][src] == p21 and lab["kind"][src] == 4
    assert (occ21[lab["q"][src]], occ21[lab["r"][src]]) == (1, 2)
    labs = cv.labels()
    a = [j for j in range(cv.nado) if tuple(labs[j]) == (1, 2, 0, 0)][0]
    assert cv.map_to(sa)[a, 1, 2] == src


# ------------------------------------------- symmetry-adapted == conventional

CASES = [
    # N, m, L, bath kind, detuning, g, kappa
    (1, 2, 3, "mats", 0.02, 0.05, 0.01),
    (2, 1, 3, "hight", 0.0, 0.05 / np.sqrt(2), 0.0),
    (3, 1, 4, "hight", 0.02, 0.05, 0.01),
    (4, 1, 4, "hight", 0.02, 0.05, 0.0),
    (3, 2, 3, "mats", 0.02, 0.05, 0.01),
    (4, 2, 3, "mats", -0.01, 0.07, 0.02),
    (3, 3, 3, "static", 0.02, 0.05, 0.01),
    (3, 2, 3, "generic", 0.1, 0.2, 0.05),
    (4, 2, 2, "generic", 0.1, 0.2, 0.05),
    (2, 4, 2, "generic", 0.1, 0.2, 0.0),
]


def _bath(kind, m):
    import oracle.bath as B

    if kind == "hight":
        return B.high_t(0.01, 0.05, 0.025)
    if kind == "mats":
        return B.matsubara(0.02, 0.05, 0.025, m - 1)
    if kind == "static":
        return B.matsubara(0.02, 0.05, 0.025, m - 2, sigma=0.02)
    return _bath_generic(m, seed=m)


@pytest.mark.parametrize("case", CASES)
def test_sa_equals_conventional_rhs(orc, case):
    """Eq. canonical-ADO-eom and Sec. IV: the unique-variable generator is an
    exact reduction of Eq. scaled-HEOM.  For ANY unique-variable vector x,
    expanding x to all conventional ADO entries and applying the conventional
    RHS equals expanding the symmetry-adapted RHS (to rounding).  Covers m > 1,
    loss, the static channel, complex c_k, c-check_k != conj(c_k), complex nu."""
    N, m, L, kind, det, g, kap = case
    bath = _bath(kind, m)
    sa = orc.SA(N, m, L, bath, det, g, kap)
    cv = orc.Conventional(N, m, L, bath, det, g, kap)
    mp = cv.map_to(sa)
    assert (mp >= 0).all()
    assert set(np.unique(mp)) == set(range(sa.nvar))  # every variable is some entry
    rng = np.random.default_rng(7)
    x = rng.standard_normal(sa.nvar) + 1j * rng.standard_normal(sa.nvar)
    dsa = sa.rhs(x)
    dcv = cv.rhs(x[mp])
    scale = np.abs(dcv).max()
    assert np.abs(dcv - dsa[mp]).max() <= 1e-13 * scale
    assert orc.errors() == 0


@pytest.mark.parametrize("case", CASES[1:6])
def test_sa_equals_conventional_propagation(orc, case):
    """Central covariance (Eq. central-covariance) under a permutation-
    invariant initial state: RK4 on both hierarchies agrees to rounding, and
    every conventional ADO entry equals its unique variable."""
    N, m, L, kind, det, g, kap = case
    bath = _bath(kind, m)
    sa = orc.SA(N, m, L, bath, det, g, kap)
    cv = orc.Conventional(N, m, L, bath, det, g, kap)
    mp = cv.map_to(sa)
    Z, P0, T0, X0 = 0.4, 0.25, 0.05, 0.1 + 0.05j
    if N == 1:
        P0 = 0.6
    x = sa.initial_state(Z, X0, np.conj(X0), P0, T0)
    xc = cv.zeros()
    xc[0] = x[mp[0]]
    ys = sa.rk4(x, 0.05, 200)
    yc = cv.rk4(xc, 0.05, 200)
    assert np.abs(yc - ys[mp]).max() <= 1e-12 * np.abs(yc).max()


def test_relabel_covariance_conventional(orc):
    """Eqs. hierarchy-relabel, term-covariance: relabelling molecules (moving
    whole local vectors) commutes with the conventional generator."""
    N, m, L = 3, 2, 3
    bath = _bath_generic(m, 11)
    cv = orc.Conventional(N, m, L, bath, 0.05, 0.1, 0.02)
    labs = cv.labels()
    index = {tuple(l): a for a, l in enumerate(labs)}
    perm = [2, 0, 1]   # pi(i)
    inv = np.argsort(perm)
    rng = np.random.default_rng(5)
    x = rng.standard_normal((cv.nado, N + 1, N + 1)) + 1j * rng.standard_normal((cv.nado, N + 1, N + 1))
    U = np.zeros((N + 1, N + 1))
    U[0, 0] = 1
    for i in range(N):
        U[perm[i] + 1, i + 1] = 1
    xp = np.zeros_like(x)
    for a, l in enumerate(labs):
        lv = np.array(l).reshape(N, m)
        pl = lv[inv].ravel()              # (pi n)_ik = n_{pi^-1(i),k}
        xp[index[tuple(pl)]] = U @ x[a] @ U.T
    d = cv.rhs(x)
    dp = cv.rhs(xp)
    for a, l in enumerate(labs):
        lv = np.array(l).reshape(N, m)
        b = index[tuple(lv[inv].ravel())]
        assert np.abs(dp[b] - U @ d[a] @ U.T).max() < 1e-13


# ----------------------------------------------------------- closed forms

def _rk_obs(orc, sa, x, dt, steps, every):
    _, obs = sa.propagate(x, dt, steps, every)
    return obs


def test_rabi_closed_form(orc):
    """L = 0 leaves the TC Hamiltonian (Eq. HS) alone.  From |c><c| with
    detuning, Z(t) = 1 - (Omega_R^2/Omega^2) sin^2(Omega t/2),
    Omega^2 = Omega_R^2 + Delta^2, Omega_R = 2 g sqrt(N) (Eq. Rabi-splitting)."""
    bath = {"c": np.array([0.1 + 0.0j]), "cc": np.array([0.1 + 0.0j]), "nu": np.array([1.0])}
    N, gsn, det = 50, 0.1, 0.03
    g = gsn / np.sqrt(N)
    sa = orc.SA(N, 1, 0, bath, det, g, 0.0)
    assert sa.npat == 1 and sa.nvar == 5
    x = sa.initial_state(1.0, 0, 0, 0, 0)
    dt, steps = 0.05, 800
    obs = _rk_obs(orc, sa, x, dt, steps, 100)
    t = np.arange(obs.shape[0]) * 100 * dt
    OR = 2 * gsn
    Om = np.sqrt(OR ** 2 + det ** 2)
    Zt = 1 - (OR ** 2 / Om ** 2) * np.sin(Om * t / 2) ** 2
    assert np.abs(obs[:, 1] - Zt).max() < 1e-9


def test_bright_resonant_closed_form(orc):
    """Resonant bright start (Eq. bright-initial-uvar), L = 0:
    P_B(t) = cos^2(g sqrt(N) t), P_D = 0."""
    bath = {"c": np.array([0.1 + 0.0j]), "cc": np.array([0.1 + 0.0j]), "nu": np.array([1.0])}
    N, gsn = 10, 0.05
    sa = orc.SA(N, 1, 0, bath, 0.0, gsn / np.sqrt(N), 0.0)
    x = sa.initial_state(0, 0, 0, 1.0 / N, 1.0 / N)
    obs = _rk_obs(orc, sa, x, 0.05, 2000, 200)
    t = np.arange(obs.shape[0]) * 200 * 0.05
    assert np.abs(obs[:, 3] - np.cos(gsn * t) ** 2).max() < 1e-9
    assert np.abs(obs[:, 4]).max() < 1e-12


def _lineshape(bath, t):
    out = 0j
    for c, nu in zip(bath["c"], bath["nu"]):
        if nu == 0:
            out += c * t * t / 2
        else:
            out += c / nu ** 2 * (np.exp(-nu * t) + nu * t - 1)
    return out


@pytest.mark.parametrize("kind,m,L,tol", [("hight", 1, 8, 1e-11), ("mats", 2, 7, 1e-9), ("static", 3, 8, 1e-9)])
def test_pure_dephasing_closed_form(orc, kind, m, L, tol):
    """g = 0: X_0(t) = X_0(0) exp(-i Delta' t - g(t)), Y_0 with g*(t) from
    c-check, T_0 = T_0(0) exp(-g - g*), Z and P_0 constant, with the bath
    lineshape g(t) = sum_k c_k/nu_k^2 (e^{-nu_k t} + nu_k t - 1) of the
    exponential BCF of Eq. BCF-exp (c t^2/2 for the static channel of
    Eq. C_static).  Hierarchy truncation error only."""
    bath = _bath(kind, m)
    N, det = 6, 0.02
    sa = orc.SA(N, m, L, bath, det, 0.0, 0.0)
    X0 = 0.1 + 0.05j
    x = sa.initial_state(0.3, X0, np.conj(X0), 0.1, 0.02)
    dt, steps = 0.02, 1000
    y = sa.rk4(x, dt, steps)
    t = dt * steps
    gt = _lineshape(bath, t)
    gct = _lineshape({"c": bath["cc"], "nu": bath["nu"]}, t)
    ix = sa.rho0_index()
    assert abs(y[ix["X0"]] - X0 * np.exp(-1j * det * t - gt)) < tol
    assert abs(y[ix["Y0"]] - np.conj(X0) * np.exp(1j * det * t - gct)) < tol
    assert abs(y[ix["T0"]] - 0.02 * np.exp(-gt - gct)) < tol
    assert abs(y[ix["Z"]] - 0.3) < 1e-14 and abs(y[ix["P0"]] - 0.1) < 1e-14


def test_loss_closed_form(orc):
    """Cavity loss (reading: Lindblad on a within the single-excitation
    manifold), g = 0: Z(t) = Z(0) e^{-kappa t}; X_0 gains e^{-kappa t/2}."""
    bath = _bath("hight", 1)
    N, det, kap = 4, 0.0, 0.01
    sa = orc.SA(N, 1, 8, bath, det, 0.0, kap)
    X0 = 0.2
    x = sa.initial_state(0.5, X0, X0, 0.125, 0.0)
    dt, steps = 0.02, 1000
    y = sa.rk4(x, dt, steps)
    t = dt * steps
    ix = sa.rho0_index()
    assert abs(y[ix["Z"]] - 0.5 * np.exp(-kap * t)) < 1e-12
    gt = _lineshape(bath, t)
    assert abs(y[ix["X0"]] - X0 * np.exp(-kap * t / 2 - gt)) < 1e-10


def test_trace_and_hermiticity_invariants(orc):
    """kappa = 0: Tr rho_S = Z + N P_0 (Eq. trace-uvar) is conserved (an exact
    linear invariant, kept by RK4).  Real nu_k with c-check_k = conj(c_k):
    every ADO stays Hermitian, Y_q = X_q*, S_{r,q} = S_{q,r}*, Z, P, T real.
    Sum rules P_B + P_D = P_exc and P_+ + P_- + P_D = Tr."""
    import oracle.bath as B

    bath = B.matsubara(0.02, 0.05, 0.025, 1)
    N, L = 12, 5
    sa = orc.SA(N, 2, L, bath, 0.02, 0.1 / np.sqrt(N), 0.0)
    th = 0.5 * np.arctan2(0.2, -0.02)
    x = sa.initial_state(np.cos(th) ** 2, np.sin(th) * np.cos(th) / np.sqrt(N),
                         np.sin(th) * np.cos(th) / np.sqrt(N), np.sin(th) ** 2 / N, np.sin(th) ** 2 / N)
    y, obs = sa.propagate(x, 0.02, 3000, 500)
    assert np.abs(obs[:, 0] - 1.0).max() < 1e-13
    assert obs[:, 7].max() < 1e-14
    assert np.abs(obs[:, 3] + obs[:, 4] - obs[:, 2]).max() < 1e-14
    assert np.abs(obs[:, 5] + obs[:, 6] + obs[:, 4] - obs[:, 0]).max() < 1e-14
    lab = sa.var_labels()
    pt = sa.patterns()
    for p in range(sa.npat):
        a = pt["var_off"][p]
        sel = slice(a, pt["var_off"][p + 1])
        kinds, qs, rs = lab["kind"][sel], lab["q"][sel], lab["r"][sel]
        vals = y[sel]
        d = {(int(k), int(q), int(r)): v for k, q, r, v in zip(kinds, qs, rs, vals)}
        for (k, q, r), v in d.items():
            if k in (0, 3, 5):
                assert abs(v.imag) < 1e-14
            if k == 1:
                assert abs(v - np.conj(d[(2, q, 0)])) < 1e-14
            if k == 4:
                assert abs(v - np.conj(d[(4, r, q)])) < 1e-14


def test_initial_state_observables(orc):
    """Eqs. cavity-initial-uvar, bright-initial-uvar, upper-/lower-polariton-
    initial with the observables of Eqs. trace-uvar .. Pminus-uvar."""
    bath = _bath("hight", 1)
    N, gsn, det = 25, 0.1, 0.04
    sa = orc.SA(N, 1, 2, bath, det, gsn / np.sqrt(N), 0.0)
    th = 0.5 * np.arctan2(2 * gsn, -det)
    s, c = np.sin(th), np.cos(th)
    up = sa.observables(sa.initial_state(c * c, s * c / np.sqrt(N), s * c / np.sqrt(N), s * s / N, s * s / N))
    lp = sa.observables(sa.initial_state(s * s, -s * c / np.sqrt(N), -s * c / np.sqrt(N), c * c / N, c * c / N))
    cav = sa.observables(sa.initial_state(1, 0, 0, 0, 0))
    br = sa.observables(sa.initial_state(0, 0, 0, 1 / N, 1 / N))
    assert abs(up[5] - 1) < 1e-14 and abs(up[6]) < 1e-14 and abs(up[4]) < 1e-14
    assert abs(lp[6] - 1) < 1e-14 and abs(lp[5]) < 1e-14
    assert abs(cav[1] - 1) < 1e-15 and abs(cav[2]) < 1e-15
    assert abs(br[3] - 1) < 1e-14 and abs(br[4]) < 1e-14 and abs(br[2] - 1) < 1e-14
    # the polaritons diagonalise the TC Hamiltonian: a UP start stays UP at L=0
    sa0 = orc.SA(N, 1, 0, bath, det, gsn / np.sqrt(N), 0.0)
    x = sa0.initial_state(c * c, s * c / np.sqrt(N), s * c / np.sqrt(N), s * s / N, s * s / N)
    _, obs = sa0.propagate(x, 0.05, 1000, 250)
    assert np.abs(obs[:, 5] - 1).max() < 1e-10


def test_no_internal_errors(orc):
    assert orc.errors() == 0


# ---- terminator (the Ishizaki-Tanimura treatment of omitted Matsubara terms,
# named in Sec. V; reading: -Delta sum_i [Q_i, [Q_i, rho_n]] on every ADO)

@pytest.mark.parametrize("case", [(2, 1, 3, "hight", 0.02, 0.05, 0.01), (3, 2, 3, "mats", 0.02, 0.05, 0.0),
                                  (3, 2, 3, "generic", 0.1, 0.2, 0.05), (4, 1, 4, "hight", 0.0, 0.03, 0.0)])
def test_terminator_sa_equals_conventional(orc, case):
    """With the terminator on, the symmetry-adapted RHS (a per-variable weight)
    still equals the conventional RHS (the double commutator with explicit Q_i
    matrices), for any vector."""
    N, m, L, kind, det, g, kap = case
    bath = _bath(kind, m)
    Delta = 0.0123
    sa = orc.SA(N, m, L, bath, det, g, kap, term=Delta)
    cv = orc.Conventional(N, m, L, bath, det, g, kap, term=Delta)
    mp = cv.map_to(sa)
    rng = np.random.default_rng(3)
    x = rng.standard_normal(sa.nvar) + 1j * rng.standard_normal(sa.nvar)
    dsa, dcv = sa.rhs(x), cv.rhs(x[mp])
    assert np.abs(dcv - dsa[mp]).max() <= 1e-13 * np.abs(dcv).max()
    # and the term is really there: it changes the RHS by -Delta w x
    d0 = orc.SA(N, m, L, bath, det, g, kap).rhs(x)
    lab = sa.var_labels()
    w = np.select([np.isin(lab["kind"], [1, 2]), np.isin(lab["kind"], [4, 5])], [1.0, 2.0], 0.0)
    assert np.abs((dsa - d0) + Delta * w * x).max() <= 1e-14 * np.abs(x).max()
    assert orc.errors() == 0


def test_terminator_closed_form(orc):
    """L = 0, g = 0: every variable evolves on its own, dX_0 = (-i Delta' - Delta) X_0,
    dT_0 = -2 Delta T_0, Z and P_0 constant.  RK4 on a scalar linear equation
    multiplies by 1 + z + z^2/2 + z^3/6 + z^4/24 (z = rate dt) per step, exactly."""
    bath = _bath("hight", 1)
    N, det, Delta = 5, 0.03, 0.02
    sa = orc.SA(N, 1, 0, bath, det, 0.0, 0.0, term=Delta)
    X0, T0 = 0.2 - 0.1j, 0.05
    x = sa.initial_state(0.5, X0, np.conj(X0), 0.1, T0)
    dt, steps = 0.05, 400
    y = sa.rk4(x, dt, steps)
    amp = lambda z: (1 + z + z ** 2 / 2 + z ** 3 / 6 + z ** 4 / 24) ** steps
    ix = sa.rho0_index()
    assert abs(y[ix["X0"]] - X0 * amp((-1j * det - Delta) * dt)) < 1e-13
    assert abs(y[ix["Y0"]] - np.conj(X0) * amp((1j * det - Delta) * dt)) < 1e-13
    assert abs(y[ix["T0"]] - T0 * amp(-2 * Delta * dt)) < 1e-14
    assert y[ix["Z"]] == 0.5 and y[ix["P0"]] == 0.1


@pytest.mark.parametrize("K", [0, 1, 2, 5])
def test_terminator_strength(orc, K):
    """oracle.bath.terminator sums the omitted Matsubara c_j / nu_j term by term;
    it must equal the closed form of the full sum, lambda (2 kT / gamma -
    cot(gamma / 2 kT)), less the first K terms, and vanish as K grows."""
    import math

    import oracle.bath as B

    lam, gam, kT = 0.02, 0.05, 0.025
    full = lam * (2 * kT / gam - 1 / math.tan(gam / (2 * kT)))
    kept = sum(4 * lam * gam * kT / ((2 * math.pi * j * kT) ** 2 - gam ** 2) for j in range(1, K + 1))
    assert abs(B.terminator(lam, gam, kT, K) - (full - kept)) < 1e-15
    assert B.terminator(lam, gam, kT, K + 1) < B.terminator(lam, gam, kT, K)


# ---- one distinguished molecule (Sec. V.F: localised and cavity-site states;
# the distinguished molecule keeps its own singleton category)

def test_distinguished_counts_text(orc):
    """Sec. V.F text, one distinguished molecule: 41391 patterns for N >= 26,
    1715600 variables for N >= 28, 27.45 MB, 5.59 times the symmetric count."""
    bath = {"c": np.array([0.1 + 0.0j]), "cc": np.array([0.1 + 0.0j]), "nu": np.array([1.0])}
    base = orc.SA(27, 1, 25, bath, cache=False).nvar
    seen = 0
    for line in open(os.path.join(GOLD, "exact_counts.txt")):
        if not line.strip() or line[0] == "#":
            continue
        kind, m, L, d, N, val = line.split()
        if int(d) != 1:
            continue
        sa = orc.SA(int(N), int(m), int(L), bath, cache=False, d=1)
        seen += 1
        if kind == "patterns":
            assert sa.npat == int(val)
            assert orc.SA(int(N) - 1, int(m), int(L), bath, cache=False, d=1).npat < int(val)
        elif kind == "variables":
            assert sa.nvar == int(val)
            assert orc.SA(int(N) - 1, int(m), int(L), bath, cache=False, d=1).nvar < int(val)
        elif kind == "megabytes":
            assert f"{16 * sa.nvar / 1e6:.2f}" == val
        elif kind == "ratio":
            assert f"{sa.nvar / base:.2f}" == val
    assert seen == 4


D_CASES = [(1, 1, 3), (2, 1, 3), (3, 1, 3), (3, 2, 3), (4, 1, 4), (4, 2, 2), (5, 1, 3), (2, 3, 2)]


@pytest.mark.parametrize("N,m,L", D_CASES)
def test_distinguished_sa_equals_conventional_rhs(orc, N, m, L):
    """With molecule 1 distinguished, the reduced generator is still an exact
    reduction of Eq. scaled-HEOM: every conventional entry maps to a variable,
    every variable is some entry, and the right-hand sides agree for any
    vector (loss and terminator on)."""
    bath = _bath_generic(m, seed=N + m + L)
    kw = dict(detuning=0.1, g=0.2, kappa=0.05, term=0.01)
    sa = orc.SA(N, m, L, bath, d=1, **kw)
    cv = orc.Conventional(N, m, L, bath, **kw)
    mp = cv.map_to(sa)
    assert (mp >= 0).all() and set(np.unique(mp)) == set(range(sa.nvar))
    rng = np.random.default_rng(5)
    x = rng.standard_normal(sa.nvar) + 1j * rng.standard_normal(sa.nvar)
    dcv, dsa = cv.rhs(x[mp]), sa.rhs(x)
    assert np.abs(dcv - dsa[mp]).max() <= 1e-13 * np.abs(dcv).max()
    assert orc.errors() == 0


@pytest.mark.parametrize("N", [2, 3, 5])
def test_distinguished_localised_propagation(orc, N):
    """rho_S(0) = |e_1><e_1| (Eq. localized_initial_condition) is not
    permutation-invariant, so it needs the distinguished molecule: RK4 on both
    hierarchies agrees to rounding, and the observables follow the dense
    reduced density matrix."""
    import oracle.bath as B

    bath = B.high_t(0.01, 0.05, 0.025)
    kw = dict(detuning=0.0, g=0.05 / np.sqrt(N), kappa=0.0)
    sa = orc.SA(N, 1, 4, bath, d=1, **kw)
    cv = orc.Conventional(N, 1, 4, bath, **kw)
    mp = cv.map_to(sa)
    rho = np.zeros((N + 1, N + 1), complex)
    rho[1, 1] = 1.0
    x = sa.initial_state_dense(rho)
    xc = cv.zeros()
    xc[0] = rho
    assert np.array_equal(x[mp[0]], rho)
    ys = sa.rk4(x, 0.05, 200)
    yc = cv.rk4(xc, 0.05, 200)
    assert np.abs(yc - ys[mp]).max() <= 1e-12
    # populations from the dense rho_S of the conventional run
    r = yc[0]
    obs = sa.observables(ys)
    Bv = np.concatenate([[0], np.ones(N) / np.sqrt(N)])
    assert abs(obs[0] - np.trace(r).real) < 1e-12
    assert abs(obs[1] - r[0, 0].real) < 1e-12
    assert abs(obs[3] - (Bv @ r @ Bv).real) < 1e-12


@pytest.mark.parametrize("N", [2, 5, 10, 100, 10 ** 12])
def test_distinguished_initial_tc_populations(orc, N):
    """Resonant initial TC populations of Sec. V.F: the localised state has
    P_+ = P_- = 1/(2N), P_D = 1 - 1/N; the cavity-site superposition
    sqrt(0.3)|e_1> + sqrt(0.7)|c> has P_D = 0.3 (1 - 1/N) and
    P_+- = (sqrt(0.7) +- sqrt(0.3/N))^2 / 2."""
    import oracle.bath as B

    sa = orc.SA(N, 1, 2, B.high_t(0.01, 0.05, 0.025), 0.0, 0.05 / np.sqrt(N), 0.0, d=1)
    ix = sa.rho0_index()
    x = sa.zeros()
    x[ix["Pd"]] = 1.0
    o = sa.observables(x)
    assert abs(o[5] - 1 / (2 * N)) < 1e-13 and abs(o[6] - 1 / (2 * N)) < 1e-13
    assert abs(o[4] - (1 - 1 / N)) < 1e-13 and abs(o[0] - 1) < 1e-15
    x = sa.zeros()
    x[ix["Pd"]], x[ix["Z"]] = 0.3, 0.7
    x[ix["Xd"]] = x[ix["Yd"]] = np.sqrt(0.21)
    o = sa.observables(x)
    assert abs(o[4] - 0.3 * (1 - 1 / N)) < 1e-13
    assert abs(o[5] - 0.5 * (np.sqrt(0.7) + np.sqrt(0.3 / N)) ** 2) < 1e-13
    assert abs(o[6] - 0.5 * (np.sqrt(0.7) - np.sqrt(0.3 / N)) ** 2) < 1e-13


def _orbits(N, m, L, d):
    """Brute force: canonical patterns and unique variables are the orbits of
    ADO labels n in N0^(N m), |n| <= L, and of (label, row, column) triples
    under the permutations of molecules d+1..N (Sec. IV, Eq. N-symmetric-pool);
    basis index 0 is the cavity, i the molecule i."""
    import itertools

    labels = [t for t in itertools.product(range(L + 1), repeat=N * m) if sum(t) <= L]
    perms = [tuple(range(d)) + p for p in itertools.permutations(range(d, N))]
    ado_orb, var_orb = set(), set()
    for t in labels:
        mol = [t[i * m:(i + 1) * m] for i in range(N)]
        imgs = []
        for p in perms:
            # molecule i's vector moves to molecule p[i]
            new = [None] * N
            for i in range(N):
                new[p[i]] = mol[i]
            imgs.append((tuple(new), p))
        ado_orb.add(min(im for im, _ in imgs))
        for a in range(N + 1):
            for b in range(N + 1):
                var_orb.add(min((im, 0 if a == 0 else p[a - 1] + 1, 0 if b == 0 else p[b - 1] + 1)
                                for im, p in imgs))
    return len(ado_orb), len(var_orb)


@pytest.mark.parametrize("N,m,L,d", [(1, 1, 3, 1), (2, 1, 3, 1), (3, 1, 3, 1), (4, 1, 3, 1), (3, 2, 2, 1),
                                     (4, 2, 2, 2), (3, 1, 4, 2), (5, 1, 3, 2), (4, 1, 3, 3), (5, 1, 2, 3),
                                     (4, 2, 2, 0), (5, 1, 3, 0)])
def test_distinguished_counts_are_orbits(orc, N, m, L, d):
    """The pattern and variable counts equal the orbit counts of the
    conventional hierarchy under the residual permutation group, found by
    brute force."""
    bath = {"c": np.full(m, 0.1 + 0j), "cc": np.full(m, 0.1 + 0j), "nu": np.ones(m)}
    sa = orc.SA(N, m, L, bath, cache=False, d=d)
    assert (sa.npat, sa.nvar) == _orbits(N, m, L, d)


@pytest.mark.parametrize("m,L,d", [(1, 4, 2), (2, 3, 2), (1, 3, 3), (1, 6, 1), (2, 4, 3)])
def test_distinguished_saturation_thresholds(orc, m, L, d):
    """Eqs. distinguished-pattern-threshold and distinguished-thresholds: the
    pattern count stops growing exactly at N = L + d, the variable count
    exactly at N = L + d + 2."""
    bath = {"c": np.full(m, 0.1 + 0j), "cc": np.full(m, 0.1 + 0j), "nu": np.ones(m)}
    sa = {N: orc.SA(N, m, L, bath, cache=False, d=d) for N in range(max(d, 1), L + d + 6)}
    assert sa[L + d - 1].npat < sa[L + d].npat == sa[L + d + 5].npat
    assert sa[L + d + 1].nvar < sa[L + d + 2].nvar == sa[L + d + 5].nvar


@pytest.mark.parametrize("N,m,L,d", [(2, 1, 3, 2), (3, 1, 3, 2), (4, 2, 2, 2), (5, 1, 3, 2), (3, 1, 3, 3),
                                     (4, 1, 3, 3), (5, 2, 2, 3)])
def test_two_three_distinguished_sa_equals_conventional(orc, N, m, L, d):
    """d = 2, 3: the reduced generator is still an exact reduction of Eq.
    scaled-HEOM (the map is onto, and the right-hand sides agree, loss and
    terminator on)."""
    bath = _bath_generic(m, seed=N + m + L + d)
    kw = dict(detuning=0.1, g=0.2, kappa=0.05, term=0.01)
    sa = orc.SA(N, m, L, bath, d=d, **kw)
    cv = orc.Conventional(N, m, L, bath, **kw)
    mp = cv.map_to(sa)
    assert (mp >= 0).all() and set(np.unique(mp)) == set(range(sa.nvar))
    rng = np.random.default_rng(6)
    x = rng.standard_normal(sa.nvar) + 1j * rng.standard_normal(sa.nvar)
    dcv, dsa = cv.rhs(x[mp]), sa.rhs(x)
    assert np.abs(dcv - dsa[mp]).max() <= 1e-13 * np.abs(dcv).max()
    # the dense initial state lands where the map puts the physical ADO
    rho = rng.standard_normal((N + 1, N + 1)) + 1j * rng.standard_normal((N + 1, N + 1))
    sym = np.zeros_like(rho)
    import itertools

    perms = list(itertools.permutations(range(d + 1, N + 1)))
    for p in perms:  # average over the residual group so the state is invariant
        idx = list(range(d + 1)) + list(p)
        sym += rho[np.ix_(idx, idx)]
    sym /= len(perms)
    x0 = sa.initial_state_dense(sym)
    assert np.allclose(x0[mp[0]], sym, atol=1e-15)
    assert orc.errors() == 0


@pytest.mark.parametrize("N", [3, 7, 100, 10 ** 12])
def test_two_distinguished_initial_populations(orc, N):
    """(|e_1> +- |e_2>)/sqrt 2 at resonance: the symmetric state has bright
    weight 2/N, so P_+ = P_- = 1/N and P_D = 1 - 2/N; the antisymmetric one
    is dark, P_D = 1 (only the S_12 terms of P_B tell them apart)."""
    import oracle.bath as B

    sa = orc.SA(N, 1, 2, B.high_t(0.01, 0.05, 0.025), 0.0, 0.05 / np.sqrt(N), 0.0, d=2)
    ix = sa.rho0_index()
    for sgn in (1.0, -1.0):
        x = sa.zeros()
        x[ix["P1"]] = x[ix["P2"]] = 0.5
        x[ix["S12"]] = x[ix["S21"]] = 0.5 * sgn
        o = sa.observables(x)
        pb = 2.0 / N if sgn > 0 else 0.0
        assert abs(o[0] - 1) < 1e-15 and abs(o[3] - pb) < 1e-15
        assert abs(o[4] - (1 - pb)) < 1e-13
        assert abs(o[5] - pb / 2) < 1e-15 and abs(o[6] - pb / 2) < 1e-15


@pytest.mark.parametrize("N,m,L", [(1, 1, 4), (2, 1, 3), (2, 2, 3), (3, 1, 3), (3, 2, 2)])
def test_all_molecules_distinguished_is_conventional(orc, N, m, L):
    """d = N leaves no permutation symmetry (Eq. N-symmetric-pool with an
    empty pool): every pattern is one ADO label, every molecule its own
    category, so the reduced hierarchy is the conventional one entry for
    entry -- C(Nm+L, L) patterns of (N+1)^2 variables, the map a bijection."""
    bath = _bath_generic(m, seed=3 * N + m + L)
    kw = dict(detuning=0.05, g=0.2, kappa=0.02, term=0.01)
    sa = orc.SA(N, m, L, bath, d=N, **kw)
    cv = orc.Conventional(N, m, L, bath, **kw)
    assert sa.npat == cv.nado and sa.nvar == cv.nado * (N + 1) ** 2
    mp = cv.map_to(sa)
    assert np.array_equal(np.sort(mp.ravel()), np.arange(sa.nvar))
    rng = np.random.default_rng(9)
    x = rng.standard_normal(sa.nvar) + 1j * rng.standard_normal(sa.nvar)
    assert np.abs(cv.rhs(x[mp]) - sa.rhs(x)[mp]).max() <= 1e-13 * np.abs(sa.rhs(x)).max()


@pytest.mark.parametrize("N", [2, 5, 40])
def test_distinguished_localised_L0_closed_form(orc, N):
    """L = 0 (no bath), resonance, d = 1: RK4 is exact on each eigen-
    component of the Liouvillian, so rho(t_n) = sum_ab a_a a_b* |a><b|
    R(-i (E_a - E_b) dt)^n with R(z) = 1 + z + z^2/2 + z^3/6 + z^4/24.  For
    |e_1> the components are the polaritons (E = +- g sqrt N, weight 1/(2N)
    each) and the dark part (E = 0, weight 1 - 1/N); the molecule-1
    population P_11 and the cavity population follow in closed form."""
    import oracle.bath as B

    g, dt, n = 0.05 / np.sqrt(N), 0.05, 300
    sa = orc.SA(N, 1, 0, B.high_t(0.01, 0.05, 0.025), 0.0, g, 0.0, d=1)
    x = sa.zeros()
    x[sa.rho0_index()["Pd"]] = 1.0
    y = sa.rk4(x, dt, n)
    R = lambda z: 1 + z + z ** 2 / 2 + z ** 3 / 6 + z ** 4 / 24
    w = g * np.sqrt(N)
    # <e_1|UP> = <e_1|LP> = 1/sqrt(2N); <e_1|dark part> = 1 - 1/N; <c|UP> = -<c|LP> = 1/sqrt 2
    E = {"U": w, "L": -w, "D": 0.0}
    a = {"U": 1 / np.sqrt(2 * N), "L": 1 / np.sqrt(2 * N), "D": None}
    e1 = {"U": 1 / np.sqrt(2 * N), "L": 1 / np.sqrt(2 * N), "D": 1.0}  # <e_1|alpha> (dark: unnormalised part)
    cav = {"U": 1 / np.sqrt(2), "L": -1 / np.sqrt(2), "D": 0.0}
    amp = {"U": a["U"], "L": a["L"], "D": 1 - 1 / N}  # amplitude times norm of the dark part
    P11 = sum(e1[p] * amp[p] * amp[q] * e1[q] * R(-1j * (E[p] - E[q]) * dt) ** n for p in E for q in E)
    Pc = sum(cav[p] * amp[p] * amp[q] * cav[q] * R(-1j * (E[p] - E[q]) * dt) ** n for p in E for q in E)
    ix = sa.rho0_index()
    assert abs(y[ix["Pd"]] - P11) < 1e-13
    assert abs(y[ix["Z"]] - Pc) < 1e-13
