"""ORACLE -- test infrastructure only.

Plain FP64 CPU reference for the symmetry-adapted HEOM of Mondal & Huo
(arXiv 2608.20657).  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` import this
package.  The product package never imports it, and the two share no code.

* ``sa_heom_oracle.c`` (compiled to ``_liborc.so`` by :func:`build`) holds
  the conventional scaled HEOM (Eq. scaled-HEOM) and the symmetry-adapted
  unique-variable equations (Secs. III-IV), both integrated with RK4.
* :mod:`oracle.bath` holds the bath decompositions (Eq. BCF-exp, Eq.
  Drude_Lorentz, Eq. C_static) in exact / extended precision.
* :mod:`oracle.counts` holds the closed-form counts (Eqs. direct-ado-count,
  canonical-count-one, uvar-count, resources-*).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sa_heom_oracle.c")
_LIB = os.path.join(_HERE, "_liborc.so")
MAXM = 8


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (plain -O2, OpenMP over patterns)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(
            ["gcc", "-O2", "-fopenmp", "-std=c11", "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"]
        )
        os.replace(tmp, _LIB)
    return _LIB


class Params(ctypes.Structure):
    _fields_ = [
        ("N", ctypes.c_longlong),
        ("m", ctypes.c_int),
        ("L", ctypes.c_int),
        ("detuning", ctypes.c_double),
        ("g", ctypes.c_double),
        ("kappa", ctypes.c_double),
        ("c_re", ctypes.c_double * MAXM),
        ("c_im", ctypes.c_double * MAXM),
        ("cc_re", ctypes.c_double * MAXM),
        ("cc_im", ctypes.c_double * MAXM),
        ("nu_re", ctypes.c_double * MAXM),
        ("nu_im", ctypes.c_double * MAXM),
        ("term", ctypes.c_double),
        ("d", ctypes.c_int),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        P = ctypes.POINTER
        vp = ctypes.c_void_p
        ll = ctypes.c_longlong
        sig = {
            "orc_num_threads": (ctypes.c_int, []),
            "orc_errors": (ll, []),
            "orc_sa_create": (vp, [P(Params), ctypes.c_int]),
            "orc_sa_destroy": (None, [vp]),
            "orc_sa_num_patterns": (ll, [vp]),
            "orc_sa_num_vars": (ll, [vp]),
            "orc_sa_num_vectors": (ctypes.c_int, [vp]),
            "orc_sa_num_categories": (ll, [vp]),
            "orc_sa_vectors": (None, [vp, vp]),
            "orc_sa_patterns": (None, [vp, vp, vp, vp, vp, vp, vp, vp]),
            "orc_sa_categories": (None, [vp, vp, vp]),
            "orc_sa_var_labels": (None, [vp, vp, vp, vp, vp]),
            "orc_sa_rhs": (None, [vp, vp, vp]),
            "orc_sa_rhs_at": (None, [vp, vp, vp, ll, vp]),
            "orc_sa_num_terms": (ll, [vp]),
            "orc_sa_terms": (None, [vp, vp, vp, vp, vp, vp, vp]),
            "orc_sa_term_coefs": (None, [vp, vp, vp]),
            "orc_sa_rk4": (None, [vp, vp, ctypes.c_double, ll]),
            "orc_sa_observables": (None, [vp, vp, vp]),
            "orc_sa_propagate": (None, [vp, vp, ctypes.c_double, ll, ll, vp]),
            "orc_conv_create": (vp, [P(Params)]),
            "orc_conv_destroy": (None, [vp]),
            "orc_conv_num_ados": (ll, [vp]),
            "orc_conv_labels": (None, [vp, vp]),
            "orc_conv_rhs": (None, [vp, vp, vp]),
            "orc_conv_rk4": (None, [vp, vp, ctypes.c_double, ll]),
            "orc_conv_to_sa": (None, [vp, vp, vp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(_lib, name)
            f.restype = res
            f.argtypes = args
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def make_params(N, m, L, bath, detuning=0.0, g=0.0, kappa=0.0, term=0.0, d=0) -> Params:
    """bath: dict with complex arrays c, cc, nu of length m (Eq. BCF-exp);
    term: terminator strength Delta of the omitted Matsubara terms (0: off);
    d: distinguished molecules (0, or 1: molecule 1 keeps its label)."""
    p = Params()
    p.N, p.m, p.L, p.d = int(N), int(m), int(L), int(d)
    p.detuning, p.g, p.kappa, p.term = float(detuning), float(g), float(kappa), float(term)
    c = np.asarray(bath["c"], dtype=complex)
    cc = np.asarray(bath["cc"], dtype=complex)
    nu = np.asarray(bath["nu"], dtype=complex)
    assert c.shape == (m,) and cc.shape == (m,) and nu.shape == (m,)
    for k in range(m):
        p.c_re[k], p.c_im[k] = c[k].real, c[k].imag
        p.cc_re[k], p.cc_im[k] = cc[k].real, cc[k].imag
        p.nu_re[k], p.nu_im[k] = nu[k].real, nu[k].imag
    return p


def errors() -> int:
    return int(lib().orc_errors())


def num_threads() -> int:
    return int(lib().orc_num_threads())


KIND = {"Z": 0, "X": 1, "Y": 2, "P": 3, "S": 4, "T": 5}


class SA:
    """Symmetry-adapted HEOM oracle (O-2).  State: complex128 array of nvar."""

    def __init__(self, N, m, L, bath, detuning=0.0, g=0.0, kappa=0.0, cache=True, term=0.0, d=0):
        self.N, self.m, self.L, self.d = int(N), int(m), int(L), int(d)
        self.params = make_params(N, m, L, bath, detuning, g, kappa, term, d)
        self._h = lib().orc_sa_create(ctypes.byref(self.params), 1 if cache else 0)
        if not self._h:
            raise ValueError("oracle rejected the parameters")
        self.npat = int(lib().orc_sa_num_patterns(self._h))
        self.nvar = int(lib().orc_sa_num_vars(self._h))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.orc_sa_destroy(h)
            self._h = None

    # ---- tables ---------------------------------------------------------
    def vectors(self) -> np.ndarray:
        V = int(lib().orc_sa_num_vectors(self._h))
        out = np.zeros((V, self.m), dtype=np.uint8)
        lib().orc_sa_vectors(self._h, _ptr(out))
        return out

    def patterns(self) -> dict:
        P, L = self.npat, self.L + self.d  # id lists: <= L symmetric entries + d distinguished
        tier = np.zeros(P, np.int32)
        r = np.zeros(P, np.int32)
        G = np.zeros(P, np.int32)
        h = np.zeros(P, np.int32)
        var_off = np.zeros(P + 1, np.int64)
        cat_off = np.zeros(P + 1, np.int64)
        ids = np.zeros((P, max(L, 1)), np.int32)
        lib().orc_sa_patterns(self._h, _ptr(tier), _ptr(r), _ptr(G), _ptr(h), _ptr(var_off), _ptr(cat_off), _ptr(ids))
        ncat = int(lib().orc_sa_num_categories(self._h))
        cat_id = np.zeros(max(ncat, 1), np.int32)
        cat_M = np.zeros(max(ncat, 1), np.int64)
        lib().orc_sa_categories(self._h, _ptr(cat_id), _ptr(cat_M))
        return dict(tier=tier, r=r, G=G, h=h, var_off=var_off, cat_off=cat_off,
                    ids=ids[:, :L], cat_id=cat_id[:ncat], cat_M=cat_M[:ncat])

    def var_labels(self) -> dict:
        n = self.nvar
        pat = np.zeros(n, np.int64)
        kind = np.zeros(n, np.int32)
        q = np.zeros(n, np.int32)
        r = np.zeros(n, np.int32)
        lib().orc_sa_var_labels(self._h, _ptr(pat), _ptr(kind), _ptr(q), _ptr(r))
        return dict(pat=pat, kind=kind, q=q, r=r)

    def terms(self) -> dict:
        n = int(lib().orc_sa_num_terms(self._h))
        var = np.zeros(n, np.int64)
        src = np.zeros(n, np.int64)
        k = np.zeros(n, np.int32)
        nn = np.zeros(n, np.int32)
        d = np.zeros(n, np.int32)
        side = np.zeros(n, np.int32)
        lib().orc_sa_terms(self._h, _ptr(var), _ptr(src), _ptr(k), _ptr(nn), _ptr(d), _ptr(side))
        re = np.zeros(n)
        im = np.zeros(n)
        lib().orc_sa_term_coefs(self._h, _ptr(re), _ptr(im))
        return dict(var=var, src=src, k=k, n=nn, dir=d, side=side, coef=re + 1j * im)

    # ---- dynamics -------------------------------------------------------
    def zeros(self) -> np.ndarray:
        return np.zeros(self.nvar, dtype=np.complex128)

    def rhs(self, x: np.ndarray) -> np.ndarray:
        x = np.ascontiguousarray(x, dtype=np.complex128)
        dx = np.empty_like(x)
        lib().orc_sa_rhs(self._h, _ptr(x), _ptr(dx))
        return dx

    def rhs_at(self, x: np.ndarray, idx) -> np.ndarray:
        x = np.ascontiguousarray(x, dtype=np.complex128)
        idx = np.ascontiguousarray(idx, dtype=np.int64)
        out = np.empty(idx.shape[0], dtype=np.complex128)
        lib().orc_sa_rhs_at(self._h, _ptr(x), _ptr(idx), int(idx.shape[0]), _ptr(out))
        return out

    def rk4(self, x: np.ndarray, dt: float, nsteps: int) -> np.ndarray:
        y = np.array(x, dtype=np.complex128, copy=True)
        lib().orc_sa_rk4(self._h, _ptr(y), float(dt), int(nsteps))
        return y

    def observables(self, x: np.ndarray) -> np.ndarray:
        x = np.ascontiguousarray(x, dtype=np.complex128)
        out = np.zeros(8)
        lib().orc_sa_observables(self._h, _ptr(x), _ptr(out))
        return out

    def propagate(self, x: np.ndarray, dt: float, nsteps: int, obs_every: int):
        y = np.array(x, dtype=np.complex128, copy=True)
        rows = 1 + (nsteps + obs_every - 1) // obs_every
        obs = np.zeros((rows, 8))
        lib().orc_sa_propagate(self._h, _ptr(y), float(dt), int(nsteps), int(obs_every), _ptr(obs))
        return y, obs

    def _phys_categories(self):
        """Categories of the physical representative (the empty pattern) with
        the basis index of a molecule in each: distinguished molecules 1..d
        (named "d" when d = 1, else "1".."d"), then the zero category "0" of
        the other N - d when N > d."""
        names = ["d"] if self.d == 1 else [str(j) for j in range(1, self.d + 1)]
        cats = [(n, j + 1) for j, n in enumerate(names)]
        if self.N > self.d:
            cats.append(("0", self.d + 1))
        return cats

    def rho0_index(self) -> dict:
        """Indices of the physical representative's variables in the canonical
        layout (Z; X_q; Y_q; P_q; S_qr row-major; T), keyed by kind and
        category name, e.g. Z, X0, Y0, P0, T0 for d = 0."""
        cats = self._phys_categories()
        G = len(cats)
        idx = {"Z": 0}
        for q, (n, _) in enumerate(cats, 1):
            idx["X" + n], idx["Y" + n], idx["P" + n] = q, G + q, 2 * G + q
        for q, (n, _) in enumerate(cats, 1):
            for r, (n2, _) in enumerate(cats, 1):
                if r != q:
                    idx["S" + n + n2] = 3 * G + 1 + (q - 1) * (G - 1) + (r - 1) - (1 if r > q else 0)
        if self.N - self.d >= 2:
            idx["T0"] = (G + 1) ** 2  # only the zero category has M >= 2
        return idx

    def initial_state_dense(self, rho) -> np.ndarray:
        """Factorised initial hierarchy from a dense (N+1)x(N+1) rho_S in the
        basis {c, e_1 .. e_N}, invariant under permutations of the molecules
        it does not distinguish (molecules d+1..N)."""
        rho = np.asarray(rho, complex)
        x = self.zeros()
        rep = dict(self._phys_categories())
        for k, j in self.rho0_index().items():
            if k == "Z":
                e = (0, 0)
            elif k == "T0":
                e = (self.d + 1, self.d + 2)
            elif k[0] == "X":
                e = (rep[k[1:]], 0)
            elif k[0] == "Y":
                e = (0, rep[k[1:]])
            elif k[0] == "P":
                e = (rep[k[1:]], rep[k[1:]])
            else:
                e = (rep[k[1]], rep[k[2]])
            x[j] = rho[e]
        return x

    def initial_state(self, Z, X0, Y0, P0, T0=0.0) -> np.ndarray:
        """Factorised initial hierarchy (Eqs. factorized-initial-zero/higher)."""
        x = self.zeros()
        ix = self.rho0_index()
        x[ix["Z"]], x[ix["X0"]], x[ix["Y0"]], x[ix["P0"]] = Z, X0, Y0, P0
        if "T0" in ix:
            x[ix["T0"]] = T0
        return x


class Conventional:
    """Conventional scaled HEOM oracle (O-1).  State: (nado, N+1, N+1)."""

    def __init__(self, N, m, L, bath, detuning=0.0, g=0.0, kappa=0.0, term=0.0):
        self.N, self.m, self.L = int(N), int(m), int(L)
        self.params = make_params(N, m, L, bath, detuning, g, kappa, term)
        self._h = lib().orc_conv_create(ctypes.byref(self.params))
        if not self._h:
            raise ValueError("oracle rejected the parameters")
        self.nado = int(lib().orc_conv_num_ados(self._h))
        self.D = self.N + 1

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.orc_conv_destroy(h)
            self._h = None

    def labels(self) -> np.ndarray:
        out = np.zeros((self.nado, self.N * self.m), np.uint8)
        lib().orc_conv_labels(self._h, _ptr(out))
        return out

    def zeros(self) -> np.ndarray:
        return np.zeros((self.nado, self.D, self.D), dtype=np.complex128)

    def rhs(self, x):
        x = np.ascontiguousarray(x, dtype=np.complex128)
        dx = np.empty_like(x)
        lib().orc_conv_rhs(self._h, _ptr(x), _ptr(dx))
        return dx

    def rk4(self, x, dt, nsteps):
        y = np.array(x, dtype=np.complex128, copy=True)
        lib().orc_conv_rk4(self._h, _ptr(y), float(dt), int(nsteps))
        return y

    def map_to(self, sa: SA) -> np.ndarray:
        out = np.zeros((self.nado, self.D, self.D), np.int64)
        lib().orc_conv_to_sa(self._h, sa._h, _ptr(out))
        return out
