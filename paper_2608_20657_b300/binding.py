"""Thin Python binding of the C ABI in ``include/sa_heom.h`` (ctypes).

Argument marshalling only: every step of the hot path runs in the CUDA
kernels of ``libsaheom.so``.  Device buffers are plain device pointers, in
practice the ``data_ptr()`` of torch tensors, and streams are
``torch.cuda.Stream.cuda_stream`` values; PyTorch is used for device memory
and streams and nothing else.  If the shared library is missing, importing
this module raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsaheom.so")
MAXM = 8
MAXD = 3         # SA_HEOM_MAXD
PHYS_SLOTS = 32  # SA_HEOM_PHYS_SLOTS
NOALLOC_MAX_INSTANCES = 4096  # SA_HEOM_NOALLOC_MAX_INSTANCES

SA_FP64, SA_FP32_AUX = 0, 1
SA_BUILD_DEVICE, SA_BUILD_HOST_ONLY, SA_BUILD_ADJOINT_REPS, SA_BUILD_PACK_INSTANCES = 0, 1, 2, 4
SA_KERNEL_RECORDS, SA_KERNEL_LISTS, SA_KERNEL_ELL = 0, 1, 2
SA_DEBUG_EXPIRE_WAIT, SA_DEBUG_CORRUPT_RECORD, SA_DEBUG_CHECK_INDICES, SA_DEBUG_CORRUPT_LIST = 1, 2, 4, 8
SA_TUNE_FORCE = 1
INIT_KINDS = {"cavity": 0, "bright": 1, "up": 2, "lp": 3, "random": 4, "localised": 5, "superposed": 6}
BATH_HIGH_T, BATH_MATSUBARA, BATH_PADE = 0, 1, 2
ERRORS = {0: "SA_OK", -1: "SA_ERR_INVALID_ARG", -2: "SA_ERR_UNSUPPORTED", -3: "SA_ERR_OOM",
          -4: "SA_ERR_CUDA", -5: "SA_ERR_TIMEOUT", -6: "SA_ERR_NUMERIC", -7: "SA_ERR_STATE"}


class SaHeomError(RuntimeError):
    def __init__(self, code: int, where: str, detail: str):
        super().__init__(f"{where}: {ERRORS.get(code, code)} ({detail})")
        self.code = code


class Params(ctypes.Structure):
    """sa_params of include/sa_heom.h."""
    _fields_ = [
        ("N", ctypes.c_int64), ("m", ctypes.c_int32), ("L", ctypes.c_int32),
        ("detuning", ctypes.c_double), ("g", ctypes.c_double), ("kappa", ctypes.c_double),
        ("c_re", ctypes.c_double * MAXM), ("c_im", ctypes.c_double * MAXM),
        ("cc_re", ctypes.c_double * MAXM), ("cc_im", ctypes.c_double * MAXM),
        ("nu_re", ctypes.c_double * MAXM), ("nu_im", ctypes.c_double * MAXM),
        ("term", ctypes.c_double), ("d", ctypes.c_int32), ("reserved", ctypes.c_int32),
    ]

    def bath(self) -> dict:
        m = self.m
        return {"c": np.array([complex(self.c_re[k], self.c_im[k]) for k in range(m)]),
                "cc": np.array([complex(self.cc_re[k], self.cc_im[k]) for k in range(m)]),
                "nu": np.array([complex(self.nu_re[k], self.nu_im[k]) for k in range(m)])}


class Counts(ctypes.Structure):
    _fields_ = [("log10_conventional_ados", ctypes.c_double), ("n_vectors", ctypes.c_int64),
                ("n_patterns", ctypes.c_int64), ("n_vars", ctypes.c_int64), ("n_categories", ctypes.c_int64),
                ("n_records", ctypes.c_int64), ("n_terms", ctypes.c_int64), ("state_bytes", ctypes.c_int64),
                ("conventional_ados", ctypes.c_uint64)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"native library {LIB_PATH} is missing; run paper_2608_20657_b300._build.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
        P = ctypes.POINTER
        sig = {
            "sa_bath_drude_lorentz": [dbl, dbl, dbl, i32, i32, dbl, P(Params)],
            "sa_bath_terminator": [dbl, dbl, dbl, i32, P(dbl)],
            "sa_heom_counts": [P(Params), P(Counts)],
            "sa_heom_build": [P(Params), i32, i32, i32, P(vp)],
            "sa_heom_build_representatives": [P(Params), i32, i32, P(vp)],
            "sa_heom_init_representatives": [vp, vp, vp],
            "sa_heom_reconstruct_dense": [vp, vp, vp, vp, vp],
            "sa_heom_info": [vp, i32, P(Counts)],
            "sa_heom_var_offset": [vp, i32, P(i64)],
            "sa_heom_state_index": [vp, i32, i64, P(i64)],
            "sa_heom_dump_packs": [vp, vp, vp, vp, vp],
            "sa_heom_dump_vectors": [vp, i32, vp],
            "sa_heom_dump_patterns": [vp, i32, vp, vp, vp, vp, vp, vp, vp],
            "sa_heom_dump_categories": [vp, i32, vp, vp],
            "sa_heom_dump_terms": [vp, i32, vp, vp, vp, vp, vp, vp],
            "sa_heom_state_bytes": [vp, P(ctypes.c_size_t)],
            "sa_heom_init_state": [vp, vp, vp, vp],
            "sa_heom_init_physical": [vp, vp, vp, vp],
            "sa_heom_state_upload": [vp, vp, vp, vp],
            "sa_heom_state_download": [vp, vp, vp, vp],
            "sa_heom_rhs": [vp, vp, vp, vp],
            "sa_heom_step": [vp, vp, dbl, vp],
            "sa_heom_propagate": [vp, vp, dbl, i64, i64, vp, vp],
            "sa_heom_prepare": [vp, vp, dbl, i64, i64],
            "sa_heom_observables": [vp, vp, vp, vp],
            "sa_heom_set_tuning": [vp, i32, i32, i32],
            "sa_heom_autotune": [vp, vp, vp, vp],
            "sa_heom_autotune_ex": [vp, vp, vp, i32, vp],
            "sa_heom_tuning_key": [vp, P(ctypes.c_uint64)],
            "sa_heom_tuning_cache_save": [ctypes.c_char_p],
            "sa_heom_tuning_cache_load": [ctypes.c_char_p],
            "sa_heom_tuning_cache_clear": [],
            "sa_heom_tuning_cache_size": [P(i64)],
            "sa_heom_set_kernel": [vp, i32],
            "sa_heom_dump_lists": [vp, vp, vp, vp, vp, vp, vp, vp, vp, vp],
            "sa_heom_dump_ell": [vp, vp, vp, vp, vp, vp, vp],
            "sa_heom_get_tuning": [vp, vp],
            "sa_heom_launches_per_step": [vp],
            "sa_heom_device_error": [vp, vp],
            "sa_heom_observables_noalloc": [vp, vp, vp, vp],
            "sa_heom_validate": [vp],
            "sa_heom_initial_vars": [P(Params), i32, vp, vp, P(i32)],
            "sa_unit_cm_to_rad_fs": [dbl, P(dbl)],
            "sa_unit_kT_rad_fs": [dbl, P(dbl)],
            "sa_heom_dump_coefficients": [vp, i32, vp, vp],
            "sa_heom_config_hash": [vp, P(ctypes.c_uint64)],
            "sa_heom_checkpoint_bytes": [vp, P(ctypes.c_size_t)],
            "sa_heom_checkpoint_save": [vp, vp, i64, vp, ctypes.c_size_t, vp],
            "sa_heom_checkpoint_load": [vp, vp, ctypes.c_size_t, vp, P(i64), vp],
            "sa_heom_set_debug": [vp, i32],
            "sa_conv_build": [P(Params), P(vp)],
            "sa_conv_info": [vp, P(i64), P(ctypes.c_size_t)],
            "sa_conv_labels": [vp, vp],
            "sa_conv_set_rho0": [vp, vp, vp, vp],
            "sa_conv_rhs": [vp, vp, vp, vp],
            "sa_conv_step": [vp, vp, dbl, i64, vp],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = i32
        L.sa_heom_destroy.argtypes = [vp]
        L.sa_heom_destroy.restype = None
        L.sa_heom_strerror.argtypes = [i32]
        L.sa_heom_strerror.restype = ctypes.c_char_p
        L.sa_heom_last_error.argtypes = []
        L.sa_heom_last_error.restype = ctypes.c_char_p
        L.sa_conv_destroy.argtypes = [vp]
        L.sa_conv_destroy.restype = None
        L.sa_conv_last_error.argtypes = []
        L.sa_conv_last_error.restype = ctypes.c_char_p
        _lib = L
    return _lib


def exported_symbols() -> list[str]:
    return ["sa_bath_drude_lorentz", "sa_bath_terminator", "sa_heom_counts", "sa_heom_build",
            "sa_heom_build_representatives", "sa_heom_init_representatives", "sa_heom_reconstruct_dense",
            "sa_heom_destroy", "sa_heom_info",
            "sa_heom_var_offset", "sa_heom_state_index", "sa_heom_dump_packs", "sa_heom_dump_vectors", "sa_heom_dump_patterns", "sa_heom_dump_categories",
            "sa_heom_dump_terms", "sa_heom_dump_coefficients", "sa_heom_state_bytes", "sa_heom_init_state", "sa_heom_init_physical",
            "sa_heom_state_upload",
            "sa_heom_state_download", "sa_heom_rhs", "sa_heom_step", "sa_heom_propagate", "sa_heom_observables",
            "sa_heom_set_tuning", "sa_heom_autotune", "sa_heom_autotune_ex", "sa_heom_tuning_key",
            "sa_heom_tuning_cache_save", "sa_heom_tuning_cache_load", "sa_heom_tuning_cache_clear",
            "sa_heom_tuning_cache_size", "sa_heom_set_kernel", "sa_heom_get_tuning", "sa_heom_prepare", "sa_heom_dump_lists", "sa_heom_dump_ell",
            "sa_heom_launches_per_step", "sa_heom_device_error",
            "sa_heom_observables_noalloc", "sa_heom_initial_vars", "sa_unit_cm_to_rad_fs", "sa_unit_kT_rad_fs",
            "sa_heom_validate", "sa_heom_set_debug", "sa_heom_config_hash",
            "sa_heom_checkpoint_bytes", "sa_heom_checkpoint_save", "sa_heom_checkpoint_load", "sa_heom_strerror", "sa_heom_last_error", "sa_conv_build",
            "sa_conv_destroy", "sa_conv_info", "sa_conv_labels", "sa_conv_set_rho0", "sa_conv_rhs", "sa_conv_step",
            "sa_conv_last_error"]


def _check(rc: int, where: str):
    if rc != 0:
        raise SaHeomError(rc, where, lib().sa_heom_last_error().decode())


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _dev(t) -> ctypes.c_void_p:
    """Device pointer of a torch tensor (or an int address)."""
    return ctypes.c_void_p(t if isinstance(t, int) else t.data_ptr())


def _stream(stream) -> ctypes.c_void_p:
    if stream is None:
        import torch

        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return ctypes.c_void_p(stream if isinstance(stream, int) else stream.cuda_stream)


def make_params(N, m=None, L=0, bath=None, detuning=0.0, g=0.0, kappa=0.0, term=0.0, d=0) -> Params:
    """sa_params from a bath dict {c, cc, nu} (complex arrays of length m);
    term: terminator strength Delta (0: off, see bath_terminator); d: 1 keeps
    molecules 1..d (d <= 3) out of the permutation symmetry."""
    p = Params()
    c = np.asarray(bath["c"], complex)
    cc = np.asarray(bath["cc"], complex)
    nu = np.asarray(bath["nu"], complex)
    m = len(c) if m is None else m
    p.N, p.m, p.L = int(N), int(m), int(L)
    p.detuning, p.g, p.kappa, p.term = float(detuning), float(g), float(kappa), float(term)
    p.d = int(d)
    for k in range(m):
        p.c_re[k], p.c_im[k] = c[k].real, c[k].imag
        p.cc_re[k], p.cc_im[k] = cc[k].real, cc[k].imag
        p.nu_re[k], p.nu_im[k] = nu[k].real, nu[k].imag
    return p


def bath_drude_lorentz(lam, gam, kT, scheme=BATH_MATSUBARA, n_poles=1, sigma=0.0) -> dict:
    """sa_bath_drude_lorentz: {c, cc, nu} of Eq. BCF-exp."""
    p = Params()
    _check(lib().sa_bath_drude_lorentz(lam, gam, kT, scheme, n_poles, sigma, ctypes.byref(p)), "sa_bath_drude_lorentz")
    return p.bath()


def bath_terminator(lam, gam, kT, n_matsubara) -> float:
    """sa_bath_terminator: Delta of the Matsubara poles beyond n_matsubara."""
    out = ctypes.c_double()
    _check(lib().sa_bath_terminator(lam, gam, kT, int(n_matsubara), ctypes.byref(out)), "sa_bath_terminator")
    return out.value


def initial_vars(p: Params, kind: str, draws: dict | None = None) -> np.ndarray:
    """sa_heom_initial_vars: the physical representative's variables of a
    factorised initial state (canonical layout, complex)."""
    d = np.zeros(9)
    if draws is not None:
        d[:8] = np.asarray(draws["A"], complex).reshape(4).view(np.float64)
        d[8] = float(draws["w_dark"])
    out = np.zeros(20)
    n = ctypes.c_int()
    _check(lib().sa_heom_initial_vars(ctypes.byref(p), INIT_KINDS[kind], _ptr(d) if draws is not None else None,
                                      _ptr(out), ctypes.byref(n)), "sa_heom_initial_vars")
    return out[:2 * n.value].view(complex).copy()


def unit_cm_to_rad_fs(e_cm: float) -> float:
    out = ctypes.c_double()
    _check(lib().sa_unit_cm_to_rad_fs(float(e_cm), ctypes.byref(out)), "sa_unit_cm_to_rad_fs")
    return out.value


def unit_kT_rad_fs(T_K: float) -> float:
    out = ctypes.c_double()
    _check(lib().sa_unit_kT_rad_fs(float(T_K), ctypes.byref(out)), "sa_unit_kT_rad_fs")
    return out.value


def tuning_cache_save(path: str):
    _check(lib().sa_heom_tuning_cache_save(str(path).encode()), "sa_heom_tuning_cache_save")


def tuning_cache_load(path: str):
    _check(lib().sa_heom_tuning_cache_load(str(path).encode()), "sa_heom_tuning_cache_load")


def tuning_cache_clear():
    _check(lib().sa_heom_tuning_cache_clear(), "sa_heom_tuning_cache_clear")


def tuning_cache_size() -> int:
    out = ctypes.c_int64()
    _check(lib().sa_heom_tuning_cache_size(ctypes.byref(out)), "sa_heom_tuning_cache_size")
    return int(out.value)


def counts(p: Params) -> dict:
    c = Counts()
    _check(lib().sa_heom_counts(ctypes.byref(p), ctypes.byref(c)), "sa_heom_counts")
    return c.as_dict()


class Heom:
    """A built batch of instances (sa_heom handle)."""

    def __init__(self, params, precision: int = SA_FP64, host_only: bool = False, representatives: bool = False,
                 adjoint: bool = False, pack: bool = False):
        """representatives: params is one d = 0 set; the handle is the batch of
        its representative propagations (sa_heom_build_representatives);
        adjoint: leave out the |c><e_1| propagation (SA_BUILD_ADJOINT_REPS);
        pack: the packed device layout (SA_BUILD_PACK_INSTANCES)."""
        flags = SA_BUILD_HOST_ONLY if host_only else SA_BUILD_DEVICE
        if pack:
            assert not representatives
            flags |= SA_BUILD_PACK_INSTANCES
        h = ctypes.c_void_p()
        if representatives:
            p = params[0] if isinstance(params, (list, tuple)) else params
            flags |= SA_BUILD_ADJOINT_REPS if adjoint else 0
            _check(lib().sa_heom_build_representatives(ctypes.byref(p), precision, flags, ctypes.byref(h)),
                   "sa_heom_build_representatives")
            params = []
            ds = [0, 1, 1, 1, 2] if p.N >= 2 else [0, 1, 1, 1]
            if adjoint:
                del ds[2]
            for d in ds:
                q = Params.from_buffer_copy(p)
                q.d = d
                params.append(q)
        else:
            if isinstance(params, Params):
                params = [params]
            arr = (Params * len(params))(*params)
            _check(lib().sa_heom_build(arr, len(params), precision, flags, ctypes.byref(h)), "sa_heom_build")
        self.params = list(params)
        self._h = h
        self.count = len(self.params)
        self.precision = precision
        tot = self.info()
        self.n_vars = tot["n_vars"]
        self.n_patterns = tot["n_patterns"]
        sb = ctypes.c_size_t()
        _check(lib().sa_heom_state_bytes(self._h, ctypes.byref(sb)), "sa_heom_state_bytes")
        self.state_bytes = int(sb.value)

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().sa_heom_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- tables ------------------------------------------------------
    def info(self, inst: int = -1) -> dict:
        c = Counts()
        _check(lib().sa_heom_info(self._h, inst, ctypes.byref(c)), "sa_heom_info")
        return c.as_dict()

    def var_offset(self, inst: int) -> int:
        v = ctypes.c_int64()
        _check(lib().sa_heom_var_offset(self._h, inst, ctypes.byref(v)), "sa_heom_var_offset")
        return v.value

    def dump_vectors(self, inst: int = 0) -> np.ndarray:
        i = self.info(inst)
        out = np.zeros((i["n_vectors"], self.params[inst].m), np.uint8)
        _check(lib().sa_heom_dump_vectors(self._h, inst, _ptr(out)), "sa_heom_dump_vectors")
        return out

    def dump_patterns(self, inst: int = 0) -> dict:
        i = self.info(inst)
        P, L = i["n_patterns"], self.params[inst].L + self.params[inst].d  # id list width L + d
        tier, r, G, h = (np.zeros(P, np.int32) for _ in range(4))
        var_off = np.zeros(P + 1, np.int64)
        cat_off = np.zeros(P + 1, np.int64)
        ids = np.zeros((P, max(L, 1)), np.int32)
        _check(lib().sa_heom_dump_patterns(self._h, inst, _ptr(tier), _ptr(r), _ptr(G), _ptr(h), _ptr(var_off),
                                           _ptr(cat_off), _ptr(ids)), "sa_heom_dump_patterns")
        nc = i["n_categories"]
        vec_id = np.zeros(max(nc, 1), np.int32)
        mult = np.zeros(max(nc, 1), np.int64)
        _check(lib().sa_heom_dump_categories(self._h, inst, _ptr(vec_id), _ptr(mult)), "sa_heom_dump_categories")
        return dict(tier=tier, r=r, G=G, h=h, var_off=var_off, cat_off=cat_off, ids=ids[:, :L],
                    cat_id=vec_id[:nc], cat_M=mult[:nc])

    def dump_terms(self, inst: int = 0) -> dict:
        n = self.info(inst)["n_terms"]
        var, src = np.zeros(n, np.int64), np.zeros(n, np.int64)
        k, nn, d, s = (np.zeros(n, np.int32) for _ in range(4))
        _check(lib().sa_heom_dump_terms(self._h, inst, _ptr(var), _ptr(src), _ptr(k), _ptr(nn), _ptr(d), _ptr(s)),
               "sa_heom_dump_terms")
        return dict(var=var, src=src, k=k, n=nn, dir=d, side=s)

    def dump_coefficients(self, inst: int = 0) -> tuple[np.ndarray, np.ndarray]:
        """Row and column coefficients (complex) by coefficient id ((k * 32) + n) * 2 + raise."""
        n = 2 * MAXM * 32 * 2
        row, col = np.zeros(n), np.zeros(n)
        _check(lib().sa_heom_dump_coefficients(self._h, inst, _ptr(row), _ptr(col)), "sa_heom_dump_coefficients")
        return row[0::2] + 1j * row[1::2], col[0::2] + 1j * col[1::2]

    # ---- device state -------------------------------------------------
    def new_state(self, device="cuda"):
        import torch

        return torch.zeros(self.state_bytes, dtype=torch.uint8, device=device)

    def init_state(self, state, rho0, stream=None):
        """rho0: (count, 5) complex: Z, X_0, Y_0, P_0, T_0."""
        r = np.zeros((self.count, 5), complex)
        r[:] = np.asarray(rho0, complex).reshape(-1, 5) if np.ndim(rho0) > 1 else np.asarray(rho0, complex)
        flat = np.ascontiguousarray(r.view(np.float64).reshape(-1))
        _check(lib().sa_heom_init_state(self._h, _ptr(flat), _dev(state), _stream(stream)), "sa_heom_init_state")

    def init_physical(self, state, phys, stream=None):
        """phys: (count, n) complex, n <= 32: each instance's physical
        representative in the canonical layout (Z, X_q, Y_q, P_q, S_qr, T)."""
        ph = np.asarray(phys, complex)
        ph = ph.reshape(self.count, -1) if ph.ndim > 1 else ph.reshape(1, -1)
        assert ph.shape[1] <= PHYS_SLOTS
        r = np.zeros((self.count, PHYS_SLOTS), complex)
        r[:, :ph.shape[1]] = ph
        flat = np.ascontiguousarray(r.view(np.float64).reshape(-1))
        _check(lib().sa_heom_init_physical(self._h, _ptr(flat), _dev(state), _stream(stream)), "sa_heom_init_physical")

    def init_representatives(self, state, stream=None):
        """sa_heom_init_representatives: each instance starts from its unit operator."""
        _check(lib().sa_heom_init_representatives(self._h, _dev(state), _stream(stream)), "sa_heom_init_representatives")

    def reconstruct_dense(self, state, rho0, out=None, stream=None):
        """sa_heom_reconstruct_dense: rho_S(t) for the dense initial operator
        rho0 ((N+1, N+1) complex128 torch tensor on the device) from the
        representatives' current state; returns out (allocated if None)."""
        import torch

        assert rho0.dtype == torch.complex128 and rho0.is_contiguous()
        if out is None:
            out = torch.empty_like(rho0)
        _check(lib().sa_heom_reconstruct_dense(self._h, _dev(state), ctypes.c_void_p(rho0.data_ptr()),
                                               ctypes.c_void_p(out.data_ptr()), _stream(stream)),
               "sa_heom_reconstruct_dense")
        return out

    def upload(self, state, x: np.ndarray, stream=None):
        x = np.ascontiguousarray(x, np.complex128)
        assert x.shape == (self.n_vars,)
        _check(lib().sa_heom_state_upload(self._h, _ptr(x), _dev(state), _stream(stream)), "sa_heom_state_upload")

    def download(self, state, stream=None, out: np.ndarray | None = None) -> np.ndarray:
        """The state as complex128; `out` (contiguous complex128 of n_vars, for
        instance a view of page-locked memory) receives it if given."""
        if out is None:
            x = np.zeros(self.n_vars, np.complex128)
        else:
            x = out
            assert x.dtype == np.complex128 and x.shape == (self.n_vars,) and x.flags.c_contiguous
        _check(lib().sa_heom_state_download(self._h, _dev(state), _ptr(x), _stream(stream)), "sa_heom_state_download")
        return x

    def rhs(self, x, dx, stream=None):
        _check(lib().sa_heom_rhs(self._h, _dev(x), _dev(dx), _stream(stream)), "sa_heom_rhs")

    def step(self, state, dt: float, stream=None):
        _check(lib().sa_heom_step(self._h, _dev(state), float(dt), _stream(stream)), "sa_heom_step")

    def propagate(self, state, dt: float, nsteps: int, obs_every: int = 0, observe: bool = True, stream=None):
        if not observe:
            _check(lib().sa_heom_propagate(self._h, _dev(state), float(dt), int(nsteps), int(obs_every), None,
                                           _stream(stream)), "sa_heom_propagate")
            return None
        oe = obs_every if obs_every > 0 else max(nsteps, 1)
        rows = 1 + (nsteps + oe - 1) // oe
        out = np.zeros((rows, self.count, 8))
        _check(lib().sa_heom_propagate(self._h, _dev(state), float(dt), int(nsteps), int(oe), _ptr(out),
                                       _stream(stream)), "sa_heom_propagate")
        return out

    def prepare(self, state, dt: float, nsteps: int, obs_every: int = 0):
        """Build now the CUDA graphs a propagate of nsteps (observables every
        obs_every steps; 0 = none) will replay."""
        _check(lib().sa_heom_prepare(self._h, _dev(state), float(dt), int(nsteps), int(obs_every)), "sa_heom_prepare")

    def observables(self, state, stream=None) -> np.ndarray:
        out = np.zeros((self.count, 8))
        _check(lib().sa_heom_observables(self._h, _dev(state), _ptr(out), _stream(stream)), "sa_heom_observables")
        return out

    def observables_noalloc(self, state, stream=None) -> np.ndarray:
        """sa_heom_observables_noalloc: observables without any device allocation."""
        out = np.zeros((self.count, 8))
        _check(lib().sa_heom_observables_noalloc(self._h, _dev(state), _ptr(out), _stream(stream)),
               "sa_heom_observables_noalloc")
        return out

    def set_tuning(self, block=0, chunk=0, queue=-1):
        _check(lib().sa_heom_set_tuning(self._h, int(block), int(chunk), int(queue)), "sa_heom_set_tuning")

    def autotune(self, state, stream=None, force: bool = False):
        """sa_heom_autotune_ex: the cached tuning for this handle's key, or
        (force, or no entry) every variant timed and the winner cached."""
        best = (ctypes.c_int * 3)()
        _check(lib().sa_heom_autotune_ex(self._h, _dev(state), _stream(stream), SA_TUNE_FORCE if force else 0, best),
               "sa_heom_autotune_ex")
        return tuple(best)

    def tuning_key(self) -> int:
        out = ctypes.c_uint64()
        _check(lib().sa_heom_tuning_key(self._h, ctypes.byref(out)), "sa_heom_tuning_key")
        return int(out.value)

    def set_kernel(self, kernel: int):
        """SA_KERNEL_RECORDS or SA_KERNEL_LISTS (rebuilds the launch tables)."""
        _check(lib().sa_heom_set_kernel(self._h, int(kernel)), "sa_heom_set_kernel")

    def dump_lists(self) -> dict:
        """Host copy of the SA_KERNEL_LISTS tables (host-only handles)."""
        sizes = np.zeros(5, np.int64)
        _check(lib().sa_heom_dump_lists(self._h, _ptr(sizes), None, None, None, None, None, None, None, None),
               "sa_heom_dump_lists")
        ni, nr, rows, nlane, nu = (int(v) for v in sizes)
        out = dict(items=np.zeros((ni, 10), np.uint32), units=np.zeros((nu, 2), np.uint32),
                   lvd=np.zeros(nlane, np.uint32), lvj=np.zeros(nlane, np.uint8),
                   rbase=np.zeros(nr + 1, np.uint32), tidx=np.zeros(32 * rows, np.uint32),
                   tcid=np.zeros(32 * rows, np.uint16), opz=np.zeros(4, np.int32))
        _check(lib().sa_heom_dump_lists(self._h, _ptr(sizes), *(_ptr(out[k]) for k in
                                                                ("items", "units", "lvd", "lvj", "rbase", "tidx",
                                                                 "tcid", "opz"))), "sa_heom_dump_lists")
        return out

    def dump_packs(self) -> dict:
        """sa_heom_dump_packs: packs (base, n, cbase, lane0), lane instances
        and (host-only handles with list tables) the item blobs."""
        sizes = np.zeros(3, np.int64)
        _check(lib().sa_heom_dump_packs(self._h, _ptr(sizes), None, None, None), "sa_heom_dump_packs")
        npk, nl, nb = (int(v) for v in sizes)
        out = dict(packs=np.zeros((npk, 4), np.uint32), lanes=np.zeros(nl, np.uint32), blobs=np.zeros(nb, np.uint8))
        _check(lib().sa_heom_dump_packs(self._h, _ptr(sizes), _ptr(out["packs"]), _ptr(out["lanes"]),
                                        _ptr(out["blobs"])), "sa_heom_dump_packs")
        return out

    def state_index(self, inst: int, var: int) -> int:
        """sa_heom_state_index: element of the device state holding variable var of instance inst."""
        out = ctypes.c_int64()
        _check(lib().sa_heom_state_index(self._h, int(inst), int(var), ctypes.byref(out)), "sa_heom_state_index")
        return int(out.value)

    def dump_ell(self) -> dict:
        """Host copy of the SA_KERNEL_ELL tables (host-only handles)."""
        sizes = np.zeros(3, np.int64)
        _check(lib().sa_heom_dump_ell(self._h, _ptr(sizes), None, None, None, None, None), "sa_heom_dump_ell")
        nw, rows, nv = (int(v) for v in sizes)
        out = dict(wpat=np.zeros(nw, np.uint32), vword=np.zeros(nv, np.uint32), rbase=np.zeros(nw + 1, np.uint32),
                   tidx=np.zeros(32 * rows, np.uint32), tcid=np.zeros(32 * rows, np.uint16))
        _check(lib().sa_heom_dump_ell(self._h, _ptr(sizes), *(_ptr(out[k]) for k in
                                                              ("wpat", "vword", "rbase", "tidx", "tcid"))),
               "sa_heom_dump_ell")
        return out

    def tuning(self) -> dict:
        out = (ctypes.c_int * 4)()
        _check(lib().sa_heom_get_tuning(self._h, out), "sa_heom_get_tuning")
        return dict(block=out[0], chunk=out[1], queue=out[2], kernel=out[3])

    def device_error(self, stream=None):
        _check(lib().sa_heom_device_error(self._h, _stream(stream)), "sa_heom_device_error")

    def config_hash(self) -> int:
        """sa_heom_config_hash: hash of the precision, parameters and table layout version."""
        out = ctypes.c_uint64()
        _check(lib().sa_heom_config_hash(self._h, ctypes.byref(out)), "sa_heom_config_hash")
        return int(out.value)

    def checkpoint(self, state, step: int, stream=None) -> bytearray:
        """sa_heom_checkpoint_save into a new host buffer."""
        n = ctypes.c_size_t()
        _check(lib().sa_heom_checkpoint_bytes(self._h, ctypes.byref(n)), "sa_heom_checkpoint_bytes")
        buf = bytearray(n.value)
        cbuf = (ctypes.c_char * n.value).from_buffer(buf)
        _check(lib().sa_heom_checkpoint_save(self._h, _dev(state), int(step), ctypes.cast(cbuf, ctypes.c_void_p),
                                             n.value, _stream(stream)), "sa_heom_checkpoint_save")
        return buf

    def resume(self, state, buf, stream=None) -> int:
        """sa_heom_checkpoint_load: the saved state into `state`; returns the saved step index."""
        buf = bytearray(buf) if not isinstance(buf, bytearray) else buf
        cbuf = (ctypes.c_char * len(buf)).from_buffer(buf)
        step = ctypes.c_int64()
        _check(lib().sa_heom_checkpoint_load(self._h, ctypes.cast(cbuf, ctypes.c_void_p), len(buf), _dev(state),
                                             ctypes.byref(step), _stream(stream)), "sa_heom_checkpoint_load")
        return int(step.value)

    def validate(self):
        """sa_heom_validate: raises SaHeomError naming the first inconsistent table entry."""
        _check(lib().sa_heom_validate(self._h), "sa_heom_validate")

    def set_debug(self, flags: int):
        """sa_heom_set_debug (SA_DEBUG_EXPIRE_WAIT, SA_DEBUG_CORRUPT_RECORD)."""
        _check(lib().sa_heom_set_debug(self._h, int(flags)), "sa_heom_set_debug")

    def launches_per_step(self) -> int:
        return int(lib().sa_heom_launches_per_step(self._h))


def _check_conv(rc: int, where: str):
    if rc != 0:
        raise SaHeomError(rc, where, lib().sa_conv_last_error().decode())


class Conventional:
    """Conventional scaled HEOM on the GPU (sa_conv_* handle): dense ADOs."""

    def __init__(self, params: Params):
        h = ctypes.c_void_p()
        _check_conv(lib().sa_conv_build(ctypes.byref(params), ctypes.byref(h)), "sa_conv_build")
        self._h = h
        self.N, self.m = params.N, params.m
        self.D = self.N + 1
        n = ctypes.c_int64()
        sb = ctypes.c_size_t()
        _check_conv(lib().sa_conv_info(self._h, ctypes.byref(n), ctypes.byref(sb)), "sa_conv_info")
        self.nado, self.state_bytes = n.value, sb.value

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().sa_conv_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def labels(self) -> np.ndarray:
        out = np.zeros((self.nado, self.N * self.m), np.uint8)
        _check_conv(lib().sa_conv_labels(self._h, _ptr(out)), "sa_conv_labels")
        return out

    def new_state(self, device="cuda"):
        import torch

        return torch.zeros(self.state_bytes, dtype=torch.uint8, device=device)

    def set_rho0(self, state, rho0, stream=None):
        r = np.ascontiguousarray(np.asarray(rho0, np.complex128).reshape(self.D, self.D))
        _check_conv(lib().sa_conv_set_rho0(self._h, _ptr(r), _dev(state), _stream(stream)), "sa_conv_set_rho0")

    def rhs(self, x, dx, stream=None):
        _check_conv(lib().sa_conv_rhs(self._h, _dev(x), _dev(dx), _stream(stream)), "sa_conv_rhs")

    def step(self, state, dt: float, nsteps: int = 1, stream=None):
        _check_conv(lib().sa_conv_step(self._h, _dev(state), float(dt), int(nsteps), _stream(stream)), "sa_conv_step")

    def to_numpy(self, state) -> np.ndarray:
        return state.view(__import__("torch").float64).cpu().numpy().view(np.complex128).reshape(
            self.nado, self.D, self.D)
