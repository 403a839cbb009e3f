"""B300-native symmetry-adapted HEOM for the Holstein-Tavis-Cummings model
(Mondal & Huo, arXiv 2608.20657).

The hot path -- the matrix-free unique-variable right-hand side fused into
RK4 -- runs in the sm_103a kernels of ``libsaheom.so`` behind the C ABI of
``include/sa_heom.h``; :mod:`.binding` marshals arguments to it.
"""
from .binding import (SA_DEBUG_CHECK_INDICES, SA_DEBUG_CORRUPT_LIST, SA_DEBUG_CORRUPT_RECORD, SA_DEBUG_EXPIRE_WAIT, MAXD, NOALLOC_MAX_INSTANCES, PHYS_SLOTS, BATH_HIGH_T, BATH_MATSUBARA, BATH_PADE, SA_FP32_AUX, SA_FP64, SA_KERNEL_ELL, SA_KERNEL_LISTS, SA_KERNEL_RECORDS,
                      Conventional, Heom, Params, SaHeomError, bath_drude_lorentz, bath_terminator, counts, lib,
                      make_params)
from .problems import in_library_units, params_from, phys_vars, rho0_vars, theta

__all__ = ["Conventional", "Heom", "Params", "SaHeomError", "bath_drude_lorentz", "bath_terminator", "counts", "lib", "make_params", "params_from",
           "rho0_vars", "theta", "SA_FP64", "SA_FP32_AUX", "SA_KERNEL_RECORDS", "SA_KERNEL_LISTS", "SA_KERNEL_ELL", "SA_DEBUG_EXPIRE_WAIT", "SA_DEBUG_CORRUPT_RECORD", "SA_DEBUG_CHECK_INDICES", "SA_DEBUG_CORRUPT_LIST", "BATH_HIGH_T", "BATH_MATSUBARA", "BATH_PADE"]
