"""ctypes loader for libkmc_gb300.so (the C ABI of include/kmc.h).

There is no CPU fallback: if the shared library is missing or cannot be
loaded, every entry point raises.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

_LIB = None

# kmc_status codes
KMC_OK = 0
KMC_EINVAL = -1
KMC_ENOMEM = -2
KMC_ECUDA = -3
KMC_ENOTBALANCED = -4
KMC_ETIMEOUT = -5
KMC_EDEVICE = -6

STATUS_NAMES = {0: "KMC_OK", -1: "KMC_EINVAL", -2: "KMC_ENOMEM", -3: "KMC_ECUDA",
                -4: "KMC_ENOTBALANCED", -5: "KMC_ETIMEOUT", -6: "KMC_EDEVICE"}

#: every symbol include/kmc.h declares
EXPORTS = [
    "kmc_create_lattice", "kmc_set_rates", "kmc_set_rate_table", "kmc_run_schedule",
    "kmc_observables", "kmc_grad", "kmc_grad_nu", "kmc_lr_estimate", "kmc_lr_observable", "kmc_enable_grad", "kmc_reset", "kmc_sync",
    "kmc_domain_state", "kmc_get_rate_table", "kmc_rate_table_error", "kmc_set_launch", "kmc_get_launch", "kmc_set_replica_params", "kmc_set_observation", "kmc_set_horizon",
    "kmc_debug_barrier", "kmc_run_schedule_noalloc", "kmc_profile", "kmc_profile_read", "kmc_profile_polls", "kmc_kernel_launches", "kmc_domain_side", "kmc_last_error", "kmc_destroy", "kmc_version",
    "kmc_ring_create", "kmc_ring_set_rates", "kmc_ring_run", "kmc_ring_state", "kmc_ring_last_error", "kmc_ring_destroy",
    "kmc_part_create", "kmc_part_set_rates", "kmc_part_run", "kmc_part_state", "kmc_part_last_error", "kmc_part_destroy",
]


class KmcError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, str(status)), message))
        self.status = status


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load the library (building it first if allowed and needed)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = lib_path()
    if build_if_missing and not _build.up_to_date():
        _build.build()
    if not os.path.exists(path):
        raise ImportError("libkmc_gb300.so is not built (%s); run python -m paper_1403_4674_gb300.build" % path)
    L = ctypes.CDLL(path)
    vp = ctypes.c_void_p
    i32, i64, u64, dbl = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
    P = ctypes.POINTER
    L.kmc_create_lattice.argtypes = [P(vp), i32, P(i32), i32, i32, i32, P(u64), vp, vp]
    L.kmc_set_rates.argtypes = [vp, dbl, P(dbl), P(dbl), dbl, i32]
    L.kmc_set_rate_table.argtypes = [vp, dbl, P(dbl), P(dbl), dbl, P(dbl)]
    L.kmc_run_schedule.argtypes = [vp, i64, i32, i32, i32, vp, vp]
    L.kmc_observables.argtypes = [vp, P(dbl), P(dbl), P(dbl), P(i64), P(i64)]
    L.kmc_grad.argtypes = [vp, vp, i32]
    L.kmc_grad_nu.argtypes = [vp, vp]
    L.kmc_lr_estimate.argtypes = [vp, vp, vp]
    L.kmc_lr_observable.argtypes = [vp, vp, i32, i32, vp]
    L.kmc_enable_grad.argtypes = [vp, i32]
    L.kmc_reset.argtypes = [vp, i32, vp]
    L.kmc_set_replica_params.argtypes = [vp, vp, vp]
    L.kmc_set_observation.argtypes = [vp, i32]
    L.kmc_set_horizon.argtypes = [vp, dbl]
    L.kmc_sync.argtypes = [vp]
    L.kmc_domain_state.argtypes = [vp, P(u64), P(i64), P(dbl)]
    L.kmc_get_rate_table.argtypes = [vp, i32, P(dbl), P(u64)]
    L.kmc_rate_table_error.argtypes = [vp, P(dbl)]
    L.kmc_set_launch.argtypes = [vp, i32, i32, i32]
    L.kmc_get_launch.argtypes = [vp, P(i32), P(i32), P(i32), P(i32), P(i32)]
    L.kmc_debug_barrier.argtypes = [vp, i32, i64]
    L.kmc_run_schedule_noalloc.argtypes = [i32, i32, i32, u64, dbl, dbl, dbl, dbl, i32, i64, i64, i32,
                                           i32, i32, vp, vp, vp, ctypes.c_char_p, i32]
    L.kmc_profile.argtypes = [vp, i32]
    L.kmc_profile_read.argtypes = [vp, P(dbl), P(i64)]
    L.kmc_profile_polls.argtypes = [vp, P(i64)]
    L.kmc_kernel_launches.argtypes = [vp]
    L.kmc_kernel_launches.restype = i64
    L.kmc_domain_side.argtypes = [vp]
    L.kmc_domain_side.restype = i32
    L.kmc_last_error.argtypes = [vp]
    L.kmc_last_error.restype = ctypes.c_char_p
    L.kmc_destroy.argtypes = [vp]
    L.kmc_destroy.restype = None
    L.kmc_version.argtypes = []
    L.kmc_version.restype = i32
    L.kmc_ring_create.argtypes = [P(vp), i32, i32, i32, i32, P(u64), P(u64), vp]
    L.kmc_ring_set_rates.argtypes = [vp, dbl, P(dbl), P(dbl), dbl, i32]
    L.kmc_ring_run.argtypes = [vp, i64, i32, i32, i32, vp, vp, vp, vp]
    L.kmc_ring_state.argtypes = [vp, P(u64), P(u64), P(i64), P(i64), P(dbl)]
    L.kmc_ring_last_error.argtypes = [vp]
    L.kmc_ring_last_error.restype = ctypes.c_char_p
    L.kmc_ring_destroy.argtypes = [vp]
    L.kmc_ring_destroy.restype = None
    L.kmc_part_create.argtypes = [P(vp), i32, i32, i32, i32, i32, P(u64), vp, vp]
    L.kmc_part_set_rates.argtypes = [vp, dbl, P(dbl), P(dbl), dbl, i32]
    L.kmc_part_run.argtypes = [vp, i64, i32, i32, i32, vp, vp]
    L.kmc_part_state.argtypes = [vp, P(u64), P(i64), P(i64), P(dbl)]
    L.kmc_part_last_error.argtypes = [vp]
    L.kmc_part_last_error.restype = ctypes.c_char_p
    L.kmc_part_destroy.argtypes = [vp]
    L.kmc_part_destroy.restype = None
    for name in EXPORTS:
        fn = getattr(L, name)
        if fn.restype is ctypes.c_int:  # default restype: kmc_status
            fn.restype = ctypes.c_int
    _LIB = L
    return L
