"""ctypes view of libucc.so (include/ucc.h).  Argument marshalling only.

The library must have been built (``paper_2301_05726_gb300.build.build()``);
there is no fallback: loading fails with an ImportError when it is missing.
"""
from __future__ import annotations

import ctypes
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libucc.so")

UCC_OK, UCC_EINVAL, UCC_ENOMEM, UCC_ECAPACITY, UCC_ETIMEOUT, UCC_ECUDA, UCC_ESTATE = range(7)
STATUS_NAMES = {0: "UCC_OK", 1: "UCC_EINVAL", 2: "UCC_ENOMEM", 3: "UCC_ECAPACITY", 4: "UCC_ETIMEOUT",
                5: "UCC_ECUDA", 6: "UCC_ESTATE"}

# Every symbol include/ucc.h declares.
EXPORTS = ["ucc_create", "ucc_set_theta", "ucc_set_options", "ucc_apply", "ucc_energy", "ucc_gradient",
           "ucc_get_wavefunction", "ucc_get_stats", "ucc_batch_run", "ucc_last_error", "ucc_destroy",
           "ucc_energy_static", "ucc_get_entropy"]


class Hamiltonian(ctypes.Structure):
    _fields_ = [("n_spatial", ctypes.c_int32), ("n_alpha", ctypes.c_int32), ("n_beta", ctypes.c_int32),
                ("e_nuc", ctypes.c_double), ("h", ctypes.POINTER(ctypes.c_double)),
                ("g", ctypes.POINTER(ctypes.c_double))]


class Ansatz(ctypes.Structure):
    _fields_ = [("n_exc", ctypes.c_int32), ("idx", ctypes.POINTER(ctypes.c_int32)),
                ("theta", ctypes.POINTER(ctypes.c_double))]


class Options(ctypes.Structure):
    _fields_ = [("n_max", ctypes.c_int64), ("n_cut", ctypes.c_int64), ("max_entries", ctypes.c_int64),
                ("probe_width", ctypes.c_int32), ("checkpoint_stride", ctypes.c_int32),
                ("tape_budget_mb", ctypes.c_int32), ("record_entropy", ctypes.c_int32),
                ("batch_wait_ms", ctypes.c_int32), ("batch_test_skip_block", ctypes.c_int32),
                ("batch_tiles", ctypes.c_int32), ("energy_route", ctypes.c_int32),
                ("energy_test_partitions", ctypes.c_int32), ("energy_test_buffer_records", ctypes.c_int32),
                ("rebuild_test_regions", ctypes.c_int32), ("pad_", ctypes.c_int32)]


class Stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in (
        "n_det", "rotations", "created", "dropped_new", "dropped_old", "cut", "peak_entries", "capacity_entries",
        "hash_slots", "rebuilds", "tape_entries", "kernel_launches", "scanned", "sigma_probes", "sigma_hits",
        "reverse_pairs", "recompute_scanned", "recompute_rotations", "recompute_created", "forward_launches",
        "reverse_launches", "probe_width", "reverse_scanned", "reverse_compactions")] + \
        [(n, ctypes.c_double) for n in ("apply_ms", "energy_ms", "reverse_ms", "forward_kernel_ms",
                                        "reverse_kernel_ms")] + [("batch_tiles", ctypes.c_int64)] + \
        [(n, ctypes.c_double) for n in ("cut_ms", "rebuild_ms")] + [("energy_route", ctypes.c_int64)]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


class UCCError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None


def load(path: str = LIB_PATH):
    """Load libucc.so and declare its signatures (no build, no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libucc.so not built at {path}; run paper_2301_05726_gb300.build.build()")
    lib = ctypes.CDLL(path)
    vp, dp, i32 = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int32
    st = ctypes.c_int
    lib.ucc_create.restype = st
    lib.ucc_create.argtypes = [ctypes.POINTER(Hamiltonian), ctypes.POINTER(Ansatz), vp, ctypes.POINTER(vp)]
    lib.ucc_set_theta.restype = st
    lib.ucc_set_theta.argtypes = [vp, vp, ctypes.c_int]
    lib.ucc_set_options.restype = st
    lib.ucc_set_options.argtypes = [vp, ctypes.POINTER(Options)]
    lib.ucc_apply.restype = st
    lib.ucc_apply.argtypes = [vp, ctypes.c_double]
    lib.ucc_energy.restype = st
    lib.ucc_energy.argtypes = [vp, dp, dp]
    lib.ucc_gradient.restype = st
    lib.ucc_gradient.argtypes = [vp, ctypes.c_double, dp, vp, ctypes.c_int]
    lib.ucc_get_wavefunction.restype = st
    lib.ucc_get_wavefunction.argtypes = [vp, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t), vp, vp, vp,
                                         ctypes.c_int]
    lib.ucc_get_entropy.restype = st
    lib.ucc_get_entropy.argtypes = [vp, dp, ctypes.c_int32]
    lib.ucc_get_stats.restype = st
    lib.ucc_get_stats.argtypes = [vp, ctypes.POINTER(Stats)]
    lib.ucc_batch_run.restype = st
    lib.ucc_batch_run.argtypes = [ctypes.c_int, ctypes.POINTER(vp), ctypes.c_double, dp, ctypes.POINTER(vp)]
    lib.ucc_last_error.restype = ctypes.c_char_p
    lib.ucc_last_error.argtypes = []
    lib.ucc_energy_static.restype = st
    lib.ucc_energy_static.argtypes = [i32, i32, i32, ctypes.c_double, vp, vp, ctypes.c_size_t, vp, vp, vp, dp, dp,
                                      vp]
    lib.ucc_destroy.restype = None
    lib.ucc_destroy.argtypes = [vp]
    _lib = lib
    return lib


def check(status):
    if status != UCC_OK:
        msg = _lib.ucc_last_error().decode(errors="replace") if _lib is not None else ""
        raise UCCError(status, msg)
