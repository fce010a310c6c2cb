"""ctypes binding of libqfdtd (include/qfdtd.h): same names, argument marshalling only.

Every function here forwards to the C entry point of the same name and returns its
status code; no arithmetic on fields happens in Python.  ``load()`` raises OSError when
the shared library has not been built (``python -m paper_2211_10185_gb300.build``).
"""
from __future__ import annotations

import ctypes as C
import os

from . import build as _build

QF_OK, QF_EINVAL, QF_ENOMEM, QF_ECUDA, QF_ESTATE, QF_ETIMEOUT, QF_ENOTCONV = range(7)
STATUS_NAMES = {0: "QF_OK", 1: "QF_EINVAL", 2: "QF_ENOMEM", 3: "QF_ECUDA", 4: "QF_ESTATE",
                5: "QF_ETIMEOUT", 6: "QF_ENOTCONV"}
QF_KIN_FDTD, QF_KIN_FFT_NAIVE, QF_KIN_FFT_SYMANZIK, QF_KIN_FFT_REL = range(4)
QF_PREC_C64, QF_PREC_C128 = 0, 1
QF_P_PLUS, QF_P_MINUS, QF_P_MINUS_PK, QF_P_D_K, QF_P_D2_K = 0, 1, 2, 3, 4
QF_BATCH_RUNNING = -1
QF_STOP_DIFFERENCE, QF_STOP_EXTRAPOLATED = 0, 1


class qf_lattice_desc(C.Structure):
    _fields_ = [("n", C.c_int), ("a", C.c_double), ("prec", C.c_int), ("n_snap", C.c_int),
                ("plateau_slots", C.c_int)]


class qf_energy(C.Structure):
    _fields_ = [("e_re", C.c_double), ("e_im", C.c_double), ("norm", C.c_double), ("de", C.c_double),
                ("step", C.c_int64), ("tau", C.c_double)]

    def as_dict(self):
        return dict(e=complex(self.e_re, self.e_im), norm=self.norm, de=self.de, step=self.step,
                    tau=self.tau)


class qf_info(C.Structure):
    _fields_ = [("dtau", C.c_double), ("step", C.c_int64), ("tau", C.c_double), ("kinetic", C.c_int),
                ("n_snapshots", C.c_int), ("workspace_bytes", C.c_size_t), ("launches", C.c_int64),
                ("temporal_block", C.c_int), ("fft_passes", C.c_int), ("field_exp2", C.c_int64)]


class qf_kernel_stat(C.Structure):
    _fields_ = [("name", C.c_char * 24), ("launches", C.c_int64), ("total_ms", C.c_double)]


_P = C.c_void_p
_D = C.POINTER(C.c_double)
# name -> (restype, argtypes)
SIGNATURES = {
    "qf_workspace_bytes": (C.c_int, [C.POINTER(qf_lattice_desc), C.POINTER(C.c_size_t)]),
    "qf_create_lattice": (C.c_int, [C.POINTER(qf_lattice_desc), _P, C.c_size_t, _P, C.POINTER(_P)]),
    "qf_destroy_lattice": (C.c_int, [_P]),
    "qf_set_potential": (C.c_int, [_P, _D, _D]),
    "qf_set_kinetic": (C.c_int, [_P, C.c_int, C.c_double, C.c_double]),
    "qf_set_wavefunction": (C.c_int, [_P, _D]),
    "qf_get_wavefunction": (C.c_int, [_P, C.c_int, _D]),
    "qf_step_n": (C.c_int, [_P, C.c_int64, C.c_double, C.c_int, C.c_int, C.POINTER(C.c_int64)]),
    "qf_energies": (C.c_int, [_P, C.POINTER(qf_energy)]),
    "qf_project_excited": (C.c_int, [_P, C.c_int, C.POINTER(qf_energy)]),
    "qf_parity_project": (C.c_int, [_P, C.c_int, C.c_int, C.c_int]),
    "qf_track_excited": (C.c_int, [_P, C.c_int, C.POINTER(qf_energy)]),
    "qf_excited_plateau": (C.c_int, [_P, C.c_int, C.POINTER(qf_energy), C.POINTER(C.c_int)]),
    "qf_get_info": (C.c_int, [_P, C.POINTER(qf_info)]),
    "qf_prolong": (C.c_int, [_P, C.c_int, _P]),
    "qf_momentum_distribution": (C.c_int, [_P, C.c_int, _D, _D, _D, C.c_int, C.POINTER(C.c_int)]),
    "qf_field_pointer": (C.c_int, [_P, C.c_int, C.POINTER(_P)]),
    "qf_profile": (C.c_int, [_P, C.c_int]),
    "qf_profile_read": (C.c_int, [_P, C.POINTER(qf_kernel_stat), C.c_int, C.POINTER(C.c_int), C.c_int]),
    "qf_fft_step_static": (C.c_int, [C.c_int, C.c_double, C.c_int, C.c_double, C.c_double, _P, _P, C.c_int,
                                     C.c_double, _P, _P]),
    "qf_batch_create": (C.c_int, [_P, C.POINTER(_P)]),
    "qf_batch_destroy": (C.c_int, [_P]),
    "qf_batch_add": (C.c_int, [_P, _P, C.c_int64, C.c_double, C.c_double]),
    "qf_batch_remove": (C.c_int, [_P, _P]),
    "qf_batch_step": (C.c_int, [_P, C.c_int64, C.c_int, C.c_int, C.POINTER(C.c_int)]),
    "qf_batch_members": (C.c_int, [_P, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int64), C.c_int]),
    "qf_batch_info": (C.c_int, [_P, C.POINTER(C.c_int64)]),
    "qf_batch_set_stopping": (C.c_int, [_P, C.c_int]),
    "qf_batch_use_graphs": (C.c_int, [_P, C.c_int]),
    "qf_batch_graph_info": (C.c_int, [_P, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "qf_batch_last_error": (C.c_char_p, [_P]),
    "qf_selftest_bounded_wait": (C.c_int, [_P]),
    "qf_use_graphs": (C.c_int, [_P, C.c_int]),
    "qf_set_temporal_blocking": (C.c_int, [_P, C.c_int]),
    "qf_use_two_pass_fft": (C.c_int, [_P, C.c_int]),
    "qf_set_fft_tiles": (C.c_int, [C.c_int, C.c_int]),
    "qf_get_fft_tiles": (C.c_int, [C.c_int, C.POINTER(C.c_int)]),
    "qf_last_error": (C.c_char_p, [_P]),
    "qf_version": (C.c_char_p, []),
}

_lib = None


def library_path() -> str:
    return _build.library_path()


def load(path: str | None = None):
    """Loads libqfdtd.so once and declares every entry point; raises OSError if absent."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or library_path()
    if not os.path.exists(p):
        raise OSError(f"libqfdtd.so not built at {p}; run python -m paper_2211_10185_gb300.build")
    lib = C.CDLL(p)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _lib = lib
    return lib


class QFError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str = ""):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)} {msg}".strip())
        self.status = status


def dptr(arr):
    """Pointer to a C-contiguous float64 numpy array (or None)."""
    if arr is None:
        return None
    assert arr.dtype.name == "float64" and arr.flags["C_CONTIGUOUS"]
    return arr.ctypes.data_as(_D)
