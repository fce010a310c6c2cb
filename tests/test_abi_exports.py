"""The C-ABI library loads and exports every entry point include/qfdtd.h declares.

Runs without a GPU: only host-side calls (version, workspace sizing, argument checks
that fail before any CUDA call) are made.
"""
import ctypes as C
import os
import re

import pytest

from paper_2211_10185_gb300 import build, qfdtd as Q

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "qfdtd.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(qf_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return Q.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "qf_step_n" in names and "qf_project_excited" in names and "qf_parity_project" in names
    for name in names:
        assert hasattr(lib, name), name
        assert name in Q.SIGNATURES, f"binding lacks {name}"


def test_version_and_workspace_sizing(lib):
    assert b"sm_103a" in lib.qf_version()
    d = Q.qf_lattice_desc(256, 0.05, Q.QF_PREC_C64, 3)
    nb = C.c_size_t()
    assert lib.qf_workspace_bytes(C.byref(d), C.byref(nb)) == Q.QF_OK
    field = 256 ** 3 * 8
    # live + scratch + V + 3 snapshots + 3 states, plus small tables
    assert 9 * field <= nb.value < 9 * field + (64 << 20)
    d128 = Q.qf_lattice_desc(256, 0.05, Q.QF_PREC_C128, 3)
    nb2 = C.c_size_t()
    assert lib.qf_workspace_bytes(C.byref(d128), C.byref(nb2)) == Q.QF_OK
    assert nb2.value > 2 * 9 * field - (64 << 20)


@pytest.mark.parametrize("n,a,prec,snap", [(7, 0.1, 0, 3), (9, 0.1, 0, 3), (6, 0.1, 0, 3), (2048, 0.1, 0, 3),
                                           (32, 0.0, 0, 3), (32, -1.0, 0, 3), (32, 0.1, 2, 3),
                                           (32, 0.1, 0, 0), (32, 0.1, 0, 4)])
def test_invalid_descriptions_are_rejected(lib, n, a, prec, snap):
    d = Q.qf_lattice_desc(n, a, prec, snap)
    nb = C.c_size_t()
    assert lib.qf_workspace_bytes(C.byref(d), C.byref(nb)) == Q.QF_EINVAL


def test_null_arguments_fail_without_touching_the_gpu(lib):
    d = Q.qf_lattice_desc(32, 0.1, 0, 3)
    h = C.c_void_p()
    assert lib.qf_create_lattice(C.byref(d), None, 0, None, C.byref(h)) == Q.QF_EINVAL
    assert lib.qf_create_lattice(C.byref(d), C.c_void_p(256), 16, None, C.byref(h)) == Q.QF_ENOMEM
    assert lib.qf_create_lattice(C.byref(d), C.c_void_p(100), 1 << 40, None, C.byref(h)) == Q.QF_EINVAL
    assert lib.qf_destroy_lattice(None) == Q.QF_OK
    assert lib.qf_step_n(None, 1, 0.0, 1, 1, None) == Q.QF_EINVAL
    assert lib.qf_last_error(None) == b"null handle"


def test_fft_variant_choice_is_host_state(lib):
    """qf_set_fft_tiles / qf_get_fft_tiles (no GPU involved): tile variants 0 and 1 for
    every FFT size, the radix-plan variants 2 and 3 only for the sizes with a second plan
    (32, 64, 512), -1 back to pending; other sizes and values are rejected.  Each choice
    is put back as it was."""
    v = C.c_int()
    for n in (8, 12, 16, 24, 32, 48, 64, 96, 128, 192, 256, 384, 512):
        assert lib.qf_get_fft_tiles(n, C.byref(v)) == Q.QF_OK
        old = v.value
        try:
            for var in (0, 1, -1):
                assert lib.qf_set_fft_tiles(n, var) == Q.QF_OK
                assert lib.qf_get_fft_tiles(n, C.byref(v)) == Q.QF_OK and v.value == var
            for var in (2, 3):
                want = Q.QF_OK if n in (32, 64, 512) else Q.QF_EINVAL
                assert lib.qf_set_fft_tiles(n, var) == want, (n, var)
            assert lib.qf_set_fft_tiles(n, 4) == Q.QF_EINVAL and lib.qf_set_fft_tiles(n, -2) == Q.QF_EINVAL
        finally:
            lib.qf_set_fft_tiles(n, old)
    assert lib.qf_set_fft_tiles(10, 0) == Q.QF_EINVAL
    assert lib.qf_get_fft_tiles(10, C.byref(v)) == Q.QF_EINVAL
