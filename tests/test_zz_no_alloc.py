"""qf_fft_step_static: the FFT step for callers that cannot allocate device memory.

Some callers cannot hand the library a workspace (no allocator of their own, memory
already owned by a host application, or a loop that must not fail on out-of-memory);
this entry point keeps its scratch in a fixed array inside the library instead.  The
tests run it twice in a row on caller-owned torch tensors and check each result against
the lattice path (qf_step_n) on the same inputs, and the first step and its five sums
against the FP64 oracle's step (Sec. 2), at the smallest sizes and at the size cap
(N = 64, where the fixed scratch is fullest), for every FFT kinetic term and for real
and complex potentials.  This file is collected last.
"""
import ctypes as C
import math

import numpy as np
import pytest

from fieldcheck import assert_field_close
from oracle import qfdtd_oracle as O
from paper_2211_10185_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel())


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2211_10185_gb300 import build, qfdtd as Q

    build.build()
    return Q.load()


@pytest.mark.parametrize("with_sums", [True, False])
@pytest.mark.parametrize("v_complex", [False, True])
@pytest.mark.parametrize("kind", [I.FFT_NAIVE, I.FFT_SYMANZIK, I.FFT_REL])
@pytest.mark.parametrize("n", [8, 12, 64])
def test_static_step_matches_the_lattice_step_twice(lib, n, kind, v_complex, with_sums):
    import torch

    from paper_2211_10185_gb300 import qfdtd as Q
    from paper_2211_10185_gb300.lattice import Lattice

    a, m = 0.2, 1.3
    v = I.cornell(n, a, 0.5, 0.2)
    if v_complex:
        v = v - 0.05j * np.abs(v)
    psi0 = I.gaussian_field(n, 21 + n)

    lat = Lattice(n, a, precision="c64")
    lat.set_potential(v)
    lat.set_kinetic(kind, m)
    lat.set_wavefunction(psi0)
    dtau = lat.info()["dtau"]

    dev = torch.device("cuda")
    psi = torch.tensor(psi0, dtype=torch.complex64, device=dev).contiguous()
    vt = torch.tensor(v, dtype=torch.complex64 if v_complex else torch.float32, device=dev).contiguous()
    sums = torch.zeros(5, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream().cuda_stream

    scale = 1.0
    for call in range(2):
        sp = C.c_void_p(sums.data_ptr()) if with_sums else None
        st = lib.qf_fft_step_static(n, a, kind, m, dtau, C.c_void_p(psi.data_ptr()), C.c_void_p(vt.data_ptr()),
                                    int(v_complex), scale, sp, C.c_void_p(stream))
        assert st == Q.QF_OK
        torch.cuda.synchronize()
        # the lattice path: a check on every step, renormalising the step after a check
        lat.step_n(1, check_every=1)
        ref_psi = lat.get_wavefunction()
        got = psi.cpu().numpy().astype(np.complex128)
        if call == 0:
            # the oracle's step from the same (complex-FP32) input field, no rescaling
            p0 = psi0.astype(np.complex64).astype(np.complex128)
            v64 = v.astype(np.complex64 if v_complex else np.float32).astype(np.complex128)
            hk = O.apply_kinetic(p0, kind, a, m)
            coef_a, coef_b = O.update_coefficients(v64, dtau)
            assert_field_close(got, coef_a * p0 - coef_b * dtau * hk, 2e-6 * (1 + math.log2(n)),
                               what=f"static step N={n}")
            if with_sums:
                s = sums.cpu().numpy()
                nrm, ek, ev = O.reductions(p0, hk, v64)
                assert s[0] == pytest.approx(nrm, rel=1e-6)
                assert abs(complex(s[1], s[2]) - ek) < 1e-5 * abs(ek)
                assert abs(complex(s[3], s[4]) - ev) < 1e-5 * abs(ev)
        assert _rel(got, ref_psi) < 2e-6 * (1 + math.log2(n))
        rms = np.sqrt(np.mean(np.abs(ref_psi) ** 2))
        assert np.max(np.abs(got - ref_psi)) < 2e-6 * (1 + math.log2(n)) * 8 * rms
        e_ref = lat.energies()
        if with_sums:
            s = sums.cpu().numpy()
            e_static = complex(s[1] + s[3], s[2] + s[4]) / s[0]
            assert abs(e_static - e_ref["e"]) < 1e-5 * abs(e_ref["e"])
            assert s[0] == pytest.approx(e_ref["norm"], rel=1e-5)
        scale = 1.0 / math.sqrt(e_ref["norm"])
    lat.close()


def test_static_step_rejects_lattices_beyond_its_fixed_scratch(lib):
    from paper_2211_10185_gb300 import qfdtd as Q

    for n in (96, 128, 10):
        assert lib.qf_fft_step_static(n, 0.1, I.FFT_NAIVE, 1.0, 1e-3, C.c_void_p(256), C.c_void_p(256), 0, 1.0,
                                      None, None) == Q.QF_EINVAL
    assert lib.qf_fft_step_static(32, 0.1, I.FDTD, 1.0, 1e-3, C.c_void_p(256), C.c_void_p(256), 0, 1.0,
                                  None, None) == Q.QF_EINVAL
