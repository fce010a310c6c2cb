"""The two-pass FFT step (N = 128 and 256, complex FP32) against the oracle and the
four-pass step.

The two-pass form splits the y transform (N/16) x 16 between its passes and keeps the
scratch field in a blocked layout; it must compute the same step as the four-pass form
to FP32 rounding, match the FP64 oracle to the usual c64 tolerance, and run bitwise the
same alone and inside a batch (both launch the same grouped kernels).
"""
import math

import numpy as np
import pytest

from fieldcheck import assert_field_close
from oracle import qfdtd_oracle as O
from paper_2211_10185_gb300 import inputs as I

pytestmark = pytest.mark.gpu

N, A = 256, 0.05
SIZES = [128, 256]


def _a(n):
    # the same physical box at every size: a = 0.05 at N = 256
    return A * N / n


@pytest.fixture(scope="module", autouse=True)
def _built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2211_10185_gb300 import build

    build.build()


def _rel(a, b):
    return np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel())


def _potential(cplx, n=N):
    v = I.cornell(n, _a(n), 0.4, 0.2)
    return v - 0.04j * np.abs(v) if cplx else v


def _dtau(kind, n=N):
    # a/4 for the relativistic term (the bench workload); the stable default otherwise
    return _a(n) / 4 if kind == I.FFT_REL else None


def _lat(kind, v, psi0, two_pass=True, m=0.3):
    from paper_2211_10185_gb300.lattice import Lattice

    n = v.shape[0]
    lat = Lattice(n, _a(n), precision="c64")
    lat.set_potential(v)
    lat.set_kinetic(kind, m, _dtau(kind, n))
    lat.set_wavefunction(psi0)
    lat.use_two_pass_fft(two_pass)
    return lat


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("kind", [I.FFT_NAIVE, I.FFT_SYMANZIK, I.FFT_REL])
def test_two_pass_step_matches_oracle_every_site(kind, cplx, n):
    v = _potential(cplx, n)
    psi0 = I.gaussian_field(n, 11 + kind)
    gpu = _lat(kind, v, psi0)
    assert gpu.info()["fft_passes"] == 2
    ref = O.Lattice(n, _a(n))
    if cplx:
        ref.set_potential(v.real, v.imag)
    else:
        ref.set_potential(v)
    ref.set_kinetic(kind, 0.3, _dtau(kind, n))
    ref.set_wavefunction(psi0)
    # step 0 with a check (sums), step 1 plain with the renormalisation (the first step
    # starts from the natural-order pass, the second from the emitted scratch field)
    for _ in range(2):
        ref.step_n(1, check_every=2)
        gpu.step_n(1, tol=0.0, check_every=2)
    assert_field_close(gpu.get_wavefunction(), ref.psi, 2e-6 * (1 + math.log2(n)), what=f"N={n}")
    e_ref, e_gpu = ref.energies(), gpu.energies()
    assert abs(e_gpu["e"] - e_ref["e"]) < 1e-5 * abs(e_ref["e"])
    assert e_gpu["norm"] == pytest.approx(e_ref["norm"], rel=1e-5)


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("kind", [I.FFT_SYMANZIK, I.FFT_REL])
def test_two_pass_and_four_pass_agree_over_many_steps(kind, n):
    v = _potential(True, n)
    psi0 = I.gaussian_field(n, 3)
    two = _lat(kind, v, psi0, True)
    four = _lat(kind, v, psi0, False)
    assert four.info()["fft_passes"] == 4
    for lat in (two, four):
        lat.step_n(193, tol=0.0, check_every=64, snap_every=64)
    assert_field_close(two.get_wavefunction(), four.get_wavefunction(), 2e-5)
    e2, e4 = two.energies(), four.energies()
    assert e2["step"] == e4["step"] == 192
    assert abs(e2["e"] - e4["e"]) < 1e-5 * abs(e4["e"])
    # excited states through the measure passes (pass A from a state slot, sums-only C)
    x2, x4 = two.project_excited(3), four.project_excited(3)
    for a, b in zip(x2, x4):
        assert abs(a["e"] - b["e"]) < 1e-5 * abs(b["e"])
    # fewer launches per steady-state step
    assert two.info()["launches"] < four.info()["launches"]


@pytest.mark.parametrize("n", SIZES)
def test_switching_forms_mid_run_keeps_the_step(n):
    v = _potential(False, n)
    psi0 = I.gaussian_field(n, 5)
    ref = _lat(I.FFT_REL, v, psi0, True)
    mix = _lat(I.FFT_REL, v, psi0, True)
    ref.step_n(6, tol=0.0, check_every=3)
    mix.step_n(3, tol=0.0, check_every=3)
    mix.use_two_pass_fft(False)   # the scratch field's blocked layout is discarded
    mix.step_n(2, tol=0.0, check_every=3)
    mix.use_two_pass_fft(True)
    mix.step_n(1, tol=0.0, check_every=3)
    assert _rel(mix.get_wavefunction(), ref.get_wavefunction()) < 1e-5


def test_two_pass_batch_members_match_alone_bitwise():
    """Members of both two-pass sizes in one batch (each size launches as its own group)."""
    from paper_2211_10185_gb300.serve import Batch

    specs = [(I.FFT_REL, False, 1, 256), (I.FFT_NAIVE, True, 2, 128), (I.FFT_SYMANZIK, False, 3, 256),
             (I.FFT_REL, True, 4, 128)]
    alone, mixed = [], []
    for kind, cplx, seed, n in specs:
        v = _potential(cplx, n)
        psi0 = I.gaussian_field(n, seed)
        alone.append(_lat(kind, v, psi0))
        mixed.append(_lat(kind, v, psi0))
    for lat in alone:
        lat.step_n(70, tol=0.0, check_every=32, snap_every=32)
    b = Batch()
    for lat in mixed:
        b.add(lat, 70, 0.0)
    while b.step(35, check_every=32) > 0:
        pass
    for la, lm in zip(alone, mixed):
        assert np.array_equal(la.get_wavefunction(), lm.get_wavefunction())
        assert la.energies()["e"] == lm.energies()["e"]


def test_batch_keeps_two_and_four_pass_members_apart():
    """Members of one size that run different step forms launch separately, and each
    matches its own form alone bitwise."""
    from paper_2211_10185_gb300.serve import Batch

    v = _potential(False)
    alone, mixed = [], []
    for seed, two in ((7, True), (8, False), (9, True)):
        psi0 = I.gaussian_field(N, seed)
        alone.append(_lat(I.FFT_REL, v, psi0, two))
        mixed.append(_lat(I.FFT_REL, v, psi0, two))
    for lat in alone:
        lat.step_n(40, tol=0.0, check_every=16, snap_every=16)
    b = Batch()
    for lat in mixed:
        b.add(lat, 40, 0.0)
    while b.step(20, check_every=16) > 0:
        pass
    for la, lm in zip(alone, mixed):
        assert lm.info()["fft_passes"] == la.info()["fft_passes"]
        assert np.array_equal(la.get_wavefunction(), lm.get_wavefunction())


def test_side_operations_between_two_pass_steps_leave_the_solve_unchanged():
    """Momentum output, parity projection of a state slot and excited-state extraction
    overwrite the scratch field; the next two-pass step must start again from natural
    order and give the same field as a lattice that did none of them."""
    v = _potential(False)
    psi0 = I.gaussian_field(N, 21)
    plain = _lat(I.FFT_REL, v, psi0)
    busy = _lat(I.FFT_REL, v, psi0)
    for lat in (plain, busy):
        lat.step_n(193, tol=0.0, check_every=64, snap_every=64)
    busy.momentum_distribution()
    busy.project_excited(3)
    busy.parity_project(O.P_MINUS, 3, 1)   # on state 1, not the live field
    for lat in (plain, busy):
        lat.step_n(70, tol=0.0, check_every=64, snap_every=64)
    # (the busy lattice restarts with pass A from natural order, the other reuses the
    # emitted scratch field: the same arithmetic in two kernels, equal to rounding)
    assert _rel(busy.get_wavefunction(), plain.get_wavefunction()) < 1e-6
    assert abs(busy.energies()["e"] - plain.energies()["e"]) < 1e-6 * abs(plain.energies()["e"])


def test_prolongation_onto_a_two_pass_lattice():
    """Warm start N=128 -> 256: the prolonged field keeps the coarse values on coincident
    sites, and the two-pass steps from it match the four-pass steps."""
    from paper_2211_10185_gb300.lattice import Lattice

    nc, ac = N // 2, 2 * A
    coarse = Lattice(nc, ac, precision="c64")
    coarse.set_potential(I.cornell(nc, ac, 0.4, 0.2))
    coarse.set_kinetic(I.FFT_REL, 0.3, A / 4)
    coarse.set_wavefunction(I.gaussian_field(nc, 4))
    coarse.step_n(64, tol=0.0, check_every=32)
    psi_c = coarse.get_wavefunction()
    fines = []
    for two in (True, False):
        fine = _lat(I.FFT_REL, _potential(False), np.zeros((N, N, N), complex), two)
        fine.prolong_from(coarse)
        fines.append(fine)
    got = fines[0].get_wavefunction()
    # coincident sites carry the coarse values (exact up to the FP32 transforms)
    assert np.abs(got[::2, ::2, ::2] - psi_c).max() < 1e-5 * np.abs(psi_c).max()
    assert np.array_equal(got, fines[1].get_wavefunction())
    for f in fines:
        f.step_n(20, tol=0.0, check_every=10)
    assert _rel(fines[0].get_wavefunction(), fines[1].get_wavefunction()) < 1e-5
