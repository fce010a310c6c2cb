"""Degenerate inputs and a closed form at the bench size, through the C ABI.

* an empty run (max_steps = 0) changes nothing;
* the zero wavefunction stays zero (norm 0: the renormalisation falls back to 1, the
  energy is NaN) for every kinetic form, as the oracle's field does;
* a plane wave under a constant potential is an eigenvector of every step: after n steps
  it is multiplied by lambda^n, lambda = (1 - dtau V/2 - dtau T(k)) / (1 + dtau V/2), with
  T(k) the kinetic symbol (Eqs. HK1-HK3) -- checked on the N=256 two-pass and four-pass
  FFT steps without the oracle.
"""
import math

import numpy as np
import pytest

from fieldcheck import assert_field_close
from oracle import qfdtd_oracle as O
from paper_2211_10185_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2211_10185_gb300 import build

    build.build()


def _lat(n, a, kind, m, v, psi, prec="c64", dtau=None):
    from paper_2211_10185_gb300.lattice import Lattice

    lat = Lattice(n, a, precision=prec)
    lat.set_potential(v)
    lat.set_kinetic(kind, m, dtau)
    lat.set_wavefunction(psi)
    return lat


def test_empty_run_changes_nothing():
    from paper_2211_10185_gb300 import qfdtd as Q

    n, a = 16, 0.3
    psi = I.gaussian_field(n, 1)
    lat = _lat(n, a, I.FFT_SYMANZIK, 1.0, I.harmonic(n, a), psi)
    st, done = lat.step_n(0, tol=0.0, check_every=4)
    assert (st, done) == (Q.QF_ENOTCONV, 0)
    assert lat.info()["step"] == 0
    assert np.allclose(lat.get_wavefunction(), psi, rtol=0, atol=1e-6 * np.abs(psi).max())


@pytest.mark.parametrize("kind,n", [(I.FDTD, 24), (I.FFT_NAIVE, 16), (I.FFT_REL, 256)])
def test_zero_wavefunction_stays_zero(kind, n):
    a = 6.0 / n
    lat = _lat(n, a, kind, 1.0, I.cornell(n, a, 0.4, 0.2), np.zeros((n, n, n), complex))
    lat.step_n(9, tol=0.0, check_every=4)
    assert not lat.get_wavefunction().any()
    e = lat.energies()
    assert e["norm"] == 0.0 and math.isnan(e["e"].real)
    ref = O.Lattice(n, a)
    ref.set_potential(I.cornell(n, a, 0.4, 0.2))
    ref.set_kinetic(kind, 1.0)
    ref.set_wavefunction(np.zeros((n, n, n), complex))
    ref.step_n(9, check_every=0)   # (the oracle leaves the energy of a zero field undefined)
    assert not ref.psi.any()


def _symbol(kind, k, a, m):
    s2 = 4 * np.sum(np.sin(np.asarray(k) / 2) ** 2)
    if kind == I.FFT_NAIVE:
        return float(np.sum(np.asarray(k) ** 2)) / (2 * m * a * a)
    if kind == I.FFT_SYMANZIK:
        return s2 / (2 * m * a * a)
    return math.sqrt(s2 + (a * m) ** 2) / a


@pytest.mark.parametrize("n,nvec", [(256, (3, -5, 7)), (128, (5, 63, -64))])
@pytest.mark.parametrize("two_pass", [True, False])
@pytest.mark.parametrize("kind", [I.FFT_NAIVE, I.FFT_SYMANZIK, I.FFT_REL])
def test_plane_wave_closed_form(kind, two_pass, n, nvec):
    """psi = exp(i k.x) with V constant is an eigenvector of the step: one factor per step.
    nvec is the momentum index per axis (x, y, z); at N = 128 it has the largest k_lo of
    the split y transform and the Nyquist index in z."""
    a, m, v0 = 12.8 / n, 0.3, 0.7
    k = [2 * math.pi * j / n for j in nvec]
    idx = np.arange(n)
    # psi[z, y, x] = exp(i (kx x + ky y + kz z)) on the lattice indices
    psi = np.exp(1j * (k[0] * idx[None, None, :] + k[1] * idx[None, :, None] + k[2] * idx[:, None, None]))
    lat = _lat(n, a, kind, m, np.full((n, n, n), v0), psi)
    lat.use_two_pass_fft(two_pass)
    dtau = lat.info()["dtau"]
    steps = 5
    lat.step_n(steps, tol=0.0, check_every=0, snap_every=0)
    lam = (1 - dtau * v0 / 2 - dtau * _symbol(kind, k, a, m)) / (1 + dtau * v0 / 2)
    got = lat.get_wavefunction()
    want = lam ** steps * psi
    assert_field_close(got, want, 2e-6 * steps * math.log2(n))


@pytest.mark.parametrize("prec,offset", [("c64", 0), ("c128", 0), ("c64", 1)])
def test_upload_from_page_locked_memory_matches_pageable(prec, offset):
    """qf_set_wavefunction reads page-locked host buffers directly from the GPU; the field
    must equal the one uploaded from ordinary (pageable) memory, also for a buffer that is
    only 8-byte aligned."""
    import torch

    n, a = 24, 0.3
    psi = I.gaussian_field(n, 3)
    flat = np.ascontiguousarray(psi.reshape(-1)).view(np.float64)
    pinned = torch.empty(2 * n ** 3 + 1, dtype=torch.float64, pin_memory=True)
    view = pinned.numpy()[offset:offset + 2 * n ** 3]
    view[:] = flat
    one = _lat(n, a, I.FFT_SYMANZIK, 1.0, I.harmonic(n, a), psi, prec)
    two = _lat(n, a, I.FFT_SYMANZIK, 1.0, I.harmonic(n, a), np.zeros_like(psi), prec)
    two.set_wavefunction_raw(view)
    assert np.array_equal(one.get_wavefunction(), two.get_wavefunction())


@pytest.mark.parametrize("prec", ["c64", "c128"])
@pytest.mark.parametrize("check_every", [64, 256])
def test_fast_decay_between_checks_stays_in_range(prec, check_every):
    """A heavy quark with the relativistic term (N=16, a=1, m=3.77) decays by ~0.59 per
    step, so between checks the field falls by 1e-15 (64 steps) to 1e-58 (256 steps):
    below what complex FP32 holds.  The steps scale by exact powers of two and the
    library removes them on readback: energies, norms and fields equal the oracle's."""
    n, a, m = 16, 1.0, 3.7744603079583525
    v = I.cornell(n, a, 0.43989095916094956, 0.11908043740877956, 0.0)
    r = I.radius(n, a)
    psi0 = np.exp(-0.5 * (r / 0.5) ** 2).astype(complex)
    lat = _lat(n, a, I.FFT_REL, m, v, psi0, prec)
    ref = O.Lattice(n, a)
    ref.set_potential(v)
    ref.set_kinetic(O.FFT_REL, m)
    ref.set_wavefunction(psi0)
    e_tol = {"c64": 1e-5, "c128": 1e-10}[prec]
    for _ in range(4):
        lat.step_n(check_every, tol=0.0, check_every=check_every)
        ref.step_n(check_every, check_every=check_every)
        eg, er = lat.energies(), ref.energies()
        assert abs(eg["e"] - er["e"]) < e_tol * abs(er["e"]), (eg["e"], er["e"])
        assert eg["norm"] == pytest.approx(er["norm"], rel=e_tol)
    assert lat.info()["field_exp2"] != 0       # the stored field was rescaled
    assert_field_close(lat.get_wavefunction(), ref.psi, {"c64": 2e-4, "c128": 1e-10}[prec])
    # the oracle's converged energy (3.5286693398...) is reached
    assert abs(lat.energies()["e"].real - 3.528669339857) < 1e-5 * 3.53
