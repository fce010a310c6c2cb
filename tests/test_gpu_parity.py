"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on identical inputs.

Tolerances: the c128 path computes the same FP64 arithmetic in another summation order,
so fields agree to ~1e-12 relative and energies to 1e-10 relative.  The c64 path stores
fields in FP32: one FFT step carries ~log2(N) * 6e-8 relative error per site, checks
compare energies at 1e-5 relative (FP64 reductions of FP32 fields).
"""
import math

import numpy as np
import pytest

from oracle import qfdtd_oracle as O
from paper_2211_10185_gb300 import inputs as I

pytestmark = pytest.mark.gpu

KINDS = [O.FDTD, O.FFT_NAIVE, O.FFT_SYMANZIK, O.FFT_REL]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2211_10185_gb300 import build

    build.build()


def _pair(n, a, kind, m, prec, potential, seed=0, dtau=None, n_snap=3):
    from paper_2211_10185_gb300.lattice import Lattice

    v = potential
    psi0 = I.gaussian_field(n, seed)
    if kind == O.FDTD:
        psi0 = I.zero_dirichlet_planes(psi0)
    ref = O.Lattice(n, a, n_snap=n_snap)
    if np.iscomplexobj(v):
        ref.set_potential(v.real, v.imag)
    else:
        ref.set_potential(v)
    ref.set_kinetic(kind, m, dtau)
    ref.set_wavefunction(psi0)
    gpu = Lattice(n, a, precision=prec, n_snap=n_snap)
    gpu.set_potential(v)
    gpu.set_kinetic(kind, m, dtau)
    gpu.set_wavefunction(psi0)
    assert gpu.info()["dtau"] == pytest.approx(ref.dtau, rel=1e-15)
    return ref, gpu


def _rel(a, b):
    return np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel())


FIELD_TOL = {"c128": 1e-12, "c64": 2e-6}
E_TOL = {"c128": 1e-10, "c64": 1e-5}


@pytest.mark.parametrize("prec", ["c128", "c64"])
@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("n", [8, 12, 16, 24, 48])
def test_one_step_matches_oracle(n, kind, prec):
    a, m = 0.2, 1.3
    v = I.cornell(n, a, 0.5, 0.2)
    ref, gpu = _pair(n, a, kind, m, prec, v, seed=n)
    ref.step_n(1, check_every=1)
    st, done = gpu.step_n(1, check_every=1)
    assert done == 1
    tol = FIELD_TOL[prec] * (1 + math.log2(n))
    assert _rel(gpu.get_wavefunction(), ref.psi) < tol
    e_ref, e_gpu = ref.energies(), gpu.energies()
    assert abs(e_gpu["e"] - e_ref["e"]) < E_TOL[prec] * abs(e_ref["e"])
    assert e_gpu["norm"] == pytest.approx(e_ref["norm"], rel=E_TOL[prec])
    assert e_gpu["step"] == 0


@pytest.mark.parametrize("prec", ["c128", "c64"])
@pytest.mark.parametrize("kind", KINDS)
def test_many_steps_with_checks_and_complex_potential(kind, prec):
    n, a, m = 32, 0.25, 1.0
    v = I.gaussian_mix(n, a, seed=3, n_gauss=8)
    ref, gpu = _pair(n, a, kind, m, prec, v, seed=7)
    ref.step_n(200, check_every=16, snap_every=16)
    gpu.step_n(200, check_every=16, snap_every=16)
    # energies of every check are compared through the last one and the field itself
    e_ref, e_gpu = ref.energies(), gpu.energies()
    assert e_gpu["step"] == e_ref["step"] == 192
    assert abs(e_gpu["e"] - e_ref["e"]) < E_TOL[prec] * abs(e_ref["e"])
    assert abs(e_gpu["de"] - e_ref["de"]) < max(1e-6 if prec == "c64" else 1e-12, 1e-3 * e_ref["de"])
    tol = {"c128": 1e-10, "c64": 2e-4}[prec]
    assert _rel(gpu.get_wavefunction(), ref.psi) < tol


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_harmonic_fdtd_converges_like_the_oracle(prec):
    # the oscillator on N = 24 Dirichlet lattice, dtau = a^2/8, |dE| < 1e-8
    n, a, m = 24, 0.2, 1.0
    ref, gpu = _pair(n, a, O.FDTD, m, prec, I.harmonic(n, a), seed=0, dtau=a * a / 8)
    tol = 1e-8 if prec == "c128" else 1e-6
    s1, d1 = ref.step_n(40000, tol=tol, check_every=64)
    s2, d2 = gpu.step_n(40000, tol=tol, check_every=64)
    assert s1 == O.OK and s2 == 0
    if prec == "c128":
        assert d1 == d2
    e_ref, e_gpu = ref.energies()["e"].real, gpu.energies()["e"].real
    assert abs(e_gpu - e_ref) < E_TOL[prec] * abs(e_ref)


@pytest.mark.parametrize("prec", ["c128", "c64"])
@pytest.mark.parametrize("kind", [O.FDTD, O.FFT_SYMANZIK])
def test_excited_states_match_oracle_at_identical_snapshots(kind, prec):
    # The snapshots hold Psi_2 at relative weight ~exp(-2 tau) (gaps of 1).  FP32 fields
    # resolve it only while that weight is well above the accumulated FP32 rounding noise
    # (~1e-7 per step), so the c64 comparison uses tau ~ 2.9 and c128 tau ~ 5.8.
    n, a, m = 16, 0.3, 1.0
    ref, gpu = _pair(n, a, kind, m, prec, I.harmonic(n, a), seed=0, dtau=a * a / 8)
    steps = 8 * 64 if prec == "c128" else 4 * 64
    ref.step_n(steps, check_every=64, snap_every=32)
    gpu.step_n(steps, check_every=64, snap_every=32)
    st, ex_ref = ref.project_excited(3)
    ex_gpu = gpu.project_excited(3)
    tol = {"c128": [1e-10, 1e-9, 1e-8], "c64": [1e-5, 1e-4, 2e-3]}[prec]
    for i in range(3):
        er, eg = ex_ref[i]["e"], ex_gpu[i]["e"]
        assert abs(eg - er) < tol[i] * abs(er), (i, eg, er)
        assert ex_gpu[i]["norm"] == pytest.approx(1.0, abs=1e-4 if prec == "c64" else 1e-12)
    for i in range(3):
        s_ref = ref.states[i]
        s_gpu = gpu.get_wavefunction(i)
        ph = np.vdot(s_gpu, s_ref)
        # states agree up to a phase; c64 GS residuals carry FP32 noise / r_i
        assert abs(abs(ph) - 1) < {"c128": 1e-8, "c64": 1e-2}[prec]


@pytest.mark.parametrize("prec", ["c128", "c64"])
@pytest.mark.parametrize("which,axis", [(O.P_PLUS, 3), (O.P_MINUS, 3), (O.P_MINUS_PK, 1), (O.P_MINUS_PK, 2),
                                        (O.P_MINUS_PK, 3), (O.P_D_K, 3), (O.P_D_K, 1), (O.P_D2_K, 3),
                                        (O.P_D2_K, 2)])
@pytest.mark.parametrize("n", [8, 12, 24])
def test_parity_projection_matches_oracle_and_is_exactly_symmetric(n, which, axis, prec):
    a = 0.3
    ref, gpu = _pair(n, a, O.FFT_NAIVE, 1.0, prec, I.harmonic(n, a), seed=n + which)
    ref.parity_project(which, axis, -1)
    gpu.parity_project(which, axis, -1)
    out = gpu.get_wavefunction()
    assert _rel(out, ref.psi) < {"c128": 1e-14, "c64": 1e-6}[prec]
    # exact symmetry of the projected field (bitwise, also in FP32)
    if which == O.P_PLUS:
        assert np.array_equal(out, O.mirror(out))
    elif which == O.P_MINUS:
        assert np.array_equal(out, -O.mirror(out))
    elif which == O.P_MINUS_PK:
        k = O._NP_AXIS[axis]
        others = tuple(x for x in (0, 1, 2) if x != k)
        assert np.array_equal(out, -O.mirror(out, (k,)))
        assert np.array_equal(out, O.mirror(out, others))
    else:
        k = O._NP_AXIS[axis]
        i, j = tuple(x for x in (0, 1, 2) if x != k)
        assert np.array_equal(out, O.mirror(out, (k,)))
        if which == O.P_D_K:
            assert np.array_equal(out, -O.mirror(out, (i,)))
            assert np.array_equal(out, -O.mirror(out, (j,)))
        else:
            assert np.array_equal(out, O.mirror(out, (i,)))
            assert np.array_equal(out, -np.swapaxes(out, i, j))


def test_parity_of_a_gs_state_target():
    n, a = 16, 0.3
    ref, gpu = _pair(n, a, O.FDTD, 1.0, "c128", I.harmonic(n, a), seed=0, dtau=a * a / 8)
    ref.step_n(6 * 64, check_every=64, snap_every=32)
    gpu.step_n(6 * 64, check_every=64, snap_every=32)
    ref.project_excited(2)
    gpu.project_excited(2)
    ref.parity_project(O.P_MINUS, 3, 1)
    gpu.parity_project(O.P_MINUS, 3, 1)
    s_gpu, s_ref = gpu.get_wavefunction(1), ref.states[1]
    assert abs(abs(np.vdot(s_gpu, s_ref)) - 1) < 1e-8


def test_state_machine_errors():
    from paper_2211_10185_gb300 import qfdtd as Q
    from paper_2211_10185_gb300.lattice import Lattice

    lat = Lattice(16, 0.2)
    with pytest.raises(Q.QFError) as e:
        lat.step_n(1)
    assert e.value.status == Q.QF_ESTATE
    with pytest.raises(Q.QFError) as e:
        lat.project_excited(2)
    assert e.value.status == Q.QF_ESTATE
    with pytest.raises(Q.QFError) as e:
        lat.set_kinetic(7, 1.0)
    assert e.value.status == Q.QF_EINVAL
    with pytest.raises(Q.QFError) as e:
        lat.parity_project(O.P_MINUS_PK, 4, -1)
    assert e.value.status == Q.QF_EINVAL
    lat10 = Lattice(10, 0.2)
    with pytest.raises(Q.QFError) as e:
        lat10.set_kinetic(O.FFT_REL, 1.0)      # no FFT plan for N = 10
    assert e.value.status == Q.QF_EINVAL
    lat10.set_kinetic(O.FDTD, 1.0)              # FDTD takes any even N


def test_bounded_wait_times_out_and_context_stays_usable():
    # a barrier nothing completes: the bounded wait must give up and report QF_ETIMEOUT,
    # after which the same handle still computes correctly
    from paper_2211_10185_gb300 import qfdtd as Q

    n, a = 16, 0.3
    ref, gpu = _pair(n, a, O.FDTD, 1.0, "c64", I.harmonic(n, a), seed=2)
    assert gpu.lib.qf_selftest_bounded_wait(gpu.h) == Q.QF_ETIMEOUT
    ref.step_n(8, check_every=4)
    gpu.step_n(8, check_every=4)
    assert abs(gpu.energies()["e"] - ref.energies()["e"]) < 1e-5 * abs(ref.energies()["e"])


@pytest.mark.parametrize("prec", ["c128", "c64"])
@pytest.mark.parametrize("n,kind", [(16, O.FFT_SYMANZIK), (24, O.FDTD), (48, O.FFT_REL)])
def test_momentum_distribution_matches_oracle(n, kind, prec):
    a = 0.3
    ref, gpu = _pair(n, a, kind, 1.0, prec, I.harmonic(n, a), seed=n)
    ref.step_n(32, check_every=16)
    gpu.step_n(32, check_every=16)
    p_r, P_r, y_r = O.momentum_distribution(ref.psi, a)
    p_g, P_g, y_g = gpu.momentum_distribution()
    assert len(P_g) == len(P_r)
    assert np.allclose(p_g, p_r, rtol=1e-14, atol=0)
    assert abs(P_g.sum() - 1) < 1e-12
    tol = {"c128": 1e-12, "c64": 3e-6}[prec]
    assert np.max(np.abs(P_g - P_r)) < tol
    assert np.max(np.abs(y_g - y_r)) < 1e3 * tol
    # integer shell sums: the same call gives bitwise the same histogram
    assert np.array_equal(gpu.momentum_distribution()[1], P_g)
    # the step after it still matches (the scratch field was reused)
    ref.step_n(1, check_every=1)
    gpu.step_n(1, check_every=1)
    assert abs(gpu.energies()["e"] - ref.energies()["e"]) < {"c128": 1e-10, "c64": 1e-5}[prec] * abs(ref.energies()["e"])


@pytest.mark.parametrize("kind,prec", [(O.FDTD, "c64"), (O.FFT_REL, "c64"), (O.FDTD, "c128"), (O.FFT_NAIVE, "c128")])
def test_graph_replay_is_bitwise_identical_to_launches(kind, prec):
    n, a = 24, 0.25
    v = I.cornell(n, a, 0.5, 0.2)
    _, g1 = _pair(n, a, kind, 1.1, prec, v, seed=4)
    _, g2 = _pair(n, a, kind, 1.1, prec, v, seed=4)
    g2.use_graphs(False)
    for lat in (g1, g2):
        lat.step_n(3 * 32 + 5, check_every=32, snap_every=32)
    assert np.array_equal(g1.get_wavefunction(), g2.get_wavefunction())
    assert g1.energies() == g2.energies()
    assert np.array_equal(g1.get_wavefunction(100), g2.get_wavefunction(100))
    assert g1.info()["step"] == g2.info()["step"] == 101


@pytest.mark.parametrize("prec", ["c128", "c64"])
@pytest.mark.parametrize("nc", [8, 12, 16, 24])
def test_prolongation_matches_oracle(nc, prec):
    from paper_2211_10185_gb300.lattice import Lattice

    a = 0.4
    coarse = Lattice(nc, a, precision=prec)
    psi = I.gaussian_field(nc, nc + 1)
    coarse.set_wavefunction(psi)
    fine = Lattice(2 * nc, a / 2, precision=prec)
    fine.prolong_from(coarse)
    ref = O.prolong(coarse.get_wavefunction())
    got = fine.get_wavefunction()
    assert _rel(got, ref) < {"c128": 1e-13, "c64": 1e-6}[prec]
    assert np.max(np.abs(got[::2, ::2, ::2] - coarse.get_wavefunction())) < {"c128": 1e-12, "c64": 1e-5}[prec]
