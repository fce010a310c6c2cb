"""The paper-shaped workloads at their full sizes, through the C ABI, against the oracle.

* N=256 relativistic workload (the bench configuration): two steps with checks,
  every site compared with the FP64 oracle.
* N=512 Gaussian-mix workload (complex V, HK2): one step with a check, every site.
* N=32 harmonic oscillator with the FDTD term in FP64: converged ground state and the
  first excited state from snapshots, against the oracle and near 3/2 and 5/2.
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


def _rel(a, b):
    return np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel())


def _pair_from_workload(name, precision=None):
    from paper_2211_10185_gb300.lattice import Lattice

    w = I.workload(name)
    n, a = w["n"], w["a"]
    v = w["potential"](n, a)
    psi0 = I.gaussian_field(n, w["seed"])
    if w["kinetic"] == I.FDTD:
        psi0 = I.zero_dirichlet_planes(psi0)
    ref = O.Lattice(n, a)
    if np.iscomplexobj(v):
        ref.set_potential(v.real, v.imag)
    else:
        ref.set_potential(v)
    ref.set_kinetic(w["kinetic"], w["m"], w["dtau"])
    ref.set_wavefunction(psi0)
    gpu = Lattice(n, a, precision=precision or w["precision"])
    gpu.set_potential(v)
    gpu.set_kinetic(w["kinetic"], w["m"], w["dtau"])
    gpu.set_wavefunction(psi0)
    return w, ref, gpu


def test_bench_workload_n256_two_steps_every_site():
    w, ref, gpu = _pair_from_workload("cornell_rel_n256")
    for _ in range(2):
        ref.step_n(1, check_every=1)
        gpu.step_n(1, check_every=1)
        e_ref, e_gpu = ref.energies(), gpu.energies()
        assert abs(e_gpu["e"] - e_ref["e"]) < 1e-5 * abs(e_ref["e"])
    # every site: relative L2 and worst site against the field's rms
    assert_field_close(gpu.get_wavefunction(), ref.psi, 2e-6 * (1 + math.log2(w["n"])), site_factor=5.0)


def test_gaussmix_workload_n512_one_step_every_site():
    w, ref, gpu = _pair_from_workload("gaussmix_symanzik_n512")
    ref.step_n(1, check_every=1)
    gpu.step_n(1, check_every=1)
    e_ref, e_gpu = ref.energies(), gpu.energies()
    assert abs(e_gpu["e"] - e_ref["e"]) < 1e-5 * abs(e_ref["e"])
    assert_field_close(gpu.get_wavefunction(), ref.psi, 2e-6 * (1 + math.log2(w["n"])))


def test_harmonic_fdtd_n32_ground_and_first_excited():
    # the plain-method configuration: N=32, a=0.15, FDTD, m=1, V=r^2/2, dtau=a^2/8, FP64,
    # until |dE| < 1e-8, then ground and first excited states
    w, ref, gpu = _pair_from_workload("ho_fdtd_n32")
    s_ref, d_ref = ref.step_n(100000, tol=w["tol"], check_every=64, snap_every=32)
    s_gpu, d_gpu = gpu.step_n(100000, tol=w["tol"], check_every=64, snap_every=32)
    assert s_ref == O.OK and s_gpu == 0 and d_ref == d_gpu
    e_ref, e_gpu = ref.energies()["e"], gpu.energies()["e"]
    assert abs(e_gpu - e_ref) < 1e-10 * abs(e_ref)
    # exact levels of this Dirichlet lattice (box |x| < 2.4 lifts them above 3/2, 5/2):
    # sums of 1D levels from a dense eigensolver on the N-1 interior sites
    n, a = w["n"], w["a"]
    x = (np.arange(1, n) - n // 2) * a
    T = (2 * np.eye(n - 1) - np.eye(n - 1, k=1) - np.eye(n - 1, k=-1)) / (2 * w["m"] * a * a)
    lev = np.linalg.eigvalsh(T + np.diag(0.5 * x * x))
    e0, e1 = 3 * lev[0], 2 * lev[0] + lev[1]
    dt = gpu.info()["dtau"]
    assert e0 - 1e-9 <= e_gpu.real < e0 + (dt * e0) ** 2
    assert 1.5 < e0 < 1.53 and 2.5 < e1 < 2.6
    st, ex_ref = ref.project_excited(2)
    ex_gpu = gpu.project_excited(2)
    assert abs(ex_gpu[0]["e"] - ex_ref[0]["e"]) < 1e-10 * abs(ex_ref[0]["e"])
    assert abs(ex_gpu[1]["e"] - ex_ref[1]["e"]) < 1e-8 * abs(ex_ref[1]["e"])
    assert abs(ex_gpu[1]["e"].real - e1) < (dt * e1) ** 2 + 1e-6


@pytest.mark.parametrize("kind,cplx", [(I.FFT_NAIVE, False), (I.FFT_SYMANZIK, True), (I.FFT_REL, True)])
def test_n256_every_fft_kinetic_and_complex_potential(kind, cplx):
    from paper_2211_10185_gb300.lattice import Lattice

    n, a, m = 256, 0.05, 0.7
    v = I.cornell(n, a, 0.4, 0.2)
    if cplx:
        v = v - 0.05j * np.abs(v)
    psi0 = I.gaussian_field(n, 31)
    ref = O.Lattice(n, a)
    if cplx:
        ref.set_potential(v.real, v.imag)
    else:
        ref.set_potential(v)
    ref.set_kinetic(kind, m)
    ref.set_wavefunction(psi0)
    gpu = Lattice(n, a, precision="c64")
    gpu.set_potential(v)
    gpu.set_kinetic(kind, m)
    gpu.set_wavefunction(psi0)
    ref.step_n(2, check_every=1)
    gpu.step_n(2, check_every=1)
    assert abs(gpu.energies()["e"] - ref.energies()["e"]) < 1e-5 * abs(ref.energies()["e"])
    assert_field_close(gpu.get_wavefunction(), ref.psi, 2e-6 * (1 + math.log2(n)))


def test_n256_excited_states_and_parity():
    w, ref, gpu = _pair_from_workload("cornell_rel_n256")
    for lat in (ref, gpu):
        lat.step_n(3 * 16, check_every=16, snap_every=16)
    st, ex_ref = ref.project_excited(3)
    ex_gpu = gpu.project_excited(3)
    for i in range(3):
        assert abs(ex_gpu[i]["e"] - ex_ref[i]["e"]) < 1e-5 * abs(ex_ref[i]["e"]), i
    ref.parity_project(O.P_MINUS_PK, 3, 1)
    gpu.parity_project(O.P_MINUS_PK, 3, 1)
    s_gpu, s_ref = gpu.get_wavefunction(1), ref.states[1]
    assert abs(abs(np.vdot(s_gpu, s_ref)) - 1) < 1e-4


def test_config2_cornell_n128_c64_c128_oracle_plateau_and_parity():
    """The N=128 Cornell workload (kappa .52, sigma .18, m 1.5, a 0.1, Eq. HK1, default dtau).

    (1) The first 192 steps from the same psi0: the FP64 oracle, the complex-FP32 and the
        FP64 GPU paths measure the same energies at every check and the same excited-state
        energies at the snapshot record (FP32 1e-5, FP64 1e-10).
    (2) Both GPU paths run to convergence: their ground-state energies agree within 1e-5;
        the FP64 path's plateau (Sec. 4's saddle point) gives E_0 < E_1 < E_2 with
        |E_i(tau_j) - E_i(tau_{j-1})| below 1e-5 |E_i| for 1S and 1P.  2S is a true saddle:
        E_2 falls by ~1e-4 per record while the states above it decay out, and rises once
        its share of the snapshots (~2e-10 near tau = 40) reaches the FP64 rounding floor,
        so the smallest difference is the slope times how near a record falls to the
        turning point (2e-6 to 3e-5 relative over runs that differ only in rounding order);
        it is bounded by 1e-4 |E_2|.  The kept states have the parity
        of 1S (even), 1P (odd) and 2S (even): projecting them leaves them unchanged.  The
        converged ground state is a fixed point of the step map, checked with the oracle's
        kinetic term.  (The FP32 path's E_1/E_2 plateau is limited here by FP32 noise: the
        2S-1P gap is small against E_1 - E_0, see the design notes.)"""
    from paper_2211_10185_gb300.lattice import Lattice

    w = I.workload("cornell_naive_n128")
    n, a, m = w["n"], w["a"], w["m"]
    v = w["potential"](n, a)
    psi0 = I.gaussian_field(n, w["seed"])
    ref = O.Lattice(n, a)
    ref.set_potential(v)
    ref.set_kinetic(w["kinetic"], m, w["dtau"])
    ref.set_wavefunction(psi0)
    lats = {}
    for prec in ("c64", "c128"):
        lat = Lattice(n, a, precision=prec, plateau_slots=3)
        lat.set_potential(v)
        lat.set_kinetic(w["kinetic"], m, w["dtau"])
        lat.set_wavefunction(psi0)
        lats[prec] = lat
    tol = {"c64": 1e-5, "c128": 1e-10}
    for _ in range(3):
        ref.step_n(64, check_every=64, snap_every=64)
        e_ref = ref.energies()["e"]
        for prec, lat in lats.items():
            lat.step_n(64, tol=0.0, check_every=64, snap_every=64)
            assert abs(lat.energies()["e"] - e_ref) < tol[prec] * abs(e_ref), prec
    st, ex_ref = ref.project_excited(3)
    for prec, lat in lats.items():
        ex = lat.track_excited(3)
        for i in range(3):
            assert abs(ex[i]["e"] - ex_ref[i]["e"]) < tol[prec] * abs(ex_ref[i]["e"]), (prec, i)
    # (2) convergence: checks every 64 steps, snapshot records every 256 (tau ~ 55)
    for prec, lat in lats.items():
        for _ in range(280):
            lat.step_n(256, tol=0.0, check_every=64, snap_every=256)
            lat.track_excited(3)
    e64, e128 = lats["c64"].energies()["e"].real, lats["c128"].energies()["e"].real
    assert abs(e64 - e128) < 1e-5 * abs(e128)
    assert lats["c128"].energies()["de"] < 1e-12
    pl = lats["c128"].excited_plateau(3)
    es = [p[1]["e"].real for p in pl]
    assert es[0] == pytest.approx(e128, rel=1e-10)
    assert es[0] < es[1] < es[2]
    for i, bound in enumerate((1e-5, 1e-5, 1e-4)):
        assert pl[i][1]["de"] < bound * abs(es[i]), (i, pl[i])
    # the kept states' parities (their admixture of the next states is ~1e-3 at the
    # plateau of E_1 and E_2, which the energies feel only squared)
    lat = lats["c128"]
    for slot, which, t in ((200, O.P_PLUS, 1e-10), (201, O.P_MINUS, 1e-5), (202, O.P_PLUS, 1e-5)):
        before = lat.get_wavefunction(slot)
        lat.parity_project(which, 3, slot)
        assert abs(abs(np.vdot(lat.get_wavefunction(slot), before)) - 1) < t, slot
    # fixed point of psi -> coef_A psi - coef_B dtau H_K psi (oracle's kinetic term)
    psi = lat.get_wavefunction()
    dt = lat.info()["dtau"]
    hk = O.apply_kinetic(psi, w["kinetic"], a, m)
    d = 1 + 0.5 * dt * v
    mp = ((2 - d) * psi - dt * hk) / d
    lam = np.vdot(psi, mp) / np.vdot(psi, psi)
    assert np.linalg.norm((mp - lam * psi).ravel()) / np.linalg.norm(psi.ravel()) < 1e-9
    for lat in lats.values():
        lat.close()
