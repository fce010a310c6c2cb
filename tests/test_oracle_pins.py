"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these re-derive an oracle formula by retyping it: each compares the oracle
with an independent computation (a naive DFT, a continuum derivative, a textbook
eigenbasis, a dense eigensolver, an operator identity) so that a dropped term, a
wrong sign or index, or a transposed operand fails at least one test.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import qfdtd_oracle as O
from paper_2211_10185_gb300 import inputs as I

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def _rand(n, seed):
    return I.gaussian_field(n, seed)


# ----------------------------------------------------------------------------------
# The FFT step is the DFT of Eqs. HK1-HK3
# ----------------------------------------------------------------------------------

@pytest.mark.parametrize("n", [8, 12])
def test_fft_is_the_naive_dft(n):
    x = _rand(n, 11)
    j = np.arange(n)
    w = np.exp(-2j * np.pi * np.outer(j, j) / n)            # 1D DFT matrix
    # naive O(N^6) triple sum written as explicit loops over output modes
    naive = np.empty_like(x)
    for kz in range(n):
        for ky in range(n):
            for kx in range(n):
                naive[kz, ky, kx] = np.sum(x * w[kz][:, None, None] * w[ky][None, :, None]
                                           * w[kx][None, None, :])
    assert np.max(np.abs(np.fft.fftn(x) - naive)) < 1e-12 * n ** 3
    assert np.max(np.abs(np.fft.ifftn(np.fft.fftn(x)) - x)) < 1e-13


def test_lattice_momenta_match_the_paper_set():
    got = np.sort(O.lattice_momenta(8)) / np.pi
    assert np.allclose(got, GOLDEN["lattice_momenta_n8_over_pi"]["value"], atol=1e-15)
    with pytest.raises(ValueError):
        O.lattice_momenta(9)


# ----------------------------------------------------------------------------------
# Kinetic terms: plane waves, operator identities, the stencil
# ----------------------------------------------------------------------------------

def _plane_wave(n, a, q):
    """exp(i p.r) sampled at x_i = (i - N/2) a with p = 2 pi q / (N a)."""
    x = (np.arange(n) - n // 2) * a
    L = n * a
    ph = [np.exp(2j * np.pi * qq * x / L) for qq in q]      # q = (qx, qy, qz)
    return ph[2][:, None, None] * ph[1][None, :, None] * ph[0][None, None, :]


@pytest.mark.parametrize("q", [(0, 0, 0), (1, 0, 0), (0, -2, 1), (3, -3, 2), (-3, 1, 4), (4, 4, 4)])
def test_hk1_plane_waves_have_continuum_energy(q):
    # -1/(2m) d^2/dx^2 exp(ipx) = p^2/(2m) exp(ipx); on the periodic lattice this is exact
    # for every p = 2 pi q/L with a p in (-pi, pi] (Eq. HK1 with the momentum set of Sec. 2).
    n, a, m = 8, 0.3, 1.7
    psi = _plane_wave(n, a, q)
    p2 = sum((2 * np.pi * qq / (n * a)) ** 2 for qq in q)
    out = O.apply_kinetic_fft(psi, O.FFT_NAIVE, a, m)
    assert np.max(np.abs(out - p2 / (2 * m) * psi)) < 1e-11 * max(1.0, p2)


def test_hk1_aliased_index_uses_negative_momentum():
    # q = -3 and q = 5 give the same lattice function on N = 8; its energy must be that of
    # |p| = 3 (2 pi / L), not 5: the momentum set is (-pi, pi].
    n, a, m = 8, 0.25, 1.0
    psi = _plane_wave(n, a, (5, 0, 0))
    out = O.apply_kinetic_fft(psi, O.FFT_NAIVE, a, m)
    p = 2 * np.pi * 3 / (n * a)
    assert np.max(np.abs(out - p * p / (2 * m) * psi)) < 1e-10


def _periodic_stencil(psi, a, m):
    """-1/(2 m a^2) sum over the 6 neighbours of (psi_nbr - psi), periodic wrap,
    written with explicit index arithmetic."""
    n = psi.shape[0]
    idx = np.arange(n)
    up, dn = (idx + 1) % n, (idx - 1) % n
    s = (psi[up, :, :] + psi[dn, :, :] + psi[:, up, :] + psi[:, dn, :]
         + psi[:, :, up] + psi[:, :, dn] - 6 * psi)
    return -s / (2 * m * a * a)


@pytest.mark.parametrize("n", [8, 12])
def test_hk2_equals_periodic_seven_point_stencil(n):
    a, m = 0.2, 0.8
    psi = _rand(n, 3)
    out = O.apply_kinetic_fft(psi, O.FFT_SYMANZIK, a, m)
    ref = _periodic_stencil(psi, a, m)
    assert np.max(np.abs(out - ref)) < 1e-12 * np.max(np.abs(ref))


def test_hk3_squared_is_2m_hk2_plus_m2():
    # Eq. HK3 squared has the symbol (4 sum sin^2 + (a m)^2)/a^2 = 2 m T_HK2 + m^2.
    n, a, m = 12, 0.15, 0.6
    psi = _rand(n, 4)
    h3h3 = O.apply_kinetic_fft(O.apply_kinetic_fft(psi, O.FFT_REL, a, m), O.FFT_REL, a, m)
    ref = 2 * m * _periodic_stencil(psi, a, m) + m * m * psi
    assert np.max(np.abs(h3h3 - ref)) < 1e-10 * np.max(np.abs(ref))


def test_hk3_constant_state_has_energy_m():
    n, a, m = 8, 0.1, 0.37
    psi = np.full((n, n, n), 0.3 - 0.2j)
    out = O.apply_kinetic_fft(psi, O.FFT_REL, a, m)
    assert np.max(np.abs(out - GOLDEN["hk3_constant_state_energy_over_m"]["value"] * m * psi)) < 1e-13
    # the non-relativistic terms give zero on a constant
    for kind in (O.FFT_NAIVE, O.FFT_SYMANZIK):
        assert np.max(np.abs(O.apply_kinetic_fft(psi, kind, a, m))) < 1e-12


def test_hk3_small_momentum_is_relativistic_dispersion():
    # sqrt(p^2 + m^2) up to O(a^2 p^4) for a smooth plane wave (Eq. HKnr, relativistic form)
    n, a, m = 32, 0.05, 2.0
    psi = _plane_wave(n, a, (1, 1, 0))
    p2 = 2 * (2 * np.pi / (n * a)) ** 2
    out = O.apply_kinetic_fft(psi, O.FFT_REL, a, m)
    e = np.vdot(psi, out).real / np.vdot(psi, psi).real
    assert abs(e - math.sqrt(p2 + m * m)) < 2 * a * a * p2 * p2


@pytest.mark.parametrize("q", [(1, 1, 1), (2, 1, 3), (7, 5, 1)])
def test_fdtd_dirichlet_sine_modes(q):
    # Textbook: on sites 1..N-1 with psi_0 = psi_N = 0, sin(pi q j / N) is an eigenvector of
    # -(psi_{j+1} + psi_{j-1} - 2 psi_j)/(2 m a^2) with eigenvalue 2 sin^2(pi q/(2N))/(m a^2).
    n, a, m = 8, 0.4, 1.3
    j = np.arange(n)
    s = [np.sin(np.pi * qq * j / n) for qq in q]
    psi = (s[2][:, None, None] * s[1][None, :, None] * s[0][None, None, :]).astype(complex)
    lam = sum(2 * np.sin(np.pi * qq / (2 * n)) ** 2 / (m * a * a) for qq in q)
    out = O.apply_kinetic_fdtd(psi, a, m)
    assert np.max(np.abs(out - lam * psi)) < 1e-12 * lam
    # values left on the Dirichlet planes are ignored
    junk = psi.copy()
    junk[0] = 5.0
    junk[:, :, 0] = -2.0
    assert np.max(np.abs(O.apply_kinetic_fdtd(junk, a, m) - lam * psi)) < 1e-12 * lam


# ----------------------------------------------------------------------------------
# The step map
# ----------------------------------------------------------------------------------

def test_step_map_on_plane_wave_with_constant_potential():
    # (psi' - psi)/dtau = -H_K psi - V (psi' + psi)/2 with H_K psi = T psi and V = v const
    # solves to psi' = [(1 - dtau v/2 - dtau T)/(1 + dtau v/2)] psi.
    n, a, m, dtau = 8, 0.3, 1.2, 0.004
    v = 0.7 - 0.3j
    q = (1, -2, 0)
    psi0 = _plane_wave(n, a, q)
    T = sum((2 * np.pi * qq / (n * a)) ** 2 for qq in q) / (2 * m)   # HK1, exact
    lat = O.Lattice(n, a)
    lat.set_potential(np.full((n, n, n), v.real), np.full((n, n, n), v.imag))
    lat.set_kinetic(O.FFT_NAIVE, m, dtau)
    lat.set_wavefunction(psi0)
    st, done = lat.step_n(7, tol=0.0, check_every=0)
    assert st == O.ENOTCONV and done == 7
    lam = (1 - dtau * v / 2 - dtau * T) / (1 + dtau * v / 2)
    assert np.max(np.abs(lat.psi - lam ** 7 * psi0)) < 1e-13


def test_checks_measure_energy_and_renormalise():
    n, a, m, dtau = 8, 0.3, 1.0, 0.01
    v = 0.25
    q = (1, 0, 0)
    psi0 = 3.0 * _plane_wave(n, a, q)
    T = (2 * np.pi / (n * a)) ** 2 / (2 * m)
    lat = O.Lattice(n, a)
    lat.set_potential(np.full((n, n, n), v))
    lat.set_kinetic(O.FFT_NAIVE, m, dtau)
    lat.set_wavefunction(psi0)
    lat.step_n(3, check_every=2)          # checks at t = 0 and t = 2
    hist = lat.history
    assert [h["step"] for h in hist] == [0, 2]
    for h in hist:
        assert abs(h["e"] - (T + v)) < 1e-12
    assert hist[0]["norm"] == pytest.approx(9.0 * n ** 3, rel=1e-13)
    # the output of step 1 (after the check at t = 0) is rescaled by 1/sqrt(norm_0)
    lam = (1 - dtau * v / 2 - dtau * T) / (1 + dtau * v / 2)
    assert hist[1]["norm"] == pytest.approx(abs(lam) ** 4 * 9.0 * n ** 3 / (9.0 * n ** 3), rel=1e-12)


def test_default_dtau_matches_the_a2_over_8_of_the_fdtd_harmonic_run():
    assert O.default_dtau(O.FDTD, 0.15, 1.0) == pytest.approx(0.15 ** 2 / 8, rel=1e-15)


# ----------------------------------------------------------------------------------
# Converged energies against dense linear algebra (separable harmonic oscillator)
# ----------------------------------------------------------------------------------

def _fixed_point_rq(n, a, m, dtau, occupations):
    """Rayleigh quotient <H_K + V> of the fixed point of the step for a separable
    state with the given 1D occupations: the fixed point psi of psi -> coef_A psi -
    coef_B dtau H_K psi obeys (H_K + c V) psi = mu psi with c = 1 - dtau mu / 2, solved
    here self-consistently with a dense 1D eigensolver on the Dirichlet interior."""
    x = (np.arange(1, n) - n // 2) * a
    M = n - 1
    T = (2 * np.eye(M) - np.eye(M, k=1) - np.eye(M, k=-1)) / (2 * m * a * a)
    V = np.diag(0.5 * x * x)
    c = 1.0
    for _ in range(200):
        w, U = np.linalg.eigh(T + c * V)
        mu = sum(w[o] for o in occupations)
        c_new = 1 - dtau * mu / 2
        if abs(c_new - c) < 1e-16:
            break
        c = c_new
    v_exp = sum(U[:, o] @ V @ U[:, o] for o in occupations)
    exact = sum(np.linalg.eigvalsh(T + V)[o] for o in occupations)
    return mu + (1 - c) * v_exp, exact


def test_harmonic_ground_and_first_excited_match_dense_eigensolver():
    n, a, m = 16, 0.3, 1.0
    dtau = a * a / 8
    lat = O.Lattice(n, a)
    lat.set_potential(I.harmonic(n, a))
    lat.set_kinetic(O.FDTD, m, dtau)
    lat.set_wavefunction(I.gaussian_field(n, 0))
    st, done = lat.step_n(20 * 64, tol=1e-13, check_every=64, snap_every=32)
    e0 = lat.energies()["e"]
    st, ex = lat.project_excited(2)
    assert st == O.OK
    rq0, ex0 = _fixed_point_rq(n, a, m, dtau, (0, 0, 0))
    rq1, ex1 = _fixed_point_rq(n, a, m, dtau, (0, 0, 1))
    assert abs(e0.imag) < 1e-14
    assert abs(e0.real - rq0) < 1e-12
    assert abs(ex[0]["e"].real - rq0) < 1e-12
    assert abs(ex[1]["e"].real - rq1) < 1e-9
    # Rayleigh quotients sit above the exact lattice eigenvalues by O(dtau^2)
    assert 0 <= e0.real - ex0 < (dtau * 1.5) ** 2
    # and near the continuum 3/2, 5/2 at this spacing
    lv = GOLDEN["harmonic_levels_over_omega"]["value"]
    assert abs(e0.real - lv[0]) < 0.03 and abs(ex[1]["e"].real - lv[1]) < 0.1


def test_second_excited_state_is_in_the_n2_band():
    n, a, m = 16, 0.3, 1.0
    dtau = a * a / 8
    lat = O.Lattice(n, a)
    lat.set_potential(I.harmonic(n, a))
    lat.set_kinetic(O.FDTD, m, dtau)
    lat.set_wavefunction(I.gaussian_field(n, 0))
    lat.step_n(12 * 64, tol=0.0, check_every=64, snap_every=32)   # tau ~ 8.6: plateau
    st, ex = lat.project_excited(3)
    # exact lattice levels of the n = 2 band: 2s-like (2e0+e2... ) and d-like combos
    x = (np.arange(1, n) - n // 2) * a
    T = (2 * np.eye(n - 1) - np.eye(n - 1, k=1) - np.eye(n - 1, k=-1)) / (2 * m * a * a)
    w = np.linalg.eigvalsh(T + np.diag(0.5 * x * x))
    band = sorted([2 * w[0] + w[2], w[0] + 2 * w[1]])
    assert band[0] - 0.02 < ex[2]["e"].real < band[1] + 0.02


# ----------------------------------------------------------------------------------
# Brute force: dense Hamiltonian at N = 8 for non-separable cases
# ----------------------------------------------------------------------------------

def _dense(kind, n, a, m, v):
    dim = n ** 3
    H = np.empty((dim, dim), dtype=complex)
    for s in range(dim):
        e = np.zeros(dim, dtype=complex)
        e[s] = 1.0
        H[:, s] = O.apply_kinetic(e.reshape(n, n, n), kind, a, m).ravel()
    return H + np.diag(v.ravel())


@pytest.mark.parametrize("kind", [O.FFT_REL, O.FFT_NAIVE])
def test_cornell_iteration_converges_to_dense_ground_state(kind):
    n, a, m = 8, 0.25, 1.5
    v = I.cornell(n, a, 0.52, 0.18)
    lat = O.Lattice(n, a)
    lat.set_potential(v)
    lat.set_kinetic(kind, m, None)
    lat.set_wavefunction(I.gaussian_field(n, 5))
    st, done = lat.step_n(200000, tol=1e-12, check_every=32)
    assert st == O.OK
    lam = np.linalg.eigvalsh(_dense(kind, n, a, m, v))
    e = lat.energies()["e"].real
    dt = lat.dtau
    assert lam[0] - 1e-9 <= e <= lam[0] + 50 * (dt * abs(lam[0])) ** 2 + 1e-9


def test_complex_potential_energy_matches_dense_eigenvalue():
    # non-Hermitian H = H_K + V with complex V (Sec. 1, non-equilibrium potentials).  The
    # fixed point of the step obeys (H_K + c V) psi = mu psi with c = 1 - dtau mu/2
    # (complex here); solve that self-consistently with a dense eigensolver, taking the
    # eigenvalue of smallest real part, and compare Rayleigh quotients.  The exact
    # eigenvalue of H is within O(dtau) of it (first order: H is not Hermitian).
    n, a, m = 8, 0.3, 1.0
    v = I.gaussian_mix(n, a, seed=3, n_gauss=4)
    lat = O.Lattice(n, a)
    lat.set_potential(v.real, v.imag)
    lat.set_kinetic(O.FFT_SYMANZIK, m, None)
    lat.set_wavefunction(I.gaussian_field(n, 6))
    st, done = lat.step_n(200000, tol=1e-13, check_every=32)
    assert st == O.OK
    H = _dense(O.FFT_SYMANZIK, n, a, m, v)
    K = H - np.diag(v.ravel())
    dtau, c = lat.dtau, 1.0
    for _ in range(100):
        w, U = np.linalg.eig(K + c * np.diag(v.ravel()))
        i = np.argmin(w.real)
        c_new = 1 - dtau * w[i] / 2
        if abs(c_new - c) < 1e-15:
            break
        c = c_new
    u = U[:, i]
    rq = np.vdot(u, H @ u) / np.vdot(u, u)
    assert abs(lat.energies()["e"] - rq) < 1e-9 * abs(rq)
    lam = np.linalg.eigvals(H)
    target = lam[np.argmin(lam.real)]
    assert abs(lat.energies()["e"] - target) < dtau * abs(target) ** 2


# ----------------------------------------------------------------------------------
# Coulomb ground state approaches -m kappa^2 / 2 (Sec. 3)
# ----------------------------------------------------------------------------------

@pytest.mark.slow
def test_coulomb_ground_state_approaches_analytic_value():
    exact = GOLDEN["coulomb_levels_over_m_kappa2"]["value"]["1s"]          # m = kappa = 1
    errs = []
    for n, a in [(24, 0.5), (32, 0.375)]:                                 # L = 12 fixed
        lat = O.Lattice(n, a)
        lat.set_potential(I.cornell(n, a, 1.0, 0.0))
        lat.set_kinetic(O.FFT_SYMANZIK, 1.0, None)
        lat.set_wavefunction(np.exp(-I.radius(n, a)) + 0j)
        st, _ = lat.step_n(50000, tol=1e-9, check_every=32)
        assert st == O.OK
        errs.append(lat.energies()["e"].real - exact)
    assert 0 < errs[1] < errs[0] < 0.05


# ----------------------------------------------------------------------------------
# Parity projectors, Sec. 3
# ----------------------------------------------------------------------------------

def test_mirror_index_map_enumerated_on_n8():
    n, a = 8, 0.5
    x = (np.arange(n) - n // 2) * a
    L = n * a
    probe = np.arange(n ** 3, dtype=float).reshape(n, n, n)
    mir = O.mirror(probe)
    for iz in range(n):
        for iy in range(n):
            for ix in range(n):
                # the site whose coordinates are -(x, y, z) modulo the period L
                jx, jy, jz = [int(np.argmin(np.abs(((x + c) + L / 2) % L - L / 2)))
                              for c in (x[ix], x[iy], x[iz])]
                assert mir[iz, iy, ix] == probe[jz, jy, jx]


def test_projector_algebra():
    n = 8
    psi = _rand(n, 9)
    pp = O.parity(psi, O.P_PLUS)
    pm = O.parity(psi, O.P_MINUS)
    assert np.max(np.abs(pp + pm - psi)) < 1e-15
    assert np.max(np.abs(O.parity(pp, O.P_PLUS) - pp)) < 1e-15
    assert np.max(np.abs(O.parity(pm, O.P_PLUS))) < 1e-15
    for k in (1, 2, 3):
        pk = O.parity(psi, O.P_MINUS_PK, k)
        assert np.max(np.abs(O.parity(pk, O.P_MINUS_PK, k) - pk)) < 1e-15
        # P-_{p_k} output is odd overall, so P+ annihilates it
        assert np.max(np.abs(O.parity(pk, O.P_PLUS))) < 1e-15


def test_projected_states_are_bitwise_mirror_symmetric():
    n = 12
    psi = _rand(n, 10)
    pp = O.parity(psi, O.P_PLUS)
    assert np.array_equal(pp, O.mirror(pp))
    pm = O.parity(psi, O.P_MINUS)
    assert np.array_equal(pm, -O.mirror(pm))
    pk = O.parity(psi, O.P_MINUS_PK, 3)
    assert np.array_equal(pk, -O.mirror(pk, (0,)))          # odd under z -> -z
    assert np.array_equal(pk, O.mirror(pk, (1, 2)))         # even under (x, y) -> -(x, y)


def test_parity_of_analytic_s_and_p_states():
    # Sec. 3: P+ Psi_s = Psi_s, P-_{p_k} Psi_s = 0, P+ Psi_p = 0, P-_{p_k} Psi_{p_k} = Psi_{p_k}.
    n, a = 16, 0.75
    x = (np.arange(n) - n // 2) * a
    X, Y, Z = x[None, None, :], x[None, :, None], x[:, None, None]
    g = np.exp(-(X ** 2 + Y ** 2 + Z ** 2) / 2) * np.ones((n, n, n))
    s = I.zero_dirichlet_planes(g + 0j)             # planes 0 are their own mirror
    pz = I.zero_dirichlet_planes(Z * g + 0j)
    px = I.zero_dirichlet_planes(X * g + 0j)
    assert np.max(np.abs(O.parity(s, O.P_PLUS) - s)) < 1e-15
    assert np.max(np.abs(O.parity(s, O.P_MINUS_PK, 3))) < 1e-15
    assert np.max(np.abs(O.parity(pz, O.P_PLUS))) < 1e-15
    # with the factor 1/4 the projector returns a p_k state unchanged, as Sec. 3 states
    # (the printed 1/2 would double it)
    assert np.max(np.abs(O.parity(pz, O.P_MINUS_PK, 3) - pz)) < 1e-15
    assert np.max(np.abs(O.parity(px, O.P_MINUS_PK, 3))) < 1e-15
    assert np.max(np.abs(O.parity(px, O.P_MINUS_PK, 1) - px)) < 1e-15
    # renormalised projection through the solver returns the normalised p_z state
    lat = O.Lattice(n, a)
    lat.set_wavefunction(pz + 0.3 * s)
    lat.parity_project(O.P_MINUS_PK, 3, -1)
    ref = pz / np.sqrt(np.vdot(pz, pz).real)
    assert np.max(np.abs(lat.psi - ref)) < 1e-14


def test_excited_state_parity_for_the_oscillator():
    # the first excited band of the oscillator is p-like: P+ removes it, P- keeps it
    n, a, m = 16, 0.3, 1.0
    lat = O.Lattice(n, a)
    lat.set_potential(I.harmonic(n, a))
    lat.set_kinetic(O.FDTD, m, a * a / 8)
    lat.set_wavefunction(I.gaussian_field(n, 0))
    lat.step_n(15 * 64, tol=0.0, check_every=64, snap_every=32)
    st, ex = lat.project_excited(2)
    v0, v1 = lat.states[0], lat.states[1]
    # the opposite-parity admixture left after imaginary time tau decays like
    # exp(-2 (E1 - E0) tau) in norm^2 (gap 1 here)
    bound = 10 * math.exp(-2 * lat.tau)
    assert np.vdot(O.parity(v0, O.P_PLUS), O.parity(v0, O.P_PLUS)).real > 1 - bound
    assert np.vdot(O.parity(v1, O.P_PLUS), O.parity(v1, O.P_PLUS)).real < bound


# ----------------------------------------------------------------------------------
# Momentum-space distribution (Sec. 3, Fig. 2 right)
# ----------------------------------------------------------------------------------

def test_momentum_distribution_of_a_gaussian_matches_its_fourier_transform():
    # psi = exp(-r^2/(2 s^2)) is well resolved (s >> a) and small at the box edge, so its
    # lattice transform at momentum p_n = 2 pi n/(N a) is the continuum one, with
    # |Psi(p)|^2 proportional to exp(-p^2 s^2); sum that over the modes of each shell,
    # enumerated one by one.
    n, a, s = 32, 0.3, 1.0
    r = I.radius(n, a)
    psi = np.exp(-r * r / (2 * s * s)) + 0j
    p, P, y = O.momentum_distribution(psi, a)
    assert P.sum() == pytest.approx(1.0, abs=1e-13)
    dp = 2 * np.pi / (n * a)
    shells = {}
    half = n // 2
    for nz in range(-half + 1, half + 1):
        for ny in range(-half + 1, half + 1):
            for nx in range(-half + 1, half + 1):
                mag = (nx * nx + ny * ny + nz * nz) ** 0.5
                b = int(mag + 0.5)
                shells[b] = shells.get(b, 0.0) + np.exp(-(dp * mag * s) ** 2)
    tot = sum(shells.values())
    for b in range(0, 10):
        assert abs(P[b] - shells[b] / tot) < 1e-5, b
    assert np.allclose(y, np.sqrt(P / dp))


def test_momentum_distribution_of_a_plane_wave_is_one_shell():
    n, a = 16, 0.5
    x = (np.arange(n) - n // 2) * a
    q = (3, 4, 0)    # |n| = 5
    L = n * a
    psi = (np.exp(2j * np.pi * q[2] * x / L)[:, None, None] * np.exp(2j * np.pi * q[1] * x / L)[None, :, None]
           * np.exp(2j * np.pi * q[0] * x / L)[None, None, :])
    p, P, y = O.momentum_distribution(psi, a)
    assert P[5] == pytest.approx(1.0, abs=1e-12)
    assert np.sum(np.abs(np.delete(P, 5))) < 1e-12
    assert p[5] == pytest.approx(5 * 2 * np.pi / (n * a))


def test_d_wave_projectors_on_analytic_states():
    # d_xy ~ x y g, d_{x^2-y^2} ~ (x^2 - y^2) g, with g = exp(-r^2/2); s ~ g, p_x ~ x g
    n, a = 16, 0.75
    x = (np.arange(n) - n // 2) * a
    X, Y, Z = x[None, None, :], x[None, :, None], x[:, None, None]
    g = np.exp(-(X ** 2 + Y ** 2 + Z ** 2) / 2) * np.ones((n, n, n))
    z = I.zero_dirichlet_planes
    s, px = z(g + 0j), z(X * g + 0j)
    dxy, dx2y2, dyz = z(X * Y * g + 0j), z((X ** 2 - Y ** 2) * g + 0j), z(Y * Z * g + 0j)
    D, D2 = O.P_D_K, O.P_D2_K
    assert np.max(np.abs(O.parity(dxy, D, 3) - dxy)) < 1e-15          # d_xy: kept by P_{d,z}
    assert np.max(np.abs(O.parity(dyz, D, 1) - dyz)) < 1e-15          # d_yz: kept by P_{d,x}
    assert np.max(np.abs(O.parity(dx2y2, D2, 3) - dx2y2)) < 1e-15     # d_{x^2-y^2}: kept by P_{d2,z}
    for f in (s, px, dx2y2, dyz):
        assert np.max(np.abs(O.parity(f, D, 3))) < 1e-15
    for f in (s, px, dxy, dyz):
        assert np.max(np.abs(O.parity(f, D2, 3))) < 1e-15


def test_d_wave_projectors_are_idempotent_and_exactly_symmetric():
    n = 12
    psi = _rand(n, 12)
    for which in (O.P_D_K, O.P_D2_K):
        for k in (1, 2, 3):
            q = O.parity(psi, which, k)
            assert np.max(np.abs(O.parity(q, which, k) - q)) < 1e-15
            kk = O._NP_AXIS[k]
            i, j = tuple(ax for ax in (0, 1, 2) if ax != kk)
            assert np.array_equal(q, O.mirror(q, (kk,)))                  # even along k
            if which == O.P_D_K:
                assert np.array_equal(q, -O.mirror(q, (i,)))              # odd along i
                assert np.array_equal(q, -O.mirror(q, (j,)))              # odd along j
            else:
                assert np.array_equal(q, O.mirror(q, (i,)))
                assert np.array_equal(q, -np.swapaxes(q, i, j))            # odd under i <-> j
            # d projections are orthogonal to P+ (s, d) ... and to P- (p, f) complements
            assert np.max(np.abs(O.parity(q, O.P_MINUS))) < 1e-15


# ----------------------------------------------------------------------------------
# Spectral prolongation N -> 2N (warm start across lattice sizes)
# ----------------------------------------------------------------------------------

def test_prolongation_keeps_coarse_values_and_band_limited_functions():
    nc = 8
    psi = _rand(nc, 13)
    f = O.prolong(psi)
    # fine site 2 j coincides with coarse site j
    assert np.max(np.abs(f[::2, ::2, ::2] - psi)) < 1e-13
    # a band-limited periodic function is reproduced at every fine site
    L = 2 * np.pi
    xc = (np.arange(nc) - nc // 2) * (L / nc)
    xf = (np.arange(2 * nc) - nc) * (L / (2 * nc))

    def fn(x):
        X, Y, Z = x[None, None, :], x[None, :, None], x[:, None, None]
        return np.exp(1j * (2 * X - Y)) + 0.5 * np.cos(3 * Z) * np.sin(X) + 0.2

    assert np.max(np.abs(O.prolong(fn(xc)) - fn(xf))) < 1e-12
    # the Nyquist mode cos(4 x) (coarse N = 8) stays real and even on the fine grid
    nyq = np.cos(4 * xc)[None, None, :] * np.ones((nc, nc, nc))
    fny = O.prolong(nyq + 0j)
    assert np.max(np.abs(fny.imag)) < 1e-13
    assert np.max(np.abs(fny[::2, ::2, ::2] - nyq)) < 1e-13


@pytest.mark.parametrize("kind", [O.FFT_NAIVE, O.FFT_SYMANZIK, O.FFT_REL])
def test_kinetic_energy_in_k_space_equals_real_space(kind):
    """Parseval: <v|H_K v> computed in position space (inverse transform, then the
    Hermitian inner product) equals sum_k T(k) |v^(k)|^2 / N^3 with the unnormalised
    forward DFT -- the identity the GPU uses for the energies of excited states.  A
    dropped 1/N^3, a conjugate or a symbol on the wrong axis order fails it."""
    rng = np.random.default_rng(11)
    for n in (8, 12):
        a, m = 0.3, 0.7
        v = rng.standard_normal((n, n, n)) + 1j * rng.standard_normal((n, n, n))
        real_space = np.vdot(v, O.apply_kinetic_fft(v, kind, a, m))
        k_space = np.sum(O.kinetic_symbol(kind, n, a, m) * np.abs(np.fft.fftn(v)) ** 2) / n ** 3
        assert abs(real_space.imag) < 1e-10 * abs(real_space)
        assert abs(real_space.real - k_space) < 1e-12 * abs(k_space)
    # a plane wave with a different momentum on each axis: the energy is the symbol at
    # exactly that (kx, ky, kz), written out here from Eqs. HK1-HK3
    j = np.arange(16)
    kx, ky, kz = 2 * np.pi * np.array([1, 2, 3]) / 16
    pw = np.exp(1j * (kx * j[None, None, :] + ky * j[None, :, None] + kz * j[:, None, None]))
    e = np.vdot(pw, O.apply_kinetic_fft(pw, kind, 0.3, 0.7)).real / np.vdot(pw, pw).real
    sym = {O.FFT_NAIVE: (kx ** 2 + ky ** 2 + kz ** 2) / (2 * 0.09 * 0.7),
           O.FFT_SYMANZIK: 4 * (np.sin(kx / 2) ** 2 + np.sin(ky / 2) ** 2 + np.sin(kz / 2) ** 2) / (2 * 0.09 * 0.7),
           O.FFT_REL: np.sqrt(4 * (np.sin(kx / 2) ** 2 + np.sin(ky / 2) ** 2 + np.sin(kz / 2) ** 2) + 0.21 ** 2) / 0.3}
    assert abs(e - sym[kind]) < 1e-10 * sym[kind]


# ----------------------------------------------------------------------------------
# The plateau ("saddle point") of E_i(tau), Sec. 4: the reported excited-state energy
# ----------------------------------------------------------------------------------

@pytest.mark.parametrize("cond", [1.0, 1e-6])
def test_gram_schmidt_matches_householder_qr(cond):
    """Sec. 1's orthogonalisation of the snapshots: the oracle's Gram-Schmidt of three
    vectors equals the Q of a Householder QR (numpy) up to a unit phase per column, also
    for snapshots that are nearly parallel (the excited shares of late snapshots are
    small: third vector = first + cond x noise)."""
    rng = np.random.default_rng(7)
    m = 4096
    a = rng.standard_normal((m, 3)) + 1j * rng.standard_normal((m, 3))
    a[:, 2] = a[:, 0] + cond * (rng.standard_normal(m) + 1j * rng.standard_normal(m))
    basis = O.gram_schmidt([a[:, j] for j in range(3)])
    q, r = np.linalg.qr(a)
    g = np.stack(basis, axis=1)
    assert np.abs(g.conj().T @ g - np.eye(3)).max() < 1e-12
    for j in range(3):
        overlap = np.vdot(q[:, j], g[:, j])
        assert abs(abs(overlap) - 1) < 1e-10, (j, overlap)
        # each v_j lies in the span of the first j + 1 vectors (triangular structure)
        coef = np.linalg.lstsq(a[:, : j + 1], g[:, j], rcond=None)[0]
        assert np.linalg.norm(a[:, : j + 1] @ coef - g[:, j]) < 1e-9


def test_plateau_index_on_hand_made_sequences():
    # differences 2, .5, .1, .05, 6.55: the flattest step ends at index 4
    assert O.plateau_index([5.0, 3.0, 2.5, 2.4, 2.45, 9.0]) == 4
    # ties: the earliest minimiser; complex values by modulus
    assert O.plateau_index([1.0, 1.0, 1.0]) == 1
    assert O.plateau_index([1 + 1j, 1 + 0.5j, 1 + 0.6j, 2 + 0j]) == 2
    assert O.plateau_index([1.0]) is None and O.plateau_index([]) is None


def test_plateau_picks_the_exact_first_excited_level_of_the_oscillator():
    """Snapshots every 64 steps (delta (E1 - E0) ~ 0.7) of the Dirichlet oscillator up to
    tau ~ 43: early records carry the higher states, late ones have lost Psi_1 below FP64
    rounding (weight e^-tau).  The chosen E_1 must be the fixed point of the step for a
    first excited state (the self-consistent dense 1D eigensolve) to 1e-9, where neither
    the earliest nor the latest record is within 1e-3."""
    n, a, m = 16, 0.3, 1.0
    dtau = a * a / 8
    lat = O.Lattice(n, a)
    lat.set_potential(I.harmonic(n, a))
    lat.set_kinetic(O.FDTD, m, dtau)
    lat.set_wavefunction(I.gaussian_field(n, 0))
    for j in range(60):
        lat.step_n(64, check_every=64, snap_every=64)
        if j >= 2:
            assert lat.track_excited(3)[0] == O.OK
    rq0, _ = _fixed_point_rq(n, a, m, dtau, (0, 0, 0))
    rq1, _ = _fixed_point_rq(n, a, m, dtau, (0, 0, 1))
    hist = lat.excited_history
    e1 = [r["e"][1] for r in hist]
    p0, p1, p2 = lat.excited_plateau(3)
    assert abs(p0["e"] - rq0) < 1e-12
    assert abs(p1["e"] - rq1) < 1e-9
    assert abs(e1[0] - rq1) > 1e-3 and abs(e1[-1] - rq1) > 1e-3
    # the running choice equals the plain argmin over the recorded sequence
    assert p1["index"] == O.plateau_index(e1)
    assert p1["e"] == e1[p1["index"]] and p1["step"] == hist[p1["index"]]["step"]
    # the kept state is the Gram-Schmidt state of that record: an eigenvector of the step
    # map psi -> coef_A psi - coef_B dtau H_K psi (written out here from Eq. HK0's stencil)
    v = p1["state"]
    pad = np.pad(v, 1)
    lap = sum(np.roll(pad, s, axis=ax) for ax in range(3) for s in (1, -1))[1:-1, 1:-1, 1:-1] - 6 * v
    mask = O.dirichlet_mask(n)
    hk = -lap / (2 * m * a * a) * mask
    d = 1 + dtau * lat.v / 2
    mv = ((2 - d) * v - dtau * hk) / d * mask
    lam = np.vdot(v, mv) / np.vdot(v, v)
    assert np.linalg.norm((mv - lam * v).ravel()) / np.linalg.norm(v.ravel()) < 1e-7
    # E_2 lies in the (lattice-split) n = 2 band of the oscillator
    x = (np.arange(1, n) - n // 2) * a
    T = (2 * np.eye(n - 1) - np.eye(n - 1, k=1) - np.eye(n - 1, k=-1)) / (2 * m * a * a)
    w = np.linalg.eigvalsh(T + np.diag(0.5 * x * x))
    band = sorted([2 * w[0] + w[2], w[0] + 2 * w[1]])
    assert band[0] - 0.02 < p2["e"].real < band[1] + 0.02


# ----------------------------------------------------------------------------------
# Stopping rules (the paper has none; readings): difference and extrapolated
# ----------------------------------------------------------------------------------

def _stop_index(rule, energies, tol):
    d_prev, prev = math.inf, None
    for j, e in enumerate(energies):
        d = abs(e - prev) if prev is not None else math.inf
        if O.check_converged(rule, d, d_prev, tol):
            return j
        prev, d_prev = e, d
    return None


def test_extrapolated_rule_bounds_the_distance_to_the_limit():
    # a slowly contracting sequence E_j = 1 + 0.01 * 0.99^j: the difference rule stops
    # where the distance left is ~99 x tol; the extrapolated rule within tol
    tol = 1e-6
    seq = [1.0 + 0.01 * 0.99 ** j for j in range(3000)]
    jd = _stop_index("difference", seq, tol)
    je = _stop_index("extrapolated", seq, tol)
    assert seq[jd] - 1.0 > 50 * tol
    assert seq[je] - 1.0 < tol and je > jd
    # a fast one (rho = 0.1): both stop right away, at the same check
    fast = [2.0 + 0.5 * 0.1 ** j for j in range(40)]
    assert _stop_index("extrapolated", fast, tol) == _stop_index("difference", fast, tol)
    # an exact repeat converges; a growing difference never does
    assert O.check_converged("extrapolated", 0.0, math.inf, tol)
    assert not O.check_converged("extrapolated", 1e-9, 1e-10, tol)
    assert not O.check_converged("extrapolated", 1e-9, math.inf, tol)


def test_extrapolated_rule_in_a_solve_stops_near_the_converged_energy():
    n, a, m = 16, 0.3, 1.0
    dtau = a * a / 8
    ref = O.Lattice(n, a)
    ref.set_potential(I.harmonic(n, a))
    ref.set_kinetic(O.FDTD, m, dtau)
    ref.set_wavefunction(I.gaussian_field(n, 0))
    ref.step_n(40 * 64, tol=1e-14, check_every=64)
    e_inf = ref.energies()["e"].real
    for rule in ("difference", "extrapolated"):
        lat = O.Lattice(n, a)
        lat.set_potential(I.harmonic(n, a))
        lat.set_kinetic(O.FDTD, m, dtau)
        lat.set_wavefunction(I.gaussian_field(n, 0))
        # check every 8 steps: slow contraction per check (rho ~ exp(-8 dtau (E1 - E0)))
        st, done = lat.step_n(40000, tol=0.0, tol_rel=1e-6, check_every=8, rule=rule)
        assert st == O.OK
        err = abs(lat.energies()["e"].real - e_inf) / e_inf
        if rule == "difference":
            assert err > 2e-6   # several times the tolerance
        else:
            assert err < 1e-6
