"""FP64 CPU oracle for the imaginary-time step of quantumfdtd v3 (arXiv 2211.10185).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline / reference arm of ``bench.py`` may import or run this module.  The product
path (the CUDA library and its Python binding) never imports it, and it shares no code
with that path: the two meet only through the seeded arrays of
``paper_2211_10185_gb300.inputs``, which the callers pass in.

Everything is complex128 / float64 numpy.  The 3D discrete Fourier transform is
numpy's (``numpy.fft.fftn`` / ``ifftn``), used as a library step; nothing is blocked,
fused or reordered beyond the equations.  Arrays are C-ordered ``[iz, iy, ix]``
(x fastest); lattice site ``i`` sits at ``x_i = (i - N/2) a``.

Notation follows the paper: lattice spacing ``a`` (the paper's A), mass ``m`` (M),
lattice momentum ``k_l = a p_l``.  ``coef_A`` / ``coef_B`` are the update
coefficients (not the spacing).

Readings of points the paper leaves open (each marked "reading" below):
  * Eq. HK0's printed prefactor is garbled; it is read as -1/(2 m a^2) times the sum
    over the six neighbour differences, the only form whose symbol is Eq. HK2's
    4 sum sin^2(k/2) / (2 a^2 m).
  * Eq. eq_iterat prints H_K; the full H = H_K + V (Eq. eq_schro) is used.
  * The time discretisation is deferred to other papers.  It is read as
    Crank-Nicolson in V and explicit in H_K: (psi' - psi)/dtau = -H_K psi - V (psi' + psi)/2,
    i.e. psi' = coef_A psi - coef_B dtau H_K psi with coef_A = (1 - dtau V/2)/(1 + dtau V/2)
    and coef_B = 1/(1 + dtau V/2).
  * Dirichlet boundaries (Sec. 1) are the planes with index 0 on any axis, held at 0;
    the interior 1..N-1 is symmetric about the origin site N/2.
  * Energies are Rayleigh quotients <psi|H|psi>/<psi|psi> (complex for complex V),
    measured every ``check_every`` steps on the step's input psi; the convergence test
    is |E_t - E_{t-check_every}| < tol (complex modulus).
  * A second stopping rule for solves served in batches ("extrapolated"): the check
    energies approach their limit geometrically, so with d = |E_t - E_{t-check_every}|,
    the previous check's d_prev > d and rho = d / d_prev, the distance left is about
    d rho / (1 - rho); converged when max(d, d rho / (1 - rho)) < tol (d = 0 counts as
    converged; never while d >= d_prev).
  * Renormalisation: after a check on psi_t with norm n_t the output of the following
    step is multiplied by 1/sqrt(n_t).  The map is linear, so this only rescales.
  * Excited states (Sec. 1, "nearby temporal snapshots ... orthogonal projection"):
    classical Gram-Schmidt, latest snapshot first, with one re-orthogonalisation pass.
  * Which tau to report an excited-state energy at (Sec. 4 asks for the saddle point of
    E_i(tau)): E_i is recorded at a sequence of snapshot sets j, and the reported value
    is E_i(tau_j) at the j >= 1 that minimises |E_i(tau_j) - E_i(tau_{j-1})| (the
    earliest such j on ties), chosen for each state i separately.
  * P^-_{p_k} (Sec. 3) is used with the factor 1/4 and renormalised afterwards; the
    other axes than k flip together.
  * Default dtau = 0.75 / T_max with T_max = 6/(m a^2) (HK0, HK2), 3 pi^2/(2 m a^2)
    (HK1), sqrt(12 + (a m)^2)/a (HK3).
"""
from __future__ import annotations

import math

import numpy as np

FDTD, FFT_NAIVE, FFT_SYMANZIK, FFT_REL = 0, 1, 2, 3
P_PLUS, P_MINUS, P_MINUS_PK, P_D_K, P_D2_K = 0, 1, 2, 3, 4

OK, EINVAL, ENOMEM, ECUDA, ESTATE, ETIMEOUT, ENOTCONV = range(7)


# --------------------------------------------------------------------------------------
# Kinetic terms, Sec. 2
# --------------------------------------------------------------------------------------

def lattice_momenta(n: int) -> np.ndarray:
    """k = a p in DFT order, taking values in {-pi + 2pi/N, ..., 0, 2pi/N, ..., pi}
    (Sec. 2, definition below Eq. HK3).  Index j <= N/2 maps to 2 pi j / N, larger j to
    2 pi (j - N) / N.  Odd N is not covered by the paper's definition."""
    if n % 2:
        raise ValueError("the lattice momenta are defined for even N only")
    j = np.arange(n)
    return 2.0 * np.pi * np.where(j <= n // 2, j, j - n) / n


def kinetic_symbol(kind: int, n: int, a: float, m: float) -> np.ndarray:
    """Multiplier T(k) of the FFT kinetic terms on the N^3 DFT grid ``[kz, ky, kx]``.

    Eq. HK1: sum_l k_l^2 / (2 a^2 m).  Eq. HK2: 4 sum_l sin^2(k_l/2) / (2 a^2 m).
    Eq. HK3: sqrt(4 sum_l sin^2(k_l/2) + (a m)^2) / a.  The 1/N^3 of the equations is
    the normalisation of the inverse transform (numpy's ifftn applies it).
    """
    k = lattice_momenta(n)
    kz, ky, kx = k[:, None, None], k[None, :, None], k[None, None, :]
    if kind == FFT_NAIVE:
        return (kx ** 2 + ky ** 2 + kz ** 2) / (2.0 * a * a * m)
    khat2 = 4.0 * (np.sin(kx / 2) ** 2 + np.sin(ky / 2) ** 2 + np.sin(kz / 2) ** 2)
    if kind == FFT_SYMANZIK:
        return khat2 / (2.0 * a * a * m)
    if kind == FFT_REL:
        return np.sqrt(khat2 + (a * m) ** 2) / a
    raise ValueError(f"not an FFT kinetic term: {kind}")


def apply_kinetic_fft(psi: np.ndarray, kind: int, a: float, m: float) -> np.ndarray:
    """H_K^(1..3) psi = IFFT[T(k) FFT[psi]] / N^3 (Eqs. HK1-HK3, periodic)."""
    n = psi.shape[0]
    return np.fft.ifftn(kinetic_symbol(kind, n, a, m) * np.fft.fftn(psi))


def dirichlet_mask(n: int) -> np.ndarray:
    """1 on interior sites (all indices != 0), 0 on the Dirichlet planes (Sec. 1)."""
    inner = (np.arange(n) != 0).astype(np.float64)
    return inner[:, None, None] * inner[None, :, None] * inner[None, None, :]


def apply_kinetic_fdtd(psi: np.ndarray, a: float, m: float) -> np.ndarray:
    """H_K^(0) psi = -1/(2 m a^2) sum_{l=+-1..+-3} [psi(r + e_l) - psi(r)] (Eq. HK0, reading),
    with psi = 0 on the Dirichlet planes.  A neighbour index that leaves [0, N) wraps to
    the plane 0, which is pinned to zero."""
    mask = dirichlet_mask(psi.shape[0])
    p = psi * mask
    acc = np.zeros_like(p)
    for axis in range(3):
        for shift in (1, -1):
            acc += np.roll(p, -shift, axis=axis) - p      # psi(r + shift e_axis) - psi(r)
    return (-1.0 / (2.0 * m * a * a)) * acc * mask


def apply_kinetic(psi: np.ndarray, kind: int, a: float, m: float) -> np.ndarray:
    if kind == FDTD:
        return apply_kinetic_fdtd(psi, a, m)
    return apply_kinetic_fft(psi, kind, a, m)


def default_dtau(kind: int, a: float, m: float) -> float:
    """dtau = 0.75 / T_max (reading; the paper defers the stability study)."""
    if kind in (FDTD, FFT_SYMANZIK):
        tmax = 6.0 / (m * a * a)
    elif kind == FFT_NAIVE:
        tmax = 3.0 * math.pi ** 2 / (2.0 * m * a * a)
    elif kind == FFT_REL:
        tmax = math.sqrt(12.0 + (a * m) ** 2) / a
    else:
        raise ValueError(kind)
    return 0.75 / tmax


# --------------------------------------------------------------------------------------
# Imaginary-time step, Sec. 2 (Eq. eq_iterat and the spectral decomposition below it)
# --------------------------------------------------------------------------------------

def update_coefficients(v: np.ndarray, dtau: float):
    """coef_A = (1 - dtau V/2)/(1 + dtau V/2), coef_B = 1/(1 + dtau V/2) (reading)."""
    coef_b = 1.0 / (1.0 + 0.5 * dtau * v)
    coef_a = (1.0 - 0.5 * dtau * v) * coef_b
    return coef_a, coef_b


def reductions(psi: np.ndarray, hk_psi: np.ndarray, v: np.ndarray):
    """<psi|psi>, <psi|H_K psi>, <psi|V psi> with the Hermitian inner product."""
    w = np.abs(psi) ** 2
    return float(np.sum(w)), complex(np.vdot(psi, hk_psi)), complex(np.sum(w * v))


def energy(psi, v, kind, a, m):
    """Rayleigh quotient E = <psi|H_K + V|psi>/<psi|psi> (Eq. eq_schro)."""
    if kind == FDTD:
        psi = psi * dirichlet_mask(psi.shape[0])
    norm, ek, ev = reductions(psi, apply_kinetic(psi, kind, a, m), v)
    return (ek + ev) / norm, norm


def check_converged(rule: str, d: float, d_prev: float, tol: float) -> bool:
    """Stopping test of a check with energy difference d (previous check's d_prev):
    "difference": d < tol; "extrapolated": max(d, d rho/(1 - rho)) < tol with
    rho = d / d_prev while d < d_prev (d = 0 converged), else not converged."""
    if not math.isfinite(d):
        return False
    if rule == "difference":
        return d < tol
    if d == 0.0:
        return True
    if not math.isfinite(d_prev) or not d < d_prev:
        return False
    rho = d / d_prev
    return max(d, d * rho / (1.0 - rho)) < tol


# --------------------------------------------------------------------------------------
# Parity projectors, Sec. 3
# --------------------------------------------------------------------------------------

def mirror(psi: np.ndarray, axes=(0, 1, 2)) -> np.ndarray:
    """psi(-x) along the given array axes: site i goes to (N - i) mod N, which is the
    site at coordinate -x_i for x_i = (i - N/2) a and maps the plane 0 to itself."""
    out = psi
    for ax in axes:
        out = np.roll(np.flip(out, axis=ax), 1, axis=ax)
    return out


# paper axis k in {1, 2, 3} = (x1, x2, x3) = (x, y, z) -> numpy axis of [iz, iy, ix]
_NP_AXIS = {1: 2, 2: 1, 3: 0}


def parity(psi: np.ndarray, which: int, axis: int = 3) -> np.ndarray:
    """P^+, P^- and P^-_{p_k} (Sec. 3) and the d-wave projectors, without renormalisation.

    P^{+-} psi(r) = (psi(r) +- psi(-r)) / 2.  P^-_{p_k} (k = ``axis``) =
    ((psi(r) + psi(r with the two other axes flipped)) - (psi(r with axis k flipped)
    + psi(-r))) / 4, summed in that grouping so that mirror images are bitwise exact.

    d-wave projectors (the "new projection operators (for instance, d-wave states)" the
    paper lists as future work; reading): with the single-axis mirrors R_i, R_j of the
    two axes other than k and R_k of axis k,
      P_{d,k}  = (1 - R_i)(1 - R_j)(1 + R_k)/8   (d_xy-like for k = z: odd in x and in y),
      P_{d2,k} = (1 - S_ij)/2 (1 + R_i)(1 + R_j)(1 + R_k)/8   (d_{x^2-y^2}-like for k = z),
    S_ij exchanging the coordinates i and j.  Both are evaluated as ((a + b) - (c + d))
    groupings of mirror images so that the symmetries hold bitwise.
    """
    if which == P_PLUS:
        return 0.5 * (psi + mirror(psi))
    if which == P_MINUS:
        return 0.5 * (psi - mirror(psi))
    k = _NP_AXIS[axis]
    i, j = tuple(ax for ax in (0, 1, 2) if ax != k)
    if which == P_MINUS_PK:
        return 0.25 * ((psi + mirror(psi, (i, j))) - (mirror(psi, (k,)) + mirror(psi)))
    if which in (P_D_K, P_D2_K):
        # (1 + R_k)/2 first: even part along k
        e = 0.5 * (psi + mirror(psi, (k,)))
        if which == P_D_K:
            # (1 - R_i)(1 - R_j)/4 = ((1 + R_i R_j) - (R_i + R_j))/4
            return 0.25 * ((e + mirror(e, (i, j))) - (mirror(e, (i,)) + mirror(e, (j,))))
        # (1 + R_i)(1 + R_j)/4, then (1 - S_ij)/2
        f = 0.25 * ((e + mirror(e, (i, j))) + (mirror(e, (i,)) + mirror(e, (j,))))
        return 0.5 * (f - np.swapaxes(f, i, j))
    raise ValueError(which)


# --------------------------------------------------------------------------------------
# Gram-Schmidt on snapshots, Sec. 1 (excited states) and the decay of Sec. 2
# --------------------------------------------------------------------------------------

def gram_schmidt(vectors):
    """Orthonormal v_0, v_1, ... from the given vectors in order (latest snapshot first):
    classical Gram-Schmidt (all coefficients from the same residual) with one
    re-orthogonalisation pass, Hermitian inner product, FP64."""
    basis = []
    for s in vectors:
        w = np.array(s, dtype=np.complex128, copy=True)
        for _ in range(2):
            coeffs = [np.vdot(v, w) for v in basis]
            for c, v in zip(coeffs, basis):
                w = w - c * v
        nrm = math.sqrt(np.vdot(w, w).real)
        basis.append(w / nrm)
    return basis


def plateau_index(energies) -> int | None:
    """Index j >= 1 of the sequence E(tau_0), E(tau_1), ... that minimises
    |E(tau_j) - E(tau_{j-1})| (the earliest on ties); None for fewer than two values."""
    best, best_j = math.inf, None
    for j in range(1, len(energies)):
        d = abs(energies[j] - energies[j - 1])
        if d < best:
            best, best_j = d, j
    return best_j


# --------------------------------------------------------------------------------------
# The solver state machine (what the C ABI exposes), Sec. 2
# --------------------------------------------------------------------------------------

class Lattice:
    """One N^3 lattice: potential, kinetic term, live psi, snapshot ring, states."""

    def __init__(self, n: int, a: float, n_snap: int = 3):
        if n < 8 or n % 2:
            raise ValueError("N must be even and >= 8")
        self.n, self.a, self.n_snap = n, float(a), n_snap
        self.v = None
        self.kind = None
        self.m = None
        self.dtau = None
        self.psi = None
        self.step = 0
        self.tau = 0.0
        self.pending_scale = None
        self.last = None            # last check: dict(e, norm, de, step, tau)
        self.prev_e = None
        self.prev_de = math.inf     # energy difference at the previous check
        self.snaps = []             # latest first
        self.states = [None, None, None]
        self.state_energies = [None, None, None]
        self.history = []           # every check record
        self.excited_history = []   # one record per track_excited(): step, tau, [E_i]
        self.plateau = [None, None, None]   # per state: chosen record, energy, state

    # -- set-up ------------------------------------------------------------------------
    def set_potential(self, v_re, v_im=None):
        v = np.asarray(v_re, dtype=np.float64).reshape(self.n, self.n, self.n)
        if v_im is not None:
            v = v + 1j * np.asarray(v_im, dtype=np.float64).reshape(v.shape)
        self.v = v.astype(np.complex128)

    def set_kinetic(self, kind: int, m: float, dtau: float | None = None):
        if kind not in (FDTD, FFT_NAIVE, FFT_SYMANZIK, FFT_REL) or m <= 0:
            raise ValueError("bad kinetic term or mass")
        self.kind, self.m = kind, float(m)
        self.dtau = default_dtau(kind, self.a, self.m) if (dtau is None or dtau <= 0) else float(dtau)

    def set_wavefunction(self, psi):
        self.psi = np.array(psi, dtype=np.complex128).reshape(self.n, self.n, self.n)
        self.pending_scale = None

    # -- one step ----------------------------------------------------------------------
    def _hk(self, psi):
        return apply_kinetic(psi, self.kind, self.a, self.m)

    def step_n(self, max_steps: int, tol: float = 0.0, check_every: int = 64,
               snap_every: int | None = None, tol_rel: float = 0.0, rule: str = "difference"):
        """Advance up to ``max_steps`` steps; returns (status, steps_done).

        Step t (0-based, counted over the lattice's life) maps psi_t to
        psi_{t+1} = coef_A psi_t - coef_B dtau H_K psi_t.  When t % check_every == 0 the
        energy of psi_t is measured first; the run stops with OK after a check that meets
        ``check_converged(rule, |E_t - E_{t-check_every}|, previous difference,
        tol + tol_rel |E_t|)``.  After step t, when (t+1) % snap_every == 0, psi_{t+1} is
        pushed into the snapshot ring (latest first).
        """
        if self.v is None or self.kind is None or self.psi is None:
            return ESTATE, 0
        if snap_every is None:
            snap_every = check_every
        coef_a, coef_b = update_coefficients(self.v, self.dtau)
        fdtd = self.kind == FDTD
        mask = dirichlet_mask(self.n) if fdtd else None
        done = 0
        status = ENOTCONV
        while done < max_steps:
            t = self.step
            psi = self.psi * mask if fdtd else self.psi
            hk = self._hk(psi)
            check = check_every > 0 and t % check_every == 0
            if check:
                norm, ek, ev = reductions(psi, hk, self.v)
                e = (ek + ev) / norm
                de = abs(e - self.prev_e) if self.prev_e is not None else math.inf
                self.last = dict(e=e, norm=norm, de=de, step=t, tau=self.tau)
                self.history.append(self.last)
            new = coef_a * psi - coef_b * self.dtau * hk
            if fdtd:
                new = new * mask
            if self.pending_scale is not None:
                new = new * self.pending_scale
                self.pending_scale = None
            if check:
                self.pending_scale = 1.0 / math.sqrt(norm) if norm > 0 else 1.0
            self.psi = new
            self.step += 1
            self.tau += self.dtau
            done += 1
            if snap_every > 0 and self.step % snap_every == 0:
                self.snaps.insert(0, self.psi.copy())
                del self.snaps[self.n_snap:]
            if check:
                converged = check_converged(rule, de, self.prev_de, tol + tol_rel * abs(e))
                self.prev_e = e
                self.prev_de = de
                if converged:
                    status = OK
                    break
        return status, done

    def energies(self):
        return self.last

    # -- excited states ----------------------------------------------------------------
    def project_excited(self, n_states: int):
        """Gram-Schmidt over the latest ``n_states`` snapshots; E_i = <v_i|H|v_i>."""
        if n_states < 1 or n_states > min(3, self.n_snap) or len(self.snaps) < n_states:
            return ESTATE, None
        basis = gram_schmidt(self.snaps[:n_states])
        out = []
        for i, vec in enumerate(basis):
            e, norm = energy(vec, self.v, self.kind, self.a, self.m)
            self.states[i] = vec
            rec = dict(e=e, norm=norm, de=0.0, step=self.step, tau=self.tau)
            self.state_energies[i] = rec
            out.append(rec)
        return OK, out

    # -- plateau of E_i(tau) (Sec. 4: the saddle point of the excited-state energies) ----
    def track_excited(self, n_states: int):
        """Gram-Schmidt of the latest ``n_states`` snapshots now (``project_excited``) and
        one record E_i(tau_j) appended to ``excited_history``.  For each state i the
        running choice is updated: record j >= 1 replaces the current choice when
        |E_i(tau_j) - E_i(tau_{j-1})| is strictly smaller than the choice's difference
        (so the earliest minimiser wins), and the state v_i of record j is kept with it."""
        st, out = self.project_excited(n_states)
        if st != OK:
            return st, None
        rec = dict(step=self.step, tau=self.tau, e=[r["e"] for r in out])
        self.excited_history.append(rec)
        j = len(self.excited_history) - 1
        if j >= 1:
            prev = self.excited_history[j - 1]["e"]
            for i in range(n_states):
                if i >= len(prev):
                    continue
                d = abs(rec["e"][i] - prev[i])
                best = self.plateau[i]
                if best is None or d < best["de"]:
                    self.plateau[i] = dict(index=j, step=rec["step"], tau=rec["tau"], e=rec["e"][i], de=d,
                                           state=self.states[i].copy())
        return OK, out

    def excited_plateau(self, n_states: int):
        """Per state i < n_states, the record chosen by ``track_excited``: dict(index,
        step, tau, e, de, state); None for a state with fewer than two records."""
        return [self.plateau[i] for i in range(n_states)]

    # -- parity ------------------------------------------------------------------------
    def parity_project(self, which: int, axis: int = 3, target: int = -1):
        """Project the live psi (target -1) or state ``target`` and renormalise.
        A projection of the live psi cancels a pending renormalisation."""
        src = self.psi if target < 0 else self.states[target]
        if src is None:
            return ESTATE
        p = parity(src, which, axis)
        norm = float(np.sum(np.abs(p) ** 2))
        if norm > 0:
            p = p * (1.0 / math.sqrt(norm))
        if target < 0:
            self.psi = p
            self.pending_scale = None
        else:
            self.states[target] = p
        return OK

    def get_wavefunction(self, slot: int = -1):
        return self.psi if slot < 0 else self.states[slot]


# --------------------------------------------------------------------------------------
# Momentum-space distribution (Sec. 3, Fig. 2 right: y(p) = sqrt(4 pi) p Psi(p))
# --------------------------------------------------------------------------------------

def momentum_distribution(psi: np.ndarray, a: float):
    """Radial momentum distribution of a lattice wavefunction.

    Psi(p) is the DFT of psi (numpy's fftn, a library step); |Psi(p)|^2 is summed over
    shells of the integer lattice momentum n = (n_x, n_y, n_z), n_l in (-N/2, N/2], with
    shell b = round(|n|).  Returns (p_b, P_b, y_b): shell momentum b 2 pi / (N a), the
    probability in the shell (sum 1, Parseval), and y_b = sqrt(P_b / dp) with
    dp = 2 pi / (N a), the magnitude of y(p) = sqrt(4 pi) p Psi(p) for which the radial
    density is y(p)^2 (reading: shell average for states that are not s-waves).
    """
    n = psi.shape[0]
    w = np.abs(np.fft.fftn(psi)) ** 2
    j = np.arange(n)
    m = np.where(j <= n // 2, j, j - n).astype(np.float64)
    kk = np.sqrt(m[:, None, None] ** 2 + m[None, :, None] ** 2 + m[None, None, :] ** 2)
    b = np.floor(kk + 0.5).astype(np.int64)
    nb = int(b.max()) + 1
    P = np.bincount(b.ravel(), weights=w.ravel(), minlength=nb) / np.sum(w)
    dp = 2 * np.pi / (n * a)
    p = np.arange(nb) * dp
    return p, P, np.sqrt(P / dp)


# --------------------------------------------------------------------------------------
# Warm start across lattice sizes: spectral prolongation N -> 2N on the same box
# --------------------------------------------------------------------------------------

def prolong(psi_c: np.ndarray) -> np.ndarray:
    """Trigonometric interpolation of an N^3 field onto the 2N^3 lattice of the same box
    (a_fine = a / 2; fine site 2 j sits on coarse site j).  The coarse DFT coefficients
    with |n_l| < N/2 are kept; the Nyquist coefficient of each axis (n_l = N/2) is split
    into equal halves at +N/2 and -N/2 (reading); all other fine modes are zero."""
    nc = psi_c.shape[0]
    nf = 2 * nc
    h = nc // 2
    c = np.fft.fftn(psi_c)
    # per axis: coarse index -> list of (fine index, weight)
    idx = []
    for j in range(nc):
        m = j if j <= h else j - nc
        if m == h:
            idx.append([(h, 0.5), (nf - h, 0.5)])
        else:
            idx.append([(m % nf, 1.0)])
    f = np.zeros((nf, nf, nf), dtype=np.complex128)
    for jz in range(nc):
        for jy in range(nc):
            for (fy, wy) in idx[jy]:
                for (fz, wz) in idx[jz]:
                    for jx in range(nc):
                        for (fx, wx) in idx[jx]:
                            f[fz, fy, fx] += (wz * wy * wx) * c[jz, jy, jx]
    return np.fft.ifftn(f) * (nf ** 3 / nc ** 3)
