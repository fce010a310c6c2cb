"""Seeded synthetic inputs shared by the CUDA path, the FP64 oracle and the benchmark.

This module holds no arithmetic of the solver: it only produces the initial
wavefunction and the external potentials, as host FP64 numpy arrays, so that both
sides of every comparison consume identical bytes.

Layout: every field is a C-ordered ``(N, N, N)`` array indexed ``[iz, iy, ix]``
(x fastest), i.e. flat site index ``(iz*N + iy)*N + ix``.  Lattice site ``i`` on an
axis sits at coordinate ``x_i = (i - N/2) * a`` so the origin is the site ``N/2``
(the paper writes Psi(r) = Psi[(A x1, A x2, A x3)], Sec. 2 below Eq. HK3).

Random numbers come from a counter-based generator: SplitMix64 (Steele, Lea and
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014) used as a
hash of ``(seed, element, draw)``, turned into normals by the Box-Muller transform.
Any element of any field can therefore be regenerated independently.
"""
from __future__ import annotations

import numpy as np

_U64 = np.uint64
_MASK53 = float(2.0 ** -53)


def splitmix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 finaliser applied to ``x + golden`` (uint64 arrays, wrapping)."""
    with np.errstate(over="ignore"):
        z = (x + _U64(0x9E3779B97F4A7C15)).astype(np.uint64)
        z = (z ^ (z >> _U64(30))) * _U64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> _U64(27))) * _U64(0x94D049BB133111EB)
        return z ^ (z >> _U64(31))


def uniform01(seed: int, counter: np.ndarray, draw: int) -> np.ndarray:
    """Uniform doubles in [0, 1) keyed by (seed, counter, draw); 53 random bits each."""
    key = (_U64(seed) << _U64(40)) | (counter.astype(np.uint64) << _U64(1)) | _U64(draw & 1)
    return (splitmix64(key) >> _U64(11)).astype(np.float64) * _MASK53


def gaussian_field(n: int, seed: int, chunk: int = 1 << 22) -> np.ndarray:
    """i.i.d. standard-normal real and imaginary parts on an N^3 lattice (complex128).

    Element ``e = 2*site + c`` (c = 0 real, 1 imaginary) uses
    ``g = sqrt(-2 ln(1-u1)) * cos(2 pi u2)`` with u1, u2 = uniform01(seed, e, 0/1).
    """
    total = 2 * n * n * n
    if total >= (1 << 39):
        raise ValueError("lattice too large for the 39-bit element counter")
    out = np.empty(total, dtype=np.float64)
    for s in range(0, total, chunk):
        e = np.arange(s, min(total, s + chunk), dtype=np.uint64)
        u1 = uniform01(seed, e, 0)
        u2 = uniform01(seed, e, 1)
        out[s:s + e.size] = np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * np.pi * u2)
    return out.view(np.complex128).reshape(n, n, n)


def zero_dirichlet_planes(psi: np.ndarray) -> np.ndarray:
    """Copy of ``psi`` with the planes ix=0, iy=0, iz=0 set to zero (FDTD inputs)."""
    out = np.array(psi, copy=True)
    out[0, :, :] = 0
    out[:, 0, :] = 0
    out[:, :, 0] = 0
    return out


def axis_coords(n: int, a: float) -> np.ndarray:
    """Coordinates x_i = (i - N/2) a of the sites on one axis."""
    return (np.arange(n, dtype=np.float64) - n // 2) * a


def radius(n: int, a: float) -> np.ndarray:
    """|r| at every site, shape (N, N, N), origin at site (N/2, N/2, N/2)."""
    x = axis_coords(n, a)
    return np.sqrt(x[:, None, None] ** 2 + x[None, :, None] ** 2 + x[None, None, :] ** 2)


def harmonic(n: int, a: float, m: float = 1.0, omega: float = 1.0) -> np.ndarray:
    """Isotropic oscillator V = m omega^2 r^2 / 2 (real)."""
    return 0.5 * m * omega * omega * radius(n, a) ** 2


def cornell(n: int, a: float, kappa: float, sigma: float, c: float = 0.0,
            r0: float | None = None) -> np.ndarray:
    """Cornell V = -kappa/r + sigma r + c with r = 0 replaced by r0 (default a/2)."""
    r = radius(n, a)
    r = np.where(r == 0.0, a / 2 if r0 is None else r0, r)
    return -kappa / r + sigma * r + c


def gaussian_mix(n: int, a: float, seed: int = 3, n_gauss: int = 32,
                 width=(0.2, 1.0), depth=(-5.0, 0.0), imag_frac: float = 0.05) -> np.ndarray:
    """Complex 'file-style' potential: V_re = sum_g d_g exp(-|r-c_g|^2/(2 w_g^2)),
    V_im = -imag_frac |V_re|.

    Parameters are drawn from ``numpy.random.default_rng(seed)`` in this order:
    centres ``uniform(-L/4, L/4, (n_gauss, 3))`` as (x, y, z), widths
    ``uniform(*width, n_gauss)``, depths ``uniform(*depth, n_gauss)``; L = N a.
    """
    rng = np.random.default_rng(seed)
    L = n * a
    centres = rng.uniform(-L / 4, L / 4, size=(n_gauss, 3))
    widths = rng.uniform(width[0], width[1], size=n_gauss)
    depths = rng.uniform(depth[0], depth[1], size=n_gauss)
    x = axis_coords(n, a)
    vre = np.zeros((n, n, n), dtype=np.float64)
    for (cx, cy, cz), w, d in zip(centres, widths, depths):
        gx = np.exp(-(x - cx) ** 2 / (2 * w * w))
        gy = np.exp(-(x - cy) ** 2 / (2 * w * w))
        gz = np.exp(-(x - cz) ** 2 / (2 * w * w))
        vre += d * (gz[:, None, None] * gy[None, :, None] * gx[None, None, :])
    return vre - 1j * imag_frac * np.abs(vre)


# Kinetic-term identifiers shared by every layer: FDTD 7-point (Eq. HK0), FFT with
# k^2 (Eq. HK1), FFT with 4 sin^2(k/2) (Eq. HK2), relativistic FFT (Eq. HK3).
FDTD, FFT_NAIVE, FFT_SYMANZIK, FFT_REL = 0, 1, 2, 3
KINETIC_NAMES = {FDTD: "fdtd", FFT_NAIVE: "fft_naive", FFT_SYMANZIK: "fft_symanzik", FFT_REL: "fft_rel"}


def workload(name: str, n: int | None = None) -> dict:
    """The paper-shaped synthetic workloads; ``n`` overrides the lattice size.

    Returns a dict with n, a, kinetic, m, dtau (None = default rule), potential
    (a callable of (n, a)), seed, precision.
    """
    w = dict(WORKLOADS[name])
    if n is not None:
        w["n"] = n
    return w


WORKLOADS = {
    # N=32 harmonic oscillator, Dirichlet FDTD, complex128, dtau = a^2/8.
    "ho_fdtd_n32": dict(n=32, a=0.15, kinetic=FDTD, m=1.0, dtau=0.15 ** 2 / 8, seed=0,
                        precision="c128", potential=lambda n, a: harmonic(n, a),
                        tol=1e-8),
    # N=128 Cornell (kappa .52, sigma .18), k^2 FFT kinetic, m = 1.5.
    "cornell_naive_n128": dict(n=128, a=0.1, kinetic=FFT_NAIVE, m=1.5, dtau=None, seed=1,
                               precision="c64",
                               potential=lambda n, a: cornell(n, a, 0.52, 0.18, 0.0),
                               tol=1e-7),
    # N=256 relativistic kinetic, m = 0.3, Coulomb + linear (kappa .4, sigma .2), dtau = a/4.
    "cornell_rel_n256": dict(n=256, a=0.05, kinetic=FFT_REL, m=0.3, dtau=0.05 / 4, seed=2,
                             precision="c64",
                             potential=lambda n, a: cornell(n, a, 0.4, 0.2, 0.0),
                             tol=1e-9),
    # N=512 4 sin^2 FFT kinetic, complex Gaussian-mix potential, m = 1.
    "gaussmix_symanzik_n512": dict(n=512, a=0.04, kinetic=FFT_SYMANZIK, m=1.0, dtau=None,
                                   seed=3, precision="c64",
                                   potential=lambda n, a: gaussian_mix(n, a, seed=3),
                                   tol=1e-7),
}
