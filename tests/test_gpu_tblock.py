"""Two FDTD steps per pass (temporal blocking) against single steps and the oracle.

The blocked kernel computes every site of both steps with the same rounded operations as
the single-step kernel, so fields, energies and snapshots must agree bitwise with the
same solve run one step per pass; against the FP64 oracle the usual complex-FP32
tolerance applies.
"""
import math

import numpy as np
import pytest

from oracle import qfdtd_oracle as O
from paper_2211_10185_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2211_10185_gb300 import build

    build.build()


def _lat(n, a, v, psi0, tblock, graphs=True, m=1.1):
    from paper_2211_10185_gb300.lattice import Lattice

    lat = Lattice(n, a, precision="c64")
    lat.set_potential(v)
    lat.set_kinetic(O.FDTD, m)
    lat.set_wavefunction(psi0)
    lat.set_temporal_blocking(tblock)
    lat.use_graphs(graphs)
    return lat


def _inputs(n, a, complex_v, seed):
    v = I.cornell(n, a, 0.45, 0.2)
    if complex_v:
        v = v - 0.07j * np.abs(v)
    return v, I.zero_dirichlet_planes(I.gaussian_field(n, seed))


@pytest.mark.parametrize("graphs", [True, False])
@pytest.mark.parametrize("complex_v", [False, True])
@pytest.mark.parametrize("n", [16, 48, 64])
def test_two_step_pass_matches_single_steps_bitwise(n, complex_v, graphs):
    a = 6.0 / n
    v, psi0 = _inputs(n, a, complex_v, seed=n + complex_v)
    one = _lat(n, a, v, psi0, 1, graphs)
    two = _lat(n, a, v, psi0, 2, graphs)
    r1 = one.step_n(200, tol=0.0, check_every=32, snap_every=32)
    r2 = two.step_n(200, tol=0.0, check_every=32, snap_every=32)
    assert r1 == r2
    assert np.array_equal(one.get_wavefunction(), two.get_wavefunction())
    e1, e2 = one.energies(), two.energies()
    assert e1["e"] == e2["e"] and e1["norm"] == e2["norm"] and e1["step"] == e2["step"]
    for j in range(3):
        assert np.array_equal(one.get_wavefunction(100 + j), two.get_wavefunction(100 + j))
    # fewer launches: 30 of the 31 steps between checks pair up
    assert two.info()["launches"] < one.info()["launches"]
    assert two.info()["temporal_block"] == 2 and two.info()["step"] == 200


@pytest.mark.parametrize("steps", [1, 2, 7, 10])
def test_two_step_pass_without_checks_matches_oracle(steps):
    n, a = 24, 0.25
    v, psi0 = _inputs(n, a, True, seed=5)
    ref = O.Lattice(n, a)
    ref.set_potential(v.real, v.imag)
    ref.set_kinetic(O.FDTD, 1.1)
    ref.set_wavefunction(psi0)
    ref.step_n(steps, check_every=0, snap_every=0)
    gpu = _lat(n, a, v, psi0, 2)
    gpu.step_n(steps, tol=0.0, check_every=0, snap_every=0)
    # the first step runs alone (fresh field), the rest in pairs, an odd last one alone
    got = gpu.get_wavefunction()
    assert np.linalg.norm((got - ref.psi).ravel()) / np.linalg.norm(ref.psi.ravel()) < 2e-6 * (1 + steps)
    # Dirichlet planes stay exactly zero
    assert not got[0].any() and not got[:, 0].any() and not got[:, :, 0].any()
    assert gpu.info()["step"] == steps


def test_snapshots_between_checks_split_pairs():
    n, a = 32, 0.2
    v, psi0 = _inputs(n, a, False, seed=9)
    one = _lat(n, a, v, psi0, 1, graphs=False)
    two = _lat(n, a, v, psi0, 2, graphs=False)
    # snapshots every 5 steps, checks every 12: pairs must not straddle either
    one.step_n(61, tol=0.0, check_every=12, snap_every=5)
    two.step_n(61, tol=0.0, check_every=12, snap_every=5)
    assert np.array_equal(one.get_wavefunction(), two.get_wavefunction())
    for j in range(3):
        assert np.array_equal(one.get_wavefunction(100 + j), two.get_wavefunction(100 + j))
    assert one.energies()["e"] == two.energies()["e"]


def test_invalid_blocking_factor_is_rejected():
    from paper_2211_10185_gb300 import qfdtd as Q

    n, a = 16, 0.3
    v, psi0 = _inputs(n, a, False, seed=1)
    lat = _lat(n, a, v, psi0, 2)
    for k in (0, 3, -1):
        with pytest.raises(Q.QFError):
            lat.set_temporal_blocking(k)
    assert lat.info()["temporal_block"] == 2


def test_two_step_pass_full_size_n256():
    """The launch configuration of the FDTD throughput runs (N=256, complex FP32): bitwise
    against single steps, and against two oracle steps."""
    n, a = 256, 0.05
    v, psi0 = _inputs(n, a, False, seed=2)
    one = _lat(n, a, v, psi0, 1, graphs=False)
    two = _lat(n, a, v, psi0, 2, graphs=False)
    # first step alone (cleans the Dirichlet planes), then one pair
    one.step_n(3, tol=0.0, check_every=0, snap_every=0)
    two.step_n(3, tol=0.0, check_every=0, snap_every=0)
    g2 = two.get_wavefunction()
    assert np.array_equal(one.get_wavefunction(), g2)
    ref = O.Lattice(n, a)
    ref.set_potential(v)
    ref.set_kinetic(O.FDTD, 1.1)
    ref.set_wavefunction(psi0)
    ref.step_n(3, check_every=0, snap_every=0)
    assert np.linalg.norm((g2 - ref.psi).ravel()) / np.linalg.norm(ref.psi.ravel()) < 2e-6 * (1 + math.log2(n))
