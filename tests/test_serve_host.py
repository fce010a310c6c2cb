"""Host-side logic of the serving layer and the bench's byte model (no GPU needed).

* the seeded request mix is reproducible and follows its stated distributions;
* admission footprints come from the library's workspace sizing (a warm start reserves
  the coarse lattice too), and only FFT-term requests with a coarse plan warm-start;
* the roofline byte model of the step kernels matches the counted design.
"""
import math

import numpy as np
import pytest

from paper_2211_10185_gb300 import inputs as I


@pytest.fixture(scope="module")
def lib():
    from paper_2211_10185_gb300 import build, qfdtd

    build.build()
    return qfdtd.load()


def test_served_mix_is_reproducible_and_in_range():
    from paper_2211_10185_gb300.serve import served_mix

    a = served_mix(300, rate=200.0, seed=4)
    b = served_mix(300, rate=200.0, seed=4)
    assert [(r.n, r.kinetic, r.mass, r.arrival) for r in a] == [(r.n, r.kinetic, r.mass, r.arrival) for r in b]
    assert served_mix(300, seed=5)[0].arrival != a[0].arrival
    arr = np.array([r.arrival for r in a])
    assert np.all(np.diff(arr) > 0)
    # Poisson arrivals at 200/s: mean gap 5 ms (loose bound for 300 draws)
    assert 0.0035 < np.diff(arr).mean() < 0.0065
    assert {r.n for r in a} <= {32, 48, 64, 96, 128, 192, 256}
    assert {r.kinetic for r in a} == {0, 1, 2, 3}
    for r in a:
        assert 0.3 <= r.kappa <= 0.6 and 0.1 <= r.sigma <= 0.25 and 0.3 <= r.mass <= 5.0
        assert math.isclose(r.a * r.n, 16.0)


def test_footprints_follow_workspace_sizing(lib):
    from paper_2211_10185_gb300.serve import Request

    fft = Request(rid=0, arrival=0.0, n=128, a=0.125, kinetic=I.FFT_REL, mass=1.0, kappa=0.4, sigma=0.2, seed=1)
    warm = Request(rid=1, arrival=0.0, n=128, a=0.125, kinetic=I.FFT_REL, mass=1.0, kappa=0.4, sigma=0.2, seed=1,
                   warm_start=True)
    fdtd = Request(rid=2, arrival=0.0, n=128, a=0.125, kinetic=I.FDTD, mass=1.0, kappa=0.4, sigma=0.2, seed=1,
                   warm_start=True)
    assert not fft.coarse() and warm.coarse() and not fdtd.coarse()
    assert fft.footprint() == fft.workspace_bytes()
    assert warm.footprint() == warm.workspace_bytes() + warm.workspace_bytes(64, 0.25)
    assert fdtd.footprint() == fdtd.workspace_bytes()
    # a field of complex FP32 is 8 N^3 bytes; the workspace holds 9 of them plus tables
    assert 9 * 8 * 128 ** 3 <= fft.workspace_bytes() < 9 * 8 * 128 ** 3 + (64 << 20)
    # no plan for N/2 = 5: no warm start
    odd = Request(rid=3, arrival=0.0, n=10, a=1.6, kinetic=I.FFT_NAIVE, mass=1.0, kappa=0.4, sigma=0.2, seed=1,
                  warm_start=True)
    assert not odd.coarse()


def test_roofline_byte_model():
    import bench

    for prec, c in (("c64", 8), ("c128", 16)):
        for v_real in (True, False):
            vb = c // 2 if v_real else c
            assert bench.design_bytes_per_site("fft_y_fwd", prec, v_real) == 2 * c
            assert bench.design_bytes_per_site("fft_x_inv_update", prec, v_real) == 4 * c + vb
            assert bench.design_bytes_per_site("fft2_yz_mid_T", prec, v_real) == 2 * c
            # two-pass steady state: 16 + 36 B per site (real V, c64) instead of 84
            assert bench.design_bytes_per_site("fft2_xy_inv_update", prec, v_real) == 4 * c + vb
            assert bench.design_bytes_per_site("stencil_2step", prec, v_real) == 2 * c + vb
            assert bench.design_bytes_per_site("gs_dots", prec, v_real) is None
    two = bench.design_bytes_per_site("fft2_yz_mid_T", "c64", True) + bench.design_bytes_per_site("fft2_xy_inv_update", "c64", True)
    four = sum(bench.design_bytes_per_site(k, "c64", True) for k in ("fft_y_fwd", "fft_z_mid_T", "fft_y_inv",
                                                                "fft_x_inv_update"))
    assert (two, four) == (52, 84)
    # the floor of a step (read psi and V, write psi'): 20 / 24 B per site-update in complex
    # FP32, 40 / 48 in FP64; a two-step stencil launch carries two updates per site
    assert bench.algorithmic_bytes_per_site_update("c64", True) == 20
    assert bench.algorithmic_bytes_per_site_update("c64", False) == 24
    assert bench.algorithmic_bytes_per_site_update("c128", True) == 40
    assert bench.algorithmic_bytes_per_site_update("c128", False) == 48
    assert bench.UPDATES_PER_LAUNCH.get("stencil_2step") == 2 and bench.UPDATES_PER_LAUNCH.get("fft2_xy_inv_update", 1) == 1
    assert bench.step_kernel("fft2_xy_inv_update") and not bench.step_kernel("fft2_yz_mid_T")


def test_oracle_on_all_cores_uses_the_workloads_default_size():
    # the bench's CPU baseline: one oracle lattice per process, lattice size from the
    # workload when none is given (n=None)
    import bench

    rate, steps, el = bench.oracle_rate_cores("ho_fdtd_n32", None, 0.2, 2, min_steps=2)
    assert steps >= 2 and el > 0
    assert rate == pytest.approx(2 * 32 ** 3 * steps / el)


def test_prepared_request_inputs_equal_the_request_arrays():
    # the server's background preparation (radius cached per lattice size) builds exactly
    # the potential and initial state of Request, on the fine and the warm-start lattices
    from paper_2211_10185_gb300.serve import request_inputs, served_mix

    for r in served_mix(24, sizes=(16, 24, 32), seed=4)[:12]:
        v, psi = request_inputs(r)
        assert np.array_equal(v, r.potential()) and np.array_equal(psi, r.initial_state())
        v2, psi2 = request_inputs(r, r.n // 2, 2 * r.a)
        assert np.array_equal(v2, r.potential(r.n // 2, 2 * r.a))
        assert np.array_equal(psi2, r.initial_state(r.n // 2, 2 * r.a))
