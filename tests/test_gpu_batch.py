"""Batches and the serving loop: each result is the same alone and in the mix.

A batch member runs the same kernels, blocks and reduction order as the lattice alone,
so fields and energies must agree bitwise; the server must retire every request within
its HBM budget with results equal to serving that request by itself.
"""
import numpy as np
import pytest

from paper_2211_10185_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2211_10185_gb300 import build

    build.build()


SPECS = [  # n, kinetic, precision, complex V
    (16, I.FFT_NAIVE, "c64", False),
    (16, I.FFT_REL, "c64", False),
    (24, I.FFT_SYMANZIK, "c64", True),
    (16, I.FFT_SYMANZIK, "c64", False),
    (32, I.FDTD, "c64", False),
    (24, I.FDTD, "c64", True),
    (16, I.FFT_NAIVE, "c128", False),
    (16, I.FDTD, "c128", False),
]


def _make(spec, seed):
    from paper_2211_10185_gb300.lattice import Lattice

    n, kind, prec, cplx = spec
    a = 6.0 / n
    v = I.cornell(n, a, 0.45, 0.2)
    if cplx:
        v = v - 0.05j * np.abs(v)
    psi = I.gaussian_field(n, seed)
    if kind == I.FDTD:
        psi = I.zero_dirichlet_planes(psi)
    lat = Lattice(n, a, precision=prec)
    lat.set_potential(v)
    lat.set_kinetic(kind, 1.0 + 0.1 * seed)
    lat.set_wavefunction(psi)
    return lat


def test_batch_members_match_step_n_bitwise():
    from paper_2211_10185_gb300.serve import Batch
    from paper_2211_10185_gb300 import qfdtd as Q

    alone = [_make(s, i) for i, s in enumerate(SPECS)]
    mixed = [_make(s, i) for i, s in enumerate(SPECS)]
    cap, tol = 700, 1e-6
    res_alone = [lat.step_n(cap, tol=tol, check_every=32, snap_every=32) for lat in alone]
    b = Batch()
    for lat in mixed:
        b.add(lat, cap, tol, 0.0)
    while b.step(96, check_every=32) > 0:
        pass
    st = b.status()
    for i, (lat_a, lat_m) in enumerate(zip(alone, mixed)):
        (s_a, d_a), (s_m, d_m) = res_alone[i], st[i]
        assert s_a == s_m and d_a == d_m, (i, res_alone[i], st[i])
        assert np.array_equal(lat_a.get_wavefunction(), lat_m.get_wavefunction()), i
        ea, em = lat_a.energies(), lat_m.energies()
        assert ea["e"] == em["e"] and ea["step"] == em["step"], i
        # snapshots and excited states agree too
        assert np.array_equal(lat_a.get_wavefunction(100), lat_m.get_wavefunction(100))
    # every member stopped by its own rule, and the fast-converging ones (dtau ~ 0.03-0.08,
    # tau up to 20-56 within the cap) did converge
    assert all(s in (Q.QF_OK, Q.QF_ENOTCONV) for s, _ in st)
    assert any(s == Q.QF_OK for s, _ in st)
    assert b.launches() > 0


def test_members_do_not_depend_on_the_mix():
    from paper_2211_10185_gb300.serve import Batch

    cap, tol = 300, 0.0
    solo = _make(SPECS[1], 1)
    b1 = Batch()
    b1.add(solo, cap, tol)
    b1.step(cap, check_every=64)
    others = [_make(s, 10 + i) for i, s in enumerate(SPECS)]
    mixed = _make(SPECS[1], 1)
    b2 = Batch()
    for i, lat in enumerate(others):
        b2.add(lat, 50 + 40 * i, tol)          # members leave at different times
        if i == 3:
            b2.add(mixed, cap, tol)
    b2.step(cap, check_every=64)
    assert np.array_equal(solo.get_wavefunction(), mixed.get_wavefunction())


def test_server_retires_all_requests_within_budget_and_matches_alone():
    from paper_2211_10185_gb300 import qfdtd as Q
    from paper_2211_10185_gb300.serve import Server, served_mix

    reqs = served_mix(14, rate=1000.0, sizes=(16, 24, 32), seed=4, max_steps=640)
    budget = 3 * max(r.workspace_bytes() for r in reqs)
    srv = Server(budget, chunk=64)
    res = srv.run(reqs, realtime=False)
    m = srv.metrics()
    assert len(res) == len(reqs) and m["solves"] == len(reqs)
    assert srv.peak_in_use <= budget
    assert m["p50_s"] <= m["p99_s"]
    by_id = {r.rid: r for r in res}
    for req in reqs[:5]:
        one = Server(budget, chunk=64)
        (r1,) = one.run([req], realtime=False)
        r2 = by_id[req.rid]
        assert r1.status == r2.status and r1.steps == r2.steps
        assert r1.energy == r2.energy
        assert r1.status in (Q.QF_OK, Q.QF_ENOTCONV)


def test_warm_start_converges_to_the_same_state_in_fewer_fine_steps():
    import dataclasses

    from paper_2211_10185_gb300 import qfdtd as Q
    from paper_2211_10185_gb300.serve import Server, served_mix

    reqs = [r for r in served_mix(40, rate=1000.0, sizes=(48, 64), seed=5, max_steps=6000, kinetics=(1, 2, 3))][:4]
    budget = 8 * max(r.footprint() for r in reqs)
    cold = Server(budget, chunk=64).run(reqs, realtime=False)
    warm_reqs = [dataclasses.replace(r, warm_start=True) for r in reqs]
    srv = Server(budget, chunk=64)
    warm = srv.run(warm_reqs, realtime=False)
    assert srv.peak_in_use <= budget
    c = {r.rid: r for r in cold}
    for r in warm:
        assert r.coarse_steps > 0
        if r.status == Q.QF_OK and c[r.rid].status == Q.QF_OK:
            # the same ground state (tolerance-level agreement), reached in fewer fine steps
            assert abs(r.energy - c[r.rid].energy) < 1e-5 * max(1.0, abs(c[r.rid].energy))
            assert r.steps <= c[r.rid].steps


def _oracle_solve(req):
    """The request solved alone by the FP64 oracle with the served stopping rule."""
    from oracle import qfdtd_oracle as O

    lat = O.Lattice(req.n, req.a)
    lat.set_potential(req.potential())
    lat.set_kinetic(req.kinetic, req.mass, req.dtau)
    lat.set_wavefunction(req.initial_state())
    st, done = lat.step_n(req.max_steps, tol=req.tol_abs, tol_rel=req.tol_rel, check_every=64, rule="extrapolated")
    return st, done, lat.energies()["e"]


def test_served_energies_match_the_oracle_within_1e5():
    """A served mix of small requests (every kinetic term), FP32 lattices batched under
    continuous admission: each converged energy is within 1e-5 relative of the FP64
    oracle solving the same request alone with the same stopping rule."""
    import multiprocessing as mp

    from paper_2211_10185_gb300 import qfdtd as Q
    from paper_2211_10185_gb300.serve import Server, served_mix

    reqs = served_mix(40, rate=1000.0, sizes=(16, 24, 32), seed=11, max_steps=12000)
    kinds_seen = set()
    sub = []
    for r in reqs:
        if len([x for x in sub if x.kinetic == r.kinetic]) < 2:
            sub.append(r)
            kinds_seen.add(r.kinetic)
    assert kinds_seen == {0, 1, 2, 3}
    srv = Server(4 * max(r.workspace_bytes() for r in sub), chunk=64)
    res = {r.rid: r for r in srv.run(sub, realtime=False)}
    with mp.get_context("spawn").Pool(min(len(sub), 8)) as pool:
        ora = pool.map(_oracle_solve, sub)
    checked = 0
    for req, (st, done, e) in zip(sub, ora):
        got = res[req.rid]
        if st != 0 or got.status != Q.QF_OK:
            continue
        checked += 1
        assert abs(got.energy - e) < 1e-5 * abs(e), (req, got.energy, e)
    assert checked >= 6


def test_fdtd_members_of_different_sizes_share_one_launch_per_step():
    """FDTD lattices of N = 16, 24, 40 and 48 (real and complex V) taking one step per
    pass advance in a single stencil launch per step, and each ends bitwise where it
    ends alone."""
    from paper_2211_10185_gb300.serve import Batch

    specs = [(16, I.FDTD, "c64", False), (24, I.FDTD, "c64", True), (40, I.FDTD, "c64", False),
             (48, I.FDTD, "c64", True)]
    alone = [_make(s, 30 + i) for i, s in enumerate(specs)]
    mixed = [_make(s, 30 + i) for i, s in enumerate(specs)]
    for lat in alone + mixed:
        lat.set_temporal_blocking(1)   # one step per launch
    for lat in alone:
        lat.step_n(37, tol=0.0, check_every=0, snap_every=0)
    b = Batch()
    for lat in mixed:
        b.add(lat, 1000, 0.0)
    b.step(37, check_every=0, snap_every=0)
    assert b.launches() == 37
    for la, lm in zip(alone, mixed):
        assert np.array_equal(la.get_wavefunction(), lm.get_wavefunction())


def test_fdtd_members_pair_their_steps_like_a_lone_lattice():
    """With two FDTD steps per pass (the default) batch members of different sizes take
    their steps in pairs, all members with real V in one launch per pair: after the
    first step (the input field is not yet known to vanish on the Dirichlet planes),
    36 steps in 18 launches.  Fields equal those of each lattice alone bitwise (a pair
    computes what two single steps do)."""
    from paper_2211_10185_gb300.serve import Batch

    specs = [(16, I.FDTD, "c64", False), (24, I.FDTD, "c64", False), (40, I.FDTD, "c64", False),
             (48, I.FDTD, "c64", False)]
    alone = [_make(s, 40 + i) for i, s in enumerate(specs)]
    mixed = [_make(s, 40 + i) for i, s in enumerate(specs)]
    for lat in alone:
        lat.step_n(37, tol=0.0, check_every=0, snap_every=0)
    b = Batch()
    for lat in mixed:
        b.add(lat, 1000, 0.0)
    b.step(37, check_every=0, snap_every=0)
    assert b.launches() == 1 + 18
    for la, lm in zip(alone, mixed):
        assert la.info()["step"] == lm.info()["step"] == 37
        assert np.array_equal(la.get_wavefunction(), lm.get_wavefunction())


@pytest.mark.parametrize("graphs", [True, False])
def test_fdtd_pairs_with_checks_snapshots_and_fft_members(graphs):
    """A batch of FDTD members (real and complex V, two sizes) and an FFT member stepped
    in check intervals with snapshots: FDTD steps pair inside each interval (in the
    captured graph or launch by launch), and every member's field, energy and snapshots
    equal those of the lattice stepped alone."""
    from paper_2211_10185_gb300.serve import Batch

    specs = [(24, I.FDTD, "c64", False), (32, I.FDTD, "c64", True), (16, I.FFT_REL, "c64", False),
             (16, I.FDTD, "c64", False)]
    alone = [_make(s, 60 + i) for i, s in enumerate(specs)]
    mixed = [_make(s, 60 + i) for i, s in enumerate(specs)]
    for lat in alone:
        lat.step_n(80, tol=0.0, check_every=16, snap_every=16)
    b = Batch()
    b.use_graphs(graphs)
    for lat in mixed:
        b.add(lat, 100000, 0.0)
    for _ in range(5):
        b.step(16, check_every=16, snap_every=16)
    if graphs:
        assert b.graph_info()[1] >= 3
    for la, lm in zip(alone, mixed):
        assert la.info()["step"] == lm.info()["step"] == 80
        assert np.array_equal(la.get_wavefunction(), lm.get_wavefunction())
        assert la.energies() == lm.energies()
        assert la.info()["n_snapshots"] == lm.info()["n_snapshots"] == 3
        for k in range(3):
            assert np.array_equal(la.get_wavefunction(100 + k), lm.get_wavefunction(100 + k))


def test_batch_graph_replay_is_bitwise_identical_to_launches():
    """A fixed batch (FFT members of two sizes, FDTD members of two sizes, an FP64
    member) stepped in check intervals: the intervals after the first check replay one
    captured graph, and every field, energy and snapshot equals the ordinary launches'."""
    from paper_2211_10185_gb300.serve import Batch

    specs = [(16, I.FFT_REL, "c64", False), (24, I.FFT_SYMANZIK, "c64", True), (32, I.FFT_NAIVE, "c64", False),
             (24, I.FDTD, "c64", False), (32, I.FDTD, "c64", True), (16, I.FFT_NAIVE, "c128", False)]
    runs = []
    for graphs in (True, False):
        lats = [_make(s, 50 + i) for i, s in enumerate(specs)]
        b = Batch()
        b.use_graphs(graphs)
        for lat in lats:
            b.add(lat, 100000, 0.0)
        for _ in range(5):
            b.step(32, check_every=32)
        runs.append((b, lats))
    (bg, lg), (bn, ln) = runs
    captures, replays = bg.graph_info()
    # graphs are keyed by the FDTD members' buffer parity and pairing: the first interval
    # (step scale 2^k != 1, single steps) and then two alternating parities (a paired
    # interval makes an odd number of buffer swaps)
    assert captures <= 3 and replays == 5
    assert bn.graph_info() == (0, 0)
    assert bg.launches() == bn.launches()
    for a, c in zip(lg, ln):
        assert np.array_equal(a.get_wavefunction(), c.get_wavefunction())
        assert a.energies() == c.energies()
        assert np.array_equal(a.get_wavefunction(100), c.get_wavefunction(100))
        assert a.info()["step"] == c.info()["step"] == 160
