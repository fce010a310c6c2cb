"""Continuous batching of many independent imaginary-time solves on one GPU.

``Batch`` binds the ``qf_batch_*`` entry points (grouped launches: every pass of all
resident FP32 lattices of one size is one kernel launch).  ``Server`` is the request
loop: requests arrive over time, are admitted while their device workspace fits the
HBM budget, stay resident in the batch across chunks of steps, and retire when they
converge or hit their step cap, freeing their memory for queued requests.  Latency is
measured from arrival to retirement.
"""
from __future__ import annotations

import ctypes as C
import concurrent.futures as cf
import dataclasses
import functools
import heapq
import math
import time

import numpy as np

from . import inputs as I
from . import qfdtd as Q
from .lattice import Lattice


class Batch:
    def __init__(self, stream=None):
        import torch

        self.lib = Q.load()
        # a stream of its own: CUDA graphs cannot capture the legacy default stream (members
        # hand over on it: qf_batch_add synchronises their streams, qf_batch_step ends
        # synchronised)
        self.stream = stream if stream is not None else torch.cuda.Stream()
        h = C.c_void_p()
        st = self.lib.qf_batch_create(C.c_void_p(self.stream.cuda_stream), C.byref(h))
        if st != Q.QF_OK:
            raise Q.QFError(st, "qf_batch_create")
        self.h = h
        self.members: list[Lattice] = []

    def _check(self, st, where):
        if st != Q.QF_OK:
            raise Q.QFError(st, where, self.lib.qf_batch_last_error(self.h).decode())

    def add(self, lat: Lattice, max_steps: int, tol_abs: float, tol_rel: float = 0.0):
        self._check(self.lib.qf_batch_add(self.h, lat.h, int(max_steps), float(tol_abs), float(tol_rel)),
                    "qf_batch_add")
        self.members.append(lat)

    def remove(self, lat: Lattice):
        self._check(self.lib.qf_batch_remove(self.h, lat.h), "qf_batch_remove")
        self.members.remove(lat)

    def step(self, steps: int, check_every: int = 64, snap_every: int | None = None) -> int:
        nr = C.c_int()
        se = check_every if snap_every is None else snap_every
        self._check(self.lib.qf_batch_step(self.h, int(steps), int(check_every), int(se), C.byref(nr)),
                    "qf_batch_step")
        return nr.value

    def status(self):
        """[(status, steps_done)] of the members in insertion order."""
        n = len(self.members)
        cnt = C.c_int()
        st = (C.c_int * max(1, n))()
        sd = (C.c_int64 * max(1, n))()
        self._check(self.lib.qf_batch_members(self.h, C.byref(cnt), st, sd, n), "qf_batch_members")
        return [(st[i], sd[i]) for i in range(cnt.value)]

    def set_stopping(self, rule: int):
        """Q.QF_STOP_DIFFERENCE or Q.QF_STOP_EXTRAPOLATED for the members' checks."""
        self._check(self.lib.qf_batch_set_stopping(self.h, int(rule)), "qf_batch_set_stopping")

    def use_graphs(self, enable: bool = True):
        self._check(self.lib.qf_batch_use_graphs(self.h, int(bool(enable))), "qf_batch_use_graphs")

    def graph_info(self) -> tuple[int, int]:
        """(graphs captured, graph replays)."""
        c, r = C.c_int64(), C.c_int64()
        self._check(self.lib.qf_batch_graph_info(self.h, C.byref(c), C.byref(r)), "qf_batch_graph_info")
        return c.value, r.value

    def launches(self) -> int:
        x = C.c_int64()
        self._check(self.lib.qf_batch_info(self.h, C.byref(x)), "qf_batch_info")
        return x.value

    def close(self):
        if getattr(self, "h", None):
            self.lib.qf_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


@dataclasses.dataclass
class Request:
    rid: int
    arrival: float          # seconds after the start of the run
    n: int
    a: float
    kinetic: int
    mass: float
    kappa: float
    sigma: float
    seed: int
    precision: str = "c64"
    tol_abs: float = 1e-7
    tol_rel: float = 1e-6
    max_steps: int = 20000
    dtau: float | None = None
    warm_start: bool = False   # solve on N/2 first, then prolong (FFT kinetic terms)

    def potential(self, n: int | None = None, a: float | None = None):
        return I.cornell(n or self.n, a or self.a, self.kappa, self.sigma, 0.0)

    def initial_state(self, n: int | None = None, a: float | None = None):
        """Seeded Gaussian blob with a seeded width (cheap to generate for large N);
        zero on the Dirichlet planes for the FDTD term."""
        n, a = n or self.n, a or self.a
        rng = np.random.default_rng(self.seed)
        w = rng.uniform(0.5, 2.0) / math.sqrt(self.mass)
        r = I.radius(n, a)
        psi = np.exp(-0.5 * (r / w) ** 2).astype(np.complex128)
        if self.kinetic == I.FDTD:
            psi = I.zero_dirichlet_planes(psi)
        return psi

    def coarse(self) -> bool:
        """Whether this request starts on the N/2 lattice (FFT terms, N/2 >= 16 with a plan)."""
        return (self.warm_start and self.kinetic != I.FDTD and self.n % 2 == 0
                and (self.n // 2) in (16, 24, 32, 48, 64, 96, 128, 192, 256))

    def workspace_bytes(self, n: int | None = None, a: float | None = None) -> int:
        lib = Q.load()
        d = Q.qf_lattice_desc(n or self.n, a or self.a,
                              Q.QF_PREC_C64 if self.precision == "c64" else Q.QF_PREC_C128, 3)
        nb = C.c_size_t()
        if lib.qf_workspace_bytes(C.byref(d), C.byref(nb)) != Q.QF_OK:
            raise ValueError("unsupported request")
        return nb.value

    def footprint(self) -> int:
        """Device bytes reserved at admission (both lattices for a warm start)."""
        fine = self.workspace_bytes()
        return fine + (self.workspace_bytes(self.n // 2, 2 * self.a) if self.coarse() else 0)


@functools.lru_cache(maxsize=16)
def _radius(n: int, a: float) -> np.ndarray:
    r = I.radius(n, a)
    r.setflags(write=False)
    return r


def request_inputs(req: "Request", n: int | None = None, a: float | None = None):
    """(potential, initial state) of a request on its lattice (or the N/2 lattice of a warm
    start): the same arrays as Request.potential / initial_state, with |r| computed once
    per lattice size."""
    n, a = n or req.n, a or req.a
    r = _radius(n, a)
    rr = np.where(r == 0.0, a / 2, r)
    v = -req.kappa / rr + req.sigma * rr + 0.0
    rng = np.random.default_rng(req.seed)
    w = rng.uniform(0.5, 2.0) / math.sqrt(req.mass)
    psi = np.exp(-0.5 * (r / w) ** 2).astype(np.complex128)
    if req.kinetic == I.FDTD:
        psi = I.zero_dirichlet_planes(psi)
    return v, psi


@dataclasses.dataclass
class Result:
    rid: int
    status: int
    steps: int
    energy: complex
    de: float
    arrival: float
    admitted: float
    finished: float
    coarse_steps: int = 0

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


def served_mix(count: int, rate: float = 200.0, sizes=(32, 48, 64, 96, 128, 192, 256), seed: int = 4,
               max_steps: int = 20000, box: float = 16.0, kinetics=(0, 1, 2, 3)) -> list[Request]:
    """Poisson arrivals (rate per second) of Cornell solves: N uniform over ``sizes``,
    kinetic term uniform over ``kinetics``, kappa ~ U[.3, .6], sigma ~ U[.1, .25],
    m ~ U[.3, 5], a = box / N, default dtau, tol = 1e-7 + 1e-6 |E| on the distance left
    to the converged energy (the batch's extrapolated stopping rule).  Drawn from
    numpy.random.default_rng(seed) in that order per request."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for rid in range(count):
        t += rng.exponential(1.0 / rate)
        n = int(rng.choice(sizes))
        kin = int(rng.choice(kinetics))
        kappa = float(rng.uniform(0.3, 0.6))
        sigma = float(rng.uniform(0.1, 0.25))
        m = float(rng.uniform(0.3, 5.0))
        out.append(Request(rid=rid, arrival=t, n=n, a=box / n, kinetic=kin, mass=m, kappa=kappa, sigma=sigma,
                           seed=1000 + rid, max_steps=max_steps))
    return out


class Server:
    """Admits requests by device-workspace footprint into one batch and advances the
    batch in chunks of ``chunk`` steps; finished solves free their memory at once.  A
    solve stops when the distance left to its converged energy, extrapolated from the
    last two check differences, is below its tolerance (QF_STOP_EXTRAPOLATED)."""

    def __init__(self, hbm_budget_bytes: int, chunk: int = 64, stream=None,
                 stopping: int = Q.QF_STOP_EXTRAPOLATED, prep_threads: int = 8,
                 prep_bytes: int = 8 << 30):
        self.budget = int(hbm_budget_bytes)
        self.chunk = int(chunk)
        self.batch = Batch(stream)
        self.batch.set_stopping(stopping)
        # host-side preparation of queued requests' inputs (potential, initial state) on a
        # thread pool while the GPU steps the batch; at most prep_bytes of them in flight
        self.prep = cf.ThreadPoolExecutor(max_workers=prep_threads)
        self.prep_bytes = int(prep_bytes)
        self.prepared: dict[tuple, cf.Future] = {}
        self.prep_in_flight = 0
        self.queue: list[Request] = []
        self.active: dict[int, tuple[Request, Lattice, float]] = {}
        self.in_use = 0
        self.peak_in_use = 0
        self.results: list[Result] = []
        self.chunks = 0

    def _prepare(self):
        """Starts host-side input generation for queued requests, in queue order, while
        the bytes in preparation stay under prep_bytes."""
        for req in self.queue:
            n, a = (req.n // 2, 2 * req.a) if req.coarse() else (req.n, req.a)
            key = (req.rid, n)
            if key in self.prepared:
                continue
            size = 24 * n ** 3
            if self.prep_in_flight + size > self.prep_bytes and self.prepared:
                break
            self.prepared[key] = self.prep.submit(request_inputs, req, n, a)
            self.prep_in_flight += size

    def _inputs(self, req: Request, n: int, a: float):
        key = (req.rid, n)
        fut = self.prepared.pop(key, None)
        if fut is None:
            return request_inputs(req, n, a)
        self.prep_in_flight -= 24 * n ** 3
        return fut.result()

    def _admit(self, now: float):
        kept = []
        for req in self.queue:
            need = req.footprint()
            if self.in_use + need > self.budget:
                kept.append(req)
                continue
            if req.coarse():
                n, a = req.n // 2, 2 * req.a
                v, psi = self._inputs(req, n, a)
                lat = Lattice(n, a, precision=req.precision, stream=self.batch.stream)
                lat.set_potential(v)
                lat.set_kinetic(req.kinetic, req.mass, req.dtau)
                lat.set_wavefunction(psi)
                self.batch.add(lat, req.max_steps, 10 * req.tol_abs, 10 * req.tol_rel)
                self.active[req.rid] = (req, lat, now, "coarse", 0)
            else:
                v, psi = self._inputs(req, req.n, req.a)
                lat = Lattice(req.n, req.a, precision=req.precision, stream=self.batch.stream)
                lat.set_potential(v)
                lat.set_kinetic(req.kinetic, req.mass, req.dtau)
                lat.set_wavefunction(psi)
                self.batch.add(lat, req.max_steps, req.tol_abs, req.tol_rel)
                self.active[req.rid] = (req, lat, now, "fine", 0)
            self.in_use += need
            self.peak_in_use = max(self.peak_in_use, self.in_use)
        self.queue = kept

    def _fine(self, req: Request) -> Lattice:
        lat = Lattice(req.n, req.a, precision=req.precision, stream=self.batch.stream)
        lat.set_potential(req.potential())
        lat.set_kinetic(req.kinetic, req.mass, req.dtau)
        return lat

    def _retire(self, now: float):
        status = self.batch.status()
        done = [(lat, st, steps) for lat, (st, steps) in zip(list(self.batch.members), status)
                if st != Q.QF_BATCH_RUNNING]
        for lat, st, steps in done:
            rid = next(r for r, v in self.active.items() if v[1] is lat)
            req, _, admitted, phase, coarse_steps = self.active.pop(rid)
            self.batch.remove(lat)
            if phase == "coarse":
                # warm start: prolong the coarse solution onto the requested lattice
                fine = self._fine(req)
                fine.prolong_from(lat)
                lat.close()
                self.batch.add(fine, req.max_steps, req.tol_abs, req.tol_rel)
                self.active[rid] = (req, fine, admitted, "fine", steps)
                self.in_use -= req.footprint() - req.workspace_bytes()
                continue
            e = lat.energies()
            self.results.append(Result(rid, st, steps, e["e"], e["de"], req.arrival, admitted, now, coarse_steps))
            self.in_use -= req.workspace_bytes()
            lat.close()

    def run(self, requests: list[Request], realtime: bool = True) -> list[Result]:
        """Serves ``requests`` (sorted by arrival).  realtime: a request joins the queue
        once the wall clock passes its arrival time; otherwise all arrive at once."""
        pending = sorted(requests, key=lambda r: r.arrival)
        t0 = time.perf_counter()
        i = 0
        while i < len(pending) or self.queue or self.active:
            now = time.perf_counter() - t0
            while i < len(pending) and (not realtime or pending[i].arrival <= now):
                self.queue.append(pending[i])
                i += 1
            self._prepare()
            self._admit(now)
            if not self.active:
                if i < len(pending) and realtime:
                    time.sleep(max(0.0, min(0.01, pending[i].arrival - now)))
                continue
            self.batch.step(self.chunk, check_every=self.chunk)
            self.chunks += 1
            self._retire(time.perf_counter() - t0)
        self.elapsed = time.perf_counter() - t0
        self.prep.shutdown(wait=True)
        return self.results

    def metrics(self) -> dict:
        lat = sorted(r.latency for r in self.results)
        if not lat:
            return {}
        pick = lambda q: lat[min(len(lat) - 1, int(math.ceil(q * len(lat))) - 1)]  # noqa: E731
        return {"solves": len(lat), "solves_per_s": len(lat) / self.elapsed, "p50_s": pick(0.50),
                "p99_s": pick(0.99), "converged": sum(r.status == Q.QF_OK for r in self.results),
                "capped": sum(r.status == Q.QF_ENOTCONV for r in self.results),
                "peak_workspace_bytes": self.peak_in_use, "launches": self.batch.launches(),
                "elapsed_s": self.elapsed, "chunks": self.chunks}
