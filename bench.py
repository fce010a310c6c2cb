"""Benchmark of the imaginary-time step on one GB300 (or N replicas under torchrun).

One bench step = one check interval of a solve: 64 imaginary-time steps of the fused
FFT kinetic step (forward FFT, T(k) multiply, inverse FFT, coef_A/coef_B update), the
FP64 norm/energy reduction and renormalisation of the check, the snapshot, then the
Gram-Schmidt extraction of the ground and two excited states from the three latest
snapshots (with their FP64 energies) and a parity projection of the first excited
state.  Metric: site-updates/s = N^3 * 64 per bench step / time.

Default workload: N = 256^3, a = 0.05, relativistic kinetic term (Eq. HK3) with m = 0.3,
Coulomb + linear potential (kappa 0.4, sigma 0.2), dtau = a/4, complex FP32 fields with
FP64 reductions.  Each field is 134 MB (> 126 MB L2) and a step streams three of them,
so no L2 flush is needed between timed steps.

``--impl reference`` times the FP64 CPU oracle (oracle/) on the host cores instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2211_10185_gb300 import inputs as I  # noqa: E402

CHUNK = 64
METRIC = "site-updates/s (fused FFT step, N=256)"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
# per-launch DRAM traffic of one ncu capture per kernel family, with the digest of the
# sources that family compiles from
TRAFFIC_FILES = {
    "fft": (os.path.join(ROOT, "profiles", "ncu_traffic_fft_step_n256.json"),
            ("qf_fft_impl.cuh", "qf_common.cuh", "qf_fft2.cuh")),
    "stencil": (os.path.join(ROOT, "profiles", "ncu_traffic_fdtd_step_n256.json"),
                ("qf_stencil.cu", "qf_stencil_tma.cuh", "qf_stencil_tb.cuh", "qf_common.cuh")),
}
FALLBACK_HBM_GBS = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="cornell_rel_n256")
    ap.add_argument("--n", type=int, default=None, help="override the lattice size")
    ap.add_argument("--precision", default=None, choices=[None, "c64", "c128"])
    ap.add_argument("--tblock", type=int, default=2, choices=[1, 2],
                    help="FDTD steps per pass over HBM (complex FP32)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-comparator", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="CPU baseline sample budget")
    ap.add_argument("--no-served", action="store_true")
    ap.add_argument("--served-requests", type=int, default=96)
    ap.add_argument("--served-cap", type=int, default=3000)
    ap.add_argument("--config4", action="store_true",
                    help="also time 200 steps of the N=512 Gaussian-mix workload (Eq. HK2, complex V); "
                         "its host inputs take about a minute to generate")
    ap.add_argument("--served-full", action="store_true",
                    help="only the served mix, at its stated size: 2000 Poisson requests (200/s), "
                         "N in {32..256}, cap 20000 steps, 170 GB; prints one JSON line")
    ap.add_argument("--fft-variants", action="store_true",
                    help="only the four-pass FFT step's tile and radix-plan variants (the autotuner's "
                         "choices), timed per size; prints one JSON line")
    return ap.parse_args()


def max_over_ranks(value: float) -> float:
    """Maximum of a per-rank float over all ranks (NCCL on GPUs, gloo on CPU); the
    value itself when not distributed."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return value
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(units_per_rank: float, world: int, seconds_max: float) -> float:
    """Whole-job rate: every rank processed units_per_rank; the job took the slowest
    rank's time (replicas, weak scaling)."""
    return world * units_per_rank / seconds_max


def workload_config(w, prec):
    kin = I.KINETIC_NAMES[w["kinetic"]]
    return {
        "workload": (f"N={w['n']}^3 a={w['a']} kinetic={kin} m={w['m']} "
                     f"dtau={'a/4' if w['dtau'] else 'default'} seed={w['seed']} {prec}"),
        "n": w["n"], "a": w["a"], "kinetic": kin, "mass": w["m"], "precision": prec,
        "chunk_steps": CHUNK, "check_every": CHUNK, "snap_every": CHUNK,
        "per_step": "64 steps + check + snapshot + 3-state Gram-Schmidt + energies (plateau record) + parity",
        "l2": "no flush: inputs larger than L2 (3 fields of 8 N^3 bytes per step)",
    }


def make_inputs(w):
    n = w["n"]
    v = w["potential"](n, w["a"])
    psi0 = I.gaussian_field(n, w["seed"])
    if w["kinetic"] == I.FDTD:
        psi0 = I.zero_dirichlet_planes(psi0)
    return v, psi0


# ---------------------------------------------------------------------------------------
# CPU oracle timing (reference arm and cpu_baseline)
# ---------------------------------------------------------------------------------------
def oracle_rate(w, v, psi0, seconds, min_steps=2):
    """Times the FP64 oracle (as it stands) on imaginary-time steps of the same workload
    for about ``seconds``; returns (site-updates/s, steps timed, seconds)."""
    from oracle import qfdtd_oracle as O

    n = w["n"]
    lat = O.Lattice(n, w["a"])
    if np.iscomplexobj(v):
        lat.set_potential(v.real, v.imag)
    else:
        lat.set_potential(v)
    lat.set_kinetic(w["kinetic"], w["m"], w["dtau"])
    lat.set_wavefunction(psi0)
    t0 = time.perf_counter()
    steps = 0
    while True:
        lat.step_n(1, check_every=CHUNK)
        steps += 1
        el = time.perf_counter() - t0
        if steps >= min_steps and el >= seconds:
            break
    return n ** 3 * steps / el, steps, el


def size_sweep(name, prec, sizes=(32, 128), gpu_steps=640, cpu_seconds=2.0):
    """The same workload at smaller N: GPU site-updates/s over ``gpu_steps`` imaginary-time
    steps (checks every 64) against the FP64 oracle on one host core for ~``cpu_seconds``."""
    import torch

    from paper_2211_10185_gb300.lattice import Lattice

    res = {}
    for n in sizes:
        w = I.workload(name, n)
        v, psi0 = make_inputs(w)
        lat = Lattice(n, w["a"], precision=prec)
        lat.set_potential(v)
        lat.set_kinetic(w["kinetic"], w["m"], w["dtau"])
        lat.set_wavefunction(psi0)
        lat.step_n(2 * CHUNK, tol=0.0, check_every=CHUNK)  # warm-up (plans, graphs, autotuning)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        lat.step_n(gpu_steps, tol=0.0, check_every=CHUNK)
        torch.cuda.synchronize()
        gpu = n ** 3 * gpu_steps / (time.perf_counter() - t0)
        lat.close()
        cpu, steps, el = oracle_rate(w, v, psi0, cpu_seconds)
        res[str(n)] = {"gpu_site_updates_per_s": gpu, "oracle_site_updates_per_s": cpu, "oracle_steps": steps,
                       "oracle_cores": 1}
    return res


def _oracle_worker(conn, name, n):
    """One host core's oracle lattice of the workload: builds it, then advances it one
    imaginary-time step (a check every 64) per message until it receives None."""
    from oracle import qfdtd_oracle as O

    w = I.workload(name, n)
    v, psi0 = make_inputs(w)
    lat = O.Lattice(w["n"], w["a"])
    if np.iscomplexobj(v):
        lat.set_potential(v.real, v.imag)
    else:
        lat.set_potential(v)
    lat.set_kinetic(w["kinetic"], w["m"], w["dtau"])
    lat.set_wavefunction(psi0)
    conn.send("ready")
    while conn.recv() is not None:
        lat.step_n(1, check_every=CHUNK)
        conn.send("done")


class OracleCores:
    """The FP64 oracle as it stands on ``procs`` host cores: one independent lattice of
    the workload per core (spawned processes; numpy's FFT runs on one thread each), all
    stepped together.  ``step()`` advances every lattice by one imaginary-time step."""

    def __init__(self, name, n, procs):
        import multiprocessing as mp

        ctx = mp.get_context("spawn")
        self.procs, self.conns = [], []
        for _ in range(procs):
            a, b = ctx.Pipe()
            p = ctx.Process(target=_oracle_worker, args=(b, name, n), daemon=True)
            p.start()
            self.procs.append(p)
            self.conns.append(a)
        for c in self.conns:
            c.recv()

    def step(self):
        for c in self.conns:
            c.send(1)
        for c in self.conns:
            c.recv()

    def close(self):
        for c in self.conns:
            c.send(None)
        for p in self.procs:
            p.join(timeout=30)


def oracle_rate_cores(name, n, seconds, procs, min_steps=2):
    """Whole-host oracle throughput: ``procs`` lattices stepped together for about
    ``seconds``; returns (site-updates/s, steps per lattice, seconds)."""
    n_sites = I.workload(name, n)["n"] ** 3
    pool = OracleCores(name, n, procs)
    try:
        pool.step()  # warm-up
        t0 = time.perf_counter()
        steps = 0
        while True:
            pool.step()
            steps += 1
            el = time.perf_counter() - t0
            if steps >= min_steps and el >= seconds:
                break
    finally:
        pool.close()
    return procs * n_sites * steps / el, steps, el


def run_reference(args):
    """The FP64 oracle as it stands, on all host cores (one lattice of the workload per
    core); one bench step = one oracle imaginary-time step of every lattice (a check step
    every 64)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = I.workload(args.workload, args.n)
    n = w["n"]
    cores = os.cpu_count() or 1
    pool = OracleCores(args.workload, args.n, cores)
    try:
        for _ in range(args.warmup):
            pool.step()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            pool.step()
        el = time.perf_counter() - t0
    finally:
        pool.close()
    rate = cores * n ** 3 * args.steps / el
    line = {
        "impl": "reference", "metric": METRIC, "value": rate, "unit": "site-updates/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded SplitMix64/Box-Muller psi0, analytic potential)",
        "config": workload_config(w, "c128 (FP64 oracle)"),
        "cpu_baseline": {"value": rate, "unit": "site-updates/s", "cores": cores, "kind": "oracle",
                         "sample": f"{args.steps} oracle imaginary-time steps of {cores} independent N={n} "
                                   f"lattices, one per host core ({el:.1f} s; numpy FFT, one thread each)"},
        "e2e": {"value": rate, "unit": "site-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------------------
# Clock sampling during the timed region
# ---------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(index)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for row in out.strip().splitlines():
            parts = [p.strip() for p in row.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx = max(mx, float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[3:7]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------------------
# Roofline bookkeeping
# ---------------------------------------------------------------------------------------
def algorithmic_bytes_per_site_update(prec, v_real):
    """The floor of one imaginary-time step: read psi and V, write psi' (8 + 4 + 8 B per
    site for complex FP32 with a real V; V complex: 8 B; FP64 doubles every term)."""
    c = 8 if prec == "c64" else 16
    return 2 * c + ((c // 2) if v_real else c)


# site-updates one launch of a kernel kind carries (per lattice site): the step's kernels
# advance every site by one step, the two-step stencil by two
UPDATES_PER_LAUNCH = {"stencil_2step": 2}


def design_bytes_per_site(kernel, prec, v_real):
    """Bytes a launch of this kernel kind moves per lattice site by its design (every
    field it reads or writes once): the counted traffic of the kernel, not the floor."""
    c = 8 if prec == "c64" else 16
    r = c // 2
    vb = r if v_real else c
    table = {
        "fft_x_fwd": 2 * c, "fft_y_fwd": 2 * c, "fft_z_mid_T": 2 * c, "fft_y_inv": 2 * c,
        # read tmp, psi, V; write psi' and the next step's x transform
        "fft_x_inv_update": 4 * c + vb,
        "stencil_step": 2 * c + vb,
        # two steps per launch: read psi_t and V, write psi_{t+2}
        "stencil_2step": 2 * c + vb,
        # two-pass FFT step (N=256 c64): y/z pass in place; x/y pass reading the scratch
        # field, psi and V, writing psi' and the next step's scratch field
        "fft2_xy_fwd": 2 * c, "fft2_yz_mid_T": 2 * c, "fft2_xy_inv_update": 4 * c + vb,
    }
    return table.get(kernel)


def step_kernel(kernel):
    """Kernel kinds that advance psi by a step (the roofline candidates)."""
    return kernel in ("fft_x_inv_update", "fft2_xy_inv_update", "stencil_step", "stencil_2step")


def source_digest(files):
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_2211_10185_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def load_traffic(kernel, n, prec):
    path, files = TRAFFIC_FILES["stencil" if kernel.startswith("stencil") else "fft"]
    try:
        rec = json.load(open(path))
    except (OSError, ValueError):
        return None, "no committed ncu traffic summary"
    if rec.get("source_digest") != source_digest(files):
        return None, "kernels changed since the ncu capture"
    k = rec.get("kernels", {}).get(kernel)
    if not k or rec.get("n") != n or rec.get("precision") != prec:
        return None, "no capture for this kernel/workload"
    return k["dram_bytes_per_launch"], rec.get("command")


def hbm_peak():
    try:
        p = json.load(open(PEAKS_FILE))
        return float(p["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs, copy burst)"
    except (OSError, ValueError, KeyError):
        return FALLBACK_HBM_GBS, "fallback"


# ---------------------------------------------------------------------------------------
# cuFFT comparator (context only): torch.fft on the same step, c64
# ---------------------------------------------------------------------------------------
def cufft_comparator(w, v, psi0, steps=10):
    import torch

    n, a, m = w["n"], w["a"], w["m"]
    dt = w["dtau"] or 0.0
    k = 2 * np.pi * np.where(np.arange(n) <= n // 2, np.arange(n), np.arange(n) - n) / n
    kh = 4 * np.sin(k / 2) ** 2
    if w["kinetic"] == I.FFT_NAIVE:
        s = k * k
    else:
        s = kh
    S = s[:, None, None] + s[None, :, None] + s[None, None, :]
    if w["kinetic"] == I.FFT_REL:
        T = np.sqrt(S + (a * m) ** 2) / a
    else:
        T = S / (2 * a * a * m)
    dev = torch.device("cuda")
    Tt = torch.tensor(T, dtype=torch.float32, device=dev)
    vt = torch.tensor(np.asarray(v), dtype=torch.complex64, device=dev)
    d = 1 + 0.5 * dt * vt
    B = 1 / d
    A = (2 - d) * B
    psi = torch.tensor(psi0, dtype=torch.complex64, device=dev)

    def one():
        nonlocal psi
        h = torch.fft.ifftn(Tt * torch.fft.fftn(psi))
        psi = A * psi - (B * dt) * h

    for _ in range(3):
        one()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        one()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    return {"impl": "torch.fft (cuFFT) + torch elementwise, c64, precomputed A/B and T",
            "ms_per_step": ms, "site_updates_per_s": n ** 3 / (ms * 1e-3)}


# ---------------------------------------------------------------------------------------
# The complex-FP64 arm of the same bench step, and the FP64 rate it runs against
# ---------------------------------------------------------------------------------------
def c128_arm(w, v, psi0, bench_steps=2):
    """The bench step with complex-FP64 fields (qf precision c128): 64 steps + check +
    snapshot + Gram-Schmidt energies + parity, timed with CUDA events on the lattice's
    stream; returns its rate and energies beside the complex-FP32 ones."""
    import torch

    from paper_2211_10185_gb300 import qfdtd as Q
    from paper_2211_10185_gb300.lattice import Lattice

    n = w["n"]
    lat = Lattice(n, w["a"], precision="c128")
    lat.set_potential(v)
    lat.set_kinetic(w["kinetic"], w["m"], w["dtau"])
    lat.set_wavefunction(psi0)
    lat.step_n(3 * CHUNK, tol=0.0, check_every=CHUNK, snap_every=CHUNK)

    def one():
        lat.step_n(CHUNK, tol=0.0, check_every=CHUNK, snap_every=CHUNK)
        ex = lat.project_excited(3)
        lat.parity_project(Q.QF_P_MINUS_PK, 3, 1)
        return ex

    one()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(lat.stream)
    for _ in range(bench_steps):
        ex = one()
    e1.record(lat.stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / bench_steps
    lat.close()
    return {"precision": "c128", "bench_steps": bench_steps, "ms_per_bench_step": ms,
            "site_updates_per_s": n ** 3 * CHUNK / (ms * 1e-3), "energies": [e["e"].real for e in ex]}


def workload_steps(name, steps=200, warm=64):
    """Plain imaginary-time steps of another workload at its own size (checks every 64,
    CUDA-graph replay between checks), timed with CUDA events on the lattice's stream; with
    the per-kernel breakdown and the dominant step kernel's roofline on the step's floor
    bytes."""
    import torch

    from paper_2211_10185_gb300.lattice import Lattice

    w = I.workload(name)
    n = w["n"]
    v, psi0 = make_inputs(w)
    v_real = not np.iscomplexobj(v)
    prec = w["precision"]
    lat = Lattice(n, w["a"], precision=prec, n_snap=1)
    lat.set_potential(v)
    lat.set_kinetic(w["kinetic"], w["m"], w["dtau"])
    lat.set_wavefunction(psi0)
    lat.step_n(warm, tol=0.0, check_every=CHUNK, snap_every=0)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(lat.stream)
    lat.step_n(steps, tol=0.0, check_every=CHUNK, snap_every=0)
    e1.record(lat.stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    lat.profile(True)
    lat.profile_read(reset=True)
    lat.step_n(CHUNK, tol=0.0, check_every=CHUNK, snap_every=0)
    prof = lat.profile_read(reset=True)
    lat.profile(False)
    peak, _ = hbm_peak()
    alg_site = algorithmic_bytes_per_site_update(prec, v_real)
    dom = max(((k, x) for k, x in prof.items() if step_kernel(k)), key=lambda kv: kv[1][1], default=None)
    roof = None
    if dom:
        k, (cnt, tot) = dom
        avg_s = tot / cnt * 1e-3
        roof = {"kernel": k, "avg_launch_us": avg_s * 1e6, "frac": alg_site * n ** 3 / avg_s / 1e9 / peak,
                "design_frac": design_bytes_per_site(k, prec, v_real) * n ** 3 / avg_s / 1e9 / peak}
    out = {"workload": workload_config(w, prec)["workload"], "steps": steps, "ms_per_step": ms / steps,
           "site_updates_per_s": n ** 3 * steps / (ms * 1e-3),
           "step_frac_of_peak": alg_site * n ** 3 * steps / (ms * 1e-3) / 1e9 / peak,
           "fft_passes": lat.info()["fft_passes"], "roofline": roof,
           "kernels": {k: {"launches": c, "avg_us": 1e3 * t / c} for k, (c, t) in prof.items()}}
    lat.close()
    return out


def fp64_peak(size=4096, reps=3):
    """Dense FP64 rate of this GPU (cuBLAS DGEMM through torch.matmul, best of reps)."""
    import torch

    a = torch.randn(size, size, dtype=torch.float64, device="cuda")
    b = torch.randn(size, size, dtype=torch.float64, device="cuda")
    torch.matmul(a, b)
    torch.cuda.synchronize()
    best = 1e30
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1) * 1e-3)
    return {"tflops": 2 * size ** 3 / best / 1e12, "how": f"torch.matmul float64 {size}^3, best of {reps}"}


# ---------------------------------------------------------------------------------------
# Served mix: Poisson arrivals of Cornell solves, continuous batching
# ---------------------------------------------------------------------------------------
SERVED_SIZES = (32, 48, 64, 96, 128, 192, 256)


def served_benchmark(n_req, cap, sizes=(32, 48, 64, 96, 128), rate=200.0, budget=170e9, n_cmp=8, warm=True):
    """Serves a seeded sample of the mixed workload in real time; then, on a subsample of
    small requests, compares the batched FP32 form with serial per-lattice FP64 solves,
    and on FFT-term requests with N >= 64, cold solves with warm-started ones."""
    import torch

    from paper_2211_10185_gb300 import qfdtd as Q
    from paper_2211_10185_gb300.serve import Server, served_mix

    reqs = served_mix(n_req, rate=rate, sizes=sizes, seed=4, max_steps=cap)
    srv = Server(int(budget), chunk=CHUNK)
    srv.run(reqs, realtime=True)
    torch.cuda.synchronize()
    out = dict(srv.metrics())
    out.update({"requests": n_req, "arrival_rate_per_s": rate, "sizes": list(sizes), "step_cap": cap,
                "tolerance": "extrapolated distance to the converged energy < 1e-7 + 1e-6 |E| (QF_STOP_EXTRAPOLATED)", "hbm_budget_bytes": int(budget), "realtime": True})
    # comparator: the same small requests, all arriving at once, FP32 batched vs FP64 alone
    sub = [r for r in reqs if r.n <= 64][:n_cmp]
    t0 = time.perf_counter()
    srv32 = Server(int(budget), chunk=CHUNK)
    r32 = {r.rid: r for r in srv32.run(sub, realtime=False)}
    torch.cuda.synchronize()
    t32 = time.perf_counter() - t0
    t0 = time.perf_counter()
    r64 = {}
    for req in sub:
        one = Server(int(budget), chunk=CHUNK)
        req64 = dataclasses_replace(req, precision="c128")
        (res,) = one.run([req64], realtime=False)
        r64[req.rid] = res
    torch.cuda.synchronize()
    t64 = time.perf_counter() - t0
    # energies are compared where both solves converged (a solve stopped by the step cap
    # reports an unconverged energy, where the two precisions' trajectories differ).  The
    # stopping tolerance is 1e-7 + 1e-6 |E|, so near E = 0 (kinetic and potential parts of
    # order 1 cancelling) it is absolute: relative errors are reported for |E| >= 0.05 and
    # absolute ones for all.
    conv = [i for i in r64 if r32[i].status == Q.QF_OK and r64[i].status == Q.QF_OK]
    abs_err = {i: abs(r32[i].energy - r64[i].energy) for i in conv}
    rel = [abs_err[i] / abs(r64[i].energy) for i in conv if abs(r64[i].energy) >= 0.05]
    out["fp32_batched_vs_fp64_alone"] = {
        "requests": len(sub), "fp32_batched_solves_per_s": len(sub) / t32, "fp64_alone_solves_per_s": len(sub) / t64,
        "converged_both": len(conv),
        "max_rel_energy_err_fp32_vs_fp64": max(rel) if rel else None,
        "max_abs_energy_err_fp32_vs_fp64": max(abs_err.values()) if abs_err else None,
        "min_abs_energy": min(abs(r64[i].energy) for i in conv) if conv else None,
        "note": "relative error over converged solves with |E| >= 0.05; absolute error over all converged",
        "same_status": all(r32[i].status == r64[i].status for i in r64)}
    if not warm:
        return out
    # warm start across N: FFT-term requests with N >= 64, all arriving at once, solved cold
    # and warm (first on the N/2 lattice of the same box, then prolonged)
    sub = [r for r in reqs if r.kinetic != 0 and r.n >= 64][:n_cmp * 2]
    runs = {}
    for warm in (False, True):
        batch = [dataclasses_replace(r, warm_start=warm) for r in sub]
        t0 = time.perf_counter()
        res = Server(int(budget), chunk=CHUNK).run(batch, realtime=False)
        torch.cuda.synchronize()
        runs[warm] = (time.perf_counter() - t0, {r.rid: r for r in res})
    (tc, cold), (tw, warm) = runs[False], runs[True]
    both = [i for i in cold if cold[i].status == Q.QF_OK and warm[i].status == Q.QF_OK]
    out["warm_start"] = {
        "requests": len(sub), "cold_solves_per_s": len(sub) / tc, "warm_solves_per_s": len(sub) / tw,
        "cold_mean_steps": statistics.mean(r.steps for r in cold.values()) if cold else None,
        "warm_mean_fine_steps": statistics.mean(r.steps for r in warm.values()) if warm else None,
        "warm_mean_coarse_steps": statistics.mean(r.coarse_steps for r in warm.values()) if warm else None,
        "converged_cold": sum(r.status == Q.QF_OK for r in cold.values()),
        "converged_warm": sum(r.status == Q.QF_OK for r in warm.values()),
        "max_rel_energy_diff_converged": (max(abs(warm[i].energy - cold[i].energy) / abs(cold[i].energy)
                                              for i in both) if both else None)}
    return out


def dataclasses_replace(obj, **kw):
    import dataclasses

    return dataclasses.replace(obj, **kw)


# ---------------------------------------------------------------------------------------
# Our arm
# ---------------------------------------------------------------------------------------
def run_ours(args):
    import torch
    import torch.distributed as dist

    from oracle import qfdtd_oracle as O  # noqa: F401  (cpu_baseline only, rank 0)
    from paper_2211_10185_gb300 import build as B
    from paper_2211_10185_gb300 import qfdtd as Q
    from paper_2211_10185_gb300.lattice import Lattice

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    B.build()
    w = I.workload(args.workload, args.n)
    prec = args.precision or w["precision"]
    n = w["n"]
    v, psi0 = make_inputs(w)
    v_real = not np.iscomplexobj(v)

    lat = Lattice(n, w["a"], precision=prec)
    lat.set_potential(v)
    lat.set_kinetic(w["kinetic"], w["m"], w["dtau"])
    lat.set_wavefunction(psi0)
    lat.set_temporal_blocking(args.tblock)

    def bench_step():
        lat.step_n(CHUNK, tol=0.0, check_every=CHUNK, snap_every=CHUNK)
        ex = lat.track_excited(3)
        lat.parity_project(Q.QF_P_MINUS_PK, 3, 1)
        return ex

    # fill the snapshot ring (3 snapshots) before the warm-up
    lat.step_n(3 * CHUNK, tol=0.0, check_every=CHUNK, snap_every=CHUNK)
    for _ in range(max(3, args.warmup)):
        bench_step()
    torch.cuda.synchronize()

    stream = lat.stream

    def timed_region(profile):
        """K bench steps bracketed by a barrier and synchronisation; CUDA events on the
        lattice's stream.  With profile, every kernel is also bracketed by events."""
        if profile:
            lat.profile(True)
            lat.profile_read(reset=True)
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(args.steps):
            ex = bench_step()
        ev1.record(stream)
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1)
        prof = None
        if profile:
            prof = lat.profile_read(reset=True)
            lat.profile(False)
        if world > 1:
            ms = max_over_ranks(ms)
            dist.barrier()
        return ms, prof, ex

    # headline: clean timed region (no per-kernel events), clocks sampled meanwhile
    clocks = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    launches0 = lat.info()["launches"]
    ms_total, _, ex = timed_region(False)
    launches = lat.info()["launches"] - launches0
    clk = clocks.stop() if clocks else None
    # per-kernel breakdown: the same K steps again with every launch bracketed by events
    ms_prof, prof, _ = timed_region(True)

    units_per_rank = n ** 3 * CHUNK * args.steps
    value = aggregate_rate(units_per_rank, world, ms_total * 1e-3)
    ms_per_step = ms_total / args.steps

    # roofline of the dominant kernel: the largest share of the timed device time among the
    # kernels that advance psi.  achieved = algorithmic bytes per launch (the step's floor,
    # read psi and V and write psi', times the site-updates one launch carries) / the
    # launch's average CUDA-event duration; the design bytes (every field the kernel moves)
    # give design_frac beside it.
    peak, peak_src = hbm_peak()
    alg_site = algorithmic_bytes_per_site_update(prec, v_real)
    dom = max(((k, v_) for k, v_ in prof.items() if step_kernel(k)), key=lambda kv: kv[1][1], default=None)
    roof = None
    kernels = {}
    for k, (cnt, tot) in prof.items():
        kernels[k] = {"launches": cnt, "avg_us": 1e3 * tot / cnt, "share": tot / ms_prof}
    if dom:
        k, (cnt, tot) = dom
        avg_s = tot / cnt * 1e-3
        alg = alg_site * UPDATES_PER_LAUNCH.get(k, 1) * n ** 3
        design_b = design_bytes_per_site(k, prec, v_real) * n ** 3
        achieved = alg / avg_s / 1e9
        traffic, tsrc = load_traffic(k, n, prec)
        roof = {"bound": "hbm", "kernel": k, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic, "peak_source": peak_src,
                "algorithmic_bytes_per_launch": alg,
                "algorithmic_bytes_per_site_update": alg_site,
                "design_bytes_per_launch": design_b, "design_frac": design_b / avg_s / 1e9 / peak,
                "dram_frac": (traffic / avg_s / 1e9 / peak) if traffic else None,
                "avg_launch_us": avg_s * 1e6, "traffic_source": tsrc}
    # whole step on the floor bytes
    c = 8 if prec == "c64" else 16
    step_frac = alg_site * units_per_rank / (ms_total * 1e-3) / 1e9 / peak
    # design bytes of a steady-state step: the per-launch bytes of the kernels one step
    # launches (from the live profile: launches per step of each kernel kind)
    steps_timed = CHUNK * args.steps
    design = sum(design_bytes_per_site(k, prec, v_real) * cnt / steps_timed
                 for k, (cnt, _) in prof.items() if design_bytes_per_site(k, prec, v_real))

    out = None
    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": "site-updates/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if prec == "c64" else "f64",
            "data": "synthetic (seeded SplitMix64/Box-Muller psi0, analytic Cornell potential); replicas per GPU",
            "config": dict(workload_config(w, prec), parallelism=f"replicas x{world}",
                           **({"temporal_block": args.tblock} if w["kinetic"] == I.FDTD and prec == "c64" else {})),
            "roofline": roof,
            "kernels": kernels,
            "profiled_region_ms_per_step": ms_prof / args.steps,
            "step_algorithmic_hbm": {"bytes_per_site_update": alg_site,
                                     "frac_of_peak": step_frac,
                                     "design_bytes_per_site_update": design,
                                     "field_passes_per_step": design / c,
                                     "note": "minimum bytes of one step (read psi, V; write psi') / bench-step "
                                             "time; design bytes: the step's kernels (GS and parity passes "
                                             "excluded), averaged over the timed steps"},
            "gpu_launches": launches,
            "clocks": clk,
            "energies_last_step": [e["e"].real for e in ex],
        }
    # end-to-end through the public API with host buffers: upload psi0 (pinned FP64) each
    # step, run the step, read the energies back
    if not args.no_e2e:
        host = torch.empty(2 * n ** 3, dtype=torch.float64, pin_memory=True)
        host.numpy()[:] = psi0.reshape(-1).view(np.float64)
        hv = host.numpy()
        e_steps = max(3, min(args.steps, 10))

        def e2e_step():
            lat.set_wavefunction_raw(hv)
            return bench_step()

        e2e_step()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(e_steps):
            e2e_step()
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        if world > 1:
            el = max_over_ranks(el)
        if out is not None:
            out["e2e"] = {"value": aggregate_rate(n ** 3 * CHUNK * e_steps, world, el), "unit": "site-updates/s",
                          "h2d_bytes_per_step": 16 * n ** 3, "d2h_bytes_per_step": 4 * 24,
                          "steps": e_steps,
                          "note": "host wall clock; FP64 psi0 uploaded from pinned memory each step, "
                                  "4 energy records (check + 3 states) read back"}
    if out is not None and not args.no_comparator and world == 1 and w["kinetic"] != I.FDTD:
        try:
            out["comparator_cufft"] = cufft_comparator(w, v, psi0)
        except Exception as exc:  # context only
            out["comparator_cufft"] = {"error": str(exc)[:200]}
    if out is not None and world == 1 and not args.no_comparator:
        try:
            out["c128_arm"] = c128_arm(w, v, psi0)
            out["fp64_peak"] = fp64_peak()
        except Exception as exc:  # context only
            out["c128_arm"] = {"error": str(exc)[:200]}
    if out is not None and world == 1 and args.config4:
        out["config4_n512"] = workload_steps("gaussmix_symanzik_n512")
    if out is not None and not args.no_served:
        lat.close()
        torch.cuda.synchronize()
        try:
            out["served"] = served_benchmark(args.served_requests, args.served_cap)
        except Exception as exc:
            out["served"] = {"error": str(exc)[:300]}
    if out is not None and world == 1 and not args.no_cpu_baseline:
        cores = os.cpu_count() or 1
        rate, steps, el = oracle_rate_cores(args.workload, args.n, args.cpu_seconds, cores)
        out["cpu_baseline"] = {"value": rate, "unit": "site-updates/s", "cores": cores, "kind": "oracle",
                               "sample": f"{steps} FP64 oracle imaginary-time steps of each of {cores} independent "
                                         f"N={n} lattices of the same workload, one per host core ({el:.1f} s; "
                                         f"numpy FFT, one thread each)"}
        rate1, steps1, el1 = oracle_rate(w, v, psi0, args.cpu_seconds / 2)
        out["cpu_baseline_one_core"] = {"value": rate1, "unit": "site-updates/s", "cores": 1, "kind": "oracle",
                                        "sample": f"{steps1} FP64 oracle steps of the same N={n} workload "
                                                  f"({el1:.1f} s, one thread)"}
    if out is not None and world == 1 and not args.no_cpu_baseline:
        try:
            out["by_size"] = size_sweep(args.workload, prec)
        except Exception as exc:
            out["by_size"] = {"error": str(exc)[:300]}
    if out is not None:
        print(json.dumps(out), flush=True)
    lat.close()
    if world > 1:
        dist.destroy_process_group()


def run_served_full(args):
    """The served mix at its stated size (one GPU): Poisson arrivals in real time, admission
    by HBM footprint into 170 GB, FP32 lattices batched with FP64 reductions; solves/s,
    p50/p99 latency from arrival to retirement, converged/capped counts, and the FP32
    batched vs FP64 per-lattice comparator on small requests."""
    import torch

    from paper_2211_10185_gb300 import build as B

    torch.cuda.set_device(0)
    B.build()
    clocks = ClockSampler(torch.cuda.current_device())
    t0 = time.perf_counter()
    served = served_benchmark(2000, 20000, sizes=SERVED_SIZES, warm=False)
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    line = {"metric": "served solves/s, p50/p99 latency to convergence", "value": served.get("solves_per_s"),
            "unit": "solves/s", "n_gpus": 1, "higher_is_better": True, "data": "synthetic (seeded served mix)",
            "config": {"workload": "2000 Cornell solves, Poisson 200/s, N in {32,48,64,96,128,192,256}, "
                                   "kinetic uniform over FDTD/HK1/HK2/HK3, kappa U[.3,.6], sigma U[.1,.25], "
                                   "m U[.3,5], a = 16/N, default dtau, cap 20000 steps, 170 GB"},
            "served": served, "wall_s": wall, "clocks": clk}
    print(json.dumps(line), flush=True)


FFT_VARIANT_SIZES = (32, 48, 64, 96, 128, 192, 384, 512)


def run_fft_variants(args):
    """The complex-FP32 four-pass FFT step in every variant the autotuner chooses from:
    tile geometry 0/1, and the second radix plan (variants 2/3) where a size has one.
    Per size and variant: a lattice (a = 16/N, Cornell kappa 0.4 sigma 0.2, Eq. HK3, m = 1,
    four-pass form), 130 warm-up steps, then 640 steps (checks every 64, CUDA-graph replay
    between checks) timed with CUDA events on the lattice's stream.  The autotuner's
    choice is put back to pending afterwards."""
    import ctypes as C

    import torch

    from paper_2211_10185_gb300 import build as B
    from paper_2211_10185_gb300 import qfdtd as Q
    from paper_2211_10185_gb300.lattice import Lattice

    torch.cuda.set_device(0)
    B.build()
    lib = Q.load()
    clocks = ClockSampler(torch.cuda.current_device())
    res = {}
    for n in FFT_VARIANT_SIZES:
        a = 16.0 / n
        v = I.cornell(n, a, 0.4, 0.2)
        psi0 = np.ones((n, n, n), complex)
        per = {}
        for variant in range(4):
            if lib.qf_set_fft_tiles(n, variant) != Q.QF_OK:
                continue  # (no second radix plan for this size)
            lat = Lattice(n, a, precision="c64", n_snap=1)
            lat.set_potential(v)
            lat.set_kinetic(I.FFT_REL, 1.0)
            lat.set_wavefunction(psi0)
            lat.use_two_pass_fft(False)
            lat.step_n(130, tol=0.0, check_every=CHUNK, snap_every=0)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(lat.stream)
            lat.step_n(640, tol=0.0, check_every=CHUNK, snap_every=0)
            e1.record(lat.stream)
            torch.cuda.synchronize()
            per[str(variant)] = e0.elapsed_time(e1) / 640 * 1e3
            lat.close()
        lib.qf_set_fft_tiles(n, -1)
        res[str(n)] = {"us_per_step": per, "fastest": min(per, key=per.get)}
    line = {"metric": "four-pass FFT step time per tile / radix-plan variant", "unit": "us/step",
            "n_gpus": 1, "higher_is_better": False, "data": "synthetic (Cornell, constant psi0)",
            "variants": {"0": "tile 0, plan 0", "1": "tile 1, plan 0", "2": "tile 0, plan 1",
                         "3": "tile 1, plan 1"},
            "results": res, "clocks": clocks.stop()}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.fft_variants:
        run_fft_variants(args)
    elif args.served_full:
        run_served_full(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
