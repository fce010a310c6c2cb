"""``Lattice``: one libqfdtd handle whose device workspace and stream come from torch.

Thin marshalling over the C ABI (include/qfdtd.h): numpy FP64 host arrays in and out,
a torch uint8 CUDA tensor as the caller-owned workspace, and a dedicated torch stream (or
a given one) for all GPU work: the library synchronises it in every call that returns
host data; torch work on other streams that reads a field (``field_tensor``) must wait
for it.  Every method maps to one C entry point.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import qfdtd as Q


def _check(lat_handle, status, where, ok=(Q.QF_OK,)):
    if status not in ok:
        lib = Q.load()
        msg = lib.qf_last_error(lat_handle).decode() if lat_handle else ""
        raise Q.QFError(status, where, msg)
    return status


class Lattice:
    def __init__(self, n: int, a: float, precision: str = "c64", n_snap: int = 3, stream=None,
                 device: int | None = None, plateau_slots: int = 0):
        import torch

        self.lib = Q.load()
        self.n, self.a = int(n), float(a)
        self.prec = Q.QF_PREC_C64 if precision == "c64" else Q.QF_PREC_C128
        self.desc = Q.qf_lattice_desc(self.n, self.a, self.prec, int(n_snap), int(plateau_slots))
        nbytes = C.c_size_t()
        _check(None, self.lib.qf_workspace_bytes(C.byref(self.desc), C.byref(nbytes)), "qf_workspace_bytes")
        dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        # a stream of its own: CUDA graphs cannot capture the legacy default stream
        self.stream = stream if stream is not None else torch.cuda.Stream(device=dev)
        # the caller (this object) owns the device memory; 256-byte alignment is guaranteed
        self.workspace = torch.empty(int(nbytes.value), dtype=torch.uint8, device=dev)
        # stream-ordered hand-over: the block may have been used on the allocating stream
        # before, and must not be reused there while this lattice's stream still runs
        self.stream.wait_stream(torch.cuda.current_stream(dev))
        self.workspace.record_stream(self.stream)
        h = C.c_void_p()
        _check(None, self.lib.qf_create_lattice(C.byref(self.desc), C.c_void_p(self.workspace.data_ptr()),
                                                nbytes.value, C.c_void_p(self.stream.cuda_stream),
                                                C.byref(h)), "qf_create_lattice")
        self.h = h

    # -- lifetime --------------------------------------------------------------------------
    def close(self):
        if getattr(self, "h", None):
            self.lib.qf_destroy_lattice(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- set-up ----------------------------------------------------------------------------
    def set_potential(self, v):
        v = np.asarray(v)
        re = np.ascontiguousarray(v.real, dtype=np.float64).reshape(-1)
        im = np.ascontiguousarray(v.imag, dtype=np.float64).reshape(-1) if np.iscomplexobj(v) else None
        _check(self.h, self.lib.qf_set_potential(self.h, Q.dptr(re), Q.dptr(im)), "qf_set_potential")

    def set_kinetic(self, kinetic: int, mass: float, dtau: float | None = None):
        _check(self.h, self.lib.qf_set_kinetic(self.h, int(kinetic), float(mass), float(dtau or 0.0)),
               "qf_set_kinetic")

    def set_wavefunction(self, psi):
        buf = np.ascontiguousarray(np.asarray(psi, dtype=np.complex128).reshape(-1)).view(np.float64)
        _check(self.h, self.lib.qf_set_wavefunction(self.h, Q.dptr(buf)), "qf_set_wavefunction")

    def set_wavefunction_raw(self, re_im: np.ndarray):
        """re_im: C-contiguous float64 array of 2 N^3 values (e.g. pinned host memory)."""
        _check(self.h, self.lib.qf_set_wavefunction(self.h, Q.dptr(re_im)), "qf_set_wavefunction")

    def get_wavefunction(self, slot: int = -1) -> np.ndarray:
        out = np.empty(2 * self.n ** 3, dtype=np.float64)
        _check(self.h, self.lib.qf_get_wavefunction(self.h, int(slot), Q.dptr(out)), "qf_get_wavefunction")
        return out.view(np.complex128).reshape(self.n, self.n, self.n)

    # -- stepping --------------------------------------------------------------------------
    def step_n(self, max_steps: int, tol: float = 0.0, check_every: int = 64, snap_every: int | None = None):
        """Returns (status, steps_done); status is QF_OK (converged) or QF_ENOTCONV."""
        done = C.c_int64()
        se = check_every if snap_every is None else snap_every
        st = self.lib.qf_step_n(self.h, int(max_steps), float(tol), int(check_every), int(se), C.byref(done))
        _check(self.h, st, "qf_step_n", ok=(Q.QF_OK, Q.QF_ENOTCONV))
        return st, done.value

    def energies(self) -> dict:
        e = Q.qf_energy()
        _check(self.h, self.lib.qf_energies(self.h, C.byref(e)), "qf_energies")
        return e.as_dict()

    def project_excited(self, n_states: int = 3):
        out = (Q.qf_energy * n_states)()
        _check(self.h, self.lib.qf_project_excited(self.h, int(n_states), out), "qf_project_excited")
        return [out[i].as_dict() for i in range(n_states)]

    def track_excited(self, n_states: int = 3):
        """Gram-Schmidt of the latest snapshots now, recorded for the plateau of E_i(tau)."""
        out = (Q.qf_energy * n_states)()
        _check(self.h, self.lib.qf_track_excited(self.h, int(n_states), out), "qf_track_excited")
        return [out[i].as_dict() for i in range(n_states)]

    def excited_plateau(self, n_states: int = 3):
        """[(record index, energy record)] of the chosen plateau record per state."""
        out = (Q.qf_energy * n_states)()
        rec = (C.c_int * n_states)()
        _check(self.h, self.lib.qf_excited_plateau(self.h, int(n_states), out, rec), "qf_excited_plateau")
        return [(rec[i], out[i].as_dict()) for i in range(n_states)]

    def parity_project(self, which: int, axis: int = 3, target: int = -1):
        _check(self.h, self.lib.qf_parity_project(self.h, int(which), int(axis), int(target)),
               "qf_parity_project")

    def prolong_from(self, coarse: "Lattice", slot: int = -1):
        """Live psi <- spectral interpolation of ``coarse``'s field (N/2 sites, spacing 2a)."""
        _check(self.h, self.lib.qf_prolong(coarse.h, int(slot), self.h), "qf_prolong")

    def momentum_distribution(self, slot: int = -1):
        """(p, prob, y) over momentum shells of the field in ``slot`` (see qfdtd.h)."""
        nb = C.c_int()
        self.lib.qf_momentum_distribution(self.h, int(slot), None, None, None, 0, C.byref(nb))
        p = np.empty(nb.value)
        prob = np.empty(nb.value)
        y = np.empty(nb.value)
        _check(self.h, self.lib.qf_momentum_distribution(self.h, int(slot), Q.dptr(p), Q.dptr(prob), Q.dptr(y),
                                                         nb.value, C.byref(nb)), "qf_momentum_distribution")
        return p, prob, y

    def info(self) -> dict:
        i = Q.qf_info()
        _check(self.h, self.lib.qf_get_info(self.h, C.byref(i)), "qf_get_info")
        return dict(dtau=i.dtau, step=i.step, tau=i.tau, kinetic=i.kinetic, n_snapshots=i.n_snapshots,
                    workspace_bytes=i.workspace_bytes, launches=i.launches, temporal_block=i.temporal_block,
                    fft_passes=i.fft_passes, field_exp2=i.field_exp2)

    def use_graphs(self, enable: bool = True):
        _check(self.h, self.lib.qf_use_graphs(self.h, int(bool(enable))), "qf_use_graphs")

    def use_two_pass_fft(self, enable: bool = True):
        """Two HBM passes per FFT step for N = 128 and 256 complex FP32 (default) or four."""
        _check(self.h, self.lib.qf_use_two_pass_fft(self.h, int(bool(enable))), "qf_use_two_pass_fft")

    def set_temporal_blocking(self, k: int):
        """FDTD steps per pass over HBM (1 or 2; complex FP32 only)."""
        _check(self.h, self.lib.qf_set_temporal_blocking(self.h, int(k)), "qf_set_temporal_blocking")

    def profile(self, enable: bool = True):
        _check(self.h, self.lib.qf_profile(self.h, int(bool(enable))), "qf_profile")

    def profile_read(self, reset: bool = False) -> dict:
        """{kernel kind: (launches, total_ms)} of the timed launches so far."""
        out = (Q.qf_kernel_stat * 32)()
        cnt = C.c_int()
        _check(self.h, self.lib.qf_profile_read(self.h, out, 32, C.byref(cnt), int(bool(reset))),
               "qf_profile_read")
        return {out[i].name.decode(): (out[i].launches, out[i].total_ms) for i in range(min(cnt.value, 32))}

    def field_pointer(self, slot: int = -1) -> int:
        p = C.c_void_p()
        _check(self.h, self.lib.qf_field_pointer(self.h, int(slot), C.byref(p)), "qf_field_pointer")
        return p.value

    def field_tensor(self, slot: int = -1):
        """torch view (complex64/complex128, shape N^3) of a device field; no copy."""
        import torch

        off = self.field_pointer(slot) - self.workspace.data_ptr()
        nbytes = self.n ** 3 * (8 if self.prec == Q.QF_PREC_C64 else 16)
        raw = self.workspace[off:off + nbytes]
        dt = torch.complex64 if self.prec == Q.QF_PREC_C64 else torch.complex128
        return raw.view(dt).view(self.n, self.n, self.n)
