"""Element-by-element comparison of complex fields for the GPU parity tests.

A relative L2 bound alone can hide a localised indexing error (one bad tile edge,
Nyquist row or radix-3 column), so every comparison also bounds the worst site:
|got - ref| <= site_factor * l2_tol * rms(ref) at every site, where l2_tol is the
arithmetic's bound on the relative rms error (c * eps * log2 N for the FFT step).
"""
import math

import numpy as np


def field_errors(got, ref):
    """(relative L2 error, worst site error / rms of ref)."""
    got = np.asarray(got)
    ref = np.asarray(ref)
    assert got.shape == ref.shape
    diff = (got - ref).ravel()
    nr = np.linalg.norm(ref.ravel())
    rms = nr / math.sqrt(ref.size)
    return np.linalg.norm(diff) / nr, np.max(np.abs(diff)) / rms


def assert_field_close(got, ref, l2_tol, site_factor=10.0, what=""):
    rel, worst = field_errors(got, ref)
    assert rel < l2_tol, f"{what} relative L2 error {rel:.3e} >= {l2_tol:.3e}"
    assert worst < site_factor * l2_tol, (
        f"{what} worst site error {worst:.3e} rms >= {site_factor * l2_tol:.3e} rms")
