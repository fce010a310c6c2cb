"""GB300 (sm_103a) implementation of the quantumfdtd v3 imaginary-time step.

The compute path is the C-ABI library ``lib/libqfdtd.so`` (declared in
``include/qfdtd.h``); ``paper_2211_10185_gb300.qfdtd`` binds it with ctypes and
``paper_2211_10185_gb300.lattice.Lattice`` wraps one handle with a torch-owned device
workspace.  Nothing here falls back to a CPU implementation: if the library is missing,
loading it raises.
"""

__all__ = ["inputs", "qfdtd", "lattice", "build"]
