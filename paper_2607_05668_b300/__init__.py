"""B300-native kinetic-relaxation lattice Boltzmann hot path (sm_103a CUDA behind a C ABI).

`lbx` is the ctypes binding of liblbx.so; `workloads` wires the benchmark cases
(ADR cascade, NSF with primitive trackers, 3D MHD with a current tracker) into it.
Importing the package fails when the CUDA library has not been built.
"""
from . import lbx  # noqa: F401  (raises ImportError if liblbx.so is missing)
from .lbx import LbxError, System, Scheme, State, Batch, lattice_velocities, probe_peaks  # noqa: F401
