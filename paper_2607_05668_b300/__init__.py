"""B300-native kinetic-relaxation lattice Boltzmann hot path (sm_103a CUDA behind a C ABI).

`lbx` is the ctypes binding of liblbx.so; `workloads` wires the benchmark cases into it
(ADR cascade, NSF with primitive trackers, 3D MHD with a current tracker, the paper's
12-component NSF and 18-component MHD cascades, the 3D homogenized NSF with its moving
solid, and the manufactured-forcing and in-place variants).
Importing the package fails when the CUDA library has not been built.
"""
from . import lbx  # noqa: F401  (raises ImportError if liblbx.so is missing)
from .lbx import LbxError, System, Scheme, State, Batch, lattice_velocities, probe_peaks  # noqa: F401
