"""Plain, slow CPU FP64 oracle of the kinetic relaxation LBM (test infrastructure).

This package re-implements the paper's scheme step by step (stencils, exact-flux
equilibrium Eq. feq, moments Eq. moments, BGK collide-and-stream Eq. lbe_update,
reference/equilibrium shift Sec. 2.4.3, manufactured forcing Sec. 4, the
sub-characteristic check Sec. 2.3.2, systems with prescribed coefficient fields such as the
homogenized NSF of Sec. 3) in float64 PyTorch CPU code written for reading, not speed.  It shares no code with the CUDA library and never imports it.

Only the tests, the smoke check and the timed CPU baseline of the benchmark may use it;
the library never routes any computation through it.
"""
from .lattice import LATTICES, Lattice, isotropy_defects  # noqa: F401
from .scheme import Scheme, lattice_steps, tau_vector, rel_norms, eoc  # noqa: F401
from . import systems, mms, subchar, adjoint, decomp  # noqa: F401
