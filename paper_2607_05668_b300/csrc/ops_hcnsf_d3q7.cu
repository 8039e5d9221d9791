// Step, init, moment and reduction kernels of the 3D homogenized NSF on D3Q7, in every storage mode.
#include "ops_impl.cuh"

namespace lbx {
bool find_ops_hcnsf_d3q7(int precision, Ops* o) { return pick_store<LatD3Q7, SysHCNSF>(precision, o); }
}  // namespace lbx
