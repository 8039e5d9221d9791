// Step, init, moment and reduction kernels of 3D MHD with the current tracker on D3Q19, in every storage mode.
#include "ops_impl.cuh"

namespace lbx {
bool find_ops_mhd_d3q19(int precision, Ops* o) { return pick_store<LatD3Q19, SysMHD>(precision, o); }
}  // namespace lbx
