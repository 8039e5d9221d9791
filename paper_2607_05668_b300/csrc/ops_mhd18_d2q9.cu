// Step, init, moment and reduction kernels of the paper's 18-component MHD on D2Q9, in every storage mode.
#include "ops_impl.cuh"

namespace lbx {
bool find_ops_mhd18_d2q9(int precision, Ops* o) { return pick_store<LatD2Q9, SysMHD18>(precision, o); }
}  // namespace lbx
