// Step, init, moment and reduction kernels of the paper's 12-component NSF on D2Q5, in every storage mode.
#include "ops_impl.cuh"

namespace lbx {
bool find_ops_nsf12_d2q5(int precision, Ops* o) { return pick_store<LatD2Q5, SysNSF12>(precision, o); }
}  // namespace lbx
