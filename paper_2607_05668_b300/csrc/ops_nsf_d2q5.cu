// Step, init, moment and reduction kernels of NSF with primitive trackers on D2Q5, in every storage mode.
#include "ops_impl.cuh"

namespace lbx {
bool find_ops_nsf_d2q5(int precision, Ops* o) { return pick_store<LatD2Q5, SysNSF>(precision, o); }
}  // namespace lbx
