// Step, init, moment and reduction kernels of ADR cascade on D2Q5 and D2Q9, in every storage mode.
#include "ops_impl.cuh"

namespace lbx {
bool find_ops_adr_d2q5(int precision, Ops* o) { return pick_store<LatD2Q5, SysADR>(precision, o); }
bool find_ops_adr_d2q9(int precision, Ops* o) { return pick_store<LatD2Q9, SysADR>(precision, o); }
}  // namespace lbx
