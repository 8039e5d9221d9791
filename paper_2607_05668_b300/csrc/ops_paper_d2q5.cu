// Step, init, moment and reduction kernels of Burgers, compressible Euler and Maxwell TM on D2Q5, in every storage mode.
#include "ops_impl.cuh"

namespace lbx {
bool find_ops_burgers_d2q5(int precision, Ops* o) { return pick_store<LatD2Q5, SysBurgers>(precision, o); }
bool find_ops_euler_d2q5(int precision, Ops* o) { return pick_store<LatD2Q5, SysEuler>(precision, o); }
bool find_ops_maxwell_d2q5(int precision, Ops* o) { return pick_store<LatD2Q5, SysMaxwell>(precision, o); }
}  // namespace lbx
