// Dispatch over (system family, lattice): each pair is instantiated in its own ops_*.cu
// translation unit (see ops_impl.cuh).
#include "lbx_internal.h"

namespace lbx {
bool find_ops_adr_d2q5(int precision, Ops* o);
bool find_ops_adr_d2q9(int precision, Ops* o);
bool find_ops_nsf_d2q5(int precision, Ops* o);
bool find_ops_nsf_d2q9(int precision, Ops* o);
bool find_ops_mhd_d3q7(int precision, Ops* o);
bool find_ops_mhd_d3q19(int precision, Ops* o);
bool find_ops_burgers_d2q5(int precision, Ops* o);
bool find_ops_euler_d2q5(int precision, Ops* o);
bool find_ops_maxwell_d2q5(int precision, Ops* o);
bool find_ops_nsf12_d2q5(int precision, Ops* o);
bool find_ops_nsf12_d2q9(int precision, Ops* o);
bool find_ops_mhd18_d2q5(int precision, Ops* o);
bool find_ops_mhd18_d2q9(int precision, Ops* o);
bool find_ops_hcnsf_d3q7(int precision, Ops* o);

bool find_ops(int family, int lattice, int precision, Ops* o) {
  switch (family) {
    case LBX_ADR_CASCADE:
      if (lattice == LBX_D2Q5) return find_ops_adr_d2q5(precision, o);
      if (lattice == LBX_D2Q9) return find_ops_adr_d2q9(precision, o);
      return false;
    case LBX_NSF_PRIM_TRACK:
      if (lattice == LBX_D2Q5) return find_ops_nsf_d2q5(precision, o);
      if (lattice == LBX_D2Q9) return find_ops_nsf_d2q9(precision, o);
      return false;
    case LBX_MHD_J_TRACK:
      if (lattice == LBX_D3Q7) return find_ops_mhd_d3q7(precision, o);
      if (lattice == LBX_D3Q19) return find_ops_mhd_d3q19(precision, o);
      return false;
    case LBX_BURGERS:
      if (lattice == LBX_D2Q5) return find_ops_burgers_d2q5(precision, o);
      return false;
    case LBX_EULER:
      if (lattice == LBX_D2Q5) return find_ops_euler_d2q5(precision, o);
      return false;
    case LBX_MAXWELL_TM:
      if (lattice == LBX_D2Q5) return find_ops_maxwell_d2q5(precision, o);
      return false;
    case LBX_NSF_CONS_TRACK:
      if (lattice == LBX_D2Q5) return find_ops_nsf12_d2q5(precision, o);
      if (lattice == LBX_D2Q9) return find_ops_nsf12_d2q9(precision, o);
      return false;
    case LBX_MHD_POWELL_2D:
      if (lattice == LBX_D2Q5) return find_ops_mhd18_d2q5(precision, o);
      if (lattice == LBX_D2Q9) return find_ops_mhd18_d2q9(precision, o);
      return false;
    case LBX_HCNSF_3D:
      if (lattice == LBX_D3Q7) return find_ops_hcnsf_d3q7(precision, o);
      return false;
  }
  return false;
}

}  // namespace lbx
