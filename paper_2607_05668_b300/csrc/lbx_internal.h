// Internal host-side structures shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <utility>

#include "lbx.h"
#include "kernels.cuh"

struct lbx_system {
  int family;
  int K, NC, D;
  double params[8];
  double Q0[24];
};

struct lbx_scheme {
  lbx_system sys;
  lbx_scheme_desc d;            // d.mms_modes is cleared: the table lives in `modes`
  lbx_mms_mode modes[LBX_MMS_MAX_MODES];
  int q;
  int nx, ny, nz;
  long long ncell;
  double dx, dt, lam, cs2;
  double tau[lbx::KMAX];
};

namespace lbx {

// Whether the step kernels read the step index (manufactured forcing, or prescribed
// coefficient fields that move with time); the device counter then advances every step.
inline bool time_dependent(const lbx_scheme& s) {
  return s.d.mms != LBX_MMS_NONE || s.d.prescribed == LBX_PRESCRIBED_ADVECTED;
}

struct Ops {
  cudaError_t (*step)(const lbx_state*, const void* A, void* B, int rel, cudaStream_t);
  // chk: null, or two words the init checks accumulate into (k_init)
  cudaError_t (*init)(const lbx_state*, const double* Q, void* A, unsigned long long* maxbits, int write,
                      unsigned long long* chk);
  cudaError_t (*gather)(const lbx_state*, const void* A, double* Qout, double* fout);
  cudaError_t (*scatter)(const lbx_state*, const double* fin, void* A);
  cudaError_t (*reduce)(const lbx_state*, const void* A, const double* Qref, double* partials, int nblk, int mode);
  const void* (*step_fn)();
  bool reg;
  // batched persistent step: insts = BatchInst<C>[n] on the device
  // fourier: the instances carry mode-table forcing (the forced instantiation)
  cudaError_t (*batch_step)(const void* A, void* B, const void* insts, const int2* tiles, int ntiles, int fourier,
                            const long long* step_ptr, int step_rel, int grid, int block, cudaStream_t);
  const void* (*batch_fn)();
  size_t (*smem_bytes)(int threads);   // dynamic shared memory of a step launch
  size_t inst_bytes;   // sizeof(BatchInst<C>)
  size_t elem_bytes;   // storage bytes per population value
  // in-place step of the given kind (1 or 2) on the single buffer F (see k_step_inplace)
  cudaError_t (*step_inplace)(const lbx_state*, void* F, int kind, int rel, cudaStream_t);
  // slab faces: copy the face slots of A into (pack = 1) or from (0) the two face buffers
  cudaError_t (*face)(const lbx_state*, void* A, void* up, void* dn, int pack, cudaStream_t);
  int face_nf;         // velocities crossing one face (c_a = +1 along the slab axis)
  // init / moments of the planes plane0 .. plane0 + nplanes - 1 of the last axis
  cudaError_t (*init_planes)(const lbx_state*, const double* Q, void* A, int plane0, int nplanes,
                             unsigned long long* chk);
  cudaError_t (*gather_planes)(const lbx_state*, const void* A, double* Qout, int plane0, int nplanes);
};

lbx_status fail(lbx_status s, const char* fmt, ...);
bool find_ops(int family, int lattice, int precision, Ops* o);
int lattice_q(int lattice);
size_t storage_size(int precision);

}  // namespace lbx

struct lbx_state {
  lbx_scheme sch;
  cudaStream_t stream = nullptr;
  cudaStream_t copy_stream = nullptr;   // host copies overlapped with kernels (created on use)
  // planes [plane_lo, plane_lo + plane_n) of the last axis that a step launch covers
  // (lbx_step_planes; plane_n = 0: all planes)
  int plane_lo = 0, plane_n = 0;
  int step_planes() const { return plane_n > 0 ? plane_n : (sch.sys.D == 3 ? sch.nz : sch.ny); }
  lbx::Ops ops{};
  void* fa = nullptr;
  void* fb = nullptr;
  bool own_a = false, own_b = false;
  bool cur_a = true;            // current populations live in fa
  bool inplace = false;         // one buffer (fa), in-place streaming in step pairs
  int half = 0;                 // in place: 1 after a pair's first step (layout not standard)
  long long step = 0;
  bool step_dirty = false;      // host counter ahead of the device counter
  bool nonfinite = false;
  long long* d_step = nullptr;
  double* d_feq0 = nullptr;     // f^eq(Q0) [K][q]
  double* d_partials = nullptr; // reduction scratch [red_blocks][K][4]
  double* d_red_out = nullptr;  // [K][4]
  int red_blocks = 0;
  void* d_mms_modes = nullptr;  // lbx::MmsMode[n] of a FOURIER forcing
  double* d_mms_tab64 = nullptr;
  float* d_mms_tab32 = nullptr;
  double* d_pf_tab64 = nullptr;  // sin/cos tables of the advected solid (HCNSF, float64 step)
  void* d_pf_trig = nullptr;     // sin/cos of the advected solid's field times of a step (4 values)
  double scale[lbx::KMAX];
  lbx::KParams<double> pd;
  lbx::KParams<float> pf;
  bool use_graph = false;       // lbx_step replays captured graphs
  int block = 128;              // threads per block of staged (shared-memory) step kernels
  int staging = 0;              // lbx_staging of staged step kernels (0 = automatic)
  unsigned int* d_err = nullptr; // device error word of the step kernels
  unsigned long long wait_ns = lbx::BULK_WAIT_NS;  // limit of the bulk-copy waits
  std::map<std::pair<long long, int>, cudaGraphExec_t> graphs;

  void* cur() const { return cur_a ? fa : fb; }
  void* nxt() const { return cur_a ? fb : fa; }
  template <typename T>
  const lbx::KParams<T>& pc() const;
};

template <>
inline const lbx::KParams<double>& lbx_state::pc<double>() const { return pd; }
template <>
inline const lbx::KParams<float>& lbx_state::pc<float>() const { return pf; }

namespace lbx {
// Bulk row copies need rows of whole 16-byte runs and 16-byte aligned population buffers.
inline bool bulk_eligible(const lbx_state* st) {
  return st->sch.nx % 8 == 0 && ((uintptr_t)st->fa % 16) == 0 && ((uintptr_t)st->fb % 16) == 0;
}
// The staging a staged step kernel uses: LBX_STAGE_AUTO resolves to bulk row copies when
// they apply and to per-thread copies otherwise.
inline int resolved_staging(const lbx_state* st) {
  if (st->staging != LBX_STAGE_AUTO) return st->staging;
  return bulk_eligible(st) ? LBX_STAGE_BULK : LBX_STAGE_THREAD;
}
void refresh_params(lbx_state* st);
lbx_status run_reduce(lbx_state* st, const double* Qref, int mode, double* host_out);
lbx_status ensure_step_counter(lbx_state* st);
lbx_status require_standard_layout(const lbx_state* st, const char* who);
void feq0_table(const lbx_scheme& s, double* out);                 // f^eq(Q0) [K][q]
cudaError_t launch_advance(long long* step, long long n, cudaStream_t s);
}  // namespace lbx
