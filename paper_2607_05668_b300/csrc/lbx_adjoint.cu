// Gradient of a final-time density misfit by the discrete adjoint of the scheme, with
// checkpoint-and-recompute (see adjoint.cuh for the per-step derivation).
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "adjoint.cuh"
#include "lbx.h"
#include "lbx_internal.h"

using namespace lbx;

namespace {

struct AdjOps {
  cudaError_t (*step)(const void* An, const void* Lnext, void* Lout, const lbx_state* st, double* tau_acc);
  cudaError_t (*seed)(const void* AN, const double* target, void* L, const lbx_state* st);
  cudaError_t (*init)(const void* L0, const double* Qinit, const lbx_state* st, double* dJdQ);
  // slab faces of an adjoint buffer: pack (1) the face slots into up / dn, or unpack (0)
  cudaError_t (*face)(void* L, void* up, void* dn, int pack, const lbx_state* st);
  size_t lam_bytes;
};

template <class Lat, template <typename> class SysT, class St>
struct AdjImpl {
  using C = typename St::C;
  using S = typename St::S;
  static dim3 block(const lbx_scheme& s) { return dim3(s.nx >= 128 ? 128 : ((s.nx + 31) / 32) * 32, 1, 1); }
  static dim3 grid(const lbx_scheme& s) {
    dim3 b = block(s);
    return dim3((s.nx + b.x - 1) / b.x, s.ny, s.nz);
  }
  static cudaError_t step(const void* An, const void* Lnext, void* Lout, const lbx_state* st, double* tau_acc) {
    k_adj_step<Lat, SysT, St><<<grid(st->sch), block(st->sch), 0, st->stream>>>(
        (const S*)An, (const C*)Lnext, (C*)Lout, st->pc<C>(), tau_acc);
    return cudaGetLastError();
  }
  static cudaError_t seed(const void* AN, const double* target, void* L, const lbx_state* st) {
    k_adj_seed<Lat, SysT, St><<<grid(st->sch), block(st->sch), 0, st->stream>>>((const S*)AN, target, (C*)L, st->pd);
    return cudaGetLastError();
  }
  static cudaError_t init(const void* L0, const double* Qinit, const lbx_state* st, double* dJdQ) {
    k_adj_init<Lat, SysT, St><<<grid(st->sch), block(st->sch), 0, st->stream>>>((const C*)L0, Qinit, st->pd, dJdQ);
    return cudaGetLastError();
  }
  static cudaError_t face(void* L, void* up, void* dn, int pack, const lbx_state* st) {
    const lbx_scheme& s = st->sch;
    const unsigned int pc = Lat::D == 3 ? (unsigned int)(s.nx * s.ny) : (unsigned int)s.nx;
    const dim3 b(128, 1, 1), g((pc + 127) / 128, FaceVel<Lat>::NF, 2);
    if (pack)
      k_adj_face<Lat, SysT, C, true><<<g, b, 0, st->stream>>>((C*)L, (C*)up, (C*)dn, s.nx, s.ny, s.nz);
    else
      k_adj_face<Lat, SysT, C, false><<<g, b, 0, st->stream>>>((C*)L, (C*)up, (C*)dn, s.nx, s.ny, s.nz);
    return cudaGetLastError();
  }
};

template <class Lat, template <typename> class SysT>
bool pick(int precision, AdjOps* o) {
  if (precision == LBX_FP64) {
    using I = AdjImpl<Lat, SysT, StoreF64>;
    *o = AdjOps{I::step, I::seed, I::init, I::face, sizeof(double)};
    return true;
  }
  if (precision == LBX_FP32_SHIFT) {
    using I = AdjImpl<Lat, SysT, StoreF32>;
    *o = AdjOps{I::step, I::seed, I::init, I::face, sizeof(float)};
    return true;
  }
  return false;
}

bool find_adj(int family, int lattice, int precision, AdjOps* o) {
  switch (family) {
    case LBX_ADR_CASCADE:
      if (lattice == LBX_D2Q5) return pick<LatD2Q5, SysADR>(precision, o);
      if (lattice == LBX_D2Q9) return pick<LatD2Q9, SysADR>(precision, o);
      return false;
    case LBX_NSF_PRIM_TRACK:
      if (lattice == LBX_D2Q5) return pick<LatD2Q5, SysNSF>(precision, o);
      if (lattice == LBX_D2Q9) return pick<LatD2Q9, SysNSF>(precision, o);
      return false;
    case LBX_MHD_J_TRACK:
      if (lattice == LBX_D3Q19) return pick<LatD3Q19, SysMHD>(precision, o);
      return false;
    case LBX_EULER:
      if (lattice == LBX_D2Q5) return pick<LatD2Q5, SysEuler>(precision, o);
      return false;
    case LBX_BURGERS:
      if (lattice == LBX_D2Q5) return pick<LatD2Q5, SysBurgers>(precision, o);
      return false;
    case LBX_MAXWELL_TM:
      if (lattice == LBX_D2Q5) return pick<LatD2Q5, SysMaxwell>(precision, o);
      return false;
    case LBX_NSF_CONS_TRACK:
      if (lattice == LBX_D2Q5) return pick<LatD2Q5, SysNSF12>(precision, o);
      return false;
  }
  return false;
}

// Deterministic float64 sum of n values by one block (fixed thread strides, fixed tree).
__global__ void k_sum_f64(const double* __restrict__ v, long long n, double* __restrict__ out) {
  __shared__ double sm[256];
  double s = 0.0;
  for (long long i = threadIdx.x; i < n; i += blockDim.x) s += v[i];
  sm[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sm[threadIdx.x] += sm[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sm[0];
}

// Device time of the phases of the last lbx_adjoint call on this thread (ms): forward
// sweep, recomputation of the segments, reverse steps, and the rest (misfit, seed, initial
// VJP, dJ/dtau reduction); allocation and host copies of the inputs are outside all four.
thread_local double g_phase_ms[4] = {-1.0, -1.0, -1.0, -1.0};

// CUDA events around the phases; a failed event call only loses the timing.
struct PhaseTimer {
  std::vector<cudaEvent_t> ev;
  cudaStream_t s;
  explicit PhaseTimer(cudaStream_t st) : s(st) {}
  int mark() {
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return -1;
    if (cudaEventRecord(e, s) != cudaSuccess) {
      cudaEventDestroy(e);
      return -1;
    }
    ev.push_back(e);
    return (int)ev.size() - 1;
  }
  double ms(int a, int b) const {
    if (a < 0 || b < 0) return 0.0;
    float v = 0.f;
    return cudaEventElapsedTime(&v, ev[a], ev[b]) == cudaSuccess ? (double)v : 0.0;
  }
  ~PhaseTimer() {
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
  }
};

}  // namespace

extern "C" lbx_status lbx_adjoint_timings(double* ms) {
  if (!ms) return fail(LBX_ERR_ARG, "lbx_adjoint_timings: null argument");
  for (int i = 0; i < 4; ++i) ms[i] = g_phase_ms[i];
  return LBX_OK;
}

extern "C" lbx_status lbx_adjoint(const lbx_scheme* sch, const double* Q_init, int64_t n_steps, int ckpt_every,
                                  const double* rho_target, void* stream, double* J, double* dJ_dQ0,
                                  double* dJ_dtau) {
  if (!sch || !Q_init || !rho_target) return fail(LBX_ERR_ARG, "lbx_adjoint: null argument");
  if (n_steps < 0 || n_steps > (int64_t(1) << 30)) return fail(LBX_ERR_ARG, "lbx_adjoint: step count out of range");
  if (ckpt_every < 1) return fail(LBX_ERR_ARG, "lbx_adjoint: ckpt_every must be >= 1");
  if (sch->d.streaming != LBX_STREAM_TWO_BUFFERS)
    return fail(LBX_ERR_UNSUPPORTED, "lbx_adjoint: two-buffer streaming needed");
  if (sch->d.slab_planes_global != 0)
    return fail(LBX_ERR_UNSUPPORTED,
                "lbx_adjoint: whole grids only; slabs run the step-wise calls (lbx_adjoint_seed, _step, _finish)");
  AdjOps adj;
  if (!find_adj(sch->sys.family, sch->d.lattice, sch->d.precision, &adj))
    return fail(LBX_ERR_UNSUPPORTED, "lbx_adjoint: FP64 or FP32_SHIFT storage of a compiled family needed");
  lbx_state* st = nullptr;
  if (lbx_status s = lbx_init(sch, Q_init, 0, stream, nullptr, nullptr, &st)) return s;
  const int K = sch->sys.K, q = sch->q;
  const long long ncell = sch->ncell;
  const size_t bytes = lbx_state_buffer_bytes(sch);
  const size_t lam_bytes = (size_t)K * q * ncell * adj.lam_bytes;
  const long long k = std::min<long long>(ckpt_every, std::max<long long>(n_steps, 1));
  const long long nck = n_steps == 0 ? 0 : (n_steps + k - 1) / k;
  char *ckpt = nullptr, *seg = nullptr;
  void *La = nullptr, *Lb = nullptr;
  double *tau_acc = nullptr, *d_tgt = nullptr, *d_Qref = nullptr, *d_Q = nullptr, *d_grad = nullptr, *d_sum = nullptr;
  lbx_status rc = LBX_OK;
  cudaError_t e = cudaSuccess;
  auto cleanup = [&]() {
    cudaFree(ckpt); cudaFree(seg); cudaFree(La); cudaFree(Lb); cudaFree(tau_acc); cudaFree(d_tgt);
    cudaFree(d_Qref); cudaFree(d_Q); cudaFree(d_grad); cudaFree(d_sum);
    lbx_state_destroy(st);
  };
#define STEP(call)                                                                                   \
  do {                                                                                               \
    e = (call);                                                                                      \
    if (e != cudaSuccess) {                                                                          \
      rc = fail(e == cudaErrorMemoryAllocation ? LBX_ERR_OOM : LBX_ERR_CUDA, "lbx_adjoint: %s: %s", #call, \
                cudaGetErrorString(e));                                                              \
      cleanup();                                                                                     \
      return rc;                                                                                     \
    }                                                                                                \
  } while (0)
  const cudaStream_t s = st->stream;
  if (nck > 0) STEP(cudaMalloc((void**)&ckpt, bytes * nck));
  if (nck > 0) STEP(cudaMalloc((void**)&seg, bytes * k));
  STEP(cudaMalloc(&La, lam_bytes));
  STEP(cudaMalloc(&Lb, lam_bytes));
  STEP(cudaMalloc((void**)&tau_acc, sizeof(double) * ncell));
  STEP(cudaMemsetAsync(tau_acc, 0, sizeof(double) * ncell, s));
  STEP(cudaMalloc((void**)&d_tgt, sizeof(double) * ncell));
  STEP(cudaMemcpyAsync(d_tgt, rho_target, sizeof(double) * ncell, cudaMemcpyHostToDevice, s));
  STEP(cudaMalloc((void**)&d_Qref, sizeof(double) * K * ncell));
  STEP(cudaMemsetAsync(d_Qref, 0, sizeof(double) * K * ncell, s));
  STEP(cudaMemcpyAsync(d_Qref, d_tgt, sizeof(double) * ncell, cudaMemcpyDeviceToDevice, s));
  STEP(cudaMalloc((void**)&d_Q, sizeof(double) * K * ncell));
  STEP(cudaMemcpyAsync(d_Q, Q_init, sizeof(double) * K * ncell, cudaMemcpyHostToDevice, s));
  STEP(cudaMalloc((void**)&d_grad, sizeof(double) * K * ncell));
  STEP(cudaMalloc((void**)&d_sum, sizeof(double)));
  for (int i = 0; i < 4; ++i) g_phase_ms[i] = -1.0;
  STEP(cudaStreamSynchronize(s));      // inputs on the device: the timed phases start here
  PhaseTimer tm(s);
  std::vector<int> seg_marks;          // per segment: start, recomputed, reversed
  const int m_fwd0 = tm.mark();
  // forward sweep, keeping the state at the start of every segment
  for (long long c = 0; c < nck; ++c) {
    STEP(cudaMemcpyAsync(ckpt + bytes * c, st->cur(), bytes, cudaMemcpyDeviceToDevice, s));
    const long long len = std::min(k, n_steps - c * k);
    if ((rc = lbx_step(st, len))) {
      cleanup();
      return rc;
    }
  }
  const int m_fwd1 = tm.mark();
  // misfit J = 1/2 sum (rho - rho*)^2 (deterministic float64 reduction)
  {
    double out[KMAX * 4];
    if ((rc = run_reduce(st, d_Qref, 1, out))) {
      cleanup();
      return rc;
    }
    if (J) *J = 0.5 * out[0];
  }
  STEP(adj.seed(st->cur(), d_tgt, La, st));

  // reverse sweep: recompute each segment from its checkpoint, then step the adjoint back
  void* Lnext = La;
  void* Lout = Lb;
  for (long long c = nck - 1; c >= 0; --c) {
    const long long len = std::min(k, n_steps - c * k);
    STEP(cudaMemcpyAsync(seg, ckpt + bytes * c, bytes, cudaMemcpyDeviceToDevice, s));
    long long base = c * k;
    STEP(cudaMemcpyAsync(st->d_step, &base, sizeof(base), cudaMemcpyHostToDevice, s));
    STEP(cudaStreamSynchronize(s));   // `base` lives on this stack frame
    seg_marks.push_back(tm.mark());
    for (long long m = 0; m + 1 < len; ++m) STEP(st->ops.step(st, seg + bytes * m, seg + bytes * (m + 1), (int)m, s));
    seg_marks.push_back(tm.mark());
    for (long long m = len - 1; m >= 0; --m) {
      STEP(adj.step(seg + bytes * m, Lnext, Lout, st, tau_acc));
      std::swap(Lnext, Lout);
    }
    seg_marks.push_back(tm.mark());
  }
  STEP(adj.init(Lnext, d_Q, st, d_grad));
  k_sum_f64<<<1, 256, 0, s>>>(tau_acc, ncell, d_sum);
  STEP(cudaGetLastError());
  const int m_end = tm.mark();
  if (dJ_dQ0) STEP(cudaMemcpyAsync(dJ_dQ0, d_grad, sizeof(double) * K * ncell, cudaMemcpyDeviceToHost, s));
  double tsum = 0.0;
  STEP(cudaMemcpyAsync(&tsum, d_sum, sizeof(double), cudaMemcpyDeviceToHost, s));
  STEP(cudaStreamSynchronize(s));
  {
    double rec = 0.0, rev = 0.0;
    for (size_t i = 0; i + 2 < seg_marks.size(); i += 3) {
      rec += tm.ms(seg_marks[i], seg_marks[i + 1]);
      rev += tm.ms(seg_marks[i + 1], seg_marks[i + 2]);
    }
    g_phase_ms[0] = tm.ms(m_fwd0, m_fwd1);
    g_phase_ms[1] = rec;
    g_phase_ms[2] = rev;
    g_phase_ms[3] = tm.ms(m_fwd0, m_end) - g_phase_ms[0] - rec - rev;
  }
  const double tau = sch->tau[0];
  if (dJ_dtau) *dJ_dtau = tsum / (tau * tau);
  cleanup();
  return LBX_OK;
#undef STEP
}

// ---------------------------------------------------------- step-wise reverse sweep
// The pieces of lbx_adjoint for a caller that runs the sweep itself: the slabs of a grid cut
// across processes, which exchange their faces between the steps (include/lbx.h).

#define CK(call)                                                                                     \
  do {                                                                                               \
    cudaError_t e_ = (call);                                                                         \
    if (e_ != cudaSuccess)                                                                           \
      return fail(e_ == cudaErrorMemoryAllocation ? LBX_ERR_OOM : LBX_ERR_CUDA, "%s: %s", #call,     \
                  cudaGetErrorString(e_));                                                           \
  } while (0)

static lbx_status adj_of(const lbx_state* st, AdjOps* o, const char* who) {
  if (!st) return fail(LBX_ERR_ARG, "%s: null state", who);
  if (st->inplace) return fail(LBX_ERR_UNSUPPORTED, "%s: two-buffer streaming needed", who);
  if (!find_adj(st->sch.sys.family, st->sch.d.lattice, st->sch.d.precision, o))
    return fail(LBX_ERR_UNSUPPORTED, "%s: FP64 or FP32_SHIFT storage of a compiled family needed", who);
  return LBX_OK;
}

extern "C" size_t lbx_adjoint_lam_bytes(const lbx_scheme* sch) {
  AdjOps o{};
  if (!sch || !find_adj(sch->sys.family, sch->d.lattice, sch->d.precision, &o)) return 0;
  return (size_t)sch->sys.K * sch->q * (size_t)sch->ncell * o.lam_bytes;
}

extern "C" size_t lbx_adjoint_halo_bytes(const lbx_scheme* sch) {
  AdjOps o{};
  Ops po{};
  if (!sch || !find_adj(sch->sys.family, sch->d.lattice, sch->d.precision, &o)) return 0;
  if (!find_ops(sch->sys.family, sch->d.lattice, sch->d.precision, &po)) return 0;
  const size_t pc = sch->sys.D == 3 ? (size_t)sch->nx * sch->ny : (size_t)sch->nx;
  return (size_t)po.face_nf * sch->sys.K * pc * o.lam_bytes;
}

extern "C" lbx_status lbx_adjoint_checkpoint(lbx_state* st, void* dst) {
  if (!st || !dst) return fail(LBX_ERR_ARG, "lbx_adjoint_checkpoint: null argument");
  if (lbx_status s = require_standard_layout(st, "lbx_adjoint_checkpoint")) return s;
  CK(cudaMemcpyAsync(dst, st->cur(), lbx_state_buffer_bytes(&st->sch), cudaMemcpyDeviceToDevice, st->stream));
  return LBX_OK;
}

extern "C" lbx_status lbx_adjoint_restore(lbx_state* st, const void* src, int64_t step) {
  if (!st || !src) return fail(LBX_ERR_ARG, "lbx_adjoint_restore: null argument");
  if (step < 0) return fail(LBX_ERR_ARG, "lbx_adjoint_restore: negative step");
  if (lbx_status s = require_standard_layout(st, "lbx_adjoint_restore")) return s;
  CK(cudaMemcpyAsync(st->cur(), src, lbx_state_buffer_bytes(&st->sch), cudaMemcpyDeviceToDevice, st->stream));
  long long base = (long long)step;
  CK(cudaMemcpyAsync(st->d_step, &base, sizeof(base), cudaMemcpyHostToDevice, st->stream));
  CK(cudaStreamSynchronize(st->stream));   // `base` lives on this stack frame
  st->step = base;
  st->step_dirty = false;
  return LBX_OK;
}

extern "C" lbx_status lbx_adjoint_seed(lbx_state* st, const double* rho_target, void* lam, double* J) {
  AdjOps adj;
  if (lbx_status s = adj_of(st, &adj, "lbx_adjoint_seed")) return s;
  if (!rho_target || !lam) return fail(LBX_ERR_ARG, "lbx_adjoint_seed: null argument");
  const int K = st->sch.sys.K;
  const size_t ncell = (size_t)st->sch.ncell;
  double* d_Qref = nullptr;
  CK(cudaMalloc((void**)&d_Qref, sizeof(double) * K * ncell));
  cudaError_t e = cudaMemsetAsync(d_Qref, 0, sizeof(double) * K * ncell, st->stream);
  if (!e) e = cudaMemcpyAsync(d_Qref, rho_target, sizeof(double) * ncell, cudaMemcpyDeviceToDevice, st->stream);
  if (e) {
    cudaFree(d_Qref);
    return fail(LBX_ERR_CUDA, "lbx_adjoint_seed: %s", cudaGetErrorString(e));
  }
  double out[KMAX * 4];
  lbx_status rc = run_reduce(st, d_Qref, 1, out);    // synchronous
  cudaFree(d_Qref);
  if (rc) return rc;
  if (J) *J = 0.5 * out[0];
  if (cudaError_t e2 = adj.seed(st->cur(), rho_target, lam, st))
    return fail(LBX_ERR_CUDA, "lbx_adjoint_seed: %s", cudaGetErrorString(e2));
  return LBX_OK;
}

extern "C" lbx_status lbx_adjoint_step(lbx_state* st, const void* An, const void* lam_next, void* lam_out,
                                       double* tau_acc) {
  AdjOps adj;
  if (lbx_status s = adj_of(st, &adj, "lbx_adjoint_step")) return s;
  if (!An || !lam_next || !lam_out || !tau_acc) return fail(LBX_ERR_ARG, "lbx_adjoint_step: null argument");
  if (lam_next == lam_out) return fail(LBX_ERR_ARG, "lbx_adjoint_step: lam_next and lam_out must differ");
  if (cudaError_t e = adj.step(An, lam_next, lam_out, st, tau_acc))
    return fail(LBX_ERR_CUDA, "lbx_adjoint_step: %s", cudaGetErrorString(e));
  return LBX_OK;
}

static lbx_status adj_face_call(lbx_state* st, void* lam, void* upper, void* lower, int pack, const char* who) {
  AdjOps adj;
  if (lbx_status s = adj_of(st, &adj, who)) return s;
  if (!lam || !upper || !lower) return fail(LBX_ERR_ARG, "%s: null argument", who);
  if (cudaError_t e = adj.face(lam, upper, lower, pack, st)) return fail(LBX_ERR_CUDA, "%s: %s", who, cudaGetErrorString(e));
  return LBX_OK;
}

extern "C" lbx_status lbx_adjoint_halo_pack(lbx_state* st, const void* lam, void* face_upper, void* face_lower) {
  return adj_face_call(st, const_cast<void*>(lam), face_upper, face_lower, 1, "lbx_adjoint_halo_pack");
}

extern "C" lbx_status lbx_adjoint_halo_unpack(lbx_state* st, void* lam, const void* face_upper, const void* face_lower) {
  return adj_face_call(st, lam, const_cast<void*>(face_upper), const_cast<void*>(face_lower), 0,
                       "lbx_adjoint_halo_unpack");
}

extern "C" lbx_status lbx_adjoint_finish(lbx_state* st, const void* lam0, const double* Q_init, double* dJ_dQ0,
                                         const double* tau_acc, double* dJ_dtau) {
  AdjOps adj;
  if (lbx_status s = adj_of(st, &adj, "lbx_adjoint_finish")) return s;
  if (!lam0 || !Q_init || !dJ_dQ0 || !tau_acc) return fail(LBX_ERR_ARG, "lbx_adjoint_finish: null argument");
  if (cudaError_t e = adj.init(lam0, Q_init, st, dJ_dQ0))
    return fail(LBX_ERR_CUDA, "lbx_adjoint_finish: %s", cudaGetErrorString(e));
  double* d_sum = nullptr;
  CK(cudaMalloc((void**)&d_sum, sizeof(double)));
  k_sum_f64<<<1, 256, 0, st->stream>>>(tau_acc, (long long)st->sch.ncell, d_sum);
  cudaError_t e = cudaGetLastError();
  double tsum = 0.0;
  if (!e) e = cudaMemcpyAsync(&tsum, d_sum, sizeof(double), cudaMemcpyDeviceToHost, st->stream);
  if (!e) e = cudaStreamSynchronize(st->stream);
  cudaFree(d_sum);
  if (e) return fail(LBX_ERR_CUDA, "lbx_adjoint_finish: %s", cudaGetErrorString(e));
  const double tau = st->sch.tau[0];
  if (dJ_dtau) *dJ_dtau = tsum / (tau * tau);
  return LBX_OK;
}

#undef CK
