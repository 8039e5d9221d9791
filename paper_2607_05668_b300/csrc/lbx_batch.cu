// Batched states: many independent 2D grids (one scheme each, same family, lattice and
// storage) advanced by one persistent launch per step over a shared tile list, with the
// time loop recorded once into a CUDA graph and replayed.  Block size and blocks per SM
// come from a measured sweep (lbx_batch_tune).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <utility>
#include <vector>

#include "lbx.h"
#include "lbx_internal.h"

using namespace lbx;

struct lbx_batch {
  int n = 0;
  int K = 0, q = 0;
  int precision = 0;
  Ops ops{};
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::vector<lbx_scheme> sch;
  std::vector<long long> off;        // element offset of each instance
  std::vector<long long> tab_off;    // offset of each instance's forcing tables
  long long total_elems = 0;
  long long total_cells = 0;
  void* fa = nullptr;
  void* fb = nullptr;
  bool cur_a = true;
  void* d_insts = nullptr;           // BatchInst<C>[n]
  double* d_feq0 = nullptr;          // [n][K][q]
  double* d_tab64 = nullptr;
  float* d_tab32 = nullptr;
  long long* d_step = nullptr;
  MmsMode* d_modes = nullptr;        // FOURIER forcing: every instance's mode table
  std::vector<long long> mode_off;   // first mode of instance j
  long long* d_eoff = nullptr;       // element offset and count of every instance (finite check)
  long long* d_ecnt = nullptr;
  int* d_flags = nullptr;
  long long step = 0;
  int2* d_tiles = nullptr;
  int ntiles = 0;
  int tiles_block = 0;
  int nsm = 148;
  lbx_batch_config cfg{128, 8, 1, 1};
  std::map<std::pair<long long, int>, cudaGraphExec_t> graphs;

  void* cur() const { return cur_a ? fa : fb; }
  void* nxt() const { return cur_a ? fb : fa; }
  char* at(void* base, int j) const { return (char*)base + off[j] * (long long)ops.elem_bytes; }
};

#define CK(call)                                                                                     \
  do {                                                                                               \
    cudaError_t e_ = (call);                                                                         \
    if (e_ != cudaSuccess)                                                                           \
      return fail(e_ == cudaErrorMemoryAllocation ? LBX_ERR_OOM : LBX_ERR_CUDA, "%s: %s", #call,     \
                  cudaGetErrorString(e_));                                                           \
  } while (0)

// A host-side view of instance j as a single state (no device memory of its own), used
// to reuse the single-grid init, gather and reduction launchers.
static void make_view(const lbx_batch* b, int j, lbx_state* v) {
  v->sch = b->sch[j];
  v->stream = b->stream;
  v->ops = b->ops;
  v->d_step = b->d_step;
  v->d_feq0 = b->d_feq0 + (size_t)j * b->K * b->q;
  v->d_mms_tab64 = b->d_tab64 ? b->d_tab64 + b->tab_off[j] : nullptr;
  v->d_mms_tab32 = b->d_tab32 ? b->d_tab32 + b->tab_off[j] : nullptr;
  v->d_mms_modes = b->d_modes ? b->d_modes + b->mode_off[j] : nullptr;
  for (int k = 0; k < KMAX; ++k) v->scale[k] = 1.0;
  refresh_params(v);
}

static void free_batch(lbx_batch* b) {
  if (!b) return;
  for (auto& g : b->graphs) cudaGraphExecDestroy(g.second);
  cudaFree(b->fa);
  cudaFree(b->fb);
  cudaFree(b->d_insts);
  cudaFree(b->d_feq0);
  cudaFree(b->d_tab64);
  cudaFree(b->d_tab32);
  cudaFree(b->d_step);
  cudaFree(b->d_modes);
  cudaFree(b->d_eoff);
  cudaFree(b->d_ecnt);
  cudaFree(b->d_flags);
  cudaFree(b->d_tiles);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

static lbx_status build_tiles(lbx_batch* b, int block) {
  if (b->d_tiles && b->tiles_block == block) return LBX_OK;
  std::vector<int2> t;
  for (int j = 0; j < b->n; ++j)
    for (long long c = 0; c < b->sch[j].ncell; c += block) t.push_back(make_int2(j, (int)c));
  int2* d = nullptr;
  CK(cudaMalloc(&d, sizeof(int2) * t.size()));
  cudaError_t e = cudaMemcpy(d, t.data(), sizeof(int2) * t.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(d);
    return fail(LBX_ERR_CUDA, "batch tiles: %s", cudaGetErrorString(e));
  }
  for (auto& g : b->graphs) cudaGraphExecDestroy(g.second);
  b->graphs.clear();
  cudaFree(b->d_tiles);
  b->d_tiles = d;
  b->ntiles = (int)t.size();
  b->tiles_block = block;
  return LBX_OK;
}

static cudaError_t launch_step(lbx_batch* b, const void* A, void* B, int rel) {
  return b->ops.batch_step(A, B, b->d_insts, b->d_tiles, b->ntiles, b->d_modes != nullptr, b->d_step, rel,
                           b->nsm * b->cfg.ctas_per_sm, b->cfg.block, b->stream);
}

// flags[j] = 1 if any stored population of instance j is NaN or infinite; block j walks
// the instance's elements with a block-size stride.
template <typename S>
__global__ void k_batch_nonfinite(const S* __restrict__ A, const long long* __restrict__ off,
                                  const long long* __restrict__ cnt, int* __restrict__ flags) {
  const int j = blockIdx.x;
  const S* a = A + off[j];
  int bad = 0;
  for (long long e = threadIdx.x; e < cnt[j]; e += blockDim.x) {
    float vf;
    double vd;
    if constexpr (sizeof(S) == 2) {
      vf = __half2float(a[e]);
      bad |= !isfinite(vf);
    } else if constexpr (sizeof(S) == 4) {
      vf = a[e];
      bad |= !isfinite(vf);
    } else {
      vd = a[e];
      bad |= !isfinite(vd);
    }
  }
  bad = __syncthreads_or(bad);
  if (threadIdx.x == 0) flags[j] = bad;
}

extern "C" lbx_status lbx_batch_create(const lbx_scheme* const* schemes, int n, const double* const* Q,
                                       void* stream, lbx_batch** out) {
  if (!schemes || !Q || !out || n < 1) return fail(LBX_ERR_ARG, "lbx_batch_create: bad arguments");
  *out = nullptr;
  if (!schemes[0]) return fail(LBX_ERR_ARG, "lbx_batch_create: null scheme 0");
  const lbx_scheme& s0 = *schemes[0];
  for (int j = 0; j < n; ++j) {
    if (!schemes[j] || !Q[j]) return fail(LBX_ERR_ARG, "lbx_batch_create: null scheme or field %d", j);
    const lbx_scheme& s = *schemes[j];
    if (s.sys.family != s0.sys.family || s.d.lattice != s0.d.lattice || s.d.precision != s0.d.precision ||
        s.d.mms != s0.d.mms)
      return fail(LBX_ERR_ARG, "lbx_batch_create: instance %d differs in family, lattice, storage or forcing", j);
    if (s.sys.D != 2) return fail(LBX_ERR_UNSUPPORTED, "lbx_batch_create: batches are 2D");
    if (s.d.streaming != LBX_STREAM_TWO_BUFFERS)
      return fail(LBX_ERR_UNSUPPORTED, "lbx_batch_create: batches use two-buffer streaming");
    if (s.d.slab_planes_global != 0)
      return fail(LBX_ERR_UNSUPPORTED, "lbx_batch_create: instances are whole grids, not slabs");
  }
  if (s0.d.precision == LBX_FP16_SCALED)
    return fail(LBX_ERR_UNSUPPORTED, "lbx_batch_create: FP16_SCALED storage is not batched");
  auto* b = new lbx_batch();
  b->n = n;
  b->K = s0.sys.K;
  b->q = s0.q;
  b->precision = s0.d.precision;
  if (!find_ops(s0.sys.family, s0.d.lattice, s0.d.precision, &b->ops)) {
    delete b;
    return fail(LBX_ERR_UNSUPPORTED, "lbx_batch_create: combination not compiled");
  }
  auto bail = [&](lbx_status st) {
    free_batch(b);
    return st;
  };
#define CKB(call)                                                                                    \
  do {                                                                                               \
    cudaError_t e_ = (call);                                                                         \
    if (e_ != cudaSuccess)                                                                           \
      return bail(fail(e_ == cudaErrorMemoryAllocation ? LBX_ERR_OOM : LBX_ERR_CUDA, "lbx_batch_create: %s: %s", \
                       #call, cudaGetErrorString(e_)));                                              \
  } while (0)
  if (stream) {
    b->stream = (cudaStream_t)stream;
  } else {
    CKB(cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking));
    b->own_stream = true;
  }
  int dev = 0;
  CKB(cudaGetDevice(&dev));
  CKB(cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, dev));
  long long tab = 0;
  const long long align = 256 / (long long)b->ops.elem_bytes;
  for (int j = 0; j < n; ++j) {
    b->sch.push_back(*schemes[j]);
    b->off.push_back(b->total_elems);
    const long long elems = (long long)b->K * b->q * schemes[j]->ncell;
    b->total_elems += (elems + align - 1) / align * align;
    b->total_cells += schemes[j]->ncell;
    b->tab_off.push_back(tab);
    if (s0.d.mms != LBX_MMS_NONE) tab += 2LL * schemes[j]->nx + 2LL * schemes[j]->ny;
  }
  const size_t bytes = (size_t)b->total_elems * b->ops.elem_bytes;
  CKB(cudaMalloc(&b->fa, bytes));
  CKB(cudaMalloc(&b->fb, bytes));
  CKB(cudaMalloc(&b->d_step, sizeof(long long)));
  CKB(cudaMemset(b->d_step, 0, sizeof(long long)));
  CKB(cudaMalloc(&b->d_feq0, sizeof(double) * n * b->K * b->q));
  if (tab > 0) {
    std::vector<double> t(tab);
    std::vector<float> tf(tab);
    for (int j = 0; j < n; ++j) {
      const int nx = b->sch[j].nx, ny = b->sch[j].ny;
      double* o = t.data() + b->tab_off[j];
      for (int i = 0; i < nx; ++i) {
        o[i] = std::sin(2.0 * M_PI * i / nx);
        o[nx + i] = std::cos(2.0 * M_PI * i / nx);
      }
      for (int i = 0; i < ny; ++i) {
        o[2 * nx + i] = std::sin(2.0 * M_PI * i / ny);
        o[2 * nx + ny + i] = std::cos(2.0 * M_PI * i / ny);
      }
    }
    for (long long i = 0; i < tab; ++i) tf[i] = (float)t[i];
    CKB(cudaMalloc(&b->d_tab64, sizeof(double) * tab));
    CKB(cudaMalloc(&b->d_tab32, sizeof(float) * tab));
    CKB(cudaMemcpy(b->d_tab64, t.data(), sizeof(double) * tab, cudaMemcpyHostToDevice));
    CKB(cudaMemcpy(b->d_tab32, tf.data(), sizeof(float) * tab, cudaMemcpyHostToDevice));
  }
  // per-instance parameters, background equilibria and initial populations
  std::vector<char> insts((size_t)n * b->ops.inst_bytes);
  std::vector<double> feq0((size_t)n * b->K * b->q);
  {
    double* dQ = nullptr;
    long long maxcell = 0;
    for (int j = 0; j < n; ++j) maxcell = std::max(maxcell, b->sch[j].ncell);
    CKB(cudaMalloc(&dQ, sizeof(double) * b->K * maxcell));
    for (int j = 0; j < n; ++j) {
      // kernel parameters through a single-instance view; f^eq(Q0) as lbx_init computes it
      lbx_state v;
      make_view(b, j, &v);
      feq0_table(b->sch[j], feq0.data() + (size_t)j * b->K * b->q);
      if (b->precision == LBX_FP64) {
        auto* bi = reinterpret_cast<BatchInst<double>*>(insts.data()) + j;
        bi->p = v.pd;
        bi->off = b->off[j];
      } else {
        auto* bi = reinterpret_cast<BatchInst<float>*>(insts.data()) + j;
        bi->p = v.pf;
        bi->off = b->off[j];
      }
    }
    cudaError_t e = cudaMemcpy(b->d_feq0, feq0.data(), sizeof(double) * feq0.size(), cudaMemcpyHostToDevice);
    for (int j = 0; j < n && e == cudaSuccess; ++j) {
      lbx_state v;
      make_view(b, j, &v);
      e = cudaMemcpyAsync(dQ, Q[j], sizeof(double) * b->K * b->sch[j].ncell, cudaMemcpyHostToDevice, b->stream);
      if (e == cudaSuccess) e = b->ops.init(&v, dQ, b->at(b->fa, j), nullptr, 1, nullptr);
      if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    }
    cudaFree(dQ);
    CKB(e);
  }
  if (s0.d.mms == LBX_MMS_FOURIER) {
    std::vector<MmsMode> md;
    for (int j = 0; j < n; ++j) {
      b->mode_off.push_back((long long)md.size());
      for (int m = 0; m < b->sch[j].d.mms_n_modes; ++m) {
        const lbx_mms_mode& a = b->sch[j].modes[m];
        MmsMode o{};
        for (int d = 0; d < 3; ++d) o.k2pi[d] = 2.0 * M_PI * a.k[d];
        o.amp = a.amp;
        o.phase = a.phase;
        o.sigma = a.sigma;
        o.omega = a.omega;
        o.psi = a.psi;
        o.p = a.p;
        md.push_back(o);
      }
    }
    CKB(cudaMalloc((void**)&b->d_modes, sizeof(MmsMode) * md.size()));
    CKB(cudaMemcpy(b->d_modes, md.data(), sizeof(MmsMode) * md.size(), cudaMemcpyHostToDevice));
    // the instance parameters were filled before the tables existed: fill them again
    for (int j = 0; j < n; ++j) {
      lbx_state v;
      make_view(b, j, &v);
      if (b->precision == LBX_FP64)
        reinterpret_cast<BatchInst<double>*>(insts.data())[j].p = v.pd;
      else
        reinterpret_cast<BatchInst<float>*>(insts.data())[j].p = v.pf;
    }
  }
  {
    std::vector<long long> eo(n), ec(n);
    for (int j = 0; j < n; ++j) {
      eo[j] = b->off[j];
      ec[j] = (long long)b->K * b->q * b->sch[j].ncell;
    }
    CKB(cudaMalloc((void**)&b->d_eoff, sizeof(long long) * n));
    CKB(cudaMalloc((void**)&b->d_ecnt, sizeof(long long) * n));
    CKB(cudaMalloc((void**)&b->d_flags, sizeof(int) * n));
    CKB(cudaMemcpy(b->d_eoff, eo.data(), sizeof(long long) * n, cudaMemcpyHostToDevice));
    CKB(cudaMemcpy(b->d_ecnt, ec.data(), sizeof(long long) * n, cudaMemcpyHostToDevice));
  }
  CKB(cudaMalloc(&b->d_insts, insts.size()));
  CKB(cudaMemcpy(b->d_insts, insts.data(), insts.size(), cudaMemcpyHostToDevice));
  if (lbx_status st = build_tiles(b, b->cfg.block)) return bail(st);
  *out = b;
  return LBX_OK;
#undef CKB
}

extern "C" lbx_status lbx_batch_info(const lbx_batch* b, int* n, int64_t* total_cells, size_t* buffer_bytes) {
  if (!b) return fail(LBX_ERR_ARG, "lbx_batch_info: null batch");
  if (n) *n = b->n;
  if (total_cells) *total_cells = b->total_cells;
  if (buffer_bytes) *buffer_bytes = (size_t)b->total_elems * b->ops.elem_bytes;
  return LBX_OK;
}

extern "C" lbx_status lbx_batch_get_config(const lbx_batch* b, lbx_batch_config* cfg) {
  if (!b || !cfg) return fail(LBX_ERR_ARG, "lbx_batch_get_config: null argument");
  *cfg = b->cfg;
  return LBX_OK;
}

extern "C" lbx_status lbx_batch_set_config(lbx_batch* b, const lbx_batch_config* cfg) {
  if (!b || !cfg) return fail(LBX_ERR_ARG, "lbx_batch_set_config: null argument");
  if (cfg->block < 32 || cfg->block > 1024 || cfg->block % 32 != 0)
    return fail(LBX_ERR_ARG, "lbx_batch_set_config: block must be a multiple of 32 in [32, 1024]");
  if (cfg->ctas_per_sm < 1 || cfg->ctas_per_sm > 64)
    return fail(LBX_ERR_ARG, "lbx_batch_set_config: ctas_per_sm must be in [1, 64]");
  if (cfg->steps_per_launch != 1)
    return fail(LBX_ERR_UNSUPPORTED, "lbx_batch_set_config: one step per launch (a step needs all neighbours)");
  if (lbx_status s = build_tiles(b, cfg->block)) return s;
  if (cfg->ctas_per_sm != b->cfg.ctas_per_sm) {
    for (auto& g : b->graphs) cudaGraphExecDestroy(g.second);
    b->graphs.clear();
  }
  b->cfg = *cfg;
  return LBX_OK;
}

// Record `steps` launches (ping-pong from the current buffer) plus the step-counter
// advance into a graph once; later calls with the same length and parity replay it.
static lbx_status graph_for(lbx_batch* b, long long steps, cudaGraphExec_t* exec) {
  const auto key = std::make_pair(steps, b->cur_a ? 1 : 0);
  auto it = b->graphs.find(key);
  if (it != b->graphs.end()) {
    *exec = it->second;
    return LBX_OK;
  }
  cudaGraph_t g = nullptr;
  CK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
  bool a = b->cur_a;
  cudaError_t e = cudaSuccess;
  for (long long r = 0; r < steps && e == cudaSuccess; ++r) {
    e = launch_step(b, a ? b->fa : b->fb, a ? b->fb : b->fa, (int)r);
    a = !a;
  }
  if (e == cudaSuccess) e = launch_advance(b->d_step, steps, b->stream);
  cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
  if (e != cudaSuccess || e2 != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return fail(LBX_ERR_CUDA, "lbx_batch_step: graph capture failed: %s",
                cudaGetErrorString(e != cudaSuccess ? e : e2));
  }
  cudaGraphExec_t ex = nullptr;
  e = cudaGraphInstantiate(&ex, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return fail(LBX_ERR_CUDA, "lbx_batch_step: graph instantiate: %s", cudaGetErrorString(e));
  b->graphs[key] = ex;
  *exec = ex;
  return LBX_OK;
}

extern "C" lbx_status lbx_batch_step(lbx_batch* b, int64_t n) {
  if (!b) return fail(LBX_ERR_ARG, "lbx_batch_step: null batch");
  if (n < 0 || n > (1LL << 30)) return fail(LBX_ERR_ARG, "lbx_batch_step: step count out of range");
  if (n == 0) return LBX_OK;
  if (b->cfg.use_graph) {
    cudaGraphExec_t ex;
    if (lbx_status s = graph_for(b, n, &ex)) return s;
    CK(cudaGraphLaunch(ex, b->stream));
  } else {
    bool a = b->cur_a;
    for (int64_t r = 0; r < n; ++r) {
      cudaError_t e = launch_step(b, a ? b->fa : b->fb, a ? b->fb : b->fa, (int)r);
      if (e != cudaSuccess) return fail(LBX_ERR_CUDA, "lbx_batch_step: %s", cudaGetErrorString(e));
      a = !a;
    }
    CK(launch_advance(b->d_step, n, b->stream));
  }
  if (n & 1) b->cur_a = !b->cur_a;
  b->step += n;
  return LBX_OK;
}

extern "C" lbx_status lbx_batch_synchronize(lbx_batch* b) {
  if (!b) return fail(LBX_ERR_ARG, "lbx_batch_synchronize: null batch");
  CK(cudaStreamSynchronize(b->stream));
  return LBX_OK;
}

extern "C" lbx_status lbx_batch_moments(lbx_batch* b, int j, double* Q_out) {
  if (!b || !Q_out || j < 0 || j >= b->n) return fail(LBX_ERR_ARG, "lbx_batch_moments: bad arguments");
  lbx_state v;
  make_view(b, j, &v);
  const size_t bytes = sizeof(double) * b->K * (size_t)b->sch[j].ncell;
  double* d = nullptr;
  CK(cudaMalloc(&d, bytes));
  cudaError_t e = b->ops.gather(&v, b->at(b->cur(), j), d, nullptr);
  if (!e) e = cudaMemcpyAsync(Q_out, d, bytes, cudaMemcpyDeviceToHost, b->stream);
  if (!e) e = cudaStreamSynchronize(b->stream);
  cudaFree(d);
  CK(e);
  return LBX_OK;
}

// Time one configuration: `trials` launches reading the current buffer and writing the
// other one, without swapping, so the state does not advance.
static lbx_status time_config(lbx_batch* b, int trials, float* ms) {
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  cudaError_t e = cudaSuccess;
  for (int w = 0; w < 2 && e == cudaSuccess; ++w) e = launch_step(b, b->cur(), b->nxt(), 0);
  if (e == cudaSuccess) e = cudaEventRecord(e0, b->stream);
  for (int r = 0; r < trials && e == cudaSuccess; ++r) e = launch_step(b, b->cur(), b->nxt(), 0);
  if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return fail(LBX_ERR_CUDA, "lbx_batch_tune: %s", cudaGetErrorString(e));
  *ms /= trials;
  return LBX_OK;
}

extern "C" lbx_status lbx_batch_tune(lbx_batch* b, int trials, char* report, size_t report_len) {
  if (!b || trials < 1) return fail(LBX_ERR_ARG, "lbx_batch_tune: bad arguments");
  const int blocks[] = {64, 128, 256, 512};
  const int per_sm[] = {2, 4, 8, 16, 32};
  lbx_batch_config best = b->cfg;
  float best_ms = 1e30f;
  std::string rep = "{\"trials\": [";
  bool first = true;
  for (int blk : blocks) {
    int max_active = 0;
    const size_t sm_bytes = b->ops.smem_bytes(blk);
    if (sm_bytes > 48 * 1024)
      cudaFuncSetAttribute(b->ops.batch_fn(), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_bytes);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&max_active, b->ops.batch_fn(), blk, sm_bytes) != cudaSuccess ||
        max_active < 1) {
      cudaGetLastError();
      continue;                                          // this block size cannot be resident
    }
    for (int c : per_sm) {
      if (c > max_active * 2) continue;                  // beyond residency only adds tail waves
      lbx_batch_config cfg{blk, c, 1, b->cfg.use_graph};
      if (lbx_status s = lbx_batch_set_config(b, &cfg)) return s;
      float ms = 0;
      if (lbx_status s = time_config(b, trials, &ms)) return s;
      char buf[160];
      snprintf(buf, sizeof(buf), "%s{\"block\": %d, \"ctas_per_sm\": %d, \"resident\": %d, \"ms\": %.5f}",
               first ? "" : ", ", blk, c, max_active, ms);
      rep += buf;
      first = false;
      if (ms < best_ms) {
        best_ms = ms;
        best = cfg;
      }
    }
  }
  if (lbx_status s = lbx_batch_set_config(b, &best)) return s;
  char buf[200];
  snprintf(buf, sizeof(buf), "], \"best\": {\"block\": %d, \"ctas_per_sm\": %d, \"steps_per_launch\": 1, \"ms\": %.5f}}",
           best.block, best.ctas_per_sm, best_ms);
  rep += buf;
  if (report && report_len > 0) {
    strncpy(report, rep.c_str(), report_len - 1);
    report[report_len - 1] = '\0';
  }
  return LBX_OK;
}

extern "C" void lbx_batch_destroy(lbx_batch* b) {
  if (b) cudaStreamSynchronize(b->stream);
  free_batch(b);
}

extern "C" lbx_status lbx_batch_check_finite(lbx_batch* b, int* finite) {
  if (!b || !finite) return fail(LBX_ERR_ARG, "lbx_batch_check_finite: null argument");
  const void* A = b->cur();
  cudaError_t e = cudaSuccess;
  switch (b->ops.elem_bytes) {
    case 2: k_batch_nonfinite<__half><<<b->n, 256, 0, b->stream>>>((const __half*)A, b->d_eoff, b->d_ecnt, b->d_flags); break;
    case 4: k_batch_nonfinite<float><<<b->n, 256, 0, b->stream>>>((const float*)A, b->d_eoff, b->d_ecnt, b->d_flags); break;
    default: k_batch_nonfinite<double><<<b->n, 256, 0, b->stream>>>((const double*)A, b->d_eoff, b->d_ecnt, b->d_flags);
  }
  e = cudaGetLastError();
  std::vector<int> h(b->n);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), b->d_flags, sizeof(int) * b->n, cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return fail(LBX_ERR_CUDA, "lbx_batch_check_finite: %s", cudaGetErrorString(e));
  for (int j = 0; j < b->n; ++j) finite[j] = h[j] ? 0 : 1;
  return LBX_OK;
}
