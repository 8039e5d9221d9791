// lbx_conserved_sums_static: the conserved-sum reduction of lbx_conserved_sums without
// any device allocation.  Its scratch (per-block partial sums and the reduced result)
// lives in one file-scope __device__ array instead of state-owned cudaMalloc memory.
//
// Who needs it: code that must not call cudaMalloc/cudaFree - a loop being recorded
// into a CUDA graph or running under a latency budget (both calls synchronise the
// device), or a host program whose device memory is entirely owned by another allocator
// (a framework's caching allocator, a hard memory cap) - can still reduce a population
// buffer it holds.
//
// The array is created when the library's module loads on a device and stays resident
// on every device that loaded the library until the process exits.  Host code cannot use
// its name as a device address (that is a host-side stand-in); the device address is
// looked up once per device with cudaGetSymbolAddress, with that device current, by the
// first call made on that device.
#include <cuda_runtime.h>

#include <mutex>

#include "lbx.h"
#include "lbx_internal.h"

using namespace lbx;

namespace {

constexpr int kMaxDevices = 64;
constexpr size_t kPartialDoubles = (size_t)LBX_STATIC_REDUCE_MAX_BLOCKS * KMAX * 4;
constexpr size_t kScratchDoubles = kPartialDoubles + KMAX * 4;
static_assert(kScratchDoubles == (size_t)LBX_STATIC_REDUCE_SCRATCH_DOUBLES,
              "LBX_STATIC_REDUCE_SCRATCH_DOUBLES must follow the largest component count");

// Per-block partials [block][k][4] followed by the reduced result [k][4].
static __device__ __align__(256) double g_reduce_scratch[kScratchDoubles];

std::mutex g_mu;
double* g_scratch_ptr[kMaxDevices] = {};

__global__ void k_pick_sums(const double* __restrict__ out, int K, double* __restrict__ sums) {
  const int k = threadIdx.x;
  if (k < K) sums[k] = out[4 * k];
}

lbx_status scratch_for_current_device(double** ptr) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(LBX_ERR_CUDA, "lbx_conserved_sums_static: cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(LBX_ERR_ARG, "lbx_conserved_sums_static: device %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_mu);
  if (g_scratch_ptr[dev] == nullptr) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_reduce_scratch);
    if (e != cudaSuccess)
      return fail(LBX_ERR_CUDA, "lbx_conserved_sums_static: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *ptr = g_scratch_ptr[dev];
  return LBX_OK;
}

}  // namespace

extern "C" lbx_status lbx_conserved_sums_static(const lbx_scheme* sch, const void* populations, double* sums,
                                                int nblocks, void* stream) {
  if (!sch || !populations || !sums) return fail(LBX_ERR_ARG, "lbx_conserved_sums_static: null argument");
  if (sch->d.precision == LBX_FP16_SCALED)
    return fail(LBX_ERR_UNSUPPORTED,
                "lbx_conserved_sums_static: FP16_SCALED populations need the state's scales; use lbx_conserved_sums");
  const int K = sch->sys.K;
  if (nblocks == 0) {
    int dev = 0, nsm = 148;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return fail(LBX_ERR_CUDA, "lbx_conserved_sums_static: cannot query the device");
    nblocks = 2 * nsm < LBX_STATIC_REDUCE_MAX_BLOCKS ? 2 * nsm : LBX_STATIC_REDUCE_MAX_BLOCKS;
  }
  if (nblocks < 1 || nblocks > LBX_STATIC_REDUCE_MAX_BLOCKS)
    return fail(LBX_ERR_ARG,
                "lbx_conserved_sums_static: nblocks = %d exceeds the static scratch (1..%d blocks, %zu doubles)",
                nblocks, LBX_STATIC_REDUCE_MAX_BLOCKS, kScratchDoubles);
  Ops ops;
  if (!find_ops(sch->sys.family, sch->d.lattice, sch->d.precision, &ops))
    return fail(LBX_ERR_UNSUPPORTED, "lbx_conserved_sums_static: family %d on lattice %d not compiled",
                sch->sys.family, sch->d.lattice);
  double* scratch = nullptr;
  if (lbx_status s = scratch_for_current_device(&scratch)) return s;
  // A host-only description of the buffer: no device memory is attached to it.
  lbx_state view;
  view.sch = *sch;
  view.stream = (cudaStream_t)stream;
  for (int k = 0; k < KMAX; ++k) view.scale[k] = 1.0;
  refresh_params(&view);
  // Every slot read below is written earlier in this call (each block writes all of its
  // partials; the final pass writes every result), so nothing needs clearing.
  double* partials = scratch;
  double* out = scratch + kPartialDoubles;
  cudaError_t e = ops.reduce(&view, populations, nullptr, partials, nblocks, 0);
  if (e != cudaSuccess) return fail(LBX_ERR_CUDA, "lbx_conserved_sums_static: reduce: %s", cudaGetErrorString(e));
  k_reduce_final<<<1, RED_FINAL_THREADS, 0, view.stream>>>(partials, nblocks, K, 0, out);
  k_pick_sums<<<1, 32, 0, view.stream>>>(out, K, sums);
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail(LBX_ERR_CUDA, "lbx_conserved_sums_static: %s", cudaGetErrorString(e));
  return LBX_OK;
}
