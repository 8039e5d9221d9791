// Launch side of the step kernels: one OpsImpl per (lattice, system family, storage)
// wraps the kernels of kernels.cuh with their launch shapes and fills the function table
// lbx::Ops that a state dispatches through.  Included by the ops_*.cu translation units,
// each of which instantiates the families it names (so the library compiles in parallel).
#pragma once

#include <cuda_runtime.h>

#include <algorithm>

#include "kernels.cuh"
#include "lbx_internal.h"

namespace lbx {

template <class Lat, template <typename> class SysT, class St>
struct OpsImpl {
  using C = typename St::C;
  using S = typename St::S;
  static constexpr int K = SysT<C>::K;
  static constexpr int MODE = StepMode<Lat, SysT, St>::value;
  static constexpr bool REG = MODE == MODE_REG;

  static dim3 block(const lbx_scheme& s) {
    int bx = s.nx >= 128 ? 128 : ((s.nx + 31) / 32) * 32;
    return dim3(bx, 1, 1);
  }
  static dim3 grid(const lbx_scheme& s, dim3 b) { return dim3((s.nx + b.x - 1) / b.x, s.ny, s.nz); }
  // A step launch's blocks along y and z: the state's plane range of the last axis.
  static dim3 step_grid(const lbx_state* st, unsigned int gx) {
    const int n = st->step_planes();
    return Lat::D == 3 ? dim3(gx, st->sch.ny, n) : dim3(gx, n, st->sch.nz);
  }
  static size_t smem(int threads) { return StepMode<Lat, SysT, St, 128>::smem_bytes; }
  // Opt a staged kernel into the shared memory it needs.
  static cudaError_t prepare(const void* fn, size_t bytes) {
    if (MODE != MODE_SMEM) return cudaSuccess;
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  }
  template <int COLS>
  static cudaError_t launch(const lbx_state* st, const void* A, void* B, const KParams<C>& p, cudaStream_t strm) {
    const size_t bytes = StepMode<Lat, SysT, St, COLS>::smem_bytes;
    static cudaError_t prep = prepare((const void*)k_step<Lat, SysT, St, MODE, COLS>, bytes);
    if (prep != cudaSuccess) return prep;
    const dim3 b(COLS, 1, 1), g = step_grid(st, (st->sch.nx + COLS - 1) / COLS);
    k_step<Lat, SysT, St, MODE, COLS><<<g, b, bytes, strm>>>((const S*)A, (S*)B, p);
    return cudaGetLastError();
  }

  // Pipelined per-thread staging: a persistent grid of the resident blocks per SM x SMs.
  template <int COLS>
  static cudaError_t launch_pipe(const lbx_state* st, const void* A, void* B, const KParams<C>& p,
                                 cudaStream_t strm) {
    const size_t bytes = PipeMode<Lat, SysT, St, COLS>::smem_bytes;
    static cudaError_t prep = prepare((const void*)k_step_pipe<Lat, SysT, St, COLS>, bytes);
    if (prep != cudaSuccess) return prep;
    static int per_sm = 0, nsm = 0;
    if (per_sm == 0) {
      int dev = 0;
      cudaError_t e = cudaGetDevice(&dev);
      if (!e) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
      if (!e) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_step_pipe<Lat, SysT, St, COLS>, COLS, bytes);
      if (e != cudaSuccess) return e;
      if (per_sm < 1) per_sm = 1;
    }
    const long long tiles = (long long)((st->sch.nx + COLS - 1) / COLS) * st->sch.ny * st->sch.nz;
    const long long g = std::min<long long>(tiles, (long long)per_sm * nsm);
    k_step_pipe<Lat, SysT, St, COLS><<<(unsigned int)g, COLS, bytes, strm>>>((const S*)A, (S*)B, p);
    return cudaGetLastError();
  }

  template <int COLS>
  static cudaError_t launch_split(const lbx_state* st, const void* A, void* B, const KParams<C>& p,
                                  cudaStream_t strm) {
    const size_t bytes = SplitMode<Lat, SysT, St, COLS>::smem_bytes;
    static cudaError_t prep = prepare((const void*)k_step_split<Lat, SysT, St, COLS>, bytes);
    if (prep != cudaSuccess) return prep;
    const dim3 b(COLS, 1, 1), g = step_grid(st, (st->sch.nx + COLS / 2 - 1) / (COLS / 2));
    k_step_split<Lat, SysT, St, COLS><<<g, b, bytes, strm>>>((const S*)A, (S*)B, p);
    return cudaGetLastError();
  }

  template <int COLS>
  static cudaError_t launch_bulk(const lbx_state* st, const void* A, void* B, const KParams<C>& p,
                                 cudaStream_t strm) {
    const size_t bytes = BulkMode<Lat, SysT, St, COLS>::smem_bytes;
    static cudaError_t prep = prepare((const void*)k_step_bulk<Lat, SysT, St, COLS>, bytes);
    if (prep != cudaSuccess) return prep;
    const dim3 b(COLS, 1, 1), g = step_grid(st, (st->sch.nx + COLS - 1) / COLS);
    k_step_bulk<Lat, SysT, St, COLS><<<g, b, bytes, strm>>>((const S*)A, (S*)B, p);
    return cudaGetLastError();
  }

  // Register-resident kernels use 128-thread blocks (narrower grids: the smallest multiple
  // of 32 covering nx); staged kernels use st->block in {32, 64, 128} and the staging
  // st->staging resolves to.
  // A moving solid's sines of this step's field times, once per float64 step before the
  // step kernel (a launch over a plane range computes them per node instead: its pieces run
  // on two streams).
  static cudaError_t prepare_trig(const lbx_state* st, KParams<C>& p, int rel, cudaStream_t strm) {
    if (sizeof(C) != 8 || p.pf_kind != 2 || st->d_pf_trig == nullptr || st->plane_n > 0) return cudaSuccess;
    C* out = reinterpret_cast<C*>(st->d_pf_trig);
    k_pf_trig<C><<<1, 1, 0, strm>>>(p.step_ptr, rel, p.dt, p.pf_flux_dt, p.pf_src_dt, out);
    p.pf_trig = out;
    return cudaGetLastError();
  }
  static cudaError_t step(const lbx_state* st, const void* A, void* B, int rel, cudaStream_t strm) {
    KParams<C> p = st->pc<C>();
    p.step_rel = rel;
    p.plane0 = st->plane_lo;
    if (cudaError_t e = prepare_trig(st, p, rel, strm)) return e;
    if (p.mms_modes != nullptr) {
      // mode-table forcing: its own instantiation, 128 threads, per-thread staging
      const size_t bytes = StepMode<Lat, SysT, St, 128>::smem_bytes;
      static cudaError_t prep = prepare((const void*)k_step<Lat, SysT, St, MODE, 128, true>, bytes);
      if (prep != cudaSuccess) return prep;
      dim3 b = MODE == MODE_REG ? block(st->sch) : dim3(128, 1, 1), g = step_grid(st, grid(st->sch, b).x);
      k_step<Lat, SysT, St, MODE, 128, true><<<g, b, bytes, strm>>>((const S*)A, (S*)B, p);
      return cudaGetLastError();
    }
    if constexpr (MODE == MODE_REG) {
      dim3 b = block(st->sch), g = step_grid(st, grid(st->sch, b).x);
      k_step<Lat, SysT, St, MODE, 128><<<g, b, 0, strm>>>((const S*)A, (S*)B, p);
      return cudaGetLastError();
    } else {
      const int mode = resolved_staging(st);
      if (mode == LBX_STAGE_BULK) {
        switch (st->block) {
          case 32: return launch_bulk<32>(st, A, B, p, strm);
          case 64: return launch_bulk<64>(st, A, B, p, strm);
          default: return launch_bulk<128>(st, A, B, p, strm);
        }
      }
      if (mode == LBX_STAGE_PIPE) {
        // two columns per thread: the largest block up to st->block whose columns fit
        constexpr size_t cap = 227 * 1024;
        if (st->block >= 128 && PipeMode<Lat, SysT, St, 128>::smem_bytes <= cap) return launch_pipe<128>(st, A, B, p, strm);
        if (st->block >= 64 && PipeMode<Lat, SysT, St, 64>::smem_bytes <= cap) return launch_pipe<64>(st, A, B, p, strm);
        return launch_pipe<32>(st, A, B, p, strm);
      }
      if (mode == LBX_STAGE_LANES2) {
        switch (st->block) {
          case 32: return launch_split<32>(st, A, B, p, strm);
          case 64: return launch_split<64>(st, A, B, p, strm);
          default: return launch_split<128>(st, A, B, p, strm);
        }
      }
      switch (st->block) {
        case 32: return launch<32>(st, A, B, p, strm);
        case 64: return launch<64>(st, A, B, p, strm);
        default: return launch<128>(st, A, B, p, strm);
      }
    }
  }
  static cudaError_t init(const lbx_state* st, const double* Q, void* A, unsigned long long* maxbits, int write,
                          unsigned long long* chk) {
    dim3 b = block(st->sch), g = grid(st->sch, b);
    k_init<Lat, SysT, St><<<g, b, 0, st->stream>>>(Q, (S*)A, st->pd, st->d_feq0, maxbits, write, 0, chk);
    return cudaGetLastError();
  }
  static cudaError_t gather(const lbx_state* st, const void* A, double* Qout, double* fout) {
    dim3 b = block(st->sch), g = grid(st->sch, b);
    k_gather<Lat, SysT, St><<<g, b, 0, st->stream>>>((const S*)A, st->pd, st->d_feq0, Qout, fout, 0);
    return cudaGetLastError();
  }
  // The same for the planes plane0 .. plane0 + nplanes - 1 of the last axis (pipelined
  // host copies: lbx_init and lbx_moments with host arrays).
  static dim3 plane_grid(const lbx_scheme& s, dim3 b, int nplanes) {
    return dim3((s.nx + b.x - 1) / b.x, Lat::D == 3 ? s.ny : nplanes, Lat::D == 3 ? nplanes : 1);
  }
  static cudaError_t init_planes(const lbx_state* st, const double* Q, void* A, int plane0, int nplanes,
                                 unsigned long long* chk) {
    dim3 b = block(st->sch), g = plane_grid(st->sch, b, nplanes);
    k_init<Lat, SysT, St><<<g, b, 0, st->stream>>>(Q, (S*)A, st->pd, st->d_feq0, nullptr, 1, plane0, chk);
    return cudaGetLastError();
  }
  static cudaError_t gather_planes(const lbx_state* st, const void* A, double* Qout, int plane0, int nplanes) {
    dim3 b = block(st->sch), g = plane_grid(st->sch, b, nplanes);
    k_gather<Lat, SysT, St><<<g, b, 0, st->stream>>>((const S*)A, st->pd, st->d_feq0, Qout, nullptr, plane0);
    return cudaGetLastError();
  }
  static cudaError_t scatter(const lbx_state* st, const double* fin, void* A) {
    dim3 b = block(st->sch), g = grid(st->sch, b);
    k_scatter<Lat, SysT, St><<<g, b, 0, st->stream>>>(fin, (S*)A, st->pd, st->d_feq0);
    return cudaGetLastError();
  }
  static cudaError_t reduce(const lbx_state* st, const void* A, const double* Qref, double* partials,
                            int nblk, int mode) {
    k_reduce<Lat, SysT, St><<<nblk, RED_THREADS, 0, st->stream>>>((const S*)A, st->pd, Qref, partials, mode);
    return cudaGetLastError();
  }
  static const void* step_fn() { return (const void*)k_step<Lat, SysT, St, MODE, 128>; }
  static cudaError_t batch_step(const void* A, void* B, const void* insts, const int2* tiles, int ntiles, int fourier,
                                const long long* step_ptr, int step_rel, int grid, int block, cudaStream_t strm) {
    if (fourier) {
      if (MODE == MODE_SMEM) {
        cudaError_t prep = prepare((const void*)k_step_batch<Lat, SysT, St, MODE, true>, smem(block));
        if (prep != cudaSuccess) return prep;
      }
      k_step_batch<Lat, SysT, St, MODE, true><<<grid, block, smem(block), strm>>>(
          (const S*)A, (S*)B, (const BatchInst<C>*)insts, tiles, ntiles, step_ptr, step_rel);
      return cudaGetLastError();
    }
    if (MODE == MODE_SMEM) {
      cudaError_t prep = prepare((const void*)k_step_batch<Lat, SysT, St, MODE>, smem(block));
      if (prep != cudaSuccess) return prep;
    }
    k_step_batch<Lat, SysT, St, MODE><<<grid, block, smem(block), strm>>>(
        (const S*)A, (S*)B, (const BatchInst<C>*)insts, tiles, ntiles, step_ptr, step_rel);
    return cudaGetLastError();
  }
  static const void* batch_fn() { return (const void*)k_step_batch<Lat, SysT, St, MODE>; }

  // In-place steps: 128-thread blocks, per-thread staging for staged systems.
  template <bool FOURIER, int KIND>
  static cudaError_t launch_inplace(const lbx_state* st, void* F, const KParams<C>& p, cudaStream_t strm) {
    const size_t bytes = StepMode<Lat, SysT, St, 128>::smem_bytes;
    static cudaError_t prep = prepare((const void*)k_step_inplace<Lat, SysT, St, MODE, 128, FOURIER, KIND>, bytes);
    if (prep != cudaSuccess) return prep;
    dim3 b = MODE == MODE_REG ? block(st->sch) : dim3(128, 1, 1), g = grid(st->sch, b);
    k_step_inplace<Lat, SysT, St, MODE, 128, FOURIER, KIND><<<g, b, bytes, strm>>>((S*)F, p);
    return cudaGetLastError();
  }
  template <int COLS, int KIND>
  static cudaError_t launch_bulk_inplace(const lbx_state* st, void* F, const KParams<C>& p, cudaStream_t strm) {
    const size_t bytes = BulkMode<Lat, SysT, St, COLS>::smem_bytes;
    static cudaError_t prep = prepare((const void*)k_step_bulk_inplace<Lat, SysT, St, COLS, KIND>, bytes);
    if (prep != cudaSuccess) return prep;
    const dim3 b(COLS, 1, 1), g((st->sch.nx + COLS - 1) / COLS, st->sch.ny, st->sch.nz);
    k_step_bulk_inplace<Lat, SysT, St, COLS, KIND><<<g, b, bytes, strm>>>((S*)F, p);
    return cudaGetLastError();
  }
  template <int KIND>
  static cudaError_t bulk_inplace(const lbx_state* st, void* F, const KParams<C>& p, cudaStream_t strm) {
    switch (st->block) {
      case 32: return launch_bulk_inplace<32, KIND>(st, F, p, strm);
      case 64: return launch_bulk_inplace<64, KIND>(st, F, p, strm);
      default: return launch_bulk_inplace<128, KIND>(st, F, p, strm);
    }
  }
  // Staged systems use bulk row copies where the staging resolves to them (st->block wide),
  // otherwise per-thread copies in 128-thread blocks; forced runs take the latter.
  static cudaError_t step_inplace(const lbx_state* st, void* F, int kind, int rel, cudaStream_t strm) {
    KParams<C> p = st->pc<C>();
    p.step_rel = rel;
    if (cudaError_t e = prepare_trig(st, p, rel, strm)) return e;
    if (p.mms_modes != nullptr)
      return kind == 1 ? launch_inplace<true, 1>(st, F, p, strm) : launch_inplace<true, 2>(st, F, p, strm);
    if constexpr (MODE == MODE_SMEM) {
      if (resolved_staging(st) == LBX_STAGE_BULK)
        return kind == 1 ? bulk_inplace<1>(st, F, p, strm) : bulk_inplace<2>(st, F, p, strm);
    }
    return kind == 1 ? launch_inplace<false, 1>(st, F, p, strm) : launch_inplace<false, 2>(st, F, p, strm);
  }
  // Slab faces (k_face): one thread per plane cell, face velocity and face.
  static cudaError_t face(const lbx_state* st, void* A, void* up, void* dn, int pack, cudaStream_t strm) {
    const lbx_scheme& s = st->sch;
    const unsigned int pc = Lat::D == 3 ? (unsigned int)(s.nx * s.ny) : (unsigned int)s.nx;
    const dim3 b(128, 1, 1), g((pc + 127) / 128, FaceVel<Lat>::NF, 2);
    if (pack)
      k_face<Lat, SysT, St, true><<<g, b, 0, strm>>>((S*)A, (S*)up, (S*)dn, st->pc<C>());
    else
      k_face<Lat, SysT, St, false><<<g, b, 0, strm>>>((S*)A, (S*)up, (S*)dn, st->pc<C>());
    return cudaGetLastError();
  }
  // staged kernels keep a fixed 128-column layout: larger blocks cannot launch
  static size_t smem_bytes(int threads) { return (MODE == MODE_SMEM && threads > 128) ? (size_t)1 << 30 : smem(threads); }
};

template <class Lat, template <typename> class SysT, class St>
inline Ops make_ops() {
  using I = OpsImpl<Lat, SysT, St>;
  return Ops{I::step,       I::init,     I::gather,
             I::scatter,    I::reduce,   I::step_fn,
             I::REG,        I::batch_step, I::batch_fn, I::smem_bytes,
             sizeof(BatchInst<typename St::C>), sizeof(typename St::S), I::step_inplace,
             I::face, FaceVel<Lat>::NF, I::init_planes, I::gather_planes};
}

template <class Lat, template <typename> class SysT>
inline bool pick_store(int precision, Ops* o) {
  switch (precision) {
    case LBX_FP64: *o = make_ops<Lat, SysT, StoreF64>(); return true;
    case LBX_FP32_SHIFT: *o = make_ops<Lat, SysT, StoreF32>(); return true;
    case LBX_FP16_SCALED: *o = make_ops<Lat, SysT, StoreF16>(); return true;
  }
  return false;
}

}  // namespace lbx
