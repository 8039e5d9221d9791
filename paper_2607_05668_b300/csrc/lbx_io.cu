// Checkpoint files and the bandwidth / FP64 peak probes used as roofline denominators.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "lbx.h"
#include "lbx_internal.h"

using namespace lbx;

#define CK(call)                                                                                     \
  do {                                                                                               \
    cudaError_t e_ = (call);                                                                         \
    if (e_ != cudaSuccess)                                                                           \
      return fail(e_ == cudaErrorMemoryAllocation ? LBX_ERR_OOM : LBX_ERR_CUDA, "%s: %s", #call,     \
                  cudaGetErrorString(e_));                                                           \
  } while (0)

// ------------------------------------------------------------------ CRC32 and hashing
// CRC-32 (IEEE 802.3, reflected polynomial 0xEDB88320), bitwise table construction.
static unsigned int crc_table[256];
static bool crc_ready = false;
static void crc_init() {
  for (unsigned int n = 0; n < 256; ++n) {
    unsigned int c = n;
    for (int k = 0; k < 8; ++k) c = (c & 1u) ? 0xEDB88320u ^ (c >> 1) : c >> 1;
    crc_table[n] = c;
  }
  crc_ready = true;
}
static unsigned int crc32_update(unsigned int crc, const unsigned char* p, size_t n) {
  if (!crc_ready) crc_init();
  crc = ~crc;
  for (size_t i = 0; i < n; ++i) crc = crc_table[(crc ^ p[i]) & 0xffu] ^ (crc >> 8);
  return ~crc;
}

// FNV-1a 64 over the fields that define the scheme and the storage scales.
static unsigned long long scheme_hash(const lbx_state* st) {
  unsigned long long h = 1469598103934665603ull;
  auto mix = [&](const void* p, size_t n) {
    const unsigned char* b = (const unsigned char*)p;
    for (size_t i = 0; i < n; ++i) {
      h ^= b[i];
      h *= 1099511628211ull;
    }
  };
  const lbx_scheme& s = st->sch;
  mix(&s.sys.family, sizeof(int));
  mix(s.sys.params, sizeof(s.sys.params));
  mix(s.sys.Q0, sizeof(s.sys.Q0));
  mix(&s.d.lattice, sizeof(int));
  mix(&s.nx, sizeof(int));
  mix(&s.ny, sizeof(int));
  mix(&s.nz, sizeof(int));
  mix(&s.d.precision, sizeof(int));
  mix(&s.dt, sizeof(double));
  mix(s.tau, sizeof(double) * s.sys.K);
  return h;
}

struct CkptHeader {
  char magic[8];            // "LBXCKPT1"
  int version;
  int family, lattice, precision;
  int nx, ny, nz, K;
  long long step;
  unsigned long long hash;
  double scale[KMAX];
  unsigned long long payload_bytes;
};

extern "C" lbx_status lbx_save(lbx_state* st, const char* path) {
  if (!st || !path) return fail(LBX_ERR_ARG, "lbx_save: null argument");
  if (lbx_status s = require_standard_layout(st, "lbx_save")) return s;
  const size_t bytes = lbx_state_buffer_bytes(&st->sch);
  std::vector<unsigned char> buf(bytes);
  CK(cudaMemcpyAsync(buf.data(), st->cur(), bytes, cudaMemcpyDeviceToHost, st->stream));
  CK(cudaStreamSynchronize(st->stream));
  CkptHeader h;
  memset(&h, 0, sizeof(h));
  memcpy(h.magic, "LBXCKPT1", 8);
  h.version = lbx_version();
  h.family = st->sch.sys.family;
  h.lattice = st->sch.d.lattice;
  h.precision = st->sch.d.precision;
  h.nx = st->sch.nx;
  h.ny = st->sch.ny;
  h.nz = st->sch.nz;
  h.K = st->sch.sys.K;
  h.step = st->step;
  h.hash = scheme_hash(st);
  for (int k = 0; k < KMAX; ++k) h.scale[k] = st->scale[k];
  h.payload_bytes = bytes;
  unsigned int crc = crc32_update(0, (const unsigned char*)&h, sizeof(h));
  crc = crc32_update(crc, buf.data(), bytes);
  FILE* f = fopen(path, "wb");
  if (!f) return fail(LBX_ERR_IO, "lbx_save: cannot open %s", path);
  bool ok = fwrite(&h, sizeof(h), 1, f) == 1 && fwrite(buf.data(), 1, bytes, f) == bytes &&
            fwrite(&crc, sizeof(crc), 1, f) == 1;
  ok = (fclose(f) == 0) && ok;
  if (!ok) return fail(LBX_ERR_IO, "lbx_save: write to %s failed", path);
  return LBX_OK;
}

extern "C" lbx_status lbx_load(lbx_state* st, const char* path) {
  if (!st || !path) return fail(LBX_ERR_ARG, "lbx_load: null argument");
  FILE* f = fopen(path, "rb");
  if (!f) return fail(LBX_ERR_IO, "lbx_load: cannot open %s", path);
  CkptHeader h;
  const size_t bytes = lbx_state_buffer_bytes(&st->sch);
  std::vector<unsigned char> buf(bytes);
  unsigned int crc_file = 0;
  bool ok = fread(&h, sizeof(h), 1, f) == 1;
  if (ok && memcmp(h.magic, "LBXCKPT1", 8) != 0) {
    fclose(f);
    return fail(LBX_ERR_IO, "lbx_load: %s is not a checkpoint", path);
  }
  if (ok && h.payload_bytes != bytes) {
    fclose(f);
    return fail(LBX_ERR_IO, "lbx_load: payload size %llu does not match this state (%zu)", h.payload_bytes, bytes);
  }
  ok = ok && fread(buf.data(), 1, bytes, f) == bytes && fread(&crc_file, sizeof(crc_file), 1, f) == 1;
  fclose(f);
  if (!ok) return fail(LBX_ERR_IO, "lbx_load: %s is truncated", path);
  unsigned int crc = crc32_update(0, (const unsigned char*)&h, sizeof(h));
  crc = crc32_update(crc, buf.data(), bytes);
  if (crc != crc_file) return fail(LBX_ERR_IO, "lbx_load: CRC mismatch in %s", path);
  // the scales are part of the stored representation: adopt them before comparing hashes
  double saved[KMAX];
  memcpy(saved, st->scale, sizeof(saved));
  memcpy(st->scale, h.scale, sizeof(saved));
  if (h.hash != scheme_hash(st)) {
    memcpy(st->scale, saved, sizeof(saved));
    return fail(LBX_ERR_IO, "lbx_load: checkpoint was written by a different scheme");
  }
  refresh_params(st);
  CK(cudaMemcpyAsync(st->cur(), buf.data(), bytes, cudaMemcpyHostToDevice, st->stream));
  st->step = h.step;
  long long v = h.step;
  CK(cudaMemcpyAsync(st->d_step, &v, sizeof(v), cudaMemcpyHostToDevice, st->stream));
  CK(cudaStreamSynchronize(st->stream));
  st->step_dirty = false;
  st->nonfinite = false;
  st->half = 0;                 // a checkpoint holds the standard layout
  return LBX_OK;
}

// ------------------------------------------------------------------------- peak probes
__global__ void k_copy4(const float4* __restrict__ a, float4* __restrict__ b, size_t n) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) b[i] = __ldg(a + i);
}

// 8 independent FMA chains per thread, `iters` rounds: 16 * iters flops per thread.
template <typename T>
__global__ void k_fma(T* out, int iters, T s) {
  T a[8];
  for (int j = 0; j < 8; ++j) a[j] = T(threadIdx.x + j) * T(1e-3);
  const T m = T(0.999999), c = T(1e-7);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = fma(a[j], m, c);
  }
  T r = 0;
  for (int j = 0; j < 8; ++j) r += a[j];
  if (r == s) out[threadIdx.x] = r;   // practically never true; keeps the chains live
}

extern "C" lbx_status lbx_probe_peaks(size_t bytes, void* stream, double* copy_gbs, double* fp64_gflops,
                                      double* fp32_gflops) {
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, nsm = 148;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  lbx_status rc = LBX_OK;
  if (copy_gbs) {
    const size_t n4 = (bytes / 2) / sizeof(float4);
    float4 *a = nullptr, *b = nullptr;
    if (cudaMalloc(&a, n4 * sizeof(float4)) != cudaSuccess || cudaMalloc(&b, n4 * sizeof(float4)) != cudaSuccess) {
      cudaFree(a);
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      return fail(LBX_ERR_OOM, "lbx_probe_peaks: cannot allocate %zu bytes", bytes);
    }
    cudaMemsetAsync(a, 0, n4 * sizeof(float4), s);
    float best = 1e30f;
    for (int r = 0; r < 6; ++r) {
      cudaEventRecord(e0, s);
      k_copy4<<<nsm * 8, 512, 0, s>>>(a, b, n4);
      cudaEventRecord(e1, s);
      cudaEventSynchronize(e1);
      float ms;
      cudaEventElapsedTime(&ms, e0, e1);
      if (r > 0 && ms < best) best = ms;
    }
    if (cudaGetLastError() != cudaSuccess) rc = fail(LBX_ERR_CUDA, "lbx_probe_peaks: copy probe failed");
    *copy_gbs = 2.0 * n4 * sizeof(float4) / (best * 1e-3) / 1e9;
    cudaFree(a);
    cudaFree(b);
  }
  auto fma_probe = [&](auto zero, double* out) {
    using T = decltype(zero);
    T* o = nullptr;
    cudaMalloc(&o, 1024 * sizeof(T));
    const int iters = sizeof(T) == 8 ? 2048 : 32768;
    const int blocks = nsm * 8, threads = 256;
    float best = 1e30f;
    for (int r = 0; r < 4; ++r) {
      cudaEventRecord(e0, s);
      k_fma<T><<<blocks, threads, 0, s>>>(o, iters, T(-12345));
      cudaEventRecord(e1, s);
      cudaEventSynchronize(e1);
      float ms;
      cudaEventElapsedTime(&ms, e0, e1);
      if (r > 0 && ms < best) best = ms;
    }
    cudaFree(o);
    *out = 16.0 * iters * (double)blocks * threads / (best * 1e-3) / 1e9;
  };
  if (fp64_gflops) fma_probe(0.0, fp64_gflops);
  if (fp32_gflops) fma_probe(0.0f, fp32_gflops);
  if (cudaGetLastError() != cudaSuccess && rc == LBX_OK) rc = fail(LBX_ERR_CUDA, "lbx_probe_peaks: FMA probe failed");
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return rc;
}
