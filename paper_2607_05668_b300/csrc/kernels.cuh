// Device kernels of the kinetic relaxation scheme (sm_103a).
//
// Storage: structure of arrays over (velocity i, node), with components interleaved in
// pairs: component k < 2 floor(K/2) of velocity i at node `cell` is element
// ((floor(k/2) q + i) ncell + cell) 2 + (k mod 2), and an odd last component has its own
// plane after the pairs (element 2 floor(K/2) q ncell + i ncell + cell); cell =
// (z ny + y) nx + x.  A warp's access to one velocity is still one contiguous run, and
// every load or store moves two components (one 2x16-bit, 2x32-bit or 2x64-bit vector).  The buffer holds
// post-collision populations of the previous step at the node they left, so the step
// kernel PULLS f_{k,i}(x, t) = A[k][i][x - c_i] (periodic), collides at x and writes
// B[k][i][x]: every store is coalesced and every load is a unit-stride run shifted by
// at most one node (Eq. lbe_update read from the arrival side).
//
// One thread owns one node.  A warp issues one 32-wide coalesced access per population
// plane (128 B for float32), and all K*q loads of a node are independent, so each
// thread keeps K*q loads in flight; that memory-level parallelism is what saturates HBM
// at moderate occupancy.  With REG the populations stay in registers between the
// moment pass and the write pass; without it (large K*q) they are re-read with
// ld.global.nc, which the first pass has just pulled into L1/L2, so DRAM sees each
// population once.
#pragma once

#include <cuda_fp16.h>
#include <stdint.h>

#include "dual.cuh"
#include "lattices.cuh"
#include "systems.cuh"


namespace lbx {

// Largest mode table (LBX_MMS_MAX_MODES; the host checks that the two agree).
constexpr int MMS_MAX_MODES = 64;

// One manufactured mode on the device (lbx_mms_mode with 2 pi k precomputed).
struct MmsMode {
  double k2pi[3];
  double amp, phase, sigma, omega, psi;
  int p, pad_;
};

template <typename T>
struct KParams {
  int nx, ny, nz, pad_;
  int oy, oz;                  // slab origin: global index of local row 0 (2D) or plane 0 (3D)
  int plane0;                  // first plane of the last axis a step launch covers (0: all)
  long long ncell;             // nodes per population plane
  T Q0[KMAX];                  // background state (shift reference)
  T F0l[KMAX][3];              // (dt/dx)/c_s^2 * Phi(Q0), used by the unshifted mode
  T omega[KMAX];               // 1 / tau_LB per component
  T omc[KMAX];                 // 1 - 1 / tau_LB (the float64 update)
  T ow[KMAX][3];               // omega_k w_i by weight class |c_i|^2 = 0, 1, 2 (float64 update)
  T tau[KMAX];                 // tau_LB per component
  T scale[KMAX];               // float16 storage scale s_k (1 otherwise)
  T inv_scale[KMAX];
  T prm[NPRM];                 // system parameters (layout per system)
  T lc;                        // (dt/dx) / c_s^2
  T dt;                        // source factor
  const T* mms_tab;            // ADR forcing tables sx[nx] cx[nx] sy[ny] cy[ny]; null = off
  T mms_c0, mms_cx, mms_cy;    // A(-1 + 8 pi^2 nu), 2 pi A a_x, 2 pi A a_y
  const long long* step_ptr;   // step index at the start of this launch sequence
  int step_rel;                // offset of this launch in the sequence
  unsigned int* err;           // device error word: bit 0 = a bounded wait timed out
  unsigned long long wait_ns;  // limit of a bounded wait for bulk copies (global-timer ns)
  T dx;                        // node spacing (coordinates of the manufactured fields)
  const MmsMode* mms_modes;    // FOURIER forcing table; null = off
  int mms_n;
  int mms_trackers;            // nonzero: the tracker components are forced as well
  T mms_mean[8];               // mean of each primitive
  int pf_kind;                 // prescribed coefficient fields (HCNSF): 0 none, 1 uniform, 2 advected
  T pf[8];                     // their parameters (see prescribed_fields)
  T pf_src_dt, pf_flux_dt;     // time offsets of the fields inside the source and the flux
  const T* pf_trig;            // advected solid: sin, cos of the field times of this step (flux,
                               // then source; k_pf_trig), or null: computed per node
  const T* pf_tab;             // advected solid, float64: sin, cos of 2 pi x_d per node index
                               // along each axis, [sx nx][cx nx][sy ny][cy ny][sz nz][cz nz];
                               // null = computed
};

// Whether the step reads the step index: manufactured forcing or time-dependent prescribed
// coefficient fields.
template <typename T>
__host__ __device__ __forceinline__ bool time_dependent(const KParams<T>& p) {
  return p.mms_tab != nullptr || p.mms_modes != nullptr || p.pf_kind == 2;
}

// Node rows of a step block: the block's y and z indices, the last axis offset by plane0
// (a launch over a range of planes of that axis).
template <class Lat, typename T>
__device__ __forceinline__ int block_y(const KParams<T>& p) {
  return (int)blockIdx.y + (Lat::D == 2 ? p.plane0 : 0);
}
template <class Lat, typename T>
__device__ __forceinline__ int block_z(const KParams<T>& p) {
  return (int)blockIdx.z + (Lat::D == 3 ? p.plane0 : 0);
}

// Element index of population (k, i) at `cell` (see the storage layout above).
template <int K, int Q>
__host__ __device__ __forceinline__ unsigned int eidx(int k, int i, unsigned int cell, unsigned int plane) {
  constexpr int KP = K / 2;
  if (k < 2 * KP) return (((unsigned int)((k >> 1) * Q + i)) * plane + cell) * 2u + (unsigned int)(k & 1);
  return 2u * (unsigned int)(KP * Q) * plane + (unsigned int)i * plane + cell;
}

// ----------------------------------------------------------------------------- storage
struct StoreF64 {
  using S = double;
  using C = double;
  static constexpr bool SHIFT = false, SCALE = false;
  static constexpr int ID = 1;
};
struct StoreF32 {
  using S = float;
  using C = float;
  static constexpr bool SHIFT = true, SCALE = false;
  static constexpr int ID = 2;
};
struct StoreF16 {
  using S = __half;
  using C = float;
  static constexpr bool SHIFT = true, SCALE = true;
  static constexpr int ID = 3;
};

__device__ __forceinline__ double ld_nc(const double* p) { return __ldg(p); }
__device__ __forceinline__ float ld_nc(const float* p) { return __ldg(p); }
__device__ __forceinline__ float ld_nc(const __half* p) { return __half2float(__ldg(p)); }

// Re-read that the compiler may not merge with the first read (asm volatile).
__device__ __forceinline__ double ld_again(const double* p) {
  double v;
  asm volatile("ld.global.nc.f64 %0, [%1];" : "=d"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ float ld_again(const float* p) {
  float v;
  asm volatile("ld.global.nc.f32 %0, [%1];" : "=f"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ float ld_again(const __half* p) {
  unsigned short v;
  asm volatile("ld.global.nc.b16 %0, [%1];" : "=h"(v) : "l"(p));
  return __half2float(__ushort_as_half(v));
}

__device__ __forceinline__ void store_f64(double* p, double v) { *p = v; }
__device__ __forceinline__ void store_f64(float* p, double v) { *p = (float)v; }
__device__ __forceinline__ void store_f64(__half* p, double v) { *p = __double2half(v); }
// The same, returning whether the stored value is finite (float16 storage overflows to inf).
__device__ __forceinline__ bool store_f64_finite(double* p, double v) {
  *p = v;
  return isfinite(v);
}
__device__ __forceinline__ bool store_f64_finite(float* p, double v) {
  const float f = (float)v;
  *p = f;
  return isfinite(f);
}
__device__ __forceinline__ bool store_f64_finite(__half* p, double v) {
  const __half h = __double2half(v);
  *p = h;
  return !__hisinf(h) && !__hisnan(h);
}

__device__ __forceinline__ void st_out(double* p, double v) { *p = v; }
__device__ __forceinline__ void st_out(float* p, float v) { *p = v; }
__device__ __forceinline__ void st_out(__half* p, float v) { *p = __float2half_rn(v); }

// Source node of the pull along c: x - c with periodic wrap; index c + 1.
struct PullIdx {
  int sx[3], sy[3], sz[3];
  __device__ __forceinline__ PullIdx(int x, int y, int z, int nx, int ny, int nz) {
    sx[0] = x == nx - 1 ? 0 : x + 1; sx[1] = x; sx[2] = x == 0 ? nx - 1 : x - 1;
    sy[0] = y == ny - 1 ? 0 : y + 1; sy[1] = y; sy[2] = y == 0 ? ny - 1 : y - 1;
    sz[0] = z == nz - 1 ? 0 : z + 1; sz[1] = z; sz[2] = z == 0 ? nz - 1 : z - 1;
  }
  template <class Lat>
  __device__ __forceinline__ unsigned int src(int i, int nx, int ny) const {
    return ((unsigned int)sz[Lat::c(i, 2) + 1] * (unsigned int)ny + (unsigned int)sy[Lat::c(i, 1) + 1]) *
               (unsigned int)nx + (unsigned int)sx[Lat::c(i, 0) + 1];
  }
};

// ADR manufactured forcing S_MMS(x, t + dt/2) for u_ex = 1 + A sin(2pi x)cos(2pi y)e^-t:
// e^{-t}[A(-1 + 8 pi^2 nu) s_x c_y + 2 pi A (a_x c_x c_y - a_y s_x s_y)].
template <typename T>
__device__ __forceinline__ T adr_mms(const KParams<T>& p, int x, int y, long long step) {
  const T th = (T(step) + T(0.5)) * p.dt;
  const T e = exp(-th);
  const T* tb = p.mms_tab;
  const T sxv = tb[x], cxv = tb[p.nx + x], syv = tb[2 * p.nx + y], cyv = tb[2 * p.nx + p.ny + y];
  return e * (p.mms_c0 * sxv * cyv + p.mms_cx * cxv * cyv - p.mms_cy * sxv * syv);
}

// Prescribed coefficient fields of the homogenized NSF family (Sec. 3, HCNSF; supplement,
// HCNSF MMS) at coordinates x and time t: cf = (alpha, u_s,x, u_s,y, u_s,z).
//   kind 0  pure fluid: alpha = 1, u_s = 0;
//   kind 1  uniform: alpha = pf[0], u_s = (pf[1], pf[2], pf[3]);
//   kind 2  advected solid: with s_d = sin(2 pi x_d), c_d = cos(2 pi x_d), rotation pattern
//           r = rot (s0 c1 c2, -c0 s1 c2, c0 c1 s2), translation c = pf[4..6], oscillation osc:
//             u_s = (r_0 cos t + c_0 + osc sin t c2, r_1 cos t + c_1 + osc cos t c0,
//                    r_2 sin t + c_2 + osc sin t c1),
//             alpha = a_mean + a_amp [z0 + z1 + z2 + 2 z0 z1 z2], z_d = sin(2 pi xi_d),
//             xi = x - d, d = r sin t + c t  (the solid displacement);
//           pf = (a_mean, a_amp, rot, osc, c_0, c_1, c_2).
// Generic in the coordinate type: dual coordinates give the fields' spatial derivative
// (the manufactured forcing differentiates the flux through alpha).
template <typename T>
__device__ __forceinline__ void sc_pi(T a, T* s, T* c) { sincospi(a, s, c); }
template <typename T>
__device__ __forceinline__ void sc_pi(Dual<T> a, Dual<T>* s, Dual<T>* c) { sincospi_dual(a, s, c); }
// sin(pi a) alone where the cosine is not needed (dual numbers need both for the derivative)
__device__ __forceinline__ double s_pi(double a) { return sinpi(a); }
__device__ __forceinline__ float s_pi(float a) { return sinpif(a); }
template <typename T>
__device__ __forceinline__ Dual<T> s_pi(Dual<T> a) {
  Dual<T> s, c;
  sincospi_dual(a, &s, &c);
  return s;
}

// The time-independent part of the advected-solid fields at x: s_d, c_d and the rotation
// pattern r (kind 2).
template <typename U>
struct SolidAt {
  U s[3], c[3], r[3];
};
template <typename T, typename U>
__device__ __forceinline__ SolidAt<U> solid_at(const KParams<T>& p, const U (&x)[3]) {
  SolidAt<U> a;
#pragma unroll
  for (int d = 0; d < 3; ++d) sc_pi(U(T(2)) * x[d], &a.s[d], &a.c[d]);
  const T rot = p.pf[2];
  a.r[0] = U(rot) * a.s[0] * a.c[1] * a.c[2];
  a.r[1] = U(-rot) * a.c[0] * a.s[1] * a.c[2];
  a.r[2] = U(rot) * a.c[0] * a.c[1] * a.s[2];
  return a;
}
// The same from the host's per-axis tables of sin(2 pi x_d) and cos(2 pi x_d) (global node
// coordinates of a slab included): two loads per axis instead of a sincospi.
template <typename T>
__device__ __forceinline__ SolidAt<T> solid_at_tab(const KParams<T>& p, int x, int y, int z) {
  SolidAt<T> a;
  const T* tb = p.pf_tab;
  const int nx = p.nx, ny = p.ny;
  a.s[0] = tb[x];
  a.c[0] = tb[nx + x];
  a.s[1] = tb[2 * nx + y];
  a.c[1] = tb[2 * nx + ny + y];
  a.s[2] = tb[2 * nx + 2 * ny + z];
  a.c[2] = tb[2 * nx + 2 * ny + p.nz + z];
  const T rot = p.pf[2];
  a.r[0] = rot * a.s[0] * a.c[1] * a.c[2];
  a.r[1] = -rot * a.c[0] * a.s[1] * a.c[2];
  a.r[2] = rot * a.c[0] * a.c[1] * a.s[2];
  return a;
}

// The node's time-independent part: from the tables in float64 (the FP64 pipe bounds that
// kernel, and the tables save three sincospi per node), computed in float32, where the two
// table loads per axis measured slower than the sincospi.
template <typename T>
__device__ __forceinline__ SolidAt<T> solid_here(const KParams<T>& p, int x, int y, int z, const T (&xc)[3]) {
  if constexpr (sizeof(T) == 8) {
    if (p.pf_tab != nullptr) return solid_at_tab(p, x, y, z);
  }
  return solid_at(p, xc);
}

// The fields at time t (st, ct = sin t, cos t) from the node's time-independent part.
template <typename T, typename U>
__device__ __forceinline__ void solid_fields(const KParams<T>& p, const U (&x)[3], const SolidAt<U>& a, T t, T st,
                                             T ct, U (&cf)[4]) {
  const T osc = p.pf[3];
  cf[1] = a.r[0] * U(ct) + U(p.pf[4]) + U(osc * st) * a.c[2];
  cf[2] = a.r[1] * U(ct) + U(p.pf[5]) + U(osc * ct) * a.c[0];
  cf[3] = a.r[2] * U(st) + U(p.pf[6]) + U(osc * st) * a.c[1];
  U z[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) z[d] = s_pi(U(T(2)) * (x[d] - a.r[d] * U(st) - U(p.pf[4 + d] * t)));
  cf[0] = U(p.pf[0]) + U(p.pf[1]) * (z[0] + z[1] + z[2] + U(T(2)) * z[0] * z[1] * z[2]);
}
template <typename T, typename U>
__device__ __forceinline__ void prescribed_fields(const KParams<T>& p, const U (&x)[3], T t, U (&cf)[4]) {
  if (p.pf_kind == 1) {
    for (int a = 0; a < 4; ++a) cf[a] = U(p.pf[a]);
    return;
  }
  if (p.pf_kind != 2) {
    cf[0] = U(T(1));
    cf[1] = cf[2] = cf[3] = U(T(0));
    return;
  }
  T st, ct;
  sincos(t, &st, &ct);
  solid_fields(p, x, solid_at(p, x), t, st, ct, cf);
}

// Time of the prescribed fields inside the flux or the source of a float64 step: t_n + offset
// with t_n = step dt, each rounded on its own (no contraction), so that the step kernels and
// k_pf_trig, which precomputes the sines once per step, agree to the bit.
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
// The table serves the float64 step (two sincos per node on the FP64 pipe: 4.5 % of the
// HCNSF FP64 step); in float32 the per-node sincos measured as fast as the table and its
// extra launch, so the float32 steps keep their own expression t + offset.
template <typename T>
__device__ __forceinline__ T field_time(T t, T off) {
  if constexpr (sizeof(T) == 8) return add_rn(t, off);
  return t + off;
}
template <typename T>
__device__ __forceinline__ void field_sincos(const KParams<T>& p, T tl, int level, T& st, T& ct) {
  if constexpr (sizeof(T) == 8) {
    if (p.pf_trig != nullptr) {
      st = p.pf_trig[2 * level];
      ct = p.pf_trig[2 * level + 1];
      return;
    }
  }
  sincos(tl, &st, &ct);
}

// sin and cos of the advected solid's flux and source times of step *step_ptr + rel (one
// thread; launched before each step kernel of a state with a moving solid).
template <typename T>
__global__ void k_pf_trig(const long long* __restrict__ step_ptr, int rel, T dt, T off_flux, T off_src,
                          T* __restrict__ out) {
  const T t = mul_rn(T(*step_ptr + rel), dt);
  sincos(add_rn(t, off_flux), &out[0], &out[1]);
  sincos(add_rn(t, off_src), &out[2], &out[3]);
}

// Flux and source at a node at state time t (the family's eval()), with the prescribed
// coefficient fields at the node for families that have them.
template <template <typename> class SysT, typename T>
__device__ __forceinline__ void eval_node(const KParams<T>& p, int x, int y, int z, T t, const T* dQ,
                                          T (&Phi)[SysT<T>::K][SysT<T>::D], T (&Src)[SysT<T>::K]) {
  using Sys = SysT<T>;
  if constexpr (NcfOf<Sys>::value > 0) {
    const T xc[3] = {T(x) * p.dx, T(y + p.oy) * p.dx, T(z + p.oz) * p.dx};
    T cf[NcfOf<Sys>::value];
    if (p.pf_kind == 2) {
      // a moving solid: the spatial factors are shared by the two time levels
      const SolidAt<T> a = solid_here(p, x, y, z, xc);
      const T tf = field_time(t, p.pf_flux_dt);
      T sf, cfl;
      field_sincos(p, tf, 0, sf, cfl);
      solid_fields(p, xc, a, tf, sf, cfl, cf);
      if (p.pf_src_dt != p.pf_flux_dt) {
        const T ts = field_time(t, p.pf_src_dt);
        T ss, csl;
        field_sincos(p, ts, 1, ss, csl);
        T cs[NcfOf<Sys>::value];
        solid_fields(p, xc, a, ts, ss, csl, cs);
        Sys::eval(p.prm, p.Q0, dQ, Phi, Src, cf, cs);
      } else {
        Sys::eval(p.prm, p.Q0, dQ, Phi, Src, cf, cf);
      }
    } else {
      prescribed_fields(p, xc, t + p.pf_flux_dt, cf);
      Sys::eval(p.prm, p.Q0, dQ, Phi, Src, cf, cf);
    }
  } else {
    Sys::eval(p.prm, p.Q0, dQ, Phi, Src);
  }
}

// Time factor of a mode at t: g = exp(sigma t) cos(omega t + psi) and its derivative.
template <typename T>
__device__ __forceinline__ void mms_time_factor(const MmsMode& md, T t, T& g, T& gt) {
  T st, ct;
  sincos(T(md.omega) * t + T(md.psi), &st, &ct);
  const T e = exp(T(md.sigma) * t);
  g = e * ct;
  gt = T(md.sigma) * g - T(md.omega) * e * st;
}

// The time factors of every mode at t + dt/2 of `step`, computed once per block into shared
// memory (all threads of a block take the same step); ends with a block barrier.
template <typename T>
__device__ __forceinline__ void mms_time_table(const KParams<T>& p, long long step, T* tf) {
  const T t = (T(step) + T(0.5)) * p.dt;
  if (p.mms_modes != nullptr)
    for (int m = (int)threadIdx.x; m < p.mms_n; m += (int)blockDim.x) mms_time_factor(p.mms_modes[m], t, tf[2 * m], tf[2 * m + 1]);
  __syncthreads();
}

// Manufactured forcing of a FOURIER table (Sec. 4): S_MMS = d_t Q_ex + div Phi(Q_ex) - S(Q_ex)
// at (x, t + dt/2), added to the conserved components of Src.  Every primitive is
// mean + sum amp sin(theta) g(t), theta = 2 pi k.x + phase, g = exp(sigma t) cos(omega t + psi),
// so its value, time derivative, gradient and Hessian follow in closed form from one sin/cos
// of theta and of the time phase per mode.  The exact augmented state (Sys::augment) is then
// formed with dual numbers that carry d/dt once and d/dx_b once per direction b (the trackers'
// derivative along b comes from the Hessian), and the flux of each direction-b state gives
// d Phi_k,b / dx_b from the same delta-form system code the step uses.  Kept out of line: it
// runs only in forced verification runs and must not cost the step kernels registers.
template <class Lat, template <typename> class SysT, typename T>
__device__ __noinline__ void mms_fourier(const KParams<T>& p, int x, int y, int z, long long step,
                                         T* __restrict__ Src, const T* __restrict__ tfac) {
  using D1 = Dual<T>;
  using SysD = SysT<D1>;
  constexpr int K = SysD::K, NC = SysD::NC, NP = SysD::NPRIM, D = Lat::D;
  const T t = (T(step) + T(0.5)) * p.dt;
  const T xc[3] = {T(x) * p.dx, T(y + p.oy) * p.dx, T(z + p.oz) * p.dx};
  T V[NP], Vt[NP], G[NP][3], Gt[NP][3], H[NP][3][3];
#pragma unroll
  for (int q = 0; q < NP; ++q) {
    V[q] = p.mms_mean[q];
    Vt[q] = T(0);
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      G[q][b] = T(0);
      Gt[q][b] = T(0);
#pragma unroll
      for (int c = 0; c < 3; ++c) H[q][b][c] = T(0);
    }
  }
  for (int m = 0; m < p.mms_n; ++m) {
    const MmsMode& md = p.mms_modes[m];
    const T k[3] = {T(md.k2pi[0]), T(md.k2pi[1]), T(md.k2pi[2])};
    T th = T(md.phase);
#pragma unroll
    for (int d = 0; d < D; ++d) th += k[d] * xc[d];
    T sn, cs, g, gt;
    sincos(th, &sn, &cs);
    if (tfac != nullptr) {
      g = tfac[2 * m];
      gt = tfac[2 * m + 1];
    } else {
      mms_time_factor(md, t, g, gt);
    }
    const T a = T(md.amp);
#pragma unroll
    for (int q = 0; q < NP; ++q) {
      if (q != md.p) continue;
      V[q] += a * sn * g;
      Vt[q] += a * sn * gt;
#pragma unroll
      for (int b = 0; b < D; ++b) {
        G[q][b] += a * cs * k[b] * g;
        Gt[q][b] += a * cs * k[b] * gt;
#pragma unroll
        for (int c = 0; c < D; ++c) H[q][b][c] -= a * sn * k[b] * k[c] * g;
      }
    }
  }
  D1 pd[NPRM], q0[K];
#pragma unroll
  for (int i = 0; i < NPRM; ++i) pd[i] = D1(p.prm[i], T(0));
#pragma unroll
  for (int k2 = 0; k2 < K; ++k2) q0[k2] = D1(p.Q0[k2], T(0));
  D1 Vd[NP], Gd[NP][3], Qd[K];
  // d/dt of the exact augmented state
#pragma unroll
  for (int q = 0; q < NP; ++q) {
    Vd[q] = D1(V[q], Vt[q]);
#pragma unroll
    for (int b = 0; b < 3; ++b) Gd[q][b] = D1(G[q][b], Gt[q][b]);
  }
  SysD::augment(pd, Vd, Gd, Qd);
  T acc[K];
#pragma unroll
  for (int k2 = 0; k2 < K; ++k2) acc[k2] = Qd[k2].d;
  // divergence of the flux and the state source
#pragma unroll 1
  for (int b = 0; b < D; ++b) {
#pragma unroll
    for (int q = 0; q < NP; ++q) {
      Vd[q] = D1(V[q], G[q][b]);
#pragma unroll
      for (int c = 0; c < 3; ++c) Gd[q][c] = D1(G[q][c], H[q][b][c]);
    }
    SysD::augment(pd, Vd, Gd, Qd);
    D1 dQd[K], Phi[K][D], S[K];
#pragma unroll
    for (int k2 = 0; k2 < K; ++k2) dQd[k2] = Qd[k2] - q0[k2];
    if constexpr (NcfOf<SysD>::value > 0) {
      // the coefficient fields at x with d/dx_b seeded: div Phi includes their gradient
      D1 xd[3], cfd[NcfOf<SysD>::value];
#pragma unroll
      for (int d = 0; d < 3; ++d) xd[d] = D1(xc[d], d == b ? T(1) : T(0));
      prescribed_fields(p, xd, t, cfd);
      SysD::eval(pd, q0, dQd, Phi, S, cfd, cfd);
    } else {
      SysD::eval(pd, q0, dQd, Phi, S);
    }
#pragma unroll
    for (int k2 = 0; k2 < K; ++k2) acc[k2] += Phi[k2][b].d - (b == 0 ? S[k2].v : T(0));
  }
#pragma unroll
  for (int k2 = 0; k2 < NC; ++k2) Src[k2] += acc[k2];
  if (p.mms_trackers) {
#pragma unroll
    for (int k2 = NC; k2 < K; ++k2) Src[k2] += acc[k2];
  }
}

// --------------------------------------------------------------------------- the step
// Population staging between the moment pass and the write pass:
//   MODE_REG   the node's K q values stay in registers (K q <= 90);
//   MODE_SMEM  each thread copies its node's K q values into its own column of dynamic
//              shared memory (cp.async for 4/8-byte values), [(k q + i) * blockDim + tid]:
//              no other thread touches the column, so no barrier is needed, and DRAM sees
//              every population once.
constexpr int MODE_REG = 0, MODE_SMEM = 1;


// COLS: threads per block of a staged launch (the column stride of its layout).
template <class Lat, template <typename> class SysT, class St, int COLS = 128>
struct StepMode {
  // register-resident or per-thread staged (also the batched kernel's choice): registers
  // hold up to 360 bytes of populations for systems of at most 12 components; larger
  // systems need the registers for their flux (18 components on D2Q5 spill at 128)
  static constexpr int value =
      ((size_t)SysT<typename St::C>::K * Lat::Q * sizeof(typename St::C) <= 360 && SysT<typename St::C>::K <= 12)
          ? MODE_REG
          : MODE_SMEM;
  static constexpr size_t smem_per_thread = (size_t)SysT<typename St::C>::K * Lat::Q * sizeof(typename St::S);
  static constexpr size_t smem_bytes = value == MODE_SMEM ? smem_per_thread * COLS : 0;
  // blocks per SM the launch bounds ask the register allocator to allow: 4 for
  // register-resident kernels (128 registers; the FP16 ones spill at 5), and for staged
  // kernels what shared memory lets reside (228 KB per SM), at most `cap` threads
  static constexpr int smem_blocks = value == MODE_SMEM ? (int)(228 * 1024 / smem_bytes) : 0;
  static constexpr int blocks_for(int cap) {
    return value == MODE_REG ? 4 : (smem_blocks < 1 ? 1 : (smem_blocks * COLS > cap ? cap / COLS : smem_blocks));
  }
  static constexpr int min_blocks = blocks_for(384);
  // the unforced two-buffer step with FP16 storage: its half-size columns leave room for 640
  // threads (96 registers, no spills), more warps to cover the memory latency; the forced
  // and in-place kernels need their registers and keep 384.  (Register-resident FP16 kernels
  // measured the same at 4, 5 and 6 blocks of 128 per SM: they keep 4.)
  static constexpr int min_blocks_step = blocks_for(sizeof(typename St::S) == 2 ? 640 : 384);
};

// Whether finish_node runs the paired FP32 arithmetic (results are bitwise the same either
// way; only the instruction stream differs).  Measured per kernel kind: it pays in every
// staged kernel and in register-resident ones of at most 60 populations per node (NSF K = 12
// on D2Q5 +4 %, Euler FP16 +6 %), and costs in the register-resident NSF on D2Q9 (90
// populations, -2 %, tighter register pairing) and in the persistent batched kernel (-5 %),
// which therefore keep the scalar form (NOPACK).
template <class Lat, template <typename> class SysT, class St, bool NOPACK>
struct PackedUpdate {
  static constexpr bool value =
      sizeof(typename St::C) == 4 && !NOPACK &&
      (StepMode<Lat, SysT, St>::value == MODE_SMEM || SysT<typename St::C>::K * Lat::Q <= 60);
};

template <typename S>
__device__ __forceinline__ void stage(S* sm, const S* g) {
  if constexpr (sizeof(S) == 2) {
    *sm = __ldg(g);
  } else {
    const unsigned int sa = (unsigned int)__cvta_generic_to_shared(sm);
    if constexpr (sizeof(S) == 4)
      asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sa), "l"(g) : "memory");
    else
      asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(g) : "memory");
  }
}
__device__ __forceinline__ void stage_wait() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Shared-memory reads the compiler must not merge or keep live across the flux evaluation
// (asm volatile), so the staged values cost no registers between the two passes.
__device__ __forceinline__ float lds_c(const float* p) {
  float v;
  asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"((unsigned int)__cvta_generic_to_shared(p)));
  return v;
}
__device__ __forceinline__ double lds_c(const double* p) {
  double v;
  asm volatile("ld.shared.f64 %0, [%1];" : "=d"(v) : "r"((unsigned int)__cvta_generic_to_shared(p)));
  return v;
}
__device__ __forceinline__ float lds_c(const __half* p) {
  unsigned short v;
  asm volatile("ld.shared.b16 %0, [%1];" : "=h"(v) : "r"((unsigned int)__cvta_generic_to_shared(p)));
  return __half2float(__ushort_as_half(v));
}

// Component pairs: vector type, global load, shared staging and read, conversion, store.
template <typename S> struct PairOf;
template <> struct PairOf<double> { using V = double2; };
template <> struct PairOf<float> { using V = float2; };
template <> struct PairOf<__half> { using V = __half2; };

__device__ __forceinline__ double2 ldg_pair(const double2* p) { return __ldg(p); }
__device__ __forceinline__ float2 ldg_pair(const float2* p) { return __ldg(p); }
__device__ __forceinline__ __half2 ldg_pair(const __half2* p) { return __ldg(p); }
__device__ __forceinline__ void split(double2 v, double& a, double& b) { a = v.x; b = v.y; }
__device__ __forceinline__ void split(float2 v, float& a, float& b) { a = v.x; b = v.y; }
__device__ __forceinline__ void split(__half2 v, float& a, float& b) { a = __low2float(v); b = __high2float(v); }
__device__ __forceinline__ void st_pair(double2* p, double a, double b) { *p = make_double2(a, b); }
__device__ __forceinline__ void st_pair(float2* p, float a, float b) { *p = make_float2(a, b); }
__device__ __forceinline__ void st_pair(__half2* p, float a, float b) { *p = __floats2half2_rn(a, b); }
template <typename V>
__device__ __forceinline__ void stage_pair(V* sm, const V* g) {
  const unsigned int sa = (unsigned int)__cvta_generic_to_shared(sm);
  if constexpr (sizeof(V) == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(g) : "memory");
  else if constexpr (sizeof(V) == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(g) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sa), "l"(g) : "memory");
}
// pair reads from shared memory that stay volatile (re-issued in each pass)
__device__ __forceinline__ void lds_pair(const double2* p, double& a, double& b) {
  asm volatile("ld.shared.v2.f64 {%0, %1}, [%2];" : "=d"(a), "=d"(b) : "r"((unsigned int)__cvta_generic_to_shared(p)));
}
__device__ __forceinline__ void lds_pair(const float2* p, float& a, float& b) {
  asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(a), "=f"(b) : "r"((unsigned int)__cvta_generic_to_shared(p)));
}
__device__ __forceinline__ void lds_pair(const __half2* p, float& a, float& b) {
  unsigned int v;
  asm volatile("ld.shared.b32 %0, [%1];" : "=r"(v) : "r"((unsigned int)__cvta_generic_to_shared(p)));
  __half2 h = *reinterpret_cast<__half2*>(&v);
  a = __low2float(h);
  b = __high2float(h);
}

// Moment accumulation straight from stored values: a component pair (or the odd component)
// added to float32/float64 moments.  For binary16 storage, add.rn.f32.f16 converts the stored
// value exactly and rounds the sum once, which is bitwise the conversion followed by an add,
// in one instruction instead of two.
__device__ __forceinline__ void acc_h2(__half2 h, float& a, float& b) {
  const unsigned int v = *reinterpret_cast<unsigned int*>(&h);
  asm("{\n\t.reg .f16 lo, hi;\n\tmov.b32 {lo, hi}, %2;\n\tadd.rn.f32.f16 %0, lo, %0;\n\t"
      "add.rn.f32.f16 %1, hi, %1;\n\t}"
      : "+f"(a), "+f"(b)
      : "r"(v));
}
__device__ __forceinline__ void acc_h1(__half h, float& a) {
  asm("add.rn.f32.f16 %0, %1, %0;" : "+f"(a) : "h"(__half_as_ushort(h)));
}
// staged pair / odd value from shared memory into the moments
__device__ __forceinline__ void acc_lds_pair(const __half2* p, float& a, float& b) {
  unsigned int v;
  asm volatile("ld.shared.b32 %0, [%1];" : "=r"(v) : "r"((unsigned int)__cvta_generic_to_shared(p)));
  acc_h2(*reinterpret_cast<__half2*>(&v), a, b);
}
__device__ __forceinline__ void acc_lds_odd(const __half* p, float& a) {
  unsigned short v;
  asm volatile("ld.shared.b16 %0, [%1];" : "=h"(v) : "r"((unsigned int)__cvta_generic_to_shared(p)));
  acc_h1(__ushort_as_half(v), a);
}

// Paired float32 arithmetic (fma/add/sub .rn.f32x2): two independent IEEE operations in one
// instruction, each lane rounded exactly as the scalar operation, so results are bitwise
// those of two scalar instructions.
__device__ __forceinline__ unsigned long long f2_bits(float2 v) { return *reinterpret_cast<unsigned long long*>(&v); }
__device__ __forceinline__ float2 bits_f2(unsigned long long b) { return *reinterpret_cast<float2*>(&b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(f2_bits(a)), "l"(f2_bits(b)), "l"(f2_bits(c)));
  return bits_f2(d);
}
__device__ __forceinline__ float2 add2(float2 a, float2 b) {
  unsigned long long d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2_bits(a)), "l"(f2_bits(b)));
  return bits_f2(d);
}
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  unsigned long long d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2_bits(a)), "l"(f2_bits(b)));
  return bits_f2(d);
}
__device__ __forceinline__ float2 mul2(float2 a, float2 b) {
  unsigned long long d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2_bits(a)), "l"(f2_bits(b)));
  return bits_f2(d);
}

__device__ __forceinline__ float to_c(__half h) { return __half2float(h); }
__device__ __forceinline__ float to_c(float v) { return v; }
__device__ __forceinline__ double to_c(double v) { return v; }

// One node of one grid: pull, moments, flux/source, equilibrium, BGK, store.  `step` is
// the index of the step being taken (only the manufactured forcing uses it).
//
// Arithmetic (Eq. lbe_update with Eq. feq): with w = 1/tau_k,
//   f_out = f + w (F_i - f),   F_i = w_i (X_k + tau_k dt S_k) + w_i c_i . phi_k,
// phi_k = (dt/dx)/c_s^2 Phi_k.  w multiplies only the small non-equilibrium difference
// F_i - f, so the sum over i conserves X_k (+ dt S_k) up to random rounding: a rounded
// coefficient never multiplies the O(f) equilibrium itself.  Opposite velocities share
// the projection P = c'_i . phi_k (c' = c_i oriented so its first nonzero entry is +1)
// and the weight class shares w_i (X_k + tau_k dt S_k), so each population costs one
// add (moment) and three fused operations.  FP16 storage works in stored units (values
// divided by s_k): X, phi and dt S are divided by s_k once per component.
// Float64 runs on the far narrower FP64 pipe, where the operation count sets the speed:
// there f_out = (1 - w) f + [w w_i (X_k + tau_k dt S_k) + (w w_i) c_i . phi_k] with
// 1 - w and w w_i per weight class from host tables, two fused operations per population.
// The rounded coefficient 1 - w on the O(f) term moves sum_i f_out by one float64 rounding
// (~1e-16 relative) per step, far below what the float64 path is checked to.
// Moments, flux and source, equilibrium, BGK and store for one node whose populations
// are available through get_pair(kp, i, a, b) / get_odd(i) (registers or a staged column).
// Destination of the post-collision populations: DstSelf stores population (k, i) of the
// node at (k, i, cell); another functor maps (k, i) to an element index (in-place steps).
struct DstSelf {};

// acc_pair(kp, i, X0, X1) / acc_odd(i, X), when given, add the populations into the moments
// without get_pair's conversion (binary16 storage: one mixed-precision add per value).
template <class Lat, template <typename> class SysT, class St, bool FOURIER = false, bool NOPACK = false,
          class GetPair, class GetOdd, class Dst = DstSelf, class AccPair = std::nullptr_t,
          class AccOdd = std::nullptr_t>
__device__ __forceinline__ void finish_node(typename St::S* __restrict__ B, const KParams<typename St::C>& p,
                                            int x, int y, int z, unsigned int cell, long long step, bool active,
                                            GetPair get_pair, GetOdd get_odd,
                                            const typename St::C* tfac = nullptr, Dst dst = Dst(),
                                            AccPair acc_pair = nullptr, AccOdd acc_odd = nullptr) {
  using T = typename St::C;
  using V = typename PairOf<typename St::S>::V;
  using Sys = SysT<T>;
  constexpr int K = Sys::K, Q = Lat::Q, D = Lat::D, KP = K / 2;
  constexpr bool ODD = (K & 1) != 0;
  const unsigned int plane = (unsigned int)p.ncell;

  // a2: moments (Eq. moments), in stored units
  T X[K];
#pragma unroll
  for (int k = 0; k < K; ++k) X[k] = T(0);
#pragma unroll
  for (int kp = 0; kp < KP; ++kp) {
    if constexpr (sizeof(T) == 4 && std::is_same<AccPair, std::nullptr_t>::value &&
                  PackedUpdate<Lat, SysT, St, NOPACK>::value) {
      float2 x2 = make_float2(0.f, 0.f);      // the pair's two sums in one paired add per velocity
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        T a, b;
        get_pair(kp, i, a, b);
        x2 = add2(x2, make_float2(a, b));
      }
      X[2 * kp] = x2.x;
      X[2 * kp + 1] = x2.y;
    } else {
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        if constexpr (std::is_same<AccPair, std::nullptr_t>::value) {
          T a, b;
          get_pair(kp, i, a, b);
          X[2 * kp] += a;
          X[2 * kp + 1] += b;
        } else {
          acc_pair(kp, i, X[2 * kp], X[2 * kp + 1]);
        }
      }
    }
  }
  if constexpr (ODD) {
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      if constexpr (std::is_same<AccOdd, std::nullptr_t>::value)
        X[K - 1] += get_odd(i);
      else
        acc_odd(i, X[K - 1]);
    }
  }

  // a3: primitives, flux and source at the node (physical units)
  T dQ[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const T xk = St::SCALE ? X[k] * p.scale[k] : X[k];
    dQ[k] = St::SHIFT ? xk : xk - p.Q0[k];
  }
  T Phi[K][D], Src[K];
  eval_node<SysT>(p, x, y, z, T(step) * p.dt, dQ, Phi, Src);
  if (Sys::FAMILY == 1 && p.mms_tab != nullptr) Src[0] += adr_mms(p, x, y, step);
  if constexpr (FOURIER) {
    if (p.mms_modes != nullptr) mms_fourier<Lat, SysT, T>(p, x, y, z, step, Src, tfac);
  }

  // a4 + a5 + a6: equilibrium (Eq. feq), BGK with source (Eq. lbe_update), store
  // destination of a pair / of the odd component (32-bit element indices from eidx: a
  // per-node 64-bit base with 32-bit row offsets measured 5-7 % slower in the staged kernels)
  auto pair_dst = [&](int kp, int i) -> V* {
    if constexpr (std::is_same<Dst, DstSelf>::value)
      return reinterpret_cast<V*>(B + eidx<K, Q>(2 * kp, i, cell, plane));
    else
      return reinterpret_cast<V*>(B + dst(2 * kp, i));
  };
  auto odd_dst = [&](int i) -> typename St::S* {
    if constexpr (std::is_same<Dst, DstSelf>::value)
      return B + eidx<K, Q>(K - 1, i, cell, plane);
    else
      return B + dst(K - 1, i);
  };
  auto out_of = [&](int k, int i, T f) -> T {
    const T inv_s = St::SCALE ? p.inv_scale[k] : T(1);
    const int sg = Lat::c(i, 0) != 0 ? Lat::c(i, 0) : (Lat::c(i, 1) != 0 ? Lat::c(i, 1) : Lat::c(i, 2));
    T P = T(0);
#pragma unroll
    for (int d = 0; d < D; ++d) {
      const int cd = Lat::c(i, d) * sg;
      const T phd = (p.lc * Phi[k][d] + (St::SHIFT ? T(0) : p.F0l[k][d])) * inv_s;
      if (cd == 1) P += phd;
      if (cd == -1) P -= phd;
    }
    const T Xs = X[k] + p.tau[k] * (p.dt * Src[k] * inv_s);
    if constexpr (sizeof(T) == 8) {
      // float64 (the arithmetic-bound kind): (1 - w) f + w F_i with w w_i from the table of
      // the weight class, two fused operations per population; the products w w_i X's are
      // shared by the class and the projection P by the opposite pair.
      const int cls = Lat::c(i, 0) * Lat::c(i, 0) + Lat::c(i, 1) * Lat::c(i, 1) + Lat::c(i, 2) * Lat::c(i, 2);
      const T owi = p.ow[k][cls];
      return fma(p.omc[k], f, fma(T(sg) * owi, P, owi * Xs));
    } else {
      const T wi = weight<Lat, T>(i);
      const T Fi = fma(T(sg) * wi, P, wi * Xs);
      return fma(p.omega[k], Fi - f, f);
    }
  };
  if constexpr (sizeof(T) == 4 && PackedUpdate<Lat, SysT, St, NOPACK>::value) {
    // float32 arithmetic: the two components of a pair share the paired FP32 pipe (the
    // same operations as out_of, lane by lane, so bitwise its results); the projection of
    // a velocity is formed once for it and its opposite, w_i X's once per weight class
#pragma unroll
    for (int kp = 0; kp < KP; ++kp) {
      const int ka = 2 * kp, kb = 2 * kp + 1;
      const T isa = St::SCALE ? p.inv_scale[ka] : T(1), isb = St::SCALE ? p.inv_scale[kb] : T(1);
      float2 ph2[D];
#pragma unroll
      for (int d = 0; d < D; ++d)
        ph2[d] = make_float2((p.lc * Phi[ka][d] + (St::SHIFT ? T(0) : p.F0l[ka][d])) * isa,
                             (p.lc * Phi[kb][d] + (St::SHIFT ? T(0) : p.F0l[kb][d])) * isb);
      const float2 xs2 = make_float2(X[ka] + p.tau[ka] * (p.dt * Src[ka] * isa), X[kb] + p.tau[kb] * (p.dt * Src[kb] * isb));
      const float2 om2 = make_float2(p.omega[ka], p.omega[kb]);
      float2 wx2[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        int i0 = -1;
#pragma unroll
        for (int i = 0; i < Q; ++i)
          if (i0 < 0 && Lat::c(i, 0) * Lat::c(i, 0) + Lat::c(i, 1) * Lat::c(i, 1) + Lat::c(i, 2) * Lat::c(i, 2) == c) i0 = i;
        const T wc = i0 < 0 ? T(0) : weight<Lat, T>(i0);
        wx2[c] = i0 < 0 ? make_float2(0.f, 0.f) : mul2(make_float2(wc, wc), xs2);
      }
      float2 P2 = make_float2(0.f, 0.f);
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        const int sg = Lat::c(i, 0) != 0 ? Lat::c(i, 0) : (Lat::c(i, 1) != 0 ? Lat::c(i, 1) : Lat::c(i, 2));
        if (i == 0 || i != opp<Lat>(i) + 1) {   // rest, or the first of an opposite pair
          bool first = true;
#pragma unroll
          for (int d = 0; d < D; ++d) {
            const int cd = Lat::c(i, d) * sg;
            if (cd == 0) continue;
            if (first) P2 = cd == 1 ? ph2[d] : sub2(make_float2(0.f, 0.f), ph2[d]);
            else P2 = cd == 1 ? add2(P2, ph2[d]) : sub2(P2, ph2[d]);
            first = false;
          }
          if (first) P2 = make_float2(0.f, 0.f);
        }
        const int cls = Lat::c(i, 0) * Lat::c(i, 0) + Lat::c(i, 1) * Lat::c(i, 1) + Lat::c(i, 2) * Lat::c(i, 2);
        const T swi = T(sg) * weight<Lat, T>(i);
        T a, b;
        get_pair(kp, i, a, b);
        const float2 f2 = make_float2(a, b);
        const float2 F2 = fma2(make_float2(swi, swi), P2, wx2[cls]);
        const float2 o2 = fma2(om2, sub2(F2, f2), f2);
        if (active) st_pair(pair_dst(kp, i), o2.x, o2.y);
      }
    }
  } else {
#pragma unroll
    for (int kp = 0; kp < KP; ++kp)
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        T a, b;
        get_pair(kp, i, a, b);
        const T oa = out_of(2 * kp, i, a), ob = out_of(2 * kp + 1, i, b);
        if (active) st_pair(pair_dst(kp, i), oa, ob);
      }
  }
  if constexpr (ODD) {
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const T o = out_of(K - 1, i, get_odd(i));
      if (active) st_out(odd_dst(i), o);
    }
  }
}

// Issue the copies of one node's pulled populations into a staged column: pairs
// [KP q][COLS] of V, then the odd component [q][COLS] of S.
template <class Lat, template <typename> class SysT, class St, int COLS>
__device__ __forceinline__ void stage_node(const typename St::S* __restrict__ A,
                                           typename PairOf<typename St::S>::V* colv, typename St::S* colo,
                                           const PullIdx& pi, const KParams<typename St::C>& p) {
  using S = typename St::S;
  using V = typename PairOf<S>::V;
  constexpr int K = SysT<typename St::C>::K, Q = Lat::Q, KP = K / 2;
  const unsigned int plane = (unsigned int)p.ncell;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const unsigned int src = pi.src<Lat>(i, p.nx, p.ny);
#pragma unroll
    for (int kp = 0; kp < KP; ++kp)
      stage_pair(colv + (kp * Q + i) * COLS, reinterpret_cast<const V*>(A + eidx<K, Q>(2 * kp, i, src, plane)));
    if constexpr ((K & 1) != 0) stage(colo + i * COLS, A + eidx<K, Q>(K - 1, i, src, plane));
  }
}

template <class Lat, template <typename> class SysT, class St, int MODE, int COLS = 128, bool FOURIER = false,
          bool NOPACK = false>
__device__ __forceinline__ void step_node(const typename St::S* __restrict__ A, typename St::S* __restrict__ B,
                                          const KParams<typename St::C>& p, int x, int y, int z,
                                          long long step, const typename St::C* tfac = nullptr) {
  using T = typename St::C;
  using S = typename St::S;
  using V = typename PairOf<S>::V;
  constexpr int K = SysT<T>::K, Q = Lat::Q, KP = K / 2;
  constexpr bool ODD = (K & 1) != 0;
  const PullIdx pi(x, y, z, p.nx, p.ny, p.nz);
  // element offsets fit in 32 bits (the host guarantees K q cells < 2^32)
  const unsigned int plane = (unsigned int)p.ncell;
  const unsigned int cell = ((unsigned int)z * (unsigned int)p.ny + (unsigned int)y) * (unsigned int)p.nx + x;
  if constexpr (MODE == MODE_REG) {
    // a1: pull every population of the node into registers, two components per access
    T fv[K][Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const unsigned int src = pi.src<Lat>(i, p.nx, p.ny);
#pragma unroll
      for (int kp = 0; kp < KP; ++kp)
        split(ldg_pair(reinterpret_cast<const V*>(A + eidx<K, Q>(2 * kp, i, src, plane))), fv[2 * kp][i],
              fv[2 * kp + 1][i]);
      if constexpr (ODD) fv[K - 1][i] = to_c(__ldg(A + eidx<K, Q>(K - 1, i, src, plane)));
    }
    finish_node<Lat, SysT, St, FOURIER, NOPACK>(
        B, p, x, y, z, cell, step, true,
        [&](int kp, int i, T& a, T& b) {
          a = fv[2 * kp][i];
          b = fv[2 * kp + 1][i];
        },
        [&](int i) -> T { return fv[ODD ? K - 1 : 0][i]; }, tfac);
  } else {
    // a1: stage every population of the node in this thread's shared-memory column
    extern __shared__ __align__(16) unsigned char lbx_smem[];
    V* colv = reinterpret_cast<V*>(lbx_smem) + threadIdx.x;
    S* colo = reinterpret_cast<S*>(reinterpret_cast<V*>(lbx_smem) + KP * Q * COLS) + threadIdx.x;
    stage_node<Lat, SysT, St, COLS>(A, colv, colo, pi, p);
    stage_wait();
    auto get_pair = [&](int kp, int i, T& a, T& b) { lds_pair(colv + (kp * Q + i) * COLS, a, b); };
    auto get_odd = [&](int i) -> T { return lds_c(colo + i * COLS); };
    if constexpr (sizeof(S) == 2)
      finish_node<Lat, SysT, St, FOURIER, NOPACK>(
          B, p, x, y, z, cell, step, true, get_pair, get_odd, tfac, DstSelf(),
          [&](int kp, int i, T& a, T& b) { acc_lds_pair(colv + (kp * Q + i) * COLS, a, b); },
          [&](int i, T& a) { acc_lds_odd(colo + i * COLS, a); });
    else
      finish_node<Lat, SysT, St, FOURIER, NOPACK>(B, p, x, y, z, cell, step, true, get_pair, get_odd, tfac);
  }
}

// ------------------------------------------------------------ two lanes per node
// Staged variant for large K q: the two adjacent lanes 2m, 2m + 1 of a warp share node m.
// Lane h takes the rest population (h = 0 only) and, of every opposite pair (i, i + 1) of
// the lattice (i odd, c_{i+1} = -c_i, first nonzero entry of c_i = +1), velocity i + h,
// whose direction is (1 - 2h) c_i.  Pulling along -c_i mirrors the neighbour table, and
// the population planes of velocity i + h sit h planes after those of i, so both lanes run
// the same instruction stream.  Each lane sums its own populations and the pair adds the
// partner's partial sums with one shuffle per component (a + b = b + a bitwise, so both
// lanes hold identical moments); both evaluate the flux, each updates its own velocities.
// Per lane this halves the staged column, the loads, the moment adds and the update, and
// the same shared memory then keeps twice as many warps resident.
template <class Lat>
struct SplitLat {
  static constexpr int NP = (Lat::Q - 1) / 2;    // opposite pairs
  static constexpr int QH = NP + 1;              // velocity slots per lane (slot 0: rest)
  static constexpr bool valid() {
    if ((Lat::Q & 1) == 0) return false;
    for (int d = 0; d < 3; ++d)
      if (Lat::c(0, d) != 0) return false;
    for (int pp = 0; pp < NP; ++pp) {
      const int i = 2 * pp + 1;
      int lead = 0;
      for (int d = 0; d < 3; ++d) {
        if (Lat::c(i + 1, d) != -Lat::c(i, d)) return false;
        if (lead == 0) lead = Lat::c(i, d);
      }
      if (lead != 1) return false;
    }
    return true;
  }
};

template <class Lat, template <typename> class SysT, class St, int COLS>
struct SplitMode {
  static constexpr size_t smem_per_thread =
      (size_t)SysT<typename St::C>::K * SplitLat<Lat>::QH * sizeof(typename St::S);
  static constexpr size_t smem_bytes = smem_per_thread * COLS;
  // blocks that shared memory lets reside (228 KB per SM, 1 KB reserved per block),
  // at most 512 threads per SM so that the flux keeps 128 registers
  static constexpr int smem_blocks = (int)(228 * 1024 / (smem_bytes + 1024));
  static constexpr int min_blocks =
      smem_blocks < 1 ? 1 : (smem_blocks * COLS > 512 ? 512 / COLS : smem_blocks);
};

template <class Lat, template <typename> class SysT, class St, int COLS>
__device__ __forceinline__ void step_node_split(const typename St::S* __restrict__ A,
                                                typename St::S* __restrict__ B,
                                                const KParams<typename St::C>& p, int x, int y, int z,
                                                long long step, int h, bool active) {
  using T = typename St::C;
  using S = typename St::S;
  using V = typename PairOf<S>::V;
  using Sys = SysT<T>;
  constexpr int K = Sys::K, Q = Lat::Q, D = Lat::D, KP = K / 2;
  constexpr int NP = SplitLat<Lat>::NP, QH = SplitLat<Lat>::QH;
  constexpr bool ODD = (K & 1) != 0;
  static_assert(SplitLat<Lat>::valid(), "lattice order must be rest, then (+c, -c) pairs");
  const unsigned int plane = (unsigned int)p.ncell;
  const unsigned int cell = ((unsigned int)z * (unsigned int)p.ny + (unsigned int)y) * (unsigned int)p.nx + x;
  // lane 1 pulls along -c_i: swap the +1 / -1 neighbours of every axis
  PullIdx pi(x, y, z, p.nx, p.ny, p.nz);
  if (h) {
    const int tx = pi.sx[0], ty = pi.sy[0], tz = pi.sz[0];
    pi.sx[0] = pi.sx[2]; pi.sx[2] = tx;
    pi.sy[0] = pi.sy[2]; pi.sy[2] = ty;
    pi.sz[0] = pi.sz[2]; pi.sz[2] = tz;
  }
  // planes of velocity i + h: pairs are interleaved (2 values per node), the odd component is not
  const S* Ap = A + (size_t)h * 2 * plane;
  const S* Ao = A + (size_t)h * plane;
  S* Bp = B + (size_t)h * 2 * plane;
  S* Bo = B + (size_t)h * plane;

  // a1: stage this lane's populations: pairs [KP QH][COLS] of V, odd component [QH][COLS]
  extern __shared__ __align__(16) unsigned char lbx_smem[];
  V* colv = reinterpret_cast<V*>(lbx_smem) + threadIdx.x;
  S* colo = reinterpret_cast<S*>(reinterpret_cast<V*>(lbx_smem) + KP * QH * COLS) + threadIdx.x;
  if (h == 0) {
#pragma unroll
    for (int kp = 0; kp < KP; ++kp)
      stage_pair(colv + kp * QH * COLS, reinterpret_cast<const V*>(A + eidx<K, Q>(2 * kp, 0, cell, plane)));
    if constexpr (ODD) stage(colo, A + eidx<K, Q>(K - 1, 0, cell, plane));
  }
#pragma unroll
  for (int pp = 0; pp < NP; ++pp) {
    const int i = 2 * pp + 1;
    const unsigned int src = pi.src<Lat>(i, p.nx, p.ny);
#pragma unroll
    for (int kp = 0; kp < KP; ++kp)
      stage_pair(colv + (kp * QH + pp + 1) * COLS, reinterpret_cast<const V*>(Ap + eidx<K, Q>(2 * kp, i, src, plane)));
    if constexpr (ODD) stage(colo + (pp + 1) * COLS, Ao + eidx<K, Q>(K - 1, i, src, plane));
  }
  stage_wait();

  // a2: moments (Eq. moments), in stored units: own populations, then the partner's sum
  T X[K];
#pragma unroll
  for (int k = 0; k < K; ++k) X[k] = T(0);
  if (h == 0) {
#pragma unroll
    for (int kp = 0; kp < KP; ++kp) lds_pair(colv + kp * QH * COLS, X[2 * kp], X[2 * kp + 1]);
    if constexpr (ODD) X[K - 1] = lds_c(colo);
  }
#pragma unroll
  for (int kp = 0; kp < KP; ++kp)
#pragma unroll
    for (int pp = 0; pp < NP; ++pp) {
      T a, b;
      lds_pair(colv + (kp * QH + pp + 1) * COLS, a, b);
      X[2 * kp] += a;
      X[2 * kp + 1] += b;
    }
  if constexpr (ODD) {
#pragma unroll
    for (int pp = 0; pp < NP; ++pp) X[K - 1] += lds_c(colo + (pp + 1) * COLS);
  }
#pragma unroll
  for (int k = 0; k < K; ++k) X[k] += __shfl_xor_sync(0xffffffffu, X[k], 1);

  // a3: primitives, flux and source at the node (physical units)
  T dQ[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const T xk = St::SCALE ? X[k] * p.scale[k] : X[k];
    dQ[k] = St::SHIFT ? xk : xk - p.Q0[k];
  }
  T Phi[K][D], Src[K];
  eval_node<SysT>(p, x, y, z, T(step) * p.dt, dQ, Phi, Src);
  if (Sys::FAMILY == 1 && p.mms_tab != nullptr) Src[0] += adr_mms(p, x, y, step);

  // a4 + a5 + a6: the arithmetic of finish_node with the sign of c' . phi set by the lane
  const T sgn = h ? T(-1) : T(1);
  auto out_of = [&](int k, int i, T f) -> T {
    const T inv_s = St::SCALE ? p.inv_scale[k] : T(1);
    const T Xs = X[k] + p.tau[k] * (p.dt * Src[k] * inv_s);
    const T wi = weight<Lat, T>(i);
    T F;
    if (i == 0) {
      F = wi * Xs;
    } else {
      T P = T(0);
#pragma unroll
      for (int d = 0; d < D; ++d) {
        const int cd = Lat::c(i, d);
        const T phd = (p.lc * Phi[k][d] + (St::SHIFT ? T(0) : p.F0l[k][d])) * inv_s;
        if (cd == 1) P += phd;
        if (cd == -1) P -= phd;
      }
      F = fma(sgn * wi, P, wi * Xs);
    }
    return fma(p.omega[k], F - f, f);
  };
  const bool rest = active && h == 0;
#pragma unroll
  for (int kp = 0; kp < KP; ++kp) {
    {
      T a, b;
      lds_pair(colv + kp * QH * COLS, a, b);
      const T oa = out_of(2 * kp, 0, a), ob = out_of(2 * kp + 1, 0, b);
      if (rest) st_pair(reinterpret_cast<V*>(B + eidx<K, Q>(2 * kp, 0, cell, plane)), oa, ob);
    }
#pragma unroll
    for (int pp = 0; pp < NP; ++pp) {
      const int i = 2 * pp + 1;
      T a, b;
      lds_pair(colv + (kp * QH + pp + 1) * COLS, a, b);
      const T oa = out_of(2 * kp, i, a), ob = out_of(2 * kp + 1, i, b);
      if (active) st_pair(reinterpret_cast<V*>(Bp + eidx<K, Q>(2 * kp, i, cell, plane)), oa, ob);
    }
  }
  if constexpr (ODD) {
    {
      const T o = out_of(K - 1, 0, lds_c(colo));
      if (rest) st_out(B + eidx<K, Q>(K - 1, 0, cell, plane), o);
    }
#pragma unroll
    for (int pp = 0; pp < NP; ++pp) {
      const int i = 2 * pp + 1;
      const T o = out_of(K - 1, i, lds_c(colo + (pp + 1) * COLS));
      if (active) st_out(Bo + eidx<K, Q>(K - 1, i, cell, plane), o);
    }
  }
}

// Blocks of COLS lanes cover COLS / 2 nodes along x.  Lanes past the row end compute on a
// clamped node and store nothing, so every lane takes part in the shuffles.
template <class Lat, template <typename> class SysT, class St, int COLS>
__global__ void __launch_bounds__(COLS, SplitMode<Lat, SysT, St, COLS>::min_blocks)
    k_step_split(const typename St::S* __restrict__ A, typename St::S* __restrict__ B,
                 const KParams<typename St::C> p) {
  const int xr = blockIdx.x * (COLS / 2) + (int)(threadIdx.x >> 1);
  const bool active = xr < p.nx;
  const int x = active ? xr : p.nx - 1;
  const long long step = time_dependent(p) ? *p.step_ptr + p.step_rel : 0;
  step_node_split<Lat, SysT, St, COLS>(A, B, p, x, block_y<Lat>(p), block_z<Lat>(p), step, (int)(threadIdx.x & 1),
                                       active);
}

// ------------------------------------------------------------ bulk-copied rows (TMA)
// Staged variant for large K q whose pulled populations reach shared memory by bulk
// copies (cp.async.bulk, executed by the TMA engine) instead of per-thread copies.  A
// block owns COLS consecutive nodes x0 .. x0 + COLS - 1 of one row; for velocity i and
// every component the pull reads one contiguous run of the row at (y - c_iy, z - c_iz),
// shifted by c_ix.  Lane i of warp 0 issues the runs of velocity i (one per component
// pair, one for an odd component), each widened by E = 16 / element-bytes elements on the
// side the shift reaches into so that it starts and ends on 16-byte boundaries, and
// clamped to the row: the periodic wrap of the two edge nodes (x = 0 pulling along +x,
// x = nx - 1 along -x) is filled by those threads with plain loads.  All copies complete
// on one mbarrier; every thread's wait is bounded (KParams::wait_ns), and a timeout raises
// p.err and skips the node.
// Needs nx % 8 == 0 and 16-byte aligned population buffers (the host checks both).
template <class Lat, template <typename> class SysT, class St, int COLS>
struct BulkMode {
  using S = typename St::S;
  using V = typename PairOf<S>::V;
  static constexpr int K = SysT<typename St::C>::K, Q = Lat::Q, KP = K / 2;
  static constexpr bool ODD = (K & 1) != 0;
  static constexpr int EP = 16 / (int)sizeof(V), EO = 16 / (int)sizeof(S);
  static constexpr int ROWP = COLS + EP, ROWO = COLS + EO;      // row pitch in elements
  static constexpr size_t smem_bytes =
      16 + (size_t)KP * Q * ROWP * sizeof(V) + (ODD ? (size_t)Q * ROWO * sizeof(S) : 0);
  static constexpr int smem_blocks = (int)(228 * 1024 / (smem_bytes + 1024));
  static constexpr int min_blocks =
      smem_blocks < 1 ? 1 : (smem_blocks * COLS > 512 ? 512 / COLS : smem_blocks);
  // offset of the pulled element of thread t in the row of velocity i (E: pad elements)
  __host__ __device__ static constexpr int shift(int i, int E) {
    return Lat::c(i, 0) == 1 ? E - 1 : (Lat::c(i, 0) == -1 ? 1 : 0);
  }
};

__device__ __forceinline__ unsigned int smem_u32(const void* p) {
  return (unsigned int)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned int bar, unsigned int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned int bar, unsigned int bytes) {
  asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned int bar) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(bar) : "memory");
}
// Suspend until phase `parity` of the barrier completes: tries of at most about a
// microsecond each while less than `limit_ns` of the global timer has passed, and no more
// than 2^22 tries; false on timeout.  The time is checked before every try, so a zero limit
// gives up at once whatever the copies' progress.  (Checking it every eighth try, or a
// __nanosleep back-off between tries, measured no faster: the timer read paces the spin.)
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ bool mbar_wait(unsigned int bar, unsigned int parity, unsigned long long limit_ns) {
  const unsigned long long t0 = global_ns();
  for (int it = 0; it < (1 << 22); ++it) {
    if (global_ns() - t0 >= limit_ns) break;
    unsigned int done;
    asm volatile(
        "{\n\t.reg .pred P;\n\tmbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, P;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity), "r"(1000u)
        : "memory");
    if (done) return true;
  }
  return false;
}
__device__ __forceinline__ void bulk_g2s(unsigned int dst, const void* src, unsigned int bytes, unsigned int bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}
// Default limit of the bounded wait for bulk copies (KParams::wait_ns), and the fixed limit
// of the second wait after a timeout, which lets the copies in flight land before the
// block leaves.
constexpr unsigned long long BULK_WAIT_NS = 1000000000ull;   // 1 s

// The bulk-staged step of one block.  KIND 0: two buffers (pull from A, write B); KIND 1, 2:
// the in-place step kinds on one buffer (A == B; see k_step_inplace): kind 1 pulls the same
// rows as KIND 0 and stores each post-collision population into the opposite slot it read
// from, kind 2 copies the node row's swapped slots unshifted and stores in the standard
// slots.  Every element a node uses is read and written by that node alone; the 16-byte
// widening of a shifted row also reads a few elements of neighbouring blocks that this
// block never uses.
template <class Lat, template <typename> class SysT, class St, int COLS, int KIND>
__device__ __forceinline__ void bulk_step_body(const typename St::S* A, typename St::S* B,
                                               const KParams<typename St::C>& p) {
  using M = BulkMode<Lat, SysT, St, COLS>;
  using T = typename St::C;
  using S = typename St::S;
  using V = typename M::V;
  constexpr int K = M::K, Q = Lat::Q, KP = M::KP, EP = M::EP, EO = M::EO;
  constexpr bool ODD = M::ODD;
  static_assert(Q <= 32, "one issuing lane per velocity");
  static_assert(KIND == 0 || opp_valid<Lat>(), "velocities must come as rest, then (+c, -c) pairs");
  extern __shared__ __align__(16) unsigned char lbx_smem[];
  V* rowv = reinterpret_cast<V*>(lbx_smem + 16);                 // [KP q][ROWP]
  S* rowo = reinterpret_cast<S*>(rowv + (size_t)KP * Q * M::ROWP); // [q][ROWO]
  const unsigned int bar = smem_u32(lbx_smem);
  const int t = (int)threadIdx.x, x0 = (int)blockIdx.x * COLS, y = block_y<Lat>(p), z = block_z<Lat>(p);
  const int nx = p.nx, ny = p.ny, nz = p.nz;
  const unsigned int plane = (unsigned int)p.ncell;
  // offset of the element a thread uses in the shared row of velocity i
  auto sh = [](int i, int E) { return KIND == 2 ? 0 : M::shift(i, E); };

  if (t == 0) mbar_init(bar, 1);
  __syncthreads();
  if (t < 32) {
    if (t < Q) {
      // lane t copies the rows of velocity t: slot sv of the rows at (y - c_y, z - c_z),
      // shifted by c_x (kind 2: the node row's opposite slot, unshifted)
      int cx = 0, cy = 0, cz = 0;
      if constexpr (KIND != 2) {
#pragma unroll
        for (int j = 0; j < Q; ++j)
          if (j == t) {
            cx = Lat::c(j, 0);
            cy = Lat::c(j, 1);
            cz = Lat::c(j, 2);
          }
      }
      const int sv = KIND == 2 ? opp<Lat>(t) : t;
      const int ys = y - cy < 0 ? ny - 1 : (y - cy >= ny ? 0 : y - cy);
      const int zs = z - cz < 0 ? nz - 1 : (z - cz >= nz ? 0 : z - cz);
      const unsigned int cell0 = ((unsigned int)zs * (unsigned int)ny + (unsigned int)ys) * (unsigned int)nx;
      const int xsp = x0 - (cx == 1 ? EP : 0), xep = x0 + COLS + (cx == -1 ? EP : 0);
      const int lop = xsp < 0 ? 0 : xsp, hip = xep > nx ? nx : xep;
      const unsigned int bp = (unsigned int)(hip - lop) * (unsigned int)sizeof(V);
      const int xso = x0 - (cx == 1 ? EO : 0), xeo = x0 + COLS + (cx == -1 ? EO : 0);
      const int loo = xso < 0 ? 0 : xso, hio = xeo > nx ? nx : xeo;
      const unsigned int bo = ODD ? (unsigned int)(hio - loo) * (unsigned int)sizeof(S) : 0u;
      mbar_expect_tx(bar, KP * bp + bo);
      const V* Av = reinterpret_cast<const V*>(A);
#pragma unroll
      for (int kp = 0; kp < KP; ++kp)
        bulk_g2s(smem_u32(rowv + (size_t)(kp * Q + t) * M::ROWP + (lop - xsp)),
                 Av + (size_t)(kp * Q + sv) * plane + cell0 + lop, bp, bar);
      if constexpr (ODD)
        bulk_g2s(smem_u32(rowo + (size_t)t * M::ROWO + (loo - xso)),
                 A + (size_t)2 * KP * Q * plane + (size_t)sv * plane + cell0 + loo, bo, bar);
    }
    __syncwarp();
    if (t == 0) mbar_arrive(bar);
  }
  const int x = x0 + t;
  const PullIdx pi(x, y, z, nx, ny, nz);

  // periodic wrap at the row ends: the slot the clamped copy left empty
  if (KIND != 2 && x < nx && (x == 0 || x == nx - 1)) {
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const int cx = Lat::c(i, 0);
      if ((cx == 1 && x == 0) || (cx == -1 && x == nx - 1)) {
        const unsigned int src = pi.src<Lat>(i, nx, ny);
#pragma unroll
        for (int kp = 0; kp < KP; ++kp)
          rowv[(size_t)(kp * Q + i) * M::ROWP + t + M::shift(i, EP)] =
              *reinterpret_cast<const V*>(A + eidx<K, Q>(2 * kp, i, src, plane));
        if constexpr (ODD) rowo[(size_t)i * M::ROWO + t + M::shift(i, EO)] = A[eidx<K, Q>(K - 1, i, src, plane)];
      }
    }
  }
  // every thread waits for the copies itself (a single waiting thread with the block held at
  // a barrier measured 2-3 % slower: the release adds latency to every tile)
  if (x >= nx) return;
  if (!mbar_wait(bar, 0, p.wait_ns)) {
    if (p.err) atomicOr(p.err, 1u);
    mbar_wait(bar, 0, BULK_WAIT_NS);         // let copies in flight land before leaving
    return;
  }
  const unsigned int cell = ((unsigned int)z * (unsigned int)ny + (unsigned int)y) * (unsigned int)nx + x;
  const long long step = time_dependent(p) ? *p.step_ptr + p.step_rel : 0;
  auto pair_at = [&](int kp, int i) { return rowv + (size_t)(kp * Q + i) * M::ROWP + t + sh(i, EP); };
  auto odd_at = [&](int i) { return rowo + (size_t)(ODD ? i : 0) * M::ROWO + t + sh(i, EO); };
  auto get_pair = [&](int kp, int i, T& a, T& b) { lds_pair(pair_at(kp, i), a, b); };
  auto get_odd = [&](int i) -> T { return lds_c(odd_at(i)); };
  auto finish = [&](auto dst) {
    if constexpr (sizeof(S) == 2)
      finish_node<Lat, SysT, St>(B, p, x, y, z, cell, step, true, get_pair, get_odd, nullptr, dst,
                                 [&](int kp, int i, T& a, T& b) { acc_lds_pair(pair_at(kp, i), a, b); },
                                 [&](int i, T& a) { acc_lds_odd(odd_at(i), a); });
    else
      finish_node<Lat, SysT, St>(B, p, x, y, z, cell, step, true, get_pair, get_odd, nullptr, dst);
  };
  if constexpr (KIND == 0) {
    finish(DstSelf());
  } else {
    finish([&](int k, int i) -> unsigned int {
      return KIND == 1 ? eidx<K, Q>(k, opp<Lat>(i), pi.src<Lat>(opp<Lat>(i), nx, ny), plane)
                       : eidx<K, Q>(k, i, cell, plane);
    });
  }
}

template <class Lat, template <typename> class SysT, class St, int COLS>
__global__ void __launch_bounds__(COLS, BulkMode<Lat, SysT, St, COLS>::min_blocks)
    k_step_bulk(const typename St::S* __restrict__ A, typename St::S* __restrict__ B,
                const KParams<typename St::C> p) {
  bulk_step_body<Lat, SysT, St, COLS, 0>(A, B, p);
}

// In-place step of kind 1 or 2 with bulk row copies (one buffer F).
template <class Lat, template <typename> class SysT, class St, int COLS, int KIND>
__global__ void __launch_bounds__(COLS, BulkMode<Lat, SysT, St, COLS>::min_blocks)
    k_step_bulk_inplace(typename St::S* F, const KParams<typename St::C> p) {
  bulk_step_body<Lat, SysT, St, COLS, KIND>(F, F, p);
}

// Register budget per thread follows the residency the populations' staging allows.
// Blocks of COLS threads along x (COLS = 128 for register-resident kernels).  FOURIER
// compiles the manufactured forcing of a mode table in (a separate instantiation, so the
// kernels of unforced runs carry none of its code).
template <class Lat, template <typename> class SysT, class St, int MODE, int COLS, bool FOURIER = false>
__global__ void __launch_bounds__(COLS, FOURIER ? StepMode<Lat, SysT, St, COLS>::min_blocks
                                                : StepMode<Lat, SysT, St, COLS>::min_blocks_step)
    k_step(const typename St::S* __restrict__ A, typename St::S* __restrict__ B, const KParams<typename St::C> p) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const long long step = time_dependent(p) ? *p.step_ptr + p.step_rel : 0;
  if constexpr (FOURIER) {
    // the modes' time factors, shared by the block (before any thread leaves)
    __shared__ typename St::C tf[2 * MMS_MAX_MODES];
    mms_time_table(p, step, tf);
    if (x >= p.nx) return;
    step_node<Lat, SysT, St, MODE, COLS, FOURIER>(A, B, p, x, block_y<Lat>(p), block_z<Lat>(p), step,
                                                  p.mms_modes != nullptr ? tf : nullptr);
  } else {
    if (x >= p.nx) return;
    step_node<Lat, SysT, St, MODE, COLS, FOURIER>(A, B, p, x, block_y<Lat>(p), block_z<Lat>(p), step);
  }
}

// ------------------------------------------------------- pipelined per-thread staging
// Persistent variant of the per-thread staged step: the grid walks tiles of COLS nodes along
// x (row segments, x fastest) with a grid-size stride, and every thread keeps two shared-
// memory columns: it issues the copies of its node in the next tile (one cp.async group per
// tile) before it updates its node in the current one, so one node's populations are always
// in flight while the flux is evaluated.  The columns are private to their thread, so the
// pipeline needs no barrier: cp.async.wait_group 1 leaves only the newest group pending.
template <class Lat, template <typename> class SysT, class St, int COLS>
struct PipeMode {
  static constexpr size_t smem_bytes = 2 * StepMode<Lat, SysT, St, COLS>::smem_per_thread * COLS;
  static constexpr int smem_blocks = (int)(228 * 1024 / (smem_bytes + 1024));
  static constexpr int min_blocks =
      smem_blocks < 1 ? 1 : (smem_blocks * COLS > 384 ? 384 / COLS : smem_blocks);
};

__device__ __forceinline__ void stage_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void stage_wait_prev() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

template <class Lat, template <typename> class SysT, class St, int COLS>
__global__ void __launch_bounds__(COLS, PipeMode<Lat, SysT, St, COLS>::min_blocks)
    k_step_pipe(const typename St::S* __restrict__ A, typename St::S* __restrict__ B,
                const KParams<typename St::C> p) {
  using T = typename St::C;
  using S = typename St::S;
  using V = typename PairOf<S>::V;
  constexpr int K = SysT<T>::K, Q = Lat::Q, KP = K / 2;
  extern __shared__ __align__(16) unsigned char lbx_smem[];
  const int t = (int)threadIdx.x;
  const size_t stage_bytes = StepMode<Lat, SysT, St, COLS>::smem_per_thread * COLS;
  V* colv[2];
  S* colo[2];
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    V* base = reinterpret_cast<V*>(lbx_smem + s * stage_bytes);
    colv[s] = base + t;
    colo[s] = reinterpret_cast<S*>(base + KP * Q * COLS) + t;
  }
  const int tiles_x = (p.nx + COLS - 1) / COLS;
  const long long ntiles = (long long)tiles_x * p.ny * p.nz;
  const long long step = time_dependent(p) ? *p.step_ptr + p.step_rel : 0;
  auto node_of = [&](long long tl, int& x, int& y, int& z) {
    const long long row = tl / tiles_x;
    x = (int)(tl - row * tiles_x) * COLS + t;
    y = (int)(row % p.ny);
    z = (int)(row / p.ny);
  };
  auto issue = [&](long long tl, int s) {
    if (tl < ntiles) {
      int x, y, z;
      node_of(tl, x, y, z);
      if (x < p.nx) stage_node<Lat, SysT, St, COLS>(A, colv[s], colo[s], PullIdx(x, y, z, p.nx, p.ny, p.nz), p);
    }
    stage_commit();                          // an empty group past the end keeps the count uniform
  };
  long long tl = blockIdx.x;
  issue(tl, 0);
  for (int s = 0; tl < ntiles; tl += gridDim.x, s ^= 1) {
    issue(tl + gridDim.x, s ^ 1);
    stage_wait_prev();
    int x, y, z;
    node_of(tl, x, y, z);
    if (x < p.nx) {
      const unsigned int cell = ((unsigned int)z * (unsigned int)p.ny + (unsigned int)y) * (unsigned int)p.nx + x;
      V* cv = colv[s];
      S* co = colo[s];
      finish_node<Lat, SysT, St>(
          B, p, x, y, z, cell, step, true, [&](int kp, int i, T& a, T& b) { lds_pair(cv + (kp * Q + i) * COLS, a, b); },
          [&](int i) -> T { return lds_c(co + i * COLS); });
    }
  }
  stage_wait();                              // nothing stays in flight past the kernel
}

// ------------------------------------------------------------ in-place (one buffer)
// Single-buffer streaming: steps alternate between two kinds so that every node reads and
// then writes one set of addresses that no other node touches, which makes the update safe
// in place.  With i' the velocity opposite to i:
//   kind 1 (from the standard layout, F[k][i][x] = post-collision f*_i of node x): node x
//          pulls f_i(x) = F[k][i][x - c_i] and stores its post-collision f*_i into the slot it
//          emptied for the opposite direction, F[k][i'][x + c_i] (x + c_i = x - c_{i'});
//   kind 2 node x reads f_i(x) = F[k][i'][x] (its own node, swapped slots) and stores f*_i
//          in F[k][i][x], which is the standard layout again.
// A kind-1 step followed by a kind-2 step moves every population exactly as two pull steps
// between two buffers, with the same arithmetic (finish_node), so the populations after an
// even number of steps are bitwise those of the two-buffer kernels, in half the memory.

// Loads of the in-place kernels: the read-only (non-coherent) path is safe although the
// kernel writes the buffer, because every element is read only by the node that owns it,
// before that node writes it, and by no thread after.
__device__ __forceinline__ double2 ld_pair_rw(const double2* p) { return __ldg(p); }
__device__ __forceinline__ float2 ld_pair_rw(const float2* p) { return __ldg(p); }
__device__ __forceinline__ __half2 ld_pair_rw(const __half2* p) { return __ldg(p); }

template <class Lat, template <typename> class SysT, class St, int MODE, int COLS, bool FOURIER, int KIND>
__device__ __forceinline__ void step_node_inplace(typename St::S* F, const KParams<typename St::C>& p, int x,
                                                  int y, int z, long long step, const typename St::C* tfac) {
  using T = typename St::C;
  using S = typename St::S;
  using V = typename PairOf<S>::V;
  constexpr int K = SysT<T>::K, Q = Lat::Q, KP = K / 2;
  constexpr bool ODD = (K & 1) != 0;
  static_assert(opp_valid<Lat>(), "velocities must come as rest, then (+c, -c) pairs");
  const PullIdx pi(x, y, z, p.nx, p.ny, p.nz);
  const unsigned int plane = (unsigned int)p.ncell;
  const unsigned int cell = ((unsigned int)z * (unsigned int)p.ny + (unsigned int)y) * (unsigned int)p.nx + x;
  // element read as population (k, i) of this node, and element receiving its f*_i
  auto src = [&](int k, int i) -> unsigned int {
    return KIND == 1 ? eidx<K, Q>(k, i, pi.src<Lat>(i, p.nx, p.ny), plane) : eidx<K, Q>(k, opp<Lat>(i), cell, plane);
  };
  auto dst = [&](int k, int i) -> unsigned int {
    return KIND == 1 ? eidx<K, Q>(k, opp<Lat>(i), pi.src<Lat>(opp<Lat>(i), p.nx, p.ny), plane)
                     : eidx<K, Q>(k, i, cell, plane);
  };
  if constexpr (MODE == MODE_REG) {
    T fv[K][Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
#pragma unroll
      for (int kp = 0; kp < KP; ++kp)
        split(ld_pair_rw(reinterpret_cast<const V*>(F + src(2 * kp, i))), fv[2 * kp][i], fv[2 * kp + 1][i]);
      if constexpr (ODD) fv[K - 1][i] = to_c(__ldg(F + src(K - 1, i)));
    }
    finish_node<Lat, SysT, St, FOURIER>(
        F, p, x, y, z, cell, step, true,
        [&](int kp, int i, T& a, T& b) {
          a = fv[2 * kp][i];
          b = fv[2 * kp + 1][i];
        },
        [&](int i) -> T { return fv[ODD ? K - 1 : 0][i]; }, tfac, dst);
  } else {
    extern __shared__ __align__(16) unsigned char lbx_smem[];
    V* colv = reinterpret_cast<V*>(lbx_smem) + threadIdx.x;
    S* colo = reinterpret_cast<S*>(reinterpret_cast<V*>(lbx_smem) + KP * Q * COLS) + threadIdx.x;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
#pragma unroll
      for (int kp = 0; kp < KP; ++kp) stage_pair(colv + (kp * Q + i) * COLS, reinterpret_cast<const V*>(F + src(2 * kp, i)));
      if constexpr (ODD) stage(colo + i * COLS, F + src(K - 1, i));
    }
    stage_wait();
    auto get_pair = [&](int kp, int i, T& a, T& b) { lds_pair(colv + (kp * Q + i) * COLS, a, b); };
    auto get_odd = [&](int i) -> T { return lds_c(colo + i * COLS); };
    if constexpr (sizeof(S) == 2)
      finish_node<Lat, SysT, St, FOURIER>(
          F, p, x, y, z, cell, step, true, get_pair, get_odd, tfac, dst,
          [&](int kp, int i, T& a, T& b) { acc_lds_pair(colv + (kp * Q + i) * COLS, a, b); },
          [&](int i, T& a) { acc_lds_odd(colo + i * COLS, a); });
    else
      finish_node<Lat, SysT, St, FOURIER>(F, p, x, y, z, cell, step, true, get_pair, get_odd, tfac, dst);
  }
}

template <class Lat, template <typename> class SysT, class St, int MODE, int COLS, bool FOURIER, int KIND>
__global__ void __launch_bounds__(COLS, StepMode<Lat, SysT, St, COLS>::min_blocks)
    k_step_inplace(typename St::S* F, const KParams<typename St::C> p) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const long long step = time_dependent(p) ? *p.step_ptr + p.step_rel : 0;
  if constexpr (FOURIER) {
    __shared__ typename St::C tf[2 * MMS_MAX_MODES];
    mms_time_table(p, step, tf);
    if (x >= p.nx) return;
    step_node_inplace<Lat, SysT, St, MODE, COLS, FOURIER, KIND>(F, p, x, blockIdx.y, blockIdx.z, step,
                                                                 p.mms_modes != nullptr ? tf : nullptr);
  } else {
    if (x >= p.nx) return;
    step_node_inplace<Lat, SysT, St, MODE, COLS, FOURIER, KIND>(F, p, x, blockIdx.y, blockIdx.z, step, nullptr);
  }
}

// Many independent 2D grids in one persistent launch.  Instance j's populations start at
// element offset off[j] of the shared buffers; the work list holds tiles of blockDim.x
// consecutive cells (row-major, so a tile of a narrow grid spans several rows), and each
// block walks the list with a grid-size stride.
template <typename T>
struct BatchInst {
  KParams<T> p;
  long long off;
};

template <class Lat, template <typename> class SysT, class St, int MODE, bool FOURIER = false>
__global__ void k_step_batch(const typename St::S* __restrict__ A, typename St::S* __restrict__ B,
                             const BatchInst<typename St::C>* __restrict__ insts, const int2* __restrict__ tiles,
                             int ntiles, const long long* __restrict__ step_ptr, int step_rel) {
  const long long step = *step_ptr + step_rel;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int2 tl = tiles[t];
    const KParams<typename St::C> p = insts[tl.x].p;
    const long long off = insts[tl.x].off;
    const int c = tl.y + (int)threadIdx.x;
    if (c < p.ncell) {
      const int y = c / p.nx;
      step_node<Lat, SysT, St, MODE, 128, FOURIER, true>(A + off, B + off, p, c - y * p.nx, y, 0, step);
    }
  }
}

// ------------------------------------------------------------ slab faces (halo exchange)
// A slab of a larger periodic grid, cut along its last axis a (y in 2D, z in 3D) into P
// local planes, steps with the local periodic wrap along a.  In the pull layout the wrap
// makes the nodes of plane 0 read their c_a = +1 populations from the slots of plane P - 1,
// and the nodes of plane P - 1 read their c_a = -1 populations from the slots of plane 0;
// no other node reads those slots.  After a step they hold this slab's outgoing populations
// (the post-collision values leaving through the upper and the lower face), and the global
// streaming (Eq. lbe_update across the faces) needs them replaced by the lower neighbour's
// plane P - 1, c_a = +1 values and the upper neighbour's plane 0, c_a = -1 values.
// k_face copies the slots of one face between the population buffer and a contiguous face
// buffer.  Face buffer layout, for each of the NF velocities with c_a = s (lattice order):
// the component pairs [KP][plane cells] of V, then the odd component [plane cells] of S.
template <class Lat>
struct FaceVel {
  static constexpr int A = Lat::D - 1;                           // the slab axis
  static constexpr int count(int s) {
    int n = 0;
    for (int i = 0; i < Lat::Q; ++i) n += Lat::c(i, A) == s ? 1 : 0;
    return n;
  }
  static constexpr int NF = count(1);
  static_assert(NF == count(-1), "the velocity set is symmetric along the slab axis");
  // the j-th velocity (lattice order) with c_a = s
  __host__ __device__ static constexpr int nth(int j, int s) {
    for (int i = 0; i < Lat::Q; ++i)
      if (Lat::c(i, A) == s && j-- == 0) return i;
    return 0;
  }
};

// One thread per (plane cell, face velocity j); blockIdx.z selects the face: 0 = the upper
// face (plane P - 1, c_a = +1), 1 = the lower face (plane 0, c_a = -1).  PACK copies the
// population buffer's slots into the face buffers, otherwise the face buffers into the slots.
template <class Lat, template <typename> class SysT, class St, bool PACK>
__global__ void k_face(typename St::S* __restrict__ A, typename St::S* __restrict__ up,
                       typename St::S* __restrict__ dn, const KParams<typename St::C> p) {
  using S = typename St::S;
  using V = typename PairOf<S>::V;
  constexpr int K = SysT<typename St::C>::K, Q = Lat::Q, KP = K / 2, NF = FaceVel<Lat>::NF;
  const unsigned int pc = Lat::D == 3 ? (unsigned int)p.nx * (unsigned int)p.ny : (unsigned int)p.nx;
  const unsigned int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= pc) return;
  const int j = (int)blockIdx.y, face = (int)blockIdx.z;
  const int sgn = face == 0 ? 1 : -1;
  int i = 0;
#pragma unroll
  for (int jj = 0; jj < NF; ++jj)
    if (jj == j) i = FaceVel<Lat>::nth(jj, sgn);
  const unsigned int planes = Lat::D == 3 ? (unsigned int)p.nz : (unsigned int)p.ny;
  const unsigned int cell = (face == 0 ? planes - 1u : 0u) * pc + c;
  const unsigned int plane = (unsigned int)p.ncell;
  S* buf = face == 0 ? up : dn;
  V* bv = reinterpret_cast<V*>(buf);
#pragma unroll
  for (int kp = 0; kp < KP; ++kp) {
    V* g = reinterpret_cast<V*>(A + eidx<K, Q>(2 * kp, i, cell, plane));
    V* h = bv + ((size_t)j * KP + kp) * pc + c;
    if (PACK) *h = *g; else *g = *h;
  }
  if constexpr ((K & 1) != 0) {
    S* g = A + eidx<K, Q>(K - 1, i, cell, plane);
    S* h = buf + (size_t)NF * KP * pc * 2 + (size_t)j * pc + c;
    if (PACK) *h = *g; else *g = *h;
  }
}

// --------------------------------------------------------------------------- init
// One node of k_init; with `check` it also returns the node's closed-form wave-speed bound
// of the initial fields and whether every value it stored is finite.
template <class Lat, template <typename> class SysT, class St>
__device__ __forceinline__ void init_node(const double* __restrict__ Qf, typename St::S* __restrict__ A,
                                          const KParams<double>& p, const double* __restrict__ feq0,
                                          unsigned long long* maxbits, int write, int x, int y, int z, bool check,
                                          double& speed, bool& finite) {
  using Sys = SysT<double>;
  constexpr int K = Sys::K, Q = Lat::Q, D = Lat::D;
  const size_t plane = (size_t)p.ncell;
  const size_t cell = ((size_t)z * p.ny + y) * p.nx + x;
  double dQ[K];
  for (int k = 0; k < K; ++k) dQ[k] = Qf[(size_t)k * plane + cell] - p.Q0[k];
  if (check) speed = Sys::max_speed(p.prm, p.Q0, dQ);
  double Phi[K][D], Src[K];
  eval_node<SysT>(p, x, y, z, 0.0, dQ, Phi, Src);      // the initial state is at t = 0
  // destination of population i: the pull at node x reads x - c_i, so the node y = x
  // stores f_i(y + c_i); here node x writes its own f_i to x - c_i.
  int dxs[3] = {x == p.nx - 1 ? 0 : x + 1, x, x == 0 ? p.nx - 1 : x - 1};
  int dys[3] = {y == p.ny - 1 ? 0 : y + 1, y, y == 0 ? p.ny - 1 : y - 1};
  int dzs[3] = {z == p.nz - 1 ? 0 : z + 1, z, z == 0 ? p.nz - 1 : z - 1};
#pragma unroll
  for (int k = 0; k < K; ++k) {
    double lp[D];
#pragma unroll
    for (int d = 0; d < D; ++d) lp[d] = p.lc * Phi[k][d];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      // c_i . (lam/c_s^2) Phi_k: the components with c_i,d = +1 or -1 added or subtracted
      // (no products with the lattice's 0 and +-1 entries; the FP64 pipe bounds this kernel)
      double cph = 0.0;
      bool none = true;
#pragma unroll
      for (int d = 0; d < D; ++d) {
        if (Lat::c(i, d) == 1) {
          cph = none ? lp[d] : cph + lp[d];
          none = false;
        } else if (Lat::c(i, d) == -1) {
          cph = none ? -lp[d] : cph - lp[d];
          none = false;
        }
      }
      const double wd = Lat::w(i) * dQ[k];
      double v = none ? wd : fma(Lat::w(i), cph, wd);     // f^eq(Q) - f^eq(Q0)
      if (!St::SHIFT) v += feq0[k * Q + i];
      if (maxbits) atomicMax(&maxbits[k], (unsigned long long)__double_as_longlong(fabs(v)));
      if (write) {
        const size_t dst = ((size_t)dzs[Lat::c(i, 2) + 1] * p.ny + dys[Lat::c(i, 1) + 1]) * p.nx +
                           dxs[Lat::c(i, 0) + 1];
        typename St::S* o = A + eidx<K, Q>(k, i, (unsigned int)dst, (unsigned int)plane);
        if (St::SCALE) v *= p.inv_scale[k];
        if (check)
          finite = store_f64_finite(o, v) && finite;
        else
          store_f64(o, v);
      }
    }
  }
}

// Populations at the (shifted) equilibrium of Q (FP64): node x computes its equilibrium
// once and writes population i where the pull of the first step reads it, x - c_i.
// With maxbits != null it also records max |value| per component (for float16 scales).
// With chk != null it records the checks of lbx_init: chk[0] = max over nodes of the
// closed-form wave-speed bound of the initial fields (bits of a non-negative double),
// chk[1] += 1 per warp that stored a non-finite value.
template <class Lat, template <typename> class SysT, class St>
__global__ void k_init(const double* __restrict__ Qf, typename St::S* __restrict__ A,
                       const KParams<double> p, const double* __restrict__ feq0,
                       unsigned long long* maxbits, int write, int plane0, unsigned long long* chk) {
  constexpr int D = Lat::D;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  // planes plane0 .. of the last axis (the whole grid from plane0 = 0)
  const int y = (int)blockIdx.y + (D == 2 ? plane0 : 0), z = (int)blockIdx.z + (D == 3 ? plane0 : 0);
  double speed = 0.0;
  bool finite = true;
  if (x < p.nx) init_node<Lat, SysT, St>(Qf, A, p, feq0, maxbits, write, x, y, z, chk != nullptr, speed, finite);
  if (chk != nullptr) {
    // whole warps (block sizes are multiples of 32; idle lanes contribute 0 and finite)
    for (int o = 16; o > 0; o >>= 1) speed = fmax(speed, __shfl_xor_sync(0xffffffffu, speed, o));
    const bool any_bad = __any_sync(0xffffffffu, !finite);
    if ((threadIdx.x & 31) == 0) {
      atomicMax(&chk[0], (unsigned long long)__double_as_longlong(speed));
      if (any_bad) atomicAdd(&chk[1], 1ull);
    }
  }
}

// ------------------------------------------------------------------ moments / gather
// Q_k(x) = sum_i f_{k,i}(x) (+ Q0 when shifted), float64; optionally the unshifted
// pre-collision populations f_{k,i}(x) as well.
template <class Lat, template <typename> class SysT, class St>
__global__ void k_gather(const typename St::S* __restrict__ A, const KParams<double> p,
                         const double* __restrict__ feq0, double* __restrict__ Qout,
                         double* __restrict__ fout, int plane0) {
  constexpr int K = SysT<double>::K, Q = Lat::Q;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= p.nx) return;
  const int y = (int)blockIdx.y + (Lat::D == 2 ? plane0 : 0), z = (int)blockIdx.z + (Lat::D == 3 ? plane0 : 0);
  const PullIdx pi(x, y, z, p.nx, p.ny, p.nz);
  const size_t plane = (size_t)p.ncell;
  const size_t cell = ((size_t)z * p.ny + y) * p.nx + x;
  if (fout == nullptr) {
    // moments only: every component pair of a velocity in one vector load, all loads of the
    // node independent (the same per-component summation order as below)
    using V = typename PairOf<typename St::S>::V;
    constexpr int KP = K / 2;
    double sm[K];
#pragma unroll
    for (int k = 0; k < K; ++k) sm[k] = 0.0;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const unsigned int src = pi.src<Lat>(i, p.nx, p.ny);
#pragma unroll
      for (int kp = 0; kp < KP; ++kp) {
        typename St::C a, b;
        split(ldg_pair(reinterpret_cast<const V*>(A + eidx<K, Q>(2 * kp, i, src, (unsigned int)plane))), a, b);
        double va = (double)a, vb = (double)b;
        if (St::SCALE) {
          va *= p.scale[2 * kp];
          vb *= p.scale[2 * kp + 1];
        }
        sm[2 * kp] += va;
        sm[2 * kp + 1] += vb;
      }
      if constexpr ((K & 1) != 0) {
        double v = (double)ld_nc(A + eidx<K, Q>(K - 1, i, src, (unsigned int)plane));
        if (St::SCALE) v *= p.scale[K - 1];
        sm[K - 1] += v;
      }
    }
    if (Qout) {
#pragma unroll
      for (int k = 0; k < K; ++k) Qout[(size_t)k * plane + cell] = sm[k] + (St::SHIFT ? p.Q0[k] : 0.0);
    }
    return;
  }
  for (int k = 0; k < K; ++k) {
    double s = 0.0;
    for (int i = 0; i < Q; ++i) {
      double v = (double)ld_nc(A + eidx<K, Q>(k, i, pi.src<Lat>(i, p.nx, p.ny), (unsigned int)plane));
      if (St::SCALE) v *= p.scale[k];
      s += v;
      fout[((size_t)k * Q + i) * plane + cell] = v + (St::SHIFT ? feq0[k * Q + i] : 0.0);
    }
    if (Qout) Qout[(size_t)k * plane + cell] = s + (St::SHIFT ? p.Q0[k] : 0.0);
  }
}

// Store given pre-collision populations f_{k,i}(x) (float64, unshifted) into the pull
// layout: A[k][i][y] = f_{k,i}(y + c_i), shifted and scaled as the storage requires.
template <class Lat, template <typename> class SysT, class St>
__global__ void k_scatter(const double* __restrict__ fin, typename St::S* __restrict__ A,
                          const KParams<double> p, const double* __restrict__ feq0) {
  constexpr int K = SysT<double>::K, Q = Lat::Q;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= p.nx) return;
  const int y = blockIdx.y, z = blockIdx.z;
  const PullIdx pi(x, y, z, p.nx, p.ny, p.nz);
  const size_t plane = (size_t)p.ncell;
  const size_t cell = ((size_t)z * p.ny + y) * p.nx + x;
  for (int k = 0; k < K; ++k)
    for (int i = 0; i < Q; ++i) {
      double v = fin[((size_t)k * Q + i) * plane + cell] - (St::SHIFT ? feq0[k * Q + i] : 0.0);
      if (St::SCALE) v *= p.inv_scale[k];
      typename St::S* o = A + eidx<K, Q>(k, i, pi.src<Lat>(i, p.nx, p.ny), (unsigned int)plane);
      store_f64(o, v);
    }
}

// ----------------------------------------------------------------------- reductions
// Deterministic FP64 reductions over nodes.  Block b handles the fixed node set
// {b*blockDim + t + j*gridDim*blockDim}; partials[b][k][4] are then summed in block order
// by k_reduce_final.  Modes:
//   0  sums:   acc0 = sum Q_k, acc3 = count of non-finite Q_k
//   1  norms:  acc0 = sum (Q_k - R_k)^2, acc1 = sum R_k^2, acc2 = max|Q_k - R_k|, acc3 = max|R_k|
//   2  subchar: acc2[0] = max over nodes of the closed-form wave-speed bound
constexpr int RED_THREADS = 256;

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

template <class Lat, template <typename> class SysT, class St>
__global__ void __launch_bounds__(RED_THREADS) k_reduce(const typename St::S* __restrict__ A,
                                                        const KParams<double> p,
                                                        const double* __restrict__ Qref,
                                                        double* __restrict__ partials, int mode) {
  using Sys = SysT<double>;
  constexpr int K = Sys::K, Q = Lat::Q;
  double a0[K], a1[K], a2[K], a3[K];
  for (int k = 0; k < K; ++k) a0[k] = a1[k] = a2[k] = a3[k] = 0.0;
  const size_t plane = (size_t)p.ncell;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t cell = (size_t)blockIdx.x * blockDim.x + threadIdx.x; cell < plane; cell += stride) {
    // 32-bit index arithmetic (cell < plane < 2^32)
    const unsigned int c32 = (unsigned int)cell, row = c32 / (unsigned int)p.nx;
    const int x = (int)(c32 - row * (unsigned int)p.nx);
    const int y = (int)(row % (unsigned int)p.ny);
    const int z = (int)(row / (unsigned int)p.ny);
    const PullIdx pi(x, y, z, p.nx, p.ny, p.nz);
    double Qv[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      double s = 0.0;
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        double v = (double)ld_nc(A + eidx<K, Q>(k, i, pi.src<Lat>(i, p.nx, p.ny), (unsigned int)plane));
        if (St::SCALE) v *= p.scale[k];
        s += v;
      }
      Qv[k] = St::SHIFT ? s : s - p.Q0[k];     // fluctuation
    }
    if (mode == 0) {
      for (int k = 0; k < K; ++k) {
        const double q = Qv[k] + p.Q0[k];
        a0[k] += q;
        a3[k] += isfinite(q) ? 0.0 : 1.0;
      }
    } else if (mode == 1) {
      for (int k = 0; k < K; ++k) {
        const double r = Qref[(size_t)k * plane + cell];
        const double e = Qv[k] + p.Q0[k] - r;
        a0[k] += e * e;
        a1[k] += r * r;
        a2[k] = fmax(a2[k], fabs(e));
        a3[k] = fmax(a3[k], fabs(r));
      }
    } else {
      a2[0] = fmax(a2[0], Sys::max_speed(p.prm, p.Q0, Qv));
    }
  }
  __shared__ double sm[RED_THREADS / 32][4];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int k = 0; k < K; ++k) {
    double r0 = warp_sum(a0[k]), r1 = warp_sum(a1[k]);
    double r2 = warp_max(a2[k]);
    double r3 = mode == 1 ? warp_max(a3[k]) : warp_sum(a3[k]);
    if (lane == 0) {
      sm[warp][0] = r0; sm[warp][1] = r1; sm[warp][2] = r2; sm[warp][3] = r3;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double t0 = 0, t1 = 0, t2 = 0, t3 = 0;
      for (int w = 0; w < RED_THREADS / 32; ++w) {
        t0 += sm[w][0]; t1 += sm[w][1]; t2 = fmax(t2, sm[w][2]);
        t3 = mode == 1 ? fmax(t3, sm[w][3]) : t3 + sm[w][3];
      }
      double* o = partials + ((size_t)blockIdx.x * K + k) * 4;
      o[0] = t0; o[1] = t1; o[2] = t2; o[3] = t3;
    }
    __syncthreads();
  }
}

// Sum (or max) the partials of `nblk` blocks in block order: out[k][4], one thread per
// (component, statistic).
constexpr int RED_FINAL_THREADS = ((KMAX * 4 + 31) / 32) * 32;
static __global__ void k_reduce_final(const double* __restrict__ partials, int nblk, int K, int mode,
                               double* __restrict__ out) {
  const int t = threadIdx.x;
  if (t >= K * 4) return;
  const int a = t & 3;
  const bool is_max = (a == 2) || (a == 3 && mode == 1);
  double acc = 0.0;
  for (int b = 0; b < nblk; ++b) {
    const double v = partials[(size_t)b * K * 4 + t];
    acc = is_max ? fmax(acc, v) : acc + v;
  }
  out[t] = acc;
}

// Advance the device step counter after a launch sequence of n steps.
static __global__ void k_advance(long long* step, long long n) { *step += n; }

}  // namespace lbx
