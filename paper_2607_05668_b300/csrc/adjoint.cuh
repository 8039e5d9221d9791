// Discrete adjoint of the collide-and-stream step (reverse sweep kernels).
//
// Forward, in the pull layout: A_{n+1}[k][j][x] = P_{k,j}(g(x)), g_{k,i}(x) = A_n[k][i][x - c_i],
//   P_{k,j} = g_{k,j} + w_k (f^eq_{k,j}(Q) - g_{k,j}) + dt w_j S_k(Q),  Q_k = sum_i g_{k,i}
// (Eq. lbe_update; w_k = 1/tau_k).  With Lam_n = dJ/dA_n and mu_{k,j}(x) = Lam_{n+1}[k][j][x]:
//   Lam_n[k][i][x - c_i] = (1 - w_k) mu_{k,i}(x) + h_k(x),
//   h_k = w_k m0_k + d/dQ_k sum_k' [ w_k' (lam/c_s^2) m1_k' . Phi_k'(Q) + dt m0_k' S_k'(Q) ],
//   m0_k = sum_j w_j mu_{k,j},  m1_k = sum_j w_j c_j mu_{k,j}   (lattice weights w_j),
// because df^eq_{k',j}/dQ_k = w_j (delta_kk' + (lam/c_s^2) c_j . dPhi_k'/dQ_k) (Eq. feq) and
// dQ_k/dg_{k,i} = 1 (Eq. moments).  The node-local derivative of the flux and source is
// taken in forward mode (dual numbers with several tangents) through the same delta-form
// system code the step uses.  The relaxation-time derivative per node is
// sum_{k conserved, j} mu_{k,j} (g_{k,j} - f^eq_{k,j}), to be divided by tau^2.
#pragma once

#include "kernels.cuh"

namespace lbx {

// Tangent directions per evaluation of the flux in adj_vjp.  Reverse sweep of NSF D2Q9 at
// 256^2 over 2000 steps, FP32: 44.2 ms with one tangent per evaluation (K evaluations),
// 39.4 ms with 2, 37.2 ms with 5, 47.0 ms with all 10 (register pressure).  Capping the
// registers for 4 or 5 resident blocks spilled and measured slower still, and so did taking
// the flux values from the first evaluation instead of a separate one (42.4 ms: they stay
// live across the chunks).
constexpr int ADJ_TANGENTS = 5;

// One chunk of adj_vjp: tangent directions C0 .. C0+N-1 (compile-time unit seeds) in one
// evaluation of the system code, then the next chunk.
template <class Lat, template <typename> class SysT, typename T, int C0>
__device__ __forceinline__ void adj_vjp_chunk(const KParams<T>& p, const T* dQ, const T (&m0)[SysT<T>::K],
                                              const T (&m1)[SysT<T>::K][Lat::D], const T* omega, T lc, T dt,
                                              T (&grad)[SysT<T>::K]) {
  constexpr int K = SysT<T>::K, D = Lat::D;
  constexpr int N = K - C0 < ADJ_TANGENTS ? K - C0 : ADJ_TANGENTS;
  using DN = DualN<T, N>;
  using SysD = SysT<DN>;
  DN pd[NPRM], q0[KMAX], x[K];
#pragma unroll
  for (int i = 0; i < NPRM; ++i) pd[i] = DN(p.prm[i]);
#pragma unroll
  for (int k = 0; k < K; ++k) {
    q0[k] = DN(p.Q0[k]);
    x[k] = DN(dQ[k]);
    if (k >= C0 && k < C0 + N) x[k].d[k - C0] = T(1);
  }
  DN Phi[K][D], S[K];
  SysD::eval(pd, q0, x, Phi, S);
#pragma unroll
  for (int j = 0; j < N; ++j) {
    T acc = T(0);
#pragma unroll
    for (int k = 0; k < K; ++k) {
      T a = T(0);
#pragma unroll
      for (int d = 0; d < D; ++d) a += m1[k][d] * Phi[k][d].d[j];
      acc += omega[k] * lc * a + dt * m0[k] * S[k].d[j];
    }
    grad[C0 + j] = acc;
  }
  if constexpr (C0 + N < K) adj_vjp_chunk<Lat, SysT, T, C0 + N>(p, dQ, m0, m1, omega, lc, dt, grad);
}

// h_k of the header at one node: w_k m0_k + gradient of
// F(Q) = sum_k' w_k' lc m1_k' . Phi_k'(Q) + dt m0_k' S_k'(Q) with respect to Q (delta form:
// Q = Q0 + dQ, the derivative with respect to dQ is the same), in forward mode: the K unit
// directions in chunks of ADJ_TANGENTS tangents per evaluation.
template <class Lat, template <typename> class SysT, typename T>
__device__ __forceinline__ void adj_vjp(const KParams<T>& p, const T* dQ, const T (&m0)[SysT<T>::K],
                                        const T (&m1)[SysT<T>::K][Lat::D], const T* omega, T lc, T dt,
                                        T (&grad)[SysT<T>::K]) {
  adj_vjp_chunk<Lat, SysT, T, 0>(p, dQ, m0, m1, omega, lc, dt, grad);
}

// One reverse step.  An: forward buffer before step n (storage type).  Lnext = Lam_{n+1},
// Lout = Lam_n (compute type, same [k][i][cell] layout).  tau_acc[cell] += the node's
// relaxation-time term (float64, one owner per node: deterministic).
template <class Lat, template <typename> class SysT, class St>
__global__ void __launch_bounds__(128) k_adj_step(const typename St::S* __restrict__ An,
                                                  const typename St::C* __restrict__ Lnext,
                                                  typename St::C* __restrict__ Lout, const KParams<typename St::C> p,
                                                  double* __restrict__ tau_acc) {
  using T = typename St::C;
  using Sys = SysT<T>;
  constexpr int K = Sys::K, NC = Sys::NC, Q = Lat::Q, D = Lat::D;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= p.nx) return;
  const int y = blockIdx.y, z = blockIdx.z;
  const PullIdx pi(x, y, z, p.nx, p.ny, p.nz);
  const size_t plane = (size_t)p.ncell;
  const size_t cell = ((size_t)z * p.ny + y) * p.nx + x;
  // forward moments of the pre-collision state
  T X[K];
#pragma unroll
  for (int k = 0; k < K; ++k) X[k] = T(0);
#pragma unroll
  for (int i = 0; i < Q; ++i)
#pragma unroll
    for (int k = 0; k < K; ++k) X[k] += (T)ld_nc(An + eidx<K, Q>(k, i, pi.src<Lat>(i, p.nx, p.ny), (unsigned int)plane));
  T dQ[K];
#pragma unroll
  for (int k = 0; k < K; ++k) dQ[k] = St::SHIFT ? X[k] : X[k] - p.Q0[k];
  T Phi[K][D], Src[K];
  Sys::eval(p.prm, p.Q0, dQ, Phi, Src);
  // moments of the incoming adjoint
  T m0[K], m1[K][D];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    m0[k] = T(0);
#pragma unroll
    for (int d = 0; d < D; ++d) m1[k][d] = T(0);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const T mu = Lnext[((size_t)k * Q + i) * plane + cell];
      const T wm = weight<Lat, T>(i) * mu;
      m0[k] += wm;
#pragma unroll
      for (int d = 0; d < D; ++d) {
        if (Lat::c(i, d) == 1) m1[k][d] += wm;
        if (Lat::c(i, d) == -1) m1[k][d] -= wm;
      }
    }
  }
  T grad[K];
  adj_vjp<Lat, SysT, T>(p, dQ, m0, m1, p.omega, p.lc, p.dt, grad);
  // outputs and the relaxation-time term
  T tacc = T(0);
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const T om = p.omega[k];
    const T h = om * m0[k] + grad[k];
    T ph[D];
#pragma unroll
    for (int d = 0; d < D; ++d) ph[d] = p.lc * Phi[k][d] + (St::SHIFT ? T(0) : p.F0l[k][d]);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const T mu = ld_again(Lnext + ((size_t)k * Q + i) * plane + cell);
      Lout[((size_t)k * Q + i) * plane + pi.src<Lat>(i, p.nx, p.ny)] = (T(1) - om) * mu + h;
      if (k < NC) {
        T cph = T(0);
#pragma unroll
        for (int d = 0; d < D; ++d) {
          if (Lat::c(i, d) == 1) cph += ph[d];
          if (Lat::c(i, d) == -1) cph -= ph[d];
        }
        const T feq = weight<Lat, T>(i) * (X[k] + cph);
        const T g = (T)ld_again(An + eidx<K, Q>(k, i, pi.src<Lat>(i, p.nx, p.ny), (unsigned int)plane));
        tacc += mu * (g - feq);
      }
    }
  }
  tau_acc[cell] += (double)tacc;
}

// Seed of the reverse sweep for J = 1/2 sum_x (rho(x) - rho*(x))^2: Lam_N[0][i][x - c_i] =
// rho(x) - rho*(x) for every i, all other components 0.  rho from the forward buffer AN.
template <class Lat, template <typename> class SysT, class St>
__global__ void k_adj_seed(const typename St::S* __restrict__ AN, const double* __restrict__ target,
                           typename St::C* __restrict__ L, const KParams<double> p) {
  using T = typename St::C;
  constexpr int K = SysT<double>::K, Q = Lat::Q;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= p.nx) return;
  const int y = blockIdx.y, z = blockIdx.z;
  const PullIdx pi(x, y, z, p.nx, p.ny, p.nz);
  const size_t plane = (size_t)p.ncell;
  const size_t cell = ((size_t)z * p.ny + y) * p.nx + x;
  double rho = St::SHIFT ? p.Q0[0] : 0.0;
  for (int i = 0; i < Q; ++i) {
    double v = (double)ld_nc(AN + eidx<K, Q>(0, i, pi.src<Lat>(i, p.nx, p.ny), (unsigned int)plane));
    rho += v;
  }
  const T r = (T)(rho - target[cell]);
  for (int k = 0; k < K; ++k)
    for (int i = 0; i < Q; ++i) L[((size_t)k * Q + i) * plane + pi.src<Lat>(i, p.nx, p.ny)] = k == 0 ? r : T(0);
}

// Gradient with respect to the initial fields: the populations start at f^eq(Q_init(x))
// stored at x - c_i, so dJ/dQ_k(x) = m0_k + sum_k' lc m1_k' . dPhi_k'/dQ_k with mu pulled from
// Lam_0 at x - c_i (float64 evaluation at Q_init(x), like the init).
template <class Lat, template <typename> class SysT, class St>
__global__ void k_adj_init(const typename St::C* __restrict__ L0, const double* __restrict__ Qinit,
                           const KParams<double> p, double* __restrict__ dJdQ) {
  constexpr int K = SysT<double>::K, Q = Lat::Q, D = Lat::D;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= p.nx) return;
  const int y = blockIdx.y, z = blockIdx.z;
  const PullIdx pi(x, y, z, p.nx, p.ny, p.nz);
  const size_t plane = (size_t)p.ncell;
  const size_t cell = ((size_t)z * p.ny + y) * p.nx + x;
  double m0[K], m1[K][D], dQ[K], zero[K], grad[K];
  for (int k = 0; k < K; ++k) {
    m0[k] = 0.0;
    zero[k] = 0.0;
    for (int d = 0; d < D; ++d) m1[k][d] = 0.0;
    for (int i = 0; i < Q; ++i) {
      const double wm = Lat::w(i) * (double)L0[((size_t)k * Q + i) * plane + pi.src<Lat>(i, p.nx, p.ny)];
      m0[k] += wm;
      for (int d = 0; d < D; ++d) m1[k][d] += Lat::c(i, d) * wm;
    }
    dQ[k] = Qinit[(size_t)k * plane + cell] - p.Q0[k];
  }
  // the step's h with unit relaxation weights and no source term: F = sum_k' lc m1_k' . Phi_k'
  double ones[KMAX];
  for (int k = 0; k < K; ++k) ones[k] = 1.0;
  adj_vjp<Lat, SysT, double>(p, dQ, zero, m1, ones, p.lc, 0.0, grad);
  for (int k = 0; k < K; ++k) dJdQ[(size_t)k * plane + cell] = m0[k] + grad[k];
}

// Slab faces of an adjoint buffer L[k][i][cell] (compute type): the slots k_face moves for
// the populations (upper face: plane P - 1, c_a = +1; lower face: plane 0, c_a = -1).  The
// reverse step writes Lam_n at x - c_i, so with the local periodic wrap the nodes of plane 0
// write the lower neighbour's plane P - 1, c_a = +1 values into this slab's upper-face slots
// and the nodes of plane P - 1 write the upper neighbour's plane 0, c_a = -1 values into the
// lower-face slots: after each reverse step the transport runs opposite to the forward
// exchange.  One thread per (plane cell, face velocity j); blockIdx.z selects the face.
// Face buffer layout: [NF velocities][K][plane cells].
template <class Lat, template <typename> class SysT, typename T, bool PACK>
__global__ void k_adj_face(T* __restrict__ L, T* __restrict__ up, T* __restrict__ dn, int nx, int ny, int nz) {
  constexpr int K = SysT<T>::K, Q = Lat::Q, NF = FaceVel<Lat>::NF;
  const unsigned int pc = Lat::D == 3 ? (unsigned int)nx * (unsigned int)ny : (unsigned int)nx;
  const unsigned int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= pc) return;
  const int j = (int)blockIdx.y, face = (int)blockIdx.z;
  const int sgn = face == 0 ? 1 : -1;
  int i = 0;
#pragma unroll
  for (int jj = 0; jj < NF; ++jj)
    if (jj == j) i = FaceVel<Lat>::nth(jj, sgn);
  const unsigned int planes = Lat::D == 3 ? (unsigned int)nz : (unsigned int)ny;
  const size_t ncell = (size_t)pc * planes;
  const size_t cell = (size_t)(face == 0 ? planes - 1u : 0u) * pc + c;
  T* buf = face == 0 ? up : dn;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    T* g = L + ((size_t)k * Q + i) * ncell + cell;
    T* h = buf + ((size_t)j * K + k) * pc + c;
    if (PACK) *h = *g; else *g = *h;
  }
}

}  // namespace lbx
