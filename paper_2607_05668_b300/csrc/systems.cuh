// Per-system flux and source of dQ/dt + div Phi(Q) = S(Q) (Eq. pde_target), evaluated
// at one node in "delta form": given the background Q0 and the fluctuation dQ = Q - Q0,
// eval() returns dPhi = Phi(Q0 + dQ) - Phi(Q0) (physical units, [K][D]) and the full
// state source S(Q0 + dQ) ([K]).  Every difference is formed algebraically from the
// fluctuations (e.g. u - u0 = (dm - u0 drho)/rho), never as a difference of two large
// numbers, which is what lets the shifted float32/float16 kernels keep the fluctuation's
// precision (Sec. 2.4.3).  Gradient trackers follow Eq. gradient_advection:
// Phi_{G_{V,b}, c} = G_{V,b} u_c - delta_bc V / tau_grad, S_G = -G / tau_grad.
//
// max_speed() is a closed-form bound of the spectral radius of sum_a n_a dPhi_a/dQ over
// unit n (Sec. 2.3.2, Eq. subchar_system), used by the sub-characteristic check.
//
// Parameters arrive as a T array `p` whose layout each system documents; the host fills
// it (physical values plus derived background quantities).
//
// augment() builds the exact augmented state of a manufactured solution from the family's
// NPRIM primitive fields V and their gradients G[p][b] = dV_p/dx_b: the conserved
// components from V, the trackers from G (the gradients of their parents, or curl B).  It
// is written for a generic scalar U so that a dual number carries one derivative of every
// input through it.
#pragma once

namespace lbx {

constexpr int KMAX = 18;
constexpr int NPRM = 24;

// ------------------------------------------------------------------------------ ADR
// Sec. 3 (ADR) with the supplement's expanded form: Q = (u, G_x, G_y),
// Phi_u = u a - nu G, Phi_{G_b,c} = G_b a_c - delta_bc u/tau_g, S_u = R u (1-u), S_G = -G/tau_g.
// p: 0 a_x, 1 a_y, 2 nu, 3 R, 4 1/tau_grad
template <typename T>
struct SysADR {
  static constexpr int K = 3, NC = 1, D = 2, FAMILY = 1, NPRIM = 1;
  // primitive: u
  template <typename U>
  __host__ __device__ static void augment(const T* p, const U (&V)[NPRIM], const U (&G)[NPRIM][3], U (&Q)[K]) {
    Q[0] = V[0];
    Q[1] = G[0][0];
    Q[2] = G[0][1];
  }
  __host__ __device__ static void eval(const T* p, const T* Q0, const T* dQ, T (&dPhi)[K][D], T (&S)[K]) {
    const T a[2] = {p[0], p[1]};
    const T nu = p[2], R = p[3], itg = p[4];
    const T du = dQ[0];
    for (int d = 0; d < 2; ++d) dPhi[0][d] = a[d] * du - nu * dQ[1 + d];
    for (int b = 0; b < 2; ++b)
      for (int c = 0; c < 2; ++c) dPhi[1 + b][c] = a[c] * dQ[1 + b] - (b == c ? du * itg : T(0));
    const T u = Q0[0] + du;
    S[0] = R * u * (T(1) - u);
    S[1] = -(Q0[1] + dQ[1]) * itg;
    S[2] = -(Q0[2] + dQ[2]) * itg;
  }
  __host__ __device__ static T max_speed(const T* p, const T* Q0, const T* dQ) {
    return sqrt(p[0] * p[0] + p[1] * p[1]) + sqrt(p[2] * p[4]);
  }
};

// ------------------------------------------------------------------------------ NSF
// Compressible NSF (Sec. 3) with trackers of the primitives u, v, T:
// Q = (rho, m_x, m_y, E, G_u(2), G_v(2), G_T(2)), u = m/rho, p = (gamma-1)(E - m.u/2),
// T = p/(rho R), tau_v = mu (L + L^T - 2/3 tr L I) with L_ab = G_{u_a,b},
// Phi_m = m u + p I - tau_v, Phi_E = (E+p) u - tau_v u - kappa G_T.
// p: 0 gamma-1, 1 R, 2 mu, 3 kappa, 4 1/tau_grad, 5 u0x, 6 u0y, 7 E0+p0, 8 R T0,
//    9 tau_v0_xx, 10 tau_v0_xy, 11 tau_v0_yy, 12 gamma, 13 1/R
template <typename T>
struct SysNSF {
  static constexpr int K = 10, NC = 4, D = 2, FAMILY = 2, NPRIM = 4;
  // primitives: rho, u, v, p; E = p/(gamma-1) + rho |u|^2/2; trackers grad u, grad v and
  // grad T with T = p/(rho R): dT/dx_b = (dp/dx_b - R T drho/dx_b) / (rho R)
  template <typename U>
  __host__ __device__ static void augment(const T* p, const U (&V)[NPRIM], const U (&G)[NPRIM][3], U (&Q)[K]) {
    const U rho = V[0], u = V[1], v = V[2], pr = V[3];
    const U rR = rho * p[1], Tm = pr / rR;
    Q[0] = rho;
    Q[1] = rho * u;
    Q[2] = rho * v;
    Q[3] = pr / p[0] + U(0.5) * rho * (u * u + v * v);
    for (int b = 0; b < 2; ++b) {
      Q[4 + b] = G[1][b];
      Q[6 + b] = G[2][b];
      Q[8 + b] = (G[3][b] - p[1] * Tm * G[0][b]) / rR;
    }
  }
  __host__ __device__ static void eval(const T* p, const T* Q0, const T* dQ, T (&dPhi)[K][D], T (&S)[K]) {
    const T gm1 = p[0], mu = p[2], kap = p[3], itg = p[4];
    const T u0[2] = {p[5], p[6]};
    const T EP0 = p[7], RT0 = p[8];
    const T drho = dQ[0], rho = Q0[0] + drho, irho = T(1) / rho;
    const T dm[2] = {dQ[1], dQ[2]};
    const T m0[2] = {Q0[1], Q0[2]};
    T du[2], u[2];
    for (int a = 0; a < 2; ++a) {
      du[a] = (dm[a] - u0[a] * drho) * irho;
      u[a] = u0[a] + du[a];
    }
    const T dke = T(0.5) * (dm[0] * u[0] + dm[1] * u[1] + m0[0] * du[0] + m0[1] * du[1]);
    const T dE = dQ[3];
    const T dp = gm1 * (dE - dke);
    const T dT = (dp - RT0 * drho) * irho * p[13];
    // viscous stress of the tracker fluctuation (linear in G)
    const T L00 = dQ[4], L01 = dQ[5], L10 = dQ[6], L11 = dQ[7];
    const T dv = T(2.0 / 3.0) * (L00 + L11);
    const T dt00 = mu * (T(2) * L00 - dv), dt11 = mu * (T(2) * L11 - dv), dt01 = mu * (L01 + L10);
    const T t0[2][2] = {{p[9], p[10]}, {p[10], p[11]}};
    const T dtv[2][2] = {{dt00, dt01}, {dt01, dt11}};
    for (int b = 0; b < 2; ++b) dPhi[0][b] = dm[b];
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b)
        dPhi[1 + a][b] = dm[a] * u[b] + m0[a] * du[b] + (a == b ? dp : T(0)) - dtv[a][b];
    for (int b = 0; b < 2; ++b) {
      // (tau_v u) - (tau_v0 u0) = tau_v(dG) u + tau_v0 du
      const T tu = dtv[b][0] * u[0] + dtv[b][1] * u[1] + t0[b][0] * du[0] + t0[b][1] * du[1];
      dPhi[3][b] = (dE + dp) * u[b] + EP0 * du[b] - tu - kap * dQ[8 + b];
    }
    const T dV[3] = {du[0], du[1], dT};
    for (int v = 0; v < 3; ++v)
      for (int b = 0; b < 2; ++b) {
        const int k = 4 + 2 * v + b;
        for (int c = 0; c < 2; ++c)
          dPhi[k][c] = dQ[k] * u[c] + Q0[k] * du[c] - (b == c ? dV[v] * itg : T(0));
      }
    for (int k = 0; k < 4; ++k) S[k] = T(0);
    for (int k = 4; k < 10; ++k) S[k] = -(Q0[k] + dQ[k]) * itg;
  }
  // |u| + sqrt(c^2 + (4/3) mu/(rho tau_g) + (gamma-1) kappa/(rho R tau_g)): acoustic speed
  // combined with the relaxation speeds of the viscous and thermal tracker couplings.
  __host__ __device__ static T max_speed(const T* p, const T* Q0, const T* dQ) {
    const T rho = Q0[0] + dQ[0];
    const T ux = (Q0[1] + dQ[1]) / rho, uy = (Q0[2] + dQ[2]) / rho;
    const T pr = p[0] * ((Q0[3] + dQ[3]) - T(0.5) * rho * (ux * ux + uy * uy));
    const T c2 = p[12] * pr / rho;
    const T s2 = c2 + (T(4.0 / 3.0) * p[2] + p[0] * p[3] / p[1]) * p[4] / rho;
    return sqrt(ux * ux + uy * uy) + sqrt(s2);
  }
};

// ------------------------------------------------------------------------------ MHD
// 3D resistive MHD (Sec. 3) with a current tracker j = curl B:
// Q = (rho, m(3), B(3), E, j(3)), p = (gamma-1)(E - m.u/2 - |B|^2/2), p_t = p + |B|^2/2,
// Phi_m = m u + p_t I - B B, Phi_B[a][b] = B_a u_b - u_a B_b + eta eps_abc j_c,
// Phi_E = (E + p_t) u - B (u.B) + eta (j x B), Phi_j[a][b] = j_a u_b - eps_abc B_c/tau_g,
// S_j = -j/tau_g.
// p: 0 gamma-1, 1 eta, 2 1/tau_grad, 3..5 u0, 6 E0 + p_t0, 7 u0.B0, 8 gamma
template <typename T>
struct SysMHD {
  static constexpr int K = 11, NC = 8, D = 3, FAMILY = 3, NPRIM = 8;
  // primitives: rho, u(3), B(3), p; E = p/(gamma-1) + rho |u|^2/2 + |B|^2/2, j = curl B
  template <typename U>
  __host__ __device__ static void augment(const T* p, const U (&V)[NPRIM], const U (&G)[NPRIM][3], U (&Q)[K]) {
    const U rho = V[0];
    U ke = U(0), b2 = U(0);
    Q[0] = rho;
    for (int a = 0; a < 3; ++a) {
      Q[1 + a] = rho * V[1 + a];
      Q[4 + a] = V[4 + a];
      ke += V[1 + a] * V[1 + a];
      b2 += V[4 + a] * V[4 + a];
    }
    Q[7] = V[7] / p[0] + U(0.5) * (rho * ke + b2);
    Q[8] = G[6][1] - G[5][2];       // j_x = dB_z/dy - dB_y/dz
    Q[9] = G[4][2] - G[6][0];       // j_y = dB_x/dz - dB_z/dx
    Q[10] = G[5][0] - G[4][1];      // j_z = dB_y/dx - dB_x/dy
  }
  __host__ __device__ static constexpr int eps(int a, int b, int c) {
    return (a - b) * (b - c) * (c - a) / 2;
  }
  __host__ __device__ static void eval(const T* p, const T* Q0, const T* dQ, T (&dPhi)[K][D], T (&S)[K]) {
    const T gm1 = p[0], eta = p[1], itg = p[2];
    const T u0[3] = {p[3], p[4], p[5]};
    const T EP0 = p[6], uB0 = p[7];
    const T drho = dQ[0], rho = Q0[0] + drho, irho = T(1) / rho;
    T dm[3], m0[3], du[3], u[3], dB[3], B0[3], B[3], dj[3], j0[3], j[3];
    for (int a = 0; a < 3; ++a) {
      dm[a] = dQ[1 + a];
      m0[a] = Q0[1 + a];
      du[a] = (dm[a] - u0[a] * drho) * irho;
      u[a] = u0[a] + du[a];
      dB[a] = dQ[4 + a];
      B0[a] = Q0[4 + a];
      B[a] = B0[a] + dB[a];
      dj[a] = dQ[8 + a];
      j0[a] = Q0[8 + a];
      j[a] = j0[a] + dj[a];
    }
    const T dE = dQ[7];
    T dke = 0, dme = 0, duB = 0;
    for (int a = 0; a < 3; ++a) {
      dke += dm[a] * u[a] + m0[a] * du[a];
      dme += dB[a] * (B[a] + B0[a]);
      duB += du[a] * B[a] + u0[a] * dB[a];
    }
    dke *= T(0.5);
    dme *= T(0.5);
    const T dp = gm1 * (dE - dke - dme);
    const T dpt = dp + dme;
    const T uB = uB0 + duB;
    for (int b = 0; b < 3; ++b) dPhi[0][b] = dm[b];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        dPhi[1 + a][b] = dm[a] * u[b] + m0[a] * du[b] + (a == b ? dpt : T(0)) - (dB[a] * B[b] + B0[a] * dB[b]);
        T ej = 0, eB = 0;
        for (int c = 0; c < 3; ++c) {
          const int e = eps(a, b, c);
          if (e != 0) {
            ej += T(e) * dj[c];
            eB += T(e) * dB[c];
          }
        }
        dPhi[4 + a][b] = (dB[a] * u[b] + B0[a] * du[b]) - (du[a] * B[b] + u0[a] * dB[b]) + eta * ej;
        dPhi[8 + a][b] = dj[a] * u[b] + j0[a] * du[b] - eB * itg;
      }
    // (j x B) - (j0 x B0) = dj x B + j0 x dB
    const T jxB[3] = {dj[1] * B[2] - dj[2] * B[1] + j0[1] * dB[2] - j0[2] * dB[1],
                      dj[2] * B[0] - dj[0] * B[2] + j0[2] * dB[0] - j0[0] * dB[2],
                      dj[0] * B[1] - dj[1] * B[0] + j0[0] * dB[1] - j0[1] * dB[0]};
    for (int b = 0; b < 3; ++b)
      dPhi[7][b] = (dE + dpt) * u[b] + EP0 * du[b] - (dB[b] * uB + B0[b] * duB) + eta * jxB[b];
    for (int k = 0; k < 8; ++k) S[k] = T(0);
    for (int a = 0; a < 3; ++a) S[8 + a] = -j[a] * itg;
  }
  // |u| + sqrt(c^2 + |B|^2/rho + eta/tau_g): fast magnetosonic bound plus the
  // relaxation speed of the resistive current coupling.
  __host__ __device__ static T max_speed(const T* p, const T* Q0, const T* dQ) {
    const T rho = Q0[0] + dQ[0];
    T u2 = 0, b2 = 0;
    for (int a = 0; a < 3; ++a) {
      const T ua = (Q0[1 + a] + dQ[1 + a]) / rho, Ba = Q0[4 + a] + dQ[4 + a];
      u2 += ua * ua;
      b2 += Ba * Ba;
    }
    const T pr = p[0] * ((Q0[7] + dQ[7]) - T(0.5) * rho * u2 - T(0.5) * b2);
    return sqrt(u2) + sqrt(p[8] * pr / rho + b2 / rho + p[1] * p[2]);
  }
};

// ------------------------------------------------------------- NSF, the paper's cascade
// Compressible NSF with trackers of the conserved fields (the paper's 12-component
// cascade, Sec. 2.1.1): Q = (rho, m_x, m_y, E, G_rho(2), G_mx(2), G_my(2), G_E(2)).
// The chain rule gives L = grad u = (G_m - u (x) G_rho)/rho,
// grad p = (gamma-1)(G_E - u.G_m + |u|^2/2 G_rho), grad T = (grad p/R - T G_rho)/rho.
// In delta form (background L0, grad T0, tau_v0 from the host; zero for a uniform
// background):  rho dL = dG_m - u0 (x) dG_rho - du (x) G_rho - drho L0,
// rho d(grad T) = d(grad p)/R - T0 dG_rho - dT G_rho - drho grad T0.
// p: 0 gamma-1, 1 R, 2 mu, 3 kappa, 4 1/tau_grad, 5-6 u0, 7 E0+p0, 8 T0, 9-12 L0 (row-major),
//    13-14 grad T0, 15-17 tau_v0 (xx, xy, yy), 18 gamma
template <typename T>
struct SysNSF12 {
  static constexpr int K = 12, NC = 4, D = 2, FAMILY = 7, NPRIM = 4;
  // primitives: rho, u, v, p; trackers: gradients of rho, rho u, rho v, E
  template <typename U>
  __host__ __device__ static void augment(const T* p, const U (&V)[NPRIM], const U (&G)[NPRIM][3], U (&Q)[K]) {
    const U rho = V[0], u = V[1], v = V[2];
    Q[0] = rho;
    Q[1] = rho * u;
    Q[2] = rho * v;
    Q[3] = V[3] / p[0] + U(0.5) * rho * (u * u + v * v);
    for (int b = 0; b < 2; ++b) {
      Q[4 + b] = G[0][b];
      Q[6 + b] = G[0][b] * u + rho * G[1][b];
      Q[8 + b] = G[0][b] * v + rho * G[2][b];
      Q[10 + b] = G[3][b] / p[0] + U(0.5) * G[0][b] * (u * u + v * v) + rho * (u * G[1][b] + v * G[2][b]);
    }
  }
  __host__ __device__ static void eval(const T* p, const T* Q0, const T* dQ, T (&dPhi)[K][D], T (&S)[K]) {
    const T gm1 = p[0], R = p[1], mu = p[2], kap = p[3], itg = p[4];
    const T u0[2] = {p[5], p[6]};
    const T EP0 = p[7], T0 = p[8];
    const T drho = dQ[0], rho = Q0[0] + drho, irho = T(1) / rho;
    const T dm[2] = {dQ[1], dQ[2]}, m0[2] = {Q0[1], Q0[2]};
    T du[2], u[2];
    for (int a = 0; a < 2; ++a) {
      du[a] = (dm[a] - u0[a] * drho) * irho;
      u[a] = u0[a] + du[a];
    }
    const T dke = T(0.5) * (dm[0] * u[0] + dm[1] * u[1] + m0[0] * du[0] + m0[1] * du[1]);
    const T dE = dQ[3], dp = gm1 * (dE - dke);
    const T dT = (dp - R * T0 * drho) * irho / R;
    // trackers (full values G, fluctuations dG)
    T Gr[2], dGr[2], Gm[2][2], dGm[2][2], dGE[2];
    for (int b = 0; b < 2; ++b) {
      dGr[b] = dQ[4 + b];
      Gr[b] = Q0[4 + b] + dGr[b];
      for (int a = 0; a < 2; ++a) {
        dGm[a][b] = dQ[6 + 2 * a + b];
        Gm[a][b] = Q0[6 + 2 * a + b] + dGm[a][b];
      }
      dGE[b] = dQ[10 + b];
    }
    T dL[2][2], dGT[2];
    const T u02 = u0[0] * u0[0] + u0[1] * u0[1];
    const T duu = du[0] * (u[0] + u0[0]) + du[1] * (u[1] + u0[1]);    // |u|^2 - |u0|^2
    for (int b = 0; b < 2; ++b) {
      for (int a = 0; a < 2; ++a)
        dL[a][b] = (dGm[a][b] - u0[a] * dGr[b] - du[a] * Gr[b] - drho * p[9 + 2 * a + b]) * irho;
      const T dGp = gm1 * (dGE[b] - (du[0] * Gm[0][b] + du[1] * Gm[1][b] + u0[0] * dGm[0][b] + u0[1] * dGm[1][b]) +
                           T(0.5) * (duu * Gr[b] + u02 * dGr[b]));
      dGT[b] = (dGp / R - T0 * dGr[b] - dT * Gr[b] - drho * p[13 + b]) * irho;
    }
    const T dv = T(2.0 / 3.0) * (dL[0][0] + dL[1][1]);
    const T dt00 = mu * (T(2) * dL[0][0] - dv), dt11 = mu * (T(2) * dL[1][1] - dv), dt01 = mu * (dL[0][1] + dL[1][0]);
    const T t0[2][2] = {{p[15], p[16]}, {p[16], p[17]}};
    const T dtv[2][2] = {{dt00, dt01}, {dt01, dt11}};
    for (int b = 0; b < 2; ++b) dPhi[0][b] = dm[b];
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b)
        dPhi[1 + a][b] = dm[a] * u[b] + m0[a] * du[b] + (a == b ? dp : T(0)) - dtv[a][b];
    for (int b = 0; b < 2; ++b) {
      const T tu = dtv[b][0] * u[0] + dtv[b][1] * u[1] + t0[b][0] * du[0] + t0[b][1] * du[1];
      dPhi[3][b] = (dE + dp) * u[b] + EP0 * du[b] - tu - kap * dGT[b];
    }
    const T dV[4] = {drho, dm[0], dm[1], dE};
    for (int v = 0; v < 4; ++v)
      for (int b = 0; b < 2; ++b) {
        const int k = 4 + 2 * v + b;
        for (int c = 0; c < 2; ++c) dPhi[k][c] = dQ[k] * u[c] + Q0[k] * du[c] - (b == c ? dV[v] * itg : T(0));
      }
    for (int k = 0; k < 4; ++k) S[k] = T(0);
    for (int k = 4; k < 12; ++k) S[k] = -(Q0[k] + dQ[k]) * itg;
  }
  // |u| + sqrt(c^2 + (4/3 mu + (gamma-1) kappa/R) / (rho tau_g)), as for SysNSF.
  __host__ __device__ static T max_speed(const T* p, const T* Q0, const T* dQ) {
    const T rho = Q0[0] + dQ[0];
    const T ux = (Q0[1] + dQ[1]) / rho, uy = (Q0[2] + dQ[2]) / rho;
    const T pr = p[0] * ((Q0[3] + dQ[3]) - T(0.5) * rho * (ux * ux + uy * uy));
    const T s2 = p[18] * pr / rho + (T(4.0 / 3.0) * p[2] + p[0] * p[3] / p[1]) * p[4] / rho;
    return sqrt(ux * ux + uy * uy) + sqrt(s2);
  }
};

// ------------------------------------------------------------- MHD, the paper's cascade
// 2D viscous, heat-conducting resistive MHD with Powell cleaning (the paper's 18-component
// cascade): Q = (rho, m_x, m_y, E, B_x, B_y, G_rho(2), G_mx(2), G_my(2), G_E(2), G_Bx(2),
// G_By(2)); p = (gamma-1)(E - rho|u|^2/2 - |B|^2/2), p_t = p + |B|^2/2, T = p/rho,
// grad p = (gamma-1)(G_E - u.G_m + |u|^2/2 G_rho - B.G_B), j_z = G_{By,x} - G_{Bx,y},
// Phi_m = m u + p_t I - B B - tau_v, Phi_E = (E + p_t) u - B (u.B) - tau_v u - kappa grad T
// + eta (j x B), Phi_B = B u - u B - eta G_B, S = -(tr G_B) (0, B, u.B, u).
// p: 0 gamma-1, 1 mu, 2 kappa, 3 eta, 4 1/tau_grad, 5-6 u0, 7 E0 + p_t0, 8 u0.B0, 9 T0,
//    10-13 L0, 14-15 grad T0, 16-18 tau_v0 (xx, xy, yy), 19 gamma
template <typename T>
struct SysMHD18 {
  static constexpr int K = 18, NC = 6, D = 2, FAMILY = 8, NPRIM = 6;
  // primitives: rho, u, v, p, B_x, B_y; trackers: gradients of rho, rho u, rho v, E, B
  template <typename U>
  __host__ __device__ static void augment(const T* p, const U (&V)[NPRIM], const U (&G)[NPRIM][3], U (&Q)[K]) {
    const U rho = V[0], u = V[1], v = V[2], bx = V[4], by = V[5];
    Q[0] = rho;
    Q[1] = rho * u;
    Q[2] = rho * v;
    Q[3] = V[3] / p[0] + U(0.5) * (rho * (u * u + v * v) + bx * bx + by * by);
    Q[4] = bx;
    Q[5] = by;
    for (int b = 0; b < 2; ++b) {
      Q[6 + b] = G[0][b];
      Q[8 + b] = G[0][b] * u + rho * G[1][b];
      Q[10 + b] = G[0][b] * v + rho * G[2][b];
      Q[12 + b] = G[3][b] / p[0] + U(0.5) * G[0][b] * (u * u + v * v) + rho * (u * G[1][b] + v * G[2][b]) +
                  bx * G[4][b] + by * G[5][b];
      Q[14 + b] = G[4][b];
      Q[16 + b] = G[5][b];
    }
  }
  __host__ __device__ static void eval(const T* p, const T* Q0, const T* dQ, T (&dPhi)[K][D], T (&S)[K]) {
    const T gm1 = p[0], mu = p[1], kap = p[2], eta = p[3], itg = p[4];
    const T u0[2] = {p[5], p[6]};
    const T EPt0 = p[7], uB0 = p[8], T0 = p[9];
    const T drho = dQ[0], rho = Q0[0] + drho, irho = T(1) / rho;
    const T dm[2] = {dQ[1], dQ[2]}, m0[2] = {Q0[1], Q0[2]};
    const T dB[2] = {dQ[4], dQ[5]}, B0[2] = {Q0[4], Q0[5]};
    T du[2], u[2], B[2];
    for (int a = 0; a < 2; ++a) {
      du[a] = (dm[a] - u0[a] * drho) * irho;
      u[a] = u0[a] + du[a];
      B[a] = B0[a] + dB[a];
    }
    const T dke = T(0.5) * (dm[0] * u[0] + dm[1] * u[1] + m0[0] * du[0] + m0[1] * du[1]);
    const T dme = T(0.5) * (dB[0] * (B[0] + B0[0]) + dB[1] * (B[1] + B0[1]));
    const T dE = dQ[3];
    const T dp = gm1 * (dE - dke - dme), dpt = dp + dme;
    const T duB = du[0] * B[0] + du[1] * B[1] + u0[0] * dB[0] + u0[1] * dB[1];
    const T uB = uB0 + duB;
    const T dT = (dp - T0 * drho) * irho;
    T Gr[2], dGr[2], Gm[2][2], dGm[2][2], dGE[2], GB[2][2], dGB[2][2];
    for (int b = 0; b < 2; ++b) {
      dGr[b] = dQ[6 + b];
      Gr[b] = Q0[6 + b] + dGr[b];
      for (int a = 0; a < 2; ++a) {
        dGm[a][b] = dQ[8 + 2 * a + b];
        Gm[a][b] = Q0[8 + 2 * a + b] + dGm[a][b];
        dGB[a][b] = dQ[14 + 2 * a + b];
        GB[a][b] = Q0[14 + 2 * a + b] + dGB[a][b];
      }
      dGE[b] = dQ[12 + b];
    }
    T dL[2][2], dGT[2];
    const T u02 = u0[0] * u0[0] + u0[1] * u0[1];
    const T duu = du[0] * (u[0] + u0[0]) + du[1] * (u[1] + u0[1]);
    for (int b = 0; b < 2; ++b) {
      for (int a = 0; a < 2; ++a)
        dL[a][b] = (dGm[a][b] - u0[a] * dGr[b] - du[a] * Gr[b] - drho * p[10 + 2 * a + b]) * irho;
      const T dGp = gm1 * (dGE[b] - (du[0] * Gm[0][b] + du[1] * Gm[1][b] + u0[0] * dGm[0][b] + u0[1] * dGm[1][b]) +
                           T(0.5) * (duu * Gr[b] + u02 * dGr[b]) -
                           (dB[0] * GB[0][b] + dB[1] * GB[1][b] + B0[0] * dGB[0][b] + B0[1] * dGB[1][b]));
      dGT[b] = (dGp - T0 * dGr[b] - dT * Gr[b] - drho * p[14 + b]) * irho;
    }
    const T dv = T(2.0 / 3.0) * (dL[0][0] + dL[1][1]);
    const T dt00 = mu * (T(2) * dL[0][0] - dv), dt11 = mu * (T(2) * dL[1][1] - dv), dt01 = mu * (dL[0][1] + dL[1][0]);
    const T t0[2][2] = {{p[16], p[17]}, {p[17], p[18]}};
    const T dtv[2][2] = {{dt00, dt01}, {dt01, dt11}};
    // j x B - j0 x B0 with j_z = G_{By,x} - G_{Bx,y}
    const T jz0 = Q0[16] - Q0[15], djz = dGB[1][0] - dGB[0][1], jz = jz0 + djz;
    const T djxB[2] = {-(djz * B[1] + jz0 * dB[1]), djz * B[0] + jz0 * dB[0]};
    (void)jz;
    for (int b = 0; b < 2; ++b) dPhi[0][b] = dm[b];
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b)
        dPhi[1 + a][b] = dm[a] * u[b] + m0[a] * du[b] + (a == b ? dpt : T(0)) - (dB[a] * B[b] + B0[a] * dB[b]) -
                         dtv[a][b];
    for (int b = 0; b < 2; ++b) {
      const T tu = dtv[b][0] * u[0] + dtv[b][1] * u[1] + t0[b][0] * du[0] + t0[b][1] * du[1];
      dPhi[3][b] = (dE + dpt) * u[b] + EPt0 * du[b] - (dB[b] * uB + B0[b] * duB) - tu - kap * dGT[b] + eta * djxB[b];
    }
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b)
        dPhi[4 + a][b] = (dB[a] * u[b] + B0[a] * du[b]) - (du[a] * B[b] + u0[a] * dB[b]) - eta * dGB[a][b];
    const T dV[6] = {drho, dm[0], dm[1], dE, dB[0], dB[1]};
    for (int v = 0; v < 6; ++v)
      for (int b = 0; b < 2; ++b) {
        const int k = 6 + 2 * v + b;
        for (int c = 0; c < 2; ++c) dPhi[k][c] = dQ[k] * u[c] + Q0[k] * du[c] - (b == c ? dV[v] * itg : T(0));
      }
    const T divB = GB[0][0] + GB[1][1];
    S[0] = T(0);
    S[1] = -divB * B[0];
    S[2] = -divB * B[1];
    S[3] = -divB * uB;
    S[4] = -divB * u[0];
    S[5] = -divB * u[1];
    for (int k = 6; k < 18; ++k) S[k] = -(Q0[k] + dQ[k]) * itg;
  }
  // |u| + sqrt(c^2 + |B|^2/rho + (4/3 mu + (gamma-1) kappa)/(rho tau_g) + eta/tau_g): fast
  // magnetosonic speed plus the relaxation speeds of the viscous, thermal and resistive
  // tracker couplings.
  __host__ __device__ static T max_speed(const T* p, const T* Q0, const T* dQ) {
    const T rho = Q0[0] + dQ[0];
    const T ux = (Q0[1] + dQ[1]) / rho, uy = (Q0[2] + dQ[2]) / rho;
    const T bx = Q0[4] + dQ[4], by = Q0[5] + dQ[5];
    const T b2 = bx * bx + by * by;
    const T pr = p[0] * ((Q0[3] + dQ[3]) - T(0.5) * rho * (ux * ux + uy * uy) - T(0.5) * b2);
    const T s2 = p[19] * pr / rho + b2 / rho + (T(4.0 / 3.0) * p[1] + p[0] * p[2]) * p[4] / rho + p[3] * p[4];
    return sqrt(ux * ux + uy * uy) + sqrt(s2);
  }
};

// -------------------------------------------------------------------------- Burgers
// Sec. 3 (inviscid Burgers): Phi = (u^2/2, u^2/2).  No parameters.
template <typename T>
struct SysBurgers {
  static constexpr int K = 1, NC = 1, D = 2, FAMILY = 4, NPRIM = 1;
  template <typename U>
  __host__ __device__ static void augment(const T* p, const U (&V)[NPRIM], const U (&G)[NPRIM][3], U (&Q)[K]) {
    Q[0] = V[0];
  }
  __host__ __device__ static void eval(const T* p, const T* Q0, const T* dQ, T (&dPhi)[K][D], T (&S)[K]) {
    const T h = T(0.5) * dQ[0] * (T(2) * Q0[0] + dQ[0]);
    dPhi[0][0] = h;
    dPhi[0][1] = h;
    S[0] = T(0);
  }
  __host__ __device__ static T max_speed(const T* p, const T* Q0, const T* dQ) {
    return T(1.4142135623730951) * fabs(Q0[0] + dQ[0]);
  }
};

// ---------------------------------------------------------------------------- Euler
// Sec. 3 (compressible Euler).  p: 0 gamma-1, 1 u0x, 2 u0y, 3 E0+p0, 4 gamma
template <typename T>
struct SysEuler {
  static constexpr int K = 4, NC = 4, D = 2, FAMILY = 5, NPRIM = 4;
  // primitives: rho, u, v, p; E = p/(gamma-1) + rho |u|^2/2
  template <typename U>
  __host__ __device__ static void augment(const T* p, const U (&V)[NPRIM], const U (&G)[NPRIM][3], U (&Q)[K]) {
    const U rho = V[0], u = V[1], v = V[2];
    Q[0] = rho;
    Q[1] = rho * u;
    Q[2] = rho * v;
    Q[3] = V[3] / p[0] + U(0.5) * rho * (u * u + v * v);
  }
  __host__ __device__ static void eval(const T* p, const T* Q0, const T* dQ, T (&dPhi)[K][D], T (&S)[K]) {
    const T gm1 = p[0];
    const T u0[2] = {p[1], p[2]};
    const T drho = dQ[0], irho = T(1) / (Q0[0] + drho);
    const T dm[2] = {dQ[1], dQ[2]}, m0[2] = {Q0[1], Q0[2]};
    T du[2], u[2];
    for (int a = 0; a < 2; ++a) {
      du[a] = (dm[a] - u0[a] * drho) * irho;
      u[a] = u0[a] + du[a];
    }
    const T dke = T(0.5) * (dm[0] * u[0] + dm[1] * u[1] + m0[0] * du[0] + m0[1] * du[1]);
    const T dE = dQ[3], dp = gm1 * (dE - dke);
    for (int b = 0; b < 2; ++b) {
      dPhi[0][b] = dm[b];
      dPhi[1][b] = dm[0] * u[b] + m0[0] * du[b] + (b == 0 ? dp : T(0));
      dPhi[2][b] = dm[1] * u[b] + m0[1] * du[b] + (b == 1 ? dp : T(0));
      dPhi[3][b] = (dE + dp) * u[b] + p[3] * du[b];
    }
    for (int k = 0; k < 4; ++k) S[k] = T(0);
  }
  __host__ __device__ static T max_speed(const T* p, const T* Q0, const T* dQ) {
    const T rho = Q0[0] + dQ[0];
    const T ux = (Q0[1] + dQ[1]) / rho, uy = (Q0[2] + dQ[2]) / rho;
    const T pr = p[0] * ((Q0[3] + dQ[3]) - T(0.5) * rho * (ux * ux + uy * uy));
    return sqrt(ux * ux + uy * uy) + sqrt(p[4] * pr / rho);
  }
};

// ------------------------------------------------------------------------ Maxwell TM
// Sec. 3 (Maxwell TM): Q = (E_z, H_x, H_y), Phi = c((-H_y, H_x), (0, E_z), (-E_z, 0)).
// p: 0 c
template <typename T>
struct SysMaxwell {
  static constexpr int K = 3, NC = 3, D = 2, FAMILY = 6, NPRIM = 3;
  template <typename U>
  __host__ __device__ static void augment(const T* p, const U (&V)[NPRIM], const U (&G)[NPRIM][3], U (&Q)[K]) {
    for (int k = 0; k < 3; ++k) Q[k] = V[k];
  }
  __host__ __device__ static void eval(const T* p, const T* Q0, const T* dQ, T (&dPhi)[K][D], T (&S)[K]) {
    const T c = p[0];
    dPhi[0][0] = -c * dQ[2];
    dPhi[0][1] = c * dQ[1];
    dPhi[1][0] = T(0);
    dPhi[1][1] = c * dQ[0];
    dPhi[2][0] = -c * dQ[0];
    dPhi[2][1] = T(0);
    S[0] = S[1] = S[2] = T(0);
  }
  __host__ __device__ static T max_speed(const T* p, const T* Q0, const T* dQ) { return fabs(p[0]); }
};

// ------------------------------------------------------ homogenized NSF (3D, prescribed)
// 3D homogenized compressible NSF (Sec. 3, HCNSF): porosity alpha(x, t) and solid velocity
// u_s(x, t) are prescribed coefficient fields, passed per node as cf = (alpha, u_s).
// Q = (rho, m(3), E, G_11, G_22, G_T(3), G_00, G_01, G_02, G_12) in the paper's order, G the
// tracked symmetric velocity gradient and G_T the tracked grad T, T = p/rho (gas constant 1):
// tau_v = mu (2 G - 2/3 tr(G) I), Phi_m = m u + p I - alpha tau_v,
// Phi_E = (E + p) u - alpha tau_v u - alpha kappa G_T,
// Phi_{G_ab, c} = G_ab u_c - (delta_ac u_b + delta_bc u_a)/(2 tau_grad),
// Phi_{G_T,b, c} = G_T,b u_c - delta_bc T/tau_grad,
// S_m = (1-alpha)/eta (rho u_s - m), S_E = S_m . u, S_G = -G/tau_grad.
// The background's tracker components are zero (checked by the host), so alpha never
// multiplies a background quantity and Phi(Q0) is the same at every node.
// p: 0 gamma-1, 1 mu, 2 kappa, 3 1/eta, 4 1/tau_grad, 5-7 u0, 8 E0+p0, 9 T0, 10 gamma
template <typename T>
struct SysHCNSF {
  static constexpr int K = 14, NC = 5, D = 3, FAMILY = 9, NPRIM = 5, NCF = 4;
  // position in Q of the symmetric-gradient component (a, b)
  __host__ __device__ static constexpr int gidx(int a, int b) {
    return a > b ? gidx(b, a) : (a == b ? (a == 0 ? 10 : 4 + a) : (a == 0 ? 10 + b : 13));
  }
  // primitives: rho, u_x, u_y, u_z, p
  template <typename U>
  __host__ __device__ static void augment(const T* p, const U (&V)[NPRIM], const U (&G)[NPRIM][3], U (&Q)[K]) {
    const U rho = V[0];
    Q[0] = rho;
    U ke = U(0);
    for (int a = 0; a < 3; ++a) {
      Q[1 + a] = rho * V[1 + a];
      ke = ke + V[1 + a] * V[1 + a];
    }
    Q[4] = V[4] / p[0] + U(0.5) * rho * ke;
    for (int a = 0; a < 3; ++a)
      for (int b = a; b < 3; ++b) Q[gidx(a, b)] = U(0.5) * (G[1 + a][b] + G[1 + b][a]);
    const U Tm = V[4] / rho;
    for (int b = 0; b < 3; ++b) Q[7 + b] = (G[4][b] - Tm * G[0][b]) / rho;
  }
  // cf: the prescribed fields in the flux; cs: those in the drag source (the same values
  // unless the source takes them at another time level)
  template <typename CF>
  __host__ __device__ static void eval(const T* p, const T* Q0, const T* dQ, T (&dPhi)[K][D], T (&S)[K],
                                       const CF (&cf)[NCF], const CF (&cs)[NCF]) {
    const T gm1 = p[0], mu = p[1], kap = p[2], ieta = p[3], itg = p[4];
    const T EP0 = p[8], T0 = p[9];
    const T alpha = cf[0];
    const T drho = dQ[0], rho = Q0[0] + drho, irho = T(1) / rho;
    T dm[3], m0[3], du[3], u[3];
    for (int a = 0; a < 3; ++a) {
      dm[a] = dQ[1 + a];
      m0[a] = Q0[1 + a];
      du[a] = (dm[a] - p[5 + a] * drho) * irho;
      u[a] = p[5 + a] + du[a];
    }
    const T dke = T(0.5) * (dm[0] * u[0] + dm[1] * u[1] + dm[2] * u[2] + m0[0] * du[0] + m0[1] * du[1] + m0[2] * du[2]);
    const T dE = dQ[4], dp = gm1 * (dE - dke);
    const T dT = (dp - T0 * drho) * irho;
    T G[3][3];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) G[a][b] = dQ[gidx(a, b)];
    const T tr3 = T(2.0 / 3.0) * (G[0][0] + G[1][1] + G[2][2]);
    T atv[3][3];                                    // alpha tau_v
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) atv[a][b] = alpha * mu * (T(2) * G[a][b] - (a == b ? tr3 : T(0)));
    for (int b = 0; b < 3; ++b) dPhi[0][b] = dm[b];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b)
        dPhi[1 + a][b] = dm[a] * u[b] + m0[a] * du[b] + (a == b ? dp : T(0)) - atv[a][b];
    for (int b = 0; b < 3; ++b)
      dPhi[4][b] = (dE + dp) * u[b] + EP0 * du[b] - (atv[b][0] * u[0] + atv[b][1] * u[1] + atv[b][2] * u[2]) -
                   alpha * kap * dQ[7 + b];
    const T hitg = T(0.5) * itg;
    for (int a = 0; a < 3; ++a)
      for (int b = a; b < 3; ++b) {
        const int k = gidx(a, b);
        for (int c = 0; c < 3; ++c)
          dPhi[k][c] = dQ[k] * u[c] - ((a == c ? du[b] : T(0)) + (b == c ? du[a] : T(0))) * hitg;
      }
    for (int b = 0; b < 3; ++b)
      for (int c = 0; c < 3; ++c) dPhi[7 + b][c] = dQ[7 + b] * u[c] - (b == c ? dT * itg : T(0));
    const T drag = (T(1) - cs[0]) * ieta;
    S[0] = T(0);
    for (int a = 0; a < 3; ++a) S[1 + a] = drag * rho * (cs[1 + a] - u[a]);
    S[4] = S[1] * u[0] + S[2] * u[1] + S[3] * u[2];
    for (int k = 5; k < K; ++k) S[k] = -(Q0[k] + dQ[k]) * itg;
  }
  // |u| + sqrt(c^2 + (4/3 mu + (gamma-1) kappa) / (rho tau_g)), the NSF bound at alpha = 1
  // (alpha <= 1 only scales the dissipative terms down).
  __host__ __device__ static T max_speed(const T* p, const T* Q0, const T* dQ) {
    const T rho = Q0[0] + dQ[0];
    T u2 = T(0);
    for (int a = 0; a < 3; ++a) {
      const T ua = (Q0[1 + a] + dQ[1 + a]) / rho;
      u2 += ua * ua;
    }
    const T pr = p[0] * ((Q0[4] + dQ[4]) - T(0.5) * rho * u2);
    const T s2 = p[10] * pr / rho + (T(4.0 / 3.0) * p[1] + p[0] * p[2]) * p[4] / rho;
    return sqrt(u2) + sqrt(s2);
  }
};

// Number of prescribed coefficient values a family's eval() takes per node (0: none).
template <class S, class = void>
struct NcfOf {
  static constexpr int value = 0;
};
template <class S>
struct NcfOf<S, decltype(void(S::NCF))> {
  static constexpr int value = S::NCF;
};

}  // namespace lbx
