// Host side of the C ABI declared in include/lbx.h: handles, parameter packing,
// dispatch over (system family, lattice, storage) and launches of the kernels in
// kernels.cuh.  Every entry point reports failures as an lbx_status with a message in
// lbx_last_error(); none aborts.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "lbx.h"
#include "kernels.cuh"
#include "lbx_internal.h"

using namespace lbx;

// ------------------------------------------------------------------------------ errors
static thread_local std::string g_err;

lbx_status lbx::fail(lbx_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

extern "C" const char* lbx_last_error(void) { return g_err.c_str(); }
extern "C" int lbx_version(void) { return 100; }

static_assert(lbx::MMS_MAX_MODES == LBX_MMS_MAX_MODES, "device mode-table bound");

// ------------------------------------------------------------------------- systems
static int family_K(int f) {
  switch (f) {
    case LBX_ADR_CASCADE: return 3;
    case LBX_NSF_PRIM_TRACK: return 10;
    case LBX_MHD_J_TRACK: return 11;
    case LBX_BURGERS: return 1;
    case LBX_EULER: return 4;
    case LBX_MAXWELL_TM: return 3;
    case LBX_NSF_CONS_TRACK: return 12;
    case LBX_MHD_POWELL_2D: return 18;
    case LBX_HCNSF_3D: return 14;
  }
  return 0;
}
static int family_NC(int f) {
  switch (f) {
    case LBX_ADR_CASCADE: return 1;
    case LBX_NSF_PRIM_TRACK: return 4;
    case LBX_MHD_J_TRACK: return 8;
    case LBX_NSF_CONS_TRACK: return 4;
    case LBX_MHD_POWELL_2D: return 6;
    case LBX_HCNSF_3D: return 5;
    default: return family_K(f);
  }
}
static int family_D(int f) { return (f == LBX_MHD_J_TRACK || f == LBX_HCNSF_3D) ? 3 : 2; }
// Primitive fields of a FOURIER manufactured solution (lbx_mms).
static int family_nprim(int f) {
  switch (f) {
    case LBX_ADR_CASCADE: return 1;
    case LBX_NSF_PRIM_TRACK: return 4;
    case LBX_MHD_J_TRACK: return 8;
    case LBX_BURGERS: return 1;
    case LBX_EULER: return 4;
    case LBX_MAXWELL_TM: return 3;
    case LBX_NSF_CONS_TRACK: return 4;
    case LBX_MHD_POWELL_2D: return 6;
    case LBX_HCNSF_3D: return 5;
  }
  return 0;
}

static const char* NAMES_ADR[] = {"u", "G_x", "G_y"};
static const char* NAMES_NSF[] = {"rho", "m_x", "m_y", "E", "G_u_x", "G_u_y", "G_v_x", "G_v_y", "G_T_x", "G_T_y"};
static const char* NAMES_MHD[] = {"rho", "m_x", "m_y", "m_z", "B_x", "B_y", "B_z", "E", "j_x", "j_y", "j_z"};
static const char* NAMES_BUR[] = {"u"};
static const char* NAMES_EUL[] = {"rho", "m_x", "m_y", "E"};
static const char* NAMES_MAX[] = {"E_z", "H_x", "H_y"};
static const char* NAMES_NSF12[] = {"rho", "m_x", "m_y", "E", "G_rho_x", "G_rho_y", "G_mx_x", "G_mx_y",
                                    "G_my_x", "G_my_y", "G_E_x", "G_E_y"};
static const char* NAMES_MHD18[] = {"rho", "m_x", "m_y", "E", "B_x", "B_y", "G_rho_x", "G_rho_y", "G_mx_x",
                                    "G_mx_y", "G_my_x", "G_my_y", "G_E_x", "G_E_y", "G_Bx_x", "G_Bx_y",
                                    "G_By_x", "G_By_y"};
static const char* NAMES_HCNSF[] = {"rho", "m_x", "m_y", "m_z", "E", "G_u11", "G_u22", "G_T_x", "G_T_y",
                                    "G_T_z", "G_u00", "G_u01", "G_u02", "G_u12"};

extern "C" lbx_status lbx_system_declare(const lbx_system_desc* desc, lbx_system** out) {
  if (!desc || !out) return fail(LBX_ERR_ARG, "lbx_system_declare: null argument");
  *out = nullptr;
  const int K = family_K(desc->family);
  if (K == 0) return fail(LBX_ERR_ARG, "lbx_system_declare: unknown family %d", desc->family);
  auto* s = new lbx_system();
  s->family = desc->family;
  s->K = K;
  s->NC = family_NC(desc->family);
  s->D = family_D(desc->family);
  memcpy(s->params, desc->params, sizeof(s->params));
  memcpy(s->Q0, desc->Q0, sizeof(s->Q0));
  if ((s->family == LBX_NSF_PRIM_TRACK || s->family == LBX_EULER || s->family == LBX_MHD_J_TRACK ||
       s->family == LBX_NSF_CONS_TRACK || s->family == LBX_MHD_POWELL_2D || s->family == LBX_HCNSF_3D) &&
      !(s->Q0[0] > 0.0)) {
    delete s;
    return fail(LBX_ERR_ARG, "lbx_system_declare: reference density Q0[0] must be > 0");
  }
  if (s->family == LBX_HCNSF_3D) {
    // the step kernel's delta form multiplies no background quantity by alpha: Phi(Q0)
    // must not depend on the prescribed fields, i.e. the background trackers are zero
    for (int k = s->NC; k < s->K; ++k)
      if (s->Q0[k] != 0.0) {
        delete s;
        return fail(LBX_ERR_ARG, "lbx_system_declare: HCNSF_3D needs Q0[%d] = 0 (tracker background)", k);
      }
    if (!(s->params[3] > 0.0)) {
      delete s;
      return fail(LBX_ERR_ARG, "lbx_system_declare: HCNSF_3D needs eta > 0");
    }
  }
  *out = s;
  return LBX_OK;
}

extern "C" lbx_status lbx_system_info(const lbx_system* s, int* K, int* n_cons, int* dim) {
  if (!s) return fail(LBX_ERR_ARG, "lbx_system_info: null system");
  if (K) *K = s->K;
  if (n_cons) *n_cons = s->NC;
  if (dim) *dim = s->D;
  return LBX_OK;
}

extern "C" const char* lbx_component_name(const lbx_system* s, int k) {
  if (!s || k < 0 || k >= s->K) return nullptr;
  switch (s->family) {
    case LBX_ADR_CASCADE: return NAMES_ADR[k];
    case LBX_NSF_PRIM_TRACK: return NAMES_NSF[k];
    case LBX_MHD_J_TRACK: return NAMES_MHD[k];
    case LBX_BURGERS: return NAMES_BUR[k];
    case LBX_EULER: return NAMES_EUL[k];
    case LBX_MAXWELL_TM: return NAMES_MAX[k];
    case LBX_NSF_CONS_TRACK: return NAMES_NSF12[k];
    case LBX_MHD_POWELL_2D: return NAMES_MHD18[k];
    case LBX_HCNSF_3D: return NAMES_HCNSF[k];
  }
  return nullptr;
}

extern "C" void lbx_system_destroy(lbx_system* s) { delete s; }

// ------------------------------------------------------------------------- lattices
template <class Lat>
static void lat_table(int* q, int* c, double* w) {
  *q = Lat::Q;
  for (int i = 0; i < Lat::Q; ++i) {
    if (c)
      for (int d = 0; d < 3; ++d) c[3 * i + d] = Lat::c(i, d);
    if (w) w[i] = Lat::w(i);
  }
}

extern "C" lbx_status lbx_lattice_velocities(int lattice, int* q, int* c, double* w) {
  if (!q) return fail(LBX_ERR_ARG, "lbx_lattice_velocities: null q");
  switch (lattice) {
    case LBX_D2Q5: lat_table<LatD2Q5>(q, c, w); return LBX_OK;
    case LBX_D2Q9: lat_table<LatD2Q9>(q, c, w); return LBX_OK;
    case LBX_D3Q7: lat_table<LatD3Q7>(q, c, w); return LBX_OK;
    case LBX_D3Q19: lat_table<LatD3Q19>(q, c, w); return LBX_OK;
  }
  return fail(LBX_ERR_ARG, "lbx_lattice_velocities: unknown lattice %d", lattice);
}

int lbx::lattice_q(int lattice) {
  switch (lattice) {
    case LBX_D2Q5: return 5;
    case LBX_D2Q9: return 9;
    case LBX_D3Q7: return 7;
    case LBX_D3Q19: return 19;
  }
  return 0;
}
static int lattice_D(int lattice) { return (lattice == LBX_D3Q7 || lattice == LBX_D3Q19) ? 3 : 2; }
static double lattice_cs2(int lattice) { return lattice == LBX_D3Q7 ? 0.25 : 1.0 / 3.0; }
static void lattice_c(int lattice, int i, int c[3]) {
  int q, tab[19 * 3];
  lbx_lattice_velocities(lattice, &q, tab, nullptr);
  for (int d = 0; d < 3; ++d) c[d] = tab[3 * i + d];
}
static double lattice_w(int lattice, int i) {
  int q;
  double w[19];
  lbx_lattice_velocities(lattice, &q, nullptr, w);
  return w[i];
}

// ------------------------------------------------------------------------- schemes
extern "C" lbx_status lbx_scheme_derive(const lbx_system* sys, const lbx_scheme_desc* d, lbx_scheme** out) {
  if (!sys || !d || !out) return fail(LBX_ERR_ARG, "lbx_scheme_derive: null argument");
  *out = nullptr;
  const int q = lattice_q(d->lattice);
  if (q == 0) return fail(LBX_ERR_ARG, "lbx_scheme_derive: unknown lattice %d", d->lattice);
  if (lattice_D(d->lattice) != sys->D)
    return fail(LBX_ERR_ARG, "lbx_scheme_derive: lattice dimension %d != system dimension %d",
                lattice_D(d->lattice), sys->D);
  const int64_t nx = d->extent[0], ny = d->extent[1], nz = sys->D == 3 ? d->extent[2] : 1;
  if (nx < 2 || ny < 2 || nz < 1 || (sys->D == 3 && nz < 2))
    return fail(LBX_ERR_ARG, "lbx_scheme_derive: extents must be >= 2");
  if (nx > (1 << 20) || ny > 65535 || nz > 65535 || (double)nx * ny * nz >= 2147483647.0 ||
      (double)family_K(sys->family) * q * nx * ny * nz >= 4294967295.0)
    return fail(LBX_ERR_ARG, "lbx_scheme_derive: grid too large (%lld x %lld x %lld)", (long long)nx,
                (long long)ny, (long long)nz);
  if (d->scaling != LBX_ACOUSTIC && d->scaling != LBX_DIFFUSIVE)
    return fail(LBX_ERR_ARG, "lbx_scheme_derive: unknown scaling %d", d->scaling);
  if (!(d->f > 0.0)) return fail(LBX_ERR_ARG, "lbx_scheme_derive: f must be > 0");
  if (d->precision < LBX_FP64 || d->precision > LBX_FP16_SCALED)
    return fail(LBX_ERR_ARG, "lbx_scheme_derive: unknown precision %d", d->precision);
  if (d->mms == LBX_MMS_ADR_SEPARABLE && (sys->family != LBX_ADR_CASCADE || sys->params[3] != 0.0))
    return fail(LBX_ERR_ARG, "lbx_scheme_derive: ADR_SEPARABLE forcing needs the ADR cascade with R = 0");
  if (d->mms != LBX_MMS_NONE && d->mms != LBX_MMS_ADR_SEPARABLE && d->mms != LBX_MMS_FOURIER)
    return fail(LBX_ERR_ARG, "lbx_scheme_derive: unknown forcing %d", d->mms);
  if (d->mms == LBX_MMS_FOURIER) {
    if (!d->mms_modes || d->mms_n_modes < 1 || d->mms_n_modes > LBX_MMS_MAX_MODES)
      return fail(LBX_ERR_ARG, "lbx_scheme_derive: FOURIER forcing needs 1..%d modes", LBX_MMS_MAX_MODES);
    for (int m = 0; m < d->mms_n_modes; ++m) {
      const lbx_mms_mode& md = d->mms_modes[m];
      if (md.p < 0 || md.p >= family_nprim(sys->family))
        return fail(LBX_ERR_ARG, "lbx_scheme_derive: mode %d names primitive %d of %d", m, md.p,
                    family_nprim(sys->family));
      if (sys->D == 2 && md.k[2] != 0)
        return fail(LBX_ERR_ARG, "lbx_scheme_derive: mode %d has k_z != 0 in 2D", m);
      if (!std::isfinite(md.amp) || !std::isfinite(md.phase) || !std::isfinite(md.sigma) ||
          !std::isfinite(md.omega) || !std::isfinite(md.psi))
        return fail(LBX_ERR_ARG, "lbx_scheme_derive: mode %d is not finite", m);
    }
  }
  if (d->prescribed != LBX_PRESCRIBED_NONE) {
    if (sys->family != LBX_HCNSF_3D)
      return fail(LBX_ERR_ARG, "lbx_scheme_derive: prescribed fields belong to HCNSF_3D only");
    if (d->prescribed != LBX_PRESCRIBED_UNIFORM && d->prescribed != LBX_PRESCRIBED_ADVECTED)
      return fail(LBX_ERR_ARG, "lbx_scheme_derive: unknown prescribed fields %d", d->prescribed);
    for (int i = 0; i < 10; ++i)
      if (!std::isfinite(d->prescribed_params[i]))
        return fail(LBX_ERR_ARG, "lbx_scheme_derive: prescribed_params[%d] is not finite", i);
  }
  if (d->streaming != LBX_STREAM_TWO_BUFFERS && d->streaming != LBX_STREAM_IN_PLACE)
    return fail(LBX_ERR_ARG, "lbx_scheme_derive: unknown streaming %d", d->streaming);
  if (d->slab_planes_global != 0) {
    const int64_t P = sys->D == 3 ? nz : ny;
    if (d->slab_planes_global < P || d->slab_origin < 0 || d->slab_origin + P > d->slab_planes_global ||
        d->slab_planes_global > (1 << 24))
      return fail(LBX_ERR_ARG, "lbx_scheme_derive: slab of %lld planes at %lld does not fit %lld global planes",
                  (long long)P, (long long)d->slab_origin, (long long)d->slab_planes_global);
    if (d->streaming != LBX_STREAM_TWO_BUFFERS)
      return fail(LBX_ERR_UNSUPPORTED, "lbx_scheme_derive: slabs need two-buffer streaming");
  } else if (d->slab_origin != 0) {
    return fail(LBX_ERR_ARG, "lbx_scheme_derive: slab_origin without slab_planes_global");
  }
  {
    int given = 0;
    for (int k = 0; k < family_K(sys->family); ++k) {
      const double v = d->fp16_scales[k];
      if (!std::isfinite(v) || v < 0.0) return fail(LBX_ERR_ARG, "lbx_scheme_derive: fp16_scales[%d] invalid", k);
      given += v > 0.0;
    }
    if (given != 0 && given != family_K(sys->family))
      return fail(LBX_ERR_ARG, "lbx_scheme_derive: give fp16_scales for all %d components or none",
                  family_K(sys->family));
    if (given != 0 && d->precision != LBX_FP16_SCALED)
      return fail(LBX_ERR_ARG, "lbx_scheme_derive: fp16_scales need FP16_SCALED storage");
  }
  const bool has_trackers = sys->K > sys->NC;
  if (has_trackers && !(d->g_tau > 0.0)) return fail(LBX_ERR_ARG, "lbx_scheme_derive: g_tau must be > 0");
  auto* s = new lbx_scheme();
  s->sys = *sys;
  s->d = *d;
  if (d->mms == LBX_MMS_FOURIER)
    for (int m = 0; m < d->mms_n_modes; ++m) s->modes[m] = d->mms_modes[m];
  else
    s->d.mms_n_modes = 0;
  s->d.mms_modes = nullptr;
  s->q = q;
  s->nx = (int)nx;
  s->ny = (int)ny;
  s->nz = (int)nz;
  s->ncell = nx * ny * nz;
  s->dx = 1.0 / (double)nx;
  s->dt = d->scaling == LBX_ACOUSTIC ? d->f * s->dx : d->f * s->dx * s->dx;
  s->lam = s->dt / s->dx;
  s->cs2 = lattice_cs2(d->lattice);
  const double tc = d->tau_lb > 0.0 ? d->tau_lb : 0.5 + d->tau_R * s->dt;
  if (!(tc > 0.5)) {
    delete s;
    return fail(LBX_ERR_ARG, "lbx_scheme_derive: conserved tau_LB = %g must exceed 1/2", tc);
  }
  for (int k = 0; k < sys->K; ++k) s->tau[k] = k < sys->NC ? tc : d->g_tau + 1.0;
  *out = s;
  return LBX_OK;
}

extern "C" lbx_status lbx_scheme_info(const lbx_scheme* s, double* dx, double* dt, double* lam, double* tau, int* q) {
  if (!s) return fail(LBX_ERR_ARG, "lbx_scheme_info: null scheme");
  if (dx) *dx = s->dx;
  if (dt) *dt = s->dt;
  if (lam) *lam = s->lam;
  if (tau)
    for (int k = 0; k < s->sys.K; ++k) tau[k] = s->tau[k];
  if (q) *q = s->q;
  return LBX_OK;
}

extern "C" void lbx_scheme_destroy(lbx_scheme* s) { delete s; }

size_t lbx::storage_size(int precision) {
  return precision == LBX_FP64 ? 8 : (precision == LBX_FP32_SHIFT ? 4 : 2);
}

extern "C" size_t lbx_state_buffer_bytes(const lbx_scheme* s) {
  if (!s) return 0;
  return (size_t)s->sys.K * s->q * (size_t)s->ncell * storage_size(s->d.precision);
}

// Phi(Q0) in plain form (host, float64), for the unshifted storage mode and f^eq(Q0).
// Background state of the conserved-gradient cascades (NSF_CONS_TRACK, MHD_POWELL_2D) at
// Q0: velocity, pressure, temperature (T = p/(rho R); R = 1 for MHD), the chain-rule
// velocity and temperature gradients and the viscous stress.  Zero gradients for a
// uniform background.
struct CascadeBg {
  double rho, u[2], p, T, L[2][2], GT[2], tv[2][2], B[2], b2, uB, jz;
};
static CascadeBg cascade_bg(int family, const double* Q, const double* P) {
  CascadeBg c{};
  const bool mhd = family == LBX_MHD_POWELL_2D;
  const double g = P[0], R = mhd ? 1.0 : P[1], mu = P[mhd ? 1 : 2];
  const int gr = mhd ? 6 : 4;                       // first tracker: G_rho
  const double* Gr = Q + gr;
  const double* Gm0 = Q + gr + 2;
  const double* Gm1 = Q + gr + 4;
  const double* GE = Q + gr + 6;
  c.rho = Q[0];
  c.u[0] = Q[1] / c.rho;
  c.u[1] = Q[2] / c.rho;
  const double u2 = c.u[0] * c.u[0] + c.u[1] * c.u[1];
  c.B[0] = mhd ? Q[4] : 0.0;
  c.B[1] = mhd ? Q[5] : 0.0;
  c.b2 = c.B[0] * c.B[0] + c.B[1] * c.B[1];
  c.uB = c.u[0] * c.B[0] + c.u[1] * c.B[1];
  c.p = (g - 1.0) * (Q[3] - 0.5 * c.rho * u2 - 0.5 * c.b2);
  c.T = c.p / (c.rho * R);
  const double* Gm[2] = {Gm0, Gm1};
  for (int b = 0; b < 2; ++b) {
    for (int a = 0; a < 2; ++a) c.L[a][b] = (Gm[a][b] - c.u[a] * Gr[b]) / c.rho;
    double Gp = (g - 1.0) * (GE[b] - (c.u[0] * Gm0[b] + c.u[1] * Gm1[b]) + 0.5 * u2 * Gr[b]);
    if (mhd) Gp -= (g - 1.0) * (c.B[0] * Q[14 + b] + c.B[1] * Q[16 + b]);
    c.GT[b] = (Gp / R - c.T * Gr[b]) / c.rho;
  }
  const double dv = 2.0 / 3.0 * (c.L[0][0] + c.L[1][1]);
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) c.tv[a][b] = mu * (c.L[a][b] + c.L[b][a] - (a == b ? dv : 0.0));
  c.jz = mhd ? Q[16] - Q[15] : 0.0;
  return c;
}

static void background_flux(const lbx_scheme* s, double F0[KMAX][3]) {
  const lbx_system& y = s->sys;
  const double* Q = y.Q0;
  const double* P = y.params;
  const double itg = (y.K > y.NC) ? 1.0 / (s->d.g_tau * s->dt) : 0.0;
  for (int k = 0; k < KMAX; ++k)
    for (int d = 0; d < 3; ++d) F0[k][d] = 0.0;
  switch (y.family) {
    case LBX_ADR_CASCADE:
      for (int d = 0; d < 2; ++d) F0[0][d] = P[d] * Q[0] - P[2] * Q[1 + d];
      for (int b = 0; b < 2; ++b)
        for (int c = 0; c < 2; ++c) F0[1 + b][c] = Q[1 + b] * P[c] - (b == c ? Q[0] * itg : 0.0);
      break;
    case LBX_NSF_PRIM_TRACK: {
      const double g = P[0], R = P[1], mu = P[2], kap = P[3];
      const double rho = Q[0], u[2] = {Q[1] / rho, Q[2] / rho};
      const double p = (g - 1.0) * (Q[3] - 0.5 * (Q[1] * u[0] + Q[2] * u[1]));
      const double T = p / (rho * R);
      const double L[2][2] = {{Q[4], Q[5]}, {Q[6], Q[7]}};
      const double dv = L[0][0] + L[1][1];
      double tv[2][2];
      for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) tv[a][b] = mu * (L[a][b] + L[b][a] - (a == b ? 2.0 / 3.0 * dv : 0.0));
      for (int b = 0; b < 2; ++b) {
        F0[0][b] = Q[1 + b];
        for (int a = 0; a < 2; ++a) F0[1 + a][b] = Q[1 + a] * u[b] + (a == b ? p : 0.0) - tv[a][b];
        F0[3][b] = (Q[3] + p) * u[b] - (tv[b][0] * u[0] + tv[b][1] * u[1]) - kap * Q[8 + b];
      }
      const double V[3] = {u[0], u[1], T};
      for (int v = 0; v < 3; ++v)
        for (int b = 0; b < 2; ++b)
          for (int c = 0; c < 2; ++c) F0[4 + 2 * v + b][c] = Q[4 + 2 * v + b] * u[c] - (b == c ? V[v] * itg : 0.0);
      break;
    }
    case LBX_MHD_J_TRACK: {
      const double g = P[0], eta = P[1];
      const double rho = Q[0];
      double u[3], B[3], j[3], ke = 0, b2 = 0, uB = 0;
      for (int a = 0; a < 3; ++a) {
        u[a] = Q[1 + a] / rho;
        B[a] = Q[4 + a];
        j[a] = Q[8 + a];
      }
      for (int a = 0; a < 3; ++a) {
        ke += 0.5 * Q[1 + a] * u[a];
        b2 += B[a] * B[a];
        uB += u[a] * B[a];
      }
      const double p = (g - 1.0) * (Q[7] - ke - 0.5 * b2), pt = p + 0.5 * b2;
      const double jxB[3] = {j[1] * B[2] - j[2] * B[1], j[2] * B[0] - j[0] * B[2], j[0] * B[1] - j[1] * B[0]};
      for (int b = 0; b < 3; ++b) {
        F0[0][b] = Q[1 + b];
        F0[7][b] = (Q[7] + pt) * u[b] - B[b] * uB + eta * jxB[b];
        for (int a = 0; a < 3; ++a) {
          double ej = 0, eB = 0;
          for (int c = 0; c < 3; ++c) {
            const int e = SysMHD<double>::eps(a, b, c);
            ej += e * j[c];
            eB += e * B[c];
          }
          F0[1 + a][b] = Q[1 + a] * u[b] + (a == b ? pt : 0.0) - B[a] * B[b];
          F0[4 + a][b] = B[a] * u[b] - u[a] * B[b] + eta * ej;
          F0[8 + a][b] = j[a] * u[b] - eB * itg;
        }
      }
      break;
    }
    case LBX_BURGERS:
      F0[0][0] = F0[0][1] = 0.5 * Q[0] * Q[0];
      break;
    case LBX_EULER: {
      const double g = P[0], rho = Q[0], u[2] = {Q[1] / rho, Q[2] / rho};
      const double p = (g - 1.0) * (Q[3] - 0.5 * (Q[1] * u[0] + Q[2] * u[1]));
      for (int b = 0; b < 2; ++b) {
        F0[0][b] = Q[1 + b];
        for (int a = 0; a < 2; ++a) F0[1 + a][b] = Q[1 + a] * u[b] + (a == b ? p : 0.0);
        F0[3][b] = (Q[3] + p) * u[b];
      }
      break;
    }
    case LBX_MAXWELL_TM: {
      const double c = P[0];
      F0[0][0] = -c * Q[2];
      F0[0][1] = c * Q[1];
      F0[1][1] = c * Q[0];
      F0[2][0] = -c * Q[0];
      break;
    }
    case LBX_HCNSF_3D: {
      // zero background trackers: no dissipative flux, alpha drops out
      const double g = P[0], rho = Q[0];
      double u[3], ke = 0.0;
      for (int a = 0; a < 3; ++a) {
        u[a] = Q[1 + a] / rho;
        ke += 0.5 * Q[1 + a] * u[a];
      }
      const double p = (g - 1.0) * (Q[4] - ke), T = p / rho;
      for (int b = 0; b < 3; ++b) {
        F0[0][b] = Q[1 + b];
        for (int a = 0; a < 3; ++a) F0[1 + a][b] = Q[1 + a] * u[b] + (a == b ? p : 0.0);
        F0[4][b] = (Q[4] + p) * u[b];
      }
      for (int a = 0; a < 3; ++a)
        for (int b = a; b < 3; ++b)
          for (int c = 0; c < 3; ++c)
            F0[SysHCNSF<double>::gidx(a, b)][c] = -0.5 * itg * ((a == c ? u[b] : 0.0) + (b == c ? u[a] : 0.0));
      for (int b = 0; b < 3; ++b) F0[7 + b][b] = -T * itg;
      break;
    }
    case LBX_NSF_CONS_TRACK:
    case LBX_MHD_POWELL_2D: {
      const bool mhd = y.family == LBX_MHD_POWELL_2D;
      const CascadeBg c = cascade_bg(y.family, Q, P);
      const double kap = P[mhd ? 2 : 3], eta = mhd ? P[3] : 0.0;
      const double pt = c.p + 0.5 * c.b2;
      const double jxB[2] = {-c.jz * c.B[1], c.jz * c.B[0]};
      for (int b = 0; b < 2; ++b) {
        F0[0][b] = Q[1 + b];
        for (int a = 0; a < 2; ++a) F0[1 + a][b] = Q[1 + a] * c.u[b] + (a == b ? pt : 0.0) - c.B[a] * c.B[b] - c.tv[a][b];
        F0[3][b] = (Q[3] + pt) * c.u[b] - c.B[b] * c.uB - (c.tv[b][0] * c.u[0] + c.tv[b][1] * c.u[1]) -
                   kap * c.GT[b] + eta * jxB[b];
        if (mhd)
          for (int a = 0; a < 2; ++a) F0[4 + a][b] = c.B[a] * c.u[b] - c.u[a] * c.B[b] - eta * Q[14 + 2 * a + b];
      }
      const int nv = mhd ? 6 : 4, gr = mhd ? 6 : 4;
      for (int v = 0; v < nv; ++v)
        for (int b = 0; b < 2; ++b)
          for (int cc = 0; cc < 2; ++cc)
            F0[gr + 2 * v + b][cc] = Q[gr + 2 * v + b] * c.u[cc] - (b == cc ? Q[v] * itg : 0.0);
      break;
    }
  }
}

// System parameter array in the layout systems.cuh documents (physical values).
static void pack_prm(const lbx_scheme* s, double prm[NPRM]) {
  for (int i = 0; i < NPRM; ++i) prm[i] = 0.0;
  const lbx_system& y = s->sys;
  const double* Q = y.Q0;
  const double* P = y.params;
  const double itg = (y.K > y.NC) ? 1.0 / (s->d.g_tau * s->dt) : 0.0;
  switch (y.family) {
    case LBX_ADR_CASCADE:
      prm[0] = P[0]; prm[1] = P[1]; prm[2] = P[2]; prm[3] = P[3]; prm[4] = itg;
      break;
    case LBX_NSF_PRIM_TRACK: {
      const double g = P[0], R = P[1], mu = P[2];
      const double rho = Q[0], u0 = Q[1] / rho, u1 = Q[2] / rho;
      const double p0 = (g - 1.0) * (Q[3] - 0.5 * (Q[1] * u0 + Q[2] * u1));
      const double L00 = Q[4], L01 = Q[5], L10 = Q[6], L11 = Q[7], dv = 2.0 / 3.0 * (L00 + L11);
      prm[0] = g - 1.0; prm[1] = R; prm[2] = mu; prm[3] = P[3]; prm[4] = itg;
      prm[5] = u0; prm[6] = u1; prm[7] = Q[3] + p0; prm[8] = p0 / rho;
      prm[9] = mu * (2 * L00 - dv); prm[10] = mu * (L01 + L10); prm[11] = mu * (2 * L11 - dv);
      prm[12] = g;
      prm[13] = 1.0 / R;
      break;
    }
    case LBX_MHD_J_TRACK: {
      const double g = P[0], rho = Q[0];
      double u[3], ke = 0, b2 = 0, uB = 0;
      for (int a = 0; a < 3; ++a) u[a] = Q[1 + a] / rho;
      for (int a = 0; a < 3; ++a) {
        ke += 0.5 * Q[1 + a] * u[a];
        b2 += Q[4 + a] * Q[4 + a];
        uB += u[a] * Q[4 + a];
      }
      const double p0 = (g - 1.0) * (Q[7] - ke - 0.5 * b2);
      prm[0] = g - 1.0; prm[1] = P[1]; prm[2] = itg;
      prm[3] = u[0]; prm[4] = u[1]; prm[5] = u[2];
      prm[6] = Q[7] + p0 + 0.5 * b2; prm[7] = uB; prm[8] = g;
      break;
    }
    case LBX_BURGERS:
      break;
    case LBX_EULER: {
      const double g = P[0], rho = Q[0], u0 = Q[1] / rho, u1 = Q[2] / rho;
      const double p0 = (g - 1.0) * (Q[3] - 0.5 * (Q[1] * u0 + Q[2] * u1));
      prm[0] = g - 1.0; prm[1] = u0; prm[2] = u1; prm[3] = Q[3] + p0; prm[4] = g;
      break;
    }
    case LBX_MAXWELL_TM:
      prm[0] = P[0];
      break;
    case LBX_NSF_CONS_TRACK: {
      const CascadeBg c = cascade_bg(y.family, Q, P);
      prm[0] = P[0] - 1.0; prm[1] = P[1]; prm[2] = P[2]; prm[3] = P[3]; prm[4] = itg;
      prm[5] = c.u[0]; prm[6] = c.u[1]; prm[7] = Q[3] + c.p; prm[8] = c.T;
      for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) prm[9 + 2 * a + b] = c.L[a][b];
      prm[13] = c.GT[0]; prm[14] = c.GT[1];
      prm[15] = c.tv[0][0]; prm[16] = c.tv[0][1]; prm[17] = c.tv[1][1];
      prm[18] = P[0];
      break;
    }
    case LBX_MHD_POWELL_2D: {
      const CascadeBg c = cascade_bg(y.family, Q, P);
      prm[0] = P[0] - 1.0; prm[1] = P[1]; prm[2] = P[2]; prm[3] = P[3]; prm[4] = itg;
      prm[5] = c.u[0]; prm[6] = c.u[1]; prm[7] = Q[3] + c.p + 0.5 * c.b2; prm[8] = c.uB; prm[9] = c.T;
      for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) prm[10 + 2 * a + b] = c.L[a][b];
      prm[14] = c.GT[0]; prm[15] = c.GT[1];
      prm[16] = c.tv[0][0]; prm[17] = c.tv[0][1]; prm[18] = c.tv[1][1];
      prm[19] = P[0];
      break;
    }
    case LBX_HCNSF_3D: {
      const double g = P[0], rho = Q[0];
      double ke = 0.0;
      for (int a = 0; a < 3; ++a) ke += 0.5 * Q[1 + a] * Q[1 + a] / rho;
      const double p0 = (g - 1.0) * (Q[4] - ke);
      prm[0] = g - 1.0; prm[1] = P[1]; prm[2] = P[2]; prm[3] = 1.0 / P[3]; prm[4] = itg;
      for (int a = 0; a < 3; ++a) prm[5 + a] = Q[1 + a] / rho;
      prm[8] = Q[4] + p0; prm[9] = p0 / rho; prm[10] = g;
      break;
    }
  }
}

template <typename T>
static void fill_params(const lbx_state* st, KParams<T>& p, const double* scale) {
  const lbx_scheme& s = st->sch;
  memset(&p, 0, sizeof(p));
  p.nx = s.nx;
  p.ny = s.ny;
  p.nz = s.nz;
  p.oy = s.sys.D == 2 ? (int)s.d.slab_origin : 0;
  p.oz = s.sys.D == 3 ? (int)s.d.slab_origin : 0;
  p.ncell = s.ncell;
  double F0[KMAX][3], prm[NPRM];
  background_flux(&s, F0);
  pack_prm(&s, prm);
  const double lc = s.lam / s.cs2;
  double wcls[3] = {0.0, 0.0, 0.0};         // lattice weight of each class |c|^2 = 0, 1, 2
  for (int i = 0; i < s.q; ++i) {
    int c[3];
    lattice_c(s.d.lattice, i, c);
    wcls[c[0] * c[0] + c[1] * c[1] + c[2] * c[2]] = lattice_w(s.d.lattice, i);
  }
  for (int k = 0; k < s.sys.K; ++k) {
    p.Q0[k] = (T)s.sys.Q0[k];
    for (int d = 0; d < 3; ++d) p.F0l[k][d] = (T)(lc * F0[k][d]);
    p.omega[k] = (T)(1.0 / s.tau[k]);
    p.omc[k] = (T)(1.0 - 1.0 / s.tau[k]);
    for (int c = 0; c < 3; ++c) p.ow[k][c] = (T)(wcls[c] / s.tau[k]);
    p.tau[k] = (T)s.tau[k];
    p.scale[k] = (T)scale[k];
    p.inv_scale[k] = (T)(1.0 / scale[k]);
  }
  for (int i = 0; i < NPRM; ++i) p.prm[i] = (T)prm[i];
  p.lc = (T)lc;
  p.dt = (T)s.dt;
  p.step_ptr = st->d_step;
  p.err = st->d_err;
  p.wait_ns = st->wait_ns;
  if (s.d.mms == LBX_MMS_ADR_SEPARABLE) {
    const double A = s.d.mms_amp, nu = s.sys.params[2], tp = 2.0 * M_PI;
    p.mms_c0 = (T)(A * (-1.0 + 2.0 * tp * tp * nu));
    p.mms_cx = (T)(tp * A * s.sys.params[0]);
    p.mms_cy = (T)(tp * A * s.sys.params[1]);
    p.mms_tab = sizeof(T) == 8 ? (const T*)st->d_mms_tab64 : (const T*)st->d_mms_tab32;
  }
  p.dx = (T)s.dx;
  if (s.d.mms == LBX_MMS_FOURIER && st->d_mms_modes) {
    p.mms_modes = (const MmsMode*)st->d_mms_modes;
    p.mms_n = s.d.mms_n_modes;
    p.mms_trackers = s.d.mms_conserved_only == 0;
    for (int q = 0; q < 8; ++q) p.mms_mean[q] = (T)s.d.mms_mean[q];
  }
  p.pf_kind = s.d.prescribed;
  p.pf_tab = sizeof(T) == 8 ? (const T*)st->d_pf_tab64 : nullptr;
  for (int i = 0; i < 8; ++i) p.pf[i] = (T)s.d.prescribed_params[i];
  const bool moving = s.d.prescribed == LBX_PRESCRIBED_ADVECTED;
  p.pf_src_dt = (T)(moving ? s.d.prescribed_params[7] * s.dt : 0.0);
  p.pf_flux_dt = (T)(moving ? s.d.prescribed_params[8] * s.dt : 0.0);
}

// ------------------------------------------------------------------------ dispatch
// Device error word (bit 0: a bounded wait in a step kernel timed out), read after a
// synchronisation; a raised word is reported once and cleared.
static lbx_status check_err_word(lbx_state* st) {
  unsigned int w = 0;
  cudaError_t e = cudaMemcpy(&w, st->d_err, sizeof(w), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && w != 0) e = cudaMemset(st->d_err, 0, sizeof(w));
  if (e != cudaSuccess) return fail(LBX_ERR_CUDA, "reading the step kernels' error word: %s", cudaGetErrorString(e));
  if (w == 0) return LBX_OK;
  return fail(LBX_ERR_TIMEOUT, "step kernel: a bounded wait for bulk copies timed out (error word %u)", w);
}


// ------------------------------------------------------------------------- states
#define CK(call)                                                                                     \
  do {                                                                                               \
    cudaError_t e_ = (call);                                                                         \
    if (e_ != cudaSuccess)                                                                           \
      return fail(e_ == cudaErrorMemoryAllocation ? LBX_ERR_OOM : LBX_ERR_CUDA, "%s: %s (%s:%d)", #call, \
                  cudaGetErrorString(e_), __FILE__, __LINE__);                                       \
  } while (0)

// Host <-> device copies of the fields in chunks of planes of the last axis, overlapped with
// the kernels that produce or consume them (lbx_init and lbx_moments with host arrays): the
// copies run on the state's second stream, ordered against the kernels by one event per
// chunk.  Returns after both streams have finished the chunks.
constexpr int kCopyChunks = 8;

static cudaError_t copy_stream_of(lbx_state* st, cudaStream_t* cs) {
  if (!st->copy_stream) {
    if (cudaError_t e = cudaStreamCreateWithFlags(&st->copy_stream, cudaStreamNonBlocking)) return e;
  }
  *cs = st->copy_stream;
  return cudaSuccess;
}

static void plane_chunk(const lbx_scheme& s, int j, int nch, int* p0, int* np) {
  const int P = s.sys.D == 3 ? s.nz : s.ny;
  const int a = (int)((long long)P * j / nch), b = (int)((long long)P * (j + 1) / nch);
  *p0 = a;
  *np = b - a;
}

// fields Qh (host) -> dQ (device) chunk by chunk, each chunk's equilibrium populations
// written as soon as its planes have arrived
static cudaError_t init_pipelined(lbx_state* st, const double* Qh, double* dQ, unsigned long long* chk) {
  const lbx_scheme& s = st->sch;
  const int P = s.sys.D == 3 ? s.nz : s.ny, nch = std::min(P, kCopyChunks);
  const size_t pc = s.sys.D == 3 ? (size_t)s.nx * s.ny : (size_t)s.nx;
  cudaStream_t cs = nullptr;
  cudaError_t e = copy_stream_of(st, &cs);
  if (e) return e;
  cudaEvent_t ev[kCopyChunks] = {};
  for (int j = 0; j < nch && !e; ++j) e = cudaEventCreateWithFlags(&ev[j], cudaEventDisableTiming);
  for (int j = 0; j < nch && !e; ++j) {
    int p0, np;
    plane_chunk(s, j, nch, &p0, &np);
    for (int k = 0; k < s.sys.K && !e; ++k) {
      const size_t off = (size_t)k * s.ncell + (size_t)p0 * pc;
      e = cudaMemcpyAsync(dQ + off, Qh + off, sizeof(double) * np * pc, cudaMemcpyHostToDevice, cs);
    }
    if (!e) e = cudaEventRecord(ev[j], cs);
    if (!e) e = cudaStreamWaitEvent(st->stream, ev[j], 0);
    if (!e) e = st->ops.init_planes(st, dQ, st->fa, p0, np, chk);
  }
  const cudaError_t e1 = cudaStreamSynchronize(cs), e2 = cudaStreamSynchronize(st->stream);
  for (int j = 0; j < nch; ++j)
    if (ev[j]) cudaEventDestroy(ev[j]);
  return e ? e : (e1 ? e1 : e2);
}

// moments of the current populations into Qh (host) chunk by chunk: each chunk's copy back
// starts as soon as its moments are computed
static cudaError_t moments_pipelined(lbx_state* st, double* d, double* Qh) {
  const lbx_scheme& s = st->sch;
  const int P = s.sys.D == 3 ? s.nz : s.ny, nch = std::min(P, kCopyChunks);
  const size_t pc = s.sys.D == 3 ? (size_t)s.nx * s.ny : (size_t)s.nx;
  cudaStream_t cs = nullptr;
  cudaError_t e = copy_stream_of(st, &cs);
  if (e) return e;
  cudaEvent_t ev[kCopyChunks] = {};
  for (int j = 0; j < nch && !e; ++j) e = cudaEventCreateWithFlags(&ev[j], cudaEventDisableTiming);
  for (int j = 0; j < nch && !e; ++j) {
    int p0, np;
    plane_chunk(s, j, nch, &p0, &np);
    e = st->ops.gather_planes(st, st->cur(), d, p0, np);
    if (!e) e = cudaEventRecord(ev[j], st->stream);
    if (!e) e = cudaStreamWaitEvent(cs, ev[j], 0);
    for (int k = 0; k < s.sys.K && !e; ++k) {
      const size_t off = (size_t)k * s.ncell + (size_t)p0 * pc;
      e = cudaMemcpyAsync(Qh + off, d + off, sizeof(double) * np * pc, cudaMemcpyDeviceToHost, cs);
    }
  }
  const cudaError_t e1 = cudaStreamSynchronize(st->stream), e2 = cudaStreamSynchronize(cs);
  for (int j = 0; j < nch; ++j)
    if (ev[j]) cudaEventDestroy(ev[j]);
  return e ? e : (e1 ? e1 : e2);
}

// Device address of page-locked host memory (pinned or registered, mapped into the device's
// address space), else null: kernels read and write such memory directly over the bus.
static void* mapped_host(const void* p) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

static void free_state(lbx_state* st) {
  if (!st) return;
  for (auto& g : st->graphs) cudaGraphExecDestroy(g.second);
  if (st->copy_stream) cudaStreamDestroy(st->copy_stream);
  if (st->own_a && st->fa) cudaFree(st->fa);
  if (st->own_b && st->fb) cudaFree(st->fb);
  cudaFree(st->d_step);
  cudaFree(st->d_err);
  cudaFree(st->d_feq0);
  cudaFree(st->d_partials);
  cudaFree(st->d_red_out);
  cudaFree(st->d_mms_modes);
  cudaFree(st->d_mms_tab64);
  cudaFree(st->d_mms_tab32);
  cudaFree(st->d_pf_tab64);
  cudaFree(st->d_pf_trig);
  delete st;
}

void lbx::feq0_table(const lbx_scheme& s, double* out) {
  double F0[KMAX][3];
  background_flux(&s, F0);
  const double lc = s.lam / s.cs2;
  for (int k = 0; k < s.sys.K; ++k)
    for (int i = 0; i < s.q; ++i) {
      int c[3];
      lattice_c(s.d.lattice, i, c);
      double cph = 0.0;
      for (int d = 0; d < 3; ++d) cph += c[d] * F0[k][d];
      out[k * s.q + i] = lattice_w(s.d.lattice, i) * (s.sys.Q0[k] + lc * cph);
    }
}

void lbx::refresh_params(lbx_state* st) {
  fill_params<double>(st, st->pd, st->scale);
  fill_params<float>(st, st->pf, st->scale);
}

lbx_status lbx::run_reduce(lbx_state* st, const double* Qref, int mode, double* host_out) {
  if (lbx_status s = require_standard_layout(st, "lbx reduction")) return s;
  const int K = st->sch.sys.K;
  if (cudaError_t e = st->ops.reduce(st, st->cur(), Qref, st->d_partials, st->red_blocks, mode))
    return fail(LBX_ERR_CUDA, "reduce launch: %s", cudaGetErrorString(e));
  k_reduce_final<<<1, RED_FINAL_THREADS, 0, st->stream>>>(st->d_partials, st->red_blocks, K, mode, st->d_red_out);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(host_out, st->d_red_out, sizeof(double) * K * 4, cudaMemcpyDeviceToHost, st->stream));
  CK(cudaStreamSynchronize(st->stream));
  return LBX_OK;
}

extern "C" lbx_status lbx_subchar_check(lbx_state* st, double* max_speed, double* bound_cs,
                                        double* bound_monotone, int* ok) {
  if (!st) return fail(LBX_ERR_ARG, "lbx_subchar_check: null state");
  double out[KMAX * 4];
  if (lbx_status s = run_reduce(st, nullptr, 2, out)) return s;
  const double ms = st->sch.lam * out[2];
  const double cs = std::sqrt(st->sch.cs2);
  if (max_speed) *max_speed = ms;
  if (bound_cs) *bound_cs = cs;
  if (bound_monotone) *bound_monotone = st->sch.cs2;
  if (ok) *ok = (ms <= cs) ? 1 : 0;
  return LBX_OK;
}

extern "C" lbx_status lbx_init(const lbx_scheme* sch, const double* Q, int q_on_device, void* stream,
                               void* f_buf_a, void* f_buf_b, lbx_state** out) {
  if (!sch || !Q || !out) return fail(LBX_ERR_ARG, "lbx_init: null argument");
  *out = nullptr;
  const bool inplace = sch->d.streaming == LBX_STREAM_IN_PLACE;
  if (inplace && f_buf_b != nullptr)
    return fail(LBX_ERR_ARG, "lbx_init: an in-place state takes one population buffer (f_buf_b must be NULL)");
  if (!inplace && (f_buf_a == nullptr) != (f_buf_b == nullptr))
    return fail(LBX_ERR_ARG, "lbx_init: pass both population buffers or neither");
  auto* st = new lbx_state();
  st->sch = *sch;
  st->stream = (cudaStream_t)stream;
  st->inplace = inplace;
  if (!find_ops(sch->sys.family, sch->d.lattice, sch->d.precision, &st->ops)) {
    delete st;
    return fail(LBX_ERR_UNSUPPORTED, "lbx_init: family %d on lattice %d not compiled", sch->sys.family,
                sch->d.lattice);
  }
  for (int k = 0; k < KMAX; ++k) st->scale[k] = 1.0;
  lbx_status rc = LBX_OK;
  double* dQ = nullptr;
  const size_t bytes = lbx_state_buffer_bytes(sch);
  const int K = sch->sys.K, q = sch->q;
  auto bail = [&](lbx_status s) {
    if (dQ && !q_on_device && dQ != mapped_host(Q)) cudaFree(dQ);
    free_state(st);
    return s;
  };
#define CKI(call)                                                                                    \
  do {                                                                                               \
    cudaError_t e_ = (call);                                                                         \
    if (e_ != cudaSuccess)                                                                           \
      return bail(fail(e_ == cudaErrorMemoryAllocation ? LBX_ERR_OOM : LBX_ERR_CUDA, "lbx_init: %s: %s", \
                       #call, cudaGetErrorString(e_)));                                              \
  } while (0)
  if (f_buf_a) {
    st->fa = f_buf_a;
    st->fb = f_buf_b;
  } else {
    CKI(cudaMalloc(&st->fa, bytes));
    st->own_a = true;
    if (!inplace) {
      CKI(cudaMalloc(&st->fb, bytes));
      st->own_b = true;
    }
  }
  CKI(cudaMalloc(&st->d_step, sizeof(long long)));
  CKI(cudaMemsetAsync(st->d_step, 0, sizeof(long long), st->stream));
  CKI(cudaMalloc(&st->d_err, sizeof(unsigned int)));
  CKI(cudaMemsetAsync(st->d_err, 0, sizeof(unsigned int), st->stream));
  CKI(cudaMalloc(&st->d_feq0, sizeof(double) * K * q));
  {
    std::vector<double> t(K * q);
    feq0_table(*sch, t.data());
    CKI(cudaMemcpyAsync(st->d_feq0, t.data(), sizeof(double) * K * q, cudaMemcpyHostToDevice, st->stream));
    CKI(cudaStreamSynchronize(st->stream));
  }
  int dev = 0, nsm = 148;
  CKI(cudaGetDevice(&dev));
  CKI(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  st->red_blocks = 2 * nsm;
  CKI(cudaMalloc(&st->d_partials, sizeof(double) * st->red_blocks * K * 4));
  CKI(cudaMalloc(&st->d_red_out, sizeof(double) * K * 4));
  if (sch->d.mms == LBX_MMS_ADR_SEPARABLE) {
    const int nx = sch->nx, ny = sch->ny;
    std::vector<double> t(2 * nx + 2 * ny);
    std::vector<float> tf(t.size());
    for (int i = 0; i < nx; ++i) {
      t[i] = std::sin(2.0 * M_PI * i / nx);
      t[nx + i] = std::cos(2.0 * M_PI * i / nx);
    }
    // rows of a slab take their global index over the whole grid's rows
    const double gy = sch->d.slab_planes_global > 0 ? (double)sch->d.slab_planes_global : (double)ny;
    const double oy = (double)sch->d.slab_origin;
    for (int j = 0; j < ny; ++j) {
      t[2 * nx + j] = std::sin(2.0 * M_PI * (j + oy) / gy);
      t[2 * nx + ny + j] = std::cos(2.0 * M_PI * (j + oy) / gy);
    }
    for (size_t i = 0; i < t.size(); ++i) tf[i] = (float)t[i];
    CKI(cudaMalloc(&st->d_mms_tab64, sizeof(double) * t.size()));
    CKI(cudaMalloc(&st->d_mms_tab32, sizeof(float) * t.size()));
    CKI(cudaMemcpyAsync(st->d_mms_tab64, t.data(), sizeof(double) * t.size(), cudaMemcpyHostToDevice, st->stream));
    CKI(cudaMemcpyAsync(st->d_mms_tab32, tf.data(), sizeof(float) * t.size(), cudaMemcpyHostToDevice, st->stream));
    CKI(cudaStreamSynchronize(st->stream));
  }
  if (sch->d.prescribed == LBX_PRESCRIBED_ADVECTED) {
    // sin and cos of 2 pi x_d at every node index of each axis (global index of a slab), for
    // the moving solid's time-independent factors in the float64 step
    const int n3[3] = {sch->nx, sch->ny, sch->nz};
    const long long o3[3] = {0, sch->sys.D == 2 ? sch->d.slab_origin : 0, sch->sys.D == 3 ? sch->d.slab_origin : 0};
    std::vector<double> t;
    for (int a = 0; a < 3; ++a) {
      for (int i = 0; i < n3[a]; ++i) t.push_back(std::sin(2.0 * M_PI * ((double)(i + o3[a]) * sch->dx)));
      for (int i = 0; i < n3[a]; ++i) t.push_back(std::cos(2.0 * M_PI * ((double)(i + o3[a]) * sch->dx)));
    }
    CKI(cudaMalloc(&st->d_pf_tab64, sizeof(double) * t.size()));
    CKI(cudaMemcpyAsync(st->d_pf_tab64, t.data(), sizeof(double) * t.size(), cudaMemcpyHostToDevice, st->stream));
    CKI(cudaMalloc(&st->d_pf_trig, 4 * sizeof(double)));
    CKI(cudaMemsetAsync(st->d_pf_trig, 0, 4 * sizeof(double), st->stream));
    CKI(cudaStreamSynchronize(st->stream));
  }
  if (sch->d.mms == LBX_MMS_FOURIER) {
    std::vector<MmsMode> md(sch->d.mms_n_modes);
    for (int m = 0; m < sch->d.mms_n_modes; ++m) {
      const lbx_mms_mode& a = sch->modes[m];
      for (int d = 0; d < 3; ++d) md[m].k2pi[d] = 2.0 * M_PI * a.k[d];
      md[m].amp = a.amp;
      md[m].phase = a.phase;
      md[m].sigma = a.sigma;
      md[m].omega = a.omega;
      md[m].psi = a.psi;
      md[m].p = a.p;
      md[m].pad_ = 0;
    }
    CKI(cudaMalloc(&st->d_mms_modes, sizeof(MmsMode) * md.size()));
    CKI(cudaMemcpyAsync(st->d_mms_modes, md.data(), sizeof(MmsMode) * md.size(), cudaMemcpyHostToDevice, st->stream));
    CKI(cudaStreamSynchronize(st->stream));
  }
  refresh_params(st);
  // fields on the device
  const size_t qbytes = sizeof(double) * K * (size_t)sch->ncell;
  // host fields without a float16 scale pass (which needs all of them first) arrive in
  // chunks of planes, each chunk initialised while the next is copied
  const bool derive_scales = sch->d.precision == LBX_FP16_SCALED && !(sch->d.fp16_scales[0] > 0.0);
  // page-locked host fields: the init kernel reads them over the bus (no staging copy)
  double* mapped = q_on_device ? nullptr : (double*)mapped_host(Q);
  const bool pipelined = !q_on_device && !mapped && !derive_scales;
  if (q_on_device || mapped) {
    dQ = mapped ? mapped : const_cast<double*>(Q);
  } else {
    CKI(cudaMalloc(&dQ, qbytes));
    if (!pipelined) CKI(cudaMemcpyAsync(dQ, Q, qbytes, cudaMemcpyHostToDevice, st->stream));
  }
  if (sch->d.precision == LBX_FP16_SCALED && sch->d.fp16_scales[0] > 0.0) {
    for (int k = 0; k < K; ++k) st->scale[k] = sch->d.fp16_scales[k];    // given (shared by slabs)
    refresh_params(st);
  } else if (sch->d.precision == LBX_FP16_SCALED) {
    unsigned long long* dmax = nullptr;
    CKI(cudaMalloc(&dmax, sizeof(unsigned long long) * K));
    cudaError_t e = cudaMemsetAsync(dmax, 0, sizeof(unsigned long long) * K, st->stream);
    if (!e) e = st->ops.init(st, dQ, st->fa, dmax, 0, nullptr);
    unsigned long long hm[KMAX];
    if (!e) e = cudaMemcpyAsync(hm, dmax, sizeof(unsigned long long) * K, cudaMemcpyDeviceToHost, st->stream);
    if (!e) e = cudaStreamSynchronize(st->stream);
    cudaFree(dmax);
    CKI(e);
    // s_k = 2^ceil(log2(4 m_k)), m_k = max |f*_k| at init, floored at 2^-10 of the largest
    // background equilibrium population of the component: a component that starts at rest
    // (fluctuation zero up to rounding, e.g. B = B0 at t = 0) keeps room to grow instead of
    // receiving a scale of its rounding residue that the first fluctuation overflows.
    std::vector<double> feq0(K * q);
    feq0_table(*sch, feq0.data());
    for (int k = 0; k < K; ++k) {
      double m;
      memcpy(&m, &hm[k], sizeof(double));
      if (!std::isfinite(m)) return bail(fail(LBX_ERR_NONFINITE, "lbx_init: non-finite initial field"));
      double b = 0.0;
      for (int i = 0; i < q; ++i) b = std::max(b, std::fabs(feq0[k * q + i]));
      m = std::max(m, std::ldexp(b, -10));
      st->scale[k] = m > 1e-30 ? std::ldexp(1.0, (int)std::ceil(std::log2(4.0 * m))) : 1.0;
    }
    refresh_params(st);
  }
  // the init kernel records the checks of the initial state (two words in the reduction
  // result buffer): the closed-form wave-speed bound of the fields and non-finite stores
  unsigned long long* chk = reinterpret_cast<unsigned long long*>(st->d_red_out);
  CKI(cudaMemsetAsync(chk, 0, 2 * sizeof(unsigned long long), st->stream));
  if (pipelined) {
    CKI(init_pipelined(st, Q, dQ, chk));
  } else {
    CKI(st->ops.init(st, dQ, st->fa, nullptr, 1, chk));
  }
  unsigned long long hchk[2] = {0, 0};
  CKI(cudaMemcpyAsync(hchk, chk, sizeof(hchk), cudaMemcpyDeviceToHost, st->stream));
  CKI(cudaStreamSynchronize(st->stream));
  if (!q_on_device && !mapped) {
    cudaFree(dQ);
    dQ = nullptr;
  }
  st->cur_a = true;
  if (hchk[1] != 0) return bail(fail(LBX_ERR_NONFINITE, "lbx_init: non-finite initial field"));
  if (!sch->d.allow_subchar_violation) {
    double speed;
    memcpy(&speed, &hchk[0], sizeof(speed));
    const double ms = sch->lam * speed;
    if (!(ms <= std::sqrt(sch->cs2)))
      return bail(fail(LBX_ERR_SUBCHAR, "lbx_init: sub-characteristic bound violated: (dt/dx) max speed %.6g > c_s %.6g",
                       ms, std::sqrt(sch->cs2)));
  }
  *out = st;
  return LBX_OK;
#undef CKI
}

// Enqueue n steps (ping-pong from the current buffer) and, with forcing, the device
// step-counter advance; does not touch the host-side bookkeeping.
static cudaError_t enqueue_steps(lbx_state* st, int64_t n, bool start_a) {
  bool a = start_a;
  for (int64_t r = 0; r < n; ++r) {
    cudaError_t e;
    if (st->inplace)   // kinds alternate 1, 2 from the start of a pair
      e = st->ops.step_inplace(st, st->fa, ((st->half + r) & 1) ? 2 : 1, (int)r, st->stream);
    else
      e = st->ops.step(st, a ? st->fa : st->fb, a ? st->fb : st->fa, (int)r, st->stream);
    if (e != cudaSuccess) return e;
    a = !a;
  }
  if (time_dependent(st->sch)) return launch_advance(st->d_step, n, st->stream);
  return cudaSuccess;
}

extern "C" lbx_status lbx_state_set_block(lbx_state* st, int block) {
  if (!st) return fail(LBX_ERR_ARG, "lbx_state_set_block: null state");
  if (block != 32 && block != 64 && block != 128)
    return fail(LBX_ERR_ARG, "lbx_state_set_block: block must be 32, 64 or 128");
  if (block != st->block) {
    for (auto& g : st->graphs) cudaGraphExecDestroy(g.second);
    st->graphs.clear();
  }
  st->block = block;
  return LBX_OK;
}

extern "C" lbx_status lbx_state_set_wait_limit(lbx_state* st, uint64_t ns) {
  if (!st) return fail(LBX_ERR_ARG, "lbx_state_set_wait_limit: null state");
  if ((unsigned long long)ns != st->wait_ns) {
    for (auto& g : st->graphs) cudaGraphExecDestroy(g.second);   // the limit is a launch parameter
    st->graphs.clear();
  }
  st->wait_ns = (unsigned long long)ns;
  refresh_params(st);
  return LBX_OK;
}

extern "C" lbx_status lbx_state_set_staging(lbx_state* st, int staging) {
  if (!st) return fail(LBX_ERR_ARG, "lbx_state_set_staging: null state");
  if (staging < LBX_STAGE_AUTO || staging > LBX_STAGE_PIPE)
    return fail(LBX_ERR_ARG, "lbx_state_set_staging: unknown staging %d", staging);
  if (staging == LBX_STAGE_BULK && !bulk_eligible(st))
    return fail(LBX_ERR_UNSUPPORTED,
                "lbx_state_set_staging: bulk row copies need nx %% 8 == 0 and 16-byte aligned buffers");
  if (staging != st->staging) {
    for (auto& g : st->graphs) cudaGraphExecDestroy(g.second);
    st->graphs.clear();
  }
  st->staging = staging;
  return LBX_OK;
}

extern "C" lbx_status lbx_state_tune(lbx_state* st, int trials, int* staging, int* block, double* ms_per_step) {
  if (!st) return fail(LBX_ERR_ARG, "lbx_state_tune: null state");
  if (trials < 1 || trials > 1000) return fail(LBX_ERR_ARG, "lbx_state_tune: trials must be in 1..1000");
  if (st->nonfinite) return fail(LBX_ERR_NONFINITE, "lbx_state_tune: state holds non-finite values");
  const int old_staging = st->staging, old_block = st->block;
  int best_s = old_staging, best_b = old_block;
  double best = -1.0;
  if (!st->ops.reg && !st->inplace) {   // in place there is no scratch buffer and one launch shape
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaEventCreate(&e0));
    if (cudaError_t e = cudaEventCreate(&e1)) {
      cudaEventDestroy(e0);
      return fail(LBX_ERR_CUDA, "lbx_state_tune: %s", cudaGetErrorString(e));
    }
    const int stagings[2] = {LBX_STAGE_THREAD, LBX_STAGE_BULK};   // the measured-fastest kinds
    const int blocks[3] = {32, 64, 128};
    cudaError_t err = cudaSuccess;
    for (int sg : stagings) {
      if (sg == LBX_STAGE_BULK && !bulk_eligible(st)) continue;
      for (int b : blocks) {
        st->staging = sg;
        st->block = b;
        // cur -> nxt only: the other buffer is rewritten by the next step anyway
        err = st->ops.step(st, st->cur(), st->nxt(), 0, st->stream);
        if (err == cudaSuccess) err = cudaEventRecord(e0, st->stream);
        for (int r = 0; r < trials && err == cudaSuccess; ++r) err = st->ops.step(st, st->cur(), st->nxt(), 0, st->stream);
        if (err == cudaSuccess) err = cudaEventRecord(e1, st->stream);
        if (err == cudaSuccess) err = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
        if (err != cudaSuccess) break;
        const double per = ms / trials;
        if (best < 0.0 || per < best) {
          best = per;
          best_s = sg;
          best_b = b;
        }
      }
      if (err != cudaSuccess) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    st->staging = old_staging;
    st->block = old_block;
    if (err != cudaSuccess) return fail(LBX_ERR_CUDA, "lbx_state_tune: %s", cudaGetErrorString(err));
    if (lbx_status s = check_err_word(st)) return s;
    if (best_s != old_staging || best_b != old_block) {
      for (auto& g : st->graphs) cudaGraphExecDestroy(g.second);
      st->graphs.clear();
    }
    st->staging = best_s;
    st->block = best_b;
  }
  if (staging) *staging = st->ops.reg ? LBX_STAGE_AUTO : st->staging;
  if (block) *block = st->ops.reg ? 128 : st->block;
  if (ms_per_step) *ms_per_step = best;
  return LBX_OK;
}

extern "C" lbx_status lbx_state_use_graph(lbx_state* st, int enable) {
  if (!st) return fail(LBX_ERR_ARG, "lbx_state_use_graph: null state");
  if (enable && st->stream == nullptr)
    return fail(LBX_ERR_STATE, "lbx_state_use_graph: graph capture needs a stream other than the legacy default");
  st->use_graph = enable != 0;
  return LBX_OK;
}

extern "C" lbx_status lbx_step(lbx_state* st, int64_t n) {
  if (!st) return fail(LBX_ERR_ARG, "lbx_step: null state");
  if (n < 0 || n > (int64_t(1) << 30)) return fail(LBX_ERR_ARG, "lbx_step: step count out of range");
  if (st->nonfinite) return fail(LBX_ERR_NONFINITE, "lbx_step: state holds non-finite values");
  if (n == 0) return LBX_OK;
  if (st->use_graph) {
    const auto key = std::make_pair((long long)n, st->inplace ? 2 + st->half : (st->cur_a ? 1 : 0));
    auto it = st->graphs.find(key);
    if (it == st->graphs.end()) {
      cudaGraph_t g = nullptr;
      CK(cudaStreamBeginCapture(st->stream, cudaStreamCaptureModeThreadLocal));
      cudaError_t e = enqueue_steps(st, n, st->cur_a);
      cudaError_t e2 = cudaStreamEndCapture(st->stream, &g);
      if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return fail(LBX_ERR_CUDA, "lbx_step: graph capture failed: %s", cudaGetErrorString(e ? e : e2));
      }
      cudaGraphExec_t ex = nullptr;
      e = cudaGraphInstantiate(&ex, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) return fail(LBX_ERR_CUDA, "lbx_step: graph instantiate: %s", cudaGetErrorString(e));
      it = st->graphs.emplace(key, ex).first;
    }
    CK(cudaGraphLaunch(it->second, st->stream));
  } else {
    cudaError_t e = enqueue_steps(st, n, st->cur_a);
    if (e != cudaSuccess) return fail(LBX_ERR_CUDA, "lbx_step: launch failed: %s", cudaGetErrorString(e));
  }
  if (!time_dependent(st->sch)) st->step_dirty = true;
  if (st->inplace)
    st->half ^= (int)(n & 1);
  else if (n & 1)
    st->cur_a = !st->cur_a;
  st->step += n;
  return LBX_OK;
}

// An in-place state between the two steps of a pair holds the pair's intermediate layout:
// calls that read or write populations refuse it.
lbx_status lbx::require_standard_layout(const lbx_state* st, const char* who) {
  if (st->inplace && st->half)
    return fail(LBX_ERR_STATE, "%s: in-place state after an odd number of steps (take one more step)", who);
  return LBX_OK;
}

// Keep the device step counter in line with the host one (steps taken without forcing).
static lbx_status sync_step_counter(lbx_state* st) {
  if (st->step_dirty) {
    long long v = st->step;
    CK(cudaMemcpyAsync(st->d_step, &v, sizeof(v), cudaMemcpyHostToDevice, st->stream));
    CK(cudaStreamSynchronize(st->stream));
    st->step_dirty = false;
  }
  return LBX_OK;
}

extern "C" lbx_status lbx_moments(lbx_state* st, double* Q_out, int out_on_device) {
  if (!st || !Q_out) return fail(LBX_ERR_ARG, "lbx_moments: null argument");
  if (lbx_status s = require_standard_layout(st, "lbx_moments")) return s;
  const size_t bytes = sizeof(double) * st->sch.sys.K * (size_t)st->sch.ncell;
  if (out_on_device) {
    if (cudaError_t e = st->ops.gather(st, st->cur(), Q_out, nullptr))
      return fail(LBX_ERR_CUDA, "lbx_moments: %s", cudaGetErrorString(e));
    return LBX_OK;
  }
  if (double* m = (double*)mapped_host(Q_out)) {
    // page-locked host memory: the moments kernel writes it over the bus
    cudaError_t e = st->ops.gather(st, st->cur(), m, nullptr);
    if (!e) e = cudaStreamSynchronize(st->stream);
    CK(e);
    return LBX_OK;
  }
  double* d = nullptr;
  CK(cudaMalloc(&d, bytes));
  const cudaError_t e = moments_pipelined(st, d, Q_out);
  cudaFree(d);
  CK(e);
  return LBX_OK;
}

extern "C" lbx_status lbx_conserved_sums(lbx_state* st, double* sums) {
  if (!st || !sums) return fail(LBX_ERR_ARG, "lbx_conserved_sums: null argument");
  double out[KMAX * 4];
  if (lbx_status s = run_reduce(st, nullptr, 0, out)) return s;
  for (int k = 0; k < st->sch.sys.K; ++k) sums[k] = out[4 * k];
  return LBX_OK;
}

extern "C" lbx_status lbx_check_finite(lbx_state* st, int* finite) {
  if (!st || !finite) return fail(LBX_ERR_ARG, "lbx_check_finite: null argument");
  double out[KMAX * 4];
  if (lbx_status s = run_reduce(st, nullptr, 0, out)) return s;
  if (lbx_status s = check_err_word(st)) return s;
  int ok = 1;
  for (int k = 0; k < st->sch.sys.K; ++k)
    if (out[4 * k + 3] != 0.0) ok = 0;
  *finite = ok;
  if (!ok) st->nonfinite = true;
  return LBX_OK;
}

extern "C" lbx_status lbx_error_norms(lbx_state* st, const double* Q_ref, int ref_on_device, double* relL2,
                                      double* relLinf) {
  if (!st || !Q_ref) return fail(LBX_ERR_ARG, "lbx_error_norms: null argument");
  const int K = st->sch.sys.K;
  const size_t bytes = sizeof(double) * K * (size_t)st->sch.ncell;
  const double* d = Q_ref;
  double* tmp = nullptr;
  if (!ref_on_device) {
    CK(cudaMalloc(&tmp, bytes));
    if (cudaError_t e = cudaMemcpyAsync(tmp, Q_ref, bytes, cudaMemcpyHostToDevice, st->stream)) {
      cudaFree(tmp);
      return fail(LBX_ERR_CUDA, "lbx_error_norms: %s", cudaGetErrorString(e));
    }
    d = tmp;
  }
  double out[KMAX * 4];
  lbx_status s = run_reduce(st, d, 1, out);
  if (tmp) cudaFree(tmp);
  if (s) return s;
  for (int k = 0; k < K; ++k) {
    if (relL2) relL2[k] = out[4 * k + 1] > 0 ? std::sqrt(out[4 * k] / out[4 * k + 1]) : std::sqrt(out[4 * k]);
    if (relLinf) relLinf[k] = out[4 * k + 3] > 0 ? out[4 * k + 2] / out[4 * k + 3] : out[4 * k + 2];
  }
  return LBX_OK;
}

extern "C" lbx_status lbx_error_stats(lbx_state* st, const double* Q_ref, int ref_on_device, double* stats) {
  if (!st || !Q_ref || !stats) return fail(LBX_ERR_ARG, "lbx_error_stats: null argument");
  const int K = st->sch.sys.K;
  const size_t bytes = sizeof(double) * K * (size_t)st->sch.ncell;
  const double* d = Q_ref;
  double* tmp = nullptr;
  if (!ref_on_device) {
    CK(cudaMalloc(&tmp, bytes));
    if (cudaError_t e = cudaMemcpyAsync(tmp, Q_ref, bytes, cudaMemcpyHostToDevice, st->stream)) {
      cudaFree(tmp);
      return fail(LBX_ERR_CUDA, "lbx_error_stats: %s", cudaGetErrorString(e));
    }
    d = tmp;
  }
  double out[KMAX * 4];
  lbx_status s = run_reduce(st, d, 1, out);
  if (tmp) cudaFree(tmp);
  if (s) return s;
  for (int i = 0; i < 4 * K; ++i) stats[i] = out[i];
  return LBX_OK;
}

// ------------------------------------------------------------------ slab faces
extern "C" size_t lbx_halo_bytes(const lbx_scheme* s) {
  if (!s) return 0;
  Ops o{};
  if (!find_ops(s->sys.family, s->d.lattice, s->d.precision, &o)) return 0;
  const size_t pc = s->sys.D == 3 ? (size_t)s->nx * s->ny : (size_t)s->nx;
  return (size_t)o.face_nf * s->sys.K * pc * storage_size(s->d.precision);
}

static lbx_status face_call(lbx_state* st, void* a, void* b, int pack, bool next, void* stream, const char* who) {
  if (!st || !a || !b) return fail(LBX_ERR_ARG, "%s: null argument", who);
  if (st->inplace) return fail(LBX_ERR_UNSUPPORTED, "%s: two-buffer states only", who);
  if (((uintptr_t)a % 16) != 0 || ((uintptr_t)b % 16) != 0)
    return fail(LBX_ERR_ARG, "%s: face buffers must be 16-byte aligned", who);
  const cudaStream_t s = stream ? (cudaStream_t)stream : st->stream;
  if (cudaError_t e = st->ops.face(st, next ? st->nxt() : st->cur(), a, b, pack, s))
    return fail(LBX_ERR_CUDA, "%s: %s", who, cudaGetErrorString(e));
  return LBX_OK;
}

extern "C" lbx_status lbx_halo_pack(lbx_state* st, void* to_upper, void* to_lower) {
  return face_call(st, to_upper, to_lower, 1, false, nullptr, "lbx_halo_pack");
}

extern "C" lbx_status lbx_halo_unpack(lbx_state* st, const void* from_lower, const void* from_upper) {
  return face_call(st, const_cast<void*>(from_lower), const_cast<void*>(from_upper), 0, false, nullptr,
                   "lbx_halo_unpack");
}

extern "C" lbx_status lbx_halo_pack_next(lbx_state* st, void* to_upper, void* to_lower, void* stream) {
  return face_call(st, to_upper, to_lower, 1, true, stream, "lbx_halo_pack_next");
}

extern "C" lbx_status lbx_halo_unpack_next(lbx_state* st, const void* from_lower, const void* from_upper,
                                           void* stream) {
  return face_call(st, const_cast<void*>(from_lower), const_cast<void*>(from_upper), 0, true, stream,
                   "lbx_halo_unpack_next");
}

extern "C" lbx_status lbx_step_planes(lbx_state* st, int64_t plane0, int64_t nplanes, void* stream) {
  if (!st) return fail(LBX_ERR_ARG, "lbx_step_planes: null state");
  if (st->inplace) return fail(LBX_ERR_UNSUPPORTED, "lbx_step_planes: two-buffer states only");
  if (st->nonfinite) return fail(LBX_ERR_NONFINITE, "lbx_step_planes: state holds non-finite values");
  const int P = st->sch.sys.D == 3 ? st->sch.nz : st->sch.ny;
  if (plane0 < 0 || nplanes < 0 || plane0 + nplanes > P)
    return fail(LBX_ERR_ARG, "lbx_step_planes: planes [%lld, %lld) outside 0..%d", (long long)plane0,
                (long long)(plane0 + nplanes), P);
  if (!st->ops.reg && resolved_staging(st) == LBX_STAGE_PIPE)
    return fail(LBX_ERR_UNSUPPORTED, "lbx_step_planes: the persistent LBX_STAGE_PIPE kernel steps whole grids only");
  if (nplanes == 0) return LBX_OK;
  st->plane_lo = (int)plane0;
  st->plane_n = (int)nplanes;
  const cudaError_t e = st->ops.step(st, st->cur(), st->nxt(), 0, stream ? (cudaStream_t)stream : st->stream);
  st->plane_lo = 0;
  st->plane_n = 0;
  if (e) return fail(LBX_ERR_CUDA, "lbx_step_planes: %s", cudaGetErrorString(e));
  return LBX_OK;
}

extern "C" lbx_status lbx_step_commit(lbx_state* st) {
  if (!st) return fail(LBX_ERR_ARG, "lbx_step_commit: null state");
  if (st->inplace) return fail(LBX_ERR_UNSUPPORTED, "lbx_step_commit: two-buffer states only");
  if (time_dependent(st->sch)) {
    if (cudaError_t e = launch_advance(st->d_step, 1, st->stream))
      return fail(LBX_ERR_CUDA, "lbx_step_commit: %s", cudaGetErrorString(e));
  } else {
    st->step_dirty = true;
  }
  st->cur_a = !st->cur_a;
  st->step += 1;
  return LBX_OK;
}

extern "C" lbx_status lbx_state_scales(const lbx_state* st, double* scales) {
  if (!st || !scales) return fail(LBX_ERR_ARG, "lbx_state_scales: null argument");
  for (int k = 0; k < st->sch.sys.K; ++k) scales[k] = st->scale[k];
  return LBX_OK;
}

extern "C" lbx_status lbx_get_populations(lbx_state* st, double* f_out) {
  if (!st || !f_out) return fail(LBX_ERR_ARG, "lbx_get_populations: null argument");
  if (lbx_status s = require_standard_layout(st, "lbx_get_populations")) return s;
  const size_t bytes = sizeof(double) * st->sch.sys.K * st->sch.q * (size_t)st->sch.ncell;
  double* d = nullptr;
  CK(cudaMalloc(&d, bytes));
  cudaError_t e = st->ops.gather(st, st->cur(), nullptr, d);
  if (!e) e = cudaMemcpyAsync(f_out, d, bytes, cudaMemcpyDeviceToHost, st->stream);
  if (!e) e = cudaStreamSynchronize(st->stream);
  cudaFree(d);
  CK(e);
  return LBX_OK;
}

extern "C" lbx_status lbx_set_populations(lbx_state* st, const double* f_in) {
  if (!st || !f_in) return fail(LBX_ERR_ARG, "lbx_set_populations: null argument");
  if (lbx_status s = require_standard_layout(st, "lbx_set_populations")) return s;
  const size_t bytes = sizeof(double) * st->sch.sys.K * st->sch.q * (size_t)st->sch.ncell;
  double* d = nullptr;
  CK(cudaMalloc(&d, bytes));
  cudaError_t e = cudaMemcpyAsync(d, f_in, bytes, cudaMemcpyHostToDevice, st->stream);
  if (!e) e = st->ops.scatter(st, d, st->cur());
  if (!e) e = cudaStreamSynchronize(st->stream);
  cudaFree(d);
  CK(e);
  st->nonfinite = false;
  return LBX_OK;
}

extern "C" lbx_status lbx_state_time(const lbx_state* st, int64_t* step, double* t) {
  if (!st) return fail(LBX_ERR_ARG, "lbx_state_time: null state");
  if (step) *step = st->step;
  if (t) *t = (double)st->step * st->sch.dt;
  return LBX_OK;
}

extern "C" void* lbx_state_populations(const lbx_state* st) { return st ? st->cur() : nullptr; }

extern "C" lbx_status lbx_synchronize(lbx_state* st) {
  if (!st) return fail(LBX_ERR_ARG, "lbx_synchronize: null state");
  CK(cudaStreamSynchronize(st->stream));
  if (lbx_status s = sync_step_counter(st)) return s;
  return check_err_word(st);
}

extern "C" void lbx_state_destroy(lbx_state* st) {
  if (st) cudaStreamSynchronize(st->stream);
  free_state(st);
}

lbx_status lbx::ensure_step_counter(lbx_state* st) { return sync_step_counter(st); }

cudaError_t lbx::launch_advance(long long* step, long long n, cudaStream_t s) {
  k_advance<<<1, 1, 0, s>>>(step, n);
  return cudaGetLastError();
}
