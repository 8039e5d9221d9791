"""Wiring of the benchmark cases into the C ABI: which family, lattice, refinement law,
relaxation slots and background state each case uses.  Parameters only; the fields come
from the seeded `synthetic` generators and every computation runs in liblbx.so.
"""
from __future__ import annotations

from . import lbx as L


def adr_system(case):
    """ADR cascade with R = 0 (u_t + a.grad u = nu lap u); a in physical units."""
    ax, ay = case.a_phys
    return L.System(L.ADR_CASCADE, params=(ax, ay, case.nu, 0.0), Q0=(1.0, 0.0, 0.0))


def adr_scheme(case, precision=L.FP64, lattice=L.D2Q5, forcing=True, tau_u=None):
    """Diffusive refinement dt = f dx^2 with tau_LB(u) given directly, trackers g_tau."""
    sysm = adr_system(case)
    return L.Scheme(sysm, lattice, (case.n, case.n), L.DIFFUSIVE, case.f,
                    tau_lb=case.tau_u if tau_u is None else tau_u, g_tau=case.g_tau,
                    precision=precision, mms=L.MMS_ADR_SEPARABLE if forcing else L.MMS_NONE,
                    mms_amp=case.amp)


def nsf_system(case):
    return L.System(L.NSF_PRIM_TRACK, params=(case.gamma, case.R, case.mu, case.kappa),
                    Q0=case.reference_state())


def nsf_scheme(case, precision=L.FP64, lattice=L.D2Q9, tau_lb=0.0, streaming=L.STREAM_TWO_BUFFERS, extent=None,
               **slab):
    """Diffusive refinement dt = f dx^2, tau_LB = 1/2 + tau_R dt, trackers g_tau.  extent and
    slab (slab_origin, slab_planes_global, fp16_scales): a slab of the grid."""
    return L.Scheme(nsf_system(case), lattice, extent or (case.n, case.n), L.DIFFUSIVE, case.f,
                    tau_lb=tau_lb, tau_R=case.tau_R, g_tau=case.g_tau, precision=precision, streaming=streaming,
                    **slab)


def mhd_system(case):
    return L.System(L.MHD_J_TRACK, params=(case.gamma, case.eta), Q0=case.reference_state())


def mhd_scheme(case, precision=L.FP32_SHIFT, lattice=L.D3Q19, streaming=L.STREAM_TWO_BUFFERS, extent=None,
               **slab):
    """Acoustic refinement dt = f dx, tau_LB = 1/2 + tau_R dt, trackers g_tau.  extent and
    slab (slab_origin, slab_planes_global, fp16_scales): a slab of the grid."""
    return L.Scheme(mhd_system(case), lattice, extent or (case.n, case.n, case.n), L.ACOUSTIC, case.f,
                    tau_R=case.tau_R, g_tau=case.g_tau, precision=precision, streaming=streaming, **slab)


# ------------------------------------------------------------- forced (manufactured) runs
_FAMILY = {"adr": L.ADR_CASCADE, "nsf": L.NSF_PRIM_TRACK, "mhd": L.MHD_J_TRACK,
           "burgers": L.BURGERS, "euler": L.EULER, "maxwell": L.MAXWELL_TM,
           "nsf12": L.NSF_CONS_TRACK, "mhd18": L.MHD_POWELL_2D, "hcnsf": L.HCNSF_3D}


def table_system(table, params, Q0):
    """The family of a manufactured mode table (duck-typed: .family) with its parameters."""
    return L.System(_FAMILY[table.family], params=params, Q0=Q0)


def forced_scheme(table, system, lattice, extent, scaling, f, precision=L.FP64, tau_lb=0.0,
                  tau_R=0.0, g_tau=0.0, conserved_only=False, prescribed=L.PRESCRIBED_NONE,
                  prescribed_params=(), streaming=L.STREAM_TWO_BUFFERS, **slab):
    """A scheme carrying the FOURIER forcing of `table` (.lbx_modes(), .mean): every
    component, or the conserved ones with conserved_only."""
    return L.Scheme(system, lattice, extent, scaling, f, tau_lb=tau_lb, tau_R=tau_R, g_tau=g_tau,
                    precision=precision, mms=L.MMS_FOURIER, mms_modes=table.lbx_modes(),
                    mms_mean=list(table.mean), mms_conserved_only=conserved_only,
                    prescribed=prescribed, prescribed_params=prescribed_params, streaming=streaming, **slab)


# ------------------------------------------------------------- the paper's own cascades
def nsf12_system(case):
    """12-component NSF with conserved-gradient trackers (case: gamma, R, mu, kappa and a
    cascade background state)."""
    return L.System(L.NSF_CONS_TRACK, params=(case.gamma, case.R, case.mu, case.kappa),
                    Q0=case.reference_state_cascade())


def nsf12_scheme(case, precision=L.FP32_SHIFT, lattice=L.D2Q5):
    """The paper's NSF recipe: diffusive dt = f dx^2, tau_LB = 1/2 + tau_R dt, trackers g_tau."""
    return L.Scheme(nsf12_system(case), lattice, (case.n, case.n), L.DIFFUSIVE, case.f,
                    tau_R=case.tau_R, g_tau=case.g_tau, precision=precision)


def mhd18_system(case):
    """18-component 2D MHD with Powell cleaning (case: gamma, mu, kappa, eta)."""
    return L.System(L.MHD_POWELL_2D, params=(case.gamma, case.mu, case.kappa, case.eta),
                    Q0=case.reference_state())


def mhd18_scheme(case, precision=L.FP32_SHIFT, lattice=L.D2Q5):
    """The paper's MHD recipe: acoustic dt = f dx, tau_LB = 1/2 + tau_R dt, trackers g_tau."""
    return L.Scheme(mhd18_system(case), lattice, (case.n, case.n), L.ACOUSTIC, case.f,
                    tau_R=case.tau_R, g_tau=case.g_tau, precision=precision)


# ------------------------------------------------- 3D homogenized NSF (prescribed fields)
def hcnsf_system(case):
    """14-component 3D homogenized NSF (case: gamma, mu, kappa, eta, a background state with
    zero trackers)."""
    return L.System(L.HCNSF_3D, params=(case.gamma, case.mu, case.kappa, case.eta),
                    Q0=case.reference_state())


def hcnsf_prescribed(case):
    """The case's advected-solid porosity and solid velocity (lbx_prescribed ADVECTED)."""
    return L.PRESCRIBED_ADVECTED, ((case.alpha_mean, case.alpha_amp, case.rot, case.osc) + tuple(case.c)
                                   + (getattr(case, "theta", 0.0), getattr(case, "theta_flux", 0.0)))


def hcnsf_scheme(case, precision=L.FP32_SHIFT, forced=False, extent=None, streaming=L.STREAM_TWO_BUFFERS,
                 **slab):
    """The paper's HCNSF recipe on D3Q7: acoustic dt = f dx, tau_LB = 1/2 + tau_R dt, trackers
    g_tau, prescribed fields of the moving solid; forced: the case's manufactured flow.  slab
    (slab_origin, slab_planes_global, fp16_scales): a z-slab of the grid (extent its own)."""
    kind, pf = hcnsf_prescribed(case)
    ext = extent or (case.n, case.n, case.n)
    if forced:
        return forced_scheme(case.table(), hcnsf_system(case), L.D3Q7, ext, L.ACOUSTIC, case.f,
                             precision=precision, tau_R=case.tau_R, g_tau=case.g_tau,
                             prescribed=kind, prescribed_params=pf, streaming=streaming, **slab)
    return L.Scheme(hcnsf_system(case), L.D3Q7, ext, L.ACOUSTIC, case.f, tau_R=case.tau_R,
                    g_tau=case.g_tau, precision=precision, prescribed=kind, prescribed_params=pf,
                    streaming=streaming, **slab)
