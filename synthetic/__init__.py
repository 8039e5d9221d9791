"""Seeded synthetic inputs shared by the CUDA path and the CPU oracle.

This module only builds input fields: node coordinates, manufactured exact fields
Q_ex(x, t) and their analytic gradients (used to start the gradient trackers), and the
random draws of the batched workload.  It holds none of the scheme's arithmetic: no
equilibrium, flux, source, collision or streaming.  Everything is float64 torch on
the CPU; callers move results where they need them.

Conventions
-----------
* Periodic unit domain [0, 1)^D, N nodes per axis, node coordinates x_i = i / N.
* Field arrays are [K, ny, nx] (2D) or [K, nz, ny, nx] (3D), x fastest, C order.
* Tracker components G_{V,b} hold d V / d x_b (index b is the derivative direction).

Component orders (fixed by this library):
  ADR cascade         (u, G_u,x, G_u,y)                                       K = 3
  NSF, primitive trk  (rho, m_x, m_y, E, G_u,x, G_u,y, G_v,x, G_v,y, G_T,x, G_T,y) K = 10
  MHD, current trk    (rho, m_x, m_y, m_z, B_x, B_y, B_z, E, j_x, j_y, j_z)    K = 11
  Burgers             (u)                                                     K = 1
  Euler               (rho, m_x, m_y, E)                                      K = 4
  Maxwell TM          (E_z, H_x, H_y)                                         K = 3
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import torch

TWO_PI = 2.0 * math.pi
DT = torch.float64


def coords(shape):
    """Node coordinates x_i = i/N along each axis, broadcast to `shape` (z, y, x order).

    Returns a tuple (x, y) for 2D or (x, y, z) for 3D of float64 tensors of `shape`.
    """
    axes = [torch.arange(n, dtype=DT) / n for n in shape]
    mesh = torch.meshgrid(*axes, indexing="ij")
    return tuple(m.contiguous() for m in reversed(mesh))  # x fastest -> (x, y[, z])


# --------------------------------------------------------------------------------------
# ADR cascade: u_t + a.grad u = nu lap u, manufactured u = 1 + 0.1 sin(2 pi x) cos(2 pi y) e^-t
# --------------------------------------------------------------------------------------

@dataclass
class AdrCase:
    """One ADR-cascade instance.  `a_lat` is the advection vector in lattice units at
    this N (a_phys = a_lat * dx / dt); diffusive refinement dt = f dx^2."""
    n: int
    a_lat: tuple = (0.1, 0.05)
    nu: float = 0.01
    f: float = 1.0
    tau_u: float = 0.8
    g_tau: float = 6.0
    amp: float = 0.1

    @property
    def dx(self):
        return 1.0 / self.n

    @property
    def dt(self):
        return self.f * self.dx * self.dx

    @property
    def a_phys(self):
        lam = self.dt / self.dx
        return (self.a_lat[0] / lam, self.a_lat[1] / lam)


def adr_exact(case: AdrCase, x, y, t):
    """Manufactured u_ex(x, y, t) = 1 + amp sin(2 pi x) cos(2 pi y) exp(-t) (torch)."""
    return 1.0 + case.amp * torch.sin(TWO_PI * x) * torch.cos(TWO_PI * y) * torch.exp(-t)


def adr_fields(case: AdrCase, t: float = 0.0):
    """Q = (u_ex, d_x u_ex, d_y u_ex) at time t, shape [3, N, N] float64."""
    x, y = coords((case.n, case.n))
    e = math.exp(-t)
    u = 1.0 + case.amp * torch.sin(TWO_PI * x) * torch.cos(TWO_PI * y) * e
    gx = case.amp * TWO_PI * torch.cos(TWO_PI * x) * torch.cos(TWO_PI * y) * e
    gy = -case.amp * TWO_PI * torch.sin(TWO_PI * x) * torch.sin(TWO_PI * y) * e
    return torch.stack([u, gx, gy])


def adr_batch_draws(n_inst: int = 512, seed: int = 0, lo_exp=5.0, hi_exp=9.0):
    """Batched ADR workload: N_j = round(2^U), U ~ U[5, 9]; a_j ~ U[-0.1, 0.1]^2 (lattice
    units at N_j); tau_j ~ U[0.6, 1.2].  numpy PCG64(seed)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ns = np.rint(2.0 ** rng.uniform(lo_exp, hi_exp, n_inst)).astype(int)
    a = rng.uniform(-0.1, 0.1, (n_inst, 2))
    tau = rng.uniform(0.6, 1.2, n_inst)
    return [AdrCase(n=int(ns[j]), a_lat=(float(a[j, 0]), float(a[j, 1])), tau_u=float(tau[j]))
            for j in range(n_inst)]


# --------------------------------------------------------------------------------------
# Seeded Fourier fields (NSF, adjoint target)
# --------------------------------------------------------------------------------------

def _modes(rng, n_modes, kmax, dim):
    ks = []
    while len(ks) < n_modes:
        k = rng.integers(-kmax, kmax + 1, dim)
        if np.any(k != 0):
            ks.append(k)
    return np.array(ks)


@dataclass
class FourierField:
    """V(x) = mean + sum_m amp_m sin(2 pi k_m . x + phase_m)."""
    mean: float
    k: np.ndarray      # [M, D] integer wavevectors
    amp: np.ndarray    # [M]
    phase: np.ndarray  # [M]

    def value(self, xs):
        v = torch.full_like(xs[0], self.mean)
        for k, a, p in zip(self.k, self.amp, self.phase):
            th = TWO_PI * sum(float(k[d]) * xs[d] for d in range(len(xs))) + float(p)
            v = v + float(a) * torch.sin(th)
        return v

    def grad(self, xs, b):
        g = torch.zeros_like(xs[0])
        for k, a, p in zip(self.k, self.amp, self.phase):
            th = TWO_PI * sum(float(k[d]) * xs[d] for d in range(len(xs))) + float(p)
            g = g + float(a) * TWO_PI * float(k[b]) * torch.cos(th)
        return g


def fourier_field(rng, mean, n_modes=4, kmax=3, amp_max=0.05, dim=2):
    k = _modes(rng, n_modes, kmax, dim)
    amp = rng.uniform(0.0, amp_max, n_modes)
    phase = rng.uniform(0.0, TWO_PI, n_modes)
    return FourierField(mean, k, amp, phase)


@dataclass
class NsfCase:
    """Compressible NSF with primitive trackers (grad u, grad v, grad T).

    Ideal gas gamma = 1.4, R = 1, rho0 = 1, T0 = 1, background Mach 0.3 along 30 deg,
    Re = 100 on the unit domain, Pr = 0.71; diffusive refinement dt = f dx^2 with f = 2,
    tau_R = 60, g_tau = 6 (the paper's NSF recipe)."""
    n: int
    seed: int = 0
    gamma: float = 1.4
    R: float = 1.0
    Pr: float = 0.71
    Re: float = 100.0
    mach: float = 0.3
    angle_deg: float = 30.0
    f: float = 2.0
    tau_R: float = 60.0
    g_tau: float = 6.0
    n_modes: int = 4
    amp_max: float = 0.05

    @property
    def c_bar(self):
        return math.sqrt(self.gamma * self.R * 1.0)

    @property
    def U0(self):
        s = self.mach * self.c_bar
        a = math.radians(self.angle_deg)
        return (s * math.cos(a), s * math.sin(a))

    @property
    def mu(self):
        return 1.0 * math.hypot(*self.U0) * 1.0 / self.Re

    @property
    def kappa(self):
        cp = self.gamma * self.R / (self.gamma - 1.0)
        return self.mu * cp / self.Pr

    @property
    def dx(self):
        return 1.0 / self.n

    @property
    def dt(self):
        return self.f * self.dx * self.dx

    def primitives(self):
        """Seeded (rho, u, v, T) Fourier fields, numpy PCG64(seed)."""
        rng = np.random.Generator(np.random.PCG64(self.seed))
        u0, v0 = self.U0
        return [fourier_field(rng, 1.0, self.n_modes, 3, self.amp_max),
                fourier_field(rng, u0, self.n_modes, 3, self.amp_max),
                fourier_field(rng, v0, self.n_modes, 3, self.amp_max),
                fourier_field(rng, 1.0, self.n_modes, 3, self.amp_max)]

    def reference_state(self):
        """Q0 = uniform background (rho0, rho0 U0, E0, trackers 0)."""
        u0, v0 = self.U0
        p0 = 1.0 * self.R * 1.0
        E0 = p0 / (self.gamma - 1.0) + 0.5 * (u0 * u0 + v0 * v0)
        return [1.0, u0, v0, E0] + [0.0] * 6


def nsf_fields(case: NsfCase):
    """Conserved state plus analytic primitive gradients, [10, N, N] float64."""
    xs = coords((case.n, case.n))
    rho_f, u_f, v_f, T_f = case.primitives()
    rho, u, v, T = (fld.value(xs) for fld in (rho_f, u_f, v_f, T_f))
    p = rho * case.R * T
    E = p / (case.gamma - 1.0) + 0.5 * rho * (u * u + v * v)
    comps = [rho, rho * u, rho * v, E]
    for fld in (u_f, v_f, T_f):
        comps += [fld.grad(xs, 0), fld.grad(xs, 1)]
    return torch.stack(comps)


def density_target(n: int, seed: int = 1, amp_max: float = 0.05):
    """rho*(x) = 1 + seeded Fourier field (<= amp_max per mode), for the misfit
    J = 1/2 sum_x (rho(x, T) - rho*(x))^2."""
    rng = np.random.Generator(np.random.PCG64(seed))
    fld = fourier_field(rng, 1.0, 4, 3, amp_max)
    return fld.value(coords((n, n)))


# --------------------------------------------------------------------------------------
# 3D resistive MHD with current tracker
# --------------------------------------------------------------------------------------

@dataclass
class MhdCase:
    """3D resistive MHD, j = curl B tracked.  rho = 1, p = 1/gamma, u and B = curl A
    built from seeded random-phase sinusoids (amplitude 0.2).  Acoustic refinement
    dt = f dx with f = 0.05, tau_R = 160, g_tau = 4 (the paper's MHD float recipe)."""
    n: int
    seed: int = 0
    gamma: float = 1.4
    eta: float = 0.01
    f: float = 0.05
    tau_R: float = 160.0
    g_tau: float = 4.0
    n_modes: int = 3
    amp: float = 0.2

    @property
    def dx(self):
        return 1.0 / self.n

    @property
    def dt(self):
        return self.f * self.dx

    def reference_state(self):
        p0 = 1.0 / self.gamma
        return [1.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, p0 / (self.gamma - 1.0), 0.0, 0.0, 0.0]

    def draws(self):
        rng = np.random.Generator(np.random.PCG64(self.seed))
        vel = [(_modes(rng, 1, 2, 3)[0], rng.uniform(-1, 1, 3), rng.uniform(0, TWO_PI))
               for _ in range(self.n_modes)]
        pot = [(_modes(rng, 1, 2, 3)[0], rng.uniform(-1, 1, 3), rng.uniform(0, TWO_PI))
               for _ in range(self.n_modes)]
        return vel, pot


def mhd_fields(case: MhdCase):
    """[11, N, N, N] float64: rho, m, B = curl A, E, j = curl B (all analytic)."""
    n = case.n
    xs = coords((n, n, n))
    vel, pot = case.draws()
    scale = case.amp / case.n_modes
    u = [torch.zeros_like(xs[0]) for _ in range(3)]
    B = [torch.zeros_like(xs[0]) for _ in range(3)]
    j = [torch.zeros_like(xs[0]) for _ in range(3)]
    for k, d, ph in vel:
        th = TWO_PI * sum(float(k[c]) * xs[c] for c in range(3)) + ph
        s = torch.sin(th)
        for c in range(3):
            u[c] = u[c] + scale * float(d[c]) * s
    for k, d, ph in pot:
        # A = scale d sin(th) / (2 pi |k|): B = scale cos(th) (k x d)/|k|,
        # j = curl B = -2 pi scale sin(th) k x (k x d) / |k|.
        kn = float(np.linalg.norm(k))
        kxd = np.cross(k, d)
        kxkxd = np.cross(k, kxd)
        th = TWO_PI * sum(float(k[c]) * xs[c] for c in range(3)) + ph
        cth, sth = torch.cos(th), torch.sin(th)
        for c in range(3):
            B[c] = B[c] + scale * float(kxd[c]) / kn * cth
            j[c] = j[c] - TWO_PI * scale * float(kxkxd[c]) / kn * sth
    rho = torch.ones_like(xs[0])
    p = torch.full_like(xs[0], 1.0 / case.gamma)
    u2 = sum(c * c for c in u)
    b2 = sum(c * c for c in B)
    E = p / (case.gamma - 1.0) + 0.5 * rho * u2 + 0.5 * b2
    return torch.stack([rho] + [rho * c for c in u] + B + [E] + j)


# --------------------------------------------------------------------------------------
# The paper's own D2Q5 manufactured solutions (supplement, MMS section)
# --------------------------------------------------------------------------------------

def burgers_exact(x, y, t, A=1.3):
    """u = A sin(2 pi x) sin(2 pi y) cos t (torch; t may be a tensor)."""
    return A * torch.sin(TWO_PI * x) * torch.sin(TWO_PI * y) * torch.cos(t)


def maxwell_exact(x, y, t, A=0.5, w=4.0):
    """TM mode: E_z, H_x, H_y with k_x = 2 pi, k_y = 4 pi, omega = 4 (torch)."""
    kx, ky = TWO_PI, 2.0 * TWO_PI
    ez = A * torch.sin(kx * x) * torch.sin(ky * y) * torch.cos(w * t)
    hx = A * torch.sin(kx * x) * torch.cos(ky * y) * torch.sin(w * t)
    hy = -A * (kx / ky) * torch.cos(kx * x) * torch.sin(ky * y) * torch.sin(w * t)
    return torch.stack([ez, hx, hy])


def adr_exact_stack(case: AdrCase):
    """Callable (x, y, t) -> [1, ...] conserved exact field for the ADR case."""
    return lambda x, y, t: adr_exact(case, x, y, t).unsqueeze(0)
