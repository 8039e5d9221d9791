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
  12-component NSF    (rho, m_x, m_y, E, G_rho(2), G_mx(2), G_my(2), G_E(2))   K = 12
  18-component MHD    (rho, m_x, m_y, E, B_x, B_y, G of the six, 2 each)      K = 18
  3D homogenized NSF  (rho, m(3), E, G_u11, G_u22, G_T(3), G_u00, G_u01, G_u02, G_u12)  K = 14
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


def density_target(n: int, seed: int = 1, amp_max: float = 0.05, dim: int = 2):
    """rho*(x) = 1 + seeded Fourier field (<= amp_max per mode) on the n^dim grid, for the
    misfit J = 1/2 sum_x (rho(x, T) - rho*(x))^2."""
    rng = np.random.Generator(np.random.PCG64(seed))
    fld = fourier_field(rng, 1.0, 4, 3, amp_max, dim=dim)
    return fld.value(coords((n,) * dim))


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


# --------------------------------------------------------------------------------------
# Manufactured solutions as mode tables of primitive fields (forced verification runs)
# --------------------------------------------------------------------------------------

# primitive fields per family, in table order
PRIMITIVES = {"adr": ("u",), "nsf": ("rho", "u", "v", "p"),
              "mhd": ("rho", "u_x", "u_y", "u_z", "B_x", "B_y", "B_z", "p"),
              "burgers": ("u",), "euler": ("rho", "u", "v", "p"), "maxwell": ("E_z", "H_x", "H_y"),
              "nsf12": ("rho", "u", "v", "p"), "mhd18": ("rho", "u", "v", "p", "B_x", "B_y"),
              "hcnsf": ("rho", "u_x", "u_y", "u_z", "p")}


@dataclass
class ModeTable:
    """Primitive fields V_p(x, t) = mean[p] + sum over the modes of p of
    amp sin(2 pi k.x + phase) exp(sigma t) cos(omega t + psi), and the conserved state the
    family assembles from them (gamma, R: the gas constants where the family has them)."""
    family: str
    mean: list
    modes: list            # (p, k, amp, phase, sigma, omega, psi), k a tuple of ints
    gamma: float = 1.4
    R: float = 1.0

    def primitives(self, xs, t):
        t = t if torch.is_tensor(t) else torch.full_like(xs[0], float(t))
        V = [torch.full_like(xs[0], float(m)) for m in self.mean]
        for (p, k, amp, phase, sigma, omega, psi) in self.modes:
            th = TWO_PI * sum(float(k[d]) * xs[d] for d in range(len(xs))) + phase
            V[p] = V[p] + amp * torch.sin(th) * torch.exp(sigma * t) * torch.cos(omega * t + psi)
        return V

    def conserved(self, V):
        g, R = self.gamma, self.R
        if self.family in ("adr", "burgers", "maxwell"):
            return torch.stack(V)
        if self.family == "mhd18":
            rho, u, v, p, bx, by = V
            E = p / (g - 1.0) + 0.5 * rho * (u * u + v * v) + 0.5 * (bx * bx + by * by)
            return torch.stack([rho, rho * u, rho * v, E, bx, by])
        if self.family == "hcnsf":
            rho, u, p = V[0], V[1:4], V[4]
            return torch.stack([rho] + [rho * c for c in u] + [p / (g - 1.0) + 0.5 * rho * sum(c * c for c in u)])
        if self.family in ("nsf", "euler", "nsf12"):
            rho, u, v, p = V
            return torch.stack([rho, rho * u, rho * v, p / (g - 1.0) + 0.5 * rho * (u * u + v * v)])
        if self.family == "mhd":
            rho, u, B, p = V[0], V[1:4], V[4:7], V[7]
            E = p / (g - 1.0) + 0.5 * rho * sum(c * c for c in u) + 0.5 * sum(c * c for c in B)
            return torch.stack([rho] + [rho * c for c in u] + list(B) + [E])
        raise ValueError(self.family)

    def exact(self, *xt):
        """Conserved exact fields at coordinates xt[:-1] and time xt[-1] (oracle callable)."""
        return self.conserved(self.primitives(xt[:-1], xt[-1]))

    def gradient(self, xs, t, p, b):
        """d V_p / d x_b, analytic."""
        t = t if torch.is_tensor(t) else torch.full_like(xs[0], float(t))
        g = torch.zeros_like(xs[0])
        for (q, k, amp, phase, sigma, omega, psi) in self.modes:
            if q != p or k[b] == 0:
                continue
            th = TWO_PI * sum(float(k[d]) * xs[d] for d in range(len(xs))) + phase
            g = g + amp * TWO_PI * k[b] * torch.cos(th) * torch.exp(sigma * t) * torch.cos(omega * t + psi)
        return g

    def augmented(self, xs, t):
        """Conserved exact fields plus the family's trackers (ADR: grad u; NSF: grad u,
        grad v, grad T; MHD: curl B), the initial state of a forced run."""
        Qc = self.exact(*xs, t)
        if self.family == "adr":
            tr = [self.gradient(xs, t, 0, b) for b in range(2)]
        elif self.family == "nsf":
            # T = p/(rho R): grad T = (grad p - R T grad rho)/(rho R)
            rho, _, _, p = self.primitives(xs, t)
            T = p / (rho * self.R)
            tr = [self.gradient(xs, t, q, b) for q in (1, 2) for b in range(2)]
            tr += [(self.gradient(xs, t, 3, b) - self.R * T * self.gradient(xs, t, 0, b)) / (rho * self.R)
                   for b in range(2)]
        elif self.family == "mhd":
            G = lambda c, b: self.gradient(xs, t, 4 + c, b)
            tr = [G(2, 1) - G(1, 2), G(0, 2) - G(2, 0), G(1, 0) - G(0, 1)]
        elif self.family == "hcnsf":
            # sym grad u and grad T (T = p/rho) in the paper's order
            V = self.primitives(xs, t)
            rho, p = V[0], V[4]
            Gs = [[self.gradient(xs, t, q, b) for b in range(3)] for q in range(5)]
            sym = lambda a, b: 0.5 * (Gs[1 + a][b] + Gs[1 + b][a])
            gT = [(Gs[4][b] - p / rho * Gs[0][b]) / rho for b in range(3)]
            tr = [sym(1, 1), sym(2, 2)] + gT + [sym(0, 0), sym(0, 1), sym(0, 2), sym(1, 2)]
        elif self.family in ("nsf12", "mhd18"):
            # gradients of the conserved fields by the product rule
            V = self.primitives(xs, t)
            rho, u, v, p = V[:4]
            g1 = self.gamma - 1.0
            tr = []
            Gs = [[self.gradient(xs, t, q, b) for b in range(2)] for q in range(len(V))]
            for b in range(2):
                tr.append(Gs[0][b])
            for q, w in ((1, u), (2, v)):
                for b in range(2):
                    tr.append(Gs[0][b] * w + rho * Gs[q][b])
            for b in range(2):
                gE = Gs[3][b] / g1 + 0.5 * Gs[0][b] * (u * u + v * v) + rho * (u * Gs[1][b] + v * Gs[2][b])
                if self.family == "mhd18":
                    gE = gE + V[4] * Gs[4][b] + V[5] * Gs[5][b]
                tr.append(gE)
            if self.family == "mhd18":
                for q in (4, 5):
                    for b in range(2):
                        tr.append(Gs[q][b])
        else:
            return Qc
        return torch.cat([Qc, torch.stack(tr)])

    def lbx_modes(self):
        return [(p, tuple(int(c) for c in k), float(a), float(ph), float(s), float(w), float(ps))
                for (p, k, a, ph, s, w, ps) in self.modes]


def _product_modes(p, amp, fx, fy, kx, ky, omega, psi):
    """amp f_x(2 pi kx x) f_y(2 pi ky y) cos(omega t + psi) as two sine modes (f in sin/cos)."""
    # sin a cos b = [sin(a+b) + sin(a-b)]/2, cos a sin b = [sin(a+b) - sin(a-b)]/2,
    # sin a sin b = [sin(a-b+pi/2) - sin(a+b+pi/2)]/2, cos a cos b = [sin(a+b+pi/2) + sin(a-b+pi/2)]/2
    h = 0.5 * amp
    plus, minus = (kx, ky, 0), (kx, -ky, 0)
    q = 0.5 * math.pi
    if (fx, fy) == ("sin", "cos"):
        return [(p, plus, h, 0.0, 0.0, omega, psi), (p, minus, h, 0.0, 0.0, omega, psi)]
    if (fx, fy) == ("cos", "sin"):
        return [(p, plus, h, 0.0, 0.0, omega, psi), (p, minus, -h, 0.0, 0.0, omega, psi)]
    if (fx, fy) == ("sin", "sin"):
        return [(p, minus, h, q, 0.0, omega, psi), (p, plus, -h, q, 0.0, omega, psi)]
    return [(p, plus, h, q, 0.0, omega, psi), (p, minus, h, q, 0.0, omega, psi)]


def _trig_product(p, amp, factors, omega, psi):
    """amp prod_d f_d(2 pi k_d x_d) cos(omega t + psi), f_d in {sin, cos}, as sine modes:
    cos a = sin(a + pi/2) and sin a sin b = [sin(a - b + pi/2) - sin(a + b + pi/2)]/2, applied
    factor by factor (a product of three factors becomes four modes)."""
    q = 0.5 * math.pi

    def factor(d, fn, kd):
        return tuple(kd if e == d else 0 for e in range(3)), (0.0 if fn == "sin" else q)

    k0, ph0 = factor(0, *factors[0])
    terms = [(float(amp), k0, ph0)]                 # (amplitude, k, phase) of sin(2 pi k.x + phase)
    for d in range(1, len(factors)):
        k1, ph1 = factor(d, *factors[d])
        out = []
        for (a, k, ph) in terms:
            out.append((0.5 * a, tuple(k[e] - k1[e] for e in range(3)), ph - ph1 + q))
            out.append((-0.5 * a, tuple(k[e] + k1[e] for e in range(3)), ph + ph1 + q))
        terms = out
    return [(p, k, a, ph, 0.0, omega, psi) for (a, k, ph) in terms]


def burgers_table(A=1.3):
    """The paper's Burgers field u = A sin(2 pi x) sin(2 pi y) cos t (supplement, MMS)."""
    return ModeTable("burgers", [0.0], _product_modes(0, A, "sin", "sin", 1, 1, 1.0, 0.0))


def maxwell_table(A=0.5, w=4.0):
    """The paper's TM field: E_z = A sin(kx x) sin(ky y) cos(w t), H_x = A sin(kx x) cos(ky y)
    sin(w t), H_y = -A (kx/ky) cos(kx x) sin(ky y) sin(w t), kx = 2 pi, ky = 4 pi."""
    s = -0.5 * math.pi                     # sin(w t) = cos(w t - pi/2)
    return ModeTable("maxwell", [0.0, 0.0, 0.0],
                     _product_modes(0, A, "sin", "sin", 1, 2, w, 0.0)
                     + _product_modes(1, A, "sin", "cos", 1, 2, w, s)
                     + _product_modes(2, -A * 0.5, "cos", "sin", 1, 2, w, s))


def euler_table(gamma=1.4):
    """The paper's Euler field in the units its scales divide out (rho0 = 1, c_s = 1):
    p0 = 1/gamma, background u0 = v0 = 3 c_s, k = 2 pi,
    rho = 1 + 0.3 sin(kx) cos(ky) cos t, u = 3 + 0.3 cos(kx) sin(ky) sin t,
    v = 3 + 0.3 sin(kx) sin(ky) sin t, p = p0 + (rho - 1) + 0.2 p0 cos(kx) sin(ky) sin t."""
    p0 = 1.0 / gamma
    s = -0.5 * math.pi
    modes = (_product_modes(0, 0.3, "sin", "cos", 1, 1, 1.0, 0.0)
             + _product_modes(1, 0.3, "cos", "sin", 1, 1, 1.0, s)
             + _product_modes(2, 0.3, "sin", "sin", 1, 1, 1.0, s)
             + _product_modes(3, 0.3, "sin", "cos", 1, 1, 1.0, 0.0)
             + _product_modes(3, 0.2 * p0, "cos", "sin", 1, 1, 1.0, s))
    return ModeTable("euler", [1.0, 3.0, 3.0, p0], modes, gamma=gamma)


def nsf_mms_table(case: NsfCase, seed: int = 2):
    """Forced NSF field: each primitive (rho, u, v, p) = the case's mean (p0 = rho0 R T0 = 1)
    + 4 seeded modes (k in [-3, 3]^2 without 0, amp U(0, 0.05), phase U(0, 2 pi)) times
    cos(t + psi), psi U(0, 2 pi)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    u0, v0 = case.U0
    modes = []
    for p in range(4):
        for k in _modes(rng, case.n_modes, 3, 2):
            modes.append((p, (int(k[0]), int(k[1]), 0), float(rng.uniform(0.0, case.amp_max)),
                          float(rng.uniform(0.0, TWO_PI)), 0.0, 1.0, float(rng.uniform(0.0, TWO_PI))))
    return ModeTable("nsf", [1.0, u0, v0, 1.0 * case.R * 1.0], modes, gamma=case.gamma, R=case.R)


@dataclass
class NsfPaperCase:
    """The paper's NSF manufactured flow (supplement, MMS section) in the units its scales
    divide out: rho0 = 1, sound speed c_s = 1 at T0 = 1, so R = 1/gamma and p0 = 1/gamma;
    mu = 3.52 Pa s / (rho0 c_s L) with rho0 = 1.225 kg/m^3, c_s = 340.2 m/s, L = 1 m;
    kappa = mu c_p / Pr, c_p = gamma R/(gamma - 1), Pr = 0.71; background (u0, v0) = (3, 2).
    Recipe: diffusive f = 2, tau_R = 60, g_tau = 6."""
    n: int
    gamma: float = 1.4
    Pr: float = 0.71
    f: float = 2.0
    tau_R: float = 60.0
    g_tau: float = 6.0

    @property
    def R(self):
        return 1.0 / self.gamma

    @property
    def mu(self):
        return 3.52 / (1.225 * 340.2)

    @property
    def kappa(self):
        return self.mu * (self.gamma * self.R / (self.gamma - 1.0)) / self.Pr

    @property
    def dx(self):
        return 1.0 / self.n

    @property
    def dt(self):
        return self.f * self.dx * self.dx

    def reference_state(self):
        p0 = 1.0 / self.gamma
        return [1.0, 3.0, 2.0, p0 / (self.gamma - 1.0) + 0.5 * 13.0] + [0.0] * 6

    def table(self, family="nsf"):
        """rho = 1 + 0.2 sin(kx) cos(ky) cos t, u = 3 + 0.2 cos(kx) sin(ky) sin t,
        v = 2 + 0.15 sin(kx) sin(ky) cos t, p = p0 + (rho - 1) + 0.2 p0 cos(kx) sin(ky) sin t."""
        p0, s = 1.0 / self.gamma, -0.5 * math.pi
        modes = (_product_modes(0, 0.2, "sin", "cos", 1, 1, 1.0, 0.0)
                 + _product_modes(1, 0.2, "cos", "sin", 1, 1, 1.0, s)
                 + _product_modes(2, 0.15, "sin", "sin", 1, 1, 1.0, 0.0)
                 + _product_modes(3, 0.2, "sin", "cos", 1, 1, 1.0, 0.0)
                 + _product_modes(3, 0.2 * p0, "cos", "sin", 1, 1, 1.0, s))
        return ModeTable(family, [1.0, 3.0, 2.0, p0], modes, gamma=self.gamma, R=self.R)

    def reference_state_cascade(self):
        """Q0 of the paper's 12-component cascade (uniform background, zero trackers)."""
        return self.reference_state()[:4] + [0.0] * 8


@dataclass
class MhdPaperCase:
    """The paper's MHD manufactured flow (supplement, MMS section), uniform along z, in the
    units its scales divide out (rho0 = 1, c_s = 1, p0 = 1/gamma, B in Alfven units):
    background u0 = v0 = 3, B0 = (0.5, 0.5, 0); eta = 3.4 m^2/s / (c_s L) = 0.01.
    Recipe of configuration 3: acoustic f = 0.05, tau_R = 160, g_tau = 4."""
    n: int
    gamma: float = 1.4
    eta: float = 0.01
    f: float = 0.05
    tau_R: float = 160.0
    g_tau: float = 4.0

    @property
    def dx(self):
        return 1.0 / self.n

    @property
    def dt(self):
        return self.f * self.dx

    def reference_state(self):
        p0 = 1.0 / self.gamma
        E0 = p0 / (self.gamma - 1.0) + 0.5 * 18.0 + 0.5 * 0.5
        return [1.0, 3.0, 3.0, 0.0, 0.5, 0.5, 0.0, E0, 0.0, 0.0, 0.0]

    def table(self):
        """rho = 1 + 0.3 sin(kx) cos(ky) cos t, p = p0 + (rho - 1) + 0.2 p0 cos(kx) sin(ky) sin t,
        u = 3 + 0.3 cos(kx) sin(ky) sin t, v = 3 + 0.3 sin(kx) sin(ky) sin t, w = 0,
        B_x = 0.5 - 0.3 cos(kx) sin(ky) sin t, B_y = 0.5 + 0.3 sin(kx) cos(ky) sin t, B_z = 0."""
        p0, s = 1.0 / self.gamma, -0.5 * math.pi
        modes = (_product_modes(0, 0.3, "sin", "cos", 1, 1, 1.0, 0.0)
                 + _product_modes(7, 0.3, "sin", "cos", 1, 1, 1.0, 0.0)
                 + _product_modes(7, 0.2 * p0, "cos", "sin", 1, 1, 1.0, s)
                 + _product_modes(1, 0.3, "cos", "sin", 1, 1, 1.0, s)
                 + _product_modes(2, 0.3, "sin", "sin", 1, 1, 1.0, s)
                 + _product_modes(4, -0.3, "cos", "sin", 1, 1, 1.0, s)
                 + _product_modes(5, 0.3, "sin", "cos", 1, 1, 1.0, s))
        return ModeTable("mhd", [1.0, 3.0, 3.0, 0.0, 0.5, 0.5, 0.0, p0], modes, gamma=self.gamma)


def mhd_mms_table(case: MhdCase, seed: int = 2):
    """Forced 3D MHD field: rho = 1 + 2 modes (amp 0.05), p = 1/gamma + 2 modes (amp 0.02),
    u from case.n_modes velocity modes and B = curl A from as many potential modes
    (amplitude case.amp / n_modes each, so div B = 0 exactly), every mode times
    cos(t + psi) with a seeded psi."""
    rng = np.random.Generator(np.random.PCG64(seed))
    scale = case.amp / case.n_modes
    modes = []

    def tphase():
        return float(rng.uniform(0.0, TWO_PI))
    for p, amp in ((0, 0.05), (7, 0.02)):
        for k in _modes(rng, 2, 2, 3):
            modes.append((p, tuple(int(c) for c in k), amp, float(rng.uniform(0.0, TWO_PI)), 0.0, 1.0, tphase()))
    for _ in range(case.n_modes):
        k, d, ph, ps = _modes(rng, 1, 2, 3)[0], rng.uniform(-1, 1, 3), float(rng.uniform(0, TWO_PI)), tphase()
        for c in range(3):
            modes.append((1 + c, tuple(int(v) for v in k), scale * float(d[c]), ph, 0.0, 1.0, ps))
    for _ in range(case.n_modes):
        k, d, ph, ps = _modes(rng, 1, 2, 3)[0], rng.uniform(-1, 1, 3), float(rng.uniform(0, TWO_PI)), tphase()
        kxd = np.cross(k, d) / float(np.linalg.norm(k))
        for c in range(3):          # B = curl of A = scale d sin(th)/(2 pi |k|): cos(th) (k x d)/|k|
            modes.append((4 + c, tuple(int(v) for v in k), scale * float(kxd[c]), ph + 0.5 * math.pi, 0.0, 1.0, ps))
    return ModeTable("mhd", [1.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 1.0 / case.gamma], modes, gamma=case.gamma)


@dataclass
class MhdPaper2DCase:
    """The paper's MHD manufactured flow on its own 2D system (18 components, Powell
    source), in the units its scales divide out: rho0 = 1, c_s = 1, p0 = 1/gamma, background
    u0 = v0 = 3, B0 = (0.5, 0.5), equal diffusivities mu = kappa = eta = 0.01
    (4.165 Pa s / (1.225 kg/m^3 x 340 m/s x 1 m) and 3.4 m^2/s / (340 m/s x 1 m)).
    Double-precision recipe: acoustic f = 0.025, tau_R = 140, g_tau = 4."""
    n: int
    gamma: float = 1.4
    mu: float = 0.01
    kappa: float = 0.01
    eta: float = 0.01
    f: float = 0.025
    tau_R: float = 140.0
    g_tau: float = 4.0

    @property
    def dx(self):
        return 1.0 / self.n

    @property
    def dt(self):
        return self.f * self.dx

    def reference_state(self):
        p0 = 1.0 / self.gamma
        E0 = p0 / (self.gamma - 1.0) + 0.5 * 18.0 + 0.5 * 0.5
        return [1.0, 3.0, 3.0, E0, 0.5, 0.5] + [0.0] * 12

    def table(self):
        """rho = 1 + 0.3 sin(kx) cos(ky) cos t, p = p0 + (rho - 1) + 0.2 p0 cos(kx) sin(ky) sin t,
        u = 3 + 0.3 cos(kx) sin(ky) sin t, v = 3 + 0.3 sin(kx) sin(ky) sin t,
        B_x = 0.5 - 0.3 cos(kx) sin(ky) sin t, B_y = 0.5 + 0.3 sin(kx) cos(ky) sin t."""
        p0, s = 1.0 / self.gamma, -0.5 * math.pi
        modes = (_product_modes(0, 0.3, "sin", "cos", 1, 1, 1.0, 0.0)
                 + _product_modes(3, 0.3, "sin", "cos", 1, 1, 1.0, 0.0)
                 + _product_modes(3, 0.2 * p0, "cos", "sin", 1, 1, 1.0, s)
                 + _product_modes(1, 0.3, "cos", "sin", 1, 1, 1.0, s)
                 + _product_modes(2, 0.3, "sin", "sin", 1, 1, 1.0, s)
                 + _product_modes(4, -0.3, "cos", "sin", 1, 1, 1.0, s)
                 + _product_modes(5, 0.3, "sin", "cos", 1, 1, 1.0, s))
        return ModeTable("mhd18", [1.0, 3.0, 3.0, p0, 0.5, 0.5], modes, gamma=self.gamma)


@dataclass
class AdrPaperCase:
    """The paper's ADR manufactured flow (supplement, MMS section):
    c = 0.5 + 0.5 sin(2 pi (x - u0 t)) cos(2 pi (y - u1 t)) e^{-t}, u = (0.1, -0.1), D = 0.01,
    reaction R c (1 - c) with R = 1.  Recipe: diffusive f = 1.9, tau_R = 50, g_tau = 6."""
    n: int
    a: tuple = (0.1, -0.1)
    D: float = 0.01
    R: float = 1.0
    f: float = 1.9
    tau_R: float = 50.0
    g_tau: float = 6.0

    @property
    def dx(self):
        return 1.0 / self.n

    @property
    def dt(self):
        return self.f * self.dx * self.dx

    def table(self):
        """sin(theta - w t) = sin(theta) cos(w t) + sin(theta + pi/2) cos(w t + pi/2), so each
        product term of the travelling wave is two standing modes decaying as e^{-t}."""
        q = 0.5 * math.pi
        modes = []
        for k, w in (((1, 1, 0), TWO_PI * (self.a[0] + self.a[1])), ((1, -1, 0), TWO_PI * (self.a[0] - self.a[1]))):
            modes += [(0, k, 0.25, 0.0, -1.0, w, 0.0), (0, k, 0.25, q, -1.0, w, q)]
        return ModeTable("adr", [0.5], modes)


def burgers_stability_grid(mach, omega, f=0.2):
    """(Ma, omega, A, tau_LB) for every pair of a Burgers stability sweep (Sec. 3, Burgers):
    Ma = lambda A / c_s with lambda = dt/dx = f (acoustic) and c_s^2 = 1/3, so the
    equilibria stay monotone in u exactly while Ma <= c_s; tau_LB = 1/omega."""
    cs = 1.0 / math.sqrt(3.0)
    return [(float(m), float(w), float(m) * cs / f, 1.0 / float(w)) for w in omega for m in mach]


@dataclass
class HcnsfPaperCase:
    """The paper's 3D homogenized NSF manufactured flow (supplement, HCNSF MMS section) in the
    units its scales divide out: rho0 = 1, c_s = sqrt(p0/rho0) = 1, p0 = 1, mean sound speed
    c_bar = sqrt(gamma), drift U0 = Ma c_bar with Ma = 0.5, amplitude A = 0.2;
    mu = kappa = 3.52 Pa s / (rho0 c_s L) and eta = 0.000348 s c_s / L with rho0 = 1.225 kg/m^3,
    c_s = 287.4 m/s, L = 1 m.  The prescribed fields and the solid displacement are read in
    the same units (amplitudes in c_s, time in L/c_s).
    Recipe: acoustic f = 0.05, tau_R = 10 (double) or 20 (float), g_tau = 3; N = 32 .. 256.
    The drag source takes the prescribed fields at the step's midpoint t^n + dt/2 and the
    equilibrium flux at t^n (theta = 1/2, theta_flux = 0)."""
    n: int
    gamma: float = 1.4
    A: float = 0.2
    Ma: float = 0.5
    f: float = 0.05
    tau_R: float = 10.0
    g_tau: float = 3.0
    alpha_mean: float = 0.5
    alpha_amp: float = 0.1
    rot: float = 0.2
    osc: float = 0.1
    c: tuple = (0.1, -0.1, 0.05)
    theta: float = 0.5       # time level of the prescribed fields in the drag source: t^n + theta dt
    theta_flux: float = 0.0  # the same inside the equilibrium flux

    @property
    def mu(self):
        return 3.52 / (1.225 * 287.4)

    @property
    def kappa(self):
        return 3.52 / (1.225 * 287.4)

    @property
    def eta(self):
        return 0.000348 * 287.4

    @property
    def U0(self):
        return self.Ma * math.sqrt(self.gamma)

    @property
    def dx(self):
        return 1.0 / self.n

    @property
    def dt(self):
        return self.f * self.dx

    def reference_state(self):
        U0 = self.U0
        return [1.0, U0, U0, U0, 1.0 / (self.gamma - 1.0) + 1.5 * U0 * U0] + [0.0] * 9

    def table(self):
        """rho = 1 + A s0 c1 s2 cos t, u_x = U0 + A c0 s1 s2 sin t, u_y = U0 + A s0 c1 s2 sin t,
        u_z = U0 + A s0 s1 c2 sin t, p = 1 + gamma (rho - 1) + A c0 s1 c2 sin t
        (s_d = sin(2 pi x_d), c_d = cos(2 pi x_d))."""
        A, g, s = self.A, self.gamma, -0.5 * math.pi
        fac = lambda a, b, c: [(a, 1), (b, 1), (c, 1)]
        modes = (_trig_product(0, A, fac("sin", "cos", "sin"), 1.0, 0.0)
                 + _trig_product(1, A, fac("cos", "sin", "sin"), 1.0, s)
                 + _trig_product(2, A, fac("sin", "cos", "sin"), 1.0, s)
                 + _trig_product(3, A, fac("sin", "sin", "cos"), 1.0, s)
                 + _trig_product(4, g * A, fac("sin", "cos", "sin"), 1.0, 0.0)
                 + _trig_product(4, A, fac("cos", "sin", "cos"), 1.0, s))
        U0 = self.U0
        return ModeTable("hcnsf", [1.0, U0, U0, U0, 1.0], modes, gamma=g)

    def prescribed(self, xx, t):
        """(alpha, u_s,x, u_s,y, u_s,z) at coordinates xx and time t: u_s is a rotation
        (amplitude rot) plus the translation c plus an oscillation (amplitude osc); alpha =
        a_mean + a_amp [sin k xi_0 + sin k xi_1 + sin k xi_2 + 2 sin k xi_0 sin k xi_1 sin k xi_2],
        xi = x - d, d = r(x) sin t + c t with r(x) the rotation's spatial pattern."""
        t = t if torch.is_tensor(t) else torch.full_like(xx[0], float(t))
        s = [torch.sin(TWO_PI * x) for x in xx]
        c = [torch.cos(TWO_PI * x) for x in xx]
        st, ct = torch.sin(t), torch.cos(t)
        r = [self.rot * s[0] * c[1] * c[2], -self.rot * c[0] * s[1] * c[2], self.rot * c[0] * c[1] * s[2]]
        us = [r[0] * ct + self.c[0] + self.osc * st * c[2],
              r[1] * ct + self.c[1] + self.osc * ct * c[0],
              r[2] * st + self.c[2] + self.osc * st * c[1]]
        sx = [torch.sin(TWO_PI * (xx[d] - r[d] * st - self.c[d] * t)) for d in range(3)]
        alpha = self.alpha_mean + self.alpha_amp * (sx[0] + sx[1] + sx[2] + 2.0 * sx[0] * sx[1] * sx[2])
        return [alpha] + us
