"""The kinetic relaxation scheme, plain FP64, push form (test infrastructure).

Steps, in the paper's order and notation:
  * lattice scaling (Sec. 2.3.1 refinement laws, supplement recipes): dx = 1/N,
    dt = f dx (acoustic) or f dx^2 (diffusive), tau_LB = 1/2 + tau_R dt for the
    conserved fields (Sec. 2.3.1), tau_LB = g_tau + 1 and tau_grad = g_tau dt for
    trackers (supplement, recipes paragraph);
  * equilibrium, Eq. feq:  f^eq_{k,i} = w_i (Q_k + c_i . [(dt/dx) Phi_k] / c_s^2);
  * moments, Eq. moments:  Q_k = sum_i f_{k,i};
  * BGK collide-and-stream, Eq. lbe_update:
      f_{k,i}(x + c_i dx, t + dt) = f - (f - f^eq)/tau_LB + dt w_i S_k^total(x, t + dt/2),
    with state sources S(Q) taken at Q^n and explicit (manufactured) forcing at the
    midpoint t + dt/2;
  * reference/equilibrium shift (Sec. 2.4.3): f* = f - f^eq(Q0, F0), F0 = Phi(Q0).

Prescribed coefficient fields c(x, t) (HCNSF porosity and solid velocity) are evaluated
at the node coordinates x = (i, j, l) dx and at the time level of the state they multiply:
t^n in the equilibrium flux and the state source of step n, t = 0 at initialisation;
`source_theta` and `flux_theta` move the source's and the flux's fields to t^n + theta dt.

Arrays: populations f are [K, q, *grid], fields Q are [K, *grid], grid = (nz,) ny, nx.
The streaming here pushes post-collision values to x + c_i with torch.roll, exactly as
Eq. lbe_update is written.
"""
from __future__ import annotations

import math

import torch

from .lattice import Lattice
from .systems import flux_at, source_at

F64 = torch.float64


def lattice_steps(N, f, scaling):
    """(dx, dt) for N nodes per unit length under the named refinement law."""
    dx = 1.0 / N
    if scaling == "acoustic":
        return dx, f * dx
    if scaling == "diffusive":
        return dx, f * dx * dx
    raise ValueError(scaling)


def tau_vector(system, dt, tau_cons=None, tau_R=None, g_tau=None):
    """Per-component tau_LB: conserved fields tau_cons (given) or 1/2 + tau_R dt;
    trackers g_tau + 1."""
    if tau_cons is None:
        tau_cons = 0.5 + tau_R * dt
    taus = []
    for k in range(system.K):
        if k < system.n_cons:
            taus.append(tau_cons)
        else:
            taus.append(float(g_tau) + 1.0)
    if any(isinstance(t, torch.Tensor) for t in taus):
        return torch.stack([t if isinstance(t, torch.Tensor) else torch.tensor(t, dtype=F64)
                            for t in taus])
    return torch.tensor(taus, dtype=F64)


class Scheme:
    def __init__(self, system, lattice: Lattice, shape, dx, dt, tau, mms=None,
                 shifted=False, Q0=None, source_theta=0.0, flux_theta=0.0, origin=None):
        self.sys = system
        self.lat = lattice
        self.shape = tuple(shape)
        self.dx, self.dt = float(dx), float(dt)
        self.lam = self.dt / self.dx
        self.tau = tau if isinstance(tau, torch.Tensor) else torch.tensor(tau, dtype=F64)
        self.c = lattice.c
        self.w = [float(x) for x in lattice.w]
        self.cs2 = float(lattice.cs2)
        self.mms = mms
        self.shifted = shifted
        self.source_theta = float(source_theta)
        self.flux_theta = float(flux_theta)
        self.Q0 = None if Q0 is None else torch.as_tensor(Q0, dtype=F64)
        # node coordinates (x, y[, z]), x fastest, for prescribed coefficient fields; `origin`
        # (grid order, as shape) offsets the node indices of a slab of a larger domain
        org = origin if origin is not None else (0,) * len(self.shape)
        axes = [(torch.arange(n, dtype=F64) + o) * self.dx for n, o in zip(self.shape, org)]
        self.xx = tuple(m.contiguous() for m in reversed(torch.meshgrid(*axes, indexing="ij")))
        if shifted:
            q0 = self.Q0.reshape((system.K,) + (1,) * len(self.shape))
            self.feq0 = self.feq(q0)      # [K, q, 1, ...] background equilibrium
        assert lattice.D == system.D

    # -- Eq. feq --------------------------------------------------------------------
    def feq(self, Q, t=0.0):
        Phi = flux_at(self.sys, Q, self.xx, t + self.flux_theta * self.dt)   # [K, D, *grid]
        out = []
        for i, ci in enumerate(self.c):
            cphi = sum(ci[d] * Phi[:, d] for d in range(self.lat.D) if ci[d] != 0)
            out.append(self.w[i] * (Q + self.lam * cphi / self.cs2))
        return torch.stack(out, dim=1)

    # -- Eq. moments ----------------------------------------------------------------
    def moments(self, f):
        Q = f.sum(dim=1)
        if self.shifted:
            Q = Q + self.Q0.reshape((self.sys.K,) + (1,) * len(self.shape))
        return Q

    def init(self, Q, t=0.0):
        """Populations at the (shifted) equilibrium of the given fields (supplement,
        recipes paragraph)."""
        f = self.feq(Q, t)
        return f - self.feq0 if self.shifted else f

    def source_total(self, Q, t):
        S = source_at(self.sys, Q, self.xx, t + self.source_theta * self.dt)
        if self.mms is not None:
            Sm = self.mms(t + 0.5 * self.dt)          # all K components, or the conserved ones
            S = S + Sm if Sm.shape[0] == self.sys.K else torch.cat([S[: self.sys.n_cons] + Sm, S[self.sys.n_cons:]])
        return S

    def collide(self, f, t):
        """Post-collision populations at every node (right-hand side of Eq. lbe_update)."""
        Q = self.moments(f)
        fe = self.feq(Q, t)
        if self.shifted:
            fe = fe - self.feq0
        S = self.source_total(Q, t)
        K = self.sys.K
        tau = self.tau.reshape((K, 1) + (1,) * len(self.shape))
        w = torch.tensor(self.w, dtype=F64).reshape((1, -1) + (1,) * len(self.shape))
        return f - (f - fe) / tau + self.dt * w * S.unsqueeze(1)

    def stream(self, post):
        """Push population i from x to x + c_i (periodic)."""
        D = self.lat.D
        out = []
        for i, ci in enumerate(self.c):
            p = post[:, i]
            shifts = tuple(ci[d] for d in range(D) if ci[d] != 0)
            dims = tuple(-(d + 1) for d in range(D) if ci[d] != 0)
            out.append(torch.roll(p, shifts=shifts, dims=dims) if shifts else p)
        return torch.stack(out, dim=1)

    def step(self, f, t):
        return self.stream(self.collide(f, t))

    def run(self, f, n_steps, t0=0.0):
        t = t0
        for n in range(n_steps):
            f = self.step(f, t0 + n * self.dt)
        return f


def rel_norms(Qh, Qex):
    """Relative discrete L2 and Linf errors per component (Sec. 4): the L2 norm is
    (N_cells^-1 sum f^2)^(1/2); the relative Linf is max|e| / max|Q_ex|."""
    K = Qh.shape[0]
    e = (Qh - Qex).reshape(K, -1)
    r = Qex.reshape(K, -1)
    l2 = torch.sqrt((e * e).mean(1)) / torch.sqrt((r * r).mean(1))
    linf = e.abs().amax(1) / r.abs().amax(1)
    return l2, linf


def eoc(ns, errs):
    """Empirical order of convergence: minus the least-squares slope of log2 e against
    log2 N over the whole sequence (Sec. 4)."""
    xs = [math.log2(n) for n in ns]
    ys = [math.log2(e) for e in errs]
    mx, my = sum(xs) / len(xs), sum(ys) / len(ys)
    num = sum((x - mx) * (y - my) for x, y in zip(xs, ys))
    den = sum((x - mx) ** 2 for x in xs)
    return -num / den
