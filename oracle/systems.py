"""Conservation-law systems dQ/dt + div Phi(Q) = S(Q) (Eq. pde_target) for the oracle.

Each system gives the augmented state Q+ = (conserved, trackers) with its algebraic
flux Phi [K, D, ...] and state source S [K, ...], written in the paper's vector form.
Gradient trackers follow Eq. gradient_advection: Phi_G = G (x) u - I (x) V / tau_grad,
S_G = -G / tau_grad, with tau_grad = g_tau * dt (Sec. 2.1.1, supplement recipes).

Tracker index convention: component G_{V,b} approximates d V / d x_b.  The flux of
component G_{V,b} in direction c is G_{V,b} u_c - delta_{bc} V / tau_grad.

Every function here is plain torch on float64 tensors whose leading axis is the
component; trailing axes are the grid (or empty for a single node).
"""
from __future__ import annotations

import torch


def _eps(a, b, c):
    """Levi-Civita symbol epsilon_{abc} for a, b, c in {0, 1, 2}."""
    return (a - b) * (b - c) * (c - a) / 2


class System:
    name = ""
    K = 0
    D = 0
    n_cons = 0

    def flux(self, Q):
        raise NotImplementedError

    def source(self, Q):
        return torch.zeros_like(Q)

    # For building the exact augmented state Q+ of a manufactured solution:
    def parents(self, Qc):
        """Fields whose gradients the trackers carry, from the conserved state."""
        return []

    def trackers_from_grads(self, dP):
        """Tracker components from dP[p][b] = d parent_p / d x_b."""
        return []


class AdrCascade(System):
    """Scalar advection-diffusion(-reaction), Sec. 3 (ADR) and supplement Sec. 4 (ADR).

    Q = (u, G_x, G_y).  Phi_u = u a - nu G;  Phi_{G_b, c} = G_b a_c - delta_bc u / tau_g;
    S_u = R u (1 - u);  S_G = -G / tau_g.  With R = 0 this is u_t + a.grad u = nu lap u.
    """
    name = "adr"
    n_cons = 1

    def __init__(self, a, nu, tau_grad, R=0.0):
        self.a = [float(x) for x in a]
        self.D = len(self.a)
        self.K = 1 + self.D
        self.nu = float(nu)
        self.tau_grad = float(tau_grad)
        self.R = float(R)

    def flux(self, Q):
        u, G = Q[0], Q[1:]
        D = self.D
        rows = [torch.stack([u * self.a[c] - self.nu * G[c] for c in range(D)])]
        for b in range(D):
            rows.append(torch.stack([G[b] * self.a[c] - (u / self.tau_grad if b == c else 0 * u)
                                     for c in range(D)]))
        return torch.stack(rows)

    def source(self, Q):
        u, G = Q[0], Q[1:]
        return torch.stack([self.R * u * (1.0 - u)] + [-G[b] / self.tau_grad for b in range(self.D)])

    def parents(self, Qc):
        return [Qc[0]]

    def trackers_from_grads(self, dP):
        return [dP[0][b] for b in range(self.D)]


class NsfPrimitive(System):
    """Compressible Navier-Stokes-Fourier (Sec. 3, Eq. for NSF), closed with trackers of
    the primitives u, v, T themselves (Algorithm 1 "track V as an auxiliary field"; the
    HCNSF case tracks grad u and grad T the same way).

    Q = (rho, m_x, m_y, E, G_u(2), G_v(2), G_T(2)), u = m/rho,
    p = (gamma-1)(E - |m|^2 / (2 rho)), T = p / (rho R),
    tau_v = mu (L + L^T - 2/3 tr(L) I) with L_ab = G_{u_a, b},
    Phi_rho = m,  Phi_m = m (x) u + p I - tau_v,  Phi_E = (E + p) u - tau_v u - kappa G_T.
    """
    name = "nsf"
    K = 10
    D = 2
    n_cons = 4

    def __init__(self, gamma, R, mu, kappa, tau_grad):
        self.gamma, self.R, self.mu, self.kappa = float(gamma), float(R), float(mu), float(kappa)
        self.tau_grad = float(tau_grad)

    def primitives(self, Q):
        rho, m, E = Q[0], Q[1:3], Q[3]
        u = m / rho
        p = (self.gamma - 1.0) * (E - 0.5 * (m[0] * m[0] + m[1] * m[1]) / rho)
        T = p / (rho * self.R)
        return rho, u, p, T

    def flux(self, Q):
        rho, u, p, T = self.primitives(Q)
        m, E = Q[1:3], Q[3]
        L = [[Q[4], Q[5]], [Q[6], Q[7]]]
        GT = [Q[8], Q[9]]
        div = L[0][0] + L[1][1]
        tv = [[self.mu * (L[a][b] + L[b][a] - (2.0 / 3.0) * div * (1.0 if a == b else 0.0))
               for b in range(2)] for a in range(2)]
        rows = [torch.stack([m[0], m[1]])]
        for a in range(2):
            rows.append(torch.stack([m[a] * u[b] + (p if a == b else 0 * p) - tv[a][b]
                                     for b in range(2)]))
        rows.append(torch.stack([(E + p) * u[b] - (tv[b][0] * u[0] + tv[b][1] * u[1])
                                 - self.kappa * GT[b] for b in range(2)]))
        parents = [u[0], u[1], T]
        for pi, V in enumerate(parents):
            for b in range(2):
                G = Q[4 + 2 * pi + b]
                rows.append(torch.stack([G * u[c] - (V / self.tau_grad if b == c else 0 * V)
                                         for c in range(2)]))
        return torch.stack(rows)

    def source(self, Q):
        S = torch.zeros_like(Q)
        S[4:] = -Q[4:] / self.tau_grad
        return S

    def parents(self, Qc):
        rho, u, p, T = self.primitives(Qc)
        return [u[0], u[1], T]

    def trackers_from_grads(self, dP):
        return [dP[p][b] for p in range(3) for b in range(2)]


class MhdCurrent(System):
    """3D resistive MHD (Sec. 3, Eq. for MHD, without viscosity and heat flux) closed with
    a tracker of the current density j = curl B instead of grad B.

    Q = (rho, m(3), B(3), E, j(3)), p = (gamma-1)(E - |m|^2/(2 rho) - |B|^2/2),
    p_tot = p + |B|^2/2,
    Phi_m = m (x) u + p_tot I - B (x) B,
    Phi_B[a][b] = B_a u_b - u_a B_b + eta eps_abc j_c   (curl form of -eta grad B),
    Phi_E = (E + p_tot) u - B (u.B) + eta (j x B),
    Phi_j[a][b] = j_a u_b - eps_abc B_c / tau_grad,  S_j = -j / tau_grad,
    whose steady state is j = curl B (the tracker construction with I (x) V replaced by
    the Levi-Civita contraction).
    """
    name = "mhd"
    K = 11
    D = 3
    n_cons = 8

    def __init__(self, gamma, eta, tau_grad):
        self.gamma, self.eta, self.tau_grad = float(gamma), float(eta), float(tau_grad)

    def flux(self, Q):
        rho, m, B, E, j = Q[0], Q[1:4], Q[4:7], Q[7], Q[8:11]
        u = m / rho
        b2 = B[0] * B[0] + B[1] * B[1] + B[2] * B[2]
        p = (self.gamma - 1.0) * (E - 0.5 * (m[0] * m[0] + m[1] * m[1] + m[2] * m[2]) / rho - 0.5 * b2)
        ptot = p + 0.5 * b2
        udb = u[0] * B[0] + u[1] * B[1] + u[2] * B[2]
        jxB = [j[1] * B[2] - j[2] * B[1], j[2] * B[0] - j[0] * B[2], j[0] * B[1] - j[1] * B[0]]
        rows = [torch.stack([m[0], m[1], m[2]])]
        for a in range(3):
            rows.append(torch.stack([m[a] * u[b] + (ptot if a == b else 0 * ptot) - B[a] * B[b]
                                     for b in range(3)]))
        for a in range(3):
            rows.append(torch.stack([B[a] * u[b] - u[a] * B[b]
                                     + self.eta * sum(_eps(a, b, c) * j[c] for c in range(3))
                                     for b in range(3)]))
        rows.append(torch.stack([(E + ptot) * u[b] - B[b] * udb + self.eta * jxB[b] for b in range(3)]))
        for a in range(3):
            rows.append(torch.stack([j[a] * u[b]
                                     - sum(_eps(a, b, c) * B[c] for c in range(3)) / self.tau_grad
                                     for b in range(3)]))
        return torch.stack(rows)

    def source(self, Q):
        S = torch.zeros_like(Q)
        S[8:] = -Q[8:] / self.tau_grad
        return S

    def parents(self, Qc):
        return [Qc[4], Qc[5], Qc[6]]

    def trackers_from_grads(self, dP):
        # j_a = eps_abc d_b B_c
        return [sum(_eps(a, b, c) * dP[c][b] for b in range(3) for c in range(3) if _eps(a, b, c) != 0)
                for a in range(3)]


class NsfConservedGradients(System):
    """Compressible Navier-Stokes-Fourier with trackers of the conserved fields, the
    paper's own 12-component cascade (Sec. 2.1.1: the chain rule expands grad u and grad T
    over the gradients of rho, rho u and E; supplement, NSF system).

    Q = (rho, m_x, m_y, E, G_rho(2), G_mx(2), G_my(2), G_E(2)), G_{V,b} ~ d V / d x_b.
    grad u = (G_m - u (x) G_rho) / rho, i.e. d u_a / d x_b = (G_{m_a,b} - u_a G_{rho,b}) / rho;
    grad p = (gamma-1)(G_E - u . G_m + |u|^2/2 G_rho), u . G_m = sum_a u_a G_{m_a};
    grad T = (grad p / R - T G_rho) / rho, T = p / (rho R).
    Phi_rho = m, Phi_m = m (x) u + p I - tau_v, Phi_E = (E + p) u - tau_v u - kappa grad T,
    tau_v = mu (L + L^T - 2/3 tr(L) I), L = grad u; trackers of V in (rho, m_x, m_y, E).
    """
    name = "nsf12"
    K = 12
    D = 2
    n_cons = 4

    def __init__(self, gamma, R, mu, kappa, tau_grad):
        self.gamma, self.R, self.mu, self.kappa = float(gamma), float(R), float(mu), float(kappa)
        self.tau_grad = float(tau_grad)

    def flux(self, Q):
        g1 = self.gamma - 1.0
        rho, m, E = Q[0], Q[1:3], Q[3]
        u = m / rho
        u2 = u[0] * u[0] + u[1] * u[1]
        p = g1 * (E - 0.5 * rho * u2)
        T = p / (rho * self.R)
        Gr, Gm, GE = Q[4:6], [Q[6:8], Q[8:10]], Q[10:12]
        L = [[(Gm[a][b] - u[a] * Gr[b]) / rho for b in range(2)] for a in range(2)]
        Gp = [g1 * (GE[b] - (u[0] * Gm[0][b] + u[1] * Gm[1][b]) + 0.5 * u2 * Gr[b]) for b in range(2)]
        GT = [(Gp[b] / self.R - T * Gr[b]) / rho for b in range(2)]
        div = L[0][0] + L[1][1]
        tv = [[self.mu * (L[a][b] + L[b][a] - (2.0 / 3.0) * div * (1.0 if a == b else 0.0))
               for b in range(2)] for a in range(2)]
        rows = [torch.stack([m[0], m[1]])]
        for a in range(2):
            rows.append(torch.stack([m[a] * u[b] + (p if a == b else 0 * p) - tv[a][b] for b in range(2)]))
        rows.append(torch.stack([(E + p) * u[b] - (tv[b][0] * u[0] + tv[b][1] * u[1])
                                 - self.kappa * GT[b] for b in range(2)]))
        for pi, V in enumerate([rho, m[0], m[1], E]):
            for b in range(2):
                G = Q[4 + 2 * pi + b]
                rows.append(torch.stack([G * u[c] - (V / self.tau_grad if b == c else 0 * V)
                                         for c in range(2)]))
        return torch.stack(rows)

    def source(self, Q):
        S = torch.zeros_like(Q)
        S[4:] = -Q[4:] / self.tau_grad
        return S

    def parents(self, Qc):
        return [Qc[0], Qc[1], Qc[2], Qc[3]]

    def trackers_from_grads(self, dP):
        return [dP[p][b] for p in range(4) for b in range(2)]


class MhdPowell2D(System):
    """2D viscous, heat-conducting resistive MHD with Powell divergence cleaning, the
    paper's own 18-component cascade (Sec. 3, MHD system; supplement, MHD system):
    trackers of rho, rho u, E and B, the chain rule for grad u and grad T (T = p / rho),
    and div B = tr G_B in the Powell source.

    Q = (rho, m_x, m_y, E, B_x, B_y, G_rho(2), G_mx(2), G_my(2), G_E(2), G_Bx(2), G_By(2)).
    p = (gamma-1)(E - |m|^2/(2 rho) - |B|^2/2), p_t = p + |B|^2/2,
    grad p = (gamma-1)(G_E - u . G_m + |u|^2/2 G_rho - B . G_B), grad T = (grad p - T G_rho)/rho,
    j_z = G_{By,x} - G_{Bx,y}, j x B = (-j_z B_y, j_z B_x),
    Phi_m = m (x) u + p_t I - B (x) B - tau_v,
    Phi_E = (E + p_t) u - B (u . B) - tau_v u - K grad T + eta (j x B),
    Phi_B = B (x) u - u (x) B - eta G_B,  S = -(div B) (0, B, u . B, u) on (rho, m, E, B).
    """
    name = "mhd18"
    K = 18
    D = 2
    n_cons = 6

    def __init__(self, gamma, mu, kappa, eta, tau_grad):
        self.gamma, self.mu, self.kappa, self.eta = float(gamma), float(mu), float(kappa), float(eta)
        self.tau_grad = float(tau_grad)

    def _parts(self, Q):
        g1 = self.gamma - 1.0
        rho, m, E, B = Q[0], Q[1:3], Q[3], Q[4:6]
        u = m / rho
        u2 = u[0] * u[0] + u[1] * u[1]
        b2 = B[0] * B[0] + B[1] * B[1]
        p = g1 * (E - 0.5 * rho * u2 - 0.5 * b2)
        return rho, m, E, B, u, u2, b2, p

    def flux(self, Q):
        g1 = self.gamma - 1.0
        rho, m, E, B, u, u2, b2, p = self._parts(Q)
        pt = p + 0.5 * b2
        T = p / rho
        Gr, Gm, GE, GB = Q[6:8], [Q[8:10], Q[10:12]], Q[12:14], [Q[14:16], Q[16:18]]
        L = [[(Gm[a][b] - u[a] * Gr[b]) / rho for b in range(2)] for a in range(2)]
        Gp = [g1 * (GE[b] - (u[0] * Gm[0][b] + u[1] * Gm[1][b]) + 0.5 * u2 * Gr[b]
                    - (B[0] * GB[0][b] + B[1] * GB[1][b])) for b in range(2)]
        GT = [(Gp[b] - T * Gr[b]) / rho for b in range(2)]
        div = L[0][0] + L[1][1]
        tv = [[self.mu * (L[a][b] + L[b][a] - (2.0 / 3.0) * div * (1.0 if a == b else 0.0))
               for b in range(2)] for a in range(2)]
        jz = GB[1][0] - GB[0][1]
        jxB = [-jz * B[1], jz * B[0]]
        uB = u[0] * B[0] + u[1] * B[1]
        rows = [torch.stack([m[0], m[1]])]
        for a in range(2):
            rows.append(torch.stack([m[a] * u[b] + (pt if a == b else 0 * pt) - B[a] * B[b] - tv[a][b]
                                     for b in range(2)]))
        rows.append(torch.stack([(E + pt) * u[b] - B[b] * uB - (tv[b][0] * u[0] + tv[b][1] * u[1])
                                 - self.kappa * GT[b] + self.eta * jxB[b] for b in range(2)]))
        for a in range(2):
            rows.append(torch.stack([B[a] * u[b] - u[a] * B[b] - self.eta * GB[a][b] for b in range(2)]))
        for pi, V in enumerate([rho, m[0], m[1], E, B[0], B[1]]):
            for b in range(2):
                G = Q[6 + 2 * pi + b]
                rows.append(torch.stack([G * u[c] - (V / self.tau_grad if b == c else 0 * V)
                                         for c in range(2)]))
        return torch.stack(rows)

    def source(self, Q):
        rho, m, E, B, u, u2, b2, p = self._parts(Q)
        divB = Q[14] + Q[17]
        S = torch.zeros_like(Q)
        S[1], S[2] = -divB * B[0], -divB * B[1]
        S[3] = -divB * (u[0] * B[0] + u[1] * B[1])
        S[4], S[5] = -divB * u[0], -divB * u[1]
        S[6:] = -Q[6:] / self.tau_grad
        return S

    def parents(self, Qc):
        return [Qc[k] for k in range(6)]

    def trackers_from_grads(self, dP):
        return [dP[p][b] for p in range(6) for b in range(2)]


class Burgers(System):
    """Inviscid Burgers, Sec. 3: Phi = (u^2/2, u^2/2) (and u^2/2 in 1D)."""
    name = "burgers"
    K = 1
    n_cons = 1

    def __init__(self, D=2):
        self.D = D

    def flux(self, Q):
        h = 0.5 * Q[0] * Q[0]
        return torch.stack([torch.stack([h] * self.D)])


class Euler(System):
    """Compressible Euler, Sec. 3: Phi = (m, m (x) u + p I, (E + p) u)."""
    name = "euler"
    K = 4
    D = 2
    n_cons = 4

    def __init__(self, gamma=1.4):
        self.gamma = float(gamma)

    def flux(self, Q):
        rho, m, E = Q[0], Q[1:3], Q[3]
        u = m / rho
        p = (self.gamma - 1.0) * (E - 0.5 * (m[0] * m[0] + m[1] * m[1]) / rho)
        rows = [torch.stack([m[0], m[1]])]
        for a in range(2):
            rows.append(torch.stack([m[a] * u[b] + (p if a == b else 0 * p) for b in range(2)]))
        rows.append(torch.stack([(E + p) * u[b] for b in range(2)]))
        return torch.stack(rows)


class MaxwellTM(System):
    """Maxwell TM mode, Sec. 3: Q = (E_z, H_x, H_y),
    Phi = (c(-H_y, H_x), c(0, E_z), c(-E_z, 0))."""
    name = "maxwell"
    K = 3
    D = 2
    n_cons = 3

    def __init__(self, c=1.0):
        self.c = float(c)

    def flux(self, Q):
        ez, hx, hy = Q[0], Q[1], Q[2]
        z = 0 * ez
        return self.c * torch.stack([torch.stack([-hy, hx]), torch.stack([z, ez]),
                                     torch.stack([-ez, z])])


class HomogenizedNsf3D(System):
    """3D homogenized compressible Navier-Stokes-Fourier (Sec. 3, HCNSF; supplement, HCNSF
    system), with prescribed porosity alpha(x, t) and solid velocity u_s(x, t).

    Q = (rho, m(3), E, G_11, G_22, G_T(3), G_00, G_01, G_02, G_12), the paper's order, where
    G_ab ~ (sym grad u)_ab and G_T ~ grad T, T = p / rho (gas constant 1),
    p = (gamma-1)(E - |m|^2/(2 rho)),  tau_v = mu (2 G - 2/3 tr(G) I),
    Phi_rho = m,  Phi_m = m (x) u + p I - alpha tau_v,
    Phi_E = (E + p) u - alpha tau_v u - alpha kappa G_T,
    Phi_{G_ab, c} = G_ab u_c - (delta_ac u_b + delta_bc u_a) / (2 tau_grad)   (sym(I (x) u)),
    Phi_{G_T,b, c} = G_T,b u_c - delta_bc T / tau_grad,
    S_m = (1-alpha)/eta (rho u_s - m),  S_E = S_m . u,  S_G = -G / tau_grad.

    `fields(xx, t)` returns (alpha, u_s,0, u_s,1, u_s,2) at node coordinates xx and time t;
    flux and source take those values as `cf`.
    """
    name = "hcnsf"
    K = 14
    D = 3
    n_cons = 5
    prescribed = True
    # (a, b) of the symmetric-gradient components, by position in Q
    SYM = {5: (1, 1), 6: (2, 2), 10: (0, 0), 11: (0, 1), 12: (0, 2), 13: (1, 2)}

    def __init__(self, gamma, mu, kappa, eta, tau_grad, fields):
        self.gamma, self.mu, self.kappa, self.eta = float(gamma), float(mu), float(kappa), float(eta)
        self.tau_grad = float(tau_grad)
        self.fields = fields

    def _parts(self, Q):
        rho, m, E = Q[0], Q[1:4], Q[4]
        u = m / rho
        p = (self.gamma - 1.0) * (E - 0.5 * (m[0] * u[0] + m[1] * u[1] + m[2] * u[2]))
        G = [[None] * 3 for _ in range(3)]
        for k, (a, b) in self.SYM.items():
            G[a][b] = G[b][a] = Q[k]
        return rho, m, E, u, p, G, Q[7:10]

    def flux(self, Q, cf):
        alpha = cf[0]
        rho, m, E, u, p, G, GT = self._parts(Q)
        tr = G[0][0] + G[1][1] + G[2][2]
        tv = [[self.mu * (2.0 * G[a][b] - (2.0 / 3.0) * tr * (1.0 if a == b else 0.0)) for b in range(3)]
              for a in range(3)]
        T = p / rho
        itg = 1.0 / self.tau_grad
        rows = [None] * self.K
        rows[0] = torch.stack([m[0], m[1], m[2]])
        for a in range(3):
            rows[1 + a] = torch.stack([m[a] * u[b] + (p if a == b else 0 * p) - alpha * tv[a][b]
                                       for b in range(3)])
        rows[4] = torch.stack([(E + p) * u[b] - alpha * (tv[b][0] * u[0] + tv[b][1] * u[1] + tv[b][2] * u[2])
                               - alpha * self.kappa * GT[b] for b in range(3)])
        for k, (a, b) in self.SYM.items():
            rows[k] = torch.stack([Q[k] * u[c] - 0.5 * itg * ((u[b] if a == c else 0 * u[b])
                                                              + (u[a] if b == c else 0 * u[a]))
                                   for c in range(3)])
        for b in range(3):
            rows[7 + b] = torch.stack([GT[b] * u[c] - (T * itg if b == c else 0 * T) for c in range(3)])
        return torch.stack(rows)

    def source(self, Q, cf):
        alpha, us = cf[0], cf[1:4]
        rho, m, E, u, p, G, GT = self._parts(Q)
        drag = (1.0 - alpha) / self.eta
        S = torch.zeros_like(Q)
        for a in range(3):
            S[1 + a] = drag * (rho * us[a] - m[a])
        S[4] = S[1] * u[0] + S[2] * u[1] + S[3] * u[2]
        S[5:] = -Q[5:] / self.tau_grad
        return S

    def parents(self, Qc):
        rho, m, E = Qc[0], Qc[1:4], Qc[4]
        u = m / rho
        p = (self.gamma - 1.0) * (E - 0.5 * (m[0] * u[0] + m[1] * u[1] + m[2] * u[2]))
        return [u[0], u[1], u[2], p / rho]

    def trackers_from_grads(self, dP):
        sym = lambda a, b: 0.5 * (dP[a][b] + dP[b][a])
        return [sym(1, 1), sym(2, 2), dP[3][0], dP[3][1], dP[3][2], sym(0, 0), sym(0, 1), sym(0, 2), sym(1, 2)]


def flux_at(system, Q, xx, t):
    """Phi(Q), or Phi(Q; c(x, t)) for a system with prescribed coefficient fields."""
    if getattr(system, "prescribed", False):
        return system.flux(Q, system.fields(xx, t))
    return system.flux(Q)


def source_at(system, Q, xx, t):
    """S(Q), or S(Q; c(x, t)) for a system with prescribed coefficient fields."""
    if getattr(system, "prescribed", False):
        return system.source(Q, system.fields(xx, t))
    return system.source(Q)
