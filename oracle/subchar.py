"""Sub-characteristic admissibility check (Sec. 2.3.2, Eqs. subchar_scalar and
subchar_system): max |eig sum_a n_a A_a(Q)| <= a over unit directions n and attained
states, with A_a = d Phi_a / d Q.  In lattice units (a = c_s dx/dt) this reads
(dt/dx) max|eig| <= c_s.  The sharper monotone-equilibrium bound of Sec. 3 (Burgers
paragraph) reads (dt/dx) max|f'| <= c_s^2.

The Jacobians come from automatic differentiation of the oracle flux and the
eigenvalues from numpy; this is a slow check, evaluated node by node.
"""
from __future__ import annotations

import math

import numpy as np
import torch


def directions(D, n):
    """n unit directions: equispaced angles on [0, pi) in 2D (the spectrum of -A_n is
    minus that of A_n), a Fibonacci sphere in 3D, +-1 in 1D."""
    if D == 1:
        return np.array([[1.0]])
    if D == 2:
        th = np.pi * np.arange(n) / n
        return np.stack([np.cos(th), np.sin(th)], 1)
    i = np.arange(n) + 0.5
    phi = np.arccos(1 - 2 * i / n)
    th = np.pi * (1 + 5 ** 0.5) * i
    return np.stack([np.cos(th) * np.sin(phi), np.sin(th) * np.sin(phi), np.cos(phi)], 1)


def flux_jacobian(system, q, cf=None):
    """J[k, a, l] = d Phi_{k,a} / d Q_l at one node state q [K] (with the node's prescribed
    coefficients cf for systems that have them)."""
    q = torch.as_tensor(q, dtype=torch.float64)
    if cf is None:
        return torch.autograd.functional.jacobian(lambda v: system.flux(v), q)
    return torch.autograd.functional.jacobian(lambda v: system.flux(v, cf), q)


def node_max_speed(system, q, dirs, cf=None):
    J = flux_jacobian(system, q, cf).numpy()
    best = 0.0
    for n in dirs:
        A = np.einsum("kal,a->kl", J, n)
        best = max(best, float(np.max(np.abs(np.linalg.eigvals(A)))))
    return best


def max_speed(system, Q, n_dirs=64, nodes=None, cf=None):
    """max over the given node indices (flattened grid; all nodes if None) and over
    n_dirs directions of the spectral radius of A_n.  cf: the prescribed coefficient fields
    on the same grid (a sequence of tensors), for systems that take them."""
    K = Q.shape[0]
    Qf = Q.reshape(K, -1)
    idx = range(Qf.shape[1]) if nodes is None else nodes
    dirs = directions(system.D, n_dirs)
    cff = None if cf is None else [c.reshape(-1) for c in cf]
    return max(node_max_speed(system, Qf[:, j], dirs, None if cff is None else [c[j] for c in cff]) for j in idx)


def check(system, Q, lam, cs2, n_dirs=64, nodes=None):
    s = max_speed(system, Q, n_dirs, nodes)
    cs = math.sqrt(cs2)
    return {"max_speed": s, "lattice_speed": lam * s, "bound_cs": cs, "bound_monotone": cs2,
            "ok": lam * s <= cs, "monotone_ok": lam * s <= cs2}
