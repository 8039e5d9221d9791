"""Shared test helpers: oracle schemes for the same cases the GPU runs."""
import math

import torch

import oracle
import synthetic as syn
from oracle import systems as S
from oracle.mms import make_mms

F64 = torch.float64


def oracle_adr(case: syn.AdrCase, lattice="D2Q5", forcing=True, shifted=False):
    sysm = S.AdrCascade(case.a_phys, case.nu, case.g_tau * case.dt)
    xs = syn.coords((case.n, case.n))
    # the closed-form ADR_SEPARABLE forcing acts on the conserved component alone
    mms = make_mms(sysm, lambda x, y, t: syn.adr_exact(case, x, y, t).unsqueeze(0), xs, dt=case.dt,
                   conserved_only=True) if forcing else None
    tau = oracle.tau_vector(sysm, case.dt, tau_cons=case.tau_u, g_tau=case.g_tau)
    return oracle.Scheme(sysm, oracle.LATTICES[lattice], (case.n, case.n), case.dx, case.dt, tau,
                         mms=mms, shifted=shifted, Q0=[1.0, 0.0, 0.0])


def oracle_nsf(case: syn.NsfCase, lattice="D2Q9"):
    sysm = S.NsfPrimitive(case.gamma, case.R, case.mu, case.kappa, case.g_tau * case.dt)
    tau = oracle.tau_vector(sysm, case.dt, tau_R=case.tau_R, g_tau=case.g_tau)
    return oracle.Scheme(sysm, oracle.LATTICES[lattice], (case.n, case.n), case.dx, case.dt, tau)


def oracle_mhd(case: syn.MhdCase, lattice="D3Q19"):
    sysm = S.MhdCurrent(case.gamma, case.eta, case.g_tau * case.dt)
    tau = oracle.tau_vector(sysm, case.dt, tau_R=case.tau_R, g_tau=case.g_tau)
    n = case.n
    return oracle.Scheme(sysm, oracle.LATTICES[lattice], (n, n, n), case.dx, case.dt, tau)


def rel_linf_per_field(a, b):
    """max|a - b| / max|b| per component (leading axis)."""
    K = a.shape[0]
    d = (a - b).reshape(K, -1).abs().amax(1)
    r = b.reshape(K, -1).abs().amax(1)
    return d / r


def fluct_rel_l2(a, b, Q0):
    """||a - b||_2 / ||b - Q0||_2 per component: error relative to the fluctuation."""
    K = a.shape[0]
    q0 = torch.as_tensor(Q0, dtype=F64).reshape((K,) + (1,) * (a.dim() - 1))
    e = (a - b).reshape(K, -1)
    r = (b - q0).reshape(K, -1)
    return torch.sqrt((e * e).sum(1)) / torch.sqrt((r * r).sum(1)).clamp_min(1e-300)


def patch_moments(make_scheme, Q, centers, steps, r):
    """The oracle's moments after `steps` steps at each of `centers` (grid-order index
    tuples), each computed on a periodic patch of side 2 r + 1 cut from the full fields Q
    [K, *grid] around the node.  With r > steps the centre's domain of dependence lies inside
    the patch, so its value is the full domain's.  make_scheme(shape, origin) builds the
    oracle scheme of a patch whose first node has grid index `origin`."""
    out = []
    for c in centers:
        sub = Q
        for d, cd in enumerate(c):
            n = Q.shape[1 + d]
            idx = torch.tensor([(cd - r + j) % n for j in range(2 * r + 1)])
            sub = sub.index_select(1 + d, idx)
        sch = make_scheme(tuple(sub.shape[1:]), tuple(cd - r for cd in c))
        Qp = sch.moments(sch.run(sch.init(sub), steps))
        out.append(Qp[(slice(None),) + (r,) * len(c)])
    return torch.stack(out, dim=1)                 # [K, n_centres]


def _primitives(kind, Q, gamma, R=1.0):
    """Tracker parents from conserved fields [K, n]: name -> [components, n]."""
    rho = Q[0]
    if kind == "nsf":
        p = (gamma - 1.0) * (Q[3] - 0.5 * (Q[1] ** 2 + Q[2] ** 2) / rho)
        return {"u": (Q[1] / rho)[None], "v": (Q[2] / rho)[None], "T": (p / (rho * R))[None]}
    if kind == "mhd":
        return {"B": Q[4:7]}
    if kind == "hcnsf":
        m2 = Q[1] ** 2 + Q[2] ** 2 + Q[3] ** 2
        p = (gamma - 1.0) * (Q[4] - 0.5 * m2 / rho)
        return {"u": Q[1:4] / rho, "T": (p / rho)[None]}
    raise ValueError(kind)


# tracker component -> parent field, per family (component orders of include/lbx.h)
TRACKER_PARENT = {
    "nsf": {4: "u", 5: "u", 6: "v", 7: "v", 8: "T", 9: "T"},
    "mhd": {8: "B", 9: "B", 10: "B"},
    "hcnsf": {5: "u", 6: "u", 7: "T", 8: "T", 9: "T", 10: "u", 11: "u", 12: "u", 13: "u"},
}


def parity_scales(kind, Q, Q0, n_cons, dx, g_tau, cs2, gamma, shifted, R=1.0):
    """Per-component scale a parity error is measured against: the largest magnitude the
    component's stored populations carry, which sets the rounding unit of its moment.
    A conserved field's populations are of the size of the field (or, shifted, of its
    fluctuation about Q0).  A tracker of V has equilibrium populations
    w_i (G + c_i . (dt/dx) Phi_G / c_s^2) with Phi_G containing -I V / tau_grad, so their size
    is (dt/dx) |V| / (c_s^2 tau_grad) = |V| / (c_s^2 g_tau dx) (shifted: |V - V0|), far larger
    than G itself at fine grids; its moment's rounding error scales with that, not with G."""
    K = Q.shape[0]
    Qf = Q.reshape(K, -1)
    q0 = torch.as_tensor(Q0, dtype=F64).reshape(K, 1)
    scale = ((Qf - q0) if shifted else Qf).abs().amax(1)
    if K > n_cons:
        prim = _primitives(kind, Qf, gamma, R)
        prim0 = _primitives(kind, q0, gamma, R)
        amp = 1.0 / (cs2 * g_tau * dx)
        for k, par in TRACKER_PARENT[kind].items():
            v = prim[par] - prim0[par] if shifted else prim[par]
            scale[k] = torch.maximum(scale[k], amp * v.abs().max())
    return scale
