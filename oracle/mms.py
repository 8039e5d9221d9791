"""Manufactured-solution forcing S_MMS = d_t Q_ex + div Phi(Q_ex) - S(Q_ex) (Sec. 4).

The derivatives are taken by forward-mode automatic differentiation of the exact
fields (torch.func.jvp), so no derivative is written by hand.  Tracker components of
the exact augmented state are the exact gradients of their parent fields (supplement,
MMS section: trackers are initialised from the spatial derivatives of the fields).

By default the forcing is the residual of the whole augmented state Q+ (conserved and
tracker components), as the paper's compiler forms it on Q+ (Sec. 4: the residual of the
analytical profiles, injected into the update); for a tracker the 1/tau_grad terms of
flux and source cancel and its forcing is d_t grad V + div(grad V (x) u).
For a system with prescribed coefficient fields c(x, t) the divergence differentiates
Phi(Q_ex(x, t); c(x, t)) along x, the coefficients included.  With
`conserved_only` the trackers are left unforced (they then lag grad V by O(tau_grad)).
"""
from __future__ import annotations

import torch
from torch.func import jvp

from .systems import flux_at, source_at


def _replace(xx, b, xb):
    out = list(xx)
    out[b] = xb
    return tuple(out)


def exact_augmented(system, exact, xx, t):
    """Q+_ex = (Q_ex, trackers = grad of the parents) at coordinates xx and time t.

    `exact(*xx, t)` returns the conserved exact fields [n_cons, *grid]."""
    Qc = exact(*xx, t)
    if system.K == system.n_cons:
        return Qc
    D = len(xx)
    dP_b = []
    for b in range(D):
        def along_b(xb, b=b):
            return torch.stack(system.parents(exact(*_replace(xx, b, xb), t)))
        _, d = jvp(along_b, (xx[b],), (torch.ones_like(xx[b]),))
        dP_b.append(d)
    n_par = dP_b[0].shape[0]
    dP = [[dP_b[b][p] for b in range(D)] for p in range(n_par)]
    return torch.cat([Qc, torch.stack(system.trackers_from_grads(dP))])


def mms_source(system, exact, xx, t, conserved_only=False):
    """S_MMS(x, t), [K, *grid] ([n_cons, *grid] with conserved_only)."""
    tt = torch.full_like(xx[0], float(t))
    return mms_source_t(system, exact, xx, tt, conserved_only)


def make_mms(system, exact, xx, dt=None, chunk=64, conserved_only=False):
    """Callable t -> S_MMS(x, t) on the fixed node coordinates xx.

    With a time step `dt`, the forcing is evaluated for `chunk` consecutive instants
    t, t + dt, ... at once (the same definition, batched along a leading time axis to
    amortise the differentiation overhead) and served from that cache."""
    if dt is None:
        return lambda t: mms_source(system, exact, xx, t, conserved_only)
    cache = {"t0": None, "vals": None}

    def fn(t):
        t0 = cache["t0"]
        if t0 is not None:
            j = round((t - t0) / dt)
            if 0 <= j < cache["vals"].shape[0] and abs(t - (t0 + j * dt)) <= 1e-9 * dt:
                return cache["vals"][j]
        ts = torch.tensor([t + j * dt for j in range(chunk)], dtype=torch.float64)
        shp = (chunk,) + tuple(xx[0].shape)
        tb = ts.reshape((chunk,) + (1,) * xx[0].dim()).expand(shp).contiguous()
        xb = tuple(x.unsqueeze(0).expand(shp).contiguous() for x in xx)
        vals = mms_source_t(system, exact, xb, tb, conserved_only)   # [K or n_cons, chunk, *grid]
        cache["t0"], cache["vals"] = t, vals.transpose(0, 1).contiguous()
        return cache["vals"][0]
    return fn


def mms_source_t(system, exact, xx, tt, conserved_only=False):
    """S_MMS with a time tensor tt of the same shape as the coordinates."""
    nk = system.n_cons if conserved_only else system.K
    _, dQdt = jvp(lambda T: exact_augmented(system, exact, xx, T)[:nk], (tt,), (torch.ones_like(tt),))
    div = torch.zeros_like(dQdt)
    for b in range(len(xx)):
        def flux_b(xb, b=b):
            xb_all = _replace(xx, b, xb)
            return flux_at(system, exact_augmented(system, exact, xb_all, tt), xb_all, tt)[:nk, b]
        _, d = jvp(flux_b, (xx[b],), (torch.ones_like(xx[b]),))
        div = div + d
    Qp = exact_augmented(system, exact, xx, tt)
    return dQdt + div - source_at(system, Qp, xx, tt)[:nk]
