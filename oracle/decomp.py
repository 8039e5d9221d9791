"""Slab domain decomposition of the oracle step (host-emulated ranks).

The grid is cut along its slowest axis (y in 2D, z in 3D).  Each rank collides its own
nodes, then streams: populations with c_slab = +1 leaving the top layer go to the next
rank, those with c_slab = -1 leaving the bottom layer to the previous rank (periodic).
This is the one exchange per step that a multi-device run of Eq. lbe_update needs.
"""
from __future__ import annotations

import torch


def _slab_dim(D):
    return -D  # tensor dim of the slowest spatial axis in [K, q, *grid]


def outgoing(scheme, post):
    """(up, down): top-layer populations with c_slab = +1, bottom layer with c_slab = -1."""
    D = scheme.lat.D
    up_i = [i for i, c in enumerate(scheme.c) if c[D - 1] == 1]
    dn_i = [i for i, c in enumerate(scheme.c) if c[D - 1] == -1]
    dim = _slab_dim(D)
    up = post[:, up_i].select(dim, -1).clone()
    dn = post[:, dn_i].select(dim, 0).clone()
    return up, dn


def stream_with_halo(scheme, post, from_below, from_above):
    """Stream locally, then overwrite the layers that wrapped around the slab with the
    populations received from the neighbouring ranks (shifted in-plane by c_i)."""
    D = scheme.lat.D
    dim = _slab_dim(D)
    f = scheme.stream(post)
    up_i = [i for i, c in enumerate(scheme.c) if c[D - 1] == 1]
    dn_i = [i for i, c in enumerate(scheme.c) if c[D - 1] == -1]
    for src, idx, layer in ((from_below, up_i, 0), (from_above, dn_i, -1)):
        for j, i in enumerate(idx):
            ci = scheme.c[i]
            v = src[:, j]
            shifts = tuple(ci[d] for d in range(D - 1) if ci[d] != 0)
            dims = tuple(-(d + 1) for d in range(D - 1) if ci[d] != 0)
            if shifts:
                v = torch.roll(v, shifts=shifts, dims=dims)
            f[:, i].select(dim, layer).copy_(v)
    return f


def run_emulated(schemes, f_slabs, n_steps, t0=0.0):
    """Advance R slabs in lock step; the exchange is a direct copy between neighbours."""
    R = len(f_slabs)
    dt = schemes[0].dt
    for n in range(n_steps):
        t = t0 + n * dt
        posts = [s.collide(f, t) for s, f in zip(schemes, f_slabs)]
        outs = [outgoing(s, p) for s, p in zip(schemes, posts)]
        f_slabs = [stream_with_halo(schemes[r], posts[r], outs[(r - 1) % R][0], outs[(r + 1) % R][1])
                   for r in range(R)]
    return f_slabs
