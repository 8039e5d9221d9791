"""One periodic grid cut into slabs along its last axis (y in 2D, z in 3D): the domain
decomposition of the collide-and-stream step across processes or GPUs.

Each slab is an lbx state whose scheme carries `slab_origin` / `slab_planes_global`; it
steps with the periodic wrap of its own planes, and after every step the populations that
left through its two faces are exchanged with the neighbouring slabs (lbx_halo_pack, a
transport, lbx_halo_unpack), which makes the streaming of Eq. lbe_update cross the faces.
This module holds the exchange schedule and the bookkeeping only: the population copies
into and out of the face buffers run in liblbx.so's kernels, and the transport is
torch.distributed point-to-point messages (NCCL between GPUs, gloo for host tensors) or,
for several slabs in one process, device-to-device copies.  Reductions are per slab and
are combined here in float64 (sums add, maxima take the maximum).
"""
from __future__ import annotations

import numpy as np
import torch

from . import lbx as L


def slab_bounds(planes, nslabs, s):
    """(origin, count) of slab s when `planes` planes are cut into `nslabs` slabs whose
    sizes differ by at most one (the first planes % nslabs slabs take one more)."""
    base, extra = divmod(planes, nslabs)
    origin = s * base + min(s, extra)
    return origin, base + (1 if s < extra else 0)


def slab_of(Q, origin, count):
    """The slab's fields: Q [K, (nz,) ny, nx] cut along its first grid axis (the slab axis)."""
    return Q.narrow(1, origin, count).contiguous()


class RingExchange:
    """The face exchange of `world` slabs in a periodic ring over torch.distributed: slab r's
    upper neighbour is r + 1 and its lower neighbour r - 1 (mod world).  Every rank posts
    the same four messages in the same order (send up, receive from below, send down,
    receive from above), so the sends and receives between two ranks pair up in order even
    when both neighbours are the same rank (world = 2).  A ring of one slab is the periodic
    grid itself: its own outgoing faces are its incoming ones."""

    def __init__(self, rank=None, world=None, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group) if rank is None else rank
        self.world = dist.get_world_size(group) if world is None else world
        self.up = (self.rank + 1) % self.world
        self.down = (self.rank - 1) % self.world

    def _peer(self, r):
        return r if self.group is None else self.dist.get_global_rank(self.group, r)

    def exchange(self, to_upper, to_lower, from_lower, from_upper):
        if self.world == 1:
            from_lower.copy_(to_upper)
            from_upper.copy_(to_lower)
            return
        d = self.dist
        ops = [d.P2POp(d.isend, to_upper, self._peer(self.up), self.group),
               d.P2POp(d.irecv, from_lower, self._peer(self.down), self.group),
               d.P2POp(d.isend, to_lower, self._peer(self.down), self.group),
               d.P2POp(d.irecv, from_upper, self._peer(self.up), self.group)]
        for req in d.batch_isend_irecv(ops):
            req.wait()

    def sum(self, values):
        """float64 sum over the ring of a per-slab array (host), e.g. conserved sums."""
        t = torch.as_tensor(np.asarray(values, dtype=np.float64))
        if self.world > 1:
            dev = "cuda" if self.dist.get_backend(self.group) == "nccl" else "cpu"
            t = t.to(dev)
            self.dist.all_reduce(t, op=self.dist.ReduceOp.SUM, group=self.group)
        return t.cpu().numpy()

    def max(self, values):
        t = torch.as_tensor(np.asarray(values, dtype=np.float64))
        if self.world > 1:
            dev = "cuda" if self.dist.get_backend(self.group) == "nccl" else "cpu"
            t = t.to(dev)
            self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX, group=self.group)
        return t.cpu().numpy()


class Slab:
    """One slab: an lbx.State and its four face buffers (device, 16-byte aligned)."""

    def __init__(self, scheme: L.Scheme, Q, stream=None, buffers=None, faces=None):
        """buffers: caller-owned population buffers (lbx_init f_buf_a, f_buf_b); faces:
        four caller-owned face buffers (to_upper, to_lower, from_lower, from_upper) of at
        least scheme.halo_bytes bytes; None: allocated here."""
        self.scheme = scheme
        self.state = L.State(scheme, Q, stream=stream, buffers=buffers)
        nb = scheme.halo_bytes
        if faces is None:
            faces = [torch.empty(nb, dtype=torch.uint8, device="cuda") for _ in range(4)]
        self.to_upper, self.to_lower, self.from_lower, self.from_upper = faces

    def pack(self):
        self.state.halo_pack(self.to_upper, self.to_lower)

    def unpack(self):
        self.state.halo_unpack(self.from_lower, self.from_upper)

    def close(self):
        self.state.close()


def step_ring(slab: Slab, ring: RingExchange, n=1):
    """n steps of one slab of a multi-process run: each step, then its face exchange.  The
    slab's state must run on torch's current stream (the stream the messages order with)."""
    for _ in range(int(n)):
        slab.state.step(1)
        slab.pack()
        ring.exchange(slab.to_upper, slab.to_lower, slab.from_lower, slab.from_upper)
        slab.unpack()


def step_local(slabs, n=1):
    """n steps of several slabs of one grid held by this process (one stream, listed from
    the lowest plane up): every slab steps, packs its faces, receives its neighbours' faces
    by device copies, and unpacks them."""
    m = len(slabs)
    for _ in range(int(n)):
        for s in slabs:
            s.state.step(1)
            s.pack()
        for i, s in enumerate(slabs):
            s.from_lower.copy_(slabs[(i - 1) % m].to_upper)
            s.from_upper.copy_(slabs[(i + 1) % m].to_lower)
        for s in slabs:
            s.unpack()


def _split_step(slabs, side, exchange):
    """One step of slabs with the exchange behind the interior: the boundary planes 0 and
    P - 1 of every slab step on `side`, whose faces are packed, exchanged (exchange(), on
    side) and unpacked into the buffer being written while the interior planes 1 .. P - 2
    step on torch's current stream (the states' stream); then that stream waits for side
    and every state commits its step (lbx_step_planes, lbx_halo_pack_next / _unpack_next,
    lbx_step_commit)."""
    main = torch.cuda.current_stream()
    side.wait_stream(main)
    for s in slabs:
        P = s.scheme.grid[0]
        s.state.step_planes(0, 1, side)
        if P > 1:
            s.state.step_planes(P - 1, 1, side)
        s.state.step_planes(1, max(P - 2, 0))
    exchange()
    main.wait_stream(side)
    for s in slabs:
        s.state.step_commit()


def side_stream():
    """The second stream of the overlapped exchange, at high priority: the block scheduler
    then dispatches its small kernels (boundary planes, pack, unpack) as soon as SMs free
    up instead of after every block of the interior launch."""
    lo, hi = torch.cuda.Stream.priority_range()
    return torch.cuda.Stream(priority=hi)


def step_ring_overlap(slab: Slab, ring: RingExchange, n=1, side=None):
    """step_ring with the face exchange hidden behind the interior planes of every step
    (bitwise the result of step_ring).  The slab's state must run on torch's current
    stream; `side` is a second stream (side_stream() if None)."""
    side = side or side_stream()

    def exchange():
        slab.state.halo_pack_next(slab.to_upper, slab.to_lower, side)
        with torch.cuda.stream(side):
            ring.exchange(slab.to_upper, slab.to_lower, slab.from_lower, slab.from_upper)
        slab.state.halo_unpack_next(slab.from_lower, slab.from_upper, side)
    for _ in range(int(n)):
        _split_step([slab], side, exchange)


def step_local_overlap(slabs, n=1, side=None):
    """step_local with the face exchange hidden behind the interior planes (bitwise the
    result of step_local)."""
    side = side or side_stream()
    m = len(slabs)

    def exchange():
        for s in slabs:
            s.state.halo_pack_next(s.to_upper, s.to_lower, side)
        with torch.cuda.stream(side):
            for i, s in enumerate(slabs):
                s.from_lower.copy_(slabs[(i - 1) % m].to_upper)
                s.from_upper.copy_(slabs[(i + 1) % m].to_lower)
        for s in slabs:
            s.state.halo_unpack_next(s.from_lower, s.from_upper, side)
    for _ in range(int(n)):
        _split_step(slabs, side, exchange)


def combine_error_stats(stats):
    """relative L2 and L-infinity per component (Sec. 4, as lbx_error_norms) from the
    [K, 4] statistics of every slab (lbx_error_stats) combined over the grid."""
    st = np.asarray(stats, dtype=np.float64)
    l2 = np.sqrt(st[:, 0] / np.where(st[:, 1] > 0, st[:, 1], 1.0))
    li = st[:, 2] / np.where(st[:, 3] > 0, st[:, 3], 1.0)
    return l2, li


def ring_error_norms(slab: Slab, Q_ref_local, ring: RingExchange):
    """Relative norms of the whole grid from one slab of a multi-process run."""
    st = slab.state.error_stats(Q_ref_local)
    s = ring.sum(st[:, :2])
    m = ring.max(st[:, 2:])
    return combine_error_stats(np.concatenate([s, m], axis=1))


def shared_fp16_scales(scales_per_slab):
    """The FP16 storage scales slabs of one grid share: the largest of each component's
    derived scales (s_k = 2^ceil(log2(4 max|f*_k|)) grows with the maximum, so the largest
    slab scale is the scale of the whole grid)."""
    return np.max(np.asarray(scales_per_slab, dtype=np.float64), axis=0)


# --------------------------------------------------------------------- adjoint sweep
def _adj_faces(scheme):
    nb = max(scheme.adjoint_halo_bytes, 16)
    return [torch.empty(nb, dtype=torch.uint8, device="cuda") for _ in range(4)]


def _adj_exchange(slabs, lams, faces, ring, reverse):
    """Face exchange of the adjoint buffers lams[s] (lbx_adjoint_halo_pack, a transport,
    lbx_adjoint_halo_unpack).  reverse (after a seed or a reverse step): each slab takes its
    upper neighbour's upper face and its lower neighbour's lower face; forward (before the
    initial VJP, which pulls): its lower neighbour's upper face and its upper neighbour's
    lower face.  faces[s] = [packed upper, packed lower, received upper, received lower]."""
    for s, lam, f in zip(slabs, lams, faces):
        s.state.adjoint_halo_pack(lam, f[0], f[1])
    if ring is not None:
        pu, pl, ru, rl = faces[0]
        if reverse:     # upper face down, lower face up
            ring.exchange(pl, pu, rl, ru)
        else:           # as the populations: upper face up, lower face down
            ring.exchange(pu, pl, ru, rl)
    else:
        m = len(slabs)
        for i, f in enumerate(faces):
            up, dn = faces[(i + 1) % m], faces[(i - 1) % m]
            f[2].copy_(up[0] if reverse else dn[0])
            f[3].copy_(dn[1] if reverse else up[1])
    for s, lam, f in zip(slabs, lams, faces):
        s.state.adjoint_halo_unpack(lam, f[2], f[3])


def slab_adjoint(slabs, Q_init, rho_target, n_steps, ckpt_every, ring=None):
    """Gradient of J = 1/2 sum_x (rho(x, T) - rho*(x))^2 over a grid cut into slabs, by the
    step-wise adjoint of liblbx.so (the reverse of Eq. lbe_update, face exchanges reversed).

    slabs: this process's slabs of the grid, freshly initialised from Q_init and listed from
    the lowest plane up (with `ring`, exactly one slab per process).  Q_init[s], rho_target[s]:
    float64 CUDA tensors [K, cells] and [cells] of slab s.  Every step of the forward sweep,
    of the recomputation and of the reverse sweep is followed by its face exchange; the
    forward state is checkpointed every ckpt_every steps and each segment is recomputed
    before its reverse steps, as lbx_adjoint does for a whole grid.
    Returns (J, [dJ/dQ_init per slab, float64 CUDA [K, cells]], dJ/dtau), J and dJ/dtau
    summed over the grid."""
    slabs = list(slabs)
    if ring is not None and len(slabs) != 1:
        raise ValueError("slab_adjoint: one slab per process with a ring")
    sch = slabs[0].scheme
    n_steps, ckpt_every = int(n_steps), int(ckpt_every)
    if n_steps < 0 or ckpt_every < 1:
        raise ValueError("slab_adjoint: n_steps >= 0 and ckpt_every >= 1")
    if sch.adjoint_lam_bytes == 0:
        raise L.LbxError(-1, "slab_adjoint: no adjoint for this family and storage")
    k = min(ckpt_every, max(n_steps, 1))
    nck = 0 if n_steps == 0 else -(-n_steps // k)

    def fwd_step():
        if ring is not None:
            step_ring(slabs[0], ring, 1)
        else:
            step_local(slabs, 1)

    def buf(nbytes):
        return torch.empty(nbytes, dtype=torch.uint8, device="cuda")

    ckpt = [[buf(s.scheme.buffer_bytes) for _ in range(nck)] for s in slabs]
    seg = [[buf(s.scheme.buffer_bytes) for _ in range(k)] for s in slabs]
    lam = [[buf(s.scheme.adjoint_lam_bytes) for _ in range(2)] for s in slabs]
    ncell = [int(np.prod(s.scheme.grid)) for s in slabs]
    tau = [torch.zeros(n, dtype=torch.float64, device="cuda") for n in ncell]
    faces = [_adj_faces(s.scheme) for s in slabs]

    # forward sweep, keeping the state at the start of every segment
    for c in range(nck):
        for s, ck in zip(slabs, ckpt):
            s.state.adjoint_checkpoint(ck[c])
        for _ in range(min(k, n_steps - c * k)):
            fwd_step()
    # misfit and seed Lam_N
    J = np.array([sum(s.state.adjoint_seed(r, lm[0]) for s, r, lm in zip(slabs, rho_target, lam))])
    cur = 0
    _adj_exchange(slabs, [lm[cur] for lm in lam], faces, ring, reverse=True)
    # reverse sweep: recompute each segment from its checkpoint, then step the adjoint back
    for c in range(nck - 1, -1, -1):
        ln = min(k, n_steps - c * k)
        for s, ck in zip(slabs, ckpt):
            s.state.adjoint_restore(ck[c], c * k)
        for j in range(ln):
            for s, sg in zip(slabs, seg):
                s.state.adjoint_checkpoint(sg[j])
            if j + 1 < ln:
                fwd_step()
        for j in range(ln - 1, -1, -1):
            for s, sg, lm, t in zip(slabs, seg, lam, tau):
                s.state.adjoint_step(sg[j], lm[cur], lm[1 - cur], t)
            cur = 1 - cur
            _adj_exchange(slabs, [lm[cur] for lm in lam], faces, ring, reverse=True)
    # the initial VJP pulls Lam_0 across the faces: forward exchange first
    _adj_exchange(slabs, [lm[cur] for lm in lam], faces, ring, reverse=False)
    grads, gt = [], np.zeros(1)
    for s, lm, q, t, n in zip(slabs, lam, Q_init, tau, ncell):
        g = torch.empty((s.scheme.system.K, n), dtype=torch.float64, device="cuda")
        gt[0] += s.state.adjoint_finish(lm[cur], q, g, t)
        grads.append(g)
    if ring is not None:
        J, gt = ring.sum(J), ring.sum(gt)
    return float(J[0]), grads, float(gt[0])
