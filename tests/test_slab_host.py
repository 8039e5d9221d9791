"""Host side of the slab decomposition (no GPU): scheme arguments, face-buffer sizes, the
slab split, and the product's ring exchange schedule (paper_2607_05668_b300.slab.
RingExchange) run as two and three gloo ranks on the CPU.

The exchange test drives RingExchange with a plain model of the library's pull layout:
a slab's array f[k, i, y, x] holds the populations that left node (y, x) along c_i, a
step pulls f[k, i, y - c_iy, x - c_ix] with the slab's own periodic wrap and applies a
node-local mixing map, and the face slots the library's k_face kernel copies (plane P - 1
for c_y = +1, plane 0 for c_y = -1) are packed, exchanged and unpacked after every step.
The slabs' pulled populations must equal the whole grid's bitwise.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import synthetic as syn

lbx = pytest.importorskip("paper_2607_05668_b300.lbx")
from paper_2607_05668_b300 import slab as SL, workloads as W  # noqa: E402

D2Q9 = np.array([[0, 0], [1, 0], [-1, 0], [0, 1], [0, -1], [1, 1], [-1, -1], [1, -1], [-1, 1]])


def test_slab_bounds_cover_the_grid_once():
    for planes in (7, 16, 1024):
        for n in (1, 2, 3, 8):
            if n > planes:
                continue
            spans = [SL.slab_bounds(planes, n, s) for s in range(n)]
            assert spans[0][0] == 0 and sum(c for _, c in spans) == planes
            assert all(spans[s][0] + spans[s][1] == spans[s + 1][0] for s in range(n - 1))
            assert max(c for _, c in spans) - min(c for _, c in spans) <= 1


def test_face_buffer_bytes_count_the_crossing_velocities():
    case = syn.NsfCase(n=32)
    sch = W.nsf_scheme(case, lbx.FP32_SHIFT, extent=(32, 8), slab_origin=8, slab_planes_global=32)
    assert sch.halo_bytes == 3 * 10 * 32 * 4                       # D2Q9: 3 of 9 cross a face
    m = syn.MhdCase(n=8)
    sm = W.mhd_scheme(m, lbx.FP16_SCALED, extent=(8, 8, 4), slab_origin=4, slab_planes_global=8)
    assert sm.halo_bytes == 5 * 11 * 64 * 2                        # D3Q19: 5 of 19, 8 x 8 plane
    sd = W.nsf_scheme(case, lbx.FP64, lattice=lbx.D2Q5)
    assert sd.halo_bytes == 1 * 10 * 32 * 8                        # D2Q5: 1 of 5; whole grid too


def test_slab_scheme_arguments_are_checked():
    case = syn.NsfCase(n=16)
    with pytest.raises(lbx.LbxError, match="fit"):
        W.nsf_scheme(case, extent=(16, 8), slab_origin=12, slab_planes_global=16)
    with pytest.raises(lbx.LbxError, match="slab_origin"):
        W.nsf_scheme(case, extent=(16, 8), slab_origin=4)
    with pytest.raises(lbx.LbxError, match="two-buffer"):
        W.nsf_scheme(case, extent=(16, 8), slab_origin=0, slab_planes_global=16, streaming=lbx.STREAM_IN_PLACE)
    with pytest.raises(lbx.LbxError, match="FP16_SCALED"):
        W.nsf_scheme(case, lbx.FP32_SHIFT, fp16_scales=[1.0] * 10)
    with pytest.raises(lbx.LbxError, match="all 10"):
        W.nsf_scheme(case, lbx.FP16_SCALED, fp16_scales=[1.0] * 4)
    W.nsf_scheme(case, lbx.FP16_SCALED, fp16_scales=[0.5] * 10)


def test_shared_fp16_scales_take_the_largest():
    s = SL.shared_fp16_scales([[0.5, 2.0, 1.0], [1.0, 0.25, 1.0]])
    assert list(s) == [1.0, 2.0, 1.0]


# ------------------------------------------------------------ the exchange schedule
def _pull(f):
    """Pre-collision populations of every node: f[k, i, y - c_iy, x - c_ix] (periodic)."""
    out = np.empty_like(f)
    for i, (cx, cy) in enumerate(D2Q9):
        out[:, i] = np.roll(np.roll(f[:, i], cy, axis=1), cx, axis=2)
    return out


def _collide(pre):
    """A node-local map that mixes velocities and components (stands in for the BGK update)."""
    m = pre.mean(axis=1, keepdims=True)
    return pre + 0.3 * (m - pre) + 0.05 * np.roll(pre, 1, axis=0) * m


UP = [i for i, c in enumerate(D2Q9) if c[1] == 1]
DN = [i for i, c in enumerate(D2Q9) if c[1] == -1]


def _pack(f):
    return torch.from_numpy(f[:, UP, -1, :].copy()), torch.from_numpy(f[:, DN, 0, :].copy())


def _unpack(f, from_lower, from_upper):
    f[:, UP, -1, :] = from_lower.numpy()
    f[:, DN, 0, :] = from_upper.numpy()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


STEPS, NX, NY, K = 6, 10, 13, 2


def _whole():
    f = np.random.default_rng(4).standard_normal((K, 9, NY, NX))
    out = [f]
    for _ in range(STEPS):
        f = _collide(_pull(f))
        out.append(f)
    return out


def _rank_main(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ring = SL.RingExchange()
        o, c = SL.slab_bounds(NY, world, rank)
        f = _whole()[0][:, :, o:o + c, :].copy()

        def exchange(f):
            tu, tl = _pack(f)
            fl, fu = torch.empty_like(tu), torch.empty_like(tl)
            ring.exchange(tu, tl, fl, fu)
            _unpack(f, fl, fu)
        exchange(f)                     # the cut of a post-step array: faces from the neighbours
        for _ in range(STEPS):
            f = _collide(_pull(f))
            exchange(f)
        np.save(os.path.join(out_dir, f"slab{rank}.npy"), _pull(f))
        tot = ring.sum(f.sum(axis=(1, 2, 3)))
        np.save(os.path.join(out_dir, f"sum{rank}.npy"), tot)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_ring_exchange_reproduces_the_whole_grid(tmp_path, world):
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, str(tmp_path))) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = np.concatenate([np.load(tmp_path / f"slab{r}.npy") for r in range(world)], axis=2)
    want = _pull(_whole()[-1])
    assert np.array_equal(got, want)
    sums = [np.load(tmp_path / f"sum{r}.npy") for r in range(world)]
    assert all(np.array_equal(s, sums[0]) for s in sums)
    np.testing.assert_allclose(sums[0], _whole()[-1].sum(axis=(1, 2, 3)), rtol=1e-12)


# --------------------------------------------- the adjoint's reversed exchange schedule
# The reverse step of the library's adjoint pushes: node x writes Lam_n[k][i][x - c_i].  The
# model below stands in for it (a node-local map of the incoming adjoint, then the push with
# the slab's own periodic wrap); the product's slab._adj_exchange packs, exchanges and
# unpacks the adjoint face slots (the slots k_adj_face copies) between the steps.  The slabs'
# adjoint arrays must equal the whole grid's bitwise after every reverse step, and after
# the forward exchange a pull (the initial VJP's access pattern) must match too.
class _FakeAdjState:
    """The adjoint face copies of lbx_adjoint_halo_pack / _unpack on host arrays."""

    def adjoint_halo_pack(self, lam, face_upper, face_lower):
        face_upper.copy_(torch.from_numpy(lam[:, UP, -1, :].copy()))
        face_lower.copy_(torch.from_numpy(lam[:, DN, 0, :].copy()))

    def adjoint_halo_unpack(self, lam, face_upper, face_lower):
        lam[:, UP, -1, :] = face_upper.numpy()
        lam[:, DN, 0, :] = face_lower.numpy()


class _FakeSlab:
    def __init__(self):
        self.state = _FakeAdjState()


def _push(lam):
    """Lam_n[k, i, x - c_i] = g(Lam_{n+1})[k, i, x] (periodic), g node-local."""
    g = 0.7 * lam + 0.1 * lam.mean(axis=1, keepdims=True) + 0.02 * np.roll(lam, 1, axis=0)
    out = np.empty_like(g)
    for i, (cx, cy) in enumerate(D2Q9):
        out[:, i] = np.roll(np.roll(g[:, i], -cy, axis=1), -cx, axis=2)
    return out


def _adj_whole():
    lam = np.random.default_rng(7).standard_normal((K, 9, NY, NX))
    out = [lam]
    for _ in range(STEPS):
        lam = _push(lam)
        out.append(lam)
    return out


def _adj_rank_main(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ring = SL.RingExchange()
        o, c = SL.slab_bounds(NY, world, rank)
        whole = _adj_whole()
        lam = whole[0][:, :, o:o + c, :].copy()
        shape = (K, len(UP), NX)
        faces = [[torch.empty(shape, dtype=torch.float64) for _ in range(4)]]
        slabs = [_FakeSlab()]
        for n in range(STEPS):
            lam = _push(lam)
            SL._adj_exchange(slabs, [lam], faces, ring, reverse=True)
            if not np.array_equal(lam, whole[n + 1][:, :, o:o + c, :]):
                raise AssertionError(f"rank {rank}: reverse step {n} differs")
        SL._adj_exchange(slabs, [lam], faces, ring, reverse=False)
        np.save(os.path.join(out_dir, f"adj{rank}.npy"), _pull(lam))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [1, 2, 3])
def test_adjoint_ring_exchange_reproduces_the_whole_grid(tmp_path, world):
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_adj_rank_main, args=(r, world, port, str(tmp_path))) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = np.concatenate([np.load(tmp_path / f"adj{r}.npy") for r in range(world)], axis=2)
    assert np.array_equal(got, _pull(_adj_whole()[-1]))


def test_adjoint_face_buffer_bytes():
    case = syn.NsfCase(n=32)
    sch = W.nsf_scheme(case, lbx.FP32_SHIFT, extent=(32, 8), slab_origin=8, slab_planes_global=32)
    assert sch.adjoint_halo_bytes == 3 * 10 * 32 * 4               # compute type float
    assert sch.adjoint_lam_bytes == 10 * 9 * 32 * 8 * 4
    sd = W.nsf_scheme(case, lbx.FP64, extent=(32, 8), slab_origin=8, slab_planes_global=32)
    assert sd.adjoint_halo_bytes == 3 * 10 * 32 * 8
    s16 = W.nsf_scheme(case, lbx.FP16_SCALED)
    assert s16.adjoint_lam_bytes == 0 and s16.adjoint_halo_bytes == 0   # no FP16 adjoint


@pytest.mark.parametrize("nslabs", [1, 2, 3])
def test_adjoint_local_exchange_reproduces_the_whole_grid(nslabs):
    """Several slabs in one process (the device-copy branch of slab._adj_exchange).  With
    three slabs the forward direction after a reverse step would not reproduce the whole
    grid (with one or two, the upper and the lower neighbour are the same slab)."""
    whole = _adj_whole()
    spans = [SL.slab_bounds(NY, nslabs, s) for s in range(nslabs)]
    for reverse in (True, False):
        lams = [whole[0][:, :, o:o + c, :].copy() for o, c in spans]
        faces = [[torch.empty((K, len(UP), NX), dtype=torch.float64) for _ in range(4)] for _ in spans]
        slabs = [_FakeSlab() for _ in spans]
        for n in range(STEPS):
            lams = [_push(lam) for lam in lams]
            SL._adj_exchange(slabs, lams, faces, None, reverse=reverse)
        ok = all(np.array_equal(lam, whole[-1][:, :, o:o + c, :]) for lam, (o, c) in zip(lams, spans))
        assert ok == (reverse or nslabs <= 2)


def test_slab_adjoint_checks_its_arguments_before_any_device_work():
    class _Ring:
        pass
    with pytest.raises(ValueError, match="one slab per process"):
        SL.slab_adjoint([object(), object()], [], [], 4, 2, ring=_Ring())
