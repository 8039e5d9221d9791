"""Slab decomposition across processes (gloo, world_size 2, CPU): each rank steps its own
y-slab of the NSF grid and exchanges the populations that cross the slab boundary with
point-to-point messages; the gathered result equals the single-domain run bitwise."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
import synthetic as syn
from tests import helpers as H

N, STEPS = 16, 5


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        case = syn.NsfCase(n=N)
        full = H.oracle_nsf(case)
        f = full.init(syn.nsf_fields(case))
        rows = N // world
        sch = H.oracle_nsf(case)
        sch.shape = (rows, N)
        fl = f[..., rank * rows:(rank + 1) * rows, :].contiguous()
        up, dn = (rank + 1) % world, (rank - 1) % world
        for n in range(STEPS):
            post = sch.collide(fl, n * sch.dt)
            send_up, send_dn = oracle.decomp.outgoing(sch, post)
            from_below, from_above = torch.empty_like(send_up), torch.empty_like(send_dn)
            # pairwise ordered exchange (even ranks send first) avoids a send/recv deadlock
            if rank % 2 == 0:
                dist.send(send_up, up); dist.recv(from_below, dn)
                dist.send(send_dn, dn); dist.recv(from_above, up)
            else:
                dist.recv(from_below, dn); dist.send(send_up, up)
                dist.recv(from_above, up); dist.send(send_dn, dn)
            fl = oracle.decomp.stream_with_halo(sch, post, from_below, from_above)
        torch.save(fl, os.path.join(out_dir, f"slab{rank}.pt"))
    finally:
        dist.destroy_process_group()


def test_two_rank_slab_decomposition_matches_single_domain(tmp_path):
    world = 2
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, str(tmp_path))) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    case = syn.NsfCase(n=N)
    full = H.oracle_nsf(case)
    ref = full.run(full.init(syn.nsf_fields(case)), STEPS)
    got = torch.cat([torch.load(tmp_path / f"slab{r}.pt") for r in range(world)], dim=-2)
    assert torch.equal(got, ref)


HC_SHAPE, HC_STEPS = (8, 6, 8), 3


def _hcnsf_scheme(shape, origin=None):
    from oracle import systems as S
    case = syn.HcnsfPaperCase(n=8)
    sysm = S.HomogenizedNsf3D(case.gamma, case.mu, case.kappa, case.eta, case.g_tau * case.dt, fields=case.prescribed)
    tau = oracle.tau_vector(sysm, case.dt, tau_R=case.tau_R, g_tau=case.g_tau)
    return case, oracle.Scheme(sysm, oracle.LATTICES["D3Q7"], shape, case.dx, case.dt, tau,
                               source_theta=case.theta, origin=origin)


def _rank_main_hcnsf(rank, world, port, out_dir):
    """The 3D homogenized NSF on z-slabs: each rank's node coordinates carry its offset, so
    the prescribed porosity and solid velocity are those of the whole domain."""
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        case, full = _hcnsf_scheme(HC_SHAPE)
        f = full.init(case.table().augmented(syn.coords(HC_SHAPE), 0.0))
        nz = HC_SHAPE[0] // world
        _, sch = _hcnsf_scheme((nz,) + HC_SHAPE[1:], origin=(rank * nz, 0, 0))
        fl = f[:, :, rank * nz:(rank + 1) * nz].contiguous()
        up, dn = (rank + 1) % world, (rank - 1) % world
        for n in range(HC_STEPS):
            post = sch.collide(fl, n * sch.dt)
            send_up, send_dn = oracle.decomp.outgoing(sch, post)
            from_below, from_above = torch.empty_like(send_up), torch.empty_like(send_dn)
            if rank % 2 == 0:
                dist.send(send_up, up); dist.recv(from_below, dn)
                dist.send(send_dn, dn); dist.recv(from_above, up)
            else:
                dist.recv(from_below, dn); dist.send(send_up, up)
                dist.recv(from_above, up); dist.send(send_dn, dn)
            fl = oracle.decomp.stream_with_halo(sch, post, from_below, from_above)
        torch.save(fl, os.path.join(out_dir, f"hc{rank}.pt"))
    finally:
        dist.destroy_process_group()


def test_two_rank_slabs_with_prescribed_fields_match_single_domain(tmp_path):
    world = 2
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_rank_main_hcnsf, args=(r, world, port, str(tmp_path))) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    case, full = _hcnsf_scheme(HC_SHAPE)
    ref = full.run(full.init(case.table().augmented(syn.coords(HC_SHAPE), 0.0)), HC_STEPS)
    got = torch.cat([torch.load(tmp_path / f"hc{r}.pt") for r in range(world)], dim=-3)
    assert torch.equal(got, ref)
