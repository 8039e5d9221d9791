#!/usr/bin/env python3
"""Benchmark of the fused collide-and-stream step on one B300 (or N replicas).

Default workload: compressible NSF with primitive trackers (K = 10) on D2Q9, a 1024^2
periodic grid, reference/equilibrium-shifted FP32 populations, seeded Fourier fields
around rho = 1, T = 1, Mach 0.3.  A step is one collide-and-stream pass over the whole
grid (one kernel launch).  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload nsf|mhd|adr|nsf12|mhd18|hcnsf] [--precision fp32|fp64|fp16]

--impl reference times the CPU FP64 oracle on bounded samples of the same workload.
Under torchrun (N > 1) every rank holds one case-sized slab of a grid N times as long along
its last axis and exchanges the faces of every step with its neighbours (NCCL, behind the
interior planes; weak scaling; --decomp replicas: independent grids); rank 0 prints the
line; the reference arm runs on rank 0 only.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import torch  # noqa: E402

import synthetic as syn  # noqa: E402

PREC = {"fp64": 1, "fp32": 2, "fp16": 3}
PREC_NAME = {"fp64": "f64", "fp32": "f32", "fp16": "f32 (f16 storage)"}
STORE_BYTES = {"fp64": 8, "fp32": 4, "fp16": 2}


def kernel_source_sha():
    h = hashlib.sha256()
    for f in ("kernels.cuh", "systems.cuh", "lattices.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2607_05668_b300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs"), "measured"
    return 6400.0, "fallback"


def profile_entry(key):
    """Entry of the committed ncu summary (profiles/ncu_traffic.json), or None when it is
    missing or was taken on other kernel sources."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p)).get(key)
    if not d or d.get("source_sha") != kernel_source_sha():
        return None
    return d


def profile_traffic(workload_key, cells=None):
    """DRAM bytes per launch of the step kernel (scaled by node count when the capture ran
    on a smaller grid of the same kernel), or None."""
    d = profile_entry(workload_key)
    if not d:
        return None
    b = d.get("dram_bytes_per_launch")
    if b is not None and cells and d.get("cells") and d["cells"] != cells:
        b = b * cells / d["cells"]
    return b


def profile_kernel(workload_key):
    """Kernel and block of the committed capture (the launch shape the tuner kept there)."""
    d = profile_entry(workload_key)
    return {"kernel": d.get("kernel_fn"), "block": d.get("block"), "cells": d.get("cells")} if d else None


class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            time.sleep(0.3)
        except FileNotFoundError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.lines:
            return None
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class PaperD2Q5Case:
    """The paper's D2Q5 systems of its Sec. 5 roofline table, each with its Table 3 recipe and
    manufactured field at t = 0 as the initial state (an unforced run: the plain step kernel).
      burgers  K = 1, acoustic f = 0.2, tau_R = 0.2, u = 1.3 sin(2 pi x) sin(2 pi y)
      euler    K = 4, acoustic f = 0.05, tau_R = 0.2, the paper's Euler field (gamma = 1.4)
      maxwell  K = 3, acoustic f = 0.2, tau_R = 0.2, the paper's TM field (c = 1)
      adrp     K = 3 (u and its two gradient trackers), diffusive f = 1.9, tau_R = 50,
               g_tau = 6, the paper's ADR field (a = (0.1, -0.1), D = 0.01, reaction R = 1)."""
    RECIPES = {"burgers": ("acoustic", 0.2, 0.2, 0.0), "euler": ("acoustic", 0.05, 0.2, 0.0),
               "maxwell": ("acoustic", 0.2, 0.2, 0.0), "adrp": ("diffusive", 1.9, 50.0, 6.0)}

    def __init__(self, name, n):
        self.name, self.n = name, n
        self.scaling, self.f, self.tau_R, self.g_tau = self.RECIPES[name]
        self.dx = 1.0 / n
        self.dt = self.f * self.dx * (self.dx if self.scaling == "diffusive" else 1.0)

    def table(self):
        if self.name == "burgers":
            return syn.burgers_table()
        if self.name == "maxwell":
            return syn.maxwell_table()
        if self.name == "euler":
            return syn.euler_table()
        return syn.AdrPaperCase(n=self.n).table()

    def system_args(self):
        """(params, Q0) of the family."""
        if self.name == "burgers":
            return (), (0.0,)
        if self.name == "maxwell":
            return (1.0,), (0.0, 0.0, 0.0)
        if self.name == "euler":
            g = 1.4
            return (g,), (1.0, 3.0, 3.0, (1.0 / g) / (g - 1.0) + 9.0)
        a = syn.AdrPaperCase(n=self.n)
        return (a.a[0], a.a[1], a.D, a.R), (0.5, 0.0, 0.0)

    def reference_state(self):
        return list(self.system_args()[1])


PAPER_D2Q5 = ("burgers", "euler", "maxwell", "adrp")


def make_case(workload, n=None):
    if workload in PAPER_D2Q5:
        return PaperD2Q5Case(workload, n or 4096)
    if workload == "nsf":
        return syn.NsfCase(n=n or 1024)
    if workload == "mhd":
        return syn.MhdCase(n=n or 256)
    if workload == "adr":
        return syn.AdrCase(n=n or 64)
    if workload == "nsf12":
        return syn.NsfPaperCase(n=n or 1024)
    if workload == "mhd18":
        return syn.MhdPaper2DCase(n=n or 512)
    if workload == "hcnsf":
        return syn.HcnsfPaperCase(n=n or 256)
    raise ValueError(workload)


def fields(workload, case):
    if workload in PAPER_D2Q5:
        return case.table().augmented(syn.coords((case.n, case.n)), 0.0)
    if workload == "nsf12":
        return case.table("nsf12").augmented(syn.coords((case.n, case.n)), 0.0)
    if workload == "mhd18":
        return case.table().augmented(syn.coords((case.n, case.n)), 0.0)
    if workload == "hcnsf":
        return case.table().augmented(syn.coords((case.n, case.n, case.n)), 0.0)
    return {"nsf": syn.nsf_fields, "mhd": syn.mhd_fields, "adr": syn.adr_fields}[workload](case)


def scheme(W, L, workload, case, prec, inplace=False, **slab):
    p = PREC[prec]
    sm = L.STREAM_IN_PLACE if inplace else L.STREAM_TWO_BUFFERS
    if slab:
        fn = {"nsf": W.nsf_scheme, "mhd": W.mhd_scheme, "hcnsf": W.hcnsf_scheme}[workload]
        return fn(case, p, **slab)
    if workload in PAPER_D2Q5:
        params, Q0 = case.system_args()
        sysm = W.table_system(case.table(), params, Q0)
        return L.Scheme(sysm, L.D2Q5, (case.n, case.n), L.ACOUSTIC if case.scaling == "acoustic" else L.DIFFUSIVE,
                        case.f, tau_R=case.tau_R, g_tau=case.g_tau, precision=p, streaming=sm)
    if workload == "nsf":
        return W.nsf_scheme(case, p, streaming=sm)
    if workload == "mhd":
        return W.mhd_scheme(case, p, streaming=sm)
    if workload == "nsf12":
        return W.nsf12_scheme(case, p)
    if workload == "mhd18":
        return W.mhd18_scheme(case, p)
    if workload == "hcnsf":
        return W.hcnsf_scheme(case, p, streaming=sm)
    assert not inplace
    return W.adr_scheme(case, p)


def kq(workload):
    return {"nsf": (10, 9), "mhd": (11, 19), "adr": (3, 5), "nsf12": (12, 5), "mhd18": (18, 5),
            "hcnsf": (14, 7), "burgers": (1, 5), "euler": (4, 5), "maxwell": (3, 5), "adrp": (3, 5)}[workload]


LATTICE_NAME = {"nsf": "d2q9", "mhd": "d3q19", "adr": "d2q5", "nsf12": "d2q5", "mhd18": "d2q5",
                "hcnsf": "d3q7", "burgers": "d2q5", "euler": "d2q5", "maxwell": "d2q5", "adrp": "d2q5"}
DIM3 = ("mhd", "hcnsf")


def config_of(workload, case, precision, K, q, ws=1):
    """The workload description both arms report."""
    dim = 3 if workload in DIM3 else 2
    grid = "x".join([str(case.n)] * dim)
    bytes_launch = 2 * K * q * STORE_BYTES[precision] * case.n ** dim
    return {"workload": f"{workload}_{LATTICE_NAME[workload]}_{grid}_{precision}", "grid": [case.n] * dim,
            "components": K, "velocities": q, "precision": precision,
            "l2": f"inputs larger than L2 (each population buffer {bytes_launch / 2 / 1e6:.0f} MB > 126 MB)"
            if bytes_launch / 2 > 126e6 else f"L2-resident ({bytes_launch / 1e6:.1f} MB of populations)",
            "parallelism": f"replicas x{ws}"}


def launches_per_step(workload, precision, decomp):
    """Kernel launches of one timed step: the step kernel; in slab mode the two boundary
    planes, the interior, pack and unpack; in float64 with the homogenized NSF's moving solid
    also the one-thread kernel of the step's field-time sines."""
    if decomp == "slab":
        return 5
    return 2 if (workload == "hcnsf" and precision == "fp64") else 1


def cells(workload, case):
    return case.n ** (3 if workload in DIM3 else 2)



# ------------------------------------------------------------------ measurements
def _timed_steps(obj, stream, steps):
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    obj.step(steps)
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / steps


def launch_desc(L, rep):
    """The step kernel lbx_state_tune kept: staging and block (register-resident: none)."""
    if rep["ms_per_step"] < 0:
        return {"kernel": "k_step (register-resident)", "block": 128}
    name = {L.STAGE_THREAD: "k_step (per-thread copies)", L.STAGE_BULK: "k_step_bulk (bulk row copies)",
            L.STAGE_PIPE: "k_step_pipe (pipelined per-thread copies)"}
    return {"kernel": name.get(rep["staging"], str(rep["staging"])), "block": rep["block"],
            "staging": rep["staging"], "tuned_ms_per_step": rep["ms_per_step"]}


def measure_grid(L, W, workload, precision, n, steps, warmup, stream, graph=False, inplace=False):
    """Time one grid workload; returns a dict of rate, ms per step and GB/s.  inplace: one
    population buffer (the steps run in pairs, so `steps` must be even)."""
    case = make_case(workload, n)
    K, q = kq(workload)
    ncell = cells(workload, case)
    st = L.State(scheme(W, L, workload, case, precision, inplace), fields(workload, case).cuda(), stream=stream)
    if inplace:
        st.set_block(64)        # no tuner in place (no scratch buffer): the staged kernels' usual best
    launch = st.tune()
    if graph:
        st.use_graph(True)
    st.step(warmup)
    st.synchronize()
    ms = _timed_steps(st, stream, steps)
    nbytes = 2 * K * q * STORE_BYTES[precision] * ncell
    out = {"lup_s": ncell / (ms * 1e-3), "ms_per_step": ms, "gbs": nbytes / (ms * 1e-3) / 1e9,
           "bytes_per_launch": nbytes, "finite": st.check_finite(), "graph": graph,
           "launch": launch_desc(L, launch) if not inplace else
           {"kernel": "in place, kinds 1 and 2 alternating (k_step_bulk_inplace for staged systems with "
                      "nx % 8 == 0, else k_step_inplace)", "block": launch["block"]},
           "population_buffers": 1 if inplace else 2}
    return out, st


def fluct_err(Qa, Qb, Q0):
    """||Qa - Qb||_2 / ||Qb - Q0||_2 per component (device tensors)."""
    K = Qa.shape[0]
    q0 = torch.tensor(Q0, dtype=torch.float64, device=Qa.device).reshape((K,) + (1,) * (Qa.dim() - 1))
    e = (Qa - Qb).reshape(K, -1).norm(dim=1)
    r = (Qb - q0).reshape(K, -1).norm(dim=1)
    return (e / r).tolist()


def measure_precision_errors(L, W, workload, n, steps, stream):
    """FP32-shift and FP16-scaled against the FP64 kernel (itself pinned to the CPU oracle
    to 1e-12) after `steps` steps at full size."""
    case = make_case(workload, n)
    Q = fields(workload, case).cuda()
    ref = L.State(scheme(W, L, workload, case, "fp64"), Q, stream=stream)
    ref.step(steps)
    R = ref.moments(device=True)
    ref.synchronize()
    ref.close()
    out = {}
    for prec in ("fp32", "fp16"):
        st = L.State(scheme(W, L, workload, case, prec), Q, stream=stream)
        st.step(steps)
        Qp = st.moments(device=True)
        st.synchronize()
        out[prec] = [float(f"{v:.3e}") for v in fluct_err(Qp, R, case.reference_state())]
        st.close()
    del R
    torch.cuda.empty_cache()
    return {"steps": steps, "grid": case.n, "fluct_rel_l2_vs_fp64": out}


def measure_batch(L, W, steps, warmup, stream, n_inst=512, seed=0, trials=5):
    cases = syn.adr_batch_draws(n_inst, seed=seed)
    schemes = [W.adr_scheme(c, L.FP32_SHIFT) for c in cases]
    b = L.Batch(schemes, [syn.adr_fields(c) for c in cases], stream=stream)
    rep = b.tune(trials=trials)
    b.step(warmup)
    b.synchronize()
    ms = _timed_steps(b, stream, steps)
    nbytes = 2 * 3 * 5 * 4 * b.total_cells
    out = {"instances": n_inst, "total_cells": b.total_cells, "lup_s": b.total_cells / (ms * 1e-3),
           "ms_per_step": ms, "gbs": nbytes / (ms * 1e-3) / 1e9, "bytes_per_launch": nbytes,
           "tuned": rep["best"], "graph": True}
    b.close()
    return out


def measure_adjoint(L, W, n=256, steps=2000, ckpt=64):
    """Config 5: gradient of the final density misfit for NSF D2Q9 FP32-shift, checkpoint
    every `ckpt` steps.  Bytes per node-step: forward 2 K q s twice (sweep + recompute) plus
    the reverse step (Lam in and out, forward state in) 3 K q s."""
    case = syn.NsfCase(n=n)
    sch = W.nsf_scheme(case, L.FP32_SHIFT)
    Q, tgt = syn.nsf_fields(case), syn.density_target(n)
    L.adjoint(sch, Q, 64, 16, tgt)        # warm-up (module load, allocations)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    J, g, gt = L.adjoint(sch, Q, steps, ckpt, tgt)
    sec = time.perf_counter() - t0
    ph = L.adjoint_timings()
    dev_s = sum(ph.values()) * 1e-3
    K, q = 10, 9
    cells2 = case.n * case.n
    fwd_b, rev_b = 2 * K * q * 4 * cells2, 3 * K * q * 4 * cells2       # per step
    nrec = steps - (steps + ckpt - 1) // ckpt                            # recomputed steps
    return {"grid": n, "steps": steps, "ckpt_every": ckpt,
            "seconds_per_gradient": dev_s, "seconds_per_gradient_wall": sec, "phases_ms": ph,
            "forward_ms_per_step": ph["forward_ms"] / steps,
            "recompute_ms_per_step": ph["recompute_ms"] / max(nrec, 1),
            "reverse_ms_per_step": ph["reverse_ms"] / steps,
            "forward_gbs": fwd_b / (ph["forward_ms"] / steps * 1e-3) / 1e9,
            "reverse_gbs": rev_b / (ph["reverse_ms"] / steps * 1e-3) / 1e9,
            "J": J, "dJ_dtau": gt,
            "note": ("seconds_per_gradient: device time of the forward sweep, recomputation, reverse steps "
                     "and the rest (CUDA events inside lbx_adjoint; allocation and host copies excluded); "
                     "the wall time includes them.  Reverse step bytes per node: Lambda in and out (FP32) "
                     "plus the forward populations (FP32), 3 K q 4.  The 256^2 working set (two population "
                     "buffers 47 MB, Lambda 47 MB) is L2-resident, so GB/s here are not HBM figures.")}


def run_variants(L, W, args, stream, peak, probe_fp64=None):
    v = {}
    t0 = time.perf_counter()
    for wl, prec, n, steps in (("nsf", "fp64", 1024, 100), ("nsf", "fp16", 1024, 1000),
                               ("mhd", "fp32", 256, 50), ("mhd", "fp16", 256, 50),
                               ("nsf12", "fp32", 1024, 500), ("nsf12", "fp16", 1024, 500),
                               ("nsf12", "fp64", 1024, 100), ("mhd18", "fp32", 512, 500),
                               ("mhd18", "fp64", 512, 100), ("hcnsf", "fp32", 256, 100),
                               ("hcnsf", "fp16", 256, 100), ("hcnsf", "fp64", 256, 20),
                               ("adr", "fp64", 64, 500), ("nsf", "fp32", 1024, "inplace"),
                               ("mhd", "fp32", 256, "inplace"), ("hcnsf", "fp32", 256, "inplace"),
                               ("burgers", "fp32", 4096, 400), ("burgers", "fp64", 4096, 100),
                               ("euler", "fp32", 4096, 200), ("euler", "fp64", 4096, 20),
                               ("maxwell", "fp32", 4096, 200), ("maxwell", "fp64", 4096, 20),
                               ("adrp", "fp32", 4096, 200), ("adrp", "fp64", 4096, 20)):
        inplace = steps == "inplace"
        steps = {"nsf": 1000, "mhd": 50, "hcnsf": 100}[wl] if inplace else steps
        # the 64^2 case is launch-latency bound: its 500 steps replay as one CUDA graph
        r, st = measure_grid(L, W, wl, prec, n, steps, 6 if wl != "adr" else 500, stream, graph=(wl == "adr"),
                             inplace=inplace)
        st.close()
        r["frac_of_hbm_peak"] = r["gbs"] / peak
        ncell = n ** (3 if wl in DIM3 else 2)
        r["traffic_per_launch"] = None if inplace else profile_traffic(f"{wl}_{prec}", ncell)
        r["traffic_kernel"] = None if inplace else profile_kernel(f"{wl}_{prec}")
        if prec == "fp64":
            fl = profile_entry(f"{wl}_fp64_flops")
            if fl:
                ach = fl["fp64_flops_per_node"] * r["lup_s"] / 1e9
                r["alu_roofline"] = {"bound": "alu", "achieved": ach, "unit": "GFLOP/s",
                                     "fp64_flops_per_node": fl["fp64_flops_per_node"],
                                     "peak_probe": probe_fp64, "frac": ach / probe_fp64 if probe_fp64 else None}
                if fl.get("fp64_inst_per_node") and probe_fp64:
                    # DADD and DMUL take a slot of the FP64 pipe as a DFMA does: the issue-slot
                    # roofline is the probe's DFMA rate (probe GFLOP/s / 2) per FP64 instruction
                    ai = fl["fp64_inst_per_node"] * r["lup_s"] / 1e9
                    r["alu_roofline"]["fp64_inst_per_node"] = fl["fp64_inst_per_node"]
                    r["alu_roofline"]["inst_frac"] = ai / (probe_fp64 / 2.0)
        v[f"{wl}_{prec}_{n}" + ("_inplace" if inplace else "")] = r
        torch.cuda.empty_cache()
    r = measure_batch(L, W, 200, 5, stream)
    r["frac_of_hbm_peak"] = r["gbs"] / peak
    v["adr_batch512_fp32"] = r
    v["adjoint_nsf256_fp32"] = measure_adjoint(L, W)
    v["precision_errors"] = {"nsf_1024": measure_precision_errors(L, W, "nsf", 1024, 2000, stream),
                             "mhd_128": measure_precision_errors(L, W, "mhd", 128, 500, stream)}
    v["seconds"] = time.perf_counter() - t0
    return v

# --------------------------------------------------------------------- our arm
def slab_kwargs(workload, case, rank, ws):
    """Slab arguments of rank `rank` when every rank holds one case-sized slab of a grid
    stacked along the last axis (weak scaling): global planes n ws, origin n rank.  The
    seeded fields are periodic with period 1 in every coordinate, so each slab's initial
    fields are the case's own."""
    if workload not in ("nsf", "mhd", "hcnsf"):
        raise SystemExit(f"--decomp slab: workload {workload} has no slab wiring")
    dim3 = workload in DIM3
    ext = (case.n, case.n, case.n) if dim3 else (case.n, case.n)
    return {"extent": ext, "slab_origin": rank * case.n, "slab_planes_global": ws * case.n}


def run_ours(args):
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2607_05668_b300 import lbx as L, workloads as W, slab as SL

    decomp = args.decomp or ("slab" if ws > 1 else "whole")
    case = make_case(args.workload, args.n)
    Q = fields(args.workload, case)
    ncell = cells(args.workload, case)
    K, q = kq(args.workload)
    stream = torch.cuda.Stream()
    ring = None
    if decomp == "slab":
        ring = SL.RingExchange(rank=0, world=1) if ws == 1 else SL.RingExchange()
        kw = slab_kwargs(args.workload, case, rank, ws)
        sch = scheme(W, L, args.workload, case, args.precision, **kw)
        if args.precision == "fp16":        # the slabs share the grid's storage scales
            probe_st = L.State(sch, Q.cuda(), stream=stream)
            kw["fp16_scales"] = list(ring.max(probe_st.scales()))
            probe_st.close()
            sch = scheme(W, L, args.workload, case, args.precision, **kw)
    else:
        sch = scheme(W, L, args.workload, case, args.precision)
    with torch.cuda.stream(stream):
        slab = SL.Slab(sch, Q.cuda(), stream=stream) if decomp == "slab" else None
    st = slab.state if slab else L.State(sch, Q.cuda(), stream=stream)

    side = SL.side_stream() if decomp == "slab" else None

    def run_steps(n, state=None, sl=None):
        if sl is not None:
            # the face exchange (pack, NCCL send/recv, unpack) on a second stream behind the
            # interior planes of every step
            with torch.cuda.stream(stream):
                SL.step_ring_overlap(sl, ring, n, side)
        else:
            state.step(n)

    if args.staging is not None:            # a fixed launch shape (profiling one staging)
        sg = {"thread": L.STAGE_THREAD, "bulk": L.STAGE_BULK, "lanes2": L.STAGE_LANES2,
              "pipe": L.STAGE_PIPE}[args.staging]
        st.set_staging(sg)
        st.set_block(args.block)
        launch = {"kernel": f"staging {args.staging} (fixed)", "block": args.block, "staging": sg}
    else:
        launch = launch_desc(L, st.tune())  # staged kernels: fastest launch shape, state unchanged
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    graph = decomp != "slab" and not args.no_graph
    with ClockSampler(local) as clk:
        # untimed: settle the clocks (an idle GPU starts a few percent slow) and, with graph
        # replay, record the K-step graph for both buffer parities before the timed call
        if graph:
            st.use_graph(True)
        run_steps(args.warmup, st, slab)
        # chunks of exactly K steps: an even K keeps the buffer parity the timed call starts
        # from, an odd K alternates it, so either way the timed call's graph (keyed by step
        # count and parity) is recorded here and not inside the timed region
        t_pre, pre = time.perf_counter(), 0
        chunk = args.steps if graph else max(args.steps, 50)
        while pre < 2 * chunk or time.perf_counter() - t_pre < 0.25:
            run_steps(chunk, st, slab)
            pre += chunk
            if pre % (8 * chunk) == 0:
                st.synchronize()
        st.synchronize()
        t_pre = time.perf_counter() - t_pre
        barrier()
        e0.record(stream)
        run_steps(args.steps, st, slab)
        e1.record(stream)
        e1.synchronize()
        barrier()
    ms = e0.elapsed_time(e1)
    if ws > 1:
        import torch.distributed as dist
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    ms_step = ms / args.steps
    finite = st.check_finite()
    value = ws * ncell * args.steps / (ms * 1e-3)

    # roofline of the step kernel: algorithmic bytes 2 K q s per node update
    bytes_launch = 2 * K * q * STORE_BYTES[args.precision] * ncell
    peak, peak_kind = measured_peaks()
    achieved = bytes_launch / (ms_step * 1e-3) / 1e9
    traffic = profile_traffic(f"{args.workload}_{args.precision}", ncell)
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": traffic, "traffic_kernel": profile_kernel(f"{args.workload}_{args.precision}"),
            "peak_kind": peak_kind, "algorithmic_bytes_per_launch": bytes_launch}
    if decomp == "slab":
        roof["note"] = "time per step includes the face exchange (pack, transport, unpack)"
    if args.precision == "fp64":
        roof["note"] = "FP64 arithmetic on B300 is far below the HBM ridge; see fp64_alu"

    # end to end through the C ABI from host memory: lbx_init with the fields in pinned host
    # memory (the init kernel reads them over the bus; then the finite and sub-characteristic
    # checks), `steps` steps, and lbx_moments into pinned host memory (the moments kernel
    # writes them over the bus).  The population buffers are allocated once, outside the timed region
    # (caller-owned buffers, as a program that solves repeatedly keeps them).
    if slab:
        slab.close()
    else:
        st.close()
    Qh = torch.empty(Q.shape, dtype=Q.dtype, pin_memory=True)
    Qh.copy_(Q)
    out_h = torch.empty(Q.shape, dtype=Q.dtype, pin_memory=True)
    # the host buffers are reused from run to run: one untimed copy each way maps them for the
    # copy engines first (the first copy into a fresh pinned buffer measured about 5x slower)
    tmp = Qh.to("cuda")
    out_h.copy_(tmp)
    del tmp
    bufs = [torch.empty(sch.buffer_bytes, dtype=torch.uint8, device="cuda") for _ in range(2)]
    faces = [torch.empty(max(sch.halo_bytes, 16), dtype=torch.uint8, device="cuda") for _ in range(4)]
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    barrier()
    t0 = time.perf_counter()
    sl2 = SL.Slab(sch, Qh, stream=stream, buffers=bufs, faces=faces) if decomp == "slab" else None
    st2 = sl2.state if sl2 else L.State(sch, Qh, stream=stream, buffers=bufs)   # synchronous (checks)
    t1 = time.perf_counter()
    if launch.get("staging") is not None:
        st2.set_staging(launch["staging"])
        st2.set_block(launch["block"])
    ev[0].record(stream)
    run_steps(args.steps, st2, sl2)
    ev[1].record(stream)
    st2.moments_into(out_h)                  # synchronous: waits for the steps
    t2 = time.perf_counter()
    e2e_s = t2 - t0
    if ws > 1:
        import torch.distributed as dist
        t = torch.tensor([e2e_s], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    st2.close()
    del bufs
    steps_ms = ev[0].elapsed_time(ev[1])
    e2e = {"value": ws * ncell * args.steps / e2e_s, "unit": "LUP/s",
           "h2d_bytes_per_step": Qh.numel() * 8 / args.steps,
           "d2h_bytes_per_step": out_h.numel() * 8 / args.steps,
           "run": f"lbx_init from pinned host fields (read by the init kernel over PCIe; checks) + "
                  f"{args.steps} steps + lbx_moments into pinned host memory (written by the moments kernel "
                  "over PCIe), per run; population buffers and pinned host buffers allocated (and the host "
                  "buffers used once) outside",
           "split_ms": {"init_incl_h2d_and_checks": (t1 - t0) * 1e3,
                        "steps": steps_ms,
                        "moments_incl_d2h_after_steps": max((t2 - t1) * 1e3 - steps_ms, 0.0),
                        "total": e2e_s * 1e3}}

    config = config_of(args.workload, case, args.precision, K, q, ws)
    if decomp == "slab":
        g = list(config["grid"])
        g[-1] = case.n * ws
        config["parallelism"] = (f"slab x{ws}: one {'z' if args.workload in DIM3 else 'y'}-slab of "
                                 f"{'x'.join(map(str, config['grid']))} per GPU of a {'x'.join(map(str, g))} "
                                 "grid, one face exchange per step (boundary planes, lbx_halo_pack_next, NCCL "
                                 "send/recv, lbx_halo_unpack_next on a second stream behind the interior planes)")
    result = {
        "metric": "Lattice updates/s", "value": value, "unit": "LUP/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": PREC_NAME[args.precision], "data": "synthetic",
        "config": config,
        "roofline": roof, "e2e": e2e, "gpu_launches": args.steps * launches_per_step(args.workload, args.precision, decomp),
        "finite": finite, "launch": launch, "clocks": clk.summary(),
        "timing": {"graph_replay": graph, "pre_warm_steps": pre, "pre_warm_s": t_pre,
                   "note": "the W warm-up steps, then untimed pre-warm steps in calls of K steps (at least "
                           "0.25 s: they settle the clocks and record the graph the timed call replays); the "
                           "K timed steps follow a barrier and a device synchronisation"},
    }
    if rank == 0 and (args.precision == "fp64" or args.probe or not args.no_variants):
        result["probe"] = L.probe_peaks(2 << 30, stream=stream)
    if rank == 0 and not args.no_variants and args.workload == "nsf" and args.precision == "fp32":
        result["variants"] = run_variants(L, W, args, stream, peak, result["probe"]["fp64_gflops"])
    if rank == 0 and not args.no_cpu:
        result["cpu_baseline"] = cpu_baseline(args, case)
    if rank == 0:
        print(json.dumps(result), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


# ----------------------------------------------------------------- CPU oracle arm
def _oracle_scheme(workload, case, shape):
    import oracle
    from oracle import systems as S
    if workload == "nsf":
        sysm = S.NsfPrimitive(case.gamma, case.R, case.mu, case.kappa, case.g_tau * case.dt)
        lat = "D2Q9"
    elif workload == "mhd":
        sysm = S.MhdCurrent(case.gamma, case.eta, case.g_tau * case.dt)
        lat = "D3Q19"
    elif workload == "nsf12":
        sysm = S.NsfConservedGradients(case.gamma, case.R, case.mu, case.kappa, case.g_tau * case.dt)
        lat = "D2Q5"
    elif workload == "mhd18":
        sysm = S.MhdPowell2D(case.gamma, case.mu, case.kappa, case.eta, case.g_tau * case.dt)
        lat = "D2Q5"
    elif workload in PAPER_D2Q5:
        params, _ = case.system_args()
        sysm = {"burgers": lambda: S.Burgers(), "euler": lambda: S.Euler(*params),
                "maxwell": lambda: S.MaxwellTM(*params),
                "adrp": lambda: S.AdrCascade(params[:2], params[2], case.g_tau * case.dt, params[3])}[workload]()
        lat = "D2Q5"
    elif workload == "hcnsf":
        sysm = S.HomogenizedNsf3D(case.gamma, case.mu, case.kappa, case.eta, case.g_tau * case.dt,
                                  fields=case.prescribed)
        lat = "D3Q7"
    else:
        sysm = S.AdrCascade(case.a_phys, case.nu, case.g_tau * case.dt)
        lat = "D2Q5"
    tau = oracle.tau_vector(sysm, case.dt, tau_R=getattr(case, "tau_R", None),
                            tau_cons=getattr(case, "tau_u", None), g_tau=case.g_tau)
    return oracle.Scheme(sysm, oracle.LATTICES[lat], shape, case.dx, case.dt, tau,
                         source_theta=getattr(case, "theta", 0.0), flux_theta=getattr(case, "theta_flux", 0.0))


def _oracle_sample(workload, case, rows):
    """The oracle on a periodic slab of `rows` rows of the full grid (same per-node work)."""
    Q = fields(workload, case)
    Qs = Q[..., :rows, :].contiguous() if workload not in DIM3 else Q[:, :rows].contiguous()
    shape = tuple(Qs.shape[1:])
    sch = _oracle_scheme(workload, case, shape)
    return sch, sch.init(Qs), int(Qs[0].numel())


def cpu_baseline(args, case, budget_s=15.0):
    cores = torch.get_num_threads()
    rows = 64 if args.workload not in DIM3 else 8
    sch, f, n = _oracle_sample(args.workload, case, rows)
    f = sch.step(f, 0.0)                      # warm up
    t0 = time.perf_counter()
    steps = 0
    while time.perf_counter() - t0 < budget_s:
        f = sch.step(f, 0.0)
        steps += 1
    el = time.perf_counter() - t0
    return {"value": steps * n / el, "unit": "LUP/s", "cores": cores, "kind": "oracle",
            "sample": f"{steps} FP64 oracle steps on a periodic {rows}-row slab of the {case.n}-wide grid "
                      f"({n} nodes), {el:.1f} s"}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    case = make_case(args.workload, args.n)
    K, q = kq(args.workload)
    # each step is one oracle step on a slab sized so the whole run stays within minutes
    budget = 150.0
    sch, f, n = _oracle_sample(args.workload, case, 8 if args.workload not in DIM3 else 2)
    t0 = time.perf_counter()
    f = sch.step(f, 0.0)
    per_step = time.perf_counter() - t0
    total = args.steps + args.warmup
    rows = max(2, min(case.n, int(8 * budget / max(per_step * total, 1e-9))))
    if args.workload in DIM3:
        rows = max(2, min(case.n, rows // 4))
    sch, f, n = _oracle_sample(args.workload, case, rows)
    for _ in range(args.warmup):
        f = sch.step(f, 0.0)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        f = sch.step(f, 0.0)
    el = time.perf_counter() - t0
    value = n * args.steps / el
    cores = torch.get_num_threads()
    sample = f"each step: one FP64 oracle step on a periodic {rows}-row slab ({n} nodes) of the {case.n}-wide grid"
    print(json.dumps({
        "impl": "reference", "metric": "Lattice updates/s", "value": value, "unit": "LUP/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": config_of(args.workload, case, args.precision, K, q, ws),
        "cpu_baseline": {"value": value, "unit": "LUP/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "LUP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="nsf",
                    choices=["nsf", "mhd", "adr", "nsf12", "mhd18", "hcnsf"] + list(PAPER_D2Q5))
    ap.add_argument("--precision", default="fp32", choices=["fp64", "fp32", "fp16"])
    ap.add_argument("--n", type=int, default=None, help="grid size override")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--probe", action="store_true", help="also run the copy / FMA peak probes")
    ap.add_argument("--no-variants", action="store_true", help="skip the other precisions and workloads")
    ap.add_argument("--staging", choices=["thread", "bulk", "lanes2", "pipe"], default=None,
                    help="staged kernels: fix the staging instead of tuning (with --block)")
    ap.add_argument("--block", type=int, default=128, choices=[32, 64, 128], help="block size with --staging")
    ap.add_argument("--no-graph", action="store_true", help="launch the timed steps one by one (no graph replay)")
    ap.add_argument("--decomp", choices=["whole", "slab", "replicas"], default=None,
                    help="multi-GPU layout: slab (default for N > 1) = one slab per GPU of one grid with a face "
                         "exchange per step; replicas = independent grids; whole (N = 1 default)")
    ap.add_argument("--adjoint-only", type=int, default=None, metavar="STEPS",
                    help="only the config-5 adjoint (NSF D2Q9 256^2 FP32, checkpoints every 64) over STEPS steps")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.adjoint_only is not None:
        from paper_2607_05668_b300 import lbx as L, workloads as W
        print(json.dumps(measure_adjoint(L, W, steps=args.adjoint_only)), flush=True)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
