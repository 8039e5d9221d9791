"""Parity at the benchmark's full sizes and in its launch configuration (the tuned staging of
`bench.py`), on sampled nodes: the oracle computes each sampled node's moments on a small
periodic patch around it (tests/helpers.patch_moments, checked against full-domain runs on
the CPU), including nodes at the domain's edges and corners."""
import pytest
import torch

import oracle
import synthetic as syn
from oracle import systems as S
from tests import helpers as H

pytestmark = pytest.mark.gpu

lbx = pytest.importorskip("paper_2607_05668_b300.lbx")
from paper_2607_05668_b300 import workloads as W  # noqa: E402

F64 = torch.float64


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")


def _gpu_nodes(st, centers):
    Qg = st.moments()
    return torch.stack([Qg[(slice(None),) + tuple(c)] for c in centers], dim=1)


def _check(kind, got, want, case, prec, n_cons, cs2, R=1.0):
    """Per field, max |diff| over the population scale of the field (tests/helpers.parity_scales):
    for a conserved field its size (FP64) or its fluctuation about Q0 (shifted FP32); for a
    tracker of V also |V| / (c_s^2 g_tau dx) (shifted: |V - V0| / ...), the size of the
    V / tau_grad term its equilibrium populations carry, which sets the rounding unit of its
    moment.  After a few steps the GPU and the oracle differ by the rounding of q populations
    of that scale per step (q eps: 2e-15 in FP64, 1e-6 in FP32), so the bounds are 1e-12
    (FP64) and 1e-4 (FP32) for every field, trackers included."""
    shifted = prec != lbx.FP64
    scale = H.parity_scales(kind, want, case.reference_state(), n_cons, case.dx, case.g_tau, cs2, case.gamma,
                            shifted, R)
    err = (got - want).abs().amax(1) / scale
    print(kind, "FP64" if prec == lbx.FP64 else "FP32", [f"{v:.2e}" for v in err.tolist()])
    assert float(err.max()) <= (1e-12 if prec == lbx.FP64 else 1e-4), err.tolist()


@pytest.mark.parametrize("prec", [lbx.FP32_SHIFT, lbx.FP64])
def test_nsf_d2q9_1024_sampled_nodes(prec):
    """The benchmark's own workload (NSF D2Q9 1024^2) after 3 steps."""
    n, steps = 1024, 3
    case = syn.NsfCase(n=n)
    Q = syn.nsf_fields(case)
    st = lbx.State(W.nsf_scheme(case, prec), Q.cuda())
    st.tune()
    st.step(steps)
    centers = [(0, 0), (n - 1, n // 3), (n // 2, n - 1), (n // 4, n // 2), (7, 9), (n - 5, n - 7)]
    ref = H.oracle_nsf(case)
    make = lambda shape, origin: oracle.Scheme(ref.sys, ref.lat, shape, case.dx, case.dt, ref.tau)
    _check("nsf", _gpu_nodes(st, centers), H.patch_moments(make, Q, centers, steps, steps + 1), case, prec, 4,
           1.0 / 3.0, case.R)


def test_mhd_d3q19_256_sampled_nodes():
    """The 3D MHD variant (D3Q19 256^3, FP32, bulk row copies as tuned) after 2 steps."""
    n, steps = 256, 2
    case = syn.MhdCase(n=n)
    Q = syn.mhd_fields(case)
    st = lbx.State(W.mhd_scheme(case, lbx.FP32_SHIFT), Q.cuda())
    st.tune()
    st.step(steps)
    centers = [(0, 0, 0), (n - 1, n // 3, 5), (n // 2, n - 1, n // 4), (3, 7, n - 1), (n // 2, n // 2, n // 2)]
    ref = H.oracle_mhd(case)
    make = lambda shape, origin: oracle.Scheme(ref.sys, ref.lat, shape, case.dx, case.dt, ref.tau)
    _check("mhd", _gpu_nodes(st, centers), H.patch_moments(make, Q, centers, steps, steps + 1), case,
           lbx.FP32_SHIFT, 8, 1.0 / 3.0)


def test_hcnsf_d3q7_256_sampled_nodes():
    """The 3D homogenized NSF variant (D3Q7 256^3, FP32, the moving solid's fields) after 2
    steps, every field (the trackers start at the exact gradients of the flow)."""
    n, steps = 256, 2
    case = syn.HcnsfPaperCase(n=n)
    Q = case.table().augmented(syn.coords((n, n, n)), 0.0)
    st = lbx.State(W.hcnsf_scheme(case, lbx.FP32_SHIFT), Q.cuda())
    st.tune()
    st.step(steps)
    # edges and corners, at coordinates where the flow's fluctuations are not small
    centers = [(37, 101, n - 5), (n - 1, 3, 77), (0, 130, n - 1), (129, 64, 31), (n - 1, n - 1, 0), (37, 101, 211)]
    sysm = S.HomogenizedNsf3D(case.gamma, case.mu, case.kappa, case.eta, case.g_tau * case.dt, fields=case.prescribed)
    tau = oracle.tau_vector(sysm, case.dt, tau_R=case.tau_R, g_tau=case.g_tau)
    make = lambda shape, origin: oracle.Scheme(sysm, oracle.LATTICES["D3Q7"], shape, case.dx, case.dt, tau,
                                               source_theta=case.theta, origin=origin)
    _check("hcnsf", _gpu_nodes(st, centers), H.patch_moments(make, Q, centers, steps, steps + 1), case,
           lbx.FP32_SHIFT, 5, 0.25)
