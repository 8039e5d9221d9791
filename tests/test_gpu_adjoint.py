"""Hand-written GPU adjoint (lbx_adjoint) against the oracle's reverse-mode gradient of its
own FP64 forward, against central finite differences (h = 1e-4, FP64), and the
checkpoint-interval invariance of the recompute."""
import numpy as np
import pytest
import torch

import oracle
import synthetic as syn
from tests import helpers as H

pytestmark = pytest.mark.gpu

lbx = pytest.importorskip("paper_2607_05668_b300.lbx")
from paper_2607_05668_b300 import workloads as W  # noqa: E402
from paper_2607_05668_b300.autograd import DensityMisfit  # noqa: E402

F64 = torch.float64


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")


def _nsf(N, tau):
    case = syn.NsfCase(n=N)
    return case, (lambda prec: W.nsf_scheme(case, prec, tau_lb=tau))


def _oracle_grad(case, Q, target, steps, tau):
    sysm = oracle.systems.NsfPrimitive(case.gamma, case.R, case.mu, case.kappa, case.g_tau * case.dt)

    def make(tc):
        t = oracle.tau_vector(sysm, case.dt, tau_cons=tc, g_tau=case.g_tau)
        return oracle.Scheme(sysm, oracle.LATTICES["D2Q9"], (case.n, case.n), case.dx, case.dt, t)
    return oracle.adjoint.misfit_and_grad(make, Q, target, steps, tau)


def _rel(a, b):
    return float((a - b).abs().max() / b.abs().max())


def test_fp64_adjoint_matches_oracle_gradient():
    N, steps, tau = 32, 40, 0.52
    case, mk = _nsf(N, tau)
    Q, tgt = syn.nsf_fields(case), syn.density_target(N)
    J, g, gt = lbx.adjoint(mk(lbx.FP64), Q, steps, 8, tgt)
    Jo, go, gto = _oracle_grad(case, Q, tgt, steps, tau)
    assert abs(J - Jo) <= 1e-12 * abs(Jo)
    assert _rel(g, go) <= 1e-10
    assert abs(gt - gto) <= 1e-10 * abs(gto)


def test_fp32_adjoint_against_fp64_oracle():
    N, steps, tau = 32, 40, 0.52
    case, mk = _nsf(N, tau)
    Q, tgt = syn.nsf_fields(case), syn.density_target(N)
    J, g, gt = lbx.adjoint(mk(lbx.FP32_SHIFT), Q, steps, 8, tgt)
    Jo, go, gto = _oracle_grad(case, Q, tgt, steps, tau)
    assert abs(J - Jo) <= 1e-4 * abs(Jo)
    rho_rel = _rel(g[0], go[0])
    print("FP32 adjoint: rel dJ/drho", rho_rel, "rel dJ/dtau", abs(gt - gto) / abs(gto))
    assert rho_rel <= 1e-4
    assert abs(gt - gto) <= 1e-4 * abs(gto)


def test_checkpoint_interval_does_not_change_the_result():
    case, mk = _nsf(24, 0.55)
    Q, tgt = syn.nsf_fields(case), syn.density_target(24)
    a = lbx.adjoint(mk(lbx.FP32_SHIFT), Q, 30, 4, tgt)
    b = lbx.adjoint(mk(lbx.FP32_SHIFT), Q, 30, 30, tgt)
    c = lbx.adjoint(mk(lbx.FP32_SHIFT), Q, 30, 7, tgt)      # uneven last segment
    assert a[0] == b[0] == c[0] and a[2] == b[2] == c[2]
    assert torch.equal(a[1], b[1]) and torch.equal(a[1], c[1])


def test_fp64_adjoint_against_central_differences():
    """h = 1e-4 central differences of the GPU FP64 forward: a random direction of the
    initial density, eight single nodes of rho (corners, edges, interior), and tau; 1e-5
    relative."""
    N, steps, tau, h = 32, 60, 0.52, 1e-4
    case, mk = _nsf(N, tau)
    Q, tgt = syn.nsf_fields(case), syn.density_target(N)
    J, g, gt = lbx.adjoint(mk(lbx.FP64), Q, steps, 16, tgt)

    def Jof(Qx, t=tau):
        sch = W.nsf_scheme(case, lbx.FP64, tau_lb=t)
        return lbx.adjoint(sch, Qx, steps, steps, tgt)[0]
    v = torch.zeros_like(Q)
    v[0] = torch.randn(Q[0].shape, dtype=F64, generator=torch.Generator().manual_seed(0))
    fd = (Jof(Q + h * v) - Jof(Q - h * v)) / (2 * h)
    assert abs(fd - float((g * v).sum())) <= 1e-5 * abs(fd)
    for (yy, xx) in ((3, 5), (17, 29), (31, 0), (0, 31), (8, 8), (22, 13), (30, 30), (12, 2)):
        e = torch.zeros_like(Q)
        e[0, yy, xx] = 1.0
        fdn = (Jof(Q + h * e) - Jof(Q - h * e)) / (2 * h)
        assert abs(fdn - float(g[0, yy, xx])) <= 1e-5 * abs(fdn) + 1e-9 * float(g[0].abs().max())
    fdt = (Jof(Q, tau + h) - Jof(Q, tau - h)) / (2 * h)
    assert abs(fdt - gt) <= 1e-5 * abs(fdt)


def test_forced_adr_adjoint_matches_oracle():
    """The forcing depends on the step index: the recompute must restore it per segment."""
    case = syn.AdrCase(n=32)
    Q, tgt = syn.adr_fields(case), 1.0 + 0.05 * torch.cos(2 * np.pi * syn.coords((32, 32))[0])
    J, g, gt = lbx.adjoint(W.adr_scheme(case, lbx.FP64), Q, 23, 5, tgt)
    och_sys = oracle.systems.AdrCascade(case.a_phys, case.nu, case.g_tau * case.dt)
    from oracle.mms import make_mms

    def make(tc):
        t = oracle.tau_vector(och_sys, case.dt, tau_cons=tc, g_tau=case.g_tau)
        xs = syn.coords((32, 32))
        mms = make_mms(och_sys, lambda x, y, T: syn.adr_exact(case, x, y, T).unsqueeze(0), xs, dt=case.dt,
                       conserved_only=True)
        return oracle.Scheme(och_sys, oracle.LATTICES["D2Q5"], (32, 32), case.dx, case.dt, t, mms=mms)
    Jo, go, gto = oracle.adjoint.misfit_and_grad(make, Q, tgt, 23, case.tau_u)
    assert abs(J - Jo) <= 1e-12 * abs(Jo)
    assert _rel(g, go) <= 1e-10 and abs(gt - gto) <= 1e-10 * abs(gto)


def test_autograd_function_returns_the_adjoint_gradients():
    case, mk = _nsf(16, 0.53)
    Q = syn.nsf_fields(case).requires_grad_(True)
    tau = torch.tensor(0.53, dtype=F64, requires_grad=True)
    tgt = syn.density_target(16)
    J = DensityMisfit.apply(Q, tau, tgt, lambda t: W.nsf_scheme(case, lbx.FP64, tau_lb=t), 12, 5)
    gQ, gt = torch.autograd.grad(3.0 * J, [Q, tau])
    J2, g2, gt2 = lbx.adjoint(mk(lbx.FP64), Q.detach(), 12, 5, tgt)
    assert float(J) == J2
    assert torch.equal(gQ, 3.0 * g2) and float(gt) == 3.0 * gt2


def test_linear_adr_adjoint_is_the_transposed_oracle_matrix_8x8():
    """Linear ADR cascade (no forcing) on 8 x 8: with the oracle's equilibrium map E
    (192 -> 960), one-step matrix M (960 x 960) and density projection P, both built column
    by column, J = 1/2 |P M^n E Q0 - rho*|^2 has the gradient E^T (M^T)^n P^T r.  The GPU
    adjoint must equal it; and, J being quadratic, a central difference of J along any
    direction equals <dJ/dQ0, v> for any step h (the tangent-adjoint dot-product identity)."""
    N, steps = 8, 6
    case = syn.AdrCase(n=N, tau_u=0.83)
    och = H.oracle_adr(case, forcing=False)
    K, q, nn = 3, 5, N * N
    nQ, nf = K * nn, K * q * nn
    E = torch.zeros(nf, nQ, dtype=F64)
    for j in range(nQ):
        e = torch.zeros(nQ, dtype=F64)
        e[j] = 1.0
        E[:, j] = och.init(e.reshape(K, N, N)).reshape(-1)
    M = torch.zeros(nf, nf, dtype=F64)
    P = torch.zeros(nn, nf, dtype=F64)
    for j in range(nf):
        e = torch.zeros(nf, dtype=F64)
        e[j] = 1.0
        f = e.reshape(K, q, N, N)
        M[:, j] = och.step(f, 0.0).reshape(-1)
        P[:, j] = och.moments(f)[0].reshape(-1)
    g = torch.Generator().manual_seed(3)
    Q = syn.adr_fields(case) + 0.01 * torch.randn((K, N, N), dtype=F64, generator=g)
    tgt = 1.0 + 0.05 * torch.randn((N, N), dtype=F64, generator=g)
    Mn = torch.linalg.matrix_power(M, steps)
    r = P @ Mn @ E @ Q.reshape(-1) - tgt.reshape(-1)
    grad_m = (E.T @ Mn.T @ P.T @ r).reshape(K, N, N)
    sch = W.adr_scheme(case, lbx.FP64, forcing=False)
    J, gq, _ = lbx.adjoint(sch, Q, steps, 4, tgt)
    assert abs(J - 0.5 * float(r @ r)) <= 1e-12 * abs(J)
    assert _rel(gq, grad_m) <= 1e-12
    v = torch.randn((K, N, N), dtype=F64, generator=g)
    for h in (1e-1, 1e-3):
        Jp = lbx.adjoint(sch, Q + h * v, steps, steps, tgt)[0]
        Jm = lbx.adjoint(sch, Q - h * v, steps, steps, tgt)[0]
        dd = float((gq * v).sum())
        assert abs((Jp - Jm) / (2 * h) - dd) <= 1e-9 * abs(dd) + 1e-12 * J / h


def test_paper_nsf12_adjoint_matches_oracle_gradient():
    """The adjoint of the paper's 12-component NSF (conserved-gradient trackers) on D2Q5,
    FP64, against the oracle's reverse-mode gradient of its own forward."""
    N, steps, tau = 24, 20, 0.55
    c = syn.NsfPaperCase(n=N)
    tab = c.table("nsf12")
    Q = tab.augmented(syn.coords((N, N)), 0.0)
    tgt = syn.density_target(N)

    def gsch(t):
        return lbx.Scheme(lbx.System(lbx.NSF_CONS_TRACK, params=(c.gamma, c.R, c.mu, c.kappa),
                                     Q0=c.reference_state_cascade()),
                          lbx.D2Q5, (N, N), lbx.DIFFUSIVE, c.f, tau_lb=t, g_tau=c.g_tau, precision=lbx.FP64)
    J, g, gt = lbx.adjoint(gsch(tau), Q, steps, 6, tgt)
    osys = oracle.systems.NsfConservedGradients(c.gamma, c.R, c.mu, c.kappa, c.g_tau * c.dt)

    def make(tc):
        t = oracle.tau_vector(osys, c.dt, tau_cons=tc, g_tau=c.g_tau)
        return oracle.Scheme(osys, oracle.LATTICES["D2Q5"], (N, N), c.dx, c.dt, t)
    Jo, go, gto = oracle.adjoint.misfit_and_grad(make, Q, tgt, steps, tau)
    assert abs(J - Jo) <= 1e-12 * abs(Jo)
    assert _rel(g, go) <= 1e-10
    assert abs(gt - gto) <= 1e-10 * abs(gto)
