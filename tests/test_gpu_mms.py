"""Manufactured forcing from mode tables on the GPU (LBX_MMS_FOURIER, Sec. 4).

1. Parity: forced FP64 runs of every family equal the CPU oracle, whose forcing comes from
   forward-mode differentiation (torch.func.jvp) of the same exact fields, to 1e-12.
2. The paper's Table 3 at its printed resolution: the GPU runs the paper's own Burgers,
   Maxwell TM and Euler fields and recipes at N = 256 and 512 up to t = 1; the relative L2
   error at N = 512 must be within 5 % of the printed value and the 256 -> 512 order within
   0.1 of the printed EOC (tests/golden/table3.txt).
3. Second-order convergence of the configurations' own systems under forcing: NSF with
   primitive trackers on D2Q9 (diffusive) and 3D MHD with the current tracker on D3Q19
   (acoustic).
"""
import math

import pytest
import torch

import oracle
import synthetic as syn
from oracle.mms import make_mms
from tests import helpers as H

pytestmark = pytest.mark.gpu

lbx = pytest.importorskip("paper_2607_05668_b300.lbx")
from paper_2607_05668_b300 import workloads as W  # noqa: E402

F64 = torch.float64
GOLDEN = __file__.rsplit("/", 1)[0] + "/golden"


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")


def _table3():
    rows = [l.split() for l in open(f"{GOLDEN}/table3.txt") if l.strip() and not l.startswith("#")]
    return {(r[0], r[1]): (float(r[2]), float(r[3])) for r in rows}


def _paper_case(name):
    """(table, GPU system, oracle system, lattice name, scaling, f, tau_R, g_tau, gas)."""
    if name == "burgers":
        tab = syn.burgers_table()
        return tab, W.table_system(tab, (), (0.0,)), oracle.systems.Burgers(), 0.2, 0.2
    if name == "maxwell":
        tab = syn.maxwell_table()
        return tab, W.table_system(tab, (1.0,), (0.0, 0.0, 0.0)), oracle.systems.MaxwellTM(1.0), 0.2, 0.2
    tab = syn.euler_table()
    g = tab.gamma
    Q0 = (1.0, 3.0, 3.0, (1.0 / g) / (g - 1.0) + 9.0)
    return tab, W.table_system(tab, (g,), Q0), oracle.systems.Euler(g), 0.05, 0.2


def _run_gpu(tab, system, lattice, N, dim, scaling, f, steps, precision=lbx.FP64, tau_R=0.0, g_tau=0.0):
    sch = W.forced_scheme(tab, system, lattice, (N,) * dim, scaling, f, precision=precision,
                          tau_R=tau_R, g_tau=g_tau)
    xs = syn.coords((N,) * dim)
    st = lbx.State(sch, tab.augmented(xs, 0.0))
    st.step(steps)
    return st, sch, xs


# ------------------------------------------------------------------------------ parity

@pytest.mark.parametrize("name", ["burgers", "maxwell", "euler"])
def test_forced_paper_systems_fp64_match_oracle(name):
    N, steps = 40, 24
    tab, gsys, osys, f, tauR = _paper_case(name)
    st, sch, xs = _run_gpu(tab, gsys, lbx.D2Q5, N, 2, lbx.ACOUSTIC, f, steps, tau_R=tauR)
    dx, dt = oracle.lattice_steps(N, f, "acoustic")
    och = oracle.Scheme(osys, oracle.LATTICES["D2Q5"], (N, N), dx, dt, oracle.tau_vector(osys, dt, tau_R=tauR),
                        mms=make_mms(osys, tab.exact, xs, dt=dt))
    Qo = och.moments(och.run(och.init(tab.augmented(xs, 0.0)), steps))
    err = H.rel_linf_per_field(st.moments(), Qo)
    assert err.max() <= 1e-12, err


def test_forced_nsf_fp64_matches_oracle():
    N, steps = 24, 10
    case = syn.NsfCase(n=N)
    tab = syn.nsf_mms_table(case)
    st, sch, xs = _run_gpu(tab, W.nsf_system(case), lbx.D2Q9, N, 2, lbx.DIFFUSIVE, case.f, steps,
                           tau_R=case.tau_R, g_tau=case.g_tau)
    och = H.oracle_nsf(case)
    och.mms = make_mms(och.sys, tab.exact, xs, dt=case.dt)
    Qo = och.moments(och.run(och.init(tab.augmented(xs, 0.0)), steps))
    err = H.rel_linf_per_field(st.moments(), Qo)
    assert err.max() <= 1e-12, err


def test_forced_mhd_fp64_matches_oracle():
    N, steps = 10, 5
    case = syn.MhdCase(n=N)
    tab = syn.mhd_mms_table(case)
    st, sch, xs = _run_gpu(tab, W.mhd_system(case), lbx.D3Q19, N, 3, lbx.ACOUSTIC, case.f, steps,
                           tau_R=case.tau_R, g_tau=case.g_tau)
    och = H.oracle_mhd(case)
    och.mms = make_mms(och.sys, tab.exact, xs, dt=case.dt)
    Qo = och.moments(och.run(och.init(tab.augmented(xs, 0.0)), steps))
    err = H.rel_linf_per_field(st.moments(), Qo)
    assert err.max() <= 1e-12, err


def test_forced_runs_reject_bad_tables():
    tab = syn.burgers_table()
    gsys = W.table_system(tab, (), (0.0,))
    with pytest.raises(lbx.LbxError, match="primitive"):
        lbx.Scheme(gsys, lbx.D2Q5, (16, 16), lbx.ACOUSTIC, 0.2, tau_R=0.2, mms=lbx.MMS_FOURIER,
                   mms_modes=[(1, (1, 1), 0.1, 0.0, 0.0, 1.0, 0.0)], mms_mean=[0.0])
    with pytest.raises(lbx.LbxError, match="modes"):
        lbx.Scheme(gsys, lbx.D2Q5, (16, 16), lbx.ACOUSTIC, 0.2, tau_R=0.2, mms=lbx.MMS_FOURIER,
                   mms_modes=[], mms_mean=[0.0])


# ----------------------------------------------------------- the paper's Table 3 at N = 512

def _rel_l2(Qg, Qex, comps):
    """Relative L2 error of a field; a vector field (several components, e.g. rho u) takes the
    Euclidean norm of its components' relative errors, as the paper's Table 3 does."""
    errs = [float(torch.sqrt(((Qg[k] - Qex[k]) ** 2).sum() / (Qex[k] ** 2).sum())) for k in comps]
    return math.sqrt(sum(e * e for e in errs))


@pytest.mark.parametrize("name", ["burgers", "maxwell", "euler"])
def test_gpu_reproduces_paper_table3_at_512(name):
    tab, gsys, _, f, tauR = _paper_case(name)
    fields = {"burgers": {"u": [0]}, "maxwell": {"Ez": [0], "Hx": [1], "Hy": [2]},
              "euler": {"rho": [0], "rhou": [1, 2], "E": [3]}}[name]
    errs = {}
    for N in (256, 512):
        dt = f / N
        n = int(round(1.0 / dt))
        st, sch, xs = _run_gpu(tab, gsys, lbx.D2Q5, N, 2, lbx.ACOUSTIC, f, n, tau_R=tauR)
        Qex = tab.exact(*xs, torch.full_like(xs[0], n * dt))
        Qg = st.moments()
        errs[N] = {fld: _rel_l2(Qg, Qex, comps) for fld, comps in fields.items()}
    tab3 = _table3()
    for fld in fields:
        ref, ref_eoc = tab3[(name, fld)]
        p = math.log2(errs[256][fld] / errs[512][fld])
        print(f"{name} {fld}: N=512 rel-L2 {errs[512][fld]:.4e} (paper {ref:.4e}), order {p:.3f} (paper {ref_eoc})")
        assert abs(errs[512][fld] - ref) / ref < 0.05
        assert abs(p - ref_eoc) < 0.1


def test_gpu_reproduces_paper_table3_adr_with_forced_trackers():
    """Table 3, scalar ADR double (a tracker-carrying system): rel-L2 1.2680e-4 and rel-Linf
    2.2901e-4 at N = 512, t = 1, recipe diffusive f = 1.9, tau_R = 50, g_tau = 6.  The match
    holds when the manufactured residual forces every component of the augmented state (the
    paper's definition on Q+); forcing the conserved field alone gives 1.3406e-4."""
    N = 512
    c = syn.AdrPaperCase(n=N)
    tab = c.table()
    gsys = lbx.System(lbx.ADR_CASCADE, params=(c.a[0], c.a[1], c.D, c.R), Q0=(0.5, 0.0, 0.0))
    n = int(round(1.0 / c.dt))
    st, sch, xs = _run_gpu(tab, gsys, lbx.D2Q5, N, 2, lbx.DIFFUSIVE, c.f, n, tau_R=c.tau_R, g_tau=c.g_tau)
    l2, li = st.error_norms(tab.augmented(xs, n * c.dt))
    print(f"adr: N=512 rel-L2 {l2[0]:.4e} (paper 1.2680e-04), rel-Linf {li[0]:.4e} (paper 2.2901e-04)")
    assert abs(l2[0] - 1.2680e-4) / 1.2680e-4 < 5e-4
    assert abs(li[0] - 2.2901e-4) / 2.2901e-4 < 5e-4


def test_conserved_only_forcing_differs_from_the_full_residual():
    N, steps = 32, 40
    c = syn.AdrPaperCase(n=N)
    tab = c.table()
    gsys = lbx.System(lbx.ADR_CASCADE, params=(c.a[0], c.a[1], c.D, c.R), Q0=(0.5, 0.0, 0.0))
    xs = syn.coords((N, N))
    out = []
    for co in (False, True):
        sch = W.forced_scheme(tab, gsys, lbx.D2Q5, (N, N), lbx.DIFFUSIVE, c.f, tau_R=c.tau_R, g_tau=c.g_tau,
                              conserved_only=co)
        st = lbx.State(sch, tab.augmented(xs, 0.0))
        st.step(steps)
        out.append(st.moments())
        dx, dt = oracle.lattice_steps(N, c.f, "diffusive")
        osys = oracle.systems.AdrCascade(c.a, c.D, c.g_tau * dt, c.R)
        och = oracle.Scheme(osys, oracle.LATTICES["D2Q5"], (N, N), dx, dt,
                            oracle.tau_vector(osys, dt, tau_R=c.tau_R, g_tau=c.g_tau),
                            mms=make_mms(osys, tab.exact, xs, dt=dt, conserved_only=co))
        Qo = och.moments(och.run(och.init(tab.augmented(xs, 0.0)), steps))
        assert H.rel_linf_per_field(out[-1], Qo).max() <= 1e-12
    assert float((out[0][1:] - out[1][1:]).abs().max()) > 1e-6


# ------------------------------------------------- second order for the configs' systems

def _fluct_rel_l2(Qg, Qex, Q0, comps):
    """||Q_h - Q_ex|| / ||Q_ex - Q0|| over the listed components together."""
    e = sum(((Qg[k] - Qex[k]) ** 2).sum() for k in comps)
    r = sum(((Qex[k] - Q0[k]) ** 2).sum() for k in comps)
    return float(torch.sqrt(e / r))


@pytest.mark.parametrize("lattice,ns", [(lbx.D2Q5, (64, 128, 256)), (lbx.D2Q9, (128, 256, 512))])
def test_forced_nsf_paper_field_is_second_order(lattice, ns):
    """The paper's NSF manufactured flow (Mach 3 and 2, k = 2 pi) through the configuration's
    primitive-tracker NSF, recipe diffusive f = 2, tau_R = 60, g_tau = 6, to t = 0.25: the
    pairwise orders of the conserved fields rise to 2 (the paper's NSF: 1.95 to 2.01 for its
    own tracker set).  D2Q9 reaches the asymptotic range one doubling later than D2Q5."""
    T = 0.25
    errs = []
    for N in ns:
        case = syn.NsfPaperCase(n=N)
        tab = case.table()
        gsys = lbx.System(lbx.NSF_PRIM_TRACK, params=(case.gamma, case.R, case.mu, case.kappa),
                          Q0=case.reference_state())
        n = int(round(T / case.dt))
        st, sch, xs = _run_gpu(tab, gsys, lattice, N, 2, lbx.DIFFUSIVE, case.f, n, tau_R=case.tau_R,
                               g_tau=case.g_tau)
        Qex = tab.exact(*xs, torch.full_like(xs[0], n * case.dt))
        errs.append(_fluct_rel_l2(st.moments(), Qex, case.reference_state(), [0, 1, 2, 3]))
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    print("NSF paper field", lattice, "errors", errs, "orders", orders)
    assert orders[0] > 1.6 and 1.85 < orders[1] < 2.3, orders


def test_forced_mhd_paper_field_d3q19_is_second_order():
    """The paper's MHD manufactured flow (Mach 3, B0 = (0.5, 0.5, 0), k = 2 pi, uniform in z)
    through the configuration's 3D current-tracker MHD on D3Q19, recipe acoustic f = 0.05,
    tau_R = 160, g_tau = 4, eta = 0.01, to t = 0.25 at N = 32, 64, 128."""
    T = 0.25
    errs = []
    for N in (32, 64, 128):
        case = syn.MhdPaperCase(n=N)
        tab = case.table()
        gsys = lbx.System(lbx.MHD_J_TRACK, params=(case.gamma, case.eta), Q0=case.reference_state())
        n = int(round(T / case.dt))
        st, sch, xs = _run_gpu(tab, gsys, lbx.D3Q19, N, 3, lbx.ACOUSTIC, case.f, n, tau_R=case.tau_R,
                               g_tau=case.g_tau)
        Qex = tab.exact(*xs, torch.full_like(xs[0], n * case.dt))
        errs.append(_fluct_rel_l2(st.moments(), Qex, case.reference_state(), list(range(8))))
        del st
        torch.cuda.empty_cache()
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    print("MHD paper field errors", errs, "orders", orders)
    assert all(1.7 < o < 2.3 for o in orders), orders
