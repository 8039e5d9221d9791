"""Slabs of one grid on one GPU: the face exchange reproduces the whole grid bitwise.

A periodic grid cut into 2 or 4 slabs along its last axis (y in 2D, z in 3D), each slab
an lbx state stepping with its own periodic wrap and exchanging the populations that cross
its faces after every step (lbx_halo_pack, device copies between the slabs,
lbx_halo_unpack, paper_2607_05668_b300.slab.step_local), must give the whole grid's
populations and moments bitwise: every node does the same arithmetic on the same inputs.
Covered: FP64, shifted FP32 and scaled FP16 (the slabs share the whole grid's scales),
NSF on D2Q9 (3 of 9 velocities cross a face), 3D MHD on D3Q19 (5 of 19, odd K), the
homogenized NSF on D3Q7 with its moving porosity (node coordinates offset by the slab
origin), and a manufactured-forced run (forcing evaluated at global coordinates); uneven
slab sizes, and a single slab exchanging with itself.
"""
import pytest
import torch

import synthetic as syn
from tests import helpers as H

pytestmark = pytest.mark.gpu

lbx = pytest.importorskip("paper_2607_05668_b300.lbx")
from paper_2607_05668_b300 import slab as SL, workloads as W  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")


def _slabs(make_scheme, Q, planes, nslabs, scales=None):
    """Slabs of the grid: make_scheme(extent_of_slab_axis, origin, fp16_scales) -> Scheme."""
    out = []
    for s in range(nslabs):
        o, c = SL.slab_bounds(planes, nslabs, s)
        out.append(SL.Slab(make_scheme(c, o, scales), SL.slab_of(Q, o, c)))
    return out


def _compare(whole, slabs, steps, planes, stepper=None):
    whole.step(steps)
    (stepper or SL.step_local)(slabs, steps)
    Qw = whole.moments()
    Qs = torch.cat([s.state.moments() for s in slabs], dim=1)
    assert torch.equal(Qs, Qw)
    fw = whole.get_populations()
    fs = torch.cat([s.state.get_populations() for s in slabs], dim=2)
    assert torch.equal(fs, fw)
    # conserved sums add over the slabs (FP64; the order of addition differs)
    tot = sum(s.state.conserved_sums() for s in slabs)
    ref = whole.conserved_sums()
    assert abs(tot - ref).max() <= 1e-12 * (abs(ref).max() + 1.0)
    # error norms from the slabs' raw statistics equal the whole grid's
    l2, li = SL.combine_error_stats(sum_stats([s.state.error_stats(SL.slab_of(Qw, *bounds(slabs, i)))
                                               for i, s in enumerate(slabs)]))
    assert l2.max() == 0.0 and li.max() == 0.0


def bounds(slabs, i):
    return slabs[i].scheme.slab_origin, slabs[i].scheme.grid[0]


def sum_stats(stats):
    import numpy as np
    st = np.stack(stats)
    return np.concatenate([st[:, :, :2].sum(0), st[:, :, 2:].max(0)], axis=1)


@pytest.mark.parametrize("precision", [lbx.FP64, lbx.FP32_SHIFT, lbx.FP16_SCALED])
@pytest.mark.parametrize("nslabs", [1, 2, 4])
def test_nsf_d2q9_slabs_equal_the_whole_grid(precision, nslabs):
    case = syn.NsfCase(n=48)
    Q = syn.nsf_fields(case)
    whole = lbx.State(W.nsf_scheme(case, precision), Q)
    scales = list(whole.scales()) if precision == lbx.FP16_SCALED else None

    def make(c, o, sc):
        return lbx.Scheme(W.nsf_system(case), lbx.D2Q9, (case.n, c), lbx.DIFFUSIVE, case.f, tau_R=case.tau_R,
                          g_tau=case.g_tau, precision=precision, slab_origin=o, slab_planes_global=case.n,
                          fp16_scales=sc)
    _compare(whole, _slabs(make, Q, case.n, nslabs, scales), 12, case.n)


@pytest.mark.parametrize("precision", [lbx.FP64, lbx.FP32_SHIFT, lbx.FP16_SCALED])
def test_mhd_d3q19_slabs_equal_the_whole_grid(precision):
    case = syn.MhdCase(n=16)
    Q = syn.mhd_fields(case)
    whole = lbx.State(W.mhd_scheme(case, precision), Q)
    whole.set_staging(lbx.STAGE_BULK)
    scales = list(whole.scales()) if precision == lbx.FP16_SCALED else None

    def make(c, o, sc):
        return lbx.Scheme(W.mhd_system(case), lbx.D3Q19, (case.n, case.n, c), lbx.ACOUSTIC, case.f,
                          tau_R=case.tau_R, g_tau=case.g_tau, precision=precision, slab_origin=o,
                          slab_planes_global=case.n, fp16_scales=sc)
    slabs = _slabs(make, Q, case.n, 3, scales)          # 6, 5, 5 planes
    for s in slabs:
        s.state.set_staging(lbx.STAGE_BULK)
    _compare(whole, slabs, 6, case.n)


@pytest.mark.parametrize("forced", [False, True])
def test_hcnsf_slabs_with_offset_coordinates_equal_the_whole_grid(forced):
    hc = syn.HcnsfPaperCase(n=16)
    Q = hc.table().augmented(syn.coords((16, 16, 16)), 0.0)
    whole = lbx.State(W.hcnsf_scheme(hc, lbx.FP64, forced=forced), Q)

    def make(c, o, sc):
        return W.hcnsf_scheme(hc, lbx.FP64, forced=forced, extent=(16, 16, c), slab_origin=o,
                              slab_planes_global=16)
    _compare(whole, _slabs(make, Q, 16, 2), 4, 16)


def test_forced_nsf_slabs_equal_the_whole_grid():
    N, steps = 24, 6
    case = syn.NsfCase(n=N)
    tab = syn.nsf_mms_table(case)
    xs = syn.coords((N, N))
    Q = tab.augmented(xs, 0.0)

    def sch(ext, **kw):
        return lbx.Scheme(W.nsf_system(case), lbx.D2Q9, ext, lbx.DIFFUSIVE, case.f, tau_R=case.tau_R,
                          g_tau=case.g_tau, mms=lbx.MMS_FOURIER, mms_modes=tab.lbx_modes(), mms_mean=list(tab.mean),
                          **kw)
    whole = lbx.State(sch((N, N)), Q)
    slabs = _slabs(lambda c, o, s: sch((N, c), slab_origin=o, slab_planes_global=N), Q, N, 2)
    _compare(whole, slabs, steps, N)
    och = H.oracle_nsf(case)
    from oracle.mms import make_mms
    och.mms = make_mms(och.sys, tab.exact, xs, dt=case.dt)
    Qo = och.moments(och.run(och.init(Q), steps))
    Qs = torch.cat([s.state.moments() for s in slabs], dim=1)
    assert H.rel_linf_per_field(Qs, Qo).max() <= 1e-12


# ------------------------------------------- the exchange hidden behind the interior planes
def test_step_pieces_equal_one_step():
    """lbx_step_planes over a split of the planes, then lbx_step_commit, is bitwise one
    lbx_step: register-resident FP32, bulk-staged FP16 3D, and the homogenized NSF with
    time-dependent fields (the device step counter advances at the commit)."""
    nsf, mhd, hc = syn.NsfCase(n=40), syn.MhdCase(n=16), syn.HcnsfPaperCase(n=16)
    hq = hc.table().augmented(syn.coords((16, 16, 16)), 0.0)
    cases = [(lambda: W.nsf_scheme(nsf, lbx.FP32_SHIFT), syn.nsf_fields(nsf), (0, 1, 17, 40)),
             (lambda: W.mhd_scheme(mhd, lbx.FP16_SCALED), syn.mhd_fields(mhd), (0, 5, 16)),
             (lambda: W.hcnsf_scheme(hc, lbx.FP64), hq, (0, 1, 15, 16))]
    for make, Q, cuts in cases:
        ref, st = lbx.State(make(), Q), lbx.State(make(), Q)
        ref.step(3)
        for _ in range(3):
            for a, b in zip(cuts[:-1], cuts[1:]):
                st.step_planes(a, b - a)
            st.step_commit()
        assert st.time == ref.time
        assert torch.equal(st.get_populations(), ref.get_populations())


def test_step_planes_refuses_bad_ranges_and_the_persistent_kernel():
    case = syn.MhdCase(n=8)
    st = lbx.State(W.mhd_scheme(case, lbx.FP32_SHIFT), syn.mhd_fields(case))
    for a, n in ((-1, 2), (0, 9), (7, 2)):
        with pytest.raises(lbx.LbxError, match="ERR_ARG"):
            st.step_planes(a, n)
    st.set_staging(lbx.STAGE_PIPE)
    with pytest.raises(lbx.LbxError, match="ERR_UNSUPPORTED"):
        st.step_planes(0, 1)


@pytest.mark.parametrize("nslabs", [1, 3])
def test_overlapped_exchange_slabs_equal_the_whole_grid(nslabs):
    """step_local_overlap: boundary planes, face exchange and unpack on a second stream while
    the interior planes step; NSF D2Q9 in FP16 (shared scales) and MHD D3Q19 in FP32 (bulk
    row copies), 1 and 3 slabs, bitwise equal to the whole grid."""
    case = syn.NsfCase(n=48)
    Q = syn.nsf_fields(case)
    whole = lbx.State(W.nsf_scheme(case, lbx.FP16_SCALED), Q)
    scales = list(whole.scales())

    def make(c, o, sc):
        return W.nsf_scheme(case, lbx.FP16_SCALED, extent=(case.n, c), slab_origin=o, slab_planes_global=case.n,
                            fp16_scales=sc)
    _compare(whole, _slabs(make, Q, case.n, nslabs, scales), 12, case.n, SL.step_local_overlap)

    m = syn.MhdCase(n=16)
    Qm = syn.mhd_fields(m)
    wm = lbx.State(W.mhd_scheme(m, lbx.FP32_SHIFT), Qm)
    slabs = _slabs(lambda c, o, sc: W.mhd_scheme(m, lbx.FP32_SHIFT, extent=(16, 16, c), slab_origin=o,
                                                 slab_planes_global=16), Qm, 16, nslabs)
    for s in slabs:
        s.state.set_staging(lbx.STAGE_BULK)
    _compare(wm, slabs, 6, 16, SL.step_local_overlap)


def test_overlapped_exchange_with_time_dependent_fields():
    """The homogenized NSF's moving porosity reads the device step counter: the pieces of a
    step and the commit keep it in order across the two streams."""
    hc = syn.HcnsfPaperCase(n=16)
    Q = hc.table().augmented(syn.coords((16, 16, 16)), 0.0)
    whole = lbx.State(W.hcnsf_scheme(hc, lbx.FP64, forced=True), Q)

    def make(c, o, sc):
        return W.hcnsf_scheme(hc, lbx.FP64, forced=True, extent=(16, 16, c), slab_origin=o, slab_planes_global=16)
    _compare(whole, _slabs(make, Q, 16, 2), 5, 16, SL.step_local_overlap)

