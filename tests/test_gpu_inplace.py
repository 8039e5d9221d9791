"""Single-buffer in-place streaming (LBX_STREAM_IN_PLACE) against the two-buffer pull
kernels: after every even number of steps the populations must be bitwise identical (the
two step kinds move populations exactly as two pull steps, with the same arithmetic), for
register-resident and staged systems, odd and even component counts, forced and unforced
runs, and all three storage precisions."""
import pytest
import torch

import synthetic as syn

pytestmark = pytest.mark.gpu

lbx = pytest.importorskip("paper_2607_05668_b300.lbx")
from paper_2607_05668_b300 import workloads as W  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")


def _nsf(prec, streaming, forced=False):
    case = syn.NsfCase(n=40)
    if forced:
        tab = syn.nsf_mms_table(case)
        sys_ = lbx.System(lbx.NSF_PRIM_TRACK, params=(case.gamma, case.R, case.mu, case.kappa),
                          Q0=case.reference_state())
        sch = lbx.Scheme(sys_, lbx.D2Q9, (40, 40), lbx.DIFFUSIVE, case.f, tau_R=case.tau_R, g_tau=case.g_tau,
                         precision=prec, mms=lbx.MMS_FOURIER, mms_modes=tab.lbx_modes(), mms_mean=list(tab.mean),
                         streaming=streaming)
        return sch, tab.augmented(syn.coords((40, 40)), 0.0)
    sys_ = lbx.System(lbx.NSF_PRIM_TRACK, params=(case.gamma, case.R, case.mu, case.kappa), Q0=case.reference_state())
    sch = lbx.Scheme(sys_, lbx.D2Q9, (40, 40), lbx.DIFFUSIVE, case.f, tau_R=case.tau_R, g_tau=case.g_tau,
                     precision=prec, streaming=streaming)
    return sch, syn.nsf_fields(case)


def _mhd(prec, streaming, forced=False):
    case = syn.MhdCase(n=20)
    sys_ = lbx.System(lbx.MHD_J_TRACK, params=(case.gamma, case.eta), Q0=case.reference_state())
    sch = lbx.Scheme(sys_, lbx.D3Q19, (20, 20, 20), lbx.ACOUSTIC, case.f, tau_R=case.tau_R, g_tau=case.g_tau,
                     precision=prec, streaming=streaming)
    return sch, syn.mhd_fields(case)


def _hcnsf(prec, streaming, forced=False):
    case = syn.HcnsfPaperCase(n=16)
    kind, pf = W.hcnsf_prescribed(case)
    kw = dict(tau_R=case.tau_R, g_tau=case.g_tau, precision=prec, prescribed=kind, prescribed_params=pf,
              streaming=streaming)
    tab = case.table()
    if forced:
        kw.update(mms=lbx.MMS_FOURIER, mms_modes=tab.lbx_modes(), mms_mean=list(tab.mean))
    sch = lbx.Scheme(W.hcnsf_system(case), lbx.D3Q7, (16, 16, 16), lbx.ACOUSTIC, case.f, **kw)
    return sch, tab.augmented(syn.coords((16, 16, 16)), 0.0)


CASES = {"nsf": _nsf, "mhd": _mhd, "hcnsf": _hcnsf}


@pytest.mark.parametrize("forced", [False, True])
@pytest.mark.parametrize("prec", [lbx.FP64, lbx.FP32_SHIFT, lbx.FP16_SCALED])
@pytest.mark.parametrize("name", ["nsf", "mhd", "hcnsf"])
def test_inplace_equals_two_buffers_bitwise(name, prec, forced):
    """NSF D2Q9 (K = 10, register-resident in FP32/FP16), MHD D3Q19 (K = 11: an odd
    component, staged), HCNSF D3Q7 (K = 14, staged, prescribed fields)."""
    if forced and name == "mhd":
        pytest.skip("the MHD case here is unforced")
    sa, Q = CASES[name](prec, lbx.STREAM_TWO_BUFFERS, forced)
    sb, _ = CASES[name](prec, lbx.STREAM_IN_PLACE, forced)
    a, b = lbx.State(sa, Q), lbx.State(sb, Q)
    for n in (2, 4):
        a.step(n)
        b.step(n)
        assert torch.equal(a.get_populations(), b.get_populations())
        assert torch.equal(a.moments(), b.moments())
    a.step(1)
    b.step(1)
    with pytest.raises(lbx.LbxError):          # the pair's intermediate layout
        b.moments()
    a.step(1)
    b.step(1)
    assert torch.equal(a.moments(), b.moments())


def test_inplace_state_allocates_one_buffer():
    case = syn.MhdCase(n=128)
    sys_ = lbx.System(lbx.MHD_J_TRACK, params=(case.gamma, case.eta), Q0=case.reference_state())
    Q = syn.mhd_fields(case)
    used = []
    for streaming in (lbx.STREAM_TWO_BUFFERS, lbx.STREAM_IN_PLACE):
        sch = lbx.Scheme(sys_, lbx.D3Q19, (128, 128, 128), lbx.ACOUSTIC, case.f, tau_R=case.tau_R,
                         g_tau=case.g_tau, precision=lbx.FP32_SHIFT, streaming=streaming)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        st = lbx.State(sch, Q)
        torch.cuda.synchronize()
        used.append(free0 - torch.cuda.mem_get_info()[0])
        st.close()
        del st
    buf = sch.buffer_bytes
    assert abs(used[0] - used[1] - buf) < 0.05 * buf, (used, buf)


def test_inplace_graph_replay_and_checkpoint(tmp_path):
    sa, Q = _nsf(lbx.FP32_SHIFT, lbx.STREAM_TWO_BUFFERS)
    sb, _ = _nsf(lbx.FP32_SHIFT, lbx.STREAM_IN_PLACE)
    s = torch.cuda.Stream()
    a, b = lbx.State(sa, Q, stream=s), lbx.State(sb, Q, stream=s)
    b.use_graph(True)
    for _ in range(3):
        a.step(3)
        b.step(3)          # alternates the pair's phase between replays
    a.step(1)
    b.step(1)
    assert torch.equal(a.moments(), b.moments())
    path = str(tmp_path / "ip.ckpt")
    b.save(path)
    c = lbx.State(sa, Q)
    c.load(path)
    a.step(2)
    c.step(2)
    assert torch.equal(a.moments(), c.moments())


@pytest.mark.parametrize("prec", [lbx.FP32_SHIFT, lbx.FP16_SCALED, lbx.FP64])
def test_inplace_bulk_and_thread_staging_equal_two_buffers(prec):
    """MHD D3Q19 at 24^3 (nx % 8 == 0): in-place kinds with bulk row copies (blocks of 32, 64
    and 128) and with per-thread copies equal the two-buffer pull bitwise."""
    case = syn.MhdCase(n=24)
    sys_ = lbx.System(lbx.MHD_J_TRACK, params=(case.gamma, case.eta), Q0=case.reference_state())
    Q = syn.mhd_fields(case)

    def make(streaming):
        return lbx.Scheme(sys_, lbx.D3Q19, (24, 24, 24), lbx.ACOUSTIC, case.f, tau_R=case.tau_R, g_tau=case.g_tau,
                          precision=prec, streaming=streaming)
    ref = lbx.State(make(lbx.STREAM_TWO_BUFFERS), Q)
    ref.step(6)
    want = ref.get_populations()
    for staging, block in ((lbx.STAGE_BULK, 32), (lbx.STAGE_BULK, 64), (lbx.STAGE_BULK, 128), (lbx.STAGE_THREAD, 128)):
        st = lbx.State(make(lbx.STREAM_IN_PLACE), Q)
        st.set_staging(staging)
        st.set_block(block)
        st.step(6)
        assert torch.equal(st.get_populations(), want), (staging, block)
