"""The bounded device-side wait of the bulk-staged step kernels.

A block of k_step_bulk (and of the in-place bulk kernels) waits on an mbarrier for the row
copies it issued, for at most the state's wait limit of global-timer time.  A limit of zero
makes every block give up before its first try while its copies complete normally: nothing
faults, each block raises the state's device error word, waits once more for its copies and
leaves its nodes unwritten.  lbx_synchronize must then report LBX_ERR_TIMEOUT (once: the word
is cleared), and after the populations are restored the default limit must give results
bitwise equal to an undisturbed run, which itself matches the CPU FP64 oracle.
"""
import pytest
import torch

import synthetic as syn
from tests import helpers as H

pytestmark = pytest.mark.gpu

lbx = pytest.importorskip("paper_2607_05668_b300.lbx")
from paper_2607_05668_b300 import workloads as W  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")


@pytest.mark.parametrize("streaming", [lbx.STREAM_TWO_BUFFERS, lbx.STREAM_IN_PLACE])
def test_zero_wait_limit_times_out_and_the_state_recovers(streaming):
    case = syn.MhdCase(n=16)                    # D3Q19, 11 components: staged, nx % 8 == 0
    Q = syn.mhd_fields(case)
    sch = W.mhd_scheme(case, lbx.FP64, streaming=streaming)
    steps = 4

    ref = lbx.State(sch, Q)
    ref.set_staging(lbx.STAGE_BULK)
    ref.step(steps)
    ref.synchronize()

    st = lbx.State(sch, Q)
    st.set_staging(lbx.STAGE_BULK)
    f0 = st.get_populations()
    st.set_wait_limit(0)
    st.step(2)                                  # in place: one pair, both kinds time out
    with pytest.raises(lbx.LbxError) as err:
        st.synchronize()
    assert err.value.name == "ERR_TIMEOUT"
    st.synchronize()                            # reported once, then cleared

    st.set_wait_limit(10 ** 9)
    st.set_populations(f0)                      # the unforced system does not read the time
    st.step(steps)
    st.synchronize()
    assert torch.equal(st.get_populations(), ref.get_populations())

    och = H.oracle_mhd(case)
    Qo = och.moments(och.run(och.init(Q), steps))
    assert H.rel_linf_per_field(st.moments(), Qo).max() <= 1e-12
