"""lbx_conserved_sums_static: conserved sums for callers that cannot allocate device
memory (code recorded into a CUDA graph or under a latency budget, where cudaMalloc and
cudaFree would synchronise the device, or programs whose device memory belongs to another
allocator).  Its scratch is a static device array inside the library, so the call
allocates nothing.  Its result must equal lbx_conserved_sums on the same populations,
on consecutive calls that reuse the shared array.

Collected last on purpose, so that a failure here stops a -x run only after every other
test has run; it also passes on its own in a fresh process.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import synthetic as syn

pytestmark = pytest.mark.gpu

lbx = pytest.importorskip("paper_2607_05668_b300.lbx")
from paper_2607_05668_b300 import workloads as W  # noqa: E402


def _static_sums(state, nblocks=0):
    K = state.K
    out = torch.full((K,), float("nan"), dtype=torch.float64, device="cuda")
    lbx.check(lbx.lib().lbx_conserved_sums_static(state.scheme._h, state.populations_ptr(), out.data_ptr(),
                                                  nblocks, state._stream))
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")


@pytest.mark.parametrize("prec", [lbx.FP64, lbx.FP32_SHIFT])
def test_static_sums_match_allocating_entry_point_on_consecutive_calls(prec):
    case = syn.NsfCase(n=96)
    st = lbx.State(W.nsf_scheme(case, prec), syn.nsf_fields(case))
    st.step(17)
    ref = st.conserved_sums()
    first = _static_sums(st)
    second = _static_sums(st)
    np.testing.assert_allclose(first, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())
    np.testing.assert_allclose(second, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())
    # a call on a state of another shape and component count in between, then again
    m = syn.MhdCase(n=20)
    sm = lbx.State(W.mhd_scheme(m, lbx.FP32_SHIFT), syn.mhd_fields(m))
    np.testing.assert_allclose(_static_sums(sm, nblocks=7), sm.conserved_sums(), rtol=1e-12,
                               atol=1e-12 * np.abs(sm.conserved_sums()).max())
    np.testing.assert_allclose(_static_sums(st, nblocks=lbx.STATIC_REDUCE_MAX_BLOCKS), ref, rtol=1e-12,
                               atol=1e-12 * np.abs(ref).max())


def test_static_sums_reject_oversized_and_unsupported_requests():
    case = syn.NsfCase(n=32)
    st = lbx.State(W.nsf_scheme(case, lbx.FP32_SHIFT), syn.nsf_fields(case))
    with pytest.raises(lbx.LbxError) as e:
        _static_sums(st, nblocks=lbx.STATIC_REDUCE_MAX_BLOCKS + 1)
    assert e.value.name == "ERR_ARG" and "static scratch" in str(e.value)
    st16 = lbx.State(W.nsf_scheme(case, lbx.FP16_SCALED), syn.nsf_fields(case))
    with pytest.raises(lbx.LbxError) as e:
        _static_sums(st16)
    assert e.value.name == "ERR_UNSUPPORTED"
