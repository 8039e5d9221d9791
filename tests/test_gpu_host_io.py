"""Host fields in and host moments out: lbx_init and lbx_moments with host arrays give the
same populations and moments as the device-side calls, bitwise.

Page-locked host arrays are read (init) and written (moments) by the kernels directly over
the bus.  Pageable ones are copied in chunks of planes of the last axis on the state's
second stream: lbx_init runs the equilibrium of each chunk as it arrives, lbx_moments
copies each chunk back while the next one's moments are computed.  Every node does the same
arithmetic either way.  Covered: 2D (chunks of rows) and 3D (chunks
of z-planes), fewer planes than chunks, pinned and pageable host memory, and FP16 storage
with derived scales (the whole-field path, which needs every field before the scales).
"""
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


def _cases():
    nsf = syn.NsfCase(n=48)
    mhd = syn.MhdCase(n=16)
    return {
        "nsf_fp32": (lambda: W.nsf_scheme(nsf, lbx.FP32_SHIFT), lambda: syn.nsf_fields(nsf)),
        "nsf_fp64_5rows": (lambda: W.nsf_scheme(nsf, lbx.FP64, extent=(48, 5), slab_origin=0,
                                                slab_planes_global=48),
                           lambda: syn.nsf_fields(nsf).narrow(1, 0, 5).contiguous()),
        "nsf_fp16": (lambda: W.nsf_scheme(nsf, lbx.FP16_SCALED), lambda: syn.nsf_fields(nsf)),
        "mhd_fp64": (lambda: W.mhd_scheme(mhd, lbx.FP64), lambda: syn.mhd_fields(mhd)),
    }


@pytest.mark.parametrize("name", ["nsf_fp32", "nsf_fp64_5rows", "nsf_fp16", "mhd_fp64"])
@pytest.mark.parametrize("pinned", [True, False])
def test_host_fields_and_host_moments_equal_the_device_path(name, pinned):
    make, fields = _cases()[name]
    Q = fields().to(torch.float64).contiguous()
    Qh = Q.pin_memory() if pinned else Q
    dev = lbx.State(make(), Q.cuda())
    host = lbx.State(make(), Qh)
    assert torch.equal(host.get_populations(), dev.get_populations())
    dev.step(3)
    host.step(3)
    out = torch.empty(Q.shape, dtype=torch.float64, pin_memory=pinned)
    host.moments_into(out)
    ref = dev.moments_into(torch.empty(Q.shape, dtype=torch.float64, device="cuda")).cpu()
    assert torch.equal(out, ref)
