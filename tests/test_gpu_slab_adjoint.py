"""The adjoint over slabs on one GPU equals the whole grid's adjoint.

A periodic grid cut into slabs along its last axis runs the gradient of
J = 1/2 sum_x (rho(x, T) - rho*(x))^2 slab by slab (paper_2607_05668_b300.slab.slab_adjoint:
lbx_adjoint_checkpoint / _restore / _seed / _step / _finish).  The reverse step of Eq.
lbe_update pushes along -c_i, so after the seed and after every reverse step the adjoint
faces travel opposite to the forward exchange, and before the initial VJP (a pull) they
travel forward.  Every node does the same arithmetic on the same inputs as lbx_adjoint on
the whole grid, so dJ/dQ_init is bitwise equal; J and dJ/dtau are sums over the nodes whose
order differs.  Covered: FP64 and shifted FP32 on D2Q9 (3 of 9 velocities cross a face),
uneven slabs, a single slab exchanging with itself, 3D MHD on D3Q19 (5 of 19, odd K), and
segments of uneven length.
"""
import pytest
import torch

import synthetic as syn

pytestmark = pytest.mark.gpu

lbx = pytest.importorskip("paper_2607_05668_b300.lbx")
from paper_2607_05668_b300 import slab as SL, workloads as W  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")


def _run(make, Q, tgt, planes, nslabs, steps, ckpt):
    """Whole-grid lbx_adjoint and the slab sweep; dJ/dQ_init of the slabs reassembled."""
    K = Q.shape[0]
    J, g, gt = lbx.adjoint(make(planes, 0, 0), Q, steps, ckpt, tgt)
    slabs, qs, ts = [], [], []
    for s in range(nslabs):
        o, c = SL.slab_bounds(planes, nslabs, s)
        Qs = SL.slab_of(Q, o, c)
        slabs.append(SL.Slab(make(c, o, planes), Qs))
        qs.append(Qs.reshape(K, -1).to("cuda", torch.float64).contiguous())
        ts.append(tgt.narrow(0, o, c).reshape(-1).to("cuda", torch.float64).contiguous())
    Js, gs, gts = SL.slab_adjoint(slabs, qs, ts, steps, ckpt)
    shape = lambda s: (K,) + s.scheme.grid                                      # noqa: E731
    g_slabs = torch.cat([gg.reshape(shape(s)).cpu() for gg, s in zip(gs, slabs)], dim=1)
    for s in slabs:
        s.close()
    return (J, g, gt), (Js, g_slabs, gts)


def _check(whole, slab):
    (J, g, gt), (Js, gs, gts) = whole, slab
    assert torch.equal(gs, g)
    assert abs(Js - J) <= 1e-13 * abs(J)
    assert abs(gts - gt) <= 1e-11 * abs(gt)


@pytest.mark.parametrize("precision,nslabs", [(lbx.FP64, 2), (lbx.FP64, 1), (lbx.FP32_SHIFT, 3)])
def test_nsf_d2q9_slab_adjoint_equals_the_whole_grid(precision, nslabs):
    N, steps, ckpt = 26, 11, 4                   # 3 slabs: 9, 9, 8 rows; segments 4, 4, 3
    case = syn.NsfCase(n=N)
    Q, tgt = syn.nsf_fields(case), syn.density_target(N)

    def make(c, o, planes):
        slab = {} if planes == 0 else {"slab_origin": o, "slab_planes_global": planes}
        return W.nsf_scheme(case, precision, tau_lb=0.52, extent=(N, c if planes else N), **slab)
    _check(*_run(make, Q, tgt, N, nslabs, steps, ckpt))


def test_mhd_d3q19_slab_adjoint_equals_the_whole_grid():
    N, steps, ckpt = 12, 7, 3
    case = syn.MhdCase(n=N)
    Q, tgt = syn.mhd_fields(case), syn.density_target(N, dim=3)

    def make(c, o, planes):
        slab = {} if planes == 0 else {"slab_origin": o, "slab_planes_global": planes}
        return W.mhd_scheme(case, lbx.FP64, extent=(N, N, c if planes else N), **slab)
    _check(*_run(make, Q, tgt, N, 2, steps, ckpt))


def test_whole_grid_adjoint_refuses_slab_schemes():
    case = syn.NsfCase(n=16)
    sch = W.nsf_scheme(case, lbx.FP64, extent=(16, 8), slab_origin=0, slab_planes_global=16)
    with pytest.raises(lbx.LbxError, match="step-wise"):
        lbx.adjoint(sch, syn.nsf_fields(case).narrow(1, 0, 8), 2, 1, syn.density_target(16)[:8])
