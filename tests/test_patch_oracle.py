"""The sampled-node oracle of the full-size parity tests (tests/helpers.patch_moments): a
node's value after n steps computed on a small periodic patch around it equals the full
domain's: bitwise, also where the patch wraps around the domain edge; to rounding under
prescribed coefficient fields, whose patch coordinates carry their offset."""
import torch

import oracle
import synthetic as syn
from oracle import systems as S
from tests import helpers as H


def test_patches_reproduce_the_full_domain_nsf():
    case = syn.NsfCase(n=24)
    full = H.oracle_nsf(case)
    Q = syn.nsf_fields(case)
    ref = full.moments(full.run(full.init(Q), 3))
    centers = [(0, 0), (23, 5), (11, 23), (7, 12)]

    def make(shape, origin):
        s = H.oracle_nsf(case)
        return oracle.Scheme(s.sys, s.lat, shape, case.dx, case.dt, s.tau)
    got = H.patch_moments(make, Q, centers, 3, 4)
    want = torch.stack([ref[:, y, x] for (y, x) in centers], dim=1)
    assert torch.equal(got, want)


def test_patches_reproduce_the_full_domain_hcnsf():
    case = syn.HcnsfPaperCase(n=12)
    shape = (12, 12, 12)
    sysm = S.HomogenizedNsf3D(case.gamma, case.mu, case.kappa, case.eta, case.g_tau * case.dt, fields=case.prescribed)
    tau = oracle.tau_vector(sysm, case.dt, tau_R=case.tau_R, g_tau=case.g_tau)
    lat = oracle.LATTICES["D3Q7"]
    Q = case.table().augmented(syn.coords(shape), 0.0)
    full = oracle.Scheme(sysm, lat, shape, case.dx, case.dt, tau, source_theta=case.theta)
    ref = full.moments(full.run(full.init(Q), 2))
    centers = [(0, 0, 0), (11, 3, 7), (5, 11, 0), (6, 6, 6)]

    def make(pshape, origin):
        return oracle.Scheme(sysm, lat, pshape, case.dx, case.dt, tau, source_theta=case.theta, origin=origin)
    got = H.patch_moments(make, Q, centers, 2, 3)
    want = torch.stack([ref[:, z, y, x] for (z, y, x) in centers], dim=1)
    # a wrapped patch node sits at x - 1 instead of x (the same fields up to the rounding
    # of their trigonometry), so agreement is to rounding rather than bitwise
    torch.testing.assert_close(got, want, rtol=1e-13, atol=1e-13)
