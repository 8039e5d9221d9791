"""The manufactured-solution inputs (synthetic.ModeTable) against closed forms.

The mode tables write the paper's product-form fields (supplement, MMS section) as sums of
sine modes; these tests evaluate both forms and the analytic tracker fields against
forward-mode differentiation (the oracle's exact_augmented), so a wrong sign, phase or
wavenumber in a table fails here and not only on the GPU."""
import math

import pytest
import torch

import oracle
import synthetic as syn
from oracle.mms import exact_augmented

TWO_PI = 2.0 * math.pi


@pytest.fixture(scope="module")
def grid():
    xs = syn.coords((20, 20))
    return xs, torch.full_like(xs[0], 0.37)


def test_burgers_and_maxwell_tables_equal_the_paper_fields(grid):
    xs, t = grid
    torch.testing.assert_close(syn.burgers_table().exact(*xs, t)[0], syn.burgers_exact(*xs, t), rtol=0, atol=4e-15)
    torch.testing.assert_close(syn.maxwell_table().exact(*xs, t), syn.maxwell_exact(*xs, t), rtol=0, atol=4e-15)


def _paper_products(xs, t, a_rho, a_u, a_v, v_time_cos, p0, u0, v0):
    kx, ky = TWO_PI * xs[0], TWO_PI * xs[1]
    drho = a_rho * torch.sin(kx) * torch.cos(ky) * torch.cos(t)
    u = u0 + a_u * torch.cos(kx) * torch.sin(ky) * torch.sin(t)
    v = v0 + a_v * torch.sin(kx) * torch.sin(ky) * (torch.cos(t) if v_time_cos else torch.sin(t))
    p = p0 + drho + 0.2 * p0 * torch.cos(kx) * torch.sin(ky) * torch.sin(t)
    return [1.0 + drho, u, v, p]


def test_euler_table_equals_the_paper_field(grid):
    xs, t = grid
    want = _paper_products(xs, t, 0.3, 0.3, 0.3, False, 1 / 1.4, 3.0, 3.0)
    for a, b in zip(syn.euler_table().primitives(xs, t), want):
        torch.testing.assert_close(a, b, rtol=0, atol=4e-15)


def test_nsf_paper_table_equals_the_paper_field(grid):
    xs, t = grid
    case = syn.NsfPaperCase(n=20)
    want = _paper_products(xs, t, 0.2, 0.2, 0.15, True, 1 / 1.4, 3.0, 2.0)
    for a, b in zip(case.table().primitives(xs, t), want):
        torch.testing.assert_close(a, b, rtol=0, atol=4e-15)
    # nondimensional constants: c_s^2 = gamma R T0 = 1, kappa = mu c_p / Pr
    assert abs(case.gamma * case.R - 1.0) < 1e-15
    assert abs(case.kappa - case.mu * 2.5 / 0.71) < 1e-15


def test_mhd_paper_table_equals_the_paper_field_and_is_solenoidal():
    xs = syn.coords((12, 12, 12))
    t = torch.full_like(xs[0], 0.41)
    case = syn.MhdPaperCase(n=12)
    V = case.table().primitives(xs, t)
    kx, ky = TWO_PI * xs[0], TWO_PI * xs[1]
    st = torch.sin(t)
    torch.testing.assert_close(V[4], 0.5 - 0.3 * torch.cos(kx) * torch.sin(ky) * st, rtol=0, atol=1e-15)
    torch.testing.assert_close(V[5], 0.5 + 0.3 * torch.sin(kx) * torch.cos(ky) * st, rtol=0, atol=1e-15)
    assert float(V[3].abs().max()) == 0.0 and float(V[6].abs().max()) == 0.0
    tab = case.table()
    div = sum(tab.gradient(xs, t, 4 + c, c) for c in range(3))
    assert float(div.abs().max()) < 1e-13
    seeded = syn.mhd_mms_table(syn.MhdCase(n=12))
    div = sum(seeded.gradient(xs, t, 4 + c, c) for c in range(3))
    assert float(div.abs().max()) < 1e-13


@pytest.mark.parametrize("which", ["nsf_seeded", "nsf_paper", "mhd_seeded", "mhd_paper"])
def test_analytic_trackers_equal_forward_mode_derivatives(which):
    if which.startswith("nsf"):
        case = syn.NsfCase(n=16) if which == "nsf_seeded" else syn.NsfPaperCase(n=16)
        tab = syn.nsf_mms_table(case) if which == "nsf_seeded" else case.table()
        sysm = oracle.systems.NsfPrimitive(case.gamma, case.R, 0.01, 0.02, 0.1)
        xs = syn.coords((16, 16))
    else:
        case = syn.MhdCase(n=8) if which == "mhd_seeded" else syn.MhdPaperCase(n=8)
        tab = syn.mhd_mms_table(case) if which == "mhd_seeded" else case.table()
        sysm = oracle.systems.MhdCurrent(case.gamma, case.eta, 0.1)
        xs = syn.coords((8, 8, 8))
    t = torch.full_like(xs[0], 0.3)
    torch.testing.assert_close(tab.augmented(xs, t), exact_augmented(sysm, tab.exact, xs, t), rtol=0, atol=1e-13)


def test_hcnsf_table_equals_the_papers_expanded_fields():
    """Supplement, HCNSF MMS, compiler-expanded fields Q_0 .. Q_4 (rho0 = c_s = 1): the mode
    table built from the physical form (U0 = Ma sqrt(gamma), p0 = rho0 c_s^2, linear response
    gamma c_s^2 drho) reproduces the printed expansions, including the printed constants
    0.591607978309962, 121/40, 161/200 and 0.0236643191323985 / 0.118321595661992."""
    xs = syn.coords((6, 6, 6))
    xs = tuple(x + 0.013 * (d + 1) for d, x in enumerate(xs))          # off the grid nodes
    t = torch.full_like(xs[0], 0.73)
    s = [torch.sin(TWO_PI * x) for x in xs]
    c = [torch.cos(TWO_PI * x) for x in xs]
    st, ct = torch.sin(t), torch.cos(t)
    U = 0.591607978309962
    Q = syn.HcnsfPaperCase(n=6).table().exact(*xs, t)
    rho = s[0] * s[2] * ct * c[1] / 5 + 1
    torch.testing.assert_close(Q[0], rho, rtol=0, atol=1e-15)
    torch.testing.assert_close(Q[1], (st * s[1] * s[2] * c[0] / 5 + U) * rho, rtol=0, atol=1e-14)
    torch.testing.assert_close(Q[2], (st * s[0] * s[2] * c[1] / 5 + U) * rho, rtol=0, atol=1e-14)
    torch.testing.assert_close(Q[3], (st * s[0] * s[1] * c[2] / 5 + U) * rho, rtol=0, atol=1e-14)
    a, b = 0.0236643191323985, 0.118321595661992
    E = (st ** 2 * s[0] ** 3 * s[1] ** 2 * s[2] * ct * c[1] * c[2] ** 2 / 250
         + st ** 2 * s[0] ** 3 * s[2] ** 3 * ct * c[1] ** 3 / 250
         + st ** 2 * s[0] ** 2 * s[1] ** 2 * c[2] ** 2 / 50
         + st ** 2 * s[0] ** 2 * s[2] ** 2 * c[1] ** 2 / 50
         + st ** 2 * s[0] * s[1] ** 2 * s[2] ** 3 * ct * c[0] ** 2 * c[1] / 250
         + st ** 2 * s[1] ** 2 * s[2] ** 2 * c[0] ** 2 / 50
         + a * st * s[0] ** 2 * s[1] * s[2] * ct * c[1] * c[2]
         + a * st * s[0] ** 2 * s[2] ** 2 * ct * c[1] ** 2
         + a * st * s[0] * s[1] * s[2] ** 2 * ct * c[0] * c[1]
         + b * st * s[0] * s[1] * c[2] + b * st * s[0] * s[2] * c[1] + b * st * s[1] * s[2] * c[0]
         + st * s[1] * c[0] * c[2] / 2 + 161 * s[0] * s[2] * ct * c[1] / 200 + 121 / 40)
    torch.testing.assert_close(Q[4], E, rtol=0, atol=1e-13)
