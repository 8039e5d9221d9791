"""The CUDA system code on the host (no GPU): systems.cuh's delta-form flux and source are
__host__ __device__, so a small host-only build evaluates them on random states and the
oracle's direct forms check them, Phi(Q0 + dQ) - Phi(Q0) and S(Q0 + dQ), for the 3D
homogenized NSF (with prescribed alpha and u_s, flux and source at different values), the
12-component NSF and the 18-component MHD, and the configurations' families (ADR cascade,
NSF with primitive trackers, 3D MHD with a current tracker, Burgers, Euler, Maxwell TM)."""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest
import torch

from oracle import systems as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2607_05668_b300", "csrc")
F64 = torch.float64

SRC = r'''
#include "systems.cuh"
using namespace lbx;
template <class Sys, int NCF>
static void run(const double* p, const double* Q0, const double* dQ, const double* cf, const double* cs,
                double* dPhi, double* Sr) {
  double P[Sys::K][Sys::D], Sv[Sys::K];
  if constexpr (NCF > 0) {
    double a[NCF], b[NCF];
    for (int i = 0; i < NCF; ++i) { a[i] = cf[i]; b[i] = cs[i]; }
    Sys::eval(p, Q0, dQ, P, Sv, a, b);
  } else {
    Sys::eval(p, Q0, dQ, P, Sv);
  }
  for (int k = 0; k < Sys::K; ++k) {
    Sr[k] = Sv[k];
    for (int d = 0; d < Sys::D; ++d) dPhi[k * Sys::D + d] = P[k][d];
  }
}
extern "C" void eval_hcnsf(const double* p, const double* Q0, const double* dQ, const double* cf, const double* cs,
                           double* dPhi, double* Sr) { run<SysHCNSF<double>, 4>(p, Q0, dQ, cf, cs, dPhi, Sr); }
extern "C" void eval_nsf12(const double* p, const double* Q0, const double* dQ, double* dPhi, double* Sr) {
  run<SysNSF12<double>, 0>(p, Q0, dQ, nullptr, nullptr, dPhi, Sr);
}
extern "C" void eval_mhd18(const double* p, const double* Q0, const double* dQ, double* dPhi, double* Sr) {
  run<SysMHD18<double>, 0>(p, Q0, dQ, nullptr, nullptr, dPhi, Sr);
}
#define PLAIN(name, Sys) \
  extern "C" void eval_##name(const double* p, const double* Q0, const double* dQ, double* dPhi, double* Sr) { \
    run<Sys<double>, 0>(p, Q0, dQ, nullptr, nullptr, dPhi, Sr); \
  }
// augment: the exact augmented state from primitives V[NPRIM] and gradients G[NPRIM][3]
template <class Sys>
static void aug(const double* p, const double* V, const double* G, double* Q) {
  double v[Sys::NPRIM], g[Sys::NPRIM][3], q[Sys::K];
  for (int i = 0; i < Sys::NPRIM; ++i) {
    v[i] = V[i];
    for (int b = 0; b < 3; ++b) g[i][b] = G[3 * i + b];
  }
  Sys::augment(p, v, g, q);
  for (int k = 0; k < Sys::K; ++k) Q[k] = q[k];
}
extern "C" void aug_hcnsf(const double* p, const double* V, const double* G, double* Q) { aug<SysHCNSF<double>>(p, V, G, Q); }
extern "C" void aug_nsf12(const double* p, const double* V, const double* G, double* Q) { aug<SysNSF12<double>>(p, V, G, Q); }
extern "C" void aug_mhd18(const double* p, const double* V, const double* G, double* Q) { aug<SysMHD18<double>>(p, V, G, Q); }
extern "C" void aug_nsf(const double* p, const double* V, const double* G, double* Q) { aug<SysNSF<double>>(p, V, G, Q); }
extern "C" void aug_mhd(const double* p, const double* V, const double* G, double* Q) { aug<SysMHD<double>>(p, V, G, Q); }
extern "C" void aug_euler(const double* p, const double* V, const double* G, double* Q) { aug<SysEuler<double>>(p, V, G, Q); }
extern "C" void aug_adr(const double* p, const double* V, const double* G, double* Q) { aug<SysADR<double>>(p, V, G, Q); }
extern "C" void aug_burgers(const double* p, const double* V, const double* G, double* Q) { aug<SysBurgers<double>>(p, V, G, Q); }
extern "C" void aug_maxwell(const double* p, const double* V, const double* G, double* Q) { aug<SysMaxwell<double>>(p, V, G, Q); }
#include "lattices.cuh"
// binary32 weights of each lattice (lattices.cuh, weight<Lat, float>) and their float sum
template <class Lat>
static int weights_f32(float* w, float* sum) {
  float acc = 0.0f;
  for (int i = 0; i < Lat::Q; ++i) {
    w[i] = weight<Lat, float>(i);
    acc += w[i];
  }
  *sum = acc;
  return Lat::Q;
}
extern "C" int weights_f32_d2q5(float* w, float* s) { return weights_f32<LatD2Q5>(w, s); }
extern "C" int weights_f32_d2q9(float* w, float* s) { return weights_f32<LatD2Q9>(w, s); }
extern "C" int weights_f32_d3q7(float* w, float* s) { return weights_f32<LatD3Q7>(w, s); }
extern "C" int weights_f32_d3q19(float* w, float* s) { return weights_f32<LatD3Q19>(w, s); }
#define SPEED(name, Sys) \
  extern "C" double speed_##name(const double* p, const double* Q0, const double* dQ) { \
    return Sys<double>::max_speed(p, Q0, dQ); \
  }
SPEED(adr, SysADR)
SPEED(nsf, SysNSF)
SPEED(mhd, SysMHD)
SPEED(burgers, SysBurgers)
SPEED(euler, SysEuler)
SPEED(maxwell, SysMaxwell)
SPEED(nsf12, SysNSF12)
SPEED(mhd18, SysMHD18)
SPEED(hcnsf, SysHCNSF)
PLAIN(adr, SysADR)
PLAIN(nsf, SysNSF)
PLAIN(mhd, SysMHD)
PLAIN(burgers, SysBurgers)
PLAIN(euler, SysEuler)
PLAIN(maxwell, SysMaxwell)
'''


@pytest.fixture(scope="module")
def host_lib(tmp_path_factory):
    nvcc = shutil.which("nvcc") or (os.path.exists("/usr/local/cuda/bin/nvcc") and "/usr/local/cuda/bin/nvcc")
    if not nvcc:
        pytest.skip("nvcc not available")
    d = tmp_path_factory.mktemp("hostsys")
    src, lib = d / "host_systems.cu", d / "libhostsys.so"
    src.write_text(SRC)
    r = subprocess.run([nvcc, "-std=c++17", "--expt-relaxed-constexpr", "-O1", "-shared", "-Xcompiler", "-fPIC",
                        "-I", CSRC, str(src), "-o", str(lib)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    return C.CDLL(str(lib))


def _ptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def test_hcnsf_host_eval_matches_oracle(host_lib):
    gam, mu, kap, eta, tg = 1.4, 0.03, 0.05, 0.1, 0.3
    g = np.random.default_rng(5)
    Q0 = np.array([1.1, 0.4, -0.2, 0.3, 3.2] + [0.0] * 9)
    ke0 = 0.5 * (Q0[1:4] ** 2).sum() / Q0[0]
    p0 = (gam - 1) * (Q0[4] - ke0)
    prm = np.zeros(24)
    prm[:11] = [gam - 1, mu, kap, 1 / eta, 1 / tg, *(Q0[1:4] / Q0[0]), Q0[4] + p0, p0 / Q0[0], gam]
    osys = S.HomogenizedNsf3D(gam, mu, kap, eta, tg, fields=None)
    for trial in range(20):
        dQ = g.uniform(-0.1, 0.1, 14)
        cf = np.array([g.uniform(0, 1), *g.uniform(-0.3, 0.3, 3)])
        cs = np.array([g.uniform(0, 1), *g.uniform(-0.3, 0.3, 3)])
        dPhi, Sr = np.zeros(42), np.zeros(14)
        host_lib.eval_hcnsf(_ptr(prm), _ptr(Q0), _ptr(dQ), _ptr(cf), _ptr(cs), _ptr(dPhi), _ptr(Sr))
        Q = torch.tensor(Q0 + dQ, dtype=F64)
        cft = [torch.tensor(v, dtype=F64) for v in cf]
        cst = [torch.tensor(v, dtype=F64) for v in cs]
        want = (osys.flux(Q, cft) - osys.flux(torch.tensor(Q0, dtype=F64), cft)).numpy().reshape(-1)
        np.testing.assert_allclose(dPhi, want, rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(Sr, osys.source(Q, cst).numpy(), rtol=1e-12, atol=1e-12)


def _cascade_prm(family, Q0, P, tg):
    """The background-dependent parameters of the cascade families (uniform background:
    zero gradients), laid out as systems.cuh documents them."""
    prm = np.zeros(24)
    rho, m = Q0[0], Q0[1:3]
    u = m / rho
    if family == "nsf12":
        g, R, mu, K = P
        p0 = (g - 1) * (Q0[3] - 0.5 * (m * u).sum())
        prm[:19] = [g - 1, R, mu, K, 1 / tg, u[0], u[1], Q0[3] + p0, p0 / (rho * R)] + [0.0] * 9 + [g]
    else:
        g, mu, K, eta = P
        B = Q0[4:6]
        b2 = (B * B).sum()
        p0 = (g - 1) * (Q0[3] - 0.5 * (m * u).sum() - 0.5 * b2)
        prm[:20] = [g - 1, mu, K, eta, 1 / tg, u[0], u[1], Q0[3] + p0 + 0.5 * b2, (u * B).sum(), p0 / rho] + [0.0] * 9 + [g]
    return prm


@pytest.mark.parametrize("family", ["nsf12", "mhd18"])
def test_cascade_host_eval_matches_oracle(host_lib, family):
    g = np.random.default_rng(7)
    tg = 0.37
    if family == "nsf12":
        P = (1.4, 0.8, 0.03, 0.05)
        Q0 = np.array([1.05, 0.3, -0.2, 2.6] + [0.0] * 8)
        osys = S.NsfConservedGradients(*P, tau_grad=tg)
        fn, K = host_lib.eval_nsf12, 12
    else:
        P = (1.4, 0.03, 0.05, 0.07)
        Q0 = np.array([1.05, 0.3, -0.2, 3.4, 0.4, -0.3] + [0.0] * 12)
        osys = S.MhdPowell2D(*P, tau_grad=tg)
        fn, K = host_lib.eval_mhd18, 18
    prm = _cascade_prm(family, Q0, P, tg)
    for trial in range(20):
        dQ = g.uniform(-0.1, 0.1, K)
        dPhi, Sr = np.zeros(2 * K), np.zeros(K)
        fn(_ptr(prm), _ptr(Q0), _ptr(dQ), _ptr(dPhi), _ptr(Sr))
        Q = torch.tensor(Q0 + dQ, dtype=F64)
        want = (osys.flux(Q) - osys.flux(torch.tensor(Q0, dtype=F64))).numpy().reshape(-1)
        np.testing.assert_allclose(dPhi, want, rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(Sr, osys.source(Q).numpy(), rtol=1e-12, atol=1e-12)


def _plain_case(name, g):
    """(oracle system, Q0, parameter array as systems.cuh lays it out, K, D) for a uniform
    background with zero trackers."""
    prm = np.zeros(24)
    tg = 0.29
    if name == "adr":
        a, nu, R = (0.4, -0.25), 0.05, 0.7
        prm[:5] = [a[0], a[1], nu, R, 1 / tg]
        return S.AdrCascade(a, nu, tg, R=R), np.array([0.6, 0.0, 0.0]), prm, 3, 2
    if name == "nsf":
        gam, R, mu, K = 1.4, 0.8, 0.03, 0.05
        Q0 = np.array([1.05, 0.3, -0.2, 2.6] + [0.0] * 6)
        u = Q0[1:3] / Q0[0]
        p0 = (gam - 1) * (Q0[3] - 0.5 * (Q0[1:3] * u).sum())
        prm[:14] = [gam - 1, R, mu, K, 1 / tg, u[0], u[1], Q0[3] + p0, p0 / Q0[0], 0, 0, 0, gam, 1 / R]  # 8: R T0
        return S.NsfPrimitive(gam, R, mu, K, tg), Q0, prm, 10, 2
    if name == "mhd":
        gam, eta = 1.4, 0.02
        Q0 = np.array([1.05, 0.3, -0.2, 0.1, 0.4, -0.3, 0.2, 3.4, 0.0, 0.0, 0.0])
        u, B = Q0[1:4] / Q0[0], Q0[4:7]
        b2 = (B * B).sum()
        p0 = (gam - 1) * (Q0[7] - 0.5 * (Q0[1:4] * u).sum() - 0.5 * b2)
        prm[:9] = [gam - 1, eta, 1 / tg, u[0], u[1], u[2], Q0[7] + p0 + 0.5 * b2, (u * B).sum(), gam]
        return S.MhdCurrent(gam, eta, tg), Q0, prm, 11, 3
    if name == "burgers":
        return S.Burgers(), np.array([0.3]), prm, 1, 2
    if name == "euler":
        gam = 1.4
        Q0 = np.array([1.05, 0.3, -0.2, 2.6])
        u = Q0[1:3] / Q0[0]
        p0 = (gam - 1) * (Q0[3] - 0.5 * (Q0[1:3] * u).sum())
        prm[:5] = [gam - 1, u[0], u[1], Q0[3] + p0, gam]
        return S.Euler(gam), Q0, prm, 4, 2
    c = 1.3
    prm[0] = c
    return S.MaxwellTM(c), np.array([0.2, -0.1, 0.3]), prm, 3, 2


@pytest.mark.parametrize("name", ["adr", "nsf", "mhd", "burgers", "euler", "maxwell"])
def test_configuration_families_host_eval_matches_oracle(host_lib, name):
    g = np.random.default_rng(11)
    osys, Q0, prm, K, D = _plain_case(name, g)
    fn = getattr(host_lib, f"eval_{name}")
    for trial in range(20):
        dQ = g.uniform(-0.1, 0.1, K)
        dPhi, Sr = np.zeros(D * K), np.zeros(K)
        fn(_ptr(prm), _ptr(Q0), _ptr(dQ), _ptr(dPhi), _ptr(Sr))
        Q = torch.tensor(Q0 + dQ, dtype=F64)
        want = (osys.flux(Q) - osys.flux(torch.tensor(Q0, dtype=F64))).numpy().reshape(-1)
        np.testing.assert_allclose(dPhi, want, rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(Sr, osys.source(Q).numpy(), rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("family", ["hcnsf", "nsf12", "mhd18", "nsf", "mhd", "euler", "adr", "burgers", "maxwell"])
def test_host_augment_matches_the_mode_tables(host_lib, family):
    """Sys::augment (the exact augmented state the manufactured forcing differentiates)
    against synthetic.ModeTable.augmented at scattered points of the paper's flows."""
    import synthetic as syn
    if family == "hcnsf":
        case = syn.HcnsfPaperCase(n=8)
        tab, dim, prm = case.table(), 3, np.array([case.gamma - 1.0] + [0.0] * 23)
    elif family == "mhd18":
        case = syn.MhdPaper2DCase(n=8)
        tab, dim, prm = case.table(), 2, np.array([case.gamma - 1.0] + [0.0] * 23)
    elif family == "mhd":
        case = syn.MhdPaperCase(n=8)
        tab, dim, prm = case.table(), 3, np.array([case.gamma - 1.0] + [0.0] * 23)
    elif family == "euler":
        tab, dim, prm = syn.euler_table(), 2, np.array([0.4] + [0.0] * 23)
    elif family == "adr":
        tab, dim, prm = syn.AdrPaperCase(n=8).table(), 2, np.zeros(24)
    elif family == "burgers":
        tab, dim, prm = syn.burgers_table(), 2, np.zeros(24)
    elif family == "maxwell":
        tab, dim, prm = syn.maxwell_table(), 2, np.zeros(24)
    else:
        case = syn.NsfPaperCase(n=8)
        tab, dim = case.table(family), 2
        prm = np.array([case.gamma - 1.0, case.R] + [0.0] * 22)
    g = np.random.default_rng(3)
    pts = [tuple(torch.tensor([float(v)], dtype=F64) for v in g.uniform(0, 1, dim)) for _ in range(6)]
    fn = getattr(host_lib, f"aug_{family}")
    for xs in pts:
        t = torch.tensor([0.61], dtype=F64)
        V = np.array([float(v[0]) for v in tab.primitives(xs, t)])
        G = np.zeros((len(V), 3))
        for q in range(len(V)):
            for b in range(dim):
                G[q, b] = float(tab.gradient(xs, t, q, b)[0])
        want = tab.augmented(xs, t)[:, 0].numpy()
        got = np.zeros(len(want))
        fn(_ptr(prm), _ptr(V), _ptr(G.reshape(-1).copy()), _ptr(got))
        np.testing.assert_allclose(got, want, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("lat", ["d2q5", "d2q9", "d3q7", "d3q19"])
def test_binary32_weights_sum_to_exactly_one(host_lib, lat):
    """The FP32 kernels' weights (moving weights on multiples of 2^-26, rest = 1 - their sum)
    add up to exactly 1 as real numbers, so sum_i w_i X = X holds without a systematic bias
    (only the per-operation rounding remains); each moving weight lies within 2^-27 of the
    exact one and the rest weight within (q - 1) 2^-27.  Exact weights in the library's own
    velocity order (lbx_lattice_velocities, a host call)."""
    from fractions import Fraction as Fr
    from paper_2607_05668_b300 import lbx
    w = np.zeros(32, dtype=np.float32)
    sm = np.zeros(1, dtype=np.float32)
    q = getattr(host_lib, f"weights_f32_{lat}")(w.ctypes.data_as(C.POINTER(C.c_float)), sm.ctypes.data_as(C.POINTER(C.c_float)))
    w = w[:q]
    assert sum(Fr(float(x)) for x in w) == 1
    _, wd = lbx.lattice_velocities(getattr(lbx, lat.upper()))
    exact = [Fr(float(v)).limit_denominator(64) for v in wd]
    assert all(abs(Fr(float(x)) - e) <= Fr(1, 2 ** 27) for x, e in zip(w[1:], exact[1:]))
    assert abs(Fr(float(w[0])) - exact[0]) <= Fr(q - 1, 2 ** 27)          # the rest weight absorbs them


def _hcnsf_case():
    gam, mu, kap, eta, tg = 1.4, 0.03, 0.05, 0.1, 0.3
    Q0 = np.array([1.1, 0.4, -0.2, 0.3, 3.2] + [0.0] * 9)
    p0 = (gam - 1) * (Q0[4] - 0.5 * (Q0[1:4] ** 2).sum() / Q0[0])
    prm = np.zeros(24)
    prm[:11] = [gam - 1, mu, kap, 1 / eta, 1 / tg, *(Q0[1:4] / Q0[0]), Q0[4] + p0, p0 / Q0[0], gam]
    return S.HomogenizedNsf3D(gam, mu, kap, eta, tg, fields=None), Q0, prm, 14, 3


@pytest.mark.parametrize("name", ["adr", "nsf", "mhd", "burgers", "euler", "maxwell", "nsf12", "mhd18", "hcnsf"])
def test_host_speed_bounds_dominate_the_oracle_eigenvalues(host_lib, name):
    """Sec. 2.3.2: each family's closed-form max_speed bounds the spectral radius of the
    directional flux Jacobian (the oracle's numeric eigenvalues over 48 directions) at random
    states, and is no more than twice it (HCNSF: the bound takes alpha = 1, the oracle a
    random alpha <= 1)."""
    from oracle import subchar
    g = np.random.default_rng(21)
    if name in ("nsf12", "mhd18"):
        tg = 0.37
        if name == "nsf12":
            P, Q0 = (1.4, 0.8, 0.03, 0.05), np.array([1.05, 0.3, -0.2, 2.6] + [0.0] * 8)
            osys = S.NsfConservedGradients(*P, tau_grad=tg)
        else:
            P, Q0 = (1.4, 0.03, 0.05, 0.07), np.array([1.05, 0.3, -0.2, 3.4, 0.4, -0.3] + [0.0] * 12)
            osys = S.MhdPowell2D(*P, tau_grad=tg)
        prm, K = _cascade_prm(name, Q0, P, tg), len(Q0)
    elif name == "hcnsf":
        osys, Q0, prm, K, _ = _hcnsf_case()
    else:
        osys, Q0, prm, K, _ = _plain_case(name, g)
    fn = getattr(host_lib, f"speed_{name}")
    fn.restype = C.c_double
    dirs = subchar.directions(osys.D, 48)
    for trial in range(8):
        dQ = g.uniform(-0.1, 0.1, K)
        bound = fn(_ptr(prm), _ptr(Q0), _ptr(dQ))
        q = torch.tensor(Q0 + dQ, dtype=F64)
        cf = None if name != "hcnsf" else [torch.tensor(v, dtype=F64) for v in (g.uniform(0, 1), 0.1, 0.0, -0.1)]
        num = subchar.node_max_speed(osys, q, dirs, cf)
        assert num * (1 - 1e-9) <= bound <= 2.0 * num + 1e-12, (bound, num)
