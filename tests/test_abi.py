"""The C-ABI library loads and exports what include/lbx.h declares; host-side argument
handling (no GPU needed)."""
import os
import re
from fractions import Fraction as Fr

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _lbx():
    try:
        from paper_2607_05668_b300 import lbx
    except ImportError as e:
        pytest.fail(f"library not built: {e}")
    return lbx


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "lbx.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(lbx_\w+)\s*\(", txt)))


def test_every_declared_symbol_is_exported():
    lbx = _lbx()
    names = declared_functions()
    assert len(names) >= 25
    missing = [n for n in names if not hasattr(lbx.lib(), n)]
    assert not missing, missing


def test_lattice_tables_are_isotropic():
    lbx = _lbx()
    for lat, cs2 in ((lbx.D2Q5, Fr(1, 3)), (lbx.D2Q9, Fr(1, 3)), (lbx.D3Q7, Fr(1, 4)), (lbx.D3Q19, Fr(1, 3))):
        c, w = lbx.lattice_velocities(lat)
        wf = [Fr(x).limit_denominator(64) for x in w]
        assert sum(wf) == 1
        for a in range(3):
            assert sum(wi * int(ci[a]) for wi, ci in zip(wf, c)) == 0
            for b in range(3):
                s = sum(wi * int(ci[a]) * int(ci[b]) for wi, ci in zip(wf, c))
                D = 3 if lat in (lbx.D3Q7, lbx.D3Q19) else 2
                assert s == (cs2 if (a == b and a < D) else 0)


def test_scheme_derivation_follows_refinement_laws():
    lbx = _lbx()
    s = lbx.System(lbx.NSF_PRIM_TRACK, (1.4, 1.0, 0.01, 0.02), (1.0, 0.3, 0.1, 3.0))
    sch = lbx.Scheme(s, lbx.D2Q9, (256, 256), lbx.DIFFUSIVE, 2.0, tau_R=60.0, g_tau=6.0)
    assert sch.dt == pytest.approx(2.0 / 256 ** 2)
    assert sch.tau[0] == pytest.approx(0.5 + 60.0 * sch.dt)
    assert sch.tau[4] == pytest.approx(7.0)
    assert sch.buffer_bytes == 10 * 9 * 256 * 256 * 8
    m = lbx.System(lbx.MHD_J_TRACK, (1.4, 0.01), (1.0,) + (0,) * 6 + (1.78,))
    sch3 = lbx.Scheme(m, lbx.D3Q19, (32, 32, 32), lbx.ACOUSTIC, 0.05, tau_R=160, g_tau=4, precision=lbx.FP16_SCALED)
    assert sch3.dt == pytest.approx(0.05 / 32) and sch3.buffer_bytes == 11 * 19 * 32 ** 3 * 2


@pytest.mark.parametrize("kw,msg", [
    (dict(lattice=3), "dimension"),            # D3Q7 for a 2D system
    (dict(tau_lb=0.4), "must exceed 1/2"),
    (dict(extent=(1, 8)), "extents"),
    (dict(f=0.0), "f must be"),
])
def test_invalid_schemes_are_rejected(kw, msg):
    lbx = _lbx()
    s = lbx.System(lbx.ADR_CASCADE, (1.0, 0.5, 0.01, 0.0), (1.0, 0.0, 0.0))
    args = dict(lattice=lbx.D2Q5, extent=(8, 8), scaling=lbx.DIFFUSIVE, f=1.0, tau_lb=0.8, g_tau=6.0)
    args.update(kw)
    with pytest.raises(lbx.LbxError) as e:
        lbx.Scheme(s, **args)
    assert e.value.name == "ERR_ARG" and msg in str(e.value)


def test_unknown_family_is_rejected():
    lbx = _lbx()
    with pytest.raises(lbx.LbxError) as e:
        lbx.System(99)
    assert e.value.name == "ERR_ARG"


def test_forcing_requires_the_adr_cascade():
    lbx = _lbx()
    s = lbx.System(lbx.BURGERS, (), (0.0,))
    with pytest.raises(lbx.LbxError):
        lbx.Scheme(s, lbx.D2Q5, (8, 8), lbx.ACOUSTIC, 0.2, tau_R=0.2, mms=lbx.MMS_ADR_SEPARABLE)


def test_init_without_device_fails_loudly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    lbx = _lbx()
    s = lbx.System(lbx.ADR_CASCADE, (1.0, 0.5, 0.01, 0.0), (1.0, 0.0, 0.0))
    sch = lbx.Scheme(s, lbx.D2Q5, (8, 8), lbx.DIFFUSIVE, 1.0, tau_lb=0.8, g_tau=6.0)
    with pytest.raises(lbx.LbxError) as e:
        lbx.State(sch, np.ones((3, 8, 8)))
    assert e.value.name == "ERR_CUDA"


def test_hcnsf_declaration_and_scheme_checks():
    """3D homogenized NSF: 14 components in the paper's order, 5 conserved, D3Q7 with the
    advected-solid fields; zero tracker background and eta > 0 required; prescribed fields
    and in-place streaming validated on the host."""
    lbx = _lbx()
    Q0 = [1.0, 0.59, 0.59, 0.59, 3.03] + [0.0] * 9
    s = lbx.System(lbx.HCNSF_3D, (1.4, 0.01, 0.01, 0.1), Q0)
    assert (s.K, s.n_cons, s.dim) == (14, 5, 3)
    assert s.names[5:8] == ["G_u11", "G_u22", "G_T_x"] and s.names[10] == "G_u00"
    pf = (0.5, 0.1, 0.2, 0.1, 0.1, -0.1, 0.05, 0.5, 0.0)
    sch = lbx.Scheme(s, lbx.D3Q7, (32, 32, 32), lbx.ACOUSTIC, 0.05, tau_R=10.0, g_tau=3.0,
                     prescribed=lbx.PRESCRIBED_ADVECTED, prescribed_params=pf, streaming=lbx.STREAM_IN_PLACE)
    assert sch.buffer_bytes == 14 * 7 * 32 ** 3 * 8 and sch.tau[5] == pytest.approx(4.0)
    bad_q0 = list(Q0)
    bad_q0[9] = 0.1
    with pytest.raises(lbx.LbxError, match="tracker background"):
        lbx.System(lbx.HCNSF_3D, (1.4, 0.01, 0.01, 0.1), bad_q0)
    with pytest.raises(lbx.LbxError, match="eta"):
        lbx.System(lbx.HCNSF_3D, (1.4, 0.01, 0.01, 0.0), Q0)
    with pytest.raises(lbx.LbxError, match="dimension"):
        lbx.Scheme(s, lbx.D2Q5, (8, 8), lbx.ACOUSTIC, 0.05, tau_R=10.0, g_tau=3.0)
    with pytest.raises(lbx.LbxError, match="unknown prescribed"):
        lbx.Scheme(s, lbx.D3Q7, (8, 8, 8), lbx.ACOUSTIC, 0.05, tau_R=10.0, g_tau=3.0, prescribed=7)
    with pytest.raises(lbx.LbxError, match="not finite"):
        lbx.Scheme(s, lbx.D3Q7, (8, 8, 8), lbx.ACOUSTIC, 0.05, tau_R=10.0, g_tau=3.0,
                   prescribed=lbx.PRESCRIBED_UNIFORM, prescribed_params=(float("nan"),))
    with pytest.raises(lbx.LbxError, match="unknown streaming"):
        lbx.Scheme(s, lbx.D3Q7, (8, 8, 8), lbx.ACOUSTIC, 0.05, tau_R=10.0, g_tau=3.0, streaming=5)
    e = lbx.System(lbx.EULER, (1.4,), (1.0, 0.1, 0.1, 2.5))
    with pytest.raises(lbx.LbxError, match="HCNSF_3D only"):
        lbx.Scheme(e, lbx.D2Q5, (8, 8), lbx.ACOUSTIC, 0.05, tau_R=1.0, prescribed=lbx.PRESCRIBED_UNIFORM,
                   prescribed_params=(0.5, 0.0, 0.0, 0.0))


def test_header_is_plain_c99(tmp_path):
    """include/lbx.h declares a C ABI: it compiles as C99 with pedantic warnings as errors."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "use_lbx.c"
    src.write_text('#include "lbx.h"\n'
                   "int main(void) {\n"
                   "  lbx_scheme_desc d = {0};\n"
                   "  d.streaming = LBX_STREAM_IN_PLACE; d.prescribed = LBX_PRESCRIBED_ADVECTED;\n"
                   "  return d.mms + d.streaming + d.prescribed - 3;\n"
                   "}\n")
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-fsyntax-only",
                        "-I", os.path.join(ROOT, "include"), str(src)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
