"""Batched persistent launch (many uneven ADR grids) against single-grid runs and the
oracle; graph replay, parity of odd step counts and the autotuner's no-advance rule."""
import math

import numpy as np
import pytest
import torch

import synthetic as syn
from tests import helpers as H

pytestmark = pytest.mark.gpu

lbx = pytest.importorskip("paper_2607_05668_b300.lbx")
from paper_2607_05668_b300 import workloads as W  # noqa: E402

SIZES = [32, 40, 64, 77, 100, 130, 33]      # narrow grids share tiles across rows; ragged tails


def _cases():
    draws = syn.adr_batch_draws(len(SIZES), seed=3)
    return [syn.AdrCase(n=n, a_lat=d.a_lat, tau_u=d.tau_u) for n, d in zip(SIZES, draws)]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")


@pytest.mark.parametrize("prec", [lbx.FP64, lbx.FP32_SHIFT])
def test_batched_instances_equal_single_grid_runs_bitwise(prec):
    cases = _cases()
    schemes = [W.adr_scheme(c, prec) for c in cases]
    b = lbx.Batch(schemes, [syn.adr_fields(c) for c in cases])
    b.set_config(block=64, ctas_per_sm=4)
    b.step(13)
    for j, c in enumerate(cases):
        st = lbx.State(W.adr_scheme(c, prec), syn.adr_fields(c))
        st.step(13)
        assert torch.equal(b.moments(j), st.moments()), j


def test_batched_fp64_matches_oracle():
    cases = _cases()[:4]
    b = lbx.Batch([W.adr_scheme(c, lbx.FP64) for c in cases], [syn.adr_fields(c) for c in cases])
    b.step(25)
    for j, c in enumerate(cases):
        och = H.oracle_adr(c)
        Qo = och.moments(och.run(och.init(syn.adr_fields(c)), 25))
        assert H.rel_linf_per_field(b.moments(j), Qo).max() <= 1e-12


def test_graph_replay_and_odd_step_counts_match_plain_launches():
    cases = _cases()
    fields = [syn.adr_fields(c) for c in cases]
    g = lbx.Batch([W.adr_scheme(c, lbx.FP32_SHIFT) for c in cases], fields)
    p = lbx.Batch([W.adr_scheme(c, lbx.FP32_SHIFT) for c in cases], fields)
    p.set_config(use_graph=False)
    for n in (3, 3, 8, 1, 3):          # repeated and odd lengths: graph cache keyed by parity
        g.step(n)
        p.step(n)
    for j in range(len(cases)):
        assert torch.equal(g.moments(j), p.moments(j))


def test_tuning_does_not_advance_the_state_and_picks_a_measured_config():
    cases = _cases()
    b = lbx.Batch([W.adr_scheme(c, lbx.FP32_SHIFT) for c in cases], [syn.adr_fields(c) for c in cases])
    b.step(4)
    before = [b.moments(j) for j in range(len(cases))]
    rep = b.tune(trials=3)
    assert len(rep["trials"]) >= 4
    best = rep["best"]
    assert best["ms"] == pytest.approx(min(t["ms"] for t in rep["trials"]))
    assert b.config["block"] == best["block"] and b.config["ctas_per_sm"] == best["ctas_per_sm"]
    for j in range(len(cases)):
        assert torch.equal(b.moments(j), before[j])
    b.step(5)
    ref = lbx.Batch([W.adr_scheme(c, lbx.FP32_SHIFT) for c in cases], [syn.adr_fields(c) for c in cases])
    ref.step(9)
    for j in range(len(cases)):
        assert torch.equal(b.moments(j), ref.moments(j))


def test_batch_rejects_mixed_families_and_fp16():
    c = syn.AdrCase(n=32)
    n = syn.NsfCase(n=32)
    with pytest.raises(lbx.LbxError):
        lbx.Batch([W.adr_scheme(c, lbx.FP64), W.nsf_scheme(n, lbx.FP64)], [syn.adr_fields(c), syn.nsf_fields(n)])
    with pytest.raises(lbx.LbxError) as e:
        lbx.Batch([W.adr_scheme(c, lbx.FP16_SCALED)], [syn.adr_fields(c)])
    assert e.value.name == "ERR_UNSUPPORTED"


# ------------------------------------------------ forced batches: the Burgers stability map

def _burgers_batch(N, grid, steps=None):
    gsys = lbx.System(lbx.BURGERS, (), (0.0,))
    xs = syn.coords((N, N))
    schemes, fields = [], []
    for (m, w, A, tau) in grid:
        tab = syn.burgers_table(A)
        schemes.append(W.forced_scheme(tab, gsys, lbx.D2Q5, (N, N), lbx.ACOUSTIC, 0.2, tau_lb=tau))
        fields.append(tab.augmented(xs, 0.0))
    b = lbx.Batch(schemes, fields)
    b.step(int(round(N / 0.2)) if steps is None else steps)      # to t = 1
    return b, schemes, fields


def _diverged(b, grid):
    """Divergent: a non-finite population, or |u| beyond ten times the manufactured amplitude."""
    fin = b.check_finite()
    return [(not f) or float(b.moments(j).abs().max()) > 10.0 * grid[j][2] for j, f in enumerate(fin)]


def test_forced_batch_equals_single_forced_runs_bitwise():
    N, steps = 48, 37
    grid = syn.burgers_stability_grid([0.3, 0.45, 0.55], [1.2, 1.9])
    b, schemes, fields = _burgers_batch(N, grid, steps)
    assert all(b.check_finite())
    for j in (0, 3, 5):
        st = lbx.State(schemes[j], fields[j])
        st.step(steps)
        assert torch.equal(b.moments(j), st.moments())
    b.close()


def test_burgers_stability_boundary_tightens_toward_the_monotone_bound():
    """Sec. 3 (Burgers stability map): run every (Ma, omega) pair to t = 1 and classify it.
    Near omega = 2 the empirical boundary approaches Ma = c_s = 1/sqrt(3) (the equilibria
    stop being monotone in u) from above and tightens under refinement; the verification
    working point Ma = 0.45 is stable; and with heavier relaxation (omega = 1) the boundary
    rises well above c_s."""
    mach = [0.45, 0.5, 0.55, 0.6, 0.65, 0.7, 0.8, 1.0, 1.2]
    bound = {}
    for N in (64, 256):
        for w in (1.0, 1.99):
            grid = syn.burgers_stability_grid(mach, [w])
            b, _, _ = _burgers_batch(N, grid)
            div = _diverged(b, grid)
            b.close()
            stable = [g[0] for g, d in zip(grid, div) if not d]
            assert 0.45 in stable, (N, w, div)
            bound[(N, w)] = max(stable)
    cs = 1.0 / math.sqrt(3.0)
    print("stability boundary (max stable Ma):", bound)
    assert cs - 0.05 <= bound[(256, 1.99)] <= bound[(64, 1.99)] <= cs + 0.15
    assert bound[(256, 1.0)] >= 0.8 and bound[(64, 1.0)] >= 0.8
