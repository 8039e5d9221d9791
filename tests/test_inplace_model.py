"""The index mapping of single-buffer in-place streaming, on the CPU (test infrastructure):
two alternating step kinds on one array reproduce two pull steps between two arrays exactly.

Layout (as the library stores populations): G[k, i, x] is the post-collision population
f*_i of node x, leaving along c_i.  A pull step reads f_i(x) = G[k, i, x - c_i].  In place:
  kind 1 reads f_i(x) = G[k, i, x - c_i] and writes f*_i(x) to G[k, i', x + c_i],
  kind 2 reads f_i(x) = G[k, i', x]       and writes f*_i(x) to G[k, i, x],
with i' the opposite velocity.  The collision is the oracle's (Eq. lbe_update without the
streaming), so only the addressing differs between the two runs."""
import pytest
import torch

import oracle
from oracle import systems as S


def _opp(lat):
    c = [tuple(v) for v in lat.c]
    return [c.index(tuple(-x for x in v)) for v in c]


def _shift(a, ci, sign, D):
    """a(x - sign c_i) along the trailing D axes of a [..., *grid] array (periodic)."""
    shifts = tuple(sign * ci[d] for d in range(D) if ci[d] != 0)
    dims = tuple(-(d + 1) for d in range(D) if ci[d] != 0)
    return torch.roll(a, shifts=shifts, dims=dims) if shifts else a


def _post(sch, f, t):
    return sch.collide(f, t)                                  # [K, q, *grid]


def _pull_step(sch, G, t):
    D = sch.lat.D
    f = torch.stack([_shift(G[:, i], sch.c[i], +1, D) for i in range(len(sch.c))], dim=1)
    return _post(sch, f, t)


def _kind1(sch, F, t):
    D, q, op = sch.lat.D, len(sch.c), _opp(sch.lat)
    f = torch.stack([_shift(F[:, i], sch.c[i], +1, D) for i in range(q)], dim=1)
    post = _post(sch, f, t)
    out = torch.empty_like(F)
    for i in range(q):                                        # slot i' at x + c_i
        out[:, op[i]] = _shift(post[:, i], sch.c[i], +1, D)
    return out


def _kind2(sch, F, t):
    q, op = len(sch.c), _opp(sch.lat)
    f = torch.stack([F[:, op[i]] for i in range(q)], dim=1)
    return _post(sch, f, t)                                   # slot i at x


@pytest.mark.parametrize("lname,shape", [("D2Q5", (6, 7)), ("D2Q9", (5, 8)), ("D3Q7", (4, 5, 6)), ("D3Q19", (4, 3, 5))])
def test_two_in_place_kinds_equal_two_pull_steps(lname, shape):
    lat = oracle.LATTICES[lname]
    D = lat.D
    sysm = S.AdrCascade([0.3, -0.2], 0.05, 0.4) if D == 2 else S.MhdCurrent(1.4, 0.02, 0.4)
    sch = oracle.Scheme(sysm, lat, shape, 0.1, 0.01, torch.linspace(0.7, 1.4, sysm.K, dtype=torch.float64))
    g = torch.Generator().manual_seed(3)
    Q = 0.05 * torch.rand((sysm.K,) + shape, generator=g, dtype=torch.float64)
    if sysm.name == "mhd":
        Q[0] += 1.0
        Q[7] += 2.5
    G = sch.init(Q)
    want = _pull_step(sch, _pull_step(sch, G, 0.0), sch.dt)
    got = _kind2(sch, _kind1(sch, G, 0.0), sch.dt)
    assert torch.equal(got, want)
    # the pair's intermediate layout is not the standard one
    assert not torch.equal(_kind1(sch, G, 0.0), _pull_step(sch, G, 0.0))
