"""Discrete velocity sets (c_i, w_i, c_s^2) for the oracle, in exact rationals.

D2Q5 and D3Q7 follow the paper's stencil table (supplement, "Discrete velocity sets of
the two stencils used in the study").  D2Q9 and D3Q19 are the standard textbook sets;
the paper allows any symmetric lattice satisfying the isotropy conditions of Sec. 2.2.1
(sum w = 1, sum w c = 0, sum w c c = c_s^2 I), which `isotropy_defects` checks exactly.
D1Q2 (c = +-1, w = 1/2, c_s^2 = 1) is the canonical two-velocity relaxation scheme of
Sec. 2.2.2 (Eq. maxwellians), used for the Lax-Friedrichs reduction check.
"""
from __future__ import annotations

from dataclasses import dataclass
from fractions import Fraction as Fr
from itertools import product

import torch


@dataclass(frozen=True)
class Lattice:
    name: str
    c: tuple          # tuple of integer velocity tuples, length q, each of length D
    w: tuple          # Fractions
    cs2: Fr

    @property
    def q(self):
        return len(self.c)

    @property
    def D(self):
        return len(self.c[0])

    def c_tensor(self):
        return torch.tensor(self.c, dtype=torch.float64)           # [q, D]

    def w_tensor(self):
        return torch.tensor([float(x) for x in self.w], dtype=torch.float64)  # [q]


def _d2q5():
    c = ((0, 0), (1, 0), (-1, 0), (0, 1), (0, -1))
    w = (Fr(1, 3),) + (Fr(1, 6),) * 4
    return Lattice("D2Q5", c, w, Fr(1, 3))


def _d2q9():
    c, w = [], []
    for cx, cy in product((-1, 0, 1), repeat=2):
        n = abs(cx) + abs(cy)
        c.append((cx, cy))
        w.append({0: Fr(4, 9), 1: Fr(1, 9), 2: Fr(1, 36)}[n])
    return Lattice("D2Q9", tuple(c), tuple(w), Fr(1, 3))


def _d3q7():
    c = ((0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1))
    w = (Fr(1, 4),) + (Fr(1, 8),) * 6
    return Lattice("D3Q7", c, w, Fr(1, 4))


def _d3q19():
    c, w = [], []
    for v in product((-1, 0, 1), repeat=3):
        n = sum(abs(x) for x in v)
        if n == 3:
            continue
        c.append(v)
        w.append({0: Fr(1, 3), 1: Fr(1, 18), 2: Fr(1, 36)}[n])
    return Lattice("D3Q19", tuple(c), tuple(w), Fr(1, 3))


def _d1q2():
    return Lattice("D1Q2", ((1,), (-1,)), (Fr(1, 2), Fr(1, 2)), Fr(1))


LATTICES = {l.name: l for l in (_d1q2(), _d2q5(), _d2q9(), _d3q7(), _d3q19())}


def isotropy_defects(lat: Lattice):
    """Exact defects of the three isotropy conditions (Sec. 2.2.1); all zero if valid."""
    D = lat.D
    s0 = sum(lat.w) - 1
    s1 = [sum(w * c[a] for w, c in zip(lat.w, lat.c)) for a in range(D)]
    s2 = [[sum(w * c[a] * c[b] for w, c in zip(lat.w, lat.c)) - (lat.cs2 if a == b else 0)
           for b in range(D)] for a in range(D)]
    return s0, s1, s2
