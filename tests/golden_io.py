"""Reader for the hand-derived fixtures under tests/golden/ (see README.txt there)."""
from __future__ import annotations

import os
from dataclasses import dataclass, field
from fractions import Fraction

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@dataclass
class Block:
    update: tuple | None
    pairs: list = field(default_factory=list)   # (s, t, d or None, sigma)
    bc: dict = field(default_factory=dict)      # v -> Fraction


@dataclass
class Fixture:
    name: str
    n: int
    directed: bool
    edges: list
    blocks: list


def load(name: str) -> Fixture:
    n = directed = None
    edges, blocks = [], [Block(None)]
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            tok = line.split()
            if tok[0] == "n":
                n = int(tok[1])
            elif tok[0] == "directed":
                directed = tok[1] == "1"
            elif tok[0] == "edge":
                edges.append((int(tok[1]), int(tok[2]), int(tok[3])))
            elif tok[0] == "pair":
                d = None if tok[3] == "inf" else int(tok[3])
                blocks[-1].pairs.append((int(tok[1]), int(tok[2]), d, int(tok[4])))
            elif tok[0] == "bc":
                blocks[-1].bc[int(tok[1])] = Fraction(tok[2])
            elif tok[0] == "update":
                assert tok[1] == "edge"
                blocks.append(Block(("edge", int(tok[2]), int(tok[3]), int(tok[4]))))
            else:
                raise ValueError(line)
    return Fixture(name, n, directed, edges, blocks)


def all_fixtures():
    return sorted(f for f in os.listdir(GOLDEN) if f.endswith(".txt") and f != "README.txt")


def graph_of(fx: Fixture):
    from paper_1311_2147_gb300 import synth
    e = np.array([(a, b) for a, b, _ in fx.edges], dtype=np.int64).reshape(-1, 2)
    return synth.Graph(fx.n, fx.directed, e[:, 0].astype(np.int32), e[:, 1].astype(np.int32),
                       np.array([w for _, _, w in fx.edges], dtype=np.int64))
