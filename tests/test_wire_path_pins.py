"""Pins of the oracle's staircase wires (an oblique wire between two
arbitrary nodes as grid-aligned segments, the staircase wire model the
paper lists among its thin-wire techniques), read back from the PEC edges
the wire leaves in the coefficients (CPU only)."""
import itertools

import numpy as np
import pytest

from oracle.oracle import OracleGrid


def pec_edges(p0, p1, n=(18, 16, 20)):
    """edges (axis, i, j, k) whose ca turned 0 because of the wire"""
    def coefs(with_wire):
        g = OracleGrid(*n, 0.1)
        if with_wire:
            g.add_wire_path(p0, p1, 0.005)
        g.finalize()
        return [g.get_coef(c) for c in range(3)]
    bare, wired = coefs(False), coefs(True)
    out = set()
    for c in range(3):
        kk, jj, ii = np.nonzero((bare[c] != 0) & (wired[c] == 0))
        out |= {(c, int(i), int(j), int(k)) for i, j, k in zip(ii, jj, kk)}
    return out


def nodes_of(edges):
    adj = {}
    for c, i, j, k in edges:
        a = (i, j, k)
        b = list(a)
        b[c] += 1
        b = tuple(b)
        adj.setdefault(a, []).append(b)
        adj.setdefault(b, []).append(a)
    return adj


def dist_to_segment(q, a, b):
    q, a, b = (np.asarray(v, float) for v in (q, a, b))
    d = b - a
    t = np.clip(np.dot(q - a, d) / np.dot(d, d), 0, 1)
    return np.linalg.norm(q - (a + t * d))


@pytest.mark.parametrize("p0,p1", [((3, 4, 5), (15, 9, 12)), ((15, 12, 3), (5, 3, 16)), ((4, 4, 4), (12, 12, 12)),
                                   ((9, 2, 8), (9, 13, 8)), ((2, 7, 15), (14, 7, 4))])
def test_staircase_is_a_grid_path_along_the_segment(p0, p1):
    """the wire's PEC edges form one simple path from p0 to p1 of exactly
    the Manhattan length, every node within one cell of the segment"""
    edges = pec_edges(p0, p1)
    assert len(edges) == sum(abs(b - a) for a, b in zip(p0, p1))
    adj = nodes_of(edges)
    deg = {v: len(nb) for v, nb in adj.items()}
    ends = sorted(v for v, dgr in deg.items() if dgr == 1)
    assert ends == sorted([tuple(p0), tuple(p1)])
    assert all(dgr <= 2 for dgr in deg.values())
    # connected: walk from p0
    seen, stack = {tuple(p0)}, [tuple(p0)]
    while stack:
        for w in adj[stack.pop()]:
            if w not in seen:
                seen.add(w)
                stack.append(w)
    assert seen == set(adj)
    assert max(dist_to_segment(v, p0, p1) for v in adj) <= 1.0


def test_axis_aligned_path_equals_plain_wire():
    """an axis-aligned path equals the plain wire between the same nodes"""
    a = pec_edges((9, 2, 8), (9, 13, 8))
    g = OracleGrid(18, 16, 20, 0.1)
    g.add_wire((9, 2, 8), (9, 13, 8), 0.005)
    g.finalize()
    h = OracleGrid(18, 16, 20, 0.1)
    h.finalize()
    b = set()
    for c in range(3):
        kk, jj, ii = np.nonzero((h.get_coef(c) != 0) & (g.get_coef(c) == 0))
        b |= {(c, int(i), int(j), int(k)) for i, j, k in zip(ii, jj, kk)}
    assert a == b
