"""Automatic joint-cut blocks (hsf_find_blocks, Sec. V) on seeded SBM-QAOA circuits.

Host-only library code, checked without a GPU against:

* brute force: the number of hubs equals the size of a minimum vertex cover of the
  crossing-gate graph, found by trying every vertex subset (tiny graphs);
* the oracle: the reordered circuit has the same statevector as the input (only
  commuting gates moved), every found block is convex and has Schmidt rank 2
  (Example 4: cascades keep rank 2), and the oracle's HSF sum over the found blocks
  equals Schroedinger;
* Table II's identity: joint paths = 2^(blocks + separate cuts), against 2^(crossing
  gates) for the standard cut.
"""
import itertools

import numpy as np
import pytest

import oracle.hsf_oracle as O
from paper_2502_06959_gb300 import hsf
from paper_2502_06959_gb300 import workloads as W


def crossing_edges(pr):
    out = []
    for g in pr.gates:
        if len(g.qubits) == 2 and (max(g.qubits) > pr.cut >= min(g.qubits)):
            out.append((max(g.qubits), min(g.qubits)))
    return out


def brute_force_cover(edges):
    verts = sorted({v for e in edges for v in e})
    for k in range(len(verts) + 1):
        for sub in itertools.combinations(verts, k):
            s = set(sub)
            if all(a in s or b in s for a, b in edges):
                return k
    return len(verts)


@pytest.mark.parametrize("sizes,p_inter,seed", [((5, 5), 0.35, 1), ((5, 6), 0.3, 2), ((6, 6), 0.25, 3),
                                                ((6, 5), 0.4, 4), ((4, 6), 0.5, 5)])
def test_hubs_are_a_minimum_vertex_cover(sizes, p_inter, seed):
    pr = W.sbm_qaoa(sizes, 0.8, p_inter, seed=seed)
    order, blocks, hubs = hsf.hsf_find_blocks(pr.n, pr.gates, pr.cut)
    assert sorted(order) == list(range(len(pr.gates)))
    assert hubs == brute_force_cover(crossing_edges(pr))
    assert len(blocks) == hubs                     # no star above the leaf cap here


@pytest.mark.parametrize("sizes,p_inter,seed", [((5, 5), 0.35, 11), ((6, 6), 0.3, 12)])
def test_found_blocks_against_the_oracle(sizes, p_inter, seed):
    pr = W.sbm_qaoa(sizes, 0.8, p_inter, seed=seed)
    q = hsf.problem_with_found_blocks(pr)
    ref = O.schrodinger(pr.n, pr.gates)
    assert np.max(np.abs(O.schrodinger(q.n, q.gates) - ref)) < 1e-13     # same circuit
    O.execution_order(q.n, q.gates, q.blocks)                              # convex, listed in order
    dec = O.decompose_blocks(q.n, q.gates, q.cut, q.blocks)
    assert all(len(d["sigma"]) == 2 for d in dec)                          # cascades: rank 2
    amps, info = O.hsf_amplitudes(q.n, q.gates, q.cut, q.blocks)
    assert info["num_paths"] == 2 ** len(q.blocks)
    assert np.max(np.abs(amps - ref)) < 1e-12


def test_table2_identity_and_leaf_cap():
    """q30-shaped instance: joint paths 2^(blocks+sep) far below the standard 2^(sep cuts);
    with a leaf cap of 2 the stars split and the block count grows, never the rank."""
    pr = W.sbm_qaoa((15, 15), 0.8, 0.1, seed=1)
    sep_cuts = len(crossing_edges(pr))
    order, blocks, hubs = hsf.hsf_find_blocks(pr.n, pr.gates, pr.cut)
    assert len(blocks) == hubs < sep_cuts
    _, blocks2, hubs2 = hsf.hsf_find_blocks(pr.n, pr.gates, pr.cut, max_leaves=2)
    assert hubs2 == hubs and len(blocks2) >= len(blocks)
    assert all(len(b) <= 2 for b in blocks2)
    # every crossing gate is in exactly one block
    q = hsf.problem_with_found_blocks(pr)
    cross = [i for i, g in enumerate(q.gates) if max(g.qubits) > q.cut >= min(g.qubits)]
    assert sorted(i for b in q.blocks for i in b) == cross


def test_non_diagonal_crossing_gates_are_plain_cuts():
    gates = [W.Gate("h", (q,)) for q in range(6)]
    gates += [W.Gate("rzz", (3, 2), param=0.3), W.Gate("cx", (4, 1)), W.Gate("rzz", (5, 2), param=0.7),
              W.Gate("rzz", (4, 0), param=1.1)]
    order, blocks, hubs = hsf.hsf_find_blocks(6, gates, 2)
    re = [gates[i] for i in order]
    kinds = [[re[i].kind for i in b] for b in blocks]
    assert ["cx"] in kinds
    assert np.max(np.abs(O.schrodinger(6, re) - O.schrodinger(6, gates))) < 1e-13


def test_rejects_bad_arguments():
    pr = W.sbm_qaoa((4, 4), 0.8, 0.5, seed=0)
    with pytest.raises(hsf.HsfError):
        hsf.hsf_find_blocks(pr.n, pr.gates, pr.cut, max_leaves=0)
    with pytest.raises(hsf.HsfError):
        hsf.hsf_find_blocks(pr.n, pr.gates, pr.n - 1)
