"""Qubit-reordering search for a better cut (hsf_search_cut; Sec. VI names reordering
the qubits to find better blocks as future work).

Host-only library code, checked without a GPU against:

* the oracle: the relabeled circuit is the same circuit (Schroedinger amplitudes under
  the bit permutation), and the reported log2 path count equals the sum of log2 ranks
  of the oracle's Schmidt decompositions (LAPACK SVD) of the blocks found on it;
* brute force: on 8 qubits every 4|4 bipartition is tried (the oracle's ranks of the
  found blocks), and the search reaches the minimum;
* the planted structure: a two-community SBM-QAOA graph with scrambled qubit labels
  is cut back along its communities (no more paths than the community cut).
"""
import itertools
import math

import numpy as np
import pytest

import oracle.hsf_oracle as O
from paper_2502_06959_gb300 import hsf
from paper_2502_06959_gb300 import workloads as W


def scrambled(pr, seed):
    rng = np.random.default_rng(seed)
    return hsf.relabel_problem(pr, [int(x) for x in rng.permutation(pr.n)])


def oracle_bits(q):
    """log2 of the oracle's joint path count over the blocks found on q."""
    dec = O.decompose_blocks(q.n, q.gates, q.cut, q.blocks)
    return sum(math.log2(len(d["sigma"])) for d in dec)


def test_single_gate_costs_are_operator_schmidt_ranks():
    # one crossing gate on qubits (2, 1) with the cut after qubit 1: cost = log2 rank
    rng = np.random.default_rng(3)
    a = rng.normal(size=(4, 4)) + 1j * rng.normal(size=(4, 4))
    u, _ = np.linalg.qr(a)
    for g in (W.Gate("cx", (2, 1)), W.Gate("swap", (2, 1)), W.Gate("iswap", (1, 2)),
              W.Gate("rzz", (2, 0), param=0.7), W.Gate("matrix", (1, 3), matrix=u)):
        gates = [W.Gate("h", (q,)) for q in range(4)] + [g]
        _, before, _ = hsf.hsf_search_cut(4, gates, 1, restarts=0)
        sig = O.schmidt_decompose(O.block_unitary(gates, [4], sorted(g.qubits, reverse=True)), 1, 1)[0]
        assert before == pytest.approx(math.log2(len(sig)))


@pytest.mark.parametrize("sizes,p_inter,seed,scramble", [((6, 6), 0.4, 1, 2), ((5, 7), 0.35, 2, 3)])
def test_searched_circuit_is_the_same_circuit_and_cost_matches_oracle(sizes, p_inter, seed, scramble):
    pr = scrambled(W.sbm_qaoa(sizes, 0.8, p_inter, seed=seed), scramble)
    q = hsf.problem_with_searched_cut(pr)
    perm = q.meta["perm"]
    assert sorted(perm) == list(range(pr.n))
    assert q.meta["log2_paths_after"] <= q.meta["log2_paths_before"]
    # the same circuit: psi'[x'] = psi[x] with bit q of x moved to bit perm[q]
    psi = O.schrodinger(pr.n, pr.gates)
    psi2 = O.schrodinger(q.n, q.gates)
    x = np.arange(1 << pr.n, dtype=np.int64)
    xp = np.zeros_like(x)
    for a, b in enumerate(perm):
        xp |= ((x >> a) & 1) << b
    assert np.max(np.abs(psi2[xp] - psi)) < 1e-13
    # the reported cost is the oracle's path count of the blocks found on it
    assert oracle_bits(q) == pytest.approx(q.meta["log2_paths_after"])


def test_search_reaches_brute_force_minimum_on_8_qubits():
    rng = np.random.default_rng(9)
    n, cut = 8, 3
    gates = [W.Gate("h", (q,)) for q in range(n)]
    for _ in range(14):
        i, j = (int(v) for v in rng.choice(n, size=2, replace=False))
        kind = ("rzz", "rzz", "cz", "cx")[int(rng.integers(4))]
        gates.append(W.Gate(kind, (i, j), param=float(rng.uniform(0.3, 2.8))))
        if rng.random() < 0.3:
            gates.append(W.Gate("rx", (i,), param=float(rng.uniform(0.3, 2.8))))
    best = None
    for b_side in itertools.combinations(range(n), cut + 1):
        bs = set(b_side)
        perm, nb, na = [0] * n, 0, 0
        for q in range(n):
            if q in bs:
                perm[q] = nb
                nb += 1
        for q in range(n):
            if q not in bs:
                perm[q] = cut + 1 + na
                na += 1
        pr = W.Problem(n=n, gates=gates, cut=cut, blocks=[])
        q = hsf.problem_with_found_blocks(hsf.relabel_problem(pr, perm))
        c = oracle_bits(q)
        best = c if best is None else min(best, c)
    _, before, after = hsf.hsf_search_cut(n, gates, cut, restarts=4, seed=1)
    assert after == pytest.approx(best)
    assert before >= after


def test_search_cuts_scrambled_communities_back():
    pr = W.sbm_qaoa((15, 15), 0.8, 0.1, seed=1)
    _, aligned, _ = hsf.hsf_search_cut(pr.n, pr.gates, pr.cut, restarts=0)
    ps = scrambled(pr, 6)
    _, before, after = hsf.hsf_search_cut(ps.n, ps.gates, ps.cut, restarts=4, seed=1)
    assert before > aligned
    assert after <= aligned


def test_search_is_deterministic_and_validates():
    pr = scrambled(W.sbm_qaoa((6, 6), 0.8, 0.4, seed=4), 1)
    r1 = hsf.hsf_search_cut(pr.n, pr.gates, pr.cut, restarts=2, seed=7)
    r2 = hsf.hsf_search_cut(pr.n, pr.gates, pr.cut, restarts=2, seed=7)
    assert r1 == r2
    for kw in (dict(cut=pr.n - 1), dict(cut=-1), dict(max_leaves=0), dict(max_leaves=9), dict(restarts=-1)):
        args = dict(cut=pr.cut, max_leaves=8, restarts=0)
        args.update(kw)
        with pytest.raises(hsf.HsfError, match="EINVAL"):
            hsf.hsf_search_cut(pr.n, pr.gates, args["cut"], args["max_leaves"], args["restarts"])
