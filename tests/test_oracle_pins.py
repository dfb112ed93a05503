"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Every check here is independent of the oracle's own formulas: worked examples of the
paper (tests/golden/), closed forms derived by hand, brute-force index-loop products,
invariants, and planted mistakes that must be caught.
"""
import json
import os

import numpy as np
import pytest

import oracle.hsf_oracle as O
from paper_2502_06959_gb300 import workloads as W
from paper_2502_06959_gb300.workloads import Gate

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def gold(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def test_bell_state_example1():
    g = gold("bell_state.json")
    gates = [Gate(k, tuple(q)) for k, q in g["gates"]]
    psi = O.schrodinger(g["n"], gates)
    ref = np.array(g["amplitudes_re"]) + 1j * np.array(g["amplitudes_im"])
    assert np.max(np.abs(psi - ref)) < 1e-15


def test_cnot_decomposition_example2():
    g = gold("cnot_schmidt.json")
    cx = O.gate_matrix(Gate("cx", (1, 0)))
    recon = sum(np.kron(np.array(t["x"]), np.array(t["y"])) for t in g["terms"])
    assert np.array_equal(recon, cx)                       # printed form equals our CNOT
    sigma, xs, ys = O.schmidt_decompose(cx, 1, 1)
    assert len(sigma) == g["schmidt_rank"]
    assert np.allclose(sigma, [np.sqrt(2), np.sqrt(2)], atol=1e-14)   # derived closed form
    assert np.max(np.abs(O.schmidt_reconstruct(sigma, xs, ys) - cx)) < 1e-14
    # the oracle's X-factors span the same operator space as {P0, P1}
    basis = np.array([np.array(t["x"]).ravel() for t in g["terms"]]).T
    for x in xs:
        coef, res, *_ = np.linalg.lstsq(basis, x.ravel(), rcond=None)
        assert np.max(np.abs(basis @ coef - x.ravel())) < 1e-13


@pytest.mark.parametrize("kind", ["swap", "cx", "cz", "rzz"])
def test_single_gate_ranks_fig3(kind):
    want = gold("fig3_ranks.json")["single_gate_ranks"][kind]
    g = Gate(kind, (1, 0), param=0.7)
    sigma, xs, ys = O.schmidt_decompose(O.gate_matrix(g), 1, 1)
    assert len(sigma) == want
    assert np.max(np.abs(O.schmidt_reconstruct(sigma, xs, ys) - O.gate_matrix(g))) < 1e-14


def test_closed_form_singular_values():
    # derived by hand: sigma(SWAP) = (1,1,1,1); sigma(RZZ(t)) = (2|cos t/2|, 2|sin t/2|)
    s, _, _ = O.schmidt_decompose(O.gate_matrix(Gate("swap", (1, 0))), 1, 1)
    assert np.allclose(s, [1, 1, 1, 1], atol=1e-14)
    for t in (0.3, 1.1, 2.0, 4.0, 5.9):
        s, _, _ = O.schmidt_decompose(O.gate_matrix(Gate("rzz", (1, 0), param=t)), 1, 1)
        ref = sorted([2 * abs(np.cos(t / 2)), 2 * abs(np.sin(t / 2))], reverse=True)
        assert np.allclose(s, ref, atol=1e-14)
    # exact rank drop: RZZ(0) = identity has rank 1
    s, _, _ = O.schmidt_decompose(np.eye(4), 1, 1)
    assert len(s) == 1 and abs(s[0] - 2) < 1e-14


def _cascade(kind, control, targets, theta=0.9):
    gates = []
    for t in targets:
        gates.append(Gate(kind, (control, t), param=theta))
    return gates


@pytest.mark.parametrize("kind", ["cx", "cz", "rzz"])
def test_cascade_rank_example4(kind):
    g = gold("cascade.json")
    n = 4
    gates = _cascade(kind, g["control"], g["targets"])
    qs = O.block_qubits(gates, range(len(gates)))
    u = O.block_unitary(gates, range(len(gates)), qs)
    assert np.allclose(u, O.circuit_unitary_bruteforce(n, gates), atol=1e-14)
    sigma, xs, ys = O.schmidt_decompose(u, 1, 3)
    assert len(sigma) == g["schmidt_rank"]
    assert np.max(np.abs(O.schmidt_reconstruct(sigma, xs, ys) - u)) < 1e-13
    if kind == "cx":       # printed form: P0 (x) I (x) I (x) I + P1 (x) X (x) X (x) X
        P0 = np.diag([1, 0]); P1 = np.diag([0, 1]); X = np.array([[0, 1], [1, 0]])
        ref = np.kron(P0, np.eye(8)) + np.kron(P1, np.kron(X, np.kron(X, X)))
        assert np.array_equal(u, ref)
        assert np.allclose(sigma, [2 * np.sqrt(2), 2 * np.sqrt(2)], atol=1e-13)
    # separate cuts would give 2^3 paths
    sep = 1
    for gg in gates:
        sep *= len(O.schmidt_decompose(O.gate_matrix(gg), 1, 1)[0])
    assert sep == g["separate_cut_paths"]


def test_joint_block_saturates_at_16_example3():
    # deep random circuit on 4 qubits, cut 2|2: joint rank saturates at 2^(2*2)
    rng = np.random.default_rng(11)
    gates = []
    for d in range(12):
        for q in range(4):
            gates.append(Gate("matrix", (q,), matrix=W.haar_u2(rng)))
        gates.append(Gate("cz", (3, 2)))
        gates.append(Gate("cz", (1, 0)))
        gates.append(Gate("cx", (2, 1)) if d % 2 == 0 else Gate("swap", (3, 0)))
    qs = O.block_qubits(gates, range(len(gates)))
    u = O.block_unitary(gates, range(len(gates)), qs)
    sigma, xs, ys = O.schmidt_decompose(u, 2, 2)
    assert len(sigma) == gold("fig3_ranks.json")["joint_2x2_saturation"]
    assert np.max(np.abs(O.schmidt_reconstruct(sigma, xs, ys) - u)) < 1e-13
    # per-gate cuts of the same block multiply the ranks instead: 2^6 * 4^6
    sep = 1
    for g in gates:
        if (max(g.qubits) >= 2) and (min(g.qubits) <= 1):
            sep *= len(O.schmidt_decompose(O.gate_matrix(g), 1, 1)[0])
    assert sep == 2 ** 6 * 4 ** 6


def test_rank_bound_and_frobenius_invariant():
    rng = np.random.default_rng(5)
    for trial in range(20):
        ka, kb = int(rng.integers(1, 3)), int(rng.integers(1, 4))
        k = ka + kb
        z = rng.standard_normal((1 << k, 1 << k)) + 1j * rng.standard_normal((1 << k, 1 << k))
        u, _ = np.linalg.qr(z)
        sigma, xs, ys = O.schmidt_decompose(u, ka, kb)
        assert len(sigma) <= min(4 ** ka, 4 ** kb)                       # Sec. IV-B
        assert abs(np.sum(sigma ** 2) - (1 << k)) < 1e-11                # ||U||_F^2 = 2^k
        assert np.max(np.abs(O.schmidt_reconstruct(sigma, xs, ys) - u)) < 1e-13
        # local unitaries on either side leave sigma unchanged
        la = np.linalg.qr(rng.standard_normal((1 << ka,) * 2) + 1j * rng.standard_normal((1 << ka,) * 2))[0]
        lb = np.linalg.qr(rng.standard_normal((1 << kb,) * 2) + 1j * rng.standard_normal((1 << kb,) * 2))[0]
        s2, _, _ = O.schmidt_decompose(np.kron(la, lb) @ u, ka, kb)
        assert np.allclose(s2, sigma, atol=1e-12)


def test_gate_definitions():
    t1, t2 = 0.37, 1.91
    r = lambda k, t: O.gate_matrix(Gate(k, (1, 0) if k == "rzz" else (0,), param=t))
    assert np.allclose(r("rzz", t1) @ r("rzz", t2), r("rzz", t1 + t2))
    assert np.allclose(r("rx", np.pi), -1j * np.array([[0, 1], [1, 0]]))
    assert np.allclose(r("rz", np.pi), np.diag([-1j, 1j]))
    for k in W.KINDS[1:]:
        nq = W.NQ[k]
        m = O.gate_matrix(Gate(k, tuple(range(nq)), param=0.4))
        assert np.allclose(m.conj().T @ m, np.eye(1 << nq), atol=1e-15)
    # first listed qubit is the most significant factor: CNOT(1,0)|10> = |11>
    psi = O.schrodinger(2, [Gate("x", (1,)), Gate("cx", (1, 0))])
    assert abs(psi[3] - 1) < 1e-15
    psi = O.schrodinger(2, [Gate("x", (1,)), Gate("cx", (0, 1))])
    assert abs(psi[2] - 1) < 1e-15
    # derivatives against central differences of the closed form
    for k in ("rx", "ry", "rz", "rzz"):
        g = Gate(k, (1, 0) if k == "rzz" else (0,), param=0.8)
        h = 1e-6
        gp = Gate(k, g.qubits, param=0.8 + h); gm = Gate(k, g.qubits, param=0.8 - h)
        fd = (O.gate_matrix(gp) - O.gate_matrix(gm)) / (2 * h)
        assert np.max(np.abs(fd - O.gate_derivative(g))) < 1e-9


@pytest.mark.parametrize("seed", range(6))
def test_schrodinger_vs_bruteforce(seed):
    n = 3 + seed % 4
    gates = W.random_circuit(n, 25, seed)
    psi = O.schrodinger(n, gates)
    u = O.circuit_unitary_bruteforce(n, gates)
    assert np.max(np.abs(u.conj().T @ u - np.eye(1 << n))) < 1e-12
    assert np.max(np.abs(psi - u[:, 0])) < 1e-13
    assert abs(np.linalg.norm(psi) - 1) < 1e-13


def _check_hsf_equals_schrodinger(pr, tol=1e-12):
    ref = O.schrodinger(pr.n, pr.gates)
    amps, info = O.hsf_amplitudes(pr.n, pr.gates, pr.cut, pr.blocks)
    assert np.max(np.abs(amps - ref)) < tol
    return info


def test_hsf_equals_schrodinger_c1_joint_and_plain():
    pr = W.workload_c1()
    info = _check_hsf_equals_schrodinger(pr)
    assert info["ranks"] == [2, 2]              # [CNOT, RZZ, CZ] on one pair: rank 2
    plain = W.singleton_blocks(pr.n, pr.gates, pr.cut)
    a_plain, ip = O.hsf_amplitudes(pr.n, pr.gates, pr.cut, plain)
    a_joint, _ = O.hsf_amplitudes(pr.n, pr.gates, pr.cut, pr.blocks)
    assert ip["num_paths"] == 64
    assert np.max(np.abs(a_plain - a_joint)) < 1e-12


@pytest.mark.parametrize("seed", range(4))
def test_hsf_equals_schrodinger_random_blocks(seed):
    pr = W.random_brickwork(10, 4, 6, block_after=(2, 4), block_kind="mixed", block_len=3,
                            seed=100 + seed)
    info = _check_hsf_equals_schrodinger(pr)
    assert all(r <= 4 for r in info["ranks"])
    # bitstring and window outputs agree with the full vector
    ref = O.schrodinger(pr.n, pr.gates)
    rng = np.random.default_rng(seed)
    bs = W.random_bitstrings(rng, pr.n, 50)
    a_bs, _ = O.hsf_amplitudes(pr.n, pr.gates, pr.cut, pr.blocks, bitstrings=bs)
    assert np.max(np.abs(a_bs - ref[bs.astype(np.int64)])) < 1e-12
    a_w, _ = O.hsf_amplitudes(pr.n, pr.gates, pr.cut, pr.blocks, window=77)
    assert np.max(np.abs(a_w - ref[:77])) < 1e-12


def test_hsf_path_ranges_partition_the_sum():
    pr = W.random_brickwork(8, 3, 5, block_after=(1, 3, 5), block_kind="rzz", block_len=2, seed=9)
    full, info = O.hsf_amplitudes(pr.n, pr.gates, pr.cut, pr.blocks)
    P = info["num_paths"]
    cuts = [0, 3, 17, P]
    parts = sum(O.hsf_amplitudes(pr.n, pr.gates, pr.cut, pr.blocks, path_range=(a, b))[0]
                for a, b in zip(cuts[:-1], cuts[1:]))
    assert np.max(np.abs(parts - full)) < 1e-13


def test_qaoa_ring_joint_vs_plain_and_two_qubit_cross_blocks():
    pr = W.qaoa_ring(10, 4, 2, seed=3)
    info = _check_hsf_equals_schrodinger(pr)
    assert info["ranks"] == [4, 4]              # two crossing RZZ per layer: rank 2 x 2
    plain = W.qaoa_ring(10, 4, 2, seed=3, joint=False)
    a, ip = O.hsf_amplitudes(plain.n, plain.gates, plain.cut, plain.blocks)
    assert ip["num_paths"] == 16
    assert np.max(np.abs(a - O.schrodinger(pr.n, pr.gates))) < 1e-12


def test_non_convex_and_missing_blocks_rejected():
    gates = [Gate("cx", (2, 1)), Gate("h", (1,)), Gate("cx", (2, 1))]
    with pytest.raises(ValueError):           # h(1) sits between two block gates
        O.hsf_amplitudes(3, gates, 1, [[0, 2]])
    with pytest.raises(ValueError):           # crossing gate 2 not in a block
        O.hsf_amplitudes(3, gates, 1, [[0]])


def test_table_path_identities():
    """Table I/II: joint paths = 2^(blocks + separate), standard = 2^(separate cuts).
    Every jointly cut group there is an RZZ cascade of Schmidt rank 2 (Sec. IV-D); the
    oracle reproduces rank 2 for RZZ stars of any size on either side."""
    t = gold("table_paths.json")
    for row in t["rows"]:
        name, q, cut, sizes, blocks, sep, sepcuts, lstd, ljoint = row
        assert sizes == [cut + 1, q - cut - 1]
        assert ljoint == blocks + sep
        assert lstd == sepcuts
    for leaves in (2, 3, 4):
        gates = [Gate("rzz", (leaves, j), param=0.3 + j) for j in range(leaves)]
        qs = O.block_qubits(gates, range(leaves))
        u = O.block_unitary(gates, range(leaves), qs)
        assert len(O.schmidt_decompose(u, 1, leaves)[0]) == 2


def test_fd_gradient_closed_form():
    # L = |<0|RX(t)|0>|^2 = cos^2(t/2), dL/dt = -sin(t)/2
    gates = [Gate("rx", (0,), param=0.0, param_id=0)]
    f = lambda th: O.loss_from_amplitudes(O.schrodinger(1, gates, th)[:1])
    for t in (0.2, 1.3, 2.9):
        g = O.fd_gradient(f, [t])
        assert abs(g[0] + np.sin(t) / 2) < 1e-9


def test_block_unitary_derivative():
    pr = W.qaoa_ring(6, 2, 1, seed=1)
    blk = pr.blocks[0]
    qs = O.block_qubits(pr.gates, blk)
    th = pr.params.copy()
    du = O.block_unitary(pr.gates, blk, qs, th, deriv_param=0)
    h = 1e-6
    tp = th.copy(); tp[0] += h
    tm = th.copy(); tm[0] -= h
    fd = (O.block_unitary(pr.gates, blk, qs, tp) - O.block_unitary(pr.gates, blk, qs, tm)) / (2 * h)
    assert np.max(np.abs(du - fd)) < 1e-9


# ---------------------------------------------------------------------------
# Planted mistakes: each plausible oracle bug must break at least one pin.
# ---------------------------------------------------------------------------

def _pins_pass():
    try:
        test_cnot_decomposition_example2()
        test_cascade_rank_example4("cx")
        test_hsf_equals_schrodinger_c1_joint_and_plain()
        return True
    except AssertionError:
        return False


def test_planted_mistakes_are_caught(monkeypatch):
    assert _pins_pass()
    real_svd = O.schmidt_decompose

    def wrong_reshuffle(a, ka, kb, tol=1e-12):     # forget the (i,j) regrouping
        s, xs, ys = real_svd(np.asarray(a).T, ka, kb, tol)
        return s, xs, ys
    monkeypatch.setattr(O, "schmidt_decompose", wrong_reshuffle)
    assert not _pins_pass()
    monkeypatch.undo()

    def dropped_conj(a, ka, kb, tol=1e-12):       # X_m from V instead of V^*
        s, xs, ys = real_svd(a, ka, kb, tol)
        return s, [x.conj() for x in xs], ys
    monkeypatch.setattr(O, "schmidt_decompose", dropped_conj)
    # CNOT factors are real; the C1 case with complex gates must catch it
    assert not _pins_pass()
    monkeypatch.undo()

    real_gm = O.gate_matrix

    def swapped_cx(g, theta=None):                 # control/target factors transposed
        m = real_gm(g, theta)
        if g.kind == "cx":
            P0 = np.diag([1, 0]).astype(complex); P1 = np.diag([0, 1]).astype(complex)
            X = np.array([[0, 1], [1, 0]], dtype=complex)
            return np.kron(np.eye(2), P0) + np.kron(X, P1)
        return m
    monkeypatch.setattr(O, "gate_matrix", swapped_cx)
    assert not _pins_pass()
    monkeypatch.undo()

    real_apply = O.apply_gate

    def reversed_qubits(psi, m, qubits, n):         # least significant qubit listed first
        return real_apply(psi, m, list(qubits)[::-1], n)
    monkeypatch.setattr(O, "apply_gate", reversed_qubits)
    assert not _pins_pass()
    monkeypatch.undo()
    assert _pins_pass()
