"""Pins of the C Schroedinger oracle (oracle/schrodinger.c, Sec. II-A) against what the
paper and the mathematics fix, independently of its own code:

* the Bell state of Example 1 (tests/golden/bell_state.json);
* the first column of the circuit unitary built entry by entry with index loops
  (``circuit_unitary_bruteforce``, n <= 6), over every supported gate kind;
* unitarity: the norm stays 1 on a 20-qubit random circuit;
* 3-qubit gates and qubit order: a CCX-like explicit 8 x 8 matrix on permuted qubits;
* planted mistakes (a transposed matrix, swapped operand order) are caught by the pins.
"""
import json
import os

import numpy as np
import pytest

import oracle.hsf_oracle as O
from oracle import schrodinger_c as SC
from paper_2502_06959_gb300 import workloads as W
from paper_2502_06959_gb300.workloads import Gate

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_bell_state_example1():
    rec = json.load(open(os.path.join(GOLDEN, "bell_state.json")))
    gates = [Gate(k, tuple(q)) for k, q in rec["gates"]]
    psi = SC.schrodinger_c(rec["n"], gates)
    want = np.array(rec["amplitudes_re"]) + 1j * np.array(rec["amplitudes_im"])
    assert np.max(np.abs(psi - want)) < 1e-15


@pytest.mark.parametrize("seed", range(6))
def test_against_bruteforce_unitary(seed):
    n = 3 + seed % 4
    gates = W.random_circuit(n, 40, seed=100 + seed)
    u = O.circuit_unitary_bruteforce(n, gates)
    psi = SC.schrodinger_c(n, gates)
    assert np.max(np.abs(psi - u[:, 0])) < 1e-13


def test_three_qubit_matrix_gate_and_order():
    rng = np.random.default_rng(5)
    z = rng.standard_normal((8, 8)) + 1j * rng.standard_normal((8, 8))
    q, r = np.linalg.qr(z)
    m = q * (np.diag(r) / np.abs(np.diag(r)))
    gates = [Gate("h", (0,)), Gate("h", (3,)), Gate("matrix", (4, 0, 2), matrix=m), Gate("cx", (2, 1))]
    u = O.circuit_unitary_bruteforce(5, gates)
    psi = SC.schrodinger_c(5, gates)
    assert np.max(np.abs(psi - u[:, 0])) < 1e-14


def test_norm_is_kept():
    gates = W.random_brickwork(20, 9, 6, block_after=(2, 4), block_kind="mixed", block_len=3, seed=8).gates
    psi = SC.schrodinger_c(20, gates)
    assert abs(np.linalg.norm(psi) - 1.0) < 1e-13


def test_planted_mistakes_are_caught():
    n = 4
    gates = W.random_circuit(n, 30, seed=71)   # holds a 2-qubit matrix and a CNOT
    u = O.circuit_unitary_bruteforce(n, gates)
    good = SC.schrodinger_c(n, gates)
    assert np.max(np.abs(good - u[:, 0])) < 1e-13
    # a transposed matrix on one gate
    bad = [Gate(g.kind, g.qubits, g.param, g.param_id, g.matrix) for g in gates]
    i = next(j for j, g in enumerate(bad) if g.kind == "matrix" and len(g.qubits) == 2)
    bad[i] = Gate("matrix", bad[i].qubits, matrix=np.asarray(bad[i].matrix).T.copy())
    assert np.max(np.abs(SC.schrodinger_c(n, bad) - u[:, 0])) > 1e-3
    # operand order of a CNOT reversed
    bad = list(gates)
    i = next(j for j, g in enumerate(bad) if g.kind == "cx")
    bad[i] = Gate("cx", tuple(reversed(bad[i].qubits)))
    assert np.max(np.abs(SC.schrodinger_c(n, bad) - u[:, 0])) > 1e-3


def test_rejects_bad_circuits():
    with pytest.raises(ValueError):
        SC.schrodinger_c(3, [Gate("cx", (1, 1))])
    with pytest.raises(ValueError):
        SC.schrodinger_c(3, [Gate("h", (3,))])
