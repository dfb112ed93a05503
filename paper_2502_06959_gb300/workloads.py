"""Seeded synthetic inputs for joint-cut HSF simulation.

This module only draws inputs: gate lists, cut positions, block memberships and
bitstrings.  It holds none of the method's arithmetic (no gate matrices other than
the Haar-random U(2) inputs themselves, no Schmidt decomposition, no simulation), so
both the FP64 oracle and the CUDA path can consume what it produces.

Circuit convention (Sec. II-A): bit q of a basis index is qubit q.  A gate on the
ordered qubits (q0, q1, ...) has its matrix row/column index in Kronecker order with
q0 as the most significant factor, so ``cx`` on (c, t) is P0 (x) I + P1 (x) X with the
control listed first (Example 2).

Angle conventions: rx/ry/rz(t) = exp(-i t P / 2), rzz(t) = exp(-i t Z(x)Z / 2).

The workload builders follow the shapes of the method's evaluation (Sec. V, Tables I
and II) and of the synthetic configurations named by the project:

* ``random_brickwork`` -- Haar-random U(2) layers, CZ brickwork inside each half, and
  jointly cut blocks on the two qubits next to the cut.
* ``qaoa_ring`` -- QAOA-style problem (RZZ on a ring) and mixer (RX) layers with the two
  ring edges that cross the cut collected into one block per layer (Sec. V).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Sequence, Tuple

import numpy as np

KINDS = ("matrix", "h", "x", "y", "z", "s", "t", "rx", "ry", "rz",
         "cx", "cz", "swap", "iswap", "rzz")
PARAM_KINDS = ("rx", "ry", "rz", "rzz")
NQ = {"h": 1, "x": 1, "y": 1, "z": 1, "s": 1, "t": 1, "rx": 1, "ry": 1, "rz": 1,
      "cx": 2, "cz": 2, "swap": 2, "iswap": 2, "rzz": 2}


@dataclass
class Gate:
    kind: str
    qubits: Tuple[int, ...]
    param: float = 0.0
    param_id: int = -1                      # index into a shared angle vector, -1 = fixed
    matrix: Optional[np.ndarray] = None     # complex (2^k, 2^k) for kind == "matrix"


@dataclass
class Problem:
    """A circuit, its horizontal cut and its cut blocks (lists of gate indices)."""
    n: int
    gates: List[Gate]
    cut: int                                # cut after qubit `cut`: b = {0..cut}, a = {cut+1..n-1}
    blocks: List[List[int]]
    name: str = ""
    bitstrings: Optional[np.ndarray] = None  # uint64, bit q = qubit q
    num_params: int = 0
    params: Optional[np.ndarray] = None
    meta: dict = field(default_factory=dict)


def haar_u2(rng: np.random.Generator) -> np.ndarray:
    """Haar-random 2x2 unitary: QR of a complex Ginibre matrix with the phase fix
    of Mezzadri (2007)."""
    z = (rng.standard_normal((2, 2)) + 1j * rng.standard_normal((2, 2))) / np.sqrt(2.0)
    q, r = np.linalg.qr(z)
    d = np.diag(r)
    return q * (d / np.abs(d))


def random_bitstrings(rng: np.random.Generator, n: int, count: int) -> np.ndarray:
    hi = rng.integers(0, 1 << 32, size=count, dtype=np.uint64)
    lo = rng.integers(0, 1 << 32, size=count, dtype=np.uint64)
    x = (hi << np.uint64(32)) | lo
    if n < 64:
        x &= np.uint64((1 << n) - 1)
    return x


def singleton_blocks(n: int, gates: Sequence[Gate], cut: int) -> List[List[int]]:
    """Plain (per-gate) cut: every gate that crosses the cut is its own block."""
    out = []
    for i, g in enumerate(gates):
        qs = g.qubits
        if any(q > cut for q in qs) and any(q <= cut for q in qs):
            out.append([i])
    return out


def _u2_layer(rng, gates, qubits):
    for q in qubits:
        gates.append(Gate("matrix", (q,), matrix=haar_u2(rng)))


def _cz_brickwork(gates, n, cut, parity):
    for q in range(parity, n - 1, 2):
        if q == cut:            # never across the cut
            continue
        gates.append(Gate("cz", (q + 1, q)))


def random_brickwork(n: int, cut: int, layers: int, block_after: Sequence[int],
                     block_kind: str, block_len: int, seed: int,
                     num_bitstrings: int = 0, name: str = "",
                     block_u2: bool = True, alt_cx: bool = False) -> Problem:
    """Layers of Haar U(2) on every qubit followed by CZ brickwork inside each half.

    After each layer index in ``block_after`` one block on the cut pair (cut+1, cut)
    is inserted.  ``block_kind``:

    * ``"rzz"`` -- ``block_len`` RZZ(theta ~ U[0, 2 pi)) gates; with ``block_u2`` a
      Haar U(2) on both block qubits sits between consecutive RZZs and belongs to the
      block (the block then has Schmidt rank 4 generically).
    * ``"cx_rzz_cz"`` -- the three gates [CNOT, RZZ(theta), CZ]; the CNOT control
      alternates between the two sides when ``alt_cx`` is set.
    * ``"mixed"`` -- ``block_len`` gates drawn from RZZ / CNOT with interleaved U(2).
    """
    rng = np.random.default_rng(seed)
    gates: List[Gate] = []
    blocks: List[List[int]] = []
    qa, qb = cut + 1, cut
    for layer in range(layers):
        _u2_layer(rng, gates, range(n))
        _cz_brickwork(gates, n, cut, layer % 2)
        if layer + 1 in block_after:
            blk = []
            if block_kind == "cx_rzz_cz":
                k = len(blocks)
                ctl, tgt = ((qa, qb) if (not alt_cx or k % 2 == 0) else (qb, qa))
                blk.append(len(gates)); gates.append(Gate("cx", (ctl, tgt)))
                blk.append(len(gates)); gates.append(Gate("rzz", (qa, qb), param=float(rng.uniform(0, 2 * np.pi))))
                blk.append(len(gates)); gates.append(Gate("cz", (qa, qb)))
            else:
                for j in range(block_len):
                    if block_kind == "rzz" or (block_kind == "mixed" and rng.random() < 0.5):
                        blk.append(len(gates))
                        gates.append(Gate("rzz", (qa, qb), param=float(rng.uniform(0, 2 * np.pi))))
                    else:
                        pair = (qa, qb) if rng.random() < 0.5 else (qb, qa)
                        blk.append(len(gates)); gates.append(Gate("cx", pair))
                    if block_u2 and j + 1 < block_len:
                        for q in (qa, qb):
                            blk.append(len(gates)); gates.append(Gate("matrix", (q,), matrix=haar_u2(rng)))
            blocks.append(blk)
    bs = random_bitstrings(rng, n, num_bitstrings) if num_bitstrings else None
    return Problem(n=n, gates=gates, cut=cut, blocks=blocks, name=name, bitstrings=bs,
                   meta=dict(seed=seed, layers=layers, block_after=list(block_after),
                             block_kind=block_kind, block_len=block_len))


def qaoa_ring(n: int, cut: int, p: int, seed: int, num_bitstrings: int = 0,
              name: str = "", joint: bool = True) -> Problem:
    """QAOA Max-Cut on a ring (Sec. V): H on every qubit, then p x [RZZ(gamma_l) on each
    ring edge (i, i+1 mod n); RX(beta_l) on every qubit].  The two ring edges that cross
    the cut, (cut, cut+1) and (n-1, 0), form one block per layer (joint cut); with
    ``joint=False`` each is its own block.  Angles are shared per layer through
    ``param_id``: gamma_l has id l, beta_l has id p + l."""
    rng = np.random.default_rng(seed)
    gammas = rng.uniform(0, 2 * np.pi, size=p)
    betas = rng.uniform(0, 2 * np.pi, size=p)
    gates: List[Gate] = [Gate("h", (q,)) for q in range(n)]
    blocks: List[List[int]] = []
    edges = [(i, (i + 1) % n) for i in range(n)]
    crossing = [e for e in edges if min(e) <= cut < max(e)]
    inside = [e for e in edges if not (min(e) <= cut < max(e))]
    for l in range(p):
        # RZZ gates commute, so the crossing edges go first in each problem layer; the
        # block made of them is then convex in the gate DAG (Sec. V, Fig. 6).
        blk = []
        for (i, j) in crossing:
            blk.append(len(gates))
            gates.append(Gate("rzz", (i, j), param=float(gammas[l]), param_id=l))
        for (i, j) in inside:
            gates.append(Gate("rzz", (i, j), param=float(gammas[l]), param_id=l))
        if joint:
            blocks.append(blk)
        else:
            blocks.extend([[b] for b in blk])
        for q in range(n):
            gates.append(Gate("rx", (q,), param=float(betas[l]), param_id=p + l))
    bs = random_bitstrings(rng, n, num_bitstrings) if num_bitstrings else None
    params = np.concatenate([gammas, betas])
    return Problem(n=n, gates=gates, cut=cut, blocks=blocks, name=name, bitstrings=bs,
                   num_params=2 * p, params=params, meta=dict(seed=seed, p=p))


def sbm_graph(sizes: Sequence[int], p_intra: float, p_inter: float, seed: int) -> List[Tuple[int, int]]:
    """Edges of a two-block stochastic block model graph (Table II: vertices of the two
    partitions joined with probability p_intra inside a partition and p_inter between
    them).  Vertices 0..sizes[0]-1 form the first partition; each pair (i < j) is drawn
    once, in lexicographic order."""
    rng = np.random.default_rng(seed)
    n = int(sum(sizes))
    part = np.concatenate([np.full(int(s), k) for k, s in enumerate(sizes)])
    edges = []
    for i in range(n):
        for j in range(i + 1, n):
            pr = p_intra if part[i] == part[j] else p_inter
            if rng.random() < pr:
                edges.append((i, j))
    return edges


def sbm_qaoa(sizes: Sequence[int] = (15, 15), p_intra: float = 0.8, p_inter: float = 0.1, seed: int = 0,
             name: str = "") -> Problem:
    """Single-layer QAOA Max-Cut on a stochastic-block-model graph (Sec. V, Table II):
    H on every qubit, RZZ(gamma) on every edge (in the generator's edge order, crossing
    and in-half edges interleaved), RX(beta) on every qubit.  Qubit q is vertex q; the cut
    lies after the first partition (Table II "cut pos." = sizes[0] - 1).  The angles are
    drawn from U[0, 2 pi) and shared through param_id (gamma: 0, beta: 1).  The blocks are
    left empty: ``hsf.problem_with_found_blocks`` (or singleton blocks) fills them."""
    rng = np.random.default_rng(seed + 7919)
    gamma, beta = (float(x) for x in rng.uniform(0, 2 * np.pi, size=2))
    n = int(sum(sizes))
    edges = sbm_graph(sizes, p_intra, p_inter, seed)
    gates: List[Gate] = [Gate("h", (q,)) for q in range(n)]
    for (i, j) in edges:
        gates.append(Gate("rzz", (j, i), param=gamma, param_id=0))
    for q in range(n):
        gates.append(Gate("rx", (q,), param=beta, param_id=1))
    cut = int(sizes[0]) - 1
    crossing = sum(1 for (i, j) in edges if i <= cut < j)
    return Problem(n=n, gates=gates, cut=cut, blocks=[], name=name or f"sbm_q{n}_pinter{p_inter}",
                   num_params=2, params=np.array([gamma, beta]),
                   meta=dict(seed=seed, sizes=list(sizes), p_intra=p_intra, p_inter=p_inter,
                             edges=len(edges), crossing=crossing, two_qubit_gates=len(edges)))


# ---------------------------------------------------------------------------
# The five named workloads (sizes fixed here, seeds fixed per workload).
# ---------------------------------------------------------------------------

def workload_c1(seed: int = 1) -> Problem:
    """n=12, split 6|6, 8 layers of Haar U(2) + in-half CZ brickwork, 2 blocks on (5,6),
    each [CNOT, RZZ(theta), CZ] with alternating CNOT orientation; all 4096 amplitudes."""
    return random_brickwork(12, 5, 8, block_after=(2, 6), block_kind="cx_rzz_cz",
                            block_len=3, seed=seed, name="c1_n12_full", alt_cx=True)


def workload_c2(seed: int = 2, num_blocks: int = 8, layers: int = 20,
                num_bitstrings: int = 4096) -> Problem:
    """n=30, split 15|15, 20 layers, 8 blocks of 4 RZZ on (14,15) with interleaved U(2)
    (rank 4 each, 4^8 = 65536 joint paths vs 2^32 per-gate paths); 4096 bitstrings."""
    after = tuple(2 * (k + 1) for k in range(num_blocks))
    return random_brickwork(30, 14, layers, block_after=after, block_kind="rzz",
                            block_len=4, seed=seed, num_bitstrings=num_bitstrings,
                            name="c2_n30_bitstrings")


def workload_c3(seed: int = 3, count: int = 64, n_choices=(20, 22, 24, 26, 28, 30, 32),
                layers: int = 8, max_paths: int = 4096) -> List[Problem]:
    """64 circuits of uneven size: n uniform over the even values in [20, 32], cut at
    n/2 - 1, 8 layers, 2-6 blocks of 2-5 RZZ/CNOT gates with interleaved U(2); the block
    count is capped so that the joint path count stays within 16..4096."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(rng.choice(n_choices))
        nb = int(rng.integers(2, 7))
        blen = int(rng.integers(2, 6))
        # block k has rank <= 4 (one qubit on each side), so 4^nb <= max_paths
        nb = max(2, min(nb, int(np.floor(np.log(max_paths) / np.log(4)))))
        after = sorted(int(x) for x in rng.choice(np.arange(1, layers + 1), size=nb, replace=False))
        pr = random_brickwork(n, n // 2 - 1, layers, block_after=tuple(after), block_kind="mixed",
                              block_len=blen, seed=int(rng.integers(1 << 31)),
                              name=f"c3_{i}_n{n}")
        out.append(pr)
    return out


def workload_c3_largest(seed: int = 3) -> Problem:
    """The largest circuit of ``workload_c3`` (most qubits, then most blocks): the one
    whose window path GEMM is timed on its own."""
    return max(workload_c3(seed=seed), key=lambda q: (q.n, len(q.blocks)))


def window_samples(n: int, window: int, count: int, seed: int) -> np.ndarray:
    """``count`` distinct seeded indices below min(window, 2^n) (uint64), sorted."""
    rng = np.random.default_rng(seed)
    top = min(window, 1 << n)
    return np.sort(rng.choice(top, size=min(count, top), replace=False)).astype(np.uint64)


def workload_c4(seed: int = 4, n: int = 28, p: int = 4, num_bitstrings: int = 1024,
                joint: bool = True) -> Problem:
    """QAOA ring, n=28, split 14|14, p=4, the 2 crossing ring edges jointly cut per
    layer; loss = sum |amp(x)|^2 over 1024 bitstrings."""
    return qaoa_ring(n, n // 2 - 1, p, seed, num_bitstrings=num_bitstrings,
                     name=f"c4_qaoa_n{n}_p{p}", joint=joint)


def workload_c5(seed: int = 5, num_blocks: int = 12, layers: int = 24,
                num_bitstrings: int = 1 << 20) -> Problem:
    """n=36, split 18|18, 24 layers, 12 blocks of 3 RZZ on (17,18) with interleaved
    U(2); 2^20 bitstrings."""
    after = tuple(2 * (k + 1) for k in range(num_blocks))
    return random_brickwork(36, 17, layers, block_after=after, block_kind="rzz",
                            block_len=3, seed=seed, num_bitstrings=num_bitstrings,
                            name="c5_n36_bitstrings")


def random_circuit(n: int, num_gates: int, seed: int, kinds=None) -> List[Gate]:
    """Random gate list over all supported kinds (for small parity cases)."""
    rng = np.random.default_rng(seed)
    kinds = kinds or ["matrix", "h", "x", "y", "z", "s", "t", "rx", "ry", "rz",
                      "cx", "cz", "swap", "iswap", "rzz", "matrix2"]
    gates = []
    for _ in range(num_gates):
        k = kinds[int(rng.integers(len(kinds)))]
        if k == "matrix2":
            qs = tuple(int(x) for x in rng.choice(n, size=2, replace=False))
            a = haar_u2(rng); b = haar_u2(rng)
            # a generic 2-qubit unitary: (a (x) b) . CZ . (c (x) d) written out as data
            z = (rng.standard_normal((4, 4)) + 1j * rng.standard_normal((4, 4)))
            q, r = np.linalg.qr(z)
            m = q * (np.diag(r) / np.abs(np.diag(r)))
            gates.append(Gate("matrix", qs, matrix=m))
            continue
        nq = 1 if k == "matrix" else NQ[k]
        qs = tuple(int(x) for x in rng.choice(n, size=nq, replace=False))
        if k == "matrix":
            gates.append(Gate("matrix", qs, matrix=haar_u2(rng)))
        elif k in PARAM_KINDS:
            gates.append(Gate(k, qs, param=float(rng.uniform(0, 2 * np.pi))))
        else:
            gates.append(Gate(k, qs))
    return gates
