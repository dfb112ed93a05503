"""FP64 CPU oracle for joint-cutting Hybrid Schroedinger-Feynman (HSF) simulation.

TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the CPU-baseline
leg of the benchmark may import this module.  It shares no code with the CUDA path:
gate matrices, block products, the Schmidt decomposition, the path enumeration and the
path sum are all written out here, plainly and slowly, in float64/complex128.

What it computes (section / equation of Herzog et al., "Joint Cutting for Hybrid
Schroedinger-Feynman Simulation of Quantum Circuits"):

* ``schrodinger``      -- Sec. II-A, Example 1: consecutive matrix-vector products on
                          the 2^n statevector starting from |0...0>.
* ``circuit_unitary_bruteforce`` -- the same circuit as an explicit 2^n x 2^n matrix
                          product, built by index loops (independent of the above; n<=10).
* ``schmidt_decompose`` -- Sec. IV-A: relabel A_{ij} into A~_{(i^b j^b),(i^a j^a)}, take
                          its SVD (eq. eq-svd) and read X_m from V*, Y_m from U, so that
                          A = sum_m sigma_m X_m (x) Y_m (eq. equ-schmidt-decompostion-res).
* ``hsf_amplitudes``   -- Sec. II-B and III-A: cut between qubit l and l+1, Schmidt-
                          decompose every block (jointly cut gate group) and, for every
                          path (one Schmidt index per block), simulate both halves and add
                          sigma-weighted Kronecker products of the two half states.
* ``fd_gradient``      -- central finite differences of a loss sum_x |amp(x)|^2 with
                          respect to shared gate angles (for the adjoint-gradient checks).

Conventions: bit q of a basis index is qubit q (Sec. II-A, i = (i_{n-1} ... i_0));
the a side holds qubits l+1..n-1 and is the left (most significant) Kronecker factor,
the b side holds qubits 0..l (Sec. IV-A).  A gate on ordered qubits (q0, q1, ...) has its
matrix index in Kronecker order with q0 most significant (CNOT = P0 (x) I + P1 (x) X,
control first, Example 2).  Rotation angles: R_P(t) = exp(-i t P / 2).

Numerical-rank reading: the paper does not state a truncation threshold for the
Schmidt rank; singular values with sigma_m <= tol * sigma_0 (tol = 1e-12) are dropped,
which only removes exact zeros up to round-off.

Parity status: every function above is pinned by tests against closed forms,
worked examples of the paper, brute-force products and invariants.
"""
from __future__ import annotations

import heapq
import itertools
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

C128 = np.complex128

# ---------------------------------------------------------------------------
# Gate matrices (standard definitions; rotations R_P(t) = exp(-i t P / 2)).
# ---------------------------------------------------------------------------
_I2 = np.eye(2, dtype=C128)
_X = np.array([[0, 1], [1, 0]], dtype=C128)
_Y = np.array([[0, -1j], [1j, 0]], dtype=C128)
_Z = np.array([[1, 0], [0, -1]], dtype=C128)
_P0 = np.array([[1, 0], [0, 0]], dtype=C128)
_P1 = np.array([[0, 0], [0, 1]], dtype=C128)


def _rot(pauli: np.ndarray, t: float) -> np.ndarray:
    # exp(-i t P/2) = cos(t/2) I - i sin(t/2) P for any P with P^2 = I
    d = pauli.shape[0]
    return np.cos(t / 2) * np.eye(d, dtype=C128) - 1j * np.sin(t / 2) * pauli


def gate_matrix(g, theta: Optional[Sequence[float]] = None) -> np.ndarray:
    """Matrix of gate ``g`` (attributes kind, qubits, param, param_id, matrix)."""
    t = g.param
    if theta is not None and g.param_id >= 0:
        t = float(theta[g.param_id])
    k = g.kind
    if k == "matrix":
        m = np.asarray(g.matrix, dtype=C128)
        assert m.shape == (1 << len(g.qubits),) * 2
        return m
    if k == "h":
        return np.array([[1, 1], [1, -1]], dtype=C128) / np.sqrt(2)
    if k == "x":
        return _X.copy()
    if k == "y":
        return _Y.copy()
    if k == "z":
        return _Z.copy()
    if k == "s":
        return np.diag([1, 1j]).astype(C128)
    if k == "t":
        return np.diag([1, np.exp(1j * np.pi / 4)]).astype(C128)
    if k == "rx":
        return _rot(_X, t)
    if k == "ry":
        return _rot(_Y, t)
    if k == "rz":
        return _rot(_Z, t)
    if k == "cx":                                   # Example 2: P0 (x) I + P1 (x) X
        return np.kron(_P0, _I2) + np.kron(_P1, _X)
    if k == "cz":
        return np.kron(_P0, _I2) + np.kron(_P1, _Z)
    if k == "swap":
        m = np.zeros((4, 4), dtype=C128)
        for a in range(2):
            for b in range(2):
                m[(b << 1) | a, (a << 1) | b] = 1
        return m
    if k == "iswap":
        return np.array([[1, 0, 0, 0], [0, 0, 1j, 0], [0, 1j, 0, 0], [0, 0, 0, 1]], dtype=C128)
    if k == "rzz":
        return _rot(np.kron(_Z, _Z), t)
    raise ValueError(f"unknown gate kind {k!r}")


def gate_derivative(g, theta: Optional[Sequence[float]] = None) -> np.ndarray:
    """d/dt of a rotation gate exp(-i t P/2) = (-i/2) P exp(-i t P/2)."""
    paulis = {"rx": _X, "ry": _Y, "rz": _Z, "rzz": np.kron(_Z, _Z)}
    return -0.5j * paulis[g.kind] @ gate_matrix(g, theta)


# ---------------------------------------------------------------------------
# O1: Schroedinger-style simulation (Sec. II-A).
# ---------------------------------------------------------------------------

def apply_gate(psi: np.ndarray, m: np.ndarray, qubits: Sequence[int], n: int) -> np.ndarray:
    """psi <- (M on `qubits`) psi for a flat 2^n vector (bit q = qubit q)."""
    k = len(qubits)
    t = psi.reshape((2,) * n)                      # axis j <-> qubit n-1-j
    axes = [n - 1 - q for q in qubits]             # first listed qubit = most significant
    t = np.moveaxis(t, axes, list(range(k)))
    shp = t.shape
    t = (m @ t.reshape(1 << k, -1)).reshape(shp)
    t = np.moveaxis(t, list(range(k)), axes)
    return np.ascontiguousarray(t).reshape(-1)


def schrodinger(n: int, gates, theta=None) -> np.ndarray:
    psi = np.zeros(1 << n, dtype=C128)
    psi[0] = 1.0
    for g in gates:
        psi = apply_gate(psi, gate_matrix(g, theta), g.qubits, n)
    return psi


def embed_bruteforce(n: int, m: np.ndarray, qubits: Sequence[int]) -> np.ndarray:
    """Full 2^n x 2^n matrix of a gate, entry by entry: <i|G|j> = M[i|_q, j|_q] when i and j
    agree on every qubit outside `qubits`, else 0."""
    dim = 1 << n
    k = len(qubits)
    full = np.zeros((dim, dim), dtype=C128)
    mask = 0
    for q in qubits:
        mask |= 1 << q
    for i in range(dim):
        si = 0
        for pos, q in enumerate(qubits):
            si |= ((i >> q) & 1) << (k - 1 - pos)
        for sj in range(1 << k):
            j = i & ~mask
            for pos, q in enumerate(qubits):
                j |= ((sj >> (k - 1 - pos)) & 1) << q
            full[i, j] = m[si, sj]
    return full


def circuit_unitary_bruteforce(n: int, gates, theta=None) -> np.ndarray:
    u = np.eye(1 << n, dtype=C128)
    for g in gates:
        u = embed_bruteforce(n, gate_matrix(g, theta), g.qubits) @ u
    return u


# ---------------------------------------------------------------------------
# Blocks and the general Schmidt decomposition (Sec. IV-A).
# ---------------------------------------------------------------------------

def block_qubits(gates, block: Sequence[int]) -> List[int]:
    qs = set()
    for gi in block:
        qs.update(gates[gi].qubits)
    return sorted(qs, reverse=True)                 # most significant first


def block_unitary(gates, block: Sequence[int], qubits: Sequence[int], theta=None,
                  deriv_param: Optional[int] = None) -> np.ndarray:
    """Product of the block's gates in circuit order (later gates on the left), on the
    block's qubits ordered most significant first.  With ``deriv_param`` = j the result
    is d/d theta_j of that product (product rule over the gates tied to angle j)."""
    k = len(qubits)
    loc = {q: k - 1 - pos for pos, q in enumerate(qubits)}   # block-local bit position
    seq = [gates[gi] for gi in block]

    def emb(m, g):
        cols = []
        for c in range(1 << k):
            e = np.zeros(1 << k, dtype=C128)
            e[c] = 1
            cols.append(apply_gate(e, m, [loc[q] for q in g.qubits], k))
        return np.stack(cols, axis=1)

    if deriv_param is None:
        u = np.eye(1 << k, dtype=C128)
        for g in seq:
            u = emb(gate_matrix(g, theta), g) @ u
        return u
    total = np.zeros((1 << k, 1 << k), dtype=C128)
    for idx, g in enumerate(seq):
        if g.param_id != deriv_param:
            continue
        u = np.eye(1 << k, dtype=C128)
        for j, h in enumerate(seq):
            m = gate_derivative(h, theta) if j == idx else gate_matrix(h, theta)
            u = emb(m, h) @ u
        total += u
    return total


def schmidt_decompose(a: np.ndarray, k_a: int, k_b: int, tol: float = 1e-12):
    """Schmidt decomposition of an operator A on k_a (high) + k_b (low) qubits.

    A~_{(i^b, j^b), (i^a, j^a)} = A_{(i^a i^b), (j^a j^b)}; A~ = U diag(sigma) V^H
    (eq. eq-svd); Y_m[i^b, j^b] = U_{(i^b j^b), m} and X_m[i^a, j^a] = V^*_{m,(i^a j^a)},
    i.e. the m-th row of V^H.  Returns (sigma, X, Y) with sigma_m > tol * sigma_0 kept,
    so that A = sum_m sigma_m X_m (x) Y_m."""
    da, db = 1 << k_a, 1 << k_b
    a4 = np.asarray(a, dtype=C128).reshape(da, db, da, db)       # [i^a, i^b, j^a, j^b]
    at = a4.transpose(1, 3, 0, 2).reshape(db * db, da * da)     # rows (i^b, j^b), cols (i^a, j^a)
    u, s, vh = np.linalg.svd(at)
    if s.size == 0 or s[0] == 0.0:
        return np.zeros(0), [], []
    r = int(np.sum(s > tol * s[0]))
    xs = [vh[m, :].reshape(da, da) for m in range(r)]
    ys = [u[:, m].reshape(db, db) for m in range(r)]
    return s[:r].copy(), xs, ys


def schmidt_reconstruct(sigma, xs, ys) -> np.ndarray:
    out = 0
    for s, x, y in zip(sigma, xs, ys):
        out = out + s * np.kron(x, y)
    return out


# ---------------------------------------------------------------------------
# O2: HSF path sum (Sec. II-B, III-A, IV-A).
# ---------------------------------------------------------------------------

def classify(n: int, gates, cut: int):
    side = []
    for g in gates:
        hi = [q > cut for q in g.qubits]
        side.append("a" if all(hi) else "b" if not any(hi) else "x")
    return side


def execution_order(n: int, gates, blocks: Sequence[Sequence[int]]):
    """A topological order of the circuit DAG in which every block is one unit.

    Raises ValueError when a block is not convex (a DAG path leaves it and comes back)
    or when the listed block order contradicts the circuit's dependencies."""
    owner = {}
    for b, blk in enumerate(blocks):
        for gi in blk:
            if gi in owner:
                raise ValueError(f"gate {gi} in two blocks")
            owner[gi] = b
    node_of = lambda gi: ("b", owner[gi]) if gi in owner else ("g", gi)
    preds: Dict[tuple, set] = {}
    succs: Dict[tuple, set] = {}
    last_on = {}
    nodes = set()
    for gi, g in enumerate(gates):
        v = node_of(gi)
        nodes.add(v)
        preds.setdefault(v, set())
        succs.setdefault(v, set())
        for q in g.qubits:
            if q in last_on:
                u = node_of(last_on[q])
                if u != v:
                    preds[v].add(u)
                    succs.setdefault(u, set()).add(v)
            last_on[q] = gi
    key = {}
    for v in nodes:
        key[v] = min(blocks[v[1]]) if v[0] == "b" else v[1]
    indeg = {v: len(preds[v]) for v in nodes}
    heap = [(key[v], v) for v in nodes if indeg[v] == 0]
    heapq.heapify(heap)
    order = []
    while heap:
        _, v = heapq.heappop(heap)
        order.append(v)
        for w in succs.get(v, ()):
            indeg[w] -= 1
            if indeg[w] == 0:
                heapq.heappush(heap, (key[w], w))
    if len(order) != len(nodes):
        raise ValueError("a block is not convex in the circuit DAG")
    # the listed block order must be compatible with the dependencies between blocks
    reach = {}
    for v in reversed(order):
        r = set()
        for w in succs.get(v, ()):
            r.add(w)
            r |= reach[w]
        reach[v] = r
    for b1 in range(len(blocks)):
        for b2 in range(b1):
            if ("b", b2) in reach[("b", b1)]:
                raise ValueError("blocks are not listed in an order compatible with the circuit")
    return order


def decompose_blocks(n: int, gates, cut: int, blocks, theta=None, tol=1e-12):
    """Per block: its qubits, its a/b split and its Schmidt terms."""
    side = classify(n, gates, cut)
    seen = set()
    for blk in blocks:
        if not any(side[gi] == "x" for gi in blk):
            raise ValueError("a block must contain a gate crossing the cut")
        seen.update(blk)
    for gi, s in enumerate(side):
        if s == "x" and gi not in seen:
            raise ValueError(f"crossing gate {gi} is not in any block")
    out = []
    for blk in blocks:
        qs = block_qubits(gates, blk)
        qa = [q for q in qs if q > cut]
        qb = [q for q in qs if q <= cut]
        u = block_unitary(gates, blk, qs, theta)
        sigma, xs, ys = schmidt_decompose(u, len(qa), len(qb), tol)
        out.append(dict(qubits=qs, qa=qa, qb=qb, u=u, sigma=sigma, x=xs, y=ys))
    return out


def hsf_amplitudes(n: int, gates, cut: int, blocks, bitstrings=None, window: int = 0,
                   path_range: Optional[Tuple[int, int]] = None, theta=None,
                   tol: float = 1e-12, decomposition=None):
    """O2: amp = sum over paths p of prod_k sigma_{m_k} psi_a^p(x_a) psi_b^p(x_b).

    Paths are tuples (m_0, ..., m_{B-1}) in mixed radix with block 0 most significant;
    ``path_range`` = (p0, p1) restricts the sum to p0 <= p < p1.  Output: the amplitudes
    at ``bitstrings`` (uint64, bit q = qubit q), else the first ``window`` amplitudes,
    else all 2^n.  Returns (amplitudes, info)."""
    order = execution_order(n, gates, blocks)
    dec = decomposition if decomposition is not None else decompose_blocks(n, gates, cut, blocks, theta, tol)
    side = classify(n, gates, cut)
    na, nb = n - cut - 1, cut + 1
    ranks = [len(d["sigma"]) for d in dec]
    total = int(np.prod(ranks)) if ranks else 1
    p0, p1 = (0, total) if path_range is None else path_range
    if bitstrings is not None:
        xs = np.asarray(bitstrings, dtype=np.uint64)
        xa = (xs >> np.uint64(nb)).astype(np.int64)
        xb = (xs & np.uint64((1 << nb) - 1)).astype(np.int64)
        out = np.zeros(len(xs), dtype=C128)
    else:
        count = (1 << n) if window == 0 else window
        out = np.zeros(count, dtype=C128)
    mats = [None if side[gi] == "x" else gate_matrix(g, theta) for gi, g in enumerate(gates)]

    def half(path, which):
        nq = na if which == "a" else nb
        off = cut + 1 if which == "a" else 0
        psi = np.zeros(1 << nq, dtype=C128)
        psi[0] = 1.0
        for kind, idx in order:
            if kind == "g":
                if side[idx] == which:
                    psi = apply_gate(psi, mats[idx], [q - off for q in gates[idx].qubits], nq)
            else:
                d = dec[idx]
                m = path[idx]
                if which == "a":
                    psi = apply_gate(psi, d["x"][m], [q - off for q in d["qa"]], nq)
                else:
                    psi = apply_gate(psi, d["y"][m], [q - off for q in d["qb"]], nq)
        return psi

    for p, path in enumerate(itertools.product(*[range(r) for r in ranks])):
        if p < p0 or p >= p1:
            continue
        w = 1.0
        for k, m in enumerate(path):
            w *= dec[k]["sigma"][m]
        pa = half(path, "a")
        pb = half(path, "b")
        if bitstrings is not None:
            out += w * pa[xa] * pb[xb]
        else:
            full = w * np.outer(pa, pb).reshape(-1)   # index x_a * 2^{n_b} + x_b
            out += full[:len(out)]
    info = dict(ranks=ranks, num_paths=total, sigma=[d["sigma"] for d in dec], n_a=na, n_b=nb)
    return out, info


# ---------------------------------------------------------------------------
# O3: loss and finite-difference gradient.
# ---------------------------------------------------------------------------

def loss_from_amplitudes(amps: np.ndarray) -> float:
    return float(np.sum(np.abs(amps) ** 2))


def fd_gradient(loss_fn, theta: Sequence[float], h: float = 1e-5) -> np.ndarray:
    """Central differences g_j = (L(t + h e_j) - L(t - h e_j)) / 2h, error O(h^2)."""
    theta = np.asarray(theta, dtype=np.float64)
    g = np.zeros_like(theta)
    for j in range(theta.size):
        tp = theta.copy(); tp[j] += h
        tm = theta.copy(); tm[j] -= h
        g[j] = (loss_fn(tp) - loss_fn(tm)) / (2 * h)
    return g
