"""Closed-form cascade decompositions (Sec. IV-D, Example 4) against the SVD route.

A block whose gates, where they touch the block's qubits on one side (the hub), are all
diagonal there gets its terms P_z (x) Y_z without an SVD.  The tests check that the plan
takes that route exactly for such blocks, that its rank equals the Schmidt rank (2 for a
one-qubit hub: C_CNOT,3 of Example 4 and the CZ / RZZ cascades), that the term weights
keep sum sigma^2 = 2^k (the Frobenius norm of a unitary block), and that amplitudes and
gradients equal the oracle's and the SVD-forced plan's.
"""
import numpy as np
import pytest

import oracle.hsf_oracle as O
from paper_2502_06959_gb300 import workloads as W
from paper_2502_06959_gb300.workloads import Gate

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2502_06959_gb300 import build
    build.build()
    from paper_2502_06959_gb300 import hsf
    hsf.load_library()


def _plan(pr, **opts):
    from paper_2502_06959_gb300 import hsf
    plan = hsf.Plan.from_problem(pr, **opts)
    desc = hsf.hsf_plan_describe(plan.handle)
    return plan, [l for l in desc.splitlines() if l.startswith("block ")]


def cascade_problem(kind, hub_side, seed):
    """n = 10 (cut after qubit 4): Haar layers, then a cascade of three gates from one hub
    qubit next to the cut to three qubits on the other side, then more layers."""
    rng = np.random.default_rng(seed)
    n, cut = 10, 4
    gates = []
    for q in range(n):
        gates.append(Gate("matrix", (q,), matrix=W.haar_u2(rng)))
    W._cz_brickwork(gates, n, cut, 0)
    hub = 5 if hub_side == "a" else 4
    leaves = [4, 3, 2] if hub_side == "a" else [5, 6, 7]
    blk = []
    for t in leaves:
        blk.append(len(gates))
        if kind == "cx":
            gates.append(Gate("cx", (hub, t)))
        elif kind == "cz":
            gates.append(Gate("cz", (t, hub)))
        else:
            gates.append(Gate("rzz", (hub, t), param=float(rng.uniform(0, 2 * np.pi))))
    for q in range(n):
        gates.append(Gate("matrix", (q,), matrix=W.haar_u2(rng)))
    W._cz_brickwork(gates, n, cut, 1)
    return W.Problem(n=n, gates=gates, cut=cut, blocks=[blk], name=f"cascade_{kind}_{hub_side}")


@pytest.mark.parametrize("kind", ["cx", "cz", "rzz"])
@pytest.mark.parametrize("hub_side", ["a", "b"])
def test_cascade_rank_two_and_amplitudes(kind, hub_side):
    pr = cascade_problem(kind, hub_side, seed=3)
    ref = O.schrodinger(pr.n, pr.gates)
    plan, lines = _plan(pr, precision="c128")
    assert len(lines) == 1 and "closed-form cascade" in lines[0] and f"side {hub_side}" in lines[0], lines
    sig = plan.sigma(0)
    assert sig.size == 2                                     # Example 4: rank 2 for any length
    assert abs(np.sum(sig ** 2) - 2 ** 4) < 1e-12            # |U_B|_F^2 = 2^k, k = 4 qubits
    got = plan.run().cpu().numpy()
    plan.close()
    assert np.max(np.abs(got - ref)) <= 1e-12
    from paper_2502_06959_gb300 import hsf
    svd, lines = _plan(pr, precision="c128", flags=hsf.FLAG_SVD_BLOCKS)
    assert "SVD" in lines[0]
    assert svd.sigma(0).size == 2
    got2 = svd.run().cpu().numpy()
    svd.close()
    assert np.max(np.abs(got2 - ref)) <= 1e-12


def test_c1_blocks_are_closed_form():
    pr = W.workload_c1()
    ref = O.schrodinger(pr.n, pr.gates)
    for prec, tol in (("c128", 1e-12), ("c64", 1e-5)):
        plan, lines = _plan(pr, precision=prec)
        assert len(lines) == 2 and all("closed-form" in l for l in lines), lines
        got = plan.run(check=True).cpu().numpy()
        plan.close()
        assert np.max(np.abs(got - ref)) <= tol


def test_non_diagonal_hub_gate_uses_the_svd():
    pr = W.workload_c2(num_bitstrings=8)
    plan, lines = _plan(pr)
    plan.close()
    assert len(lines) == 8 and all("SVD" in l for l in lines), lines


def test_qaoa_two_edge_blocks_rank_four_and_gradients():
    """C4-shaped blocks (two crossing RZZ per layer: a two-qubit hub, 4 terms) at n = 12:
    amplitudes and the adjoint gradient (block angles included) agree with the SVD route
    and with the oracle's central differences."""
    import torch
    from paper_2502_06959_gb300 import hsf
    pr = W.qaoa_ring(12, 5, 2, seed=6, num_bitstrings=64)
    plan, lines = _plan(pr, precision="c128")
    assert len(lines) == 2 and all("closed-form" in l and "rank 4" in l for l in lines), lines
    plan.close()
    bits = torch.from_numpy(pr.bitstrings.view(np.int64)).cuda()

    def loss_and_grad(flags):
        theta = torch.tensor(pr.params, dtype=torch.float64, requires_grad=True)
        amps = hsf.HSFAmplitudes.apply(theta, pr, bits, "c128") if not flags else None
        if flags:
            p = hsf.Plan.from_problem(pr, precision="c128", flags=flags, angles=pr.params)
            a = p.run(bits)
            g = p.grad(bits, 2 * a, pr.num_params).cpu().numpy()
            p.close()
            return float((a.abs() ** 2).sum()), g
        loss = (amps.abs() ** 2).sum()
        loss.backward()
        return float(loss), theta.grad.numpy()

    l_cf, g_cf = loss_and_grad(0)
    l_svd, g_svd = loss_and_grad(hsf.FLAG_SVD_BLOCKS)
    assert abs(l_cf - l_svd) <= 1e-12
    assert np.max(np.abs(g_cf - g_svd)) <= 1e-10 * max(1.0, np.max(np.abs(g_svd)))

    def loss_fn(t):
        psi = O.schrodinger(pr.n, pr.gates, theta=t)
        return O.loss_from_amplitudes(psi[pr.bitstrings.astype(np.int64)])

    fd = O.fd_gradient(loss_fn, pr.params, h=1e-5)
    assert np.max(np.abs(g_cf - fd)) <= 1e-6 * max(1.0, np.max(np.abs(fd)))


def big_cascade_problem(leaves, seed):
    """n = 14 (cut after qubit 6): a cascade of RZZ and CNOT gates from hub qubit 7 (side
    a) to `leaves` qubits of side b, between Haar layers (more than 3 block qubits on
    side b: the factor is kept as one small op per gate)."""
    rng = np.random.default_rng(seed)
    n, cut = 14, 6
    gates = [Gate("matrix", (q,), matrix=W.haar_u2(rng)) for q in range(n)]
    W._cz_brickwork(gates, n, cut, 0)
    blk = []
    for j, t in enumerate(range(cut, cut - leaves, -1)):
        blk.append(len(gates))
        if j % 2:
            gates.append(Gate("cx", (7, t)))
        else:
            gates.append(Gate("rzz", (t, 7), param=float(rng.uniform(0, 2 * np.pi))))
    gates += [Gate("matrix", (q,), matrix=W.haar_u2(rng)) for q in range(n)]
    W._cz_brickwork(gates, n, cut, 1)
    return W.Problem(n=n, gates=gates, cut=cut, blocks=[blk], name=f"cascade{leaves}")


@pytest.mark.parametrize("leaves", [4, 6])
def test_cascade_with_more_than_three_leaves(leaves):
    pr = big_cascade_problem(leaves, seed=leaves)
    ref = O.schrodinger(pr.n, pr.gates)
    for prec, tol in (("c128", 1e-12), ("c64", 1e-5)):
        plan, lines = _plan(pr, precision=prec)
        assert len(lines) == 1 and "closed-form" in lines[0] and f"1|{leaves}" in lines[0], lines
        assert plan.info["num_paths"] == 2
        got = plan.run(check=True).cpu().numpy()
        plan.close()
        assert np.max(np.abs(got - ref)) <= tol


def test_sbm_qaoa_found_blocks_joint_plain_schrodinger():
    """A q20-shaped SBM-QAOA instance (10|10, p_inter 0.3): the library's own blocks
    (hsf_find_blocks) against the standard per-gate cut and the full-state plan, all at
    the first 10^5 amplitudes, against the oracle."""
    from paper_2502_06959_gb300 import hsf
    pr = W.sbm_qaoa((10, 10), 0.8, 0.3, seed=21)
    q = hsf.problem_with_found_blocks(pr)
    ref = O.schrodinger(pr.n, pr.gates)[:100000]
    plain = W.Problem(n=q.n, gates=q.gates, cut=q.cut, blocks=W.singleton_blocks(q.n, q.gates, q.cut))
    for prob, prec in ((q, "c64"), (q, "c128"), (plain, "c64")):
        plan = hsf.Plan.from_problem(prob, precision=prec, gemm="fp32")
        P = plan.info["num_paths"]
        got = plan.run(window=100000, check=True).cpu().numpy()
        plan.close()
        assert P == 2 ** len(prob.blocks)
        assert np.max(np.abs(got - ref)) <= (1e-12 if prec == "c128" else 1e-5)
    plan = hsf.Plan.schrodinger(pr.n, pr.gates, precision="c64")
    got = plan.run(window=100000, check=True).cpu().numpy()
    plan.close()
    assert np.max(np.abs(got - ref)) <= 1e-5


def test_searched_cut_of_scrambled_sbm_qaoa():
    """A q20-shaped SBM-QAOA instance with scrambled qubit labels: hsf_search_cut
    relabels it, the planner runs the blocks found on the relabeled circuit with exactly
    2^(reported log2 paths) paths, and the amplitudes equal the oracle's Schroedinger
    amplitudes of the input circuit under the bit permutation."""
    from paper_2502_06959_gb300 import hsf
    pr = W.sbm_qaoa((10, 10), 0.8, 0.2, seed=22)
    rng = np.random.default_rng(4)
    ps = hsf.relabel_problem(pr, [int(x) for x in rng.permutation(pr.n)])
    q = hsf.problem_with_searched_cut(ps)
    assert q.meta["log2_paths_after"] < q.meta["log2_paths_before"]
    perm = q.meta["perm"]
    ref = O.schrodinger(ps.n, ps.gates)
    x = np.arange(1 << ps.n, dtype=np.int64)
    xp = np.zeros_like(x)
    for a, b in enumerate(perm):
        xp |= ((x >> a) & 1) << b
    ref_new = np.empty_like(ref)
    ref_new[xp] = ref                           # amplitudes of the relabeled circuit
    plan = hsf.Plan.from_problem(q, precision="c64", gemm="fp32")
    assert plan.info["num_paths"] == round(2 ** q.meta["log2_paths_after"])
    got = plan.run(window=1 << 16, check=True).cpu().numpy()
    plan.close()
    assert np.max(np.abs(got - ref_new[:1 << 16])) <= 1e-5
