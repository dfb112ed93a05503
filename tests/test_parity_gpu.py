"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances: the half states and per-path products run in the plan's precision; the
cross-path sum is FP64.  complex128 plans must match within 1e-12 (max abs); complex64
plans within the FP32 bound 1e-5 (max abs) and, so that the bound keeps meaning at
large n where amplitudes are ~2^{-n/2}, also within 1e-4 of the largest reference
amplitude (FP32 unit round-off 6e-8 times a few hundred gates, with margin).
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


def H():
    from paper_2502_06959_gb300 import hsf
    return hsf


def check(got, ref, prec):
    err = float(np.max(np.abs(got - ref))) if ref.size else 0.0
    if prec == "c128":
        assert err <= 1e-12, err
    else:
        scale = float(np.max(np.abs(ref))) if ref.size else 1.0
        assert err <= 1e-5, err
        assert err <= 1e-4 * scale, (err, scale)
    return err


def distinct_sigma(pr):
    """True when no block has a repeated singular value, i.e. every single path (and
    so every partial path sum) is unique; within a degenerate subspace any orthonormal
    Schmidt basis is correct and only the full path sum is fixed."""
    plan = H().Plan(pr.n, pr.gates, pr.cut, pr.blocks, precision="c128")
    sig = [plan.sigma(k) for k in range(len(pr.blocks))]
    plan.close()
    return all(np.all(np.abs(np.diff(v)) > 1e-6 * v[0]) for v in sig)


def gpu_amps(pr, prec="c64", bitstrings=None, window=0, path_range=(0, 0), blocks=None, **opts):
    import torch
    plan = H().Plan(pr.n, pr.gates, pr.cut, pr.blocks if blocks is None else blocks,
                    precision=prec, **opts)
    bs = None
    if bitstrings is not None:
        bs = torch.from_numpy(np.asarray(bitstrings, dtype=np.uint64).view(np.int64)).cuda()
    out = plan.run(bs, window=window, path_range=path_range)
    torch.cuda.synchronize()
    res = out.cpu().numpy()
    info = plan.info
    plan.close()
    return res, info


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_c1_all_amplitudes(prec):
    pr = W.workload_c1()
    ref = O.schrodinger(pr.n, pr.gates)
    got, info = gpu_amps(pr, prec)
    assert info["num_paths"] == 4
    check(got, ref, prec)


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_c1_plain_cut_equals_joint(prec):
    pr = W.workload_c1()
    plain = W.singleton_blocks(pr.n, pr.gates, pr.cut)
    got, info = gpu_amps(pr, prec, blocks=plain)
    assert info["num_paths"] == 64
    check(got, O.schrodinger(pr.n, pr.gates), prec)


def _sigma_cases():
    cases = []
    c1 = W.workload_c1()
    cases.append((c1, c1.blocks))
    c2 = W.workload_c2(layers=6, num_blocks=2, num_bitstrings=0)
    cases.append((c2, c2.blocks))
    c4 = W.workload_c4(n=12)
    cases.append((c4, c4.blocks))
    rng = np.random.default_rng(7)
    for ka, kb in ((2, 2), (3, 3), (1, 3), (3, 1), (2, 1)):
        n = ka + kb
        gates = []
        for d in range(8):
            for q in range(n):
                gates.append(Gate("matrix", (q,), matrix=W.haar_u2(rng)))
            for q in range(n - 1):
                gates.append(Gate("cz", (q + 1, q)))
        cases.append((W.Problem(n, gates, kb - 1, [list(range(len(gates)))]), None))
    return cases


def test_block_svd_matches_lapack():
    for pr, blocks in _sigma_cases():
        blocks = pr.blocks if blocks is None else blocks
        dec = O.decompose_blocks(pr.n, pr.gates, pr.cut, blocks)
        # the device SVD itself: cascade blocks would otherwise get closed-form terms,
        # whose weights are not the singular values
        plan = H().Plan(pr.n, pr.gates, pr.cut, blocks, precision="c128", flags=H().FLAG_SVD_BLOCKS)
        for k, d in enumerate(dec):
            s = plan.sigma(k)
            assert len(s) == len(d["sigma"])
            assert np.max(np.abs(s - d["sigma"])) < 1e-13
            assert abs(np.sum(s ** 2) - (1 << len(d["qubits"]))) < 1e-11
        plan.close()


def test_cascade_and_closed_form_ranks():
    for kind in ("cx", "cz", "rzz", "swap"):
        gates = [Gate(kind, (3, t), param=0.9) for t in (2, 1, 0)] if kind != "swap" else [Gate("swap", (1, 0))]
        n = 4 if kind != "swap" else 2
        cut = 2 if kind != "swap" else 0
        plan = H().Plan(n, gates, cut, [list(range(len(gates)))], precision="c128")
        s = plan.sigma(0)
        if kind == "swap":
            assert np.allclose(s, [1, 1, 1, 1], atol=1e-14)
        else:
            assert len(s) == 2
        plan.close()


@pytest.mark.parametrize("seed", range(8))
@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_random_circuits_all_gate_kinds(seed, prec):
    rng = np.random.default_rng(1000 + seed)
    n = int(rng.integers(4, 11))
    cut = int(rng.integers(0, n - 1))
    gates = W.random_circuit(n, 40, seed)
    # group crossing gates: consecutive crossing gates sharing a qubit pair become one
    # block when that keeps the block convex, else singletons
    blocks = W.singleton_blocks(n, gates, cut)
    ref = O.schrodinger(n, gates)
    pr = W.Problem(n, gates, cut, blocks)
    got, _ = gpu_amps(pr, prec)
    check(got, ref, prec)


@pytest.mark.parametrize("tile_bits", [3, 4, 5])
@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_multi_pass_tiles(tile_bits, prec):
    pr = W.random_brickwork(14, 6, 6, block_after=(2, 4), block_kind="mixed", block_len=3, seed=77)
    ref = O.schrodinger(pr.n, pr.gates)
    got, _ = gpu_amps(pr, prec, tile_bits=tile_bits)
    check(got, ref, prec)


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_bitstrings_windows_and_path_ranges(prec):
    pr = W.random_brickwork(12, 5, 6, block_after=(1, 3, 5), block_kind="mixed", block_len=3, seed=5)
    ref = O.schrodinger(pr.n, pr.gates)
    rng = np.random.default_rng(3)
    bs = W.random_bitstrings(rng, pr.n, 333)
    got, info = gpu_amps(pr, prec, bitstrings=bs)
    check(got, ref[bs.astype(np.int64)], prec)
    for w in (1, 63, 64, 65, 1000):
        got, _ = gpu_amps(pr, prec, window=w)
        check(got, ref[:w], prec)
    P = info["num_paths"]
    for (a, b) in ((0, 1), (1, 7), (5, P), (P - 1, P)):
        want, _ = O.hsf_amplitudes(pr.n, pr.gates, pr.cut, pr.blocks, bitstrings=bs, path_range=(a, b))
        got, _ = gpu_amps(pr, prec, bitstrings=bs, path_range=(a, b))
        check(got, want, prec)


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_light_cone_order_and_chunking_do_not_change_results(prec):
    from paper_2502_06959_gb300 import hsf
    import torch
    pr = W.random_brickwork(12, 5, 8, block_after=(2, 4, 6), block_kind="rzz", block_len=3, seed=8)
    ref = O.schrodinger(pr.n, pr.gates)
    got, _ = gpu_amps(pr, prec, flags=hsf.FLAG_NO_LIGHTCONE)
    check(got, ref, prec)
    got, _ = gpu_amps(pr, prec)
    check(got, ref, prec)
    # a tight workspace budget forces several path chunks
    plan = hsf.Plan(pr.n, pr.gates, pr.cut, pr.blocks, precision=prec)
    full = hsf.hsf_workspace_size(plan.handle, 0, 0, 0)
    budget = full
    while True:                      # the smallest budget that still holds one chunk
        try:
            need = hsf.hsf_workspace_size(plan.handle, 0, 0, budget // 2)
        except hsf.HsfError:
            break
        budget = need
    assert budget < full
    out = plan.run(None, budget=budget)
    torch.cuda.synchronize()
    check(out.cpu().numpy(), ref, prec)
    plan.close()


def test_edge_cases():
    # no crossing gate: one path; gates only on one side; minimal n; cut at either end
    cases = [
        W.Problem(2, [Gate("h", (1,)), Gate("cx", (1, 0))], 0, [[1]]),             # Example 1
        W.Problem(3, [Gate("h", (0,)), Gate("x", (2,))], 0, []),
        W.Problem(5, [], 2, []),
        W.Problem(6, W.random_circuit(6, 20, 4, kinds=["matrix", "rzz", "cx"]), 4, None),
        W.Problem(6, W.random_circuit(6, 20, 5, kinds=["matrix", "rzz", "cx"]), 0, None),
    ]
    for pr in cases:
        if pr.blocks is None:
            pr.blocks = W.singleton_blocks(pr.n, pr.gates, pr.cut)
        ref = O.schrodinger(pr.n, pr.gates)
        for prec in ("c128", "c64"):
            got, _ = gpu_amps(pr, prec)
            check(got, ref, prec)
    # Example 1 exactly
    got, _ = gpu_amps(cases[0], "c128")
    assert np.max(np.abs(got - np.array([1, 0, 0, 1]) / np.sqrt(2))) < 1e-15
    # a zero-length bitstring request and an empty path range give empty / zero output
    got, _ = gpu_amps(cases[3], "c64", bitstrings=np.zeros(0, dtype=np.uint64))
    assert got.size == 0
    got, _ = gpu_amps(cases[3], "c64", bitstrings=np.arange(5, dtype=np.uint64), path_range=(2, 2))
    assert np.all(got == 0)


def test_c4_qaoa_bitstrings():
    pr = W.workload_c4()
    want, info = O.hsf_amplitudes(pr.n, pr.gates, pr.cut, pr.blocks, bitstrings=pr.bitstrings)
    assert info["num_paths"] == 256
    got, ginfo = gpu_amps(pr, "c64", bitstrings=pr.bitstrings)
    assert ginfo["num_paths"] == 256
    check(got, want, "c64")


def test_c2_reduced_full_width():
    """n = 30 (15|15) with the C2 generator, 2 blocks and 6 layers (16 paths):
    every amplitude of 4096 bitstrings against the oracle's full path sum."""
    pr = W.workload_c2(num_blocks=2, layers=6)
    want, info = O.hsf_amplitudes(pr.n, pr.gates, pr.cut, pr.blocks, bitstrings=pr.bitstrings)
    assert info["num_paths"] == 16
    got, _ = gpu_amps(pr, "c64", bitstrings=pr.bitstrings)
    check(got, want, "c64")


@pytest.mark.parametrize("path_range", [(0, 48), (40000, 40016), (65536 - 16, 65536)])
def test_c2_full_size_sampled_paths(path_range):
    """The full n = 30 workload (8 blocks, 20 layers, 4^8 paths) in the launch
    configuration the benchmark times, restricted to a range of paths that the
    oracle sums one path at a time."""
    pr = W.workload_c2()
    want, info = O.hsf_amplitudes(pr.n, pr.gates, pr.cut, pr.blocks, bitstrings=pr.bitstrings,
                                  path_range=path_range)
    assert info["num_paths"] == 4 ** 8
    got, ginfo = gpu_amps(pr, "c64", bitstrings=pr.bitstrings, path_range=path_range)
    assert ginfo["num_paths"] == 4 ** 8
    check(got, want, "c64")


@pytest.mark.parametrize("prec", ["c128", "c64"])
@pytest.mark.parametrize("seed", range(4))
def test_leaf_contraction_matches_materialised_leaves(prec, seed):
    """The leaf level contracted at the bitstrings equals the materialised leaves
    summed by gather-dot, and both equal the oracle (several digits per block,
    unaligned path ranges)."""
    from paper_2502_06959_gb300 import hsf
    pr = W.random_brickwork(12, 5, 7, block_after=(2, 4, 7), block_kind="mixed", block_len=3,
                            seed=40 + seed)
    rng = np.random.default_rng(seed)
    bs = W.random_bitstrings(rng, pr.n, 257)
    ref = O.schrodinger(pr.n, pr.gates)[bs.astype(np.int64)]
    got, info = gpu_amps(pr, prec, bitstrings=bs)
    assert info["leaf_bits"] > 0
    check(got, ref, prec)
    got2, info2 = gpu_amps(pr, prec, bitstrings=bs, flags=hsf.FLAG_NO_LEAF_CONTRACT)
    check(got2, ref, prec)
    P = info["num_paths"]
    for (a, b) in ((1, P - 1), (3, 6), (P // 2 + 1, P // 2 + 2)):
        want, _ = O.hsf_amplitudes(pr.n, pr.gates, pr.cut, pr.blocks, bitstrings=bs, path_range=(a, b))
        got, _ = gpu_amps(pr, prec, bitstrings=bs, path_range=(a, b))
        check(got, want, prec)


def _leaf_rank_problem(rank, tail, seed):
    """A 12-qubit brickwork whose last block has Schmidt rank 1, 2, 4 or 8, followed by
    `tail` further layers (which widen the leaf program's light cone)."""
    pr = W.random_brickwork(12, 5, 3, block_after=(2,), block_kind="rzz", block_len=2, seed=seed)
    rng = np.random.default_rng(seed + 1000)
    g = list(pr.gates)
    blk = []

    def add(gate):
        blk.append(len(g))
        g.append(gate)

    if rank == 1:                       # CZ CZ = identity: one product term
        add(W.Gate("cz", (6, 5)))
        add(W.Gate("cz", (6, 5)))
    elif rank == 2:
        add(W.Gate("rzz", (6, 5), param=float(rng.uniform(0, 2 * np.pi))))
    elif rank == 4:
        add(W.Gate("cx", (5, 6)))
        add(W.Gate("matrix", (6,), matrix=W.haar_u2(rng)))
        add(W.Gate("matrix", (5,), matrix=W.haar_u2(rng)))
        add(W.Gate("rzz", (6, 5), param=float(rng.uniform(0, 2 * np.pi))))
    else:                               # three crossing pairs: rank 2^3
        add(W.Gate("cz", (6, 5)))
        add(W.Gate("cz", (7, 4)))
        add(W.Gate("cz", (8, 3)))
    for t in range(tail):
        W._u2_layer(rng, g, range(12))
        W._cz_brickwork(g, 12, 5, t % 2)
    return W.Problem(n=12, gates=g, cut=5, blocks=list(pr.blocks) + [blk])


@pytest.mark.parametrize("prec", ["c128", "c64"])
@pytest.mark.parametrize("rank", [1, 2, 4, 8])
@pytest.mark.parametrize("tail", [0, 1, 2])
def test_leaf_contraction_every_rank_and_width(prec, rank, tail):
    """Leaf contraction for every operator count the kernels specialise on (1, 2, 4, 8
    threads per bitstring) and leaf programs of several widths, against the state
    vector and against materialised leaves."""
    from paper_2502_06959_gb300 import hsf
    pr = _leaf_rank_problem(rank, tail, seed=70 + rank + 10 * tail)
    rng = np.random.default_rng(rank + 10 * tail)
    bs = W.random_bitstrings(rng, pr.n, 300)
    ref = O.schrodinger(pr.n, pr.gates)[bs.astype(np.int64)]
    got, info = gpu_amps(pr, prec, bitstrings=bs)
    if tail == 0:
        assert info["leaf_bits"] > 0
    check(got, ref, prec)
    got2, _ = gpu_amps(pr, prec, bitstrings=bs, flags=hsf.FLAG_NO_LEAF_CONTRACT)
    check(got2, ref, prec)


@pytest.mark.parametrize("rank,tail", [(1, 0), (2, 1), (4, 0), (4, 1), (8, 0)])
def test_leaf_contraction_many_bitstrings(rank, tail):
    """Above 65536 bitstrings the complex64 leaf contraction runs as one wave of CTAs
    that walk the parents together; every rank and leaf width it takes, against the
    state vector, plus a path range that starts and ends inside a parent's digits."""
    pr = _leaf_rank_problem(rank, tail, seed=90 + rank + 10 * tail)
    rng = np.random.default_rng(7 + rank)
    bs = W.random_bitstrings(rng, pr.n, 70000)
    ref = O.schrodinger(pr.n, pr.gates)[bs.astype(np.int64)]
    got, info = gpu_amps(pr, "c64", bitstrings=bs)
    check(got, ref, "c64")
    if not distinct_sigma(pr):
        return    # single paths are not unique when a block has repeated singular values
    P = info["num_paths"]
    sub = bs[:512]
    want, _ = O.hsf_amplitudes(pr.n, pr.gates, pr.cut, pr.blocks, bitstrings=sub, path_range=(1, P - 1))
    got_r, _ = gpu_amps(pr, "c64", bitstrings=bs, path_range=(1, P - 1))
    check(got_r[:512], want, "c64")


def test_c2_plan_uses_leaf_contraction_and_register_kernel():
    pr = W.workload_c2(num_bitstrings=16)
    plan = H().Plan.from_problem(pr)
    assert plan.info["leaf_bits"] == 4
    assert plan.info["tree_nodes"] == sum(4 ** k for k in range(9))
    plan.close()


@pytest.mark.parametrize("gemm,tol_rel", [("fp32", 1e-4), ("bf16x3", 1e-4), ("tf32x3", 1e-4), ("tf32", 5e-3)])
def test_tensor_core_path_gemm_window(gemm, tol_rel):
    """Full / window output through the tensor-core path GEMM (tcgen05): several M, N
    and K tiles, ragged edges, against the oracle.  Plain TF32 keeps ~10 mantissa bits,
    so it is checked at a looser relative bound (it is reported, not a parity form)."""
    import torch
    from paper_2502_06959_gb300 import hsf
    pr = W.random_brickwork(20, 9, 6, block_after=(1, 2, 3, 4, 5), block_kind="mixed", block_len=3, seed=21)
    ref = O.schrodinger(pr.n, pr.gates)
    for window in (1 << 20, 300000, 1000):
        plan = hsf.Plan.from_problem(pr, precision="c64", gemm=gemm)
        out = plan.run(window=window, check=True)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        info = plan.info
        plan.close()
        want = ref[:window]
        err = float(np.max(np.abs(got - want)))
        scale = float(np.max(np.abs(want)))
        assert info["num_paths"] > 128
        assert err <= tol_rel * scale, (gemm, window, err, scale)
        if gemm != "tf32":
            assert err <= 1e-5


def test_tensor_core_gemm_c1_full():
    import torch
    from paper_2502_06959_gb300 import hsf
    pr = W.workload_c1()
    ref = O.schrodinger(pr.n, pr.gates)
    for gemm in ("bf16x3", "tf32x3"):
        plan = hsf.Plan.from_problem(pr, precision="c64", gemm=gemm)
        out = plan.run(check=True).cpu().numpy()
        plan.close()
        check(out, ref, "c64")


@pytest.mark.parametrize("path_range", [(0, 4), (1 << 23, (1 << 23) + 2)])
def test_c5_n36_sampled_paths(path_range):
    """n = 36 (18|18, the full state would be 512 GB), 12 blocks (4^12 paths), 2^20
    bitstrings, in the benchmark's launch configuration, on path ranges the oracle sums
    path by path."""
    pr = W.workload_c5()
    want, info = O.hsf_amplitudes(pr.n, pr.gates, pr.cut, pr.blocks, bitstrings=pr.bitstrings,
                                  path_range=path_range)
    assert info["num_paths"] == 4 ** 12
    got, ginfo = gpu_amps(pr, "c64", bitstrings=pr.bitstrings, path_range=path_range)
    assert ginfo["num_paths"] == 4 ** 12
    check(got, want, "c64")


def test_leaf_kernel_shapes_covered():
    """The (leaf width, operator count) pairs that the leaf-rank problems above reach:
    they must include chunk-split shapes (2^width >= 2 x operators, 2 or more operators)
    at two widths, so that the split kernel's reduce-scatter over 2 and 4 lanes is
    checked against the oracle there."""
    from paper_2502_06959_gb300 import hsf
    shapes = set()
    for rank in (1, 2, 4, 8):
        for tail in (0, 1, 2):
            pr = _leaf_rank_problem(rank, tail, seed=70 + rank + 10 * tail)
            plan = hsf.Plan.from_problem(pr, precision="c64")
            info = plan.info
            plan.close()
            if info["leaf_bits"] > 0:
                shapes.add((int(info["leaf_bits"]), rank))
    split = {(c, r) for (c, r) in shapes if r >= 2 and (1 << c) >= 2 * r}
    assert len({r for (_, r) in split}) >= 2, shapes


def test_factored_leaf_against_oracle_and_direct():
    """Rank-4 last blocks (one qubit per side): where the leaf spans 2 to 4 chunk bits
    its operators factor as S (F_m (x) I), and the factored kernel (digit sum folded
    into a 4 x 4 bilinear form) must equal the oracle over all paths and over path
    ranges that cut a parent's digits (first parent from digit 1 or 3, last parent up
    to digit 1 or 3, a single parent).  The leaf widens with the tail layers; the
    factored kernel must have run for at least one of them."""
    from paper_2502_06959_gb300 import hsf
    widths = set()
    for tail in (0, 1, 2, 3):
        pr = _leaf_rank_problem(4, tail, seed=170 + tail)
        rng = np.random.default_rng(tail + 300)
        bs = W.random_bitstrings(rng, pr.n, 333)
        plan = hsf.Plan.from_problem(pr, precision="c64")
        desc = hsf.hsf_plan_describe(plan.handle)
        c = int(plan.info["leaf_bits"])
        plan.close()
        if "leaf=factored" in desc:
            widths.add(c)
        ref = O.schrodinger(pr.n, pr.gates)[bs.astype(np.int64)]
        got, info = gpu_amps(pr, "c64", bitstrings=bs)
        check(got, ref, "c64")
        P = info["num_paths"]
        for (a, b) in ((1, P), (0, P - 1), (3, P - 3), (5, 7), (P // 2 + 1, P // 2 + 3), (4, 8)):
            want, _ = O.hsf_amplitudes(pr.n, pr.gates, pr.cut, pr.blocks, bitstrings=bs, path_range=(a, b))
            got, _ = gpu_amps(pr, "c64", bitstrings=bs, path_range=(a, b))
            check(got, want, "c64")
    assert widths, "no leaf took the factored kernel"


def test_c2_leaf_is_factored():
    """The benchmark circuit's leaf (last block rank 4, one qubit per side) runs the
    factored leaf kernel."""
    from paper_2502_06959_gb300 import hsf
    pr = W.workload_c2()
    plan = hsf.Plan.from_problem(pr, precision="c64")
    desc = hsf.hsf_plan_describe(plan.handle)
    plan.close()
    assert "leaf=factored" in desc


def _run_profiled(pr, bs, flags=0, path_range=(0, 0), budget=0):
    """Amplitudes of `bs` and the per-kind launch statistics of that one run."""
    import torch
    from paper_2502_06959_gb300 import hsf
    plan = hsf.Plan.from_problem(pr, precision="c64", flags=flags)
    dbs = torch.from_numpy(np.asarray(bs, dtype=np.uint64).view(np.int64)).cuda()
    hsf.hsf_set_profiling(True)
    try:
        out = plan.run(dbs, path_range=path_range, budget=budget)
        torch.cuda.synchronize()
        stats = hsf.hsf_profile_collect(plan.handle)
    finally:
        hsf.hsf_set_profiling(False)
    res = out.cpu().numpy()
    plan.close()
    return res, stats


def _took_dot_form(stats_dots, stats_rows):
    """The leaf's counted FLOP per (parent, bitstring): 8 (4 x 16 + 20) = 672 from stored
    chunks, 8 x 20 = 160 from the dots; the same units in both runs."""
    return stats_dots["leaf"]["flops"] * 672.0 == pytest.approx(stats_rows["leaf"]["flops"] * 160.0, rel=1e-12)


@pytest.mark.parametrize("count", [1, 37, 4096])
def test_leaf_dot_form_equals_stored_children(count):
    """C2 (n = 30, 4^8 paths) at the benchmark's launch sizes: level 7 writing the four
    leaf dots per (child, bitstring) (HSF_FLAG_LEAF_DOTS) must give the same bits as
    level 7 storing its children and the factored leaf kernel reading them (the dots are
    formed from the same FP32 values in the same order, and the bilinear form is summed
    in the same order), over all paths and over ranges whose first or last parent has
    only part of its digits."""
    from paper_2502_06959_gb300 import hsf
    pr = W.workload_c2()
    bs = pr.bitstrings[:count]
    for path_range in ((0, 0), (1, 47), (40001, 40003), (65535, 65536)):
        a, sa = _run_profiled(pr, bs, hsf.FLAG_LEAF_DOTS, path_range)
        b, sb = _run_profiled(pr, bs, 0, path_range)
        assert _took_dot_form(sa, sb), path_range
        assert np.array_equal(a, b), (path_range, np.max(np.abs(a - b)))


def test_leaf_dot_form_over_path_chunks():
    """A workspace budget that splits the first 4096 C2 paths into four chunks (each
    chunk's dots overwrite the previous chunk's): the dot form against the oracle's
    path sum over a range cutting a parent, and against the stored-children run over
    all 4096 paths."""
    from paper_2502_06959_gb300 import hsf
    pr = W.workload_c2()
    bs = pr.bitstrings[:333]
    ref, sr = _run_profiled(pr, bs, 0, (0, 4096))
    got, sg = _run_profiled(pr, bs, hsf.FLAG_LEAF_DOTS, (0, 4096), budget=256 << 20)
    assert _took_dot_form(sg, sr)
    check(got, ref, "c64")
    want, _ = O.hsf_amplitudes(pr.n, pr.gates, pr.cut, pr.blocks, bitstrings=bs, path_range=(1021, 1030))
    got, _ = _run_profiled(pr, bs, hsf.FLAG_LEAF_DOTS, (1021, 1030), budget=256 << 20)
    check(got, want, "c64")
