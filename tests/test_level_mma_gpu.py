"""GPU parity of the tensor-core tree level.

A tree level whose program (Schmidt factor, then the gates it hoists) acts only on the
6 lowest storage bits of a half state with h >= 13 qubits runs as one tensor-core product
per Schmidt digit (FP16 hi/lo parts of power-of-two scaled operands, three products).  These cases check it against the FP64 oracle (complex64
bound: 1e-5 max abs and 1e-4 of the largest reference amplitude) and against the same
plan swept on the CUDA cores, for bitstring and window outputs, over path ranges that
start and end inside a parent's group of digits.
"""
import numpy as np
import pytest

import oracle.hsf_oracle as O
from paper_2502_06959_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2502_06959_gb300 import build
    build.build()
    from paper_2502_06959_gb300 import hsf
    hsf.load_library()


def check(got, ref):
    err = float(np.max(np.abs(got - ref))) if ref.size else 0.0
    scale = float(np.max(np.abs(ref))) if ref.size else 1.0
    assert err <= 1e-5, err
    assert err <= 1e-4 * scale, (err, scale)
    return err


def run(pr, bits=None, window=0, path_range=(0, 0), **opts):
    import torch
    from paper_2502_06959_gb300 import hsf
    plan = hsf.Plan(pr.n, pr.gates, pr.cut, pr.blocks, precision="c64", **opts)
    bs = None
    if bits is not None:
        bs = torch.from_numpy(np.asarray(bits, dtype=np.uint64).view(np.int64)).cuda()
    out = plan.run(bs, window=window, path_range=path_range)
    torch.cuda.synchronize()
    desc = hsf.hsf_plan_describe(plan.handle)
    res = out.cpu().numpy()
    plan.close()
    return res, desc


def problem(n, kind, seed, blocks_after=(2, 4, 6, 7), layers=8):
    return W.random_brickwork(n, n // 2 - 1, layers, block_after=blocks_after, block_kind=kind,
                              block_len=2, seed=seed)


@pytest.mark.parametrize("n,kind,seed", [(26, "rzz", 1), (26, "mixed", 2), (28, "cx_rzz_cz", 3)])
def test_tc_level_bitstrings_against_oracle(n, kind, seed):
    from paper_2502_06959_gb300 import hsf
    pr = problem(n, kind, seed)
    rng = np.random.default_rng(seed)
    bits = W.random_bitstrings(rng, n, 200)
    got, desc = run(pr, bits)
    assert "tensor-core product" in desc, desc
    ref_cc, desc_cc = run(pr, bits, flags=hsf.FLAG_NO_TC_LEVEL)
    assert "tensor-core product" not in desc_cc
    check(got, ref_cc)
    # the split product keeps FP32-level accuracy: a dropped lo part (one FP16 product)
    # or a wrong row scale would show up as ~5e-4 relative error or worse
    assert np.max(np.abs(got - ref_cc)) <= 2e-5 * np.max(np.abs(ref_cc))
    plan = hsf.Plan(pr.n, pr.gates, pr.cut, pr.blocks, precision="c64")
    P = int(plan.info["num_paths"])
    # single paths are unique only when no block has a repeated singular value (within a
    # degenerate subspace any orthonormal Schmidt basis is correct); otherwise compare
    # the full path sum, which is unique
    sig = [plan.sigma(k) for k in range(len(pr.blocks))]
    plan.close()
    distinct = all(np.all(np.abs(np.diff(s)) > 1e-6 * s[0]) for s in sig)
    ranges = ((0, 3), (1, 6), (P // 2 - 1, P // 2 + 5), (P - 5, P)) if distinct else ((0, P),)
    for (a, b) in ranges:
        want, _ = O.hsf_amplitudes(pr.n, pr.gates, pr.cut, pr.blocks, bitstrings=bits, path_range=(a, b))
        got_r, _ = run(pr, bits, path_range=(a, b))
        check(got_r, want)


def test_tc_level_window_against_cuda_cores_and_oracle():
    from paper_2502_06959_gb300 import hsf
    pr = problem(26, "mixed", 5)
    win = 1 << 18
    got, desc = run(pr, window=win, path_range=(3, 11))
    assert "tensor-core product" in desc
    ref_cc, _ = run(pr, window=win, path_range=(3, 11), flags=hsf.FLAG_NO_TC_LEVEL)
    check(got, ref_cc)
    rng = np.random.default_rng(9)
    idx = rng.choice(win, size=64, replace=False).astype(np.uint64)
    want, _ = O.hsf_amplitudes(pr.n, pr.gates, pr.cut, pr.blocks, bitstrings=idx, path_range=(3, 11))
    check(got[idx.astype(np.int64)], want)


def test_tc_level_in_n30_plan():
    """The deepest materialised level of the n = 30 workload runs on the tensor cores."""
    from paper_2502_06959_gb300 import hsf
    pr = W.workload_c2(num_bitstrings=16)
    plan = hsf.Plan.from_problem(pr)
    desc = hsf.hsf_plan_describe(plan.handle)
    plan.close()
    # level 7: the whole level is the product (FP16 parts, no ops after it)
    lines = [l for l in desc.splitlines() if l.startswith(" level 7:")]
    assert len(lines) == 2 and all("product (FP16x3)" in l and "then 0 passes" in l for l in lines), desc
    # level 6: its leading ops (factor and the gates on the 6 low bits) as the product
    # (TF32 parts), the rest (on storage bits below 11) applied by the product's epilogue
    lines = [l for l in desc.splitlines() if l.startswith(" level 6:")]
    assert len(lines) == 2 and all("product (TF32x3)" in l and "ops in its epilogue" in l for l in lines), desc


def _storage_bits(desc, n, cut):
    """Global qubit -> storage bit on its side, from the plan description's store lists
    (side b holds qubits 0..cut, side a the rest)."""
    import re
    st = {m.group(1): [int(v) for v in m.group(2).split(",")]
          for m in re.finditer(r"side ([ab]): h=\d+ store=\[([0-9,]*)\]", desc)}
    return {q: (st["b"][q] if q <= cut else st["a"][q - cut - 1]) for q in range(n)}


def test_fp16_level_keeps_small_amplitudes():
    """The FP16 split scales every 64-amplitude parent row by its own power of two.

    With near-identity single-qubit rotations the amplitude of a bitstring falls by about
    three orders of magnitude per 1 it holds.  With the 1s on qubits stored at bit 6 or
    above, the magnitude changes from row to row (a row is the 64 amplitudes on storage
    bits 0..5) and the rows span far more than FP16's exponent range (2^29 from its
    smallest normal to its largest value).  Unscaled FP16 parts would flush the small
    rows; scaled ones keep those amplitudes to FP32-level relative accuracy, as the
    CUDA-core sweep does.  (Within a row the split is accurate to about 2^-22 of the
    row's largest amplitude, an absolute bound, which the standard check covers.)
    """
    from paper_2502_06959_gb300 import hsf
    pr = problem(26, "rzz", 11)
    theta = 2e-3
    c, sn = np.cos(theta / 2), np.sin(theta / 2)
    rx = np.array([[c, -1j * sn], [-1j * sn, c]])
    for g in pr.gates:
        if g.kind == "matrix" and len(g.qubits) == 1:
            g.matrix = rx
    _, desc = run(pr, np.zeros(1, dtype=np.uint64))
    assert "product (FP16x3)" in desc, desc
    sbit = _storage_bits(desc, pr.n, pr.cut)
    high = [q for q in range(pr.n) if sbit[q] >= 6]
    rng = np.random.default_rng(11)
    bits = []
    for k in range(0, 9):                      # bitstrings with k ones on high storage bits
        for _ in range(6):
            b = 0
            for q in rng.choice(high, size=k, replace=False):
                b |= 1 << int(q)
            bits.append(b)
    extra = W.random_bitstrings(rng, pr.n, 64)  # any bitstrings: absolute accuracy
    bits = np.concatenate([np.array(bits, dtype=np.uint64), np.asarray(extra, dtype=np.uint64)])
    got, _ = run(pr, bits)
    ref, desc_cc = run(pr, bits, flags=hsf.FLAG_NO_TC_LEVEL)
    assert "tensor-core product" not in desc_cc
    check(got, ref)
    nh = 9 * 6
    mag = np.abs(ref[:nh])
    assert mag.min() < 1e-12 * mag.max(), (mag.min(), mag.max())   # the range is really there
    rel = np.abs(got[:nh] - ref[:nh]) / mag
    assert np.max(rel) <= 1e-4, (np.max(rel), mag[np.argmax(rel)])
