"""GPU adjoint gradients against central finite differences of the FP64 oracle.

Loss L = sum_s |amp(s)|^2 over seeded bitstrings.  The oracle gradient is the central
difference of L computed by the oracle's Schroedinger simulation (small n) or HSF path
sum (n = 28), with step h = 1e-5 (error O(h^2)); complex128 plans must agree to 1e-7
relative to max|grad|, complex64 plans to 2e-4 (FP32 states, with unitary gates undone
in FP32 on the way back).
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


def fd_grad(pr, bits, theta, amp_fn, h=1e-5):
    f = lambda th: O.loss_from_amplitudes(amp_fn(th))
    return O.fd_gradient(f, theta, h)


def schrodinger_at(pr, bits):
    idx = np.asarray(bits, dtype=np.int64)
    return lambda th: O.schrodinger(pr.n, pr.gates, th)[idx]


def gpu_grad(pr, bits, theta, prec):
    import torch
    from paper_2502_06959_gb300 import hsf
    plan = hsf.Plan(pr.n, pr.gates, pr.cut, pr.blocks, precision=prec, angles=theta)
    b = torch.from_numpy(np.asarray(bits, dtype=np.uint64).view(np.int64)).cuda()
    amps = plan.run(b)
    g = plan.grad(b, 2 * amps, len(theta))
    hsf.hsf_sync(plan.handle)
    out = g.cpu().numpy()
    plan.close()
    return out


def mixed_circuit(n, cut, seed, layers=3):
    """Rotations of every supported kind with shared angles, inside both halves and
    inside jointly cut blocks."""
    rng = np.random.default_rng(seed)
    gates, blocks = [], []
    nparam = 6
    for layer in range(layers):
        for q in range(n):
            k = ["rx", "ry", "rz"][(q + layer) % 3]
            gates.append(Gate(k, (q,), param=0.0, param_id=int(rng.integers(nparam))))
        for q in range(0, n - 1):
            if q == cut:
                continue
            gates.append(Gate("rzz", (q + 1, q), param=0.0, param_id=int(rng.integers(nparam))))
        blk = []
        for j in range(2):
            blk.append(len(gates)); gates.append(Gate("rzz", (cut + 1, cut), param_id=int(rng.integers(nparam))))
            blk.append(len(gates)); gates.append(Gate("matrix", (cut,), matrix=W.haar_u2(rng)))
        blk.append(len(gates)); gates.append(Gate("cx", (cut + 1, cut)))
        blocks.append(blk)
    theta = rng.uniform(0, 2 * np.pi, nparam)
    return W.Problem(n, gates, cut, blocks, num_params=nparam, params=theta)


@pytest.mark.parametrize("prec,tol", [("c128", 1e-7), ("c64", 2e-4)])
def test_qaoa_ring_gradient_small(prec, tol):
    pr = W.qaoa_ring(10, 4, 2, seed=7)
    bits = W.random_bitstrings(np.random.default_rng(1), pr.n, 60)
    g = gpu_grad(pr, bits, pr.params, prec)
    ref = fd_grad(pr, bits, pr.params, schrodinger_at(pr, bits))
    assert np.max(np.abs(g - ref)) <= tol * np.max(np.abs(ref)), (g, ref)


@pytest.mark.parametrize("prec,tol", [("c128", 1e-7), ("c64", 2e-4)])
@pytest.mark.parametrize("seed", range(3))
def test_mixed_rotation_gradient(prec, tol, seed):
    pr = mixed_circuit(9, 4, seed)
    bits = W.random_bitstrings(np.random.default_rng(seed), pr.n, 40)
    g = gpu_grad(pr, bits, pr.params, prec)
    ref = fd_grad(pr, bits, pr.params, schrodinger_at(pr, bits))
    assert np.max(np.abs(g - ref)) <= tol * np.max(np.abs(ref)), (g, ref)


def test_autograd_function_matches_oracle():
    import torch
    from paper_2502_06959_gb300 import hsf
    pr = W.qaoa_ring(8, 3, 2, seed=11)
    bits = W.random_bitstrings(np.random.default_rng(2), pr.n, 30)
    b = torch.from_numpy(bits.view(np.int64)).cuda()
    theta = torch.tensor(pr.params, dtype=torch.float64, requires_grad=True)
    amps = hsf.HSFAmplitudes.apply(theta, pr, b, "c128")
    loss = (amps.abs() ** 2).sum()
    loss.backward()
    ref = fd_grad(pr, bits, pr.params, schrodinger_at(pr, bits))
    assert abs(loss.item() - O.loss_from_amplitudes(schrodinger_at(pr, bits)(pr.params))) < 1e-12
    assert np.max(np.abs(theta.grad.numpy() - ref)) <= 1e-7 * np.max(np.abs(ref))


def test_c4_qaoa_gradient_full_size():
    """n = 28 (14|14), p = 4, 1024 bitstrings, joint blocks: adjoint gradient against
    central differences of the oracle's HSF path sum for a gamma and a beta angle."""
    pr = W.workload_c4()
    g = gpu_grad(pr, pr.bitstrings, pr.params, "c64")

    def amps(th):
        return O.hsf_amplitudes(pr.n, pr.gates, pr.cut, pr.blocks, bitstrings=pr.bitstrings, theta=th)[0]
    for j in (1, 5):
        h = 1e-4
        tp = pr.params.copy(); tp[j] += h
        tm = pr.params.copy(); tm[j] -= h
        fd = (O.loss_from_amplitudes(amps(tp)) - O.loss_from_amplitudes(amps(tm))) / (2 * h)
        assert abs(g[j] - fd) <= 2e-4 * np.max(np.abs(g)) + 1e-6 * abs(fd), (j, g[j], fd)


def gpu_grad_budget(pr, bits, theta, prec, budget):
    import torch
    from paper_2502_06959_gb300 import hsf
    plan = hsf.Plan(pr.n, pr.gates, pr.cut, pr.blocks, precision=prec, angles=theta)
    b = torch.from_numpy(np.asarray(bits, dtype=np.uint64).view(np.int64)).cuda()
    amps = plan.run(b)
    need = hsf.hsf_grad_workspace_size(plan.handle, b.numel(), budget)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    g = torch.empty(len(theta), dtype=torch.float64, device="cuda")
    gout = (2 * amps).contiguous()
    st = torch.cuda.current_stream()
    hsf.hsf_grad(plan.handle, b.data_ptr(), b.numel(), gout.data_ptr(), g.data_ptr(), len(theta), ws.data_ptr(),
                 need, st.cuda_stream)
    hsf.hsf_sync(plan.handle, st.cuda_stream)
    out = g.cpu().numpy()
    plan.close()
    return out, need


def test_chunked_adjoint_equals_whole_tree_and_fd():
    """Forward states recomputed per subtree chunk (small workspace) give the gradient of
    the whole-tree layout, and both match the oracle's central differences."""
    from paper_2502_06959_gb300 import hsf
    pr = mixed_circuit(12, 5, 4, layers=6)
    bits = W.random_bitstrings(np.random.default_rng(4), pr.n, 50)
    g0, full = gpu_grad_budget(pr, bits, pr.params, "c128", 0)
    # the smallest budget that holds a layout: the tree is then walked in subtree chunks
    plan = hsf.Plan(pr.n, pr.gates, pr.cut, pr.blocks, precision="c128", angles=pr.params)
    budget = None
    for f in np.linspace(0.1, 1.0, 19):
        try:
            hsf.hsf_grad_workspace_size(plan.handle, bits.size, int(full * f))
            budget = int(full * f)
            break
        except hsf.HsfError:
            continue
    plan.close()
    assert budget is not None and budget <= 0.7 * full, (budget, full)
    g1, small = gpu_grad_budget(pr, bits, pr.params, "c128", budget)
    assert small <= budget < full
    assert np.max(np.abs(g1 - g0)) <= 1e-12 * np.max(np.abs(g0))
    ref = fd_grad(pr, bits, pr.params, schrodinger_at(pr, bits))
    assert np.max(np.abs(g1 - ref)) <= 1e-7 * np.max(np.abs(ref))


def test_c4_all_angles_against_stored_fd():
    """All 8 angles of the n = 28 QAOA workload (1024 bitstrings): the complex128 adjoint
    within 1e-6 of max|g| of the stored FP64 central differences (oracle HSF path sum,
    tests/golden/c4_fd_gradient.json), the complex64 adjoint within 1e-4."""
    import json
    import os
    rec = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "c4_fd_gradient.json")))
    pr = W.workload_c4()
    assert np.allclose(rec["theta"], pr.params, rtol=0, atol=0)
    ref = np.array(rec["grad_richardson"])
    assert rec["fd_error_bound"] <= 1e-3 * np.max(np.abs(ref))
    scale = np.max(np.abs(ref))
    g128 = gpu_grad(pr, pr.bitstrings, pr.params, "c128")
    assert np.max(np.abs(g128 - ref)) <= 1e-6 * scale, (g128, ref)
    g64 = gpu_grad(pr, pr.bitstrings, pr.params, "c64")
    assert np.max(np.abs(g64 - ref)) <= 1e-4 * scale, (g64, ref)


def test_c2_shaped_gradient_in_the_run_workspace():
    """n = 30, 8 jointly cut blocks, 65536 paths: angles on every block's RZZ gates (one
    shared angle) and on in-half RY rotations.  The gradient runs in a workspace no
    larger than the forward run's (the whole tree would need ~90 GB in complex64), and
    matches central differences of the library's own complex128 forward."""
    import torch
    from paper_2502_06959_gb300 import hsf
    pr = W.workload_c2(num_bitstrings=256)
    gates = list(pr.gates)
    for gi in sorted(set(i for b in pr.blocks for i in b)):
        if gates[gi].kind == "rzz":
            gates[gi] = Gate("rzz", gates[gi].qubits, param=gates[gi].param, param_id=0)
    ry = [i for i, g in enumerate(gates) if g.kind == "matrix" and len(g.qubits) == 1
          and not any(i in b for b in pr.blocks)]
    rng = np.random.default_rng(5)
    for j, gi in enumerate(rng.choice(ry, size=6, replace=False)):
        gates[gi] = Gate("ry", gates[gi].qubits, param=0.0, param_id=1 + j % 2)
    theta = np.array([0.7, 1.3, -0.4])
    q = W.Problem(pr.n, gates, pr.cut, pr.blocks, num_params=3, params=theta, bitstrings=pr.bitstrings)
    plan = hsf.Plan(q.n, q.gates, q.cut, q.blocks, precision="c128", angles=theta)
    run_ws = hsf.hsf_workspace_size(plan.handle, 256, 0, int(torch.cuda.mem_get_info()[0] * 0.25))
    plan.close()
    g, need = gpu_grad_budget(q, q.bitstrings, theta, "c128", run_ws)
    assert need <= run_ws

    def loss(th):
        p = hsf.Plan(q.n, q.gates, q.cut, q.blocks, precision="c128", angles=th)
        b = torch.from_numpy(q.bitstrings.view(np.int64)).cuda()
        v = float((p.run(b).abs() ** 2).sum())
        p.close()
        return v
    fd = O.fd_gradient(loss, theta, h=1e-5)
    assert np.max(np.abs(g - fd)) <= 1e-6 * np.max(np.abs(fd)), (g, fd)
