"""Thin ctypes binding of libhsf (include/hsf.h): argument marshalling only.

Every numerical step runs in the library's CUDA kernels.  The functions keep the C
names (``hsf_plan_create``, ``hsf_run``, ...); ``Plan`` is a small owner object that
frees the native plan and caches a device workspace allocated through PyTorch.

The library is loaded from this package directory; if it is missing the import of
this module raises (there is no fallback path).
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhsf.so")

HSF_OK = 0
STATUS = {0: "HSF_OK", 1: "HSF_EINVAL", 2: "HSF_EBLOCK", 3: "HSF_ERANK", 4: "HSF_ENOMEM",
          5: "HSF_ECUDA", 6: "HSF_ETIMEOUT", 7: "HSF_ENUMERIC", 8: "HSF_ENOTSUP"}
KIND = {"matrix": 0, "h": 1, "x": 2, "y": 3, "z": 4, "s": 5, "t": 6, "rx": 7, "ry": 8, "rz": 9,
        "cx": 10, "cz": 11, "swap": 12, "iswap": 13, "rzz": 14}
PREC = {"c64": 0, "c128": 1}
GEMM = {"fp32": 0, "bf16x3": 1, "tf32x3": 2, "tf32": 3}
FLAG_NO_LIGHTCONE = 1
FLAG_NO_LEAF_CONTRACT = 2
FLAG_NO_REGISTER_SWEEP = 4
FLAG_IDENTITY_STORAGE = 8
FLAG_REG5 = 16
FLAG_REG3 = 32
FLAG_NO_TC_LEVEL = 64
FLAG_SVD_BLOCKS = 128
FLAG_LEAF_DOTS = 256


class HsfError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class hsf_gate(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("nq", ctypes.c_int32), ("q", ctypes.c_int32 * 4),
                ("param", ctypes.c_double), ("param_id", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("mat", ctypes.POINTER(ctypes.c_double))]


class hsf_circuit(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("num_gates", ctypes.c_int32),
                ("gates", ctypes.POINTER(hsf_gate))]


class hsf_blocks(ctypes.Structure):
    _fields_ = [("num_blocks", ctypes.c_int32), ("offsets", ctypes.POINTER(ctypes.c_int32)),
                ("gate_idx", ctypes.POINTER(ctypes.c_int32))]


class hsf_plan_opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("gemm_mode", ctypes.c_int32),
                ("rank_tol", ctypes.c_double), ("max_paths", ctypes.c_uint64),
                ("tile_bits", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("angles", ctypes.POINTER(ctypes.c_double)), ("num_angles", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class hsf_batch_item(ctypes.Structure):
    _fields_ = [("plan", ctypes.c_void_p), ("bitstrings", ctypes.c_void_p), ("num", ctypes.c_size_t),
                ("window", ctypes.c_uint64), ("out", ctypes.c_void_p)]


class hsf_plan_info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("n_a", ctypes.c_int32), ("n_b", ctypes.c_int32),
                ("num_blocks", ctypes.c_int32), ("num_paths", ctypes.c_uint64),
                ("precision", ctypes.c_int32), ("max_rank", ctypes.c_int32),
                ("tree_nodes", ctypes.c_int64), ("num_launches", ctypes.c_int64),
                ("leaf_bits", ctypes.c_int32), ("num_params", ctypes.c_int32)]


# symbol -> (restype, argtypes); also the list the load test checks against the header
SIGNATURES = {
    "hsf_plan_create": (ctypes.c_int, [ctypes.POINTER(hsf_circuit), ctypes.c_int32,
                                       ctypes.POINTER(hsf_blocks), ctypes.POINTER(hsf_plan_opts),
                                       ctypes.POINTER(ctypes.c_void_p)]),
    "hsf_plan_get_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(hsf_plan_info)]),
    "hsf_plan_create_schrodinger": (ctypes.c_int, [ctypes.POINTER(hsf_circuit), ctypes.POINTER(hsf_plan_opts),
                                                   ctypes.POINTER(ctypes.c_void_p)]),
    "hsf_plan_get_sigma": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32,
                                          ctypes.POINTER(ctypes.c_double), ctypes.c_int32,
                                          ctypes.POINTER(ctypes.c_int32)]),
    "hsf_plan_destroy": (None, [ctypes.c_void_p]),
    "hsf_workspace_size": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_uint64,
                                          ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]),
    "hsf_run": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_uint64,
                               ctypes.c_uint64, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p,
                               ctypes.c_size_t, ctypes.c_void_p]),
    "hsf_run_static": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_uint64,
                                      ctypes.c_uint64, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p]),
    "hsf_sync": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "hsf_plan_describe": (ctypes.c_int64, [ctypes.c_void_p, ctypes.c_char_p, ctypes.c_int64]),
    "hsf_batch_workspace_size": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(ctypes.c_size_t)]),
    "hsf_batch_create": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_size_t,
                                        ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
    "hsf_batch_launch": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "hsf_batch_nodes": (ctypes.c_int64, [ctypes.c_void_p]),
    "hsf_batch_destroy": (None, [ctypes.c_void_p]),
    "hsf_tune": (ctypes.c_int, [ctypes.POINTER(hsf_circuit), ctypes.c_int32, ctypes.POINTER(hsf_blocks),
                                ctypes.POINTER(hsf_plan_opts), ctypes.c_size_t, ctypes.c_void_p, ctypes.c_uint64,
                                ctypes.c_char_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]),
    "hsf_grad_workspace_size": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_size_t,
                                               ctypes.POINTER(ctypes.c_size_t)]),
    "hsf_grad": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p,
                                ctypes.c_int32, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    "hsf_set_allocator": (None, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "hsf_find_blocks": (ctypes.c_int, [ctypes.POINTER(hsf_circuit), ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                       ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]),
    "hsf_search_cut": (ctypes.c_int, [ctypes.POINTER(hsf_circuit), ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                      ctypes.c_uint64, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(ctypes.c_double)]),
    "hsf_last_error": (ctypes.c_char_p, []),
    "hsf_set_profiling": (None, [ctypes.c_int32]),
    "hsf_profile_collect": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32]),
    "hsf_launch_count": (ctypes.c_uint64, []),
    "hsf_version": (ctypes.c_char_p, []),
}

KERNEL_KINDS = ("sweep", "gather", "reduce", "window", "other", "leaf", "level_mma", "level_f16", "pack")


class hsf_kernel_stat(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64), ("ms", ctypes.c_double), ("bytes", ctypes.c_double),
                ("flops", ctypes.c_double)]


_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libhsf.so (raises OSError if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OSError(f"{path} not found: build it with `python -m paper_2502_06959_gb300.build`")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(code: int):
    if code != HSF_OK:
        raise HsfError(code, load_library().hsf_last_error().decode())


# numpy twin of hsf_gate (same field offsets), so a gate list marshals in a few array
# operations instead of one ctypes attribute write per field
_GATE_DTYPE = np.dtype({"names": ["kind", "nq", "q", "param", "param_id", "reserved", "mat"],
                        "formats": [np.int32, np.int32, (np.int32, 4), np.float64, np.int32, np.int32,
                                    np.uint64],
                        "offsets": [hsf_gate.kind.offset, hsf_gate.nq.offset, hsf_gate.q.offset,
                                    hsf_gate.param.offset, hsf_gate.param_id.offset,
                                    hsf_gate.reserved.offset, hsf_gate.mat.offset],
                        "itemsize": ctypes.sizeof(hsf_gate)})


def _marshal(n: int, gates, blocks: Sequence[Sequence[int]]):
    ng = len(gates)
    arr = np.zeros(max(1, ng), dtype=_GATE_DTYPE)
    keep = [arr]
    if ng:
        arr["kind"][:ng] = [KIND[g.kind] for g in gates]
        arr["nq"][:ng] = [len(g.qubits) for g in gates]
        arr["q"][:ng] = [tuple(g.qubits) + (0,) * (4 - len(g.qubits)) for g in gates]
        arr["param"][:ng] = [g.param for g in gates]
        arr["param_id"][:ng] = [g.param_id for g in gates]
        mi = [i for i, g in enumerate(gates) if g.kind == "matrix"]
        if mi:
            # all explicit 2x2 / 4x4 matrices in one buffer; each gate points at its slice
            mats = [np.asarray(gates[i].matrix, dtype=np.complex128).ravel() for i in mi]
            sizes = np.array([m.size for m in mats])
            buf = np.ascontiguousarray(np.concatenate(mats)).view(np.float64)
            keep.append(buf)
            starts = np.concatenate(([0], np.cumsum(sizes)[:-1])) * 16
            arr["mat"][mi] = buf.ctypes.data + starts
    circ = hsf_circuit(n, ng, ctypes.cast(arr.ctypes.data, ctypes.POINTER(hsf_gate)))
    offs = np.zeros(len(blocks) + 1, dtype=np.int32)
    idx = []
    for b, blk in enumerate(blocks):
        idx.extend(int(x) for x in blk)
        offs[b + 1] = len(idx)
    idx = np.asarray(idx if idx else [0], dtype=np.int32)
    keep += [offs, idx]
    bl = hsf_blocks(len(blocks), offs.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                    idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    return circ, bl, keep


class Marshalled:
    """A circuit and its blocks in the C ABI's structs, built once: planning the same
    circuit again (new angles, or every step of a benchmark) then skips the Python-side
    conversion of the gate list."""

    def __init__(self, n: int, gates, blocks):
        self.n = n
        self.circ, self.bl, self._keep = _marshal(n, gates, blocks)


def hsf_plan_create(n: int, gates, cut: int, blocks, precision: str = "c64", gemm: str = "fp32",
                    rank_tol: float = 0.0, max_paths: int = 0, tile_bits: int = 0, flags: int = 0,
                    angles: Optional[Sequence[float]] = None, marshalled: Optional[Marshalled] = None) -> int:
    """hsf_plan_create; `marshalled` (from Marshalled(n, gates, blocks)) reuses the C
    structs of an earlier conversion of the same circuit."""
    lib = load_library()
    if marshalled is not None:
        circ, bl, keep = marshalled.circ, marshalled.bl, []
    else:
        circ, bl, keep = _marshal(n, gates, blocks)
    opts = hsf_plan_opts()
    opts.precision = PREC[precision]
    opts.gemm_mode = GEMM[gemm]
    opts.rank_tol = rank_tol
    opts.max_paths = max_paths
    opts.tile_bits = tile_bits
    opts.flags = flags
    if angles is not None:
        ang = np.ascontiguousarray(angles, dtype=np.float64)
        keep.append(ang)
        opts.angles = ang.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        opts.num_angles = ang.size
    out = ctypes.c_void_p()
    _check(lib.hsf_plan_create(ctypes.byref(circ), cut, ctypes.byref(bl), ctypes.byref(opts),
                               ctypes.byref(out)))
    return out.value


def hsf_plan_create_schrodinger(n: int, gates, precision: str = "c64", tile_bits: int = 0, flags: int = 0,
                                angles: Optional[Sequence[float]] = None) -> int:
    """Full-statevector plan of the circuit (no cut, no blocks); run it with hsf_run."""
    lib = load_library()
    circ, _, keep = _marshal(n, gates, [])
    opts = hsf_plan_opts()
    opts.precision = PREC[precision]
    opts.tile_bits = tile_bits
    opts.flags = flags
    if angles is not None:
        ang = np.ascontiguousarray(angles, dtype=np.float64)
        keep.append(ang)
        opts.angles = ang.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        opts.num_angles = ang.size
    out = ctypes.c_void_p()
    _check(lib.hsf_plan_create_schrodinger(ctypes.byref(circ), ctypes.byref(opts), ctypes.byref(out)))
    return out.value


def hsf_find_blocks(n: int, gates, cut: int, max_leaves: int = 8):
    """Joint-cut blocks found by the library (hsf_find_blocks): returns (order, blocks,
    hubs) where order[i] is the input index of the i-th gate of the reordered circuit and
    blocks index the reordered circuit."""
    lib = load_library()
    circ, _, keep = _marshal(n, gates, [])
    G = len(gates)
    order = np.zeros(max(G, 1), dtype=np.int32)
    cap = max(G, 1)
    offs = np.zeros(cap + 1, dtype=np.int32)
    idx = np.zeros(max(G, 1), dtype=np.int32)
    nb, hubs = ctypes.c_int32(), ctypes.c_int32()
    _check(lib.hsf_find_blocks(ctypes.byref(circ), cut, max_leaves, order.ctypes.data, offs.ctypes.data,
                               idx.ctypes.data, cap, ctypes.byref(nb), ctypes.byref(hubs)))
    blocks = [[int(x) for x in idx[offs[b]:offs[b + 1]]] for b in range(nb.value)]
    return [int(x) for x in order[:G]], blocks, int(hubs.value)


def problem_with_found_blocks(problem, max_leaves: int = 8):
    """The problem's circuit reordered and cut into the blocks hsf_find_blocks finds."""
    import copy
    order, blocks, hubs = hsf_find_blocks(problem.n, problem.gates, problem.cut, max_leaves)
    out = copy.copy(problem)
    out.gates = [problem.gates[i] for i in order]
    out.blocks = blocks
    out.meta = dict(problem.meta, hubs=hubs, found_blocks=len(blocks))
    return out


def hsf_search_cut(n: int, gates, cut: int, max_leaves: int = 8, restarts: int = 4, seed: int = 1):
    """Qubit-reordering search (hsf_search_cut): returns (perm, log2_paths_before,
    log2_paths_after) where perm[q] is the new label of qubit q."""
    lib = load_library()
    circ, _, keep = _marshal(n, gates, [])
    perm = np.zeros(n, dtype=np.int32)
    before, after = ctypes.c_double(), ctypes.c_double()
    _check(lib.hsf_search_cut(ctypes.byref(circ), cut, max_leaves, restarts, seed, perm.ctypes.data,
                              ctypes.byref(before), ctypes.byref(after)))
    return [int(x) for x in perm], float(before.value), float(after.value)


def relabel_problem(problem, perm):
    """The same circuit with qubit q renamed perm[q] (gates, bitstrings); blocks are
    dropped (find them again on the relabeled circuit)."""
    import copy
    from . import workloads as W
    out = copy.copy(problem)
    out.gates = [W.Gate(g.kind, tuple(perm[q] for q in g.qubits), g.param, g.param_id, g.matrix)
                 for g in problem.gates]
    out.blocks = []
    if problem.bitstrings is not None:
        src = problem.bitstrings.astype(np.uint64)
        dst = np.zeros_like(src)
        for q, t in enumerate(perm):
            dst |= ((src >> np.uint64(q)) & np.uint64(1)) << np.uint64(t)
        out.bitstrings = dst
    out.meta = dict(problem.meta, perm=list(perm))
    return out


def problem_with_searched_cut(problem, max_leaves: int = 8, restarts: int = 4, seed: int = 1):
    """hsf_search_cut, then the relabeled circuit cut into the blocks hsf_find_blocks
    finds (the cut position stays problem.cut)."""
    perm, before, after = hsf_search_cut(problem.n, problem.gates, problem.cut, max_leaves, restarts, seed)
    out = problem_with_found_blocks(relabel_problem(problem, perm), max_leaves)
    out.meta = dict(out.meta, log2_paths_before=before, log2_paths_after=after)
    return out


def hsf_plan_get_info(plan: int) -> dict:
    info = hsf_plan_info()
    _check(load_library().hsf_plan_get_info(plan, ctypes.byref(info)))
    return {f: getattr(info, f) for f, _ in hsf_plan_info._fields_}


def hsf_plan_get_sigma(plan: int, block: int) -> np.ndarray:
    buf = (ctypes.c_double * 64)()
    rank = ctypes.c_int32()
    _check(load_library().hsf_plan_get_sigma(plan, block, buf, 64, ctypes.byref(rank)))
    return np.array(buf[:rank.value])


def hsf_plan_destroy(plan: int) -> None:
    if plan:
        load_library().hsf_plan_destroy(plan)


def hsf_workspace_size(plan: int, num_bitstrings: int = 0, window: int = 0, budget: int = 0) -> int:
    out = ctypes.c_size_t()
    _check(load_library().hsf_workspace_size(plan, num_bitstrings, window, budget, ctypes.byref(out)))
    return out.value


def hsf_run(plan: int, bitstrings_ptr: int, num: int, window: int, path_begin: int, path_end: int,
            out_ptr: int, workspace_ptr: int, workspace_bytes: int, stream: int = 0) -> None:
    """workspace_ptr = 0: the plan owns its workspace (see hsf_set_allocator)."""
    _check(load_library().hsf_run(plan, bitstrings_ptr or None, num, window, path_begin, path_end,
                                  out_ptr, workspace_ptr or None, workspace_bytes, stream or None))


_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)
_allocator_refs = []


def use_torch_allocator(on: bool = True) -> None:
    """Route plan-owned workspaces (hsf_run with workspace 0) through PyTorch's caching
    allocator (hsf_set_allocator); on=False restores the library's cudaMalloc default."""
    import torch
    lib = load_library()
    if not on:
        lib.hsf_set_allocator(None, None, None)
        _allocator_refs.clear()
        return

    def _alloc(ctx, nbytes, stream):
        try:
            return int(torch.cuda.caching_allocator_alloc(int(nbytes), stream=stream or 0))
        except Exception:
            return None

    def _free(ctx, ptr, stream):
        try:
            torch.cuda.caching_allocator_delete(int(ptr))
        except Exception:
            pass

    fa, ff = _ALLOC_FN(_alloc), _FREE_FN(_free)
    _allocator_refs[:] = [fa, ff]          # the library keeps the function pointers
    lib.hsf_set_allocator(ctypes.cast(fa, ctypes.c_void_p), ctypes.cast(ff, ctypes.c_void_p), None)


def hsf_set_profiling(on: bool) -> None:
    load_library().hsf_set_profiling(1 if on else 0)


def hsf_profile_collect(plan: int) -> dict:
    arr = (hsf_kernel_stat * len(KERNEL_KINDS))()
    _check(load_library().hsf_profile_collect(plan, arr, len(KERNEL_KINDS)))
    return {k: dict(launches=arr[i].launches, ms=arr[i].ms, bytes=arr[i].bytes, flops=arr[i].flops)
            for i, k in enumerate(KERNEL_KINDS)}


def hsf_launch_count() -> int:
    return int(load_library().hsf_launch_count())


def hsf_run_static(plan: int, bitstrings_ptr: int, num: int, window: int, path_begin: int,
                   path_end: int, out_ptr: int, stream: int = 0) -> None:
    """hsf_run without a workspace argument: for callers that cannot allocate device
    memory (the library's fixed 32 MiB scratch array is used instead)."""
    _check(load_library().hsf_run_static(plan, bitstrings_ptr or None, num, window, path_begin,
                                         path_end, out_ptr, stream or None))


def hsf_grad_workspace_size(plan: int, num_bitstrings: int, budget: int = 0) -> int:
    out = ctypes.c_size_t()
    _check(load_library().hsf_grad_workspace_size(plan, num_bitstrings, budget, ctypes.byref(out)))
    return out.value


def hsf_grad(plan: int, bitstrings_ptr: int, num: int, gout_ptr: int, grad_ptr: int, num_params: int,
             workspace_ptr: int, workspace_bytes: int, stream: int = 0) -> None:
    _check(load_library().hsf_grad(plan, bitstrings_ptr, num, gout_ptr, grad_ptr, num_params,
                                   workspace_ptr, workspace_bytes, stream or None))


def hsf_tune(n: int, gates, cut: int, blocks, num: int = 0, bitstrings_ptr: int = 0, window: int = 0,
             cache_path: Optional[str] = None, precision: str = "c64", gemm: str = "fp32",
             budget: int = 0) -> dict:
    """Autotune the configuration for this circuit shape and request; returns the plan
    options (tile_bits, flags, gemm) to pass to hsf_plan_create and the workspace budget
    ("budget") that sets the path batch."""
    import torch
    lib = load_library()
    circ, bl, keep = _marshal(n, gates, blocks)
    opts = hsf_plan_opts()
    opts.precision = PREC[precision]
    opts.gemm_mode = GEMM[gemm]
    probe = hsf_plan_create(n, gates, cut, blocks, precision=precision, gemm=gemm)
    if budget == 0:
        budget = int(torch.cuda.mem_get_info()[0] * 0.5)
    need = hsf_workspace_size(probe, num, window, budget)
    hsf_plan_destroy(probe)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    best_budget = ctypes.c_size_t()
    _check(lib.hsf_tune(ctypes.byref(circ), cut, ctypes.byref(bl), ctypes.byref(opts), num,
                        bitstrings_ptr or None, window, cache_path.encode() if cache_path else None,
                        ws.data_ptr(), need, ctypes.byref(best_budget)))
    inv = {v: k for k, v in GEMM.items()}
    return {"tile_bits": opts.tile_bits, "flags": opts.flags, "gemm": inv.get(opts.gemm_mode, gemm),
            "budget": int(best_budget.value)}


class Batch:
    """A CUDA graph holding hsf_run of every (plan, request) item; launch() replays it."""

    def __init__(self, items, stream=None):
        import torch
        lib = load_library()
        self.items = items          # keep plans, inputs and outputs alive
        arr = (hsf_batch_item * len(items))()
        for i, it in enumerate(items):
            bits = it.get("bitstrings")
            arr[i].plan = it["plan"].handle
            arr[i].bitstrings = bits.data_ptr() if bits is not None else None
            arr[i].num = bits.numel() if bits is not None else 0
            arr[i].window = it.get("window", 0)
            arr[i].out = it["out"].data_ptr()
        need = ctypes.c_size_t()
        _check(lib.hsf_batch_workspace_size(arr, len(items), ctypes.byref(need)))
        self.ws = torch.empty(need.value, dtype=torch.uint8, device="cuda")
        # stream capture needs a non-default stream
        if stream is None or stream.cuda_stream == 0:
            stream = torch.cuda.Stream()
        self.stream = stream
        h = ctypes.c_void_p()
        _check(lib.hsf_batch_create(arr, len(items), self.ws.data_ptr(), self.ws.numel(),
                                    self.stream.cuda_stream, ctypes.byref(h)))
        self.handle = h.value
        self.nodes = int(lib.hsf_batch_nodes(self.handle))

    def launch(self, stream=None):
        st = stream or self.stream
        _check(load_library().hsf_batch_launch(self.handle, st.cuda_stream))

    def close(self):
        if self.handle:
            load_library().hsf_batch_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def hsf_plan_describe(plan: int) -> str:
    lib = load_library()
    n = lib.hsf_plan_describe(plan, None, 0)
    buf = ctypes.create_string_buffer(int(n))
    lib.hsf_plan_describe(plan, buf, n)
    return buf.value.decode()


def hsf_sync(plan: int, stream: int = 0) -> None:
    _check(load_library().hsf_sync(plan, stream or None))


def hsf_version() -> str:
    return load_library().hsf_version().decode()


class Plan:
    """Owner of a native plan plus a cached PyTorch workspace.

    ``run`` returns a complex128 CUDA tensor with the requested amplitudes."""

    def __init__(self, n: int, gates, cut: int, blocks, **opts):
        self.n = n
        self.cut = cut
        self.handle = hsf_plan_create(n, gates, cut, blocks, **opts)
        self.info = hsf_plan_get_info(self.handle)
        self._ws = None

    @classmethod
    def from_problem(cls, problem, **opts):
        return cls(problem.n, problem.gates, problem.cut, problem.blocks, **opts)

    @classmethod
    def schrodinger(cls, n: int, gates, **opts):
        """A full-statevector plan of the circuit (hsf_plan_create_schrodinger)."""
        self = cls.__new__(cls)
        self.n = n
        self.cut = -1
        self.handle = hsf_plan_create_schrodinger(n, gates, **opts)
        self.info = hsf_plan_get_info(self.handle)
        self._ws = None
        return self

    def sigma(self, block: int) -> np.ndarray:
        return hsf_plan_get_sigma(self.handle, block)

    def workspace(self, num_bitstrings: int = 0, window: int = 0, budget: int = 0):
        import torch
        if budget == 0:
            free, _ = torch.cuda.mem_get_info()
            budget = int(free * 0.6)
        need = hsf_workspace_size(self.handle, num_bitstrings, window, budget)
        if self._ws is None or self._ws.numel() < need:
            self._ws = None
            self._ws = torch.empty(need, dtype=torch.uint8, device="cuda")
        return self._ws

    def run(self, bitstrings=None, window: int = 0, path_range=(0, 0), out=None, stream=None,
            budget: int = 0, check: bool = False):
        import torch
        num = 0 if bitstrings is None else int(bitstrings.numel())
        if bitstrings is not None and num == 0:
            return torch.empty(0, dtype=torch.complex128, device="cuda")
        count = num if num else (window if window else (1 << self.n))
        if out is None:
            out = torch.empty(count, dtype=torch.complex128, device="cuda")
        ws = self.workspace(num, window, budget)
        st = stream if stream is not None else torch.cuda.current_stream()
        hsf_run(self.handle, bitstrings.data_ptr() if num else 0, num, window,
                int(path_range[0]), int(path_range[1]), out.data_ptr(), ws.data_ptr(), ws.numel(),
                st.cuda_stream)
        if check:
            hsf_sync(self.handle, st.cuda_stream)
        return out

    def grad(self, bitstrings, gout, num_params: int = 0, stream=None, budget: int = 0):
        """dL/dtheta (float64 CUDA tensor) for the upstream gradient gout (complex128,
        one per bitstring).  The workspace is sized for `budget` bytes (0: half the free
        device memory); the library then recomputes forward states per path chunk."""
        import torch
        num = int(bitstrings.numel())
        num_params = max(num_params, int(self.info["num_params"]))
        if budget == 0:
            budget = int(torch.cuda.mem_get_info()[0] * 0.5)
        need = hsf_grad_workspace_size(self.handle, num, budget)
        ws = torch.empty(max(need, 256), dtype=torch.uint8, device="cuda")
        g = torch.empty(max(num_params, 1), dtype=torch.float64, device="cuda")
        st = stream if stream is not None else torch.cuda.current_stream()
        gout = gout.to(torch.complex128).contiguous()
        hsf_grad(self.handle, bitstrings.data_ptr(), num, gout.data_ptr(), g.data_ptr(), num_params,
                 ws.data_ptr(), ws.numel(), st.cuda_stream)
        return g[:num_params]

    def close(self):
        if self.handle:
            hsf_plan_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _autograd_function():
    import torch

    class HSFAmplitudes(torch.autograd.Function):
        """amps = HSFAmplitudes.apply(angles, problem, bitstrings, precision)

        Forward: plan the circuit with the given shared angles (param_id j takes
        angles[j]) and return the complex128 amplitudes at the bitstrings.  Backward:
        the library's adjoint pass (hsf_grad) maps the upstream gradient of the
        amplitudes to dL/dangles."""

        @staticmethod
        def forward(ctx, angles, problem, bitstrings, precision="c64"):
            ang = angles.detach().to("cpu", torch.float64).numpy()
            plan = Plan(problem.n, problem.gates, problem.cut, problem.blocks, precision=precision,
                        angles=ang)
            amps = plan.run(bitstrings)
            ctx.plan = plan
            ctx.bits = bitstrings
            ctx.nparams = angles.numel()
            ctx.dtype = angles.dtype
            ctx.device = angles.device
            return amps

        @staticmethod
        def backward(ctx, gout):
            g = ctx.plan.grad(ctx.bits, gout, ctx.nparams)
            ctx.plan.close()
            return g.to(device=ctx.device, dtype=ctx.dtype), None, None, None

    return HSFAmplitudes


_FUNCTION = None


def __getattr__(name):
    global _FUNCTION
    if name == "HSFAmplitudes":
        if _FUNCTION is None:
            _FUNCTION = _autograd_function()
        return _FUNCTION
    raise AttributeError(name)
