"""ctypes front end of the C Schroedinger oracle (oracle/schrodinger.c, O1 of Sec. II-A).

TEST INFRASTRUCTURE ONLY: importable by the tests, the smoke check, the scripts that
write stored expected values under tests/golden/ and the benchmark's CPU-baseline leg.

The gate matrices come from ``hsf_oracle.gate_matrix`` (the oracle's own closed-form
definitions); the C code only applies them one gate at a time to the full statevector.
The library is compiled with gcc into this directory on first use (or by ``build()``).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Optional, Sequence

import numpy as np

from .hsf_oracle import gate_matrix

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "schrodinger.c")
LIB = os.path.join(HERE, "liboracle_sv.so")

_lib = None


def build(force: bool = False) -> str:
    """Compile liboracle_sv.so with gcc (plain C, OpenMP)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".{os.getpid()}.tmp"
        subprocess.run(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", SRC, "-o", tmp],
                       check=True)
        os.replace(tmp, LIB)
    return LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(LIB)
        P = ctypes.c_void_p
        lib.oracle_schrodinger.restype = ctypes.c_int
        lib.oracle_schrodinger.argtypes = [ctypes.c_int, ctypes.c_int, P, P, P, P, P]
        lib.oracle_apply_gates.restype = ctypes.c_int
        lib.oracle_apply_gates.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, P, P, P, P, P]
        _lib = lib
    return _lib


class _Marshalled:
    def __init__(self, gates, theta=None):
        G = len(gates)
        self.nq = np.zeros(max(G, 1), dtype=np.int32)
        self.qubits = np.zeros(4 * max(G, 1), dtype=np.int32)
        self.off = np.zeros(max(G, 1), dtype=np.int64)
        mats = []
        pos = 0
        for i, g in enumerate(gates):
            m = np.ascontiguousarray(gate_matrix(g, theta), dtype=np.complex128)
            k = len(g.qubits)
            assert m.shape == (1 << k, 1 << k)
            self.nq[i] = k
            self.qubits[4 * i:4 * i + k] = g.qubits
            self.off[i] = pos
            mats.append(m.ravel())
            pos += m.size
        self.mats = np.concatenate(mats) if mats else np.zeros(1, dtype=np.complex128)
        self.G = G

    def ptrs(self):
        return (self.nq.ctypes.data, self.qubits.ctypes.data, self.mats.ctypes.data, self.off.ctypes.data)


def schrodinger_c(n: int, gates, theta: Optional[Sequence[float]] = None, out: Optional[np.ndarray] = None):
    """Full statevector G_T ... G_1 |0...0> (complex128, 2^n entries)."""
    lib = _load()
    mg = _Marshalled(gates, theta)
    psi = out if out is not None else np.empty(1 << n, dtype=np.complex128)
    assert psi.dtype == np.complex128 and psi.size == (1 << n) and psi.flags.c_contiguous
    rc = lib.oracle_schrodinger(n, mg.G, *mg.ptrs(), psi.ctypes.data)
    if rc != 0:
        raise ValueError("oracle_schrodinger rejected the circuit")
    return psi


def apply_gates_c(n: int, gates, psi: np.ndarray, g0: int, g1: int, theta=None) -> None:
    """psi <- gates [g0, g1) applied in order, in place (for bounded timing samples)."""
    lib = _load()
    mg = _Marshalled(gates, theta)
    rc = lib.oracle_apply_gates(n, g0, g1, *mg.ptrs(), psi.ctypes.data)
    if rc != 0:
        raise ValueError("oracle_apply_gates rejected the circuit")
