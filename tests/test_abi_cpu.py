"""CPU checks of the C ABI: the library builds, loads and exports every symbol the
header declares; the ctypes structs match the C layout; and argument validation
rejects bad circuits, cuts and blocks before any device work."""
import ctypes
import os
import re
import subprocess
import tempfile

import numpy as np
import pytest

from paper_2502_06959_gb300 import build as B
from paper_2502_06959_gb300 import hsf as H
from paper_2502_06959_gb300 import workloads as W
from paper_2502_06959_gb300.workloads import Gate

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hsf.h")


@pytest.fixture(scope="module")
def lib():
    B.build()
    return H.load_library()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hsf_[a-z_0-9]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert "hsf_run" in names and "hsf_plan_create" in names
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\b(hsf_[a-z_0-9]+)\b", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        getattr(lib, n)
    # the binding marshals exactly the declared entry points
    assert set(H.SIGNATURES) <= set(names)


def test_flag_constants_match_header():
    """Every HSF_FLAG_* of the header has the same value as the binding's FLAG_*."""
    text = open(HEADER).read()
    flags = dict(re.findall(r"#define HSF_FLAG_([A-Z0-9_]+)\s+(\d+)", text))
    assert "LEAF_DOTS" in flags and "NO_LEAF_CONTRACT" in flags
    for name, value in flags.items():
        assert getattr(H, "FLAG_" + name) == int(value), name
    assert len(set(flags.values())) == len(flags), "flag bits are distinct"


def test_struct_layouts_match_header():
    src = r"""
    #include <stdio.h>
    #include <stddef.h>
    #include "hsf.h"
    int main(void) {
      printf("%zu %zu %zu %zu %zu\n", sizeof(hsf_gate), offsetof(hsf_gate, param),
             offsetof(hsf_gate, mat), sizeof(hsf_circuit), sizeof(hsf_blocks));
      printf("%zu %zu %zu %zu\n", sizeof(hsf_plan_opts), offsetof(hsf_plan_opts, max_paths),
             offsetof(hsf_plan_opts, angles), sizeof(hsf_plan_info));
      return 0;
    }
    """
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "l.c")
        open(c, "w").write(src)
        exe = os.path.join(d, "l")
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        vals = [int(x) for x in subprocess.check_output([exe]).split()]
    got = [ctypes.sizeof(H.hsf_gate), H.hsf_gate.param.offset, H.hsf_gate.mat.offset,
           ctypes.sizeof(H.hsf_circuit), ctypes.sizeof(H.hsf_blocks),
           ctypes.sizeof(H.hsf_plan_opts), H.hsf_plan_opts.max_paths.offset,
           H.hsf_plan_opts.angles.offset, ctypes.sizeof(H.hsf_plan_info)]
    assert vals == got


def test_version_string(lib):
    assert "sm_103a" in H.hsf_version()


def _expect(code, *args, **kw):
    with pytest.raises(H.HsfError) as ei:
        H.hsf_plan_create(*args, **kw)
    assert ei.value.code == code, str(ei.value)
    assert H.load_library().hsf_last_error()


def test_validation_errors(lib):
    g = [Gate("h", (0,)), Gate("cx", (2, 1)), Gate("h", (1,)), Gate("cx", (2, 1))]
    _expect(1, 3, [Gate("h", (5,))], 1, [])                         # qubit out of range
    _expect(1, 3, g, 2, [[1], [3]])                                 # cut outside 0..n-2
    _expect(1, 3, [Gate("cx", (1, 1))], 0, [])                      # repeated qubit
    _expect(2, 3, g, 1, [[1]])                                      # crossing gate 3 not in a block
    _expect(2, 3, g, 1, [[1, 3]])                                   # non-convex: h(1) between
    _expect(2, 3, g, 1, [[1], [1, 3]])                              # gate in two blocks
    _expect(2, 3, g, 1, [[1], [3], [0]])                            # block without a crossing gate
    _expect(2, 3, g, 1, [[3], [1]])                                 # blocks out of dependency order
    big = [Gate("cx", (7, 0)), Gate("cx", (6, 1)), Gate("cx", (5, 2)), Gate("cx", (4, 3))]
    _expect(3, 8, big + [Gate("cx", (7, 3))], 3, [[0, 1, 2, 3, 4]])  # 4|4 block exceeds 3 per side
    _expect(1, 3, g, 1, [[1], [3]], precision="c64", tile_bits=2)   # tile too small
    bad = Gate("matrix", (0,), matrix=np.full((2, 2), np.nan))
    _expect(1, 2, [bad], 0, [])
