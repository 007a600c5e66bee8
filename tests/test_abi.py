"""The C-ABI library builds for sm_103a, loads, and exports every symbol that
include/lsm.h declares.  No compute call is made here (no GPU needed)."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_1909_13356_gb300 as lsm
from paper_1909_13356_gb300 import build as lsm_build

HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "lsm.h")


def declared_symbols():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[\w\s\*]+?\b(lsm_\w+)\s*\(", src, flags=re.M)))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for s in ("lsm_create", "lsm_mesh_upload", "lsm_eval_phi_grad", "lsm_solve_charts"):
        assert s in syms
    assert set(syms) == set(lsm.EXPORTS)


def test_library_builds_and_exports_every_symbol():
    path = lsm_build.build()
    L = ctypes.CDLL(path)
    for s in declared_symbols():
        assert hasattr(L, s), s


def test_library_is_built_for_sm_103a():
    assert "arch=compute_103a,code=sm_103a" in " ".join(lsm_build.ARCH)


def test_oracle_and_library_share_no_code():
    """The oracle and the CUDA path are independent: neither includes or
    imports the other."""
    root = os.path.dirname(os.path.dirname(__file__))
    bad = re.compile(r"(import\s+oracle|from\s+oracle|#include\s+[\"<].*oracle)")
    for dirpath, _, files in os.walk(os.path.join(root, "paper_1909_13356_gb300")):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                assert not bad.search(open(os.path.join(dirpath, f)).read()), f
    for f in ("oracle.c", "__init__.py"):
        txt = open(os.path.join(root, "oracle", f)).read()
        assert "lsm.h" not in txt and "paper_1909_13356_gb300" not in txt


def test_create_without_device_fails_cleanly():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(lsm.LsmError):
        lsm.Context(0)


def test_binding_declares_argument_types_for_every_export():
    """Every entry point has ctypes argument types, so doubles and 64-bit
    integers cross the boundary with the header's types."""
    L = lsm.load()
    for s in lsm.EXPORTS:
        assert getattr(L, s).argtypes is not None, s


def test_options_struct_matches_header_layout():
    """The binding's lsm_options has the header's fields, in the header's
    order and with the header's types (read from include/lsm.h)."""
    with open(HEADER) as f:
        text = f.read()
    end = text.index("} lsm_options;")
    body = text[text.rindex("typedef struct {", 0, end):end]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = re.findall(r"\b(double|float|int32_t)\s+(\w+)\s*;", body)
    ctypes_of = {"double": ctypes.c_double, "float": ctypes.c_float, "int32_t": ctypes.c_int32}
    assert [(n, ctypes_of[t]) for t, n in fields] == list(lsm._Options._fields_)
    size = sum(ctypes.sizeof(ctypes_of[t]) for t, _ in fields)
    assert size % 8 == 0   # no tail padding: the same size under any packing
    assert ctypes.sizeof(lsm._Options) == size


def test_refined_nodes_match_the_oracle_rule(oracle_mod):
    """lsm_refined_nodes (host code of the library): per triangle the order's
    Duffy rule composited over 4^level midpoint children, against the
    oracle's composite rule."""
    levels = np.array([0, 2, 1, 0, 3], dtype=np.int32)
    tri, uvw = lsm.refined_nodes(8, levels)
    otri, ouv, ow = oracle_mod.refined_nodes(len(levels), 6, levels)
    assert np.array_equal(tri, otri)
    assert np.allclose(uvw[:, :2], ouv, rtol=0, atol=1e-15)
    assert np.allclose(uvw[:, 2], ow, rtol=1e-13, atol=0)
    with pytest.raises(lsm.LsmError):
        lsm.refined_nodes(8, np.array([5]))


def test_out_of_range_options_are_rejected_before_any_device_call():
    """lsm_create checks its options first: an out-of-range treecode option
    returns LSM_E_INVALID_ARG (-1), with or without a GPU."""
    L = lsm.load()
    for field, value in (("tree_grid", 3), ("tree_grid", -1), ("tree_degree", 13), ("tree_theta", 1.0),
                         ("tree_ff_degree", 17), ("tree_min_sources", -2), ("ff_block", 96),
                         ("mixed_block", 32), ("newton_tree_degree", 13), ("newton_tree_degree", -2),
                         ("newton_tree_theta", 1.0), ("newton_cutoff", -1.0), ("newton_cutoff", 17.0)):
        opt = lsm._Options()
        setattr(opt, field, value)
        h = ctypes.c_void_p()
        assert L.lsm_create(ctypes.byref(h), 0, ctypes.byref(opt)) == -1, field
