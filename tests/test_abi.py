"""The C ABI library loads and exports every declared symbol (no GPU needed),
and host-side argument validation rejects bad input before touching a device."""
import ctypes
import os
import re

import numpy as np
import pytest

from conftest import ROOT


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "sssp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\*?\s+\*?(sssp_\w+)\s*\(", src, flags=re.M)))


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("sssp_graph_create", "sssp_graph_destroy", "sssp_solve", "sssp_last_status"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2105_06145_gb300 import sssp
    lib = ctypes.CDLL(sssp.LIB_PATH)
    for name in _declared_functions():
        assert hasattr(lib, name), name
    assert set(_declared_functions()) <= set(sssp.EXPORTED) | {"sssp_solve_host_ptr"}


def test_host_validation_without_gpu():
    from paper_2105_06145_gb300 import sssp
    off = np.array([0, 1, 2], dtype=np.uint64)
    tgt = np.array([1, 5], dtype=np.uint32)  # 5 >= n
    w = np.array([1, 1], dtype=np.uint32)
    with pytest.raises(sssp.SSSPError) as e:
        sssp.sssp_graph_create(2, 2, off, tgt, w)
    assert e.value.code == sssp.SSSP_ERR_INVALID_ARG
    bad_off = np.array([0, 2, 1], dtype=np.uint64)  # not monotone
    with pytest.raises(sssp.SSSPError):
        sssp.sssp_graph_create(2, 1, bad_off, tgt[:1], w[:1])
    with pytest.raises(sssp.SSSPError):
        sssp.sssp_graph_create(0, 0, np.zeros(1, np.uint64), tgt, w)
    assert sssp._lib.sssp_solve(None, 0, 0, 1, None, None) == sssp.SSSP_ERR_INVALID_ARG
    assert sssp._lib.sssp_rho_threshold(None, 4, None, 8, 1, 0, 1, 0, 2, 0, None, None) == \
        sssp.SSSP_ERR_INVALID_ARG
    assert sssp.sssp_status_string(sssp.SSSP_ERR_TIMEOUT) == "device-wide wait timed out"


def test_symmetry_verification_without_gpu():
    """SSSP_GRAPH_VERIFY rejects a graph that is not symmetric before any device
    work (an asymmetric edge or a reverse edge with another weight)."""
    from paper_2105_06145_gb300 import sssp
    off = np.array([0, 1, 2, 2], dtype=np.uint64)
    tgt = np.array([1, 2], dtype=np.uint32)            # 0->1, 1->2: no reverses
    w = np.array([5, 6], dtype=np.uint32)
    with pytest.raises(sssp.SSSPError) as e:
        sssp.sssp_graph_create_ex(3, 2, off, tgt, w, sssp.SSSP_GRAPH_SYMMETRIC | sssp.SSSP_GRAPH_VERIFY)
    assert e.value.code == sssp.SSSP_ERR_INVALID_ARG
    off = np.array([0, 1, 2], dtype=np.uint64)
    tgt = np.array([1, 0], dtype=np.uint32)
    w = np.array([5, 6], dtype=np.uint32)              # weights differ
    with pytest.raises(sssp.SSSPError):
        sssp.sssp_graph_create_ex(2, 2, off, tgt, w, sssp.SSSP_GRAPH_SYMMETRIC | sssp.SSSP_GRAPH_VERIFY)
    with pytest.raises(sssp.SSSPError):
        sssp.sssp_graph_create_ex(2, 2, off, tgt, w, 1 << 7)  # unknown flag


def _header_constants():
    src = open(os.path.join(ROOT, "include", "sssp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    consts = {k: int(v.rstrip("uU"), 0) for k, v in re.findall(r"#define\s+(SSSP_\w+)\s+(-?\w+)", src)
              if re.fullmatch(r"-?(0x[0-9a-fA-F]+|\d+)[uU]?", v)}
    for body in re.findall(r"typedef\s+enum\s*\{(.*?)\}", src, flags=re.S):
        for k, v in re.findall(r"(SSSP_\w+)\s*=\s*(-?\d+)", body):
            consts[k] = int(v)
    return consts


def test_binding_constants_match_the_header():
    """Every numeric constant the header defines (algorithms, statuses, flags,
    shapes, limits) has the same value in the Python binding."""
    from paper_2105_06145_gb300 import sssp
    consts = _header_constants()
    assert {"SSSP_RHO", "SSSP_DELTA_STAR", "SSSP_BELLMAN_FORD", "SSSP_ERR_TIMEOUT",
            "SSSP_SOLVE_BIDIRECTIONAL", "SSSP_GRAPH_REORDER"} <= set(consts)
    missing = [k for k in consts if not hasattr(sssp, k)]
    assert not missing, missing
    for k, v in consts.items():
        assert getattr(sssp, k) == v, (k, getattr(sssp, k), v)


def test_binding_struct_layouts_match_the_header(tmp_path):
    """Sizes and field offsets of every struct the binding passes across the
    boundary, as gcc lays them out from the header, equal the ctypes ones."""
    import shutil
    import subprocess
    from paper_2105_06145_gb300 import sssp
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = [sssp.sssp_step_trace, sssp.sssp_stats, sssp.sssp_options, sssp.sssp_server_config,
               sssp.sssp_query_info, sssp.sssp_tuning]
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "sssp.h"', "int main(void) {"]
    for st in structs:
        n = st.__name__
        lines.append(f'printf("{n} sizeof %zu\\n", sizeof({n}));')
        for f, _ in st._fields_:
            lines.append(f'printf("{n} {f} %zu\\n", offsetof({n}, {f}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.check_call([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = {}
    for ln in subprocess.check_output([str(exe)], text=True).split("\n"):
        if ln:
            s, f, v = ln.split()
            got[(s, f)] = int(v)
    for st in structs:
        n = st.__name__
        assert got[(n, "sizeof")] == ctypes.sizeof(st), n
        for f, _ in st._fields_:
            assert got[(n, f)] == getattr(st, f).offset, (n, f)
    dt = np.dtype(sssp.TRACE_DTYPE)
    assert dt.itemsize == got[("sssp_step_trace", "sizeof")]
    for f in dt.names:
        assert dt.fields[f][1] == got[("sssp_step_trace", f)], f


def test_binding_arity_matches_the_header():
    """Every function the binding types has as many parameters as the header
    declares (a drifted prototype would pass garbage through ctypes)."""
    from paper_2105_06145_gb300 import sssp
    src = open(os.path.join(ROOT, "include", "sssp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    protos = dict(re.findall(r"\b(sssp_\w+)\s*\(([^;{]*?)\)\s*;", src, flags=re.S))
    checked = 0
    for name, params in protos.items():
        fn = getattr(sssp._lib, name, None)
        if fn is None or fn.argtypes is None:
            continue
        p = params.strip()
        n = 0 if p in ("", "void") else p.count(",") + 1
        assert len(fn.argtypes) == n, (name, len(fn.argtypes), n)
        checked += 1
    assert checked >= 30, checked
