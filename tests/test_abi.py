"""CPU-side checks of the C ABI library: it builds, loads, exports every
symbol include/opmos.h declares, and fails loudly without a device."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

import paper_2411_16667_gb300 as pkg
from paper_2411_16667_gb300 import opmos

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    text = open(os.path.join(ROOT, "include", "opmos.h")).read()
    return sorted(set(re.findall(r"OPMOS_API\s+[\w\s\*]+?\b(opmos_\w+)\(", text)))


def _declared_test_symbols():
    text = open(os.path.join(ROOT, "include", "opmos_test.h")).read()
    return sorted(set(re.findall(r"OPMOS_API\s+[\w\s\*]+?\b(opmos_\w+)\(", text)))


def test_header_declares_the_binding_exports():
    assert _declared_symbols() == sorted(opmos.EXPORTS)
    assert _declared_test_symbols() == sorted(opmos.TEST_EXPORTS)


def test_library_exports_the_test_hooks():
    lib = ctypes.CDLL(pkg.build())
    for name in _declared_test_symbols():
        assert hasattr(lib, name), name


def test_library_builds_and_exports_every_symbol():
    path = pkg.build()
    lib = ctypes.CDLL(path)
    for name in _declared_symbols():
        assert hasattr(lib, name), name


def test_options_struct_matches_defaults():
    o = opmos.opmos_default_options()
    assert (o.window, o.lanes_per_label, o.tile, o.delta) == (1024, 8, 32, 1)
    assert o.mem_budget_bytes == 8 << 30
    assert ctypes.sizeof(opmos.Options) == 64 and o.alone_window == 0
    assert o.alone_labels == 1_000_000
    assert ctypes.sizeof(opmos.Stats) == 30 * 8


@pytest.mark.skipif(opmos.opmos_device_count() > 0, reason="only meaningful without a GPU")
def test_no_device_fails_loudly():
    import synth
    g, _ = synth.config1()
    with pytest.raises(opmos.OpmosError) as e:
        opmos.opmos_graph.from_synth(g)
    assert e.value.code == opmos.ERR_CUDA


def test_missing_library_fails_loudly(tmp_path):
    saved = opmos._lib
    try:
        opmos._lib = None
        with pytest.raises(opmos.OpmosError):
            opmos.lib(str(tmp_path / "missing.so"))
    finally:
        opmos._lib = saved


def _run_c_client(tmp_path):
    lib = pkg.build()
    exe = tmp_path / "client"
    subprocess.check_call(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                           os.path.join(ROOT, "tests", "c_abi_client.c"), lib,
                           f"-Wl,-rpath,{os.path.dirname(lib)}", "-o", str(exe)])
    p = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert p.returncode == 0, f"exit {p.returncode}: {p.stdout} {p.stderr}"
    return p.stdout


def test_plain_c_client_links_and_behaves(tmp_path):
    """A C program built against the header alone and linked to the library:
    defaults are filled in, and without a device compute calls fail with
    OPMOS_ERR_CUDA and a message (with one, it checks a two-path front)."""
    _run_c_client(tmp_path)


@pytest.mark.gpu
def test_plain_c_client_solves_on_the_device(tmp_path):
    """The same C program on a GPU: its device branch solves the two-path
    graph of Sec. 1 and checks the front {(4,5), (5,4)} and a path."""
    if opmos.opmos_device_count() == 0:
        pytest.fail("no CUDA device visible to the library")
    assert "front (4,5) (5,4)" in _run_c_client(tmp_path)


def test_paths_are_views_of_the_flat_arrays():
    """Result.paths over opmos_result_paths' layout: path i's nodes are
    nodes[offsets[i]:offsets[i+1]] and its arcs edges[offsets[i]-i:offsets[i+1]-i-1]."""
    offs = np.array([0, 3, 4, 7], np.uint32)
    nodes = np.array([10, 11, 12, 20, 30, 31, 32], np.uint32)
    edges = np.array([100, 101, 300, 301], np.uint64)
    p = opmos.Paths(offs, nodes, edges)
    assert len(p) == 3
    assert p[0][0].tolist() == [10, 11, 12] and p[0][1].tolist() == [100, 101]
    assert p[1][0].tolist() == [20] and p[1][1].size == 0
    assert p[-1][0].tolist() == [30, 31, 32] and p[-1][1].tolist() == [300, 301]
    assert [n.tolist() for n, _ in p[1:]] == [[20], [30, 31, 32]]
    assert [len(n) for n, _ in p] == [3, 1, 3]
    with pytest.raises(IndexError):
        p[3]
