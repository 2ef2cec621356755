"""CPU checks of the C ABI: the library builds for sm_103a, loads without a
GPU, exports every entry point include/vga_hyperball.h declares, and the
Python binding declares a signature for each.  The host-only LEB128 encoder is
compared byte for byte with the oracle's encoder.  No device work here."""
import os
import re
import subprocess

import numpy as np
import pytest

import oracle
import workloads
from paper_2604_08374_gb300 import build as vga_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "vga_hyperball.h")


def header_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*([a-z_][a-z0-9_]*)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def built_lib():
    path = vga_build.build()
    import paper_2604_08374_gb300 as vga
    return vga, path


def test_header_declares_the_boundary():
    names = header_functions()
    for required in ("vga_graph_load", "vga_graph_free", "vga_graph_load_file", "hyperball_run", "hyperball_run_dev",
                     "hyperball_run_trace", "vga_last_error", "vga_csr_encode", "vga_visibility_build"):
        assert required in names


def test_library_exports_every_declared_symbol(built_lib):
    vga, path = built_lib
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    for name in header_functions():
        assert name in exported, name
    L = vga.lib()
    for name in header_functions():
        assert hasattr(L, name)
        assert name in vga.SIGNATURES, f"binding lacks a signature for {name}"


def test_version_and_error_string(built_lib):
    vga, _ = built_lib
    assert "sm_103a" in vga.version()
    assert vga.lib().vga_last_error() is not None


@pytest.mark.parametrize("seed", [1, 2])
def test_encoder_matches_oracle(built_lib, seed):
    vga, _ = built_lib
    obst = workloads.tiny(seed)
    _, cells = oracle.main_component(obst)
    row_ptr, col = oracle.visibility_csr(obst, cells)
    ref_off, ref_bytes = oracle.csr_encode(row_ptr, col)
    off, b = vga.vga_csr_encode(row_ptr, col)
    assert np.array_equal(off, ref_off)
    assert bytes(b) == bytes(ref_bytes)


@pytest.mark.parametrize("case", ["tiny3", "maze", "ties", "all_obstacles", "one_cell"])
def test_main_component_count_matches_oracle(built_lib, case):
    # the builder's host step (largest 4-connected free component, ties to the
    # lowest raster index) against the oracle's, with no device work
    vga, _ = built_lib
    if case == "tiny3":
        obst = workloads.tiny(3)
    elif case == "maze":
        obst = (np.random.default_rng(5).random((23, 31)) < 0.45).astype(np.uint8)
    elif case == "ties":  # two equal free halves split by a wall
        obst = np.zeros((6, 9), np.uint8)
        obst[:, 4] = 1
    elif case == "all_obstacles":
        obst = np.ones((4, 5), np.uint8)
    else:
        obst = np.zeros((1, 1), np.uint8)
    _, cells = oracle.main_component(obst)
    assert vga.vga_visibility_count(obst) == len(cells)


def test_encoder_rejects_unsorted_lists(built_lib):
    vga, _ = built_lib
    with pytest.raises(vga.VgaError) as e:
        vga.vga_csr_encode(np.array([0, 3], np.uint64), np.array([1, 5, 5], np.uint32))
    assert e.value.status == vga.VGA_EINVAL


def test_encoder_wide_ids(built_lib):
    vga, _ = built_lib
    col = np.array([0, 127, 128, 16383, 16384, 2**21, 2**28, 2**32 - 1], np.uint32)
    row_ptr = np.array([0, len(col)], np.uint64)
    off, b = vga.vga_csr_encode(row_ptr, col)
    ref_off, ref_b = oracle.csr_encode(row_ptr, col)
    assert bytes(b) == bytes(ref_b)
    assert oracle.decode_list(b, 0, len(b), 2**32).tolist() == col.tolist()


STRUCTS = [("vga_tuning", "VgaTuning"), ("vga_job", "VgaJob"), ("vga_server_config", "VgaServerConfig"),
           ("vga_server_stats_t", "VgaServerStats"), ("vga_profile", "VgaProfile"), ("vga_tune_entry", "VgaTuneEntry")]


def test_ctypes_structs_match_the_header(built_lib, tmp_path):
    # the binding's ctypes mirrors must have the C structs' size and field
    # offsets (a C program compiled against the header prints them)
    vga, _ = built_lib
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "vga_hyperball.h"', "int main(void) {"]
    for cname, pyname in STRUCTS:
        cls = getattr(vga, pyname)
        lines.append(f'    printf("{pyname} sizeof %zu\\n", sizeof({cname}));')
        for field, _ in cls._fields_:
            lines.append(f'    printf("{pyname} {field} %zu\\n", offsetof({cname}, {field}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    seen = 0
    for line in out:
        if not line:
            continue
        pyname, field, value = line.split()
        cls = getattr(vga, pyname)
        got = __import__("ctypes").sizeof(cls) if field == "sizeof" else getattr(cls, field).offset
        assert got == int(value), (pyname, field)
        seen += 1
    assert seen == sum(len(getattr(vga, p)._fields_) + 1 for _, p in STRUCTS)
