"""CPU oracle for GPU HyperBall over a visibility graph (test infrastructure).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library under
``paper_2604_08374_gb300/`` never imports it and shares no code with it.

The arithmetic lives in ``vga_oracle.c`` (plain C, fp64, built with
``-ffp-contract=off``); this module compiles it with gcc and marshals numpy
arrays through ctypes.  Each wrapper names the passage of the paper
("City-Scale Visibility Graph Analysis via GPU-Accelerated HyperBall") that the
C function follows.

Parity pins live in ``tests/test_oracle_*.py``; every function here has one
(the readings of the paper each function takes are listed in the header of
``vga_oracle.c``).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vga_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "libvga_oracle.so")
_lock = threading.Lock()
_lib = None

u8p = np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS")
u32p = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")
i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
u64p = np.ctypeslib.ndpointer(dtype=np.uint64, flags="C_CONTIGUOUS")
i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C11, no FMA contraction)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fPIC", "-shared",
                               "-pthread", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _nullable(ptype):
    """ndpointer that also accepts None."""
    class _P(ptype):
        @classmethod
        def from_param(cls, obj):
            if obj is None:
                return None
            return ptype.from_param(obj)
    return _P


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            L.orc_segment_meets_cell.argtypes = [C.c_int] * 6
            L.orc_segment_meets_cell.restype = C.c_int
            for name in ("orc_visible_bruteforce", "orc_visible_dda"):
                f = getattr(L, name)
                f.argtypes = [u8p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int]
                f.restype = C.c_int
            L.orc_main_component.argtypes = [u8p, C.c_int, C.c_int, i32p]
            L.orc_main_component.restype = C.c_int64
            L.orc_visible_from.argtypes = [u8p, C.c_int, C.c_int, i64p, C.c_int64, C.c_int64, _nullable(u32p)]
            L.orc_visible_from.restype = C.c_int64
            L.orc_visibility_lists.argtypes = [u8p, C.c_int, C.c_int, i64p, C.c_int64, _nullable(i64p), C.c_int64,
                                               _nullable(i64p), _nullable(u64p), _nullable(u32p), C.c_int]
            L.orc_visibility_lists.restype = None
            L.orc_leb128_put.argtypes = [C.c_uint64, _nullable(u8p)]
            L.orc_leb128_put.restype = C.c_int
            L.orc_csr_encode.argtypes = [C.c_int64, u64p, u32p, u64p, _nullable(u8p)]
            L.orc_csr_encode.restype = C.c_uint64
            L.orc_decode_list.argtypes = [u8p, C.c_uint64, C.c_uint64, C.c_int64, _nullable(u32p)]
            L.orc_decode_list.restype = C.c_int64
            L.orc_splitmix64.argtypes = [C.c_uint64]
            L.orc_splitmix64.restype = C.c_uint64
            L.orc_hll_hash.argtypes = [C.c_uint64, C.c_uint64, C.c_int, C.POINTER(C.c_uint32), C.POINTER(C.c_uint8)]
            L.orc_hll_hash.restype = None
            L.orc_hll_init.argtypes = [C.c_int64, C.c_int, C.c_uint64, u8p]
            L.orc_hll_init.restype = None
            L.orc_hll_alpha.argtypes = [C.c_int]
            L.orc_hll_alpha.restype = C.c_double
            L.orc_u128_to_double.argtypes = [C.c_uint64, C.c_uint64]
            L.orc_u128_to_double.restype = C.c_double
            L.orc_hll_estimate.argtypes = [u8p, C.c_int]
            L.orc_hll_estimate.restype = C.c_double
            L.orc_accumulate.argtypes = [C.c_double, C.c_int, C.c_double, C.c_double]
            L.orc_accumulate.restype = C.c_double
            L.orc_union_pass.argtypes = [C.c_int64, C.c_int, u64p, u8p, u8p, u8p, _nullable(i64p), C.c_int64,
                                         C.c_int, C.POINTER(C.c_uint64)]
            L.orc_union_pass.restype = C.c_int
            L.orc_hyperball.argtypes = [C.c_int64, u64p, u8p, _nullable(u32p), C.c_int, C.c_int, C.c_uint64,
                                        C.c_int, C.c_int, f64p, f64p, C.POINTER(C.c_int), _nullable(u8p),
                                        _nullable(f64p), C.c_int]
            L.orc_hyperball.restype = C.c_int
            L.orc_hyperball_bits.argtypes = [C.c_int64, u64p, u8p, _nullable(u32p), C.c_int, C.c_int, C.c_uint64,
                                             C.c_int, C.c_int, C.c_int, f64p, f64p, C.POINTER(C.c_int),
                                             _nullable(u8p), _nullable(f64p), C.c_int]
            L.orc_hyperball_bits.restype = C.c_int
            L.orc_hll_init_bits.argtypes = [C.c_int64, C.c_int, C.c_uint64, C.c_int, u8p]
            L.orc_hll_init_bits.restype = None
            L.orc_bfs.argtypes = [C.c_int64, u64p, u8p, C.c_int64, i32p]
            L.orc_bfs.restype = C.c_int
            L.orc_dvalue.argtypes = [C.c_double]
            L.orc_dvalue.restype = C.c_double
            L.orc_metrics.argtypes = [C.c_int64, f64p, _nullable(u32p), u32p, f64p]
            L.orc_metrics.restype = None
            L.orc_hilbert_index.argtypes = [C.c_int, C.c_uint32, C.c_uint32]
            L.orc_hilbert_index.restype = C.c_uint64
            _lib = L
    return _lib


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


# --------------------------------------------------------------------------
# Visibility and graph construction (Sec. 3.1, Sec. 3.2)
# --------------------------------------------------------------------------

def segment_meets_cell(x1, y1, x2, y2, i, j) -> bool:
    """Closed segment between cell centres vs the closed square of cell (i, j)."""
    return bool(lib().orc_segment_meets_cell(x1, y1, x2, y2, i, j))


def visible_bruteforce(obst: np.ndarray, a, b) -> bool:
    H, W = obst.shape
    return bool(lib().orc_visible_bruteforce(np.ascontiguousarray(obst, np.uint8), W, H, a[0], a[1], b[0], b[1]))


def visible_dda(obst: np.ndarray, a, b) -> bool:
    H, W = obst.shape
    return bool(lib().orc_visible_dda(np.ascontiguousarray(obst, np.uint8), W, H, a[0], a[1], b[0], b[1]))


def main_component(obst: np.ndarray):
    """Largest 4-connected free component, numbered in raster order.

    Returns (node_of_cell[H*W] int32 with -1 off the component, cell_of_node[N] int64)."""
    obst = np.ascontiguousarray(obst, np.uint8)
    H, W = obst.shape
    node_of_cell = np.empty(H * W, np.int32)
    n = lib().orc_main_component(obst, W, H, node_of_cell)
    cell_of_node = np.flatnonzero(node_of_cell >= 0).astype(np.int64)
    assert len(cell_of_node) == n
    return node_of_cell, cell_of_node


def visible_from(obst: np.ndarray, cell_of_node: np.ndarray, u: int) -> np.ndarray:
    """Sorted neighbour ids of node u (supercover rule)."""
    obst = np.ascontiguousarray(obst, np.uint8)
    H, W = obst.shape
    n = len(cell_of_node)
    cnt = lib().orc_visible_from(obst, W, H, cell_of_node, n, u, None)
    out = np.empty(max(cnt, 1), np.uint32)
    lib().orc_visible_from(obst, W, H, cell_of_node, n, u, out)
    return out[:cnt]


def visibility_csr(obst: np.ndarray, cell_of_node: np.ndarray, nodes=None, nthreads=None):
    """Plain CSR (row_ptr u64, col u32) of the visibility lists of `nodes` (all nodes by default)."""
    obst = np.ascontiguousarray(obst, np.uint8)
    H, W = obst.shape
    n = len(cell_of_node)
    nthreads = nthreads or default_threads()
    sel = None if nodes is None else np.ascontiguousarray(nodes, np.int64)
    k = n if sel is None else len(sel)
    counts = np.zeros(max(k, 1), np.int64)
    lib().orc_visibility_lists(obst, W, H, cell_of_node, n, sel, k, counts, None, None, nthreads)
    row_ptr = np.zeros(k + 1, np.uint64)
    row_ptr[1:] = np.cumsum(counts[:k])
    col = np.empty(max(int(row_ptr[-1]), 1), np.uint32)
    lib().orc_visibility_lists(obst, W, H, cell_of_node, n, sel, k, None, row_ptr, col, nthreads)
    return row_ptr, col[: int(row_ptr[-1])]


def leb128(value: int) -> bytes:
    buf = np.zeros(10, np.uint8)
    k = lib().orc_leb128_put(value, buf)
    return bytes(buf[:k])


def csr_encode(row_ptr: np.ndarray, col: np.ndarray):
    """Delta + LEB128 encoding (Sec. 3.2).  Returns (offsets u64[n+1], bytes u8)."""
    row_ptr = np.ascontiguousarray(row_ptr, np.uint64)
    col = np.ascontiguousarray(col, np.uint32)
    if len(col) == 0:
        col = np.zeros(1, np.uint32)
    n = len(row_ptr) - 1
    offsets = np.zeros(n + 1, np.uint64)
    nb = lib().orc_csr_encode(n, row_ptr, col, offsets, None)
    out = np.zeros(max(nb, 1), np.uint8)
    lib().orc_csr_encode(n, row_ptr, col, offsets, out)
    return offsets, out[:nb]


def decode_list(bytes_: np.ndarray, begin: int, end: int, n: int):
    """NeighborIter of Sec. 3.2; returns the ids or None when malformed."""
    bytes_ = np.ascontiguousarray(bytes_, np.uint8)
    if len(bytes_) == 0:
        bytes_ = np.zeros(1, np.uint8)
    cnt = lib().orc_decode_list(bytes_, begin, end, n, None)
    if cnt < 0:
        return None
    out = np.empty(max(cnt, 1), np.uint32)
    lib().orc_decode_list(bytes_, begin, end, n, out)
    return out[:cnt]


def decode_csr(offsets: np.ndarray, bytes_: np.ndarray):
    n = len(offsets) - 1
    rows = [decode_list(bytes_, int(offsets[v]), int(offsets[v + 1]), n) for v in range(n)]
    row_ptr = np.zeros(n + 1, np.uint64)
    row_ptr[1:] = np.cumsum([len(r) for r in rows])
    col = np.concatenate(rows).astype(np.uint32) if n else np.zeros(0, np.uint32)
    return row_ptr, col


def hilbert_index(k: int, x: int, y: int) -> int:
    """Position of cell (x, y) along the Hilbert curve of a 2^k x 2^k square."""
    return int(lib().orc_hilbert_index(k, x, y))


def hilbert_order(obst: np.ndarray, cell_of_node: np.ndarray) -> np.ndarray:
    """The main component's cells renumbered along the Hilbert curve of the
    smallest 2^k square covering the grid (Sec. 3.2 "Optional Hilbert
    reordering"): returns cell_of_node sorted by Hilbert index."""
    H, W = obst.shape
    k = max(1, int(np.ceil(np.log2(max(W, H)))))
    keys = np.array([hilbert_index(k, int(c % W), int(c // W)) for c in cell_of_node], np.uint64)
    return cell_of_node[np.argsort(keys, kind="stable")]


def build_graph(obst: np.ndarray, nthreads=None, order: str = "raster"):
    """Obstacle grid -> (offsets, bytes, cell_of_node) of the main component,
    nodes numbered in raster order or along the Hilbert curve."""
    _, cell_of_node = main_component(obst)
    if order == "hilbert":
        cell_of_node = hilbert_order(obst, cell_of_node)
    row_ptr, col = visibility_csr(obst, cell_of_node, nthreads=nthreads)
    offsets, bytes_ = csr_encode(row_ptr, col)
    return offsets, bytes_, cell_of_node


# --------------------------------------------------------------------------
# HyperLogLog and HyperBall (Sec. 2.3, Sec. 3.3, Alg. 1)
# --------------------------------------------------------------------------

def splitmix64(x: int) -> int:
    return int(lib().orc_splitmix64(x))


def hll_hash(v: int, seed: int, p: int):
    j = C.c_uint32()
    rho = C.c_uint8()
    lib().orc_hll_hash(v, seed, p, C.byref(j), C.byref(rho))
    return int(j.value), int(rho.value)


def hll_init(n: int, p: int, seed: int, reg_bits: int = 8) -> np.ndarray:
    regs = np.zeros(max(n, 1) << p, np.uint8)
    lib().orc_hll_init_bits(n, p, seed, reg_bits, regs)
    return regs[: n << p].reshape(n, 1 << p)


def hll_alpha(p: int) -> float:
    return float(lib().orc_hll_alpha(p))


def u128_to_double(x: int) -> float:
    return float(lib().orc_u128_to_double((x >> 64) & ((1 << 64) - 1), x & ((1 << 64) - 1)))


def hll_estimate(reg: np.ndarray, p: int) -> float:
    return float(lib().orc_hll_estimate(np.ascontiguousarray(reg, np.uint8), p))


def accumulate(sum_d: float, t: int, c_t: float, c_prev: float) -> float:
    return float(lib().orc_accumulate(sum_d, t, c_t, c_prev))


def union_pass(offsets, bytes_, cur: np.ndarray, p: int, nodes=None, nthreads=None):
    """Eq. hll-union over all nodes (or the listed ones).  Returns (next, changed, edges)."""
    offsets = np.ascontiguousarray(offsets, np.uint64)
    bytes_ = np.ascontiguousarray(bytes_, np.uint8)
    if len(bytes_) == 0:
        bytes_ = np.zeros(1, np.uint8)
    n = len(offsets) - 1
    cur = np.ascontiguousarray(cur, np.uint8).reshape(-1)
    sel = None if nodes is None else np.ascontiguousarray(nodes, np.int64)
    k = n if sel is None else len(sel)
    nxt = np.zeros(max(k, 1) << p, np.uint8)
    edges = C.c_uint64()
    rc = lib().orc_union_pass(n, p, offsets, bytes_, cur, nxt, sel, k, nthreads or default_threads(),
                              C.byref(edges))
    if rc < 0:
        raise ValueError("malformed CSR")
    return nxt[: k << p].reshape(k, 1 << p), bool(rc), int(edges.value)


def hyperball(offsets, bytes_, p: int, d: int, seed: int = 0, conv_mode: int = 0, comp_size=None,
              nthreads=None, trace: int = -1, reg_bits: int = 8):
    """Algorithm 1.  Returns dict(mean_depth, ball, iterations[, regs, c]).
    reg_bits=4: the paper's 4-bit registers (rho clamped to 15).

    trace >= 0 also returns the registers (trace+1, N, m) and estimates
    (trace+1, N) after each pass, index 0 being the initial counters."""
    offsets = np.ascontiguousarray(offsets, np.uint64)
    bytes_ = np.ascontiguousarray(bytes_, np.uint8)
    if len(bytes_) == 0:
        bytes_ = np.zeros(1, np.uint8)
    n = len(offsets) - 1
    m = 1 << p
    md = np.zeros(max(n, 1), np.float64)
    ball = np.zeros(max(n, 1), np.float64)
    it = C.c_int()
    regs = c = None
    if trace >= 0:
        regs = np.zeros(max((trace + 1) * n * m, 1), np.uint8)
        c = np.zeros(max((trace + 1) * n, 1), np.float64)
    cs = None if comp_size is None else np.ascontiguousarray(comp_size, np.uint32)
    rc = lib().orc_hyperball_bits(n, offsets, bytes_, cs, p, d, seed, conv_mode, reg_bits,
                                  nthreads or default_threads(), md, ball, C.byref(it), regs, c, trace)
    if rc != 0:
        raise ValueError("malformed CSR")
    out = {"mean_depth": md[:n], "ball": ball[:n], "iterations": int(it.value)}
    if trace >= 0:
        out["regs"] = regs[: (trace + 1) * n * m].reshape(trace + 1, n, m)
        out["c"] = c[: (trace + 1) * n].reshape(trace + 1, n)
    return out


def bfs(offsets, bytes_, src: int):
    """Exact hop distances from src (-1 = unreachable) and the eccentricity."""
    offsets = np.ascontiguousarray(offsets, np.uint64)
    bytes_ = np.ascontiguousarray(bytes_, np.uint8)
    if len(bytes_) == 0:
        bytes_ = np.zeros(1, np.uint8)
    n = len(offsets) - 1
    dist = np.empty(max(n, 1), np.int32)
    ecc = lib().orc_bfs(n, offsets, bytes_, src, dist)
    if ecc < 0:
        raise ValueError("malformed CSR")
    return dist[:n], int(ecc)


# --------------------------------------------------------------------------
# Closed-form metrics (Sec. 3.3 "Metric derivation")
# --------------------------------------------------------------------------

def dvalue(k: float) -> float:
    """RA of the root of a diamond-shaped graph with k nodes (RRA normaliser)."""
    return float(lib().orc_dvalue(k))


def metrics(mean_depth, degree, comp_size=None):
    """(N, 4) array of Integration [HH], Integration [Tekl], P-value, Point First Moment."""
    md = np.ascontiguousarray(mean_depth, np.float64)
    n = len(md)
    deg = np.ascontiguousarray(degree, np.uint32)
    cs = None if comp_size is None else np.ascontiguousarray(comp_size, np.uint32)
    out = np.zeros(max(4 * n, 1), np.float64)
    lib().orc_metrics(n, md if n else np.zeros(1), cs, deg if n else np.zeros(1, np.uint32), out)
    return out[: 4 * n].reshape(n, 4)
