"""GB300 HyperBall for visibility graph analysis -- Python binding.

Thin ctypes marshalling over the C ABI declared in ``include/vga_hyperball.h``
(same names).  Every step of the computation runs in the CUDA library
``libvga_hyperball.so`` built from ``csrc/`` for sm_103a; this module only
converts numpy arrays and torch tensors to pointers.  There is no CPU
fallback: if the library is missing, importing the binding's functions raises.

Paper: "City-Scale Visibility Graph Analysis via GPU-Accelerated HyperBall"
(arXiv 2604.08374): delta-compressed LEB128 CSR (Sec. 3.2), HyperBall
(Sec. 3.3, Algorithm 1), GPU pipeline (Sec. 3.4).
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libvga_hyperball.so")

VGA_OK, VGA_EINVAL, VGA_ENOMEM, VGA_ECORRUPT, VGA_ECUDA, VGA_ETIMEOUT, VGA_EBUSY, VGA_EIO = 0, -1, -2, -3, -4, -5, -6, -7
STATUS_NAMES = {0: "VGA_OK", -1: "VGA_EINVAL", -2: "VGA_ENOMEM", -3: "VGA_ECORRUPT", -4: "VGA_ECUDA",
                -5: "VGA_ETIMEOUT", -6: "VGA_EBUSY", -7: "VGA_EIO"}

# Every entry point the header declares, with its ctypes signature.
vp, i32, u32, u64, i64, f64 = C.c_void_p, C.c_int, C.c_uint32, C.c_uint64, C.c_int64, C.c_double


class VgaTuning(C.Structure):
    _fields_ = [("slice_bytes", C.c_int), ("warps_per_cta", C.c_int), ("l2_budget_mb", C.c_int),
                ("union_mode", C.c_int), ("register_bits", C.c_int), ("hub_lookups", C.c_int),
                ("table_levels", C.c_int), ("l2_window", C.c_int), ("first_pass", C.c_int),
                ("track_changes", C.c_int), ("group_nodes", C.c_int)]


class VgaJob(C.Structure):
    _fields_ = [("graph", C.c_void_p), ("p", C.c_int), ("d", C.c_int), ("seed", C.c_uint64), ("conv_mode", C.c_int),
                ("union_mode", C.c_int), ("mean_depth_dev", C.c_void_p), ("ball_size_dev", C.c_void_p),
                ("iterations", C.c_int), ("status", C.c_int)]


class VgaServerConfig(C.Structure):
    _fields_ = [("hbm_budget_bytes", C.c_uint64), ("max_batch", C.c_int), ("solo_nodes", C.c_int),
                ("lane_priority", C.c_int), ("batched_share", C.c_int), ("reserved", C.c_int * 2)]


class VgaServerStats(C.Structure):
    _fields_ = [("submitted", C.c_uint64), ("completed", C.c_uint64), ("queued", C.c_uint64),
                ("batched_passes", C.c_uint64), ("budget_used", C.c_uint64), ("budget_peak", C.c_uint64),
                ("batched_peak", C.c_uint64)]


class VgaProfile(C.Structure):
    _fields_ = [("kernel_launches", C.c_uint64), ("union_launches", C.c_uint64), ("union_ms", C.c_double),
                ("union_edges", C.c_uint64), ("union_gather_bytes", C.c_uint64), ("union_hbm_bytes", C.c_uint64),
                ("slice_bytes", C.c_int), ("union_mode", C.c_int), ("table_rows", C.c_int), ("reserved", C.c_int),
                ("first_pass_launches", C.c_uint64), ("first_pass_ms", C.c_double),
                ("first_pass_edges", C.c_uint64), ("tracked_launches", C.c_uint64), ("tracked_ms", C.c_double)]


class VgaTuneEntry(C.Structure):
    _fields_ = [("degree_log2", C.c_int), ("union_mode", C.c_int), ("slice_bytes", C.c_int),
                ("warps_per_cta", C.c_int), ("hub_lookups", C.c_int), ("p", C.c_int), ("geu_per_s", C.c_double),
                ("tuned_edges", C.c_uint64), ("group_nodes", C.c_int), ("reserved", C.c_int)]


TUNE_FIELDS = ("degree_log2", "union_mode", "slice_bytes", "warps_per_cta", "hub_lookups", "p", "geu_per_s",
               "tuned_edges", "group_nodes")


SIGNATURES = {
    "vga_last_error": ([], C.c_char_p),
    "vga_version": ([], C.c_char_p),
    "vga_csr_encode": ([u32, vp, vp, vp, vp, C.POINTER(u64)], i32),
    "vga_graph_load": ([u32, vp, vp, u64, vp, C.POINTER(vp)], i32),
    "vga_graph_load_device": ([u32, vp, vp, u64, vp, vp, C.POINTER(vp)], i32),
    "vga_graph_load_file": ([C.c_char_p, C.POINTER(vp)], i32),
    "vga_graph_save_file": ([vp, C.c_char_p], i32),
    "vga_graph_free": ([vp], None),
    "vga_graph_info": ([vp, C.POINTER(u32), C.POINTER(u64), C.POINTER(u64)], i32),
    "vga_graph_copy_csr": ([vp, vp, vp, vp], i32),
    "vga_graph_set_cells": ([vp, i32, i32, vp], i32),
    "vga_visibility_build": ([i32, i32, vp, vp, C.POINTER(vp)], i32),
    "vga_visibility_count": ([i32, i32, vp, C.POINTER(u32)], i32),
    "vga_visibility_build_ordered": ([i32, i32, vp, i32, vp, C.POINTER(vp)], i32),
    "hyperball_run": ([vp, i32, i32, u64, vp, vp, C.POINTER(i32)], i32),
    "hyperball_workspace_bytes": ([vp, i32, C.POINTER(u64)], i32),
    "hyperball_run_dev": ([vp, i32, i32, u64, i32, vp, vp, C.POINTER(i32), vp, u64, vp, C.POINTER(VgaTuning)], i32),
    "hyperball_run_trace": ([vp, i32, i32, u64, i32, vp, vp, C.POINTER(i32), vp, vp, i32, C.POINTER(VgaTuning)],
                            i32),
    "hyperball_run_noalloc": ([vp, i32, i32, u64, i32, vp, vp, C.POINTER(i32), vp], i32),
    "vga_metrics": ([vp, vp, vp, vp], i32),
    "hyperball_batch_workspace_bytes": ([C.POINTER(VgaJob), i32, C.POINTER(u64)], i32),
    "hyperball_run_batch": ([C.POINTER(VgaJob), i32, vp, u64, vp, i32], i32),
    "vga_server_create": ([C.POINTER(VgaServerConfig), C.POINTER(vp)], i32),
    "vga_server_submit": ([vp, vp, i32, i32, u64, i32, vp, vp, C.POINTER(u64)], i32),
    "vga_server_wait": ([vp, u64, f64, C.POINTER(i32), C.POINTER(f64), C.POINTER(f64)], i32),
    "vga_server_stats": ([vp, C.POINTER(VgaServerStats)], i32),
    "vga_server_destroy": ([vp], None),
    "vga_profile_enable": ([i32], i32),
    "vga_profile_reset": ([], i32),
    "vga_profile_read": ([C.POINTER(VgaProfile)], i32),
    "vga_bench_gather": ([u64, i32, u64, i32, vp, C.POINTER(f64)], i32),
    "vga_shard_create": ([vp, i32, u64, i32, i32, C.POINTER(VgaTuning), C.POINTER(vp)], i32),
    "vga_shard_info": ([vp, C.POINTER(i32), C.POINTER(i32), C.POINTER(i32), C.POINTER(u64)], i32),
    "vga_shard_start": ([vp, vp, vp], i32),
    "vga_shard_union": ([vp, vp, C.POINTER(u32), vp], i32),
    "vga_shard_estimate": ([vp, vp, C.POINTER(u32), vp], i32),
    "vga_shard_finalize": ([vp, vp, vp, vp], i32),
    "vga_shard_free": ([vp], None),
    "vga_set_table_scheme_nodes": ([u32], i32),
    "vga_set_visibility_sweep_limits": ([i32, u32], i32),
    "vga_autotune": ([C.POINTER(vp), i32, i32, vp, C.POINTER(VgaTuneEntry), i32, C.POINTER(i32), i32], i32),
    "vga_tune_table_set": ([C.POINTER(VgaTuneEntry), i32], i32),
    "vga_tune_table_get": ([C.POINTER(VgaTuneEntry), i32, C.POINTER(i32)], i32),
}

_lock = threading.Lock()
_lib = None


class VgaError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


def lib():
    """Load libvga_hyperball.so (build it first with build.build())."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(f"{LIB_PATH} is missing: run paper_2604_08374_gb300.build.build() "
                                  "(the library has no CPU fallback)")
            L = C.CDLL(LIB_PATH)
            for name, (args, res) in SIGNATURES.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = res
            _lib = L
    return _lib


def _check(status: int):
    if status != VGA_OK:
        raise VgaError(status, lib().vga_last_error().decode(errors="replace"))


def _ptr(a) -> int | None:
    """Data pointer of a numpy array or torch tensor (None passes NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data if a.size else None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr() or None
    raise TypeError(f"unsupported buffer type {type(a)}")


def _tuning(slice_bytes=0, warps_per_cta=0, l2_budget_mb=0, union_mode=0, register_bits=0, hub_lookups=0,
            table_levels=0, l2_window=0, first_pass=0, track_changes=0, group_nodes=0):
    if not (slice_bytes or warps_per_cta or l2_budget_mb or union_mode or register_bits or hub_lookups
            or table_levels or l2_window or first_pass or track_changes or group_nodes):
        return None
    t = VgaTuning()
    t.slice_bytes, t.warps_per_cta, t.l2_budget_mb, t.union_mode = slice_bytes, warps_per_cta, l2_budget_mb, union_mode
    t.register_bits, t.hub_lookups, t.table_levels = register_bits, hub_lookups, table_levels
    t.l2_window, t.first_pass, t.track_changes = l2_window, first_pass, track_changes
    t.group_nodes = group_nodes
    return C.pointer(t)


def version() -> str:
    return lib().vga_version().decode()


# --------------------------------------------------------------------------
# Compressed CSR (Sec. 3.2)
# --------------------------------------------------------------------------

def vga_csr_encode(row_ptr: np.ndarray, col: np.ndarray):
    """Delta + LEB128 encode sorted neighbour lists -> (offsets u64[n+1], bytes u8)."""
    row_ptr = np.ascontiguousarray(row_ptr, np.uint64)
    col = np.ascontiguousarray(col, np.uint32)
    n = len(row_ptr) - 1
    offsets = np.zeros(n + 1, np.uint64)
    nb = C.c_uint64()
    _check(lib().vga_csr_encode(n, _ptr(row_ptr), _ptr(col), _ptr(offsets), None, C.byref(nb)))
    out = np.zeros(max(nb.value, 1), np.uint8)
    _check(lib().vga_csr_encode(n, _ptr(row_ptr), _ptr(col), _ptr(offsets), _ptr(out), C.byref(nb)))
    return offsets, out[: nb.value]


class Graph:
    """A device-resident compressed visibility graph (owns a vga_graph*)."""

    def __init__(self, handle: int):
        self._h = C.c_void_p(handle)
        n, e, b = C.c_uint32(), C.c_uint64(), C.c_uint64()
        _check(lib().vga_graph_info(self._h, C.byref(n), C.byref(e), C.byref(b)))
        self.n_nodes, self.n_edges, self.n_bytes = n.value, e.value, b.value

    @property
    def handle(self):
        if self._h is None or not self._h.value:
            raise ValueError("graph has been freed")
        return self._h

    def free(self):
        if self._h is not None and self._h.value:
            lib().vga_graph_free(self._h)
        self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.free()

    def copy_csr(self):
        """(offsets, bytes, degrees) copied back to host memory."""
        offsets = np.zeros(self.n_nodes + 1, np.uint64)
        bytes_ = np.zeros(max(self.n_bytes, 1), np.uint8)
        deg = np.zeros(max(self.n_nodes, 1), np.uint32)
        _check(lib().vga_graph_copy_csr(self.handle, _ptr(offsets), _ptr(bytes_), _ptr(deg)))
        return offsets, bytes_[: self.n_bytes], deg[: self.n_nodes]

    def save(self, path: str):
        _check(lib().vga_graph_save_file(self.handle, path.encode()))

    def set_cells(self, W: int, H: int, cell_of_node):
        """Attach every node's grid cell (y * W + x on a W x H grid); the grouped
        union then groups 2 x 2 blocks of cells.  None detaches it."""
        if cell_of_node is None:
            _check(lib().vga_graph_set_cells(self.handle, 0, 0, None))
            return
        cells = np.ascontiguousarray(cell_of_node, np.uint64)
        if len(cells) != self.n_nodes:
            raise ValueError("need one cell per node")
        _check(lib().vga_graph_set_cells(self.handle, W, H, _ptr(cells) if self.n_nodes else None))


def vga_graph_load(offsets: np.ndarray, bytes_: np.ndarray, comp_size=None) -> Graph:
    """Copy a compressed CSR (host arrays) to the device; validated there."""
    offsets = np.ascontiguousarray(offsets, np.uint64)
    bytes_ = np.ascontiguousarray(bytes_, np.uint8)
    n = len(offsets) - 1
    cs = None if comp_size is None else np.ascontiguousarray(comp_size, np.uint32)
    h = C.c_void_p()
    _check(lib().vga_graph_load(n, _ptr(offsets), _ptr(bytes_), len(bytes_), _ptr(cs), C.byref(h)))
    return Graph(h.value)


def vga_graph_load_device(offsets_dev, bytes_dev, n_bytes: int, comp_size=None, stream=None) -> Graph:
    """Load from device buffers (torch tensors): offsets u64 (n+1), bytes u8."""
    n = offsets_dev.numel() - 1
    cs = None if comp_size is None else np.ascontiguousarray(comp_size, np.uint32)
    h = C.c_void_p()
    _check(lib().vga_graph_load_device(n, _ptr(offsets_dev), _ptr(bytes_dev), n_bytes, _ptr(cs),
                                       _stream_ptr(stream), C.byref(h)))
    return Graph(h.value)


def vga_graph_load_file(path: str) -> Graph:
    h = C.c_void_p()
    _check(lib().vga_graph_load_file(path.encode(), C.byref(h)))
    return Graph(h.value)


# --------------------------------------------------------------------------
# Visibility builder (Sec. 3.1)
# --------------------------------------------------------------------------

def vga_visibility_count(obst: np.ndarray) -> int:
    obst = np.ascontiguousarray(obst, np.uint8)
    H, W = obst.shape
    n = C.c_uint32()
    _check(lib().vga_visibility_count(W, H, _ptr(obst), C.byref(n)))
    return n.value


def vga_visibility_build(obst: np.ndarray, return_cells: bool = False, order: str = "raster"):
    """Build the supercover visibility graph of an obstacle grid on the GPU,
    nodes in raster or Hilbert order."""
    obst = np.ascontiguousarray(obst, np.uint8)
    H, W = obst.shape
    cells = np.zeros(max(H * W, 1), np.uint64)
    h = C.c_void_p()
    _check(lib().vga_visibility_build_ordered(W, H, _ptr(obst), {"raster": 0, "hilbert": 1}[order], _ptr(cells),
                                              C.byref(h)))
    g = Graph(h.value)
    if return_cells:
        return g, cells[: g.n_nodes]
    return g


# --------------------------------------------------------------------------
# HyperBall (Sec. 3.3, Algorithm 1)
# --------------------------------------------------------------------------

def _stream_ptr(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream or None
    return int(stream) or None


def hyperball_run(g: Graph, p: int = 10, d: int = 0, seed: int = 0):
    """Algorithm 1 with host outputs -> (mean_depth, ball_size, iterations)."""
    md = np.zeros(max(g.n_nodes, 1), np.float64)
    ball = np.zeros(max(g.n_nodes, 1), np.float64)
    it = C.c_int()
    _check(lib().hyperball_run(g.handle, p, d, seed, _ptr(md), _ptr(ball), C.byref(it)))
    return md[: g.n_nodes], ball[: g.n_nodes], it.value


def hyperball_workspace_bytes(g: Graph, p: int) -> int:
    """Workspace bytes of hyperball_run_dev with automatic tuning."""
    b = C.c_uint64()
    _check(lib().hyperball_workspace_bytes(g.handle, p, C.byref(b)))
    return b.value


def hyperball_run_dev(g: Graph, p: int, d: int, seed: int, mean_depth_dev, ball_size_dev, conv_mode: int = 0,
                      workspace=None, stream=None, slice_bytes: int = 0, warps_per_cta: int = 0,
                      l2_budget_mb: int = 0, union_mode: int = 0, register_bits: int = 0,
                      hub_lookups: int = 0, table_levels: int = 0, l2_window: int = 0,
                      first_pass: int = 0, track_changes: int = 0, group_nodes: int = 0) -> int:
    """Algorithm 1 into device tensors (float64, N each); returns passes run."""
    it = C.c_int()
    ws_bytes = 0 if workspace is None else workspace.numel() * workspace.element_size()
    _check(lib().hyperball_run_dev(g.handle, p, d, seed, conv_mode, _ptr(mean_depth_dev), _ptr(ball_size_dev),
                                   C.byref(it), _ptr(workspace), ws_bytes, _stream_ptr(stream),
                                   _tuning(slice_bytes, warps_per_cta, l2_budget_mb, union_mode, register_bits,
                                           hub_lookups, table_levels, l2_window, first_pass, track_changes,
                                           group_nodes)))
    return it.value


def hyperball_run_noalloc(g: Graph, p: int, d: int, seed: int, mean_depth_dev, ball_size_dev, conv_mode: int = 0,
                          stream=None) -> int:
    """Algorithm 1 into device tensors using the library's fixed 64 MiB scratch
    instead of any device allocation (for callers that cannot allocate).
    Returns passes run; raises VgaError(VGA_EINVAL) if the run needs more."""
    it = C.c_int()
    _check(lib().hyperball_run_noalloc(g.handle, p, d, seed, conv_mode, _ptr(mean_depth_dev), _ptr(ball_size_dev),
                                       C.byref(it), _stream_ptr(stream)))
    return it.value


def hyperball_run_trace(g: Graph, p: int, d: int, seed: int = 0, conv_mode: int = 0, max_trace: int = 8,
                        slice_bytes: int = 0, warps_per_cta: int = 0, union_mode: int = 0, register_bits: int = 0,
                        hub_lookups: int = 0, table_levels: int = 0, first_pass: int = 0,
                        track_changes: int = 0, group_nodes: int = 0):
    """Run with per-pass register and estimate dumps (bit-exact checks).

    Returns dict(mean_depth, ball, iterations, regs[(max_trace+1), N, m], c[(max_trace+1), N])."""
    n, m = g.n_nodes, 1 << p
    md = np.zeros(max(n, 1), np.float64)
    ball = np.zeros(max(n, 1), np.float64)
    regs = np.zeros(max((max_trace + 1) * n * m, 1), np.uint8)
    cc = np.zeros(max((max_trace + 1) * n, 1), np.float64)
    it = C.c_int()
    _check(lib().hyperball_run_trace(g.handle, p, d, seed, conv_mode, _ptr(md), _ptr(ball), C.byref(it),
                                     _ptr(regs), _ptr(cc), max_trace,
                                     _tuning(slice_bytes, warps_per_cta, union_mode=union_mode,
                                             register_bits=register_bits, hub_lookups=hub_lookups,
                                             table_levels=table_levels, first_pass=first_pass,
                                             track_changes=track_changes, group_nodes=group_nodes)))
    return {"mean_depth": md[:n], "ball": ball[:n], "iterations": it.value,
            "regs": regs[: (max_trace + 1) * n * m].reshape(max_trace + 1, n, m),
            "c": cc[: (max_trace + 1) * n].reshape(max_trace + 1, n)}


def _job_array(jobs):
    arr = (VgaJob * max(len(jobs), 1))()
    for k, j in enumerate(jobs):
        arr[k].graph = j["graph"].handle.value
        arr[k].p, arr[k].d, arr[k].seed = j["p"], j.get("d", 0), j.get("seed", 0)
        arr[k].conv_mode = j.get("conv_mode", 0)
        arr[k].union_mode = j.get("union_mode", 0)
        arr[k].mean_depth_dev = _ptr(j.get("mean_depth"))
        arr[k].ball_size_dev = _ptr(j.get("ball"))
    return arr


def hyperball_batch_workspace_bytes(jobs) -> int:
    arr = _job_array(jobs)
    b = C.c_uint64()
    _check(lib().hyperball_batch_workspace_bytes(arr, len(jobs), C.byref(b)))
    return b.value


def hyperball_run_batch(jobs, workspace=None, stream=None, use_graph: bool = True):
    """Run many analyses together.  jobs: dicts with graph, p, d, seed,
    conv_mode and device tensors mean_depth / ball (float64, N each, optional).
    Returns the passes run per job."""
    arr = _job_array(jobs)
    ws_bytes = 0 if workspace is None else workspace.numel() * workspace.element_size()
    _check(lib().hyperball_run_batch(arr, len(jobs), _ptr(workspace), ws_bytes, _stream_ptr(stream),
                                     1 if use_graph else 0))
    return [arr[k].iterations for k in range(len(jobs))]


class Server:
    """Request loop with continuous batching (vga_server_*).  Results arrive in
    host numpy arrays; keep graphs loaded until their requests are waited for."""

    def __init__(self, hbm_budget_bytes: int = 0, max_batch: int = 0, solo_nodes: int = 0, lane_priority: int = 0,
                 batched_share: int = 0):
        cfg = VgaServerConfig()
        cfg.hbm_budget_bytes, cfg.max_batch, cfg.solo_nodes = hbm_budget_bytes, max_batch, solo_nodes
        cfg.lane_priority, cfg.batched_share = lane_priority, batched_share
        h = C.c_void_p()
        _check(lib().vga_server_create(C.byref(cfg), C.byref(h)))
        self._h = h
        self._outputs = {}

    def submit(self, g: Graph, p: int, d: int, seed: int = 0, conv_mode: int = 0) -> int:
        md = np.empty(max(g.n_nodes, 1), np.float64)
        ball = np.empty(max(g.n_nodes, 1), np.float64)
        rid = C.c_uint64()
        _check(lib().vga_server_submit(self._h, g.handle, p, d, seed, conv_mode, _ptr(md), _ptr(ball),
                                       C.byref(rid)))
        self._outputs[rid.value] = (md, ball, g.n_nodes)
        return rid.value

    def wait(self, rid: int, timeout_s: float = 0.0):
        """-> dict(mean_depth, ball, iterations, latency_s, queued_s)."""
        it, lat, q = C.c_int(), C.c_double(), C.c_double()
        status = lib().vga_server_wait(self._h, rid, timeout_s, C.byref(it), C.byref(lat), C.byref(q))
        if status == VGA_ETIMEOUT:
            _check(status)
        md, ball, n = self._outputs.pop(rid)
        _check(status)
        return {"mean_depth": md[:n], "ball": ball[:n], "iterations": it.value, "latency_s": lat.value,
                "queued_s": q.value}

    def stats(self) -> dict:
        st = VgaServerStats()
        _check(lib().vga_server_stats(self._h, C.byref(st)))
        return {name: getattr(st, name) for name, _ in VgaServerStats._fields_}

    def close(self):
        if self._h is not None and self._h.value:
            lib().vga_server_destroy(self._h)
        self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def vga_metrics(g: Graph, mean_depth_dev, out_dev=None, stream=None):
    """Closed-form metrics (Sec. 3.3): (N, 4) device tensor of HH, Tekl, P-value, PFM."""
    if out_dev is None:
        import torch
        out_dev = torch.empty((g.n_nodes, 4), dtype=torch.float64, device=mean_depth_dev.device)
    _check(lib().vga_metrics(g.handle, _ptr(mean_depth_dev), _ptr(out_dev), _stream_ptr(stream)))
    return out_dev


# --------------------------------------------------------------------------
# Measurement
# --------------------------------------------------------------------------

def vga_profile_enable(on: bool = True):
    _check(lib().vga_profile_enable(1 if on else 0))


def vga_profile_reset():
    _check(lib().vga_profile_reset())


def vga_profile_read() -> dict:
    p = VgaProfile()
    _check(lib().vga_profile_read(C.byref(p)))
    return {name: getattr(p, name) for name, _ in VgaProfile._fields_ if name != "reserved"}


def vga_bench_gather(resident_bytes: int, chunk_bytes: int, gathers: int, consumer: int = 1, stream=None) -> float:
    """Gather bandwidth (GB/s) with the union kernel's access pattern.

    consumer=1 xors the loaded words (the L2 gather roofline when the buffer
    fits in L2); consumer=0 folds them with the union's bytewise max;
    consumer=2 streams the buffer with coalesced loads instead (the
    shape-independent L2 read ceiling)."""
    out = C.c_double()
    _check(lib().vga_bench_gather(resident_bytes, chunk_bytes, gathers, consumer, _stream_ptr(stream),
                                  C.byref(out)))
    return out.value


def _entries_out(arr, n):
    return [{f: getattr(arr[k], f) for f in TUNE_FIELDS} for k in range(n)]


def vga_autotune(graphs, p: int = 10, stream=None, install: bool = True):
    """Time the union's launch choices on `graphs` and return one entry (dict)
    per degree bucket; with install=True they also become the process-wide
    table consulted by every analysis that leaves its tuning fields at 0."""
    gs = list(graphs)
    handles = (C.c_void_p * max(len(gs), 1))(*[g.handle.value for g in gs])
    out = (VgaTuneEntry * 64)()
    n = C.c_int()
    _check(lib().vga_autotune(handles, len(gs), p, _stream_ptr(stream), out, 64, C.byref(n), int(install)))
    return _entries_out(out, n.value)


def vga_tune_table_set(entries):
    """Install tuning entries (dicts with TUNE_FIELDS keys); [] clears the table."""
    arr = (VgaTuneEntry * max(len(entries), 1))()
    for k, e in enumerate(entries):
        for f in TUNE_FIELDS:
            if f in e:
                setattr(arr[k], f, e[f])
    _check(lib().vga_tune_table_set(arr, len(entries)))


def vga_tune_table_get():
    """The installed tuning table as a list of dicts."""
    out = (VgaTuneEntry * 64)()
    n = C.c_int()
    _check(lib().vga_tune_table_get(out, 64, C.byref(n)))
    return _entries_out(out, min(n.value, 64))


class Shard:
    """Register-range shard of one analysis (vga_shard_*): slices
    [slice_first, slice_first + slice_count) of every node's counter."""

    def __init__(self, handle):
        self.handle = handle
        first, count, width, pb = C.c_int(), C.c_int(), C.c_int(), C.c_uint64()
        _check(lib().vga_shard_info(handle, C.byref(first), C.byref(count), C.byref(width), C.byref(pb)))
        self.slice_first, self.slice_count, self.slice_bytes = first.value, count.value, width.value
        self.partial_bytes = pb.value

    def start(self, partial, stream=None):
        _check(lib().vga_shard_start(self.handle, _ptr(partial), _stream_ptr(stream)))

    def union(self, partial, stream=None) -> int:
        changed = C.c_uint32()
        _check(lib().vga_shard_union(self.handle, _ptr(partial), C.byref(changed), _stream_ptr(stream)))
        return changed.value

    def estimate(self, all_partials, stream=None) -> int:
        inc = C.c_uint32()
        _check(lib().vga_shard_estimate(self.handle, _ptr(all_partials), C.byref(inc), _stream_ptr(stream)))
        return inc.value

    def finalize(self, mean_depth_dev, ball_size_dev, stream=None):
        _check(lib().vga_shard_finalize(self.handle, _ptr(mean_depth_dev), _ptr(ball_size_dev),
                                        _stream_ptr(stream)))

    def free(self):
        if self.handle:
            lib().vga_shard_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def vga_shard_create(g: Graph, p: int, seed: int, shard: int, n_shards: int, slice_bytes: int = 0,
                     warps_per_cta: int = 0, union_mode: int = 0, register_bits: int = 0,
                     hub_lookups: int = 0, table_levels: int = 0, first_pass: int = 0,
                     track_changes: int = 0, group_nodes: int = 0) -> Shard:
    h = C.c_void_p()
    _check(lib().vga_shard_create(g.handle, p, seed, shard, n_shards,
                                  _tuning(slice_bytes, warps_per_cta, 0, union_mode, register_bits, hub_lookups,
                                          table_levels, first_pass=first_pass, track_changes=track_changes,
                                          group_nodes=group_nodes),
                                  C.byref(h)))
    return Shard(h)


def vga_set_visibility_sweep_limits(smem_list_cap: int = 0, smem_bitmap_nodes: int = 0):
    """Builder test hook: cap the interval lists kept in shared memory
    (1..48, 0 = 48) and keep the node bitmap in global memory for graphs above
    `smem_bitmap_nodes` nodes (0 = only when shared memory is too small)."""
    _check(lib().vga_set_visibility_sweep_limits(smem_list_cap, smem_bitmap_nodes))


def vga_set_table_scheme_nodes(nodes: int = 0):
    """Graphs loaded from now on with at least `nodes` nodes get 3-row tables of
    range maxima (0: automatic, from the L2 size)."""
    _check(lib().vga_set_table_scheme_nodes(nodes))
