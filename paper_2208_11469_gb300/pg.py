"""Python binding of libpg (include/pg.h): argument marshalling only.

Every function here passes torch device tensors to one C-ABI entry point of
the same name (without the `pg_` prefix) on the current torch CUDA stream.
All compute runs in the library's CUDA kernels. If the library has not been
built, or no CUDA device is present, the calls raise — there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import struct
import threading
from dataclasses import dataclass, field

import torch

from . import build as _build

# ----------------------------------------------------------------- constants
OK = 0
ERR = {0: "PG_OK", -1: "PG_ERR_INVALID_ARG", -2: "PG_ERR_INVALID_GRAPH", -3: "PG_ERR_TOO_LARGE",
       -4: "PG_ERR_NO_MEMORY", -5: "PG_ERR_CUDA", -6: "PG_ERR_TIMEOUT", -7: "PG_ERR_NOT_FOUND",
       -8: "PG_ERR_BUSY", -9: "PG_ERR_UNSUPPORTED", -10: "PG_ERR_CANCELLED"}
SK_BLOOM, SK_KHASH, SK_1HASH = 1, 2, 3
EST_EXACT, EST_BF_AND, EST_BF_L, EST_KH, EST_1H, EST_1H_LITERAL = 0, 1, 2, 3, 4, 5
EST_BF_OR, EST_BF_SS, EST_1H_KMV = 6, 7, 8
CSR_CODES = {0: "ok", 1: "bad_row_ptr", 2: "out_of_range", 3: "unsorted", 4: "self_loop", 5: "asymmetric"}

# Every symbol include/pg.h declares.
SYMBOLS = [
    "pg_status_string", "pg_last_error", "pg_version", "pg_validate_csr", "pg_edge_index_bytes",
    "pg_build_edge_index", "pg_edge_index_upper_off", "pg_sketch_stride",
    "pg_bloom_bits_for_budget", "pg_build_workspace_bytes", "pg_build_bloom", "pg_build_minhash",
    "pg_upload_build", "pg_sketch_save", "pg_sketch_load_header", "pg_sketch_load",
    "pg_hist_bins", "pg_workspace_bytes", "pg_triangle_count", "pg_clustering",
    "pg_jaccard_pairs", "pg_similarity_pairs", "pg_edge_counts", "pg_kernel_launches", "pg_analyze", "pg_triangle_count_noalloc",
    "pg_partial_sums", "pg_finalize_sums",
    "pg_jarvis_patrick_workspace_bytes", "pg_jarvis_patrick", "pg_clique4_workspace_bytes", "pg_clique4_count",
    "pg_batch_autotune", "pg_batch_workspace_bytes", "pg_batch_create", "pg_batch_run", "pg_batch_run_host",
    "pg_batch_destroy",
    "pg_server_reserved_bytes", "pg_server_create", "pg_submit", "pg_submit_many", "pg_poll_many", "pg_poll",
    "pg_cancel", "pg_server_stats_get", "pg_server_destroy",
]
REQ_PAIRS, REQ_SUBGRAPH_TC = 1, 2


class PGError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        super().__init__(f"{where}: {ERR.get(status, status)}: {detail}")
        self.status = status


class Csr(ctypes.Structure):
    _fields_ = [("row_ptr", ctypes.c_void_p), ("col", ctypes.c_void_p), ("n", ctypes.c_int32),
                ("nnz", ctypes.c_int64)]


class SketchDesc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("bits", ctypes.c_uint32), ("b", ctypes.c_uint32),
                ("k", ctypes.c_uint32), ("seed", ctypes.c_uint32), ("n", ctypes.c_int32),
                ("stride_bytes", ctypes.c_int64), ("data", ctypes.c_void_p)]


class Outputs(ctypes.Structure):
    _fields_ = [("tc", ctypes.c_void_p), ("lcc", ctypes.c_void_p), ("tri", ctypes.c_void_p),
                ("edge_cn", ctypes.c_void_p), ("edge_jac", ctypes.c_void_p), ("edge_count", ctypes.c_void_p),
                ("edge_aux", ctypes.c_void_p), ("hist", ctypes.c_void_p), ("edge_overlap", ctypes.c_void_p),
                ("edge_total", ctypes.c_void_p)]


class Similarity(ctypes.Structure):
    _fields_ = [("cn", ctypes.c_void_p), ("jac", ctypes.c_void_p), ("overlap", ctypes.c_void_p),
                ("total", ctypes.c_void_p)]


class BatchConfig(ctypes.Structure):
    _fields_ = [("bits", ctypes.c_uint32), ("b", ctypes.c_uint32), ("variant", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class ServerOpts(ctypes.Structure):
    _fields_ = [("streams", ctypes.c_int32), ("max_inflight", ctypes.c_int32), ("iteration_pairs", ctypes.c_int64),
                ("pinned_bytes", ctypes.c_size_t), ("sub_bits", ctypes.c_uint32), ("sub_b", ctypes.c_uint32),
                ("sub_seed", ctypes.c_uint32), ("reserved", ctypes.c_int32)]


class Request(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("estimator", ctypes.c_int32), ("count", ctypes.c_int64),
                ("data", ctypes.c_void_p), ("cn", ctypes.c_void_p), ("jac", ctypes.c_void_p)]


class TcResult(ctypes.Structure):
    _fields_ = [("edges", ctypes.c_uint64), ("count_sum", ctypes.c_uint64), ("exact_tc", ctypes.c_uint64),
                ("reserved", ctypes.c_uint64), ("est_tc", ctypes.c_double), ("est_tc_alt", ctypes.c_double)]


class Response(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("kind", ctypes.c_int32), ("count", ctypes.c_int64),
                ("tc", TcResult), ("queue_us", ctypes.c_double), ("total_us", ctypes.c_double)]


def _np_dtypes():
    import numpy as np
    req = np.dtype([("kind", "<i4"), ("estimator", "<i4"), ("count", "<i8"), ("data", "<u8"), ("cn", "<u8"),
                    ("jac", "<u8")])
    resp = np.dtype([("status", "<i4"), ("kind", "<i4"), ("count", "<i8"), ("edges", "<u8"),
                     ("count_sum", "<u8"), ("exact_tc", "<u8"), ("reserved", "<u8"), ("est_tc", "<f8"),
                     ("est_tc_alt", "<f8"), ("queue_us", "<f8"), ("total_us", "<f8")])
    assert req.itemsize == ctypes.sizeof(Request) and resp.itemsize == ctypes.sizeof(Response)
    return req, resp


REQUEST_DTYPE, RESPONSE_DTYPE = _np_dtypes()


class ServerStats(ctypes.Structure):
    _fields_ = [(nm, ctypes.c_uint64) for nm in
                ("submitted", "completed", "cancelled", "failed", "pair_launches", "pairs", "subgraphs", "queued",
                 "running", "arena_used", "arena_peak", "arena_bytes", "pair_kernel_ns")]


TC_RESULT_BYTES = 48
_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def lib() -> ctypes.CDLL:
    """Load libpg.so (built in-tree by paper_2208_11469_gb300.build)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if not os.path.exists(path):
                raise RuntimeError(f"{path} is missing: run paper_2208_11469_gb300.build.build() first")
            L = ctypes.CDLL(path)
            vp, i32, i64, u32, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_size_t
            P = ctypes.POINTER
            sig = {
                "pg_status_string": (ctypes.c_char_p, [i32]),
                "pg_last_error": (ctypes.c_char_p, []),
                "pg_version": (i32, []),
                "pg_validate_csr": (i32, [P(Csr), i32, vp, vp]),
                "pg_edge_index_bytes": (sz, [i32, i64]),
                "pg_build_edge_index": (i32, [P(Csr), vp, sz, vp]),
                "pg_edge_index_upper_off": (vp, [vp]),
                "pg_sketch_stride": (i64, [i32, u32, u32]),
                "pg_bloom_bits_for_budget": (u32, [ctypes.c_double, i32, i64]),
                "pg_build_workspace_bytes": (sz, [P(Csr)]),
                "pg_build_bloom": (i32, [P(Csr), P(SketchDesc), vp, sz, vp]),
                "pg_build_minhash": (i32, [P(Csr), P(SketchDesc), vp, sz, vp]),
                "pg_upload_build": (i32, [vp, vp, P(Csr), P(SketchDesc), i32, vp, sz, i64, vp, vp]),
                "pg_sketch_save": (i32, [P(SketchDesc), ctypes.c_char_p, vp]),
                "pg_sketch_load_header": (i32, [ctypes.c_char_p, P(SketchDesc)]),
                "pg_sketch_load": (i32, [P(SketchDesc), ctypes.c_char_p, vp]),
                "pg_hist_bins": (i64, [P(SketchDesc), i32]),
                "pg_workspace_bytes": (sz, [P(Csr), P(SketchDesc), i32]),
                "pg_triangle_count": (i32, [P(Csr), vp, P(SketchDesc), i32, vp, sz, vp, vp]),
                "pg_clustering": (i32, [P(Csr), vp, P(SketchDesc), i32, vp, sz, vp, vp, vp, vp]),
                "pg_jaccard_pairs": (i32, [P(Csr), vp, P(SketchDesc), i32, vp, i64, vp, sz, vp, vp, vp]),
                "pg_similarity_pairs": (i32, [P(Csr), vp, P(SketchDesc), i32, vp, i64, vp, sz, P(Similarity), vp]),
                "pg_edge_counts": (i32, [P(Csr), vp, P(SketchDesc), i32, vp, i64, vp, sz, vp, vp, vp, vp]),
                "pg_kernel_launches": (ctypes.c_uint64, []),
                "pg_analyze": (i32, [P(Csr), vp, P(SketchDesc), i32, vp, sz, P(Outputs), vp]),
                "pg_triangle_count_noalloc": (i32, [P(Csr), vp, P(SketchDesc), i32, vp, vp]),
                "pg_partial_sums": (i32, [P(Csr), vp, P(SketchDesc), i32, i32, i32, vp, sz, vp, vp, vp]),
                "pg_finalize_sums": (i32, [P(Csr), P(SketchDesc), i32, vp, vp, vp, vp, vp, vp]),
                "pg_jarvis_patrick_workspace_bytes": (sz, [P(Csr), P(SketchDesc), i32]),
                "pg_clique4_workspace_bytes": (sz, [P(Csr), i32, u32]),
                "pg_clique4_count": (i32, [P(Csr), i32, u32, u32, u32, vp, sz, vp, vp]),
                "pg_jarvis_patrick": (i32, [P(Csr), vp, P(SketchDesc), i32, ctypes.c_double, vp, sz, vp, vp, vp]),
                "pg_batch_autotune": (i32, [vp, vp, i32, ctypes.c_double, P(BatchConfig)]),
                "pg_batch_workspace_bytes": (sz, [P(Csr), i32, vp, P(BatchConfig)]),
                "pg_batch_create": (i32, [P(Csr), i32, vp, P(BatchConfig), u32, vp, sz, vp, vp, vp, vp,
                                          P(vp)]),
                "pg_batch_run": (i32, [vp, vp]),
                "pg_batch_run_host": (i32, [vp, vp, vp, i64, vp, vp]),
                "pg_batch_destroy": (i32, [vp]),
                "pg_server_reserved_bytes": (sz, [P(Csr), P(ServerOpts)]),
                "pg_server_create": (i32, [P(Csr), P(P(SketchDesc)), i32, vp, sz, P(ServerOpts), P(vp)]),
                "pg_submit": (i32, [vp, P(Request), P(ctypes.c_uint64)]),
                "pg_poll": (i32, [vp, ctypes.c_uint64, P(Response), i64]),
                "pg_submit_many": (i32, [vp, vp, i64, vp]),
                "pg_poll_many": (i32, [vp, vp, i64, vp, i64, P(i64)]),
                "pg_cancel": (i32, [vp, ctypes.c_uint64]),
                "pg_server_stats_get": (i32, [vp, P(ServerStats)]),
                "pg_server_destroy": (i32, [vp]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _check(status: int, where: str):
    if status != OK:
        raise PGError(status, where, lib().pg_last_error().decode(errors="replace"))


def _stream() -> int:
    return torch.cuda.current_stream().cuda_stream


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _dev_bytes(nbytes: int, device) -> torch.Tensor:
    # 16-byte aligned by the caching allocator (its blocks are 512-byte aligned)
    return torch.empty(max(int(nbytes), 16), dtype=torch.uint8, device=device)


# -------------------------------------------------------------------- graph
@dataclass
class Graph:
    """An int32 CSR graph resident on the device, with its upper-edge index."""
    row_ptr: torch.Tensor
    col: torch.Tensor
    index: torch.Tensor | None = None
    _m: int | None = field(default=None, repr=False)

    @property
    def n(self) -> int:
        return self.row_ptr.numel() - 1

    @property
    def nnz(self) -> int:
        return self.col.numel()

    @property
    def device(self):
        return self.row_ptr.device

    def csr(self) -> Csr:
        return Csr(self.row_ptr.data_ptr(), self.col.data_ptr() if self.col.numel() else None,
                   self.n, self.nnz)

    @property
    def upper_off(self) -> torch.Tensor:
        return self.index[: 4 * (self.n + 1)].view(torch.int32)

    @property
    def m(self) -> int:
        if self._m is None:
            self._m = int(self.upper_off[self.n].item())
        return self._m

    def degrees(self) -> torch.Tensor:
        return (self.row_ptr[1:] - self.row_ptr[:-1])


def graph(row_ptr: torch.Tensor, col: torch.Tensor, build_index: bool = True) -> Graph:
    if row_ptr.dtype != torch.int32 or col.dtype != torch.int32:
        raise TypeError("row_ptr and col must be int32")
    if not row_ptr.is_cuda or not col.is_cuda:
        raise ValueError("row_ptr and col must be CUDA tensors")
    g = Graph(row_ptr.contiguous(), col.contiguous())
    if build_index:
        build_edge_index(g)
    return g


def build_edge_index(g: Graph) -> torch.Tensor:
    L = lib()
    nbytes = L.pg_edge_index_bytes(g.n, g.nnz)
    idx = _dev_bytes(nbytes, g.device)
    c = g.csr()
    _check(L.pg_build_edge_index(ctypes.byref(c), _ptr(idx), idx.numel(), _stream()), "pg_build_edge_index")
    g.index = idx
    g._m = None
    return idx


def build_edge_index_into(g: Graph) -> None:
    """Rebuild the upper-edge index in the graph's existing index buffer."""
    c = g.csr()
    _check(lib().pg_build_edge_index(ctypes.byref(c), _ptr(g.index), g.index.numel(), _stream()),
           "pg_build_edge_index")


def validate_csr(g: Graph, check_symmetry: bool = True):
    """Returns (code_name, index) after synchronising the stream."""
    res = torch.zeros(2, dtype=torch.int64, device=g.device)
    c = g.csr()
    _check(lib().pg_validate_csr(ctypes.byref(c), int(check_symmetry), _ptr(res), _stream()), "pg_validate_csr")
    r = res.cpu()
    return CSR_CODES.get(int(r[0]), int(r[0])), int(r[1])


# ----------------------------------------------------------------- sketches
@dataclass
class Sketch:
    kind: int
    bits: int
    b: int
    k: int
    seed: int
    n: int
    stride: int
    data: torch.Tensor

    def desc(self) -> SketchDesc:
        return SketchDesc(self.kind, self.bits, self.b, self.k, self.seed & 0xFFFFFFFF, self.n,
                          self.stride, self.data.data_ptr() if self.data.numel() else None)

    def rows_u8(self) -> torch.Tensor:
        return self.data.view(self.n, self.stride)


def sketch_stride(kind: int, bits: int = 0, k: int = 0) -> int:
    return int(lib().pg_sketch_stride(kind, bits, k))


def bloom_bits_for_budget(s: float, n: int, nnz: int) -> int:
    return int(lib().pg_bloom_bits_for_budget(float(s), n, nnz))


def alloc_sketch(g: Graph, kind: int, *, bits: int = 0, b: int = 0, k: int = 0, seed: int = 1,
                 stride: int | None = None) -> Sketch:
    st = sketch_stride(kind, bits, k) if stride is None else int(stride)
    data = _dev_bytes(g.n * st, g.device)
    return Sketch(kind, bits, b, k, seed, g.n, st, data)


def sketch_save(sk: Sketch, path: str) -> None:
    """pg_sketch_save: write the sketch rows and descriptor to a file."""
    d = sk.desc()
    _check(lib().pg_sketch_save(ctypes.byref(d), os.fsencode(path), _stream()), "pg_sketch_save")


def sketch_load(path: str, device="cuda") -> Sketch:
    """pg_sketch_load_header + pg_sketch_load: a sketch read back from a file."""
    d = SketchDesc()
    _check(lib().pg_sketch_load_header(os.fsencode(path), ctypes.byref(d)), "pg_sketch_load_header")
    data = _dev_bytes(d.n * d.stride_bytes, torch.device(device))
    sk = Sketch(d.kind, d.bits, d.b, d.k, d.seed, d.n, d.stride_bytes, data)
    d2 = sk.desc()
    _check(lib().pg_sketch_load(ctypes.byref(d2), os.fsencode(path), _stream()), "pg_sketch_load")
    return sk


def build_workspace_bytes(g: Graph) -> int:
    c = g.csr()
    return int(lib().pg_build_workspace_bytes(ctypes.byref(c)))


def build_bloom(g: Graph, bits: int, b: int, seed: int, stride: int | None = None,
                out: Sketch | None = None, workspace: torch.Tensor | None = None) -> Sketch:
    sk = out if out is not None else alloc_sketch(g, SK_BLOOM, bits=bits, b=b, seed=seed, stride=stride)
    ws = workspace if workspace is not None else _dev_bytes(build_workspace_bytes(g), g.device)
    c, d = g.csr(), sk.desc()
    _check(lib().pg_build_bloom(ctypes.byref(c), ctypes.byref(d), _ptr(ws), ws.numel(), _stream()), "pg_build_bloom")
    return sk


def build_minhash(g: Graph, kind: int, k: int, seed: int, stride: int | None = None,
                  out: Sketch | None = None, workspace: torch.Tensor | None = None) -> Sketch:
    sk = out if out is not None else alloc_sketch(g, kind, k=k, seed=seed, stride=stride)
    ws = workspace if workspace is not None else _dev_bytes(build_workspace_bytes(g), g.device)
    c, d = g.csr(), sk.desc()
    _check(lib().pg_build_minhash(ctypes.byref(c), ctypes.byref(d), _ptr(ws), ws.numel(), _stream()),
           "pg_build_minhash")
    return sk


def upload_build(g: Graph, host_row_ptr: torch.Tensor, host_col: torch.Tensor, sketches, *,
                 workspace: torch.Tensor | None = None, chunk_entries: int | None = None, copy_stream=None):
    """pg_upload_build: copy the CSR from host tensors (page-locked for overlap)
    into g's device buffers in row chunks on copy_stream (a torch.cuda.Stream;
    None: a stream of this module) while the current stream builds every
    sketch's rows of each chunk as it lands. The sketches must be allocated
    for g (alloc_sketch) and carry their kind and parameters."""
    assert host_row_ptr.device.type == "cpu" and host_col.device.type == "cpu"
    assert host_row_ptr.dtype == torch.int32 and host_col.dtype == torch.int32
    assert host_row_ptr.is_contiguous() and host_col.is_contiguous()
    ws = workspace if workspace is not None else _dev_bytes(build_workspace_bytes(g), g.device)
    if chunk_entries is None:
        chunk_entries = max(1 << 20, g.nnz // 8)
    if copy_stream is None:
        global _upload_stream
        if _upload_stream is None:
            _upload_stream = torch.cuda.Stream(device=g.device)
        copy_stream = _upload_stream
    descs = (SketchDesc * max(len(sketches), 1))(*[sk.desc() for sk in sketches])
    c = g.csr()
    _check(lib().pg_upload_build(host_row_ptr.data_ptr(), host_col.data_ptr(), ctypes.byref(c), descs,
                                 len(sketches), _ptr(ws), ws.numel(), int(chunk_entries),
                                 copy_stream.cuda_stream, _stream()), "pg_upload_build")


_upload_stream = None


# ----------------------------------------------------------------- analysis
def workspace_bytes(g: Graph, sk: Sketch | None, est: int) -> int:
    c = g.csr()
    d = sk.desc() if sk is not None else None
    return int(lib().pg_workspace_bytes(ctypes.byref(c), ctypes.byref(d) if d is not None else None, est))


def hist_bins(sk: Sketch | None, est: int) -> int:
    if sk is None:
        return 0
    d = sk.desc()
    return int(lib().pg_hist_bins(ctypes.byref(d), est))


def workspace(g: Graph, sk: Sketch | None, est: int) -> torch.Tensor:
    return _dev_bytes(workspace_bytes(g, sk, est), g.device)


def tc_result_buffer(device) -> torch.Tensor:
    return torch.zeros(TC_RESULT_BYTES, dtype=torch.uint8, device=device)


def read_tc_result(buf: torch.Tensor) -> dict:
    raw = bytes(buf.cpu().numpy().tobytes())
    edges, count_sum, exact_tc, _, est_tc, est_tc_alt = struct.unpack("<QQQQdd", raw)
    return {"edges": edges, "count_sum": count_sum, "exact_tc": exact_tc, "est_tc": est_tc,
            "est_tc_alt": est_tc_alt}


def _sk_args(sk):
    if sk is None:
        return None, None
    d = sk.desc()
    return d, ctypes.byref(d)


def triangle_count(g: Graph, sk: Sketch | None, est: int, *, ws: torch.Tensor | None = None,
                   out: torch.Tensor | None = None, read: bool = True):
    ws = ws if ws is not None else workspace(g, sk, est)
    out = out if out is not None else tc_result_buffer(g.device)
    c = g.csr()
    d, dref = _sk_args(sk)
    _check(lib().pg_triangle_count(ctypes.byref(c), _ptr(g.index), dref, est, _ptr(ws), ws.numel(),
                                   _ptr(out), _stream()), "pg_triangle_count")
    return read_tc_result(out) if read else out


def clustering(g: Graph, sk: Sketch | None, est: int, *, want_tri: bool = True, want_tc: bool = True,
               ws: torch.Tensor | None = None, lcc: torch.Tensor | None = None,
               tri: torch.Tensor | None = None, tc: torch.Tensor | None = None):
    """Returns (lcc float32[n], tri float64[n] or None, tc result buffer or None)."""
    ws = ws if ws is not None else workspace(g, sk, est)
    lcc = lcc if lcc is not None else torch.empty(g.n, dtype=torch.float32, device=g.device)
    if want_tri and tri is None:
        tri = torch.empty(g.n, dtype=torch.float64, device=g.device)
    if want_tc and tc is None:
        tc = tc_result_buffer(g.device)
    c = g.csr()
    d, dref = _sk_args(sk)
    _check(lib().pg_clustering(ctypes.byref(c), _ptr(g.index), dref, est, _ptr(ws), ws.numel(), _ptr(lcc),
                               _ptr(tri) if want_tri else None, _ptr(tc) if want_tc else None, _stream()),
           "pg_clustering")
    return lcc, (tri if want_tri else None), (tc if want_tc else None)


def _pairs_arg(pairs):
    if pairs is None:
        return None, 0
    if pairs.dtype != torch.int32 or not pairs.is_cuda:
        raise TypeError("pairs must be a CUDA int32 tensor of shape [P, 2]")
    pairs = pairs.contiguous()
    return pairs, pairs.numel() // 2


def jaccard_pairs(g: Graph, sk: Sketch | None, est: int, pairs: torch.Tensor | None = None, *,
                  ws: torch.Tensor | None = None, want_cn: bool = True, want_jac: bool = True):
    pairs, P = _pairs_arg(pairs)
    count = P if pairs is not None else g.m
    ws = ws if ws is not None else workspace(g, sk, est)
    cn = torch.empty(count, dtype=torch.float32, device=g.device) if want_cn else None
    jac = torch.empty(count, dtype=torch.float32, device=g.device) if want_jac else None
    c = g.csr()
    d, dref = _sk_args(sk)
    _check(lib().pg_jaccard_pairs(ctypes.byref(c), _ptr(g.index), dref, est, _ptr(pairs), P, _ptr(ws),
                                  ws.numel(), _ptr(cn), _ptr(jac), _stream()), "pg_jaccard_pairs")
    return cn, jac


def similarity_pairs(g: Graph, sk: Sketch | None, est: int, pairs: torch.Tensor | None = None, *,
                     ws: torch.Tensor | None = None):
    """pg_similarity_pairs: dict of float32 tensors cn, jac, overlap, total
    (per pair, or per upper edge with pairs None)."""
    pairs, P = _pairs_arg(pairs)
    count = P if pairs is not None else g.m
    ws = ws if ws is not None else workspace(g, sk, est)
    out = {nm: torch.empty(max(count, 1), dtype=torch.float32, device=g.device)
           for nm in ("cn", "jac", "overlap", "total")}
    sim = Similarity(*[out[nm].data_ptr() for nm in ("cn", "jac", "overlap", "total")])
    c = g.csr()
    d, dref = _sk_args(sk)
    _check(lib().pg_similarity_pairs(ctypes.byref(c), _ptr(g.index), dref, est, _ptr(pairs), P, _ptr(ws),
                                     ws.numel(), ctypes.byref(sim), _stream()), "pg_similarity_pairs")
    return {nm: t[:count] for nm, t in out.items()}


def edge_counts(g: Graph, sk: Sketch | None, est: int, pairs: torch.Tensor | None = None, *,
                want_aux: bool = False, want_hist: bool = False, ws: torch.Tensor | None = None):
    pairs, P = _pairs_arg(pairs)
    count = P if pairs is not None else g.m
    ws = ws if ws is not None else workspace(g, sk, est)
    cnt = torch.empty(count, dtype=torch.int32, device=g.device)
    aux = torch.empty(count, dtype=torch.int32, device=g.device) if want_aux else None
    hist = torch.empty(max(hist_bins(sk, est), 1), dtype=torch.int64, device=g.device) if want_hist else None
    c = g.csr()
    d, dref = _sk_args(sk)
    _check(lib().pg_edge_counts(ctypes.byref(c), _ptr(g.index), dref, est, _ptr(pairs), P, _ptr(ws),
                                ws.numel(), _ptr(cnt), _ptr(aux), _ptr(hist), _stream()), "pg_edge_counts")
    return cnt, aux, hist


def kernel_launches() -> int:
    return int(lib().pg_kernel_launches())


def analyze(g: Graph, sk: Sketch | None, est: int, *, tc=None, lcc=None, tri=None, edge_cn=None,
            edge_jac=None, edge_count=None, edge_aux=None, hist=None, edge_overlap=None, edge_total=None,
            ws: torch.Tensor | None = None):
    """One fused pass (pg_analyze). Pass preallocated device tensors for the
    outputs wanted; None leaves an output out."""
    ws = ws if ws is not None else workspace(g, sk, est)
    o = Outputs(*[t.data_ptr() if t is not None else None
                  for t in (tc, lcc, tri, edge_cn, edge_jac, edge_count, edge_aux, hist, edge_overlap,
                            edge_total)])
    c = g.csr()
    d, dref = _sk_args(sk)
    _check(lib().pg_analyze(ctypes.byref(c), _ptr(g.index), dref, est, _ptr(ws), ws.numel(), ctypes.byref(o),
                            _stream()), "pg_analyze")


def triangle_count_noalloc(g: Graph, sk: Sketch, est: int, *, out: torch.Tensor | None = None,
                           read: bool = True):
    """pg_triangle_count_noalloc: the sketched triangle count with its scratch
    in the library's static device array (no workspace; see include/pg.h)."""
    out = out if out is not None else tc_result_buffer(g.device)
    c = g.csr()
    d, dref = _sk_args(sk)
    _check(lib().pg_triangle_count_noalloc(ctypes.byref(c), _ptr(g.index), dref, est, _ptr(out), _stream()),
           "pg_triangle_count_noalloc")
    return read_tc_result(out) if read else out


# -------------------------------------------------- vertex-partitioned runs
def partial_sums(g: Graph, sk: Sketch, est: int, u_begin: int, u_end: int, *, sums: torch.Tensor | None = None,
                 hist: torch.Tensor | None = None, ws: torch.Tensor | None = None):
    """pg_partial_sums: the estimates of the upper edges (u, v) with
    u_begin <= u < u_end added into sums (double [n]) at both endpoints and
    their counts into hist (int64 [hist_bins]); both are zeroed here when
    not given."""
    ws = ws if ws is not None else workspace(g, sk, est)
    if sums is None:
        sums = torch.zeros(g.n, dtype=torch.float64, device=g.device)
    if hist is None:
        hist = torch.zeros(max(hist_bins(sk, est), 1), dtype=torch.int64, device=g.device)
    c = g.csr()
    d, dref = _sk_args(sk)
    _check(lib().pg_partial_sums(ctypes.byref(c), _ptr(g.index), dref, est, int(u_begin), int(u_end), _ptr(ws),
                                 ws.numel(), _ptr(sums), _ptr(hist), _stream()), "pg_partial_sums")
    return sums, hist


def finalize_sums(g: Graph, sk: Sketch, est: int, hist: torch.Tensor, sums: torch.Tensor, *,
                  tc: torch.Tensor | None = None, lcc: torch.Tensor | None = None, tri: torch.Tensor | None = None):
    """pg_finalize_sums: TC from a summed histogram, T = sums / 2 and LCC."""
    tc = tc if tc is not None else tc_result_buffer(g.device)
    lcc = lcc if lcc is not None else torch.empty(g.n, dtype=torch.float32, device=g.device)
    tri = tri if tri is not None else torch.empty(g.n, dtype=torch.float64, device=g.device)
    c = g.csr()
    d, dref = _sk_args(sk)
    _check(lib().pg_finalize_sums(ctypes.byref(c), dref, est, _ptr(hist), _ptr(sums), _ptr(tc), _ptr(lcc), _ptr(tri),
                                  _stream()), "pg_finalize_sums")
    return tc, lcc, tri


# ------------------------------------------------------------ Jarvis-Patrick
def jarvis_patrick(g: Graph, sk: Sketch | None, est: int, tau: float, *, labels: torch.Tensor | None = None,
                   want_labels: bool = True, ws: torch.Tensor | None = None, out: torch.Tensor | None = None,
                   read: bool = True):
    """pg_jarvis_patrick: returns (labels int32 [n] or None, result dict or
    the device result buffer when read=False)."""
    c = g.csr()
    d, dref = _sk_args(sk)
    if ws is None:
        ws = _dev_bytes(lib().pg_jarvis_patrick_workspace_bytes(ctypes.byref(c), dref, est), g.device)
    if want_labels and labels is None:
        labels = torch.empty(max(g.n, 1), dtype=torch.int32, device=g.device)
    out = out if out is not None else torch.zeros(32, dtype=torch.uint8, device=g.device)
    _check(lib().pg_jarvis_patrick(ctypes.byref(c), _ptr(g.index), dref, est, float(tau), _ptr(ws), ws.numel(),
                                   _ptr(labels) if want_labels else None, _ptr(out), _stream()),
           "pg_jarvis_patrick")
    if not read:
        return (labels[: g.n] if want_labels else None), out
    clusters, kept, edges, _ = struct.unpack("<qqqq", bytes(out.cpu().numpy().tobytes()))
    return (labels[: g.n] if want_labels else None), {"clusters": clusters, "kept": kept, "edges": edges}


# ---------------------------------------------------------------- 4-cliques
def clique4_count(g: Graph, est: int, bits: int = 256, b: int = 2, seed: int = 1, *,
                  ws: torch.Tensor | None = None, out: torch.Tensor | None = None, read: bool = True):
    """pg_clique4_count: 4-cliques, exact or with the innermost intersection
    estimated from Bloom filters of the oriented neighbourhoods."""
    c = g.csr()
    if ws is None:
        ws = _dev_bytes(lib().pg_clique4_workspace_bytes(ctypes.byref(c), est, bits), g.device)
    out = out if out is not None else torch.zeros(48, dtype=torch.uint8, device=g.device)
    _check(lib().pg_clique4_count(ctypes.byref(c), est, bits, b, seed, _ptr(ws), ws.numel(), _ptr(out), _stream()),
           "pg_clique4_count")
    if not read:
        return out
    tri, exact, cs, _, e, ea = struct.unpack("<QQQQdd", bytes(out.cpu().numpy().tobytes()))
    return {"triangles": tri, "exact": exact, "count_sum": cs, "est": e, "est_alt": ea}


# -------------------------------------------------------------------- batch
def batch_autotune(n, nnz, budget: float):
    """pg_batch_autotune over host arrays of per-graph vertex and entry
    counts: returns a list of (bits, b) per graph."""
    import numpy as np
    n = np.ascontiguousarray(n, dtype=np.int32)
    nnz = np.ascontiguousarray(nnz, dtype=np.int64)
    G = len(n)
    cfg = (BatchConfig * max(G, 1))()
    _check(lib().pg_batch_autotune(n.ctypes.data_as(ctypes.c_void_p), nnz.ctypes.data_as(ctypes.c_void_p), G,
                                   float(budget), cfg), "pg_batch_autotune")
    return [(cfg[i].bits, cfg[i].b) for i in range(G)]


class Batch:
    """pg_batch_*: G graphs as one block-diagonal CSR (graph i = vertices
    voff[i] .. voff[i+1]-1), each with its own Bloom (bits, b); one run
    computes every graph's triangle count and every vertex's LCC. Owns its
    workspace and outputs; `run()` enqueues on the current stream (captured
    as a CUDA graph on first use there)."""

    def __init__(self, g: Graph, voff, configs, seed: int = 1, *, want_tri: bool = False):
        import numpy as np
        self.g = g
        self.voff = np.ascontiguousarray(voff, dtype=np.int32)
        self.G = len(self.voff) - 1
        self.cfg = (BatchConfig * self.G)()
        for i, c in enumerate(configs):
            bits, b = c[0], c[1]
            variant = c[2] if len(c) > 2 else 0
            self.cfg[i] = BatchConfig(bits, b, variant, 0)
        self._csr = g.csr()
        vp = self.voff.ctypes.data_as(ctypes.c_void_p)
        nbytes = lib().pg_batch_workspace_bytes(ctypes.byref(self._csr), self.G, vp, self.cfg)
        if nbytes == 0:
            raise PGError(-1, "pg_batch_workspace_bytes", lib().pg_last_error().decode(errors="replace"))
        self.ws = _dev_bytes(nbytes, g.device)
        self.tc = torch.zeros(self.G * TC_RESULT_BYTES, dtype=torch.uint8, device=g.device)
        self.lcc = torch.zeros(g.n, dtype=torch.float32, device=g.device)
        self.tri = torch.zeros(g.n, dtype=torch.float64, device=g.device) if want_tri else None
        h = ctypes.c_void_p()
        _check(lib().pg_batch_create(ctypes.byref(self._csr), self.G, vp, self.cfg, seed, _ptr(self.ws),
                                     self.ws.numel(), _ptr(self.tc), _ptr(self.lcc), _ptr(self.tri), _stream(),
                                     ctypes.byref(h)), "pg_batch_create")
        self._h = h

    @property
    def variants(self):
        return [self.cfg[i].variant for i in range(self.G)]

    def run(self, stream: int | None = None):
        _check(lib().pg_batch_run(self._h, _stream() if stream is None else stream), "pg_batch_run")

    def run_host(self, host_row_ptr: torch.Tensor, host_col: torch.Tensor, chunk_entries: int | None = None,
                 copy_stream=None):
        """pg_batch_run_host: one run from host tensors of the union CSR
        (page-locked for overlap), uploaded in chunks of whole graphs on
        copy_stream (a torch.cuda.Stream; None: a stream of this module)
        while the current stream works on the chunks already copied."""
        assert host_row_ptr.device.type == "cpu" and host_col.device.type == "cpu"
        assert host_row_ptr.dtype == torch.int32 and host_col.dtype == torch.int32
        assert host_row_ptr.is_contiguous() and host_col.is_contiguous()
        if chunk_entries is None:
            chunk_entries = max(1 << 20, self.g.nnz // 16)
        if copy_stream is None:
            global _upload_stream
            if _upload_stream is None:
                _upload_stream = torch.cuda.Stream(device=self.g.device)
            copy_stream = _upload_stream
        _check(lib().pg_batch_run_host(self._h, host_row_ptr.data_ptr(), host_col.data_ptr(), int(chunk_entries),
                                       copy_stream.cuda_stream, _stream()), "pg_batch_run_host")

    def results(self):
        """Per-graph dicts of the triangle-count result (synchronises)."""
        raw = self.tc.cpu().numpy().tobytes()
        out = []
        for i in range(self.G):
            edges, count_sum, exact_tc, _, est_tc, est_tc_alt = struct.unpack_from("<QQQQdd", raw, 48 * i)
            out.append({"edges": edges, "count_sum": count_sum, "exact_tc": exact_tc, "est_tc": est_tc,
                        "est_tc_alt": est_tc_alt})
        return out

    def est_tc(self) -> torch.Tensor:
        """Per-graph triangle-count estimates as a device float64 view."""
        return self.tc.view(self.G, 6 * 8).view(torch.float64)[:, 4]

    def close(self):
        if getattr(self, "_h", None):
            lib().pg_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ serving
def pinned_empty(shape, dtype):
    """A numpy array in page-locked host memory: a view of a pinned torch
    tensor, which the array's base keeps alive."""
    import numpy as np
    dt = np.dtype(dtype)
    n = int(np.prod(shape))
    t = torch.empty(max(n * dt.itemsize, 16), dtype=torch.uint8, pin_memory=True)
    return t.numpy()[: n * dt.itemsize].view(dt).reshape(shape)


class Server:
    """pg_server_*: a request loop over the resident graph `g` and its
    sketches (see include/pg.h). Requests take and return host numpy arrays;
    the arena is a device tensor owned here."""

    def __init__(self, g: Graph, sketches, arena_bytes: int, *, streams: int = 0, max_inflight: int = 0,
                 iteration_pairs: int = 0, pinned_bytes: int = 0, sub_bits: int = 0, sub_b: int = 0,
                 sub_seed: int = 0):
        self.g = g
        self._descs = [sk.desc() for sk in sketches]
        self._sketches = list(sketches)
        arr = (ctypes.POINTER(SketchDesc) * max(len(self._descs), 1))(*[ctypes.pointer(d) for d in self._descs])
        self._arr = arr
        self.opts = ServerOpts(streams, max_inflight, iteration_pairs, pinned_bytes, sub_bits, sub_b, sub_seed, 0)
        self._csr = g.csr()
        self.arena = _dev_bytes(arena_bytes, g.device)
        h = ctypes.c_void_p()
        torch.cuda.synchronize()
        _check(lib().pg_server_create(ctypes.byref(self._csr), arr, len(self._descs), _ptr(self.arena),
                                      self.arena.numel(), ctypes.byref(self.opts), ctypes.byref(h)),
               "pg_server_create")
        self._h = h
        self._live = {}  # ticket -> arrays kept alive until the response is collected

    @staticmethod
    def reserved_bytes(g: Graph, **opts) -> int:
        o = ServerOpts(opts.get("streams", 0), opts.get("max_inflight", 0), opts.get("iteration_pairs", 0),
                       opts.get("pinned_bytes", 0), opts.get("sub_bits", 0), opts.get("sub_b", 0),
                       opts.get("sub_seed", 0), 0)
        c = g.csr()
        return int(lib().pg_server_reserved_bytes(ctypes.byref(c), ctypes.byref(o)))

    def submit_pairs(self, pairs, est: int, want_cn: bool = True, want_jac: bool = True) -> int:
        import numpy as np
        pairs = np.ascontiguousarray(pairs, dtype=np.int32).reshape(-1, 2)
        P = pairs.shape[0]
        cn = np.empty(P, np.float32) if want_cn else None
        jac = np.empty(P, np.float32) if want_jac else None
        req = Request(REQ_PAIRS, est, P, pairs.ctypes.data if P else None,
                      cn.ctypes.data if cn is not None and P else None,
                      jac.ctypes.data if jac is not None and P else None)
        t = ctypes.c_uint64()
        _check(lib().pg_submit(self._h, ctypes.byref(req), ctypes.byref(t)), "pg_submit")
        self._live[t.value] = (pairs, cn, jac)
        return t.value

    def submit_subgraph(self, vertices, est: int) -> int:
        import numpy as np
        v = np.ascontiguousarray(vertices, dtype=np.int32).reshape(-1)
        req = Request(REQ_SUBGRAPH_TC, est, v.size, v.ctypes.data if v.size else None, None, None)
        t = ctypes.c_uint64()
        _check(lib().pg_submit(self._h, ctypes.byref(req), ctypes.byref(t)), "pg_submit")
        self._live[t.value] = (v, None, None)
        return t.value

    def submit_pairs_many(self, pairs, offsets, est: int, want_cn: bool = True, want_jac: bool = True,
                          pinned: bool = False):
        """Many pair requests in one call: request i is pairs[offsets[i]:offsets[i+1]]
        (pairs int32 [P, 2]). Returns (tickets uint64 [R], cn float32 [P] or None,
        jac float32 [P] or None); request i's outputs are the same slice.
        pinned=True puts the outputs in page-locked memory; with a page-locked
        `pairs` too (pinned_empty), the GPU reads and writes them in place."""
        import numpy as np
        pairs = np.ascontiguousarray(pairs, dtype=np.int32).reshape(-1, 2)
        offsets = np.asarray(offsets, dtype=np.int64)
        R = offsets.size - 1
        alloc = (lambda k: pinned_empty(k, np.float32)) if pinned else (lambda k: np.empty(k, np.float32))
        cn = alloc(max(pairs.shape[0], 1)) if want_cn else None
        jac = alloc(max(pairs.shape[0], 1)) if want_jac else None
        reqs = np.zeros(R, dtype=REQUEST_DTYPE)
        counts = np.diff(offsets)
        reqs["kind"] = REQ_PAIRS
        reqs["estimator"] = est
        reqs["count"] = counts
        nz = counts > 0
        reqs["data"] = np.where(nz, pairs.ctypes.data + 8 * offsets[:-1], 0)
        if cn is not None:
            reqs["cn"] = np.where(nz, cn.ctypes.data + 4 * offsets[:-1], 0)
        if jac is not None:
            reqs["jac"] = np.where(nz, jac.ctypes.data + 4 * offsets[:-1], 0)
        tickets = np.zeros(R, dtype=np.uint64)
        _check(lib().pg_submit_many(self._h, reqs.ctypes.data, R, tickets.ctypes.data), "pg_submit_many")
        keep = (pairs, cn, jac)
        for t in tickets.tolist():
            self._live[t] = keep
        return tickets, cn, jac

    def submit_many(self, reqs_list):
        """Mixed requests in one call: a list of ("pairs", int32 [P, 2], est) or
        ("sub", int32 vertices, est). Pair outputs are returned per request in
        the response of poll_many via `outputs`. Returns (tickets, outputs)."""
        import numpy as np
        R = len(reqs_list)
        reqs = np.zeros(R, dtype=REQUEST_DTYPE)
        outputs, keep = [], []
        for i, (kind, x, est) in enumerate(reqs_list):
            if kind == "pairs":
                x = np.ascontiguousarray(x, dtype=np.int32).reshape(-1, 2)
                cn = np.empty(max(x.shape[0], 1), np.float32)
                jac = np.empty(max(x.shape[0], 1), np.float32)
                reqs[i] = (REQ_PAIRS, est, x.shape[0], x.ctypes.data if x.shape[0] else 0,
                           cn.ctypes.data if x.shape[0] else 0, jac.ctypes.data if x.shape[0] else 0)
                outputs.append((cn[: x.shape[0]], jac[: x.shape[0]]))
                keep.append((x, cn, jac))
            else:
                x = np.ascontiguousarray(x, dtype=np.int32).reshape(-1)
                reqs[i] = (REQ_SUBGRAPH_TC, est, x.size, x.ctypes.data if x.size else 0, 0, 0)
                outputs.append(None)
                keep.append((x, None, None))
        tickets = np.zeros(R, dtype=np.uint64)
        _check(lib().pg_submit_many(self._h, reqs.ctypes.data, R, tickets.ctypes.data), "pg_submit_many")
        for t, k in zip(tickets.tolist(), keep):
            self._live[t] = k
        return tickets, outputs

    def poll_many(self, tickets, timeout_us: int = 0):
        """Responses (numpy structured array, RESPONSE_DTYPE) of the tickets;
        status -8 for those still running after timeout_us."""
        import numpy as np
        tickets = np.ascontiguousarray(tickets, dtype=np.uint64)
        out = np.zeros(tickets.size, dtype=RESPONSE_DTYPE)
        nd = ctypes.c_int64()
        st = lib().pg_poll_many(self._h, tickets.ctypes.data, tickets.size, out.ctypes.data, int(timeout_us),
                                ctypes.byref(nd))
        if st not in (0, -8):
            _check(st, "pg_poll_many")
        for t, s_ in zip(tickets.tolist(), out["status"].tolist()):
            if s_ != -8:
                self._live.pop(t, None)
        return out

    def poll(self, ticket: int, timeout_us: int = 0):
        """The response as a dict (with 'cn'/'jac' arrays for pairs), or None
        while the request runs. Raises PGError for unknown tickets."""
        r = Response()
        st = lib().pg_poll(self._h, ticket, ctypes.byref(r), int(timeout_us))
        if st == -8:
            return None
        _check(st, "pg_poll")
        _, cn, jac = self._live.pop(ticket, (None, None, None))
        tc = {nm: getattr(r.tc, nm) for nm, _ in TcResult._fields_ if nm != "reserved"}
        return {"status": r.status, "kind": r.kind, "count": r.count, "tc": tc, "queue_us": r.queue_us,
                "total_us": r.total_us, "cn": cn, "jac": jac}

    def wait(self, ticket: int, timeout_s: float = 60.0):
        r = self.poll(ticket, int(timeout_s * 1e6))
        if r is None:
            raise PGError(-6, "Server.wait", f"ticket {ticket} not complete after {timeout_s} s")
        return r

    def cancel(self, ticket: int) -> int:
        return int(lib().pg_cancel(self._h, ticket))

    def stats(self) -> dict:
        s = ServerStats()
        _check(lib().pg_server_stats_get(self._h, ctypes.byref(s)), "pg_server_stats_get")
        return {nm: getattr(s, nm) for nm, _ in ServerStats._fields_}

    def close(self):
        if getattr(self, "_h", None):
            _check(lib().pg_server_destroy(self._h), "pg_server_destroy")
            self._h = None
            self._live.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
