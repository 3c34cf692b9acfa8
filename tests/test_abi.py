"""Host-side checks of the C ABI that need no GPU: the library builds for
sm_103a, loads, exports every function include/pg.h declares, and rejects
bad arguments with status codes before touching the device."""
import ctypes
import os
import re

import pytest

from paper_2208_11469_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pg.h")


@pytest.fixture(scope="module")
def L():
    import shutil
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    B.build()
    from paper_2208_11469_gb300 import pg
    return pg.lib()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(pg_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


def test_header_declares_the_binding_symbols():
    from paper_2208_11469_gb300 import pg
    assert set(declared_functions()) == set(pg.SYMBOLS)


def test_every_declared_symbol_is_exported(L):
    for name in declared_functions():
        assert hasattr(L, name), name


def test_status_strings_and_version(L):
    assert L.pg_status_string(0) == b"PG_OK"
    assert L.pg_status_string(-4) == b"PG_ERR_NO_MEMORY"
    assert L.pg_version() >> 16 == 1


def test_sizing_helpers(L):
    from paper_2208_11469_gb300 import pg
    assert pg.sketch_stride(pg.SK_BLOOM, 448, 0) == 64
    assert pg.sketch_stride(pg.SK_BLOOM, 192, 0) == 32
    assert pg.sketch_stride(pg.SK_BLOOM, 960, 0) == 128
    assert pg.sketch_stride(pg.SK_KHASH, 0, 64) == 256
    assert pg.sketch_stride(pg.SK_1HASH, 0, 30) == 128
    # storage budget s of the CSR bytes (Sec. V-A): R-MAT scale 24 / ef 32 at 25% and 50%
    n, nnz = 1 << 24, 1_023_887_446
    assert pg.bloom_bits_for_budget(0.25, n, nnz) == 448
    assert pg.bloom_bits_for_budget(0.50, n, nnz) == 960
    assert pg.bloom_bits_for_budget(0.25, 4096, 65536) == 128  # 136 bits -> one 64-bit word less
    assert L.pg_edge_index_bytes(0, 0) > 0
    assert L.pg_edge_index_bytes(10, 100) >= 4 * 11 + 8 * 50


def _csr(n=4, nnz=6, rp=0x1000, col=0x2000):
    from paper_2208_11469_gb300 import pg
    return pg.Csr(rp, col, n, nnz)


def test_argument_errors_return_codes(L):
    from paper_2208_11469_gb300 import pg
    byref = ctypes.byref
    # NULL graph
    assert L.pg_build_edge_index(None, ctypes.c_void_p(0x1000), 1 << 20, None) == -1
    # nnz beyond int32 CSR
    g = _csr(nnz=1 << 31)
    assert L.pg_build_edge_index(byref(g), ctypes.c_void_p(0x1000), 1 << 20, None) == -3
    assert b"int32" in L.pg_last_error()
    # index buffer too small
    g = _csr()
    assert L.pg_build_edge_index(byref(g), ctypes.c_void_p(0x1000), 4, None) == -4
    # misaligned sketch data / bad parameters
    sk = pg.SketchDesc(pg.SK_BLOOM, 100, 2, 0, 1, 4, 16, 0x3000)
    assert L.pg_build_bloom(byref(g), byref(sk), ctypes.c_void_p(0x4000), 1 << 20, None) == -1
    sk = pg.SketchDesc(pg.SK_BLOOM, 2048, 2, 0, 1, 4, 256, 0x3000)
    assert L.pg_build_bloom(byref(g), byref(sk), ctypes.c_void_p(0x4000), 1 << 20, None) == -9
    sk = pg.SketchDesc(pg.SK_BLOOM, 256, 2, 0, 1, 4, 32, 0x3008)
    assert L.pg_build_bloom(byref(g), byref(sk), ctypes.c_void_p(0x4000), 1 << 20, None) == -1
    sk = pg.SketchDesc(pg.SK_BLOOM, 256, 2, 0, 1, 5, 32, 0x3000)  # rows != n
    assert L.pg_build_bloom(byref(g), byref(sk), ctypes.c_void_p(0x4000), 1 << 20, None) == -1
    sk = pg.SketchDesc(pg.SK_1HASH, 0, 0, 64, 1, 4, 256, 0x3000)  # 1-Hash k > 32
    assert L.pg_build_minhash(byref(g), byref(sk), ctypes.c_void_p(0x4000), 1 << 20, None) == -9
    # estimator / sketch mismatch
    sk = pg.SketchDesc(pg.SK_KHASH, 0, 0, 16, 1, 4, 64, 0x3000)
    out = ctypes.c_void_p(0x5000)
    assert L.pg_triangle_count(byref(g), ctypes.c_void_p(0x6000), byref(sk), pg.EST_BF_AND,
                               ctypes.c_void_p(0x7000), 1 << 20, out, None) == -1
    # workspace too small
    need = L.pg_workspace_bytes(byref(g), byref(sk), pg.EST_KH)
    assert need > 0
    assert L.pg_triangle_count(byref(g), ctypes.c_void_p(0x6000), byref(sk), pg.EST_KH,
                               ctypes.c_void_p(0x7000), need - 1, out, None) == -4
    # missing edge index
    assert L.pg_triangle_count(byref(g), None, byref(sk), pg.EST_KH,
                               ctypes.c_void_p(0x7000), need, out, None) == -1
    # unknown estimator
    assert L.pg_triangle_count(byref(g), ctypes.c_void_p(0x6000), byref(sk), 42,
                               ctypes.c_void_p(0x7000), need, out, None) == -1
    # KMV reads 1-Hash rows; its totals need two more histogram bins than 1-Hash
    assert L.pg_triangle_count(byref(g), ctypes.c_void_p(0x6000), byref(sk), pg.EST_1H_KMV,
                               ctypes.c_void_p(0x7000), need, out, None) == -1
    sk1 = pg.SketchDesc(pg.SK_1HASH, 0, 0, 16, 1, 4, 64, 0x3000)
    assert L.pg_hist_bins(byref(sk1), pg.EST_1H_KMV) == L.pg_hist_bins(byref(sk1), pg.EST_1H) + 2
    # odd pairs pointer
    assert L.pg_jaccard_pairs(byref(g), None, byref(sk), pg.EST_KH, ctypes.c_void_p(0x8004), 3,
                              ctypes.c_void_p(0x7000), need, None, None, None) == -1


def test_sketch_file_header_errors(tmp_path):
    """pg_sketch_load_header is host-only: a missing file, a file that is not
    a sketch and a truncated header are refused with the documented codes."""
    import ctypes
    from paper_2208_11469_gb300 import pg
    L = pg.lib()
    d = pg.SketchDesc()
    assert L.pg_sketch_load_header(str(tmp_path / "none.pgs").encode(), ctypes.byref(d)) == -7
    bad = tmp_path / "bad.pgs"
    bad.write_bytes(b"NOTASKETCH" + bytes(100))
    assert L.pg_sketch_load_header(str(bad).encode(), ctypes.byref(d)) == -1
    short = tmp_path / "short.pgs"
    short.write_bytes(b"PGSKTCH1" + bytes(10))
    assert L.pg_sketch_load_header(str(short).encode(), ctypes.byref(d)) == -1
    # a well-formed header (as pg_sketch_save writes it) is read back field by field
    import struct
    good = tmp_path / "good.pgs"
    good.write_bytes(struct.pack("<8siiIIIIiiqq8s", b"PGSKTCH1", 1, 1, 448, 2, 0, 7, 3, 0, 64, 192, bytes(8)))
    assert L.pg_sketch_load_header(str(good).encode(), ctypes.byref(d)) == 0
    assert (d.kind, d.bits, d.b, d.k, d.seed, d.n, d.stride_bytes) == (1, 448, 2, 0, 7, 3, 64)


def test_upload_and_host_run_argument_errors(L):
    """pg_upload_build and pg_batch_run_host check their host-side arguments
    before any CUDA call: a NULL batch or host CSR, host offsets that do not
    run from 0 to nnz, a non-positive chunk size, a bad sketch and a small
    build workspace are refused with their codes."""
    import numpy as np
    from paper_2208_11469_gb300 import pg
    byref = ctypes.byref
    g = _csr(n=4, nnz=6)
    rp = np.array([0, 2, 3, 5, 6], dtype=np.int32)
    cl = np.array([1, 2, 0, 0, 3, 2], dtype=np.int32)
    vp = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    sk = (pg.SketchDesc * 1)(pg.SketchDesc(pg.SK_BLOOM, 256, 2, 0, 1, 4, 32, 0x3000))
    ws_need = L.pg_build_workspace_bytes(byref(g))

    def up(rp_, cl_, sks, count, ws_bytes=ws_need, chunk=2):
        return L.pg_upload_build(rp_, cl_, byref(g), sks, count, ctypes.c_void_p(0x4000), ws_bytes, chunk, None,
                                 None)

    assert up(None, vp(cl), sk, 1) == -1
    assert up(vp(rp), None, sk, 1) == -1
    bad = rp.copy()
    bad[-1] = 7  # does not end at nnz
    assert up(vp(bad), vp(cl), sk, 1) == -1
    assert "0 to nnz" in L.pg_last_error().decode()
    assert up(vp(rp), vp(cl), sk, 1, chunk=0) == -1
    assert up(vp(rp), vp(cl), sk, 1, ws_bytes=ws_need - 1 if ws_need > 0 else 0) in (-1, -4)
    wrong = (pg.SketchDesc * 1)(pg.SketchDesc(pg.SK_BLOOM, 256, 2, 0, 1, 5, 32, 0x3000))  # rows != n
    assert up(vp(rp), vp(cl), wrong, 1) == -1
    assert up(vp(rp), vp(cl), None, 1) == -1
    assert L.pg_batch_run_host(None, vp(rp), vp(cl), 16, None, None) == -1
