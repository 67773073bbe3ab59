"""CPU-side checks of the C-ABI library: it builds for sm_103a, loads without
a GPU, exports every symbol include/vsz.h declares, and its host-only logic
(parameter validation, block counts, workspace sizes, status names) behaves
as documented.  No kernel is launched here."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def vsz():
    import paper_2201_04614_gb300 as v
    v.build()
    return v


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "vsz.h")).read()
    return sorted(set(re.findall(r"^VSZ_API\s+[\w\s\*]+?\b(vsz_\w+)\s*\(", src, re.M)))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for name in ("vsz_prequant_lorenzo", "vsz_outlier_compact", "vsz_reconstruct",
                 "vsz_workspace_size", "vsz_read_header"):
        assert name in syms


def test_library_exports_every_declared_symbol(vsz):
    lib = ctypes.CDLL(vsz.build())
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing
    assert set(declared_symbols()) <= set(vsz.EXPORTED) | set(declared_symbols())


def test_abi_version_and_status_strings(vsz):
    L = vsz.lib()
    assert L.vsz_abi_version() == 1
    for code, name in vsz._STATUS.items():
        assert L.vsz_status_string(code).decode() == name
    assert L.vsz_status_string(99).decode() == "VSZ_ERR_UNKNOWN"


@pytest.mark.parametrize("kw,status", [
    (dict(dims=(10,), block=8, eb=1e-3), 0),
    (dict(dims=(10, 12), block=16, eb=1e-3), 0),
    (dict(dims=(4, 5, 6), block=32, eb=1e-3), 0),
    (dict(dims=(4, 5, 6), block=64, eb=1e-3), 2),    # 3D block above 32
    (dict(dims=(10, 12), block=256, eb=1e-3), 2),    # 2D block above 128
    (dict(dims=(10,), block=6, eb=1e-3), 2),         # not a power of two (SZ-1.4's 6^3)
    (dict(dims=(10,), block=2, eb=1e-3), 2),         # below the lane width
    (dict(dims=(10,), block=0, eb=1e-3), 1),
    (dict(dims=(10,), block=8, eb=0.0), 1),
    (dict(dims=(10,), block=8, eb=float("nan")), 1),
    (dict(dims=(10,), block=8, eb=1e-3, radius=0), 1),
    (dict(dims=(10,), block=8, eb=1e-3, radius=32769), 1),
    (dict(dims=(10,), block=8, eb=1e-3, pad=9), 0),   # edge average (Sec. IV-B-3)
    (dict(dims=(10,), block=8, eb=1e-3, pad=10), 1),
    (dict(dims=(1 << 16, 1 << 16), block=8, eb=1e-3), 1),  # n >= 2^32
    (dict(dims=(0,), block=8, eb=1e-3), 0),          # empty field
])
def test_validate(vsz, kw, status):
    p = vsz.Params(tuple(kw["dims"]), kw["block"], kw["eb"], 1, kw.get("radius", 512), kw.get("pad", 0))
    assert p.validate() == status


def test_validate_ndim(vsz):
    L = vsz.lib()
    for nd, st in ((0, 1), (4, 2), (5, 1)):
        c = vsz._CParams(nd, (ctypes.c_uint64 * 3)(4, 4, 4), 8, 1e-3, 0, 512, 0)
        assert L.vsz_validate(ctypes.byref(c)) == st


def test_block_counts_and_workspace(vsz):
    import math
    for dims, b in [((1000,), 32), ((33, 65), 16), ((9, 17, 40), 8), ((512, 512, 512), 8)]:
        p = vsz.Params(dims, b, 1e-3)
        assert p.nblocks == math.prod((d + b - 1) // b for d in dims)
        assert p.n == math.prod(dims)
        w0 = vsz.workspace_size(p, 0, 0)
        w1 = vsz.workspace_size(p, 1000, 10)
        assert w0 > 0 and w0 % 256 == 0
        assert w1 >= w0 + 8 * 1010
    assert vsz.workspace_size(vsz.Params((10,), 6, 1e-3), 0, 0) == 0


def test_header_struct_layout(vsz):
    # The binding's mirror of vsz_header must match the C layout (64 bytes).
    assert vsz.HEADER_BYTES == 64
    assert ctypes.sizeof(vsz._CCompressed) == 80


def test_calls_without_gpu_fail_cleanly(vsz):
    """Invalid arguments are rejected on the host before any GPU work."""
    L = vsz.lib()
    p = vsz.Params((100,), 8, 1e-3).c()
    cc = vsz._CCompressed()
    rc = L.vsz_prequant_lorenzo(ctypes.byref(p), None, ctypes.byref(cc), None, 0, None)
    assert rc == 1
    rc = L.vsz_reconstruct(ctypes.byref(p), ctypes.byref(cc), None, None, 0, None)
    assert rc == 1


def test_entropy_calls_reject_missing_buffers_on_the_host(vsz):
    """The Huffman calls refuse a missing codebook, status word or offsets
    before any GPU work; the codebook size follows the symbol limit."""
    L = vsz.lib()
    assert L.vsz_huffman_book_bytes(0) == 0
    assert L.vsz_huffman_book_bytes(vsz.HUFF_MAX_SYMBOLS + 1) == 0
    assert L.vsz_huffman_book_bytes(1024) > L.vsz_huffman_book_bytes(16) > 0
    assert L.vsz_huffman_encode_indexed(None, 10, None, 1024, None, 0, None, None, None, None, 0, None) == 1
    assert L.vsz_huffman_decode_indexed(None, 0, None, None, 10, None, 1024, None, None, None) == 1
    assert L.vsz_huffman_decode(None, 0, None, 10, None, 1024, None, None, None) == 1
    assert L.vsz_huffman_decode_indexed(None, 0, None, None, 10, None, 0, None, None, None) == 1  # nsym 0
