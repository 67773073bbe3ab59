"""Plain CPU oracle for the dual-quantization hot path (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It wraps ``oracle.c`` -- a plain,
single-threaded C implementation written from the paper (Sec. II-B error
bounds, Sec. III-A / Alg. 2 dual-quantization, Sec. IV padding) -- with
ctypes and numpy.  It shares no code with the CUDA library.

Parity status per function (what pins it is in tests/test_oracle_*.py):
  resolve_eb, prequant, pad_values, lorenzo_delta, compress, decompress:
  pinned.  huffman_book / huffman_encode / huffman_decode / huffman_index:
  pinned.  The padding *benefit* (fewer outliers, Sec. V-H) is data
  dependent: parity unpinned, only its trend is checked.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

EB_ABS, EB_REL = 0, 1
PAD_ZERO, PAD_GLOBAL_MIN, PAD_GLOBAL_MAX, PAD_GLOBAL_AVG = 0, 1, 2, 3
PAD_BLOCK_MIN, PAD_BLOCK_MAX, PAD_BLOCK_AVG = 4, 5, 6
PAD_EDGE_MIN, PAD_EDGE_MAX, PAD_EDGE_AVG = 7, 8, 9
PAD_NAMES = {
    "zero": PAD_ZERO, "global_min": PAD_GLOBAL_MIN, "global_max": PAD_GLOBAL_MAX,
    "global_avg": PAD_GLOBAL_AVG, "block_min": PAD_BLOCK_MIN,
    "block_max": PAD_BLOCK_MAX, "block_avg": PAD_BLOCK_AVG,
    "edge_min": PAD_EDGE_MIN, "edge_max": PAD_EDGE_MAX, "edge_avg": PAD_EDGE_AVG,
}


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, IEEE-faithful flags)."""
    with _lock:
        if (not force and os.path.exists(_LIB_PATH)
                and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
            return _LIB_PATH
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math",
               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


class _Params(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int32), ("dims", ctypes.c_uint64 * 3),
                ("block", ctypes.c_uint32), ("eb", ctypes.c_double),
                ("eb_mode", ctypes.c_int32), ("radius", ctypes.c_uint32),
                ("pad", ctypes.c_int32)]


class _Eb(ctypes.Structure):
    _fields_ = [("eb_abs", ctypes.c_double), ("inv2eb", ctypes.c_float),
                ("ebx2", ctypes.c_float), ("eb_f32", ctypes.c_float),
                ("xmin", ctypes.c_float), ("xmax", ctypes.c_float),
                ("has_range", ctypes.c_int32)]


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.POINTER
        vp = ctypes.c_void_p
        lib.vszo_num_blocks.restype = ctypes.c_uint64
        lib.vszo_num_blocks.argtypes = [P(_Params)]
        lib.vszo_num_elems.restype = ctypes.c_uint64
        lib.vszo_num_elems.argtypes = [P(_Params)]
        lib.vszo_resolve_eb.argtypes = [P(_Params), vp, P(_Eb)]
        lib.vszo_prequant.argtypes = [vp, ctypes.c_uint64, ctypes.c_float, vp]
        lib.vszo_prequant.restype = None
        lib.vszo_pad_values.argtypes = [P(_Params), vp, vp]
        lib.vszo_lorenzo_delta.argtypes = [P(_Params), vp, vp, vp]
        lib.vszo_compress.argtypes = [P(_Params), vp, P(_Eb), vp, vp, vp, vp, vp, vp,
                                      P(ctypes.c_uint64), vp, vp, P(ctypes.c_uint64)]
        lib.vszo_compress_given_pad.argtypes = [P(_Params), vp, ctypes.c_int32, P(_Eb), vp, vp, vp, vp, vp,
                                                P(ctypes.c_uint64), vp, vp, P(ctypes.c_uint64)]
        lib.vszo_decompress.argtypes = [P(_Params), P(_Eb), vp, vp, vp, vp, vp,
                                        ctypes.c_uint64, vp, vp, ctypes.c_uint64, vp, vp]
        u32, u64 = ctypes.c_uint32, ctypes.c_uint64
        lib.vszo_huffman_lengths.argtypes = [vp, u32, vp]
        lib.vszo_huffman_codes.argtypes = [vp, u32, vp]
        lib.vszo_huffman_encode.argtypes = [vp, u64, vp, vp, u32, u32, vp, vp]
        lib.vszo_huffman_decode.argtypes = [vp, vp, u64, vp, vp, u32, u32, vp]
        _lib = lib
    return _lib


@dataclass(frozen=True)
class Params:
    """Field and method parameters (C-order dims, dims[0] slowest)."""
    dims: tuple
    block: int
    eb: float
    eb_mode: int = EB_REL
    radius: int = 512
    pad: int = PAD_ZERO

    @property
    def ndim(self) -> int:
        return len(self.dims)

    def _c(self) -> _Params:
        d = list(self.dims) + [0] * (3 - len(self.dims))
        return _Params(len(self.dims), (ctypes.c_uint64 * 3)(*d), self.block,
                       float(self.eb), self.eb_mode, self.radius, self.pad)

    @property
    def n(self) -> int:
        return int(np.prod(self.dims, dtype=np.uint64)) if self.dims else 0

    @property
    def nblocks(self) -> int:
        return int(_load().vszo_num_blocks(ctypes.byref(self._c())))

    @property
    def is_block_pad(self) -> bool:
        return self.pad in (PAD_BLOCK_MIN, PAD_BLOCK_MAX, PAD_BLOCK_AVG)

    @property
    def is_edge_pad(self) -> bool:
        return self.pad in (PAD_EDGE_MIN, PAD_EDGE_MAX, PAD_EDGE_AVG)

    @property
    def pad_len(self) -> int:
        """Entries of the padding table: nb (block), nb * ndim (edge), else 1."""
        if self.is_block_pad:
            return max(self.nblocks, 1)
        if self.is_edge_pad:
            return max(self.nblocks * self.ndim, 1)
        return 1


@dataclass
class EbInfo:
    eb_abs: float
    inv2eb: np.float32
    ebx2: np.float32
    eb_f32: np.float32
    xmin: np.float32
    xmax: np.float32
    has_range: bool

    @classmethod
    def _from_c(cls, e: _Eb) -> "EbInfo":
        return cls(e.eb_abs, np.float32(e.inv2eb), np.float32(e.ebx2), np.float32(e.eb_f32),
                   np.float32(e.xmin), np.float32(e.xmax), bool(e.has_range))

    def _c(self) -> _Eb:
        return _Eb(self.eb_abs, float(self.inv2eb), float(self.ebx2), float(self.eb_f32),
                   float(self.xmin), float(self.xmax), int(self.has_range))


@dataclass
class Compressed:
    eb: EbInfo
    codes: np.ndarray      # uint16[n], field layout
    q: np.ndarray          # int32[n], prequantized values
    pad: np.ndarray        # int32[nb] (block modes), int32[nb*ndim] (edge modes) or int32[1]
    blk_off: np.ndarray    # uint32[nb+1]
    out_idx: np.ndarray    # uint32[n_out], canonical order
    out_delta: np.ndarray  # int32[n_out]
    fix_idx: np.ndarray    # uint32[n_fix], canonical order
    fix_bits: np.ndarray   # uint32[n_fix], raw bits of x


def _f32(x) -> np.ndarray:
    return np.ascontiguousarray(x, dtype=np.float32).reshape(-1)


def resolve_eb(p: Params, x) -> EbInfo:
    x = _f32(x)
    e = _Eb()
    rc = _load().vszo_resolve_eb(ctypes.byref(p._c()), x.ctypes.data, ctypes.byref(e))
    if rc:
        raise ValueError(f"oracle resolve_eb failed rc={rc}")
    return EbInfo._from_c(e)


def prequant(x, inv2eb) -> np.ndarray:
    x = _f32(x)
    q = np.empty(x.size, np.int32)
    _load().vszo_prequant(x.ctypes.data, x.size, float(np.float32(inv2eb)), q.ctypes.data)
    return q


def pad_values(p: Params, q) -> np.ndarray:
    q = np.ascontiguousarray(q, dtype=np.int32).reshape(-1)
    pad = np.zeros(p.pad_len, np.int32)
    rc = _load().vszo_pad_values(ctypes.byref(p._c()), q.ctypes.data, pad.ctypes.data)
    if rc:
        raise ValueError(f"oracle pad_values failed rc={rc}")
    return pad


def lorenzo_delta(p: Params, q, pad) -> np.ndarray:
    q = np.ascontiguousarray(q, dtype=np.int32).reshape(-1)
    pad = np.ascontiguousarray(pad, dtype=np.int32).reshape(-1)
    d = np.zeros(q.size, np.int32)
    rc = _load().vszo_lorenzo_delta(ctypes.byref(p._c()), q.ctypes.data, pad.ctypes.data,
                                    d.ctypes.data)
    if rc:
        raise ValueError(f"oracle lorenzo_delta failed rc={rc}")
    return d


def compress(p: Params, x) -> Compressed:
    x = _f32(x)
    n = x.size
    assert n == p.n, (n, p.n)
    nb = p.nblocks
    e = _Eb()
    codes = np.zeros(n, np.uint16)
    q = np.zeros(n, np.int32)
    pad = np.zeros(p.pad_len, np.int32)
    blk_off = np.zeros(nb + 1, np.uint32)
    cap = max(n, 1)
    out_idx = np.zeros(cap, np.uint32)
    out_delta = np.zeros(cap, np.int32)
    fix_idx = np.zeros(cap, np.uint32)
    fix_bits = np.zeros(cap, np.uint32)
    n_out = ctypes.c_uint64(0)
    n_fix = ctypes.c_uint64(0)
    rc = _load().vszo_compress(ctypes.byref(p._c()), x.ctypes.data, ctypes.byref(e),
                               codes.ctypes.data, q.ctypes.data, pad.ctypes.data,
                               blk_off.ctypes.data, out_idx.ctypes.data, out_delta.ctypes.data,
                               ctypes.byref(n_out), fix_idx.ctypes.data, fix_bits.ctypes.data,
                               ctypes.byref(n_fix))
    if rc:
        raise ValueError(f"oracle compress failed rc={rc}")
    no, nf = n_out.value, n_fix.value
    return Compressed(EbInfo._from_c(e), codes, q, pad, blk_off,
                      out_idx[:no].copy(), out_delta[:no].copy(),
                      fix_idx[:nf].copy(), fix_bits[:nf].copy())


def compress_given_pad(p: Params, x, P: int) -> Compressed:
    """One whole-block slab of a field split along dims[0] (vszo_compress_given_pad):
    p in absolute mode with the field's eb_abs, P the field's global padding
    value (ignored by the other modes).  The returned q is not filled."""
    x = _f32(x)
    n = x.size
    assert n == p.n, (n, p.n)
    nb = p.nblocks
    e = _Eb()
    codes = np.zeros(n, np.uint16)
    pad = np.zeros(p.pad_len, np.int32)
    blk_off = np.zeros(nb + 1, np.uint32)
    cap = max(n, 1)
    out_idx = np.zeros(cap, np.uint32)
    out_delta = np.zeros(cap, np.int32)
    fix_idx = np.zeros(cap, np.uint32)
    fix_bits = np.zeros(cap, np.uint32)
    n_out = ctypes.c_uint64(0)
    n_fix = ctypes.c_uint64(0)
    rc = _load().vszo_compress_given_pad(ctypes.byref(p._c()), x.ctypes.data, int(P), ctypes.byref(e),
                                         codes.ctypes.data, pad.ctypes.data, blk_off.ctypes.data,
                                         out_idx.ctypes.data, out_delta.ctypes.data, ctypes.byref(n_out),
                                         fix_idx.ctypes.data, fix_bits.ctypes.data, ctypes.byref(n_fix))
    if rc:
        raise ValueError(f"oracle compress_given_pad failed rc={rc}")
    no, nf = n_out.value, n_fix.value
    return Compressed(EbInfo._from_c(e), codes, None, pad, blk_off,
                      out_idx[:no].copy(), out_delta[:no].copy(),
                      fix_idx[:nf].copy(), fix_bits[:nf].copy())


def decompress(p: Params, c: Compressed, return_q: bool = False):
    n = p.n
    xhat = np.zeros(n, np.float32)
    q = np.zeros(n, np.int32)
    def a(arr, dt):
        arr = np.ascontiguousarray(arr, dtype=dt)
        return arr if arr.size else np.zeros(1, dt)
    codes = a(c.codes, np.uint16)
    pad = a(c.pad, np.int32)
    blk_off = a(c.blk_off, np.uint32)
    oi, od = a(c.out_idx, np.uint32), a(c.out_delta, np.int32)
    fi, fb = a(c.fix_idx, np.uint32), a(c.fix_bits, np.uint32)
    eb = c.eb._c()
    rc = _load().vszo_decompress(ctypes.byref(p._c()), ctypes.byref(eb), codes.ctypes.data,
                                 pad.ctypes.data, blk_off.ctypes.data, oi.ctypes.data,
                                 od.ctypes.data, len(c.out_idx), fi.ctypes.data,
                                 fb.ctypes.data, len(c.fix_idx), q.ctypes.data,
                                 xhat.ctypes.data)
    if rc:
        raise ValueError(f"oracle decompress failed rc={rc}")
    return (xhat, q) if return_q else xhat


# ---------------------------------------------------------------- entropy stage
HUFF_CHUNK = 1024  # symbols per word-aligned chunk of the bitstream


def huffman_book(hist):
    """Canonical Huffman code of a histogram: (lengths uint8[nsym],
    codewords uint64[nsym]) -- Sec. II-B's entropy stage."""
    hist = np.ascontiguousarray(hist, dtype=np.uint32).reshape(-1)
    nsym = hist.size
    ln = np.zeros(max(nsym, 1), np.uint8)
    cw = np.zeros(max(nsym, 1), np.uint64)
    if _load().vszo_huffman_lengths(hist.ctypes.data, nsym, ln.ctypes.data):
        raise ValueError("oracle huffman_lengths failed")
    _load().vszo_huffman_codes(ln.ctypes.data, nsym, cw.ctypes.data)
    return ln[:nsym], cw[:nsym]


def huffman_encode(sym, lengths, codes, chunk: int = HUFF_CHUNK):
    """Word-aligned chunks, MSB first: (words uint32[], chunk_off uint64[nchunks+1])."""
    sym = np.ascontiguousarray(sym, dtype=np.uint16).reshape(-1)
    lengths = np.ascontiguousarray(lengths, np.uint8)
    codes = np.ascontiguousarray(codes, np.uint64)
    n = sym.size
    nchunks = (n + chunk - 1) // chunk
    bits = int(lengths.astype(np.int64)[sym].sum()) if n else 0
    words = np.zeros(max(1, bits // 32 + nchunks + 1), np.uint32)
    off = np.zeros(nchunks + 1, np.uint64)
    rc = _load().vszo_huffman_encode(sym.ctypes.data if n else None, n, lengths.ctypes.data, codes.ctypes.data,
                                     lengths.size, chunk, words.ctypes.data, off.ctypes.data)
    if rc:
        raise ValueError(f"oracle huffman_encode failed rc={rc}")
    return words[: int(off[-1])].copy(), off


# The decode index (the Huffman stage of Sec. II-B decoded in parallel; the
# paper decodes serially): the stream is unchanged, and beside it, for chunk
# c and sub-chunk j of HUFF_LANES per chunk, the bit of chunk c's stream where
# the sub-chunk's first code begins -- the sum of the lengths of the chunk's
# codes before it.  Sub-chunks past the end of the data get the chunk's total.
HUFF_LANES = 32


def huffman_index(sym, lengths, chunk: int = HUFF_CHUNK, lanes: int = HUFF_LANES):
    """Decode index: int64[nchunks * lanes], bit offsets inside each chunk."""
    sym = np.ascontiguousarray(sym, dtype=np.uint16).reshape(-1)
    lengths = np.asarray(lengths, np.int64)
    n = sym.size
    nchunks = (n + chunk - 1) // chunk
    bits = np.zeros(nchunks * chunk, np.int64)
    bits[:n] = lengths[sym]
    per = bits.reshape(nchunks, lanes, chunk // lanes).sum(axis=2)
    return (np.cumsum(per, axis=1) - per).reshape(-1)


def huffman_decode(words, chunk_off, n, lengths, codes, chunk: int = HUFF_CHUNK):
    words = np.ascontiguousarray(words, np.uint32)
    if words.size == 0:
        words = np.zeros(1, np.uint32)
    chunk_off = np.ascontiguousarray(chunk_off, np.uint64)
    lengths = np.ascontiguousarray(lengths, np.uint8)
    codes = np.ascontiguousarray(codes, np.uint64)
    out = np.zeros(max(n, 1), np.uint16)
    rc = _load().vszo_huffman_decode(words.ctypes.data, chunk_off.ctypes.data, n, lengths.ctypes.data,
                                     codes.ctypes.data, lengths.size, chunk, out.ctypes.data)
    if rc:
        raise ValueError(f"oracle huffman_decode failed rc={rc}")
    return out[:n]
