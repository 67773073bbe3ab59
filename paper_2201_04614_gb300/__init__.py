"""GB300 dual-quantization (the vecSZ hot path, arXiv 2201.04614).

Thin Python binding of the C ABI in include/vsz.h (libvsz.so).  It only
marshals arguments: every step of compression and reconstruction runs in the
library's CUDA kernels.  PyTorch supplies device memory and streams.  There
is no CPU fallback: without a CUDA device or the built library every call
raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

from . import buildlib as _build

__all__ = [
    "VszError", "Params", "Field", "Batch", "lib", "build", "EB_ABS", "EB_REL", "PAD_MODES",
    "num_blocks", "workspace_size", "trace_enable", "trace_read",
]

EB_ABS, EB_REL = 0, 1
PAD_MODES = {
    "zero": 0, "global_min": 1, "global_max": 2, "global_avg": 3,
    "block_min": 4, "block_max": 5, "block_avg": 6, "edge_min": 7, "edge_max": 8, "edge_avg": 9,
}
_STATUS = {0: "VSZ_OK", 1: "VSZ_ERR_INVALID_ARG", 2: "VSZ_ERR_UNSUPPORTED",
           3: "VSZ_ERR_CAPACITY", 4: "VSZ_ERR_CUDA", 5: "VSZ_ERR_CORRUPT", 6: "VSZ_ERR_TOO_LARGE"}
NOALLOC_WS_BYTES = 16 << 20  # VSZ_NOALLOC_WS_BYTES
RECON_WS_BYTES = 256         # VSZ_RECON_WS_BYTES


class VszError(RuntimeError):
    """A call of the library returned a non-zero vsz_status (`status`)."""

    def __init__(self, status: int, what: str, detail: str = ""):
        self.status = status
        super().__init__(f"{what}: {_STATUS.get(status, status)}{(' (' + detail + ')') if detail else ''}")


class _CParams(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int32), ("dims", ctypes.c_uint64 * 3), ("block", ctypes.c_uint32),
                ("eb", ctypes.c_double), ("eb_mode", ctypes.c_int32), ("radius", ctypes.c_uint32),
                ("pad", ctypes.c_int32)]


class _CHeader(ctypes.Structure):
    _fields_ = [("eb_abs", ctypes.c_double), ("inv2eb", ctypes.c_float), ("ebx2", ctypes.c_float),
                ("eb_f32", ctypes.c_float), ("xmin", ctypes.c_float), ("xmax", ctypes.c_float),
                ("pad_global", ctypes.c_int32), ("has_range", ctypes.c_uint32),
                ("status", ctypes.c_uint32), ("recon_status", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32), ("n_out", ctypes.c_uint64), ("n_fix", ctypes.c_uint64)]


class _CCompressed(ctypes.Structure):
    _fields_ = [("codes", ctypes.c_void_p), ("pad", ctypes.c_void_p), ("blk_off", ctypes.c_void_p),
                ("out_idx", ctypes.c_void_p), ("out_delta", ctypes.c_void_p), ("out_cap", ctypes.c_uint64),
                ("fix_idx", ctypes.c_void_p), ("fix_bits", ctypes.c_void_p), ("fix_cap", ctypes.c_uint64),
                ("hdr", ctypes.c_void_p)]


class _CFieldJob(ctypes.Structure):
    _fields_ = [("params", _CParams), ("d_x", ctypes.c_void_p), ("out", _CCompressed)]


class _CBatchClass(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int32), ("block", ctypes.c_uint32), ("pad_kind", ctypes.c_int32),
                ("nfields", ctypes.c_int32), ("tiles", ctypes.c_uint64), ("warps", ctypes.c_int32),
                ("ctas_per_sm", ctypes.c_int32), ("ms", ctypes.c_float), ("ms_default", ctypes.c_float),
                ("concurrent", ctypes.c_int32), ("kind", ctypes.c_int32)]


class _CHostField(ctypes.Structure):
    _fields_ = [("codes", ctypes.c_void_p), ("pad", ctypes.c_void_p), ("blk_off", ctypes.c_void_p),
                ("out_idx", ctypes.c_void_p), ("out_delta", ctypes.c_void_p), ("out_cap", ctypes.c_uint64),
                ("fix_idx", ctypes.c_void_p), ("fix_bits", ctypes.c_void_p), ("fix_cap", ctypes.c_uint64),
                ("hdr", ctypes.c_void_p)]


class _CTrace(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 24), ("ndim", ctypes.c_int32), ("block", ctypes.c_uint32),
                ("n", ctypes.c_uint64), ("ms", ctypes.c_float), ("reserved", ctypes.c_uint32)]


HEADER_BYTES = ctypes.sizeof(_CHeader)
EXPORTED = ["vsz_status_string", "vsz_last_cuda_error", "vsz_abi_version", "vsz_validate",
            "vsz_num_elems", "vsz_num_blocks", "vsz_workspace_size", "vsz_workspace_size_dense", "vsz_prequant_lorenzo",
            "vsz_outlier_compact", "vsz_compress", "vsz_reconstruct", "vsz_reconstruct_q",
            "vsz_code_histogram", "vsz_read_header", "vsz_trace_enable", "vsz_trace_read",
            "vsz_compress_noalloc", "vsz_batch_workspace_size", "vsz_batch_create", "vsz_batch_submit",
            "vsz_batch_destroy", "vsz_batch_num_classes", "vsz_batch_get_class", "vsz_batch_set_shape",
            "vsz_batch_set_concurrent", "vsz_batch_set_concurrent_each", "vsz_batch_autotune", "vsz_batch_set_outputs",
            "vsz_batch_reconstruct",
            "vsz_batch_compress_host", "vsz_slab_range", "vsz_slab_qstats", "vsz_compress_slab", "vsz_slab_rebase",
            "vsz_huffman_book_bytes", "vsz_huffman_book", "vsz_huffman_book_read", "vsz_huffman_encode",
            "vsz_huffman_encode_workspace_size", "vsz_sampling_autotune_workspace_size", "vsz_sampling_autotune",
            "vsz_sync_status", "vsz_shutdown", "vsz_debug_fail_alloc", "vsz_debug_bounds_word",
            "vsz_huffman_decode", "vsz_huffman_encode_indexed", "vsz_huffman_decode_indexed",
            "vsz_tuner_features_workspace_size", "vsz_tuner_features",
            "vsz_tuner_sweep_workspace_size", "vsz_tuner_sweep", "vsz_tuner_guard_workspace_size",
            "vsz_tuner_guard", "vsz_tuner_guard_sample_dims", "vsz_mlp_forward", "vsz_mlp_grad_workspace_size",
            "vsz_mlp_grad", "vsz_mlp_adam"]

_lib = None


def build(force: bool = False) -> str:
    """Compile libvsz.so in-tree for sm_103a (nvcc) if its sources changed; its path."""
    return _build.build(force=force)


def lib():
    """Load libvsz.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = os.environ.get("VSZ_LIBRARY") or _build.LIB_PATH  # a variant build (tile-shape experiments)
    if path == _build.LIB_PATH and (not os.path.exists(path) or _build.is_stale()):
        _build.build()
    L = ctypes.CDLL(path)
    P = ctypes.POINTER
    vp, u64, sz = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_size_t
    L.vsz_status_string.restype = ctypes.c_char_p
    L.vsz_status_string.argtypes = [ctypes.c_int]
    L.vsz_last_cuda_error.restype = ctypes.c_char_p
    L.vsz_last_cuda_error.argtypes = []
    L.vsz_abi_version.restype = ctypes.c_int
    L.vsz_validate.argtypes = [P(_CParams)]
    L.vsz_num_elems.restype = u64
    L.vsz_num_elems.argtypes = [P(_CParams)]
    L.vsz_num_blocks.restype = u64
    L.vsz_num_blocks.argtypes = [P(_CParams)]
    L.vsz_workspace_size.restype = sz
    L.vsz_workspace_size.argtypes = [P(_CParams), u64, u64]
    L.vsz_workspace_size_dense.restype = sz
    L.vsz_workspace_size_dense.argtypes = [P(_CParams), u64, u64]
    for name in ("vsz_prequant_lorenzo", "vsz_compress"):
        getattr(L, name).argtypes = [P(_CParams), vp, P(_CCompressed), vp, sz, vp]
    L.vsz_outlier_compact.argtypes = [P(_CParams), P(_CCompressed), vp, sz, vp]
    L.vsz_compress_noalloc.argtypes = [P(_CParams), vp, P(_CCompressed), vp]
    L.vsz_reconstruct.argtypes = [P(_CParams), P(_CCompressed), vp, vp, sz, vp]
    L.vsz_reconstruct_q.argtypes = [P(_CParams), P(_CCompressed), vp, vp, sz, vp]
    L.vsz_code_histogram.argtypes = [P(_CParams), vp, vp, vp]
    L.vsz_read_header.argtypes = [P(_CCompressed), P(_CHeader), vp]
    L.vsz_sync_status.argtypes = [P(_CCompressed), vp]
    L.vsz_batch_workspace_size.restype = sz
    L.vsz_batch_workspace_size.argtypes = [P(_CFieldJob), ctypes.c_int]
    L.vsz_batch_create.argtypes = [P(_CFieldJob), ctypes.c_int, vp, sz, ctypes.c_int, P(ctypes.c_void_p)]
    L.vsz_batch_submit.argtypes = [vp, vp]
    L.vsz_batch_destroy.argtypes = [vp]
    L.vsz_batch_num_classes.argtypes = [vp]
    L.vsz_batch_get_class.argtypes = [vp, ctypes.c_int, P(_CBatchClass)]
    L.vsz_batch_set_shape.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    L.vsz_batch_set_concurrent.argtypes = [vp, ctypes.c_int]
    L.vsz_batch_set_concurrent_each.argtypes = [vp, ctypes.c_int, ctypes.c_int]
    L.vsz_batch_autotune.argtypes = [vp, vp, ctypes.c_int]
    L.vsz_batch_set_outputs.argtypes = [vp, P(ctypes.c_void_p)]
    L.vsz_huffman_book_bytes.restype = sz
    L.vsz_huffman_book_bytes.argtypes = [ctypes.c_uint32]
    L.vsz_huffman_book.argtypes = [vp, ctypes.c_uint32, vp, sz, vp]
    L.vsz_huffman_book_read.argtypes = [vp, ctypes.c_uint32, vp, vp, P(ctypes.c_uint32), vp]
    L.vsz_huffman_encode_workspace_size.restype = sz
    L.vsz_huffman_encode_workspace_size.argtypes = [u64]
    L.vsz_huffman_encode.argtypes = [vp, u64, vp, ctypes.c_uint32, vp, u64, vp, vp, vp, sz, vp]
    L.vsz_huffman_decode.argtypes = [vp, u64, vp, u64, vp, ctypes.c_uint32, vp, vp, vp]
    L.vsz_huffman_encode_indexed.argtypes = [vp, u64, vp, ctypes.c_uint32, vp, u64, vp, vp, vp, vp, sz, vp]
    L.vsz_huffman_decode_indexed.argtypes = [vp, u64, vp, vp, u64, vp, ctypes.c_uint32, vp, vp, vp]
    L.vsz_batch_reconstruct.argtypes = [vp, vp]
    L.vsz_batch_compress_host.argtypes = [vp, P(ctypes.c_void_p), P(_CHostField), vp]
    L.vsz_slab_range.argtypes = [vp, u64, vp, vp]
    L.vsz_slab_qstats.argtypes = [P(_CParams), vp, vp, vp]
    L.vsz_compress_slab.argtypes = [P(_CParams), ctypes.c_int32, vp, P(_CCompressed), vp, sz, vp]
    L.vsz_slab_rebase.argtypes = [P(_CParams), P(_CCompressed), u64, u64, vp]
    L.vsz_trace_enable.argtypes = [ctypes.c_int]
    L.vsz_debug_bounds_word.argtypes = [P(ctypes.c_uint32)]
    L.vsz_trace_read.argtypes = [P(_CTrace), ctypes.c_int]
    for name in EXPORTED:
        if name.startswith(("vsz_tuner", "vsz_mlp", "vsz_sampling")):
            continue  # bound by tuner.py
        if name not in ("vsz_status_string", "vsz_last_cuda_error", "vsz_abi_version",
                        "vsz_num_elems", "vsz_num_blocks", "vsz_workspace_size", "vsz_workspace_size_dense",
                        "vsz_batch_workspace_size",
                        "vsz_huffman_book_bytes", "vsz_huffman_encode_workspace_size"):
            getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def debug_bounds_word():
    """The first out-of-bounds site recorded by a bounds-checking build (and
    clears it); None for the normal build."""
    v = ctypes.c_uint32(0)
    rc = lib().vsz_debug_bounds_word(ctypes.byref(v))
    return None if rc == 2 else int(v.value)


def trace_enable(on: bool = True) -> None:
    """Bracket every library kernel launch with CUDA events (profiling aid)."""
    _check(lib().vsz_trace_enable(1 if on else 0), "vsz_trace_enable")


def trace_read(max_records: int = 1 << 16) -> list:
    """Wait for the traced launches and return [{name, ndim, block, n, ms}], oldest first."""
    buf = (_CTrace * max_records)()
    k = lib().vsz_trace_read(buf, max_records)
    return [{"name": r.name.decode(), "ndim": r.ndim, "block": r.block, "n": r.n, "ms": r.ms}
            for r in buf[: min(k, max_records)]]


def _check(rc: int, what: str):
    if rc != 0:
        detail = lib().vsz_last_cuda_error().decode() if rc == 4 else ""
        raise VszError(rc, what, detail)


@dataclass(frozen=True)
class Params:
    """Field dims (C-order, dims[0] slowest), block edge, error bound and its
    mode, radius R, padding mode -- the paper's statement of the problem."""
    dims: tuple
    block: int
    eb: float
    eb_mode: int = EB_REL
    radius: int = 512
    pad: int = 0

    @classmethod
    def make(cls, dims, block, eb, eb_mode="rel", radius=512, pad="zero") -> "Params":
        """The paper's statement of the problem: C-order dims, block edge, error
        bound (absolute or value-range relative, Sec. II-B), radius R of the
        codes, padding mode by name (PAD_MODES, Sec. IV)."""
        em = {"abs": EB_ABS, "rel": EB_REL}[eb_mode] if isinstance(eb_mode, str) else int(eb_mode)
        pm = PAD_MODES[pad] if isinstance(pad, str) else int(pad)
        return cls(tuple(int(d) for d in dims), int(block), float(eb), em, int(radius), pm)

    def c(self) -> _CParams:
        """The vsz_params struct of the C ABI."""
        d = list(self.dims) + [0] * (3 - len(self.dims))
        return _CParams(len(self.dims), (ctypes.c_uint64 * 3)(*d), self.block, self.eb,
                        self.eb_mode, self.radius, self.pad)

    @property
    def n(self) -> int:
        """Values in the field."""
        return int(lib().vsz_num_elems(ctypes.byref(self.c())))

    @property
    def nblocks(self) -> int:
        """Blocks of the field, partial blocks at the + edges included (Sec. III-A)."""
        return int(lib().vsz_num_blocks(ctypes.byref(self.c())))

    @property
    def is_block_pad(self) -> bool:
        """A per-block padding value (Sec. IV-B-2)."""
        return self.pad in (4, 5, 6)

    @property
    def is_edge_pad(self) -> bool:
        """Per-block and per-axis padding values (Sec. IV-B-3)."""
        return self.pad in (7, 8, 9)

    @property
    def pad_len(self) -> int:
        """Entries of the padding table: nb (block), nb * ndim (edge), 0 otherwise."""
        return self.nblocks if self.is_block_pad else self.nblocks * len(self.dims) if self.is_edge_pad else 0

    def validate(self) -> int:
        """vsz_validate: 0, or the status a call with these parameters would return."""
        return int(lib().vsz_validate(ctypes.byref(self.c())))


def num_blocks(p: Params) -> int:
    """Blocks of the field of `p`."""
    return p.nblocks


def workspace_size(p: Params, out_cap: int, fix_cap: int) -> int:
    """Bytes of the compression workspace for these list capacities (vsz_workspace_size)."""
    return int(lib().vsz_workspace_size(ctypes.byref(p.c()), out_cap, fix_cap))


def workspace_size_dense(p: Params, out_cap: int, fix_cap: int) -> int:
    """Bytes of a workspace with the dense-outlier buffers of a 2D/3D field
    (vsz_workspace_size_dense): outlier-dense tiles are then read once."""
    return int(lib().vsz_workspace_size_dense(ctypes.byref(p.c()), out_cap, fix_cap))


def _stream_handle(stream) -> ctypes.c_void_p:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t) -> ctypes.c_void_p:
    return ctypes.c_void_p(t.data_ptr() if t is not None and t.numel() > 0 else 0)


def _need(t, name: str, itemsize: int, count: int) -> None:
    """Raise unless t is a contiguous CUDA tensor of itemsize-byte elements
    holding at least count of them: the C ABI trusts the sizes it is given,
    so a short buffer must be refused here, before any call."""
    if t is None or not getattr(t, "is_cuda", False):
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.element_size() != itemsize or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous tensor of {itemsize}-byte elements")
    if t.numel() < count:
        raise ValueError(f"{name} holds {t.numel()} elements, the call needs {count}")


class Field:
    """Device buffers of one compressed field, and the calls on them.

    codes int16[n] (uint16 codes), pad int32[nb] (block padding modes),
    blk_off int32[nb+1] (uint32 offsets), out_idx/out_delta int32[out_cap],
    fix_idx/fix_bits int32[fix_cap], hdr (device vsz_header), ws (workspace).
    """

    def __init__(self, params: Params, out_cap: int | None = None, fix_cap: int | None = None,
                 device=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("paper_2201_04614_gb300 needs a CUDA device (no CPU fallback)")
        rc = params.validate()
        _check(rc, "vsz_validate")
        self.p = params
        dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        n, nb = params.n, params.nblocks
        self.n, self.nb = n, nb
        self.out_cap = int(out_cap if out_cap is not None else max(1024, n))
        self.fix_cap = int(fix_cap if fix_cap is not None else max(1024, n // 64))
        i32 = torch.int32
        self.codes = torch.empty(max(n, 1), dtype=torch.int16, device=dev)
        self.pad = torch.empty(max(params.pad_len, 1), dtype=i32, device=dev) if params.pad_len or \
            params.is_block_pad or params.is_edge_pad else None
        self.blk_off = torch.empty(nb + 1, dtype=i32, device=dev)
        self.out_idx = torch.empty(max(self.out_cap, 1), dtype=i32, device=dev)
        self.out_delta = torch.empty(max(self.out_cap, 1), dtype=i32, device=dev)
        self.fix_idx = torch.empty(max(self.fix_cap, 1), dtype=i32, device=dev)
        self.fix_bits = torch.empty(max(self.fix_cap, 1), dtype=i32, device=dev)
        self.hdr = torch.zeros((HEADER_BYTES + 7) // 8, dtype=torch.int64, device=dev)
        self.ws_bytes = workspace_size_dense(params, self.out_cap, self.fix_cap)
        self.ws = torch.empty(self.ws_bytes, dtype=torch.uint8, device=dev)
        self.rws = torch.zeros(RECON_WS_BYTES // 4, dtype=torch.int32, device=dev)
        self._cp = params.c()
        self._cc = _CCompressed(self.codes.data_ptr(), self.pad.data_ptr() if self.pad is not None else 0,
                                self.blk_off.data_ptr(), self.out_idx.data_ptr(), self.out_delta.data_ptr(),
                                self.out_cap, self.fix_idx.data_ptr(), self.fix_bits.data_ptr(),
                                self.fix_cap, self.hdr.data_ptr())

    # ---- calls through the C ABI -------------------------------------------
    def _x(self, x):
        import torch
        if not (isinstance(x, torch.Tensor) and x.is_cuda and x.dtype == torch.float32 and x.is_contiguous()):
            raise TypeError("x must be a contiguous float32 CUDA tensor")
        if x.numel() != self.n:
            raise ValueError(f"x has {x.numel()} elements, params describe {self.n}")
        return ctypes.c_void_p(x.data_ptr() if self.n else 0)

    def prequant_lorenzo(self, x, stream=None):
        """Error-bound resolution and the fused prequantization, Lorenzo
        prediction, post-quantization and guard (Sec. III-A, Alg. 2;
        vsz_prequant_lorenzo).  The outliers stay staged until
        outlier_compact."""
        _check(lib().vsz_prequant_lorenzo(ctypes.byref(self._cp), self._x(x), ctypes.byref(self._cc),
                                          _ptr(self.ws), self.ws_bytes, _stream_handle(stream)),
               "vsz_prequant_lorenzo")

    def outlier_compact(self, stream=None):
        """The outlier and fixup lists in canonical block-major order, and the
        block offsets (vsz_outlier_compact)."""
        _check(lib().vsz_outlier_compact(ctypes.byref(self._cp), ctypes.byref(self._cc), _ptr(self.ws),
                                         self.ws_bytes, _stream_handle(stream)), "vsz_outlier_compact")

    def compress(self, x, stream=None):
        """prequant_lorenzo followed by outlier_compact (vsz_compress); x a
        contiguous float32 CUDA tensor of n values."""
        _check(lib().vsz_compress(ctypes.byref(self._cp), self._x(x), ctypes.byref(self._cc), _ptr(self.ws),
                                  self.ws_bytes, _stream_handle(stream)), "vsz_compress")

    def compress_noalloc(self, x, stream=None):
        """Compression through vsz_compress_noalloc: the library's fixed
        workspace instead of self.ws (for callers that cannot allocate)."""
        _check(lib().vsz_compress_noalloc(ctypes.byref(self._cp), self._x(x), ctypes.byref(self._cc),
                                          _stream_handle(stream)), "vsz_compress_noalloc")

    def reconstruct(self, out=None, stream=None):
        """The inverse (Sec. III-A): per-block prefix sums of the residuals,
        x_hat = q * 2eb, fixups restored (vsz_reconstruct); returns x_hat."""
        import torch
        if out is None:
            out = torch.empty(max(self.n, 1), dtype=torch.float32, device=self.codes.device)
        _need(out, "out", 4, self.n)
        _check(lib().vsz_reconstruct(ctypes.byref(self._cp), ctypes.byref(self._cc), _ptr(out), _ptr(self.rws),
                                     RECON_WS_BYTES, _stream_handle(stream)), "vsz_reconstruct")
        return out[: self.n]

    def reconstruct_q(self, out=None, stream=None):
        """The inverse's prequantized integers q (vsz_reconstruct_q)."""
        import torch
        if out is None:
            out = torch.empty(max(self.n, 1), dtype=torch.int32, device=self.codes.device)
        _need(out, "out", 4, self.n)
        _check(lib().vsz_reconstruct_q(ctypes.byref(self._cp), ctypes.byref(self._cc), _ptr(out), _ptr(self.rws),
                                       RECON_WS_BYTES, _stream_handle(stream)), "vsz_reconstruct_q")
        return out[: self.n]

    def code_histogram(self, out=None, stream=None):
        """The 2R-bin histogram of the codes (vsz_code_histogram; the entropy
        stage and the tuner's labels, Sec. II-B)."""
        import torch
        if out is None:
            out = torch.empty(2 * self.p.radius, dtype=torch.int32, device=self.codes.device)
        _need(out, "out", 4, 2 * self.p.radius)
        _check(lib().vsz_code_histogram(ctypes.byref(self._cp), _ptr(self.codes), _ptr(out),
                                        _stream_handle(stream)), "vsz_code_histogram")
        return out

    def sync_status(self, stream=None) -> int:
        """The device-recorded error of this field (vsz_sync_status): 0, 3 or 5."""
        return int(lib().vsz_sync_status(ctypes.byref(self._cc), _stream_handle(stream)))

    def header(self, stream=None) -> dict:
        """The device header as a dict (resolved error bound, range, P,
        counts, status); synchronizes the stream."""
        h = _CHeader()
        _check(lib().vsz_read_header(ctypes.byref(self._cc), ctypes.byref(h), _stream_handle(stream)),
               "vsz_read_header")
        return {k: getattr(h, k) for k, _ in _CHeader._fields_}

    # ---- host copies of the results (synchronizing) ------------------------
    def to_host(self) -> dict:
        """Codes, pads, offsets, outliers and fixups as numpy arrays."""
        import numpy as np
        h = self.header()
        no, nf = int(h["n_out"]), int(h["n_fix"])
        if h["status"] != 0:
            raise VszError(int(h["status"]), "compression")
        return {
            "header": h,
            "codes": self.codes[: self.n].cpu().numpy().view(np.uint16),
            "pad": self.pad[: max(self.p.pad_len, 0)].cpu().numpy() if self.pad is not None else None,
            "blk_off": self.blk_off.cpu().numpy().view(np.uint32),
            "out_idx": self.out_idx[:no].cpu().numpy().view(np.uint32),
            "out_delta": self.out_delta[:no].cpu().numpy(),
            "fix_idx": self.fix_idx[:nf].cpu().numpy().view(np.uint32),
            "fix_bits": self.fix_bits[:nf].cpu().numpy().view(np.uint32),
        }


class Batch:
    """Many fields compressed together (vsz_batch_*): a fixed number of
    launches whatever the number of fields, optionally replayed as a CUDA
    graph.  `fields` are Field objects (their output buffers are used) and
    `xs` the matching contiguous float32 CUDA inputs; both must stay alive
    and in place while the batch exists (the plan holds their pointers)."""

    def __init__(self, fields, xs, use_graph: bool = True):
        import torch
        if len(fields) != len(xs) or not fields:
            raise ValueError("one input per field, at least one field")
        self.fields, self.xs = list(fields), list(xs)
        jobs = (_CFieldJob * len(fields))()
        for i, (f, x) in enumerate(zip(fields, xs)):
            jobs[i].params = f._cp
            jobs[i].d_x = f._x(x)
            jobs[i].out = f._cc
        self._jobs = jobs
        L = lib()
        self.ws_bytes = int(L.vsz_batch_workspace_size(jobs, len(fields)))
        if self.ws_bytes == 0:
            raise VszError(1, "vsz_batch_workspace_size")
        self.ws = torch.empty(self.ws_bytes, dtype=torch.uint8, device=fields[0].codes.device)
        h = ctypes.c_void_p()
        _check(L.vsz_batch_create(jobs, len(fields), _ptr(self.ws), self.ws_bytes, 1 if use_graph else 0,
                                  ctypes.byref(h)), "vsz_batch_create")
        self._h = h

    def submit(self, stream=None):
        """Compress every field of the plan (vsz_batch_submit)."""
        _check(lib().vsz_batch_submit(self._h, _stream_handle(stream)), "vsz_batch_submit")

    def set_outputs(self, outs):
        """One contiguous float32 CUDA output per field (vsz_batch_set_outputs);
        they must stay alive and in place while the plan uses them."""
        if len(outs) != len(self.fields):
            raise ValueError("one output per field")
        for f, o in zip(self.fields, outs):
            if f.n and (o is None or o.dtype.itemsize != 4 or not o.is_contiguous() or o.numel() < f.n):
                raise ValueError("each output must be a contiguous float32 tensor of n values")
        arr = (ctypes.c_void_p * len(outs))(*[(o.data_ptr() if o is not None and o.numel() else None) for o in outs])
        _check(lib().vsz_batch_set_outputs(self._h, arr), "vsz_batch_set_outputs")
        self.outs = list(outs)

    def reconstruct(self, stream=None):
        """Reconstruct every field into its output (vsz_batch_reconstruct)."""
        _check(lib().vsz_batch_reconstruct(self._h, _stream_handle(stream)), "vsz_batch_reconstruct")

    def host_outputs(self, caps=None) -> list:
        """Page-locked host buffers for compress_host: per field a dict of
        CPU tensors shaped like the field's device outputs; caps[i] =
        (outliers, fixups) sizes the host lists (default: the device lists'
        capacities)."""
        import torch
        outs = []
        for i, f in enumerate(self.fields):
            oc, fc = caps[i] if caps is not None else (f.out_cap, f.fix_cap)

            def pin(n, dt):
                return torch.empty(max(int(n), 1), dtype=dt).pin_memory()
            outs.append({"codes": pin(f.n, torch.int16), "blk_off": pin(f.nb + 1, torch.int32),
                         "pad": pin(f.p.pad_len, torch.int32) if f.p.pad_len else None,
                         "out_idx": pin(oc, torch.int32), "out_delta": pin(oc, torch.int32),
                         "fix_idx": pin(fc, torch.int32), "fix_bits": pin(fc, torch.int32),
                         "header": _CHeader()})
        return outs

    def compress_host(self, h_xs, h_outs, stream=None):
        """Host memory to host memory (vsz_batch_compress_host): copies each
        field's input from the CPU tensor h_xs[i] to its device input,
        compresses the batch, and copies every field's header, codes, block
        offsets, padding table and exact-length lists into h_outs[i] (from
        host_outputs()).  Blocking."""
        if len(h_xs) != len(self.fields) or len(h_outs) != len(self.fields):
            raise ValueError("one host input and one host output per field")
        xs = (ctypes.c_void_p * len(h_xs))()
        hf = (_CHostField * len(h_xs))()
        for i, (f, x, o) in enumerate(zip(self.fields, h_xs, h_outs)):
            if f.n and (x.device.type != "cpu" or x.dtype.itemsize != 4 or not x.is_contiguous()
                        or x.numel() < f.n):
                raise ValueError("each host input must be a contiguous float32 CPU tensor of n values")
            xs[i] = x.data_ptr() if f.n else None
            hf[i].codes = o["codes"].data_ptr()
            hf[i].pad = o["pad"].data_ptr() if o["pad"] is not None else None
            hf[i].blk_off = o["blk_off"].data_ptr()
            hf[i].out_idx, hf[i].out_delta = o["out_idx"].data_ptr(), o["out_delta"].data_ptr()
            hf[i].out_cap = min(int(f.out_cap), o["out_idx"].numel(), o["out_delta"].numel())
            hf[i].fix_idx, hf[i].fix_bits = o["fix_idx"].data_ptr(), o["fix_bits"].data_ptr()
            hf[i].fix_cap = min(int(f.fix_cap), o["fix_idx"].numel(), o["fix_bits"].numel())
            hf[i].hdr = ctypes.addressof(o["header"])
        _check(lib().vsz_batch_compress_host(self._h, xs, hf, _stream_handle(stream)), "vsz_batch_compress_host")
        return [{k: getattr(o["header"], k) for k, _ in _CHeader._fields_} for o in h_outs]

    def classes(self) -> list:
        """The plan's classes (rank, block, padding kind) with their launch
        shapes and the last autotune's times (vsz_batch_get_class)."""
        L = lib()
        out = []
        for c in range(L.vsz_batch_num_classes(self._h)):
            k = _CBatchClass()
            _check(L.vsz_batch_get_class(self._h, c, ctypes.byref(k)), "vsz_batch_get_class")
            out.append({f: getattr(k, f) for f, _ in _CBatchClass._fields_})
        return out

    def set_shape(self, c: int, warps: int = 0, ctas_per_sm: int = 0):
        """Launch shape of class c (0 = default); no shape changes a result."""
        _check(lib().vsz_batch_set_shape(self._h, c, warps, ctas_per_sm), "vsz_batch_set_shape")

    def set_concurrent(self, on: bool):
        """Run the class kernels of each sequence as parallel branches."""
        _check(lib().vsz_batch_set_concurrent(self._h, 1 if on else 0), "vsz_batch_set_concurrent")

    def set_concurrent_each(self, compress_on: bool, reconstruct_on: bool):
        """set_concurrent for the compression and the reconstruction sequence separately."""
        _check(lib().vsz_batch_set_concurrent_each(self._h, 1 if compress_on else 0, 1 if reconstruct_on else 0),
               "vsz_batch_set_concurrent_each")

    def concurrency(self) -> tuple:
        """(compression, reconstruction) concurrent flags of the plan."""
        cls = self.classes()
        c = any(k["concurrent"] for k in cls if k["kind"] == 0)
        r = any(k["concurrent"] for k in cls if k["kind"] == 1)
        return c, r

    def autotune(self, stream=None, reps: int = 3, cache: str | None = None) -> list:
        """Tile autotuner (vsz_batch_autotune): synchronous; returns classes().
        With `cache` (a JSON file), shapes found earlier on this GPU model for
        the same classes are applied instead of searching again, and a new
        search is recorded there."""
        if cache and self.load_shapes(cache):
            return self.classes()
        _check(lib().vsz_batch_autotune(self._h, _stream_handle(stream), reps), "vsz_batch_autotune")
        if cache:
            self.save_shapes(cache)
        return self.classes()

    @staticmethod
    def _device_key() -> str:
        import torch
        pr = torch.cuda.get_device_properties(torch.cuda.current_device())
        return f"{pr.name}|{pr.multi_processor_count} SMs"

    @staticmethod
    def _class_key(c: dict) -> str:
        return f"{c['kind']}:{c['ndim']}:{c['block']}:{c['pad_kind']}"

    def save_shapes(self, path: str) -> None:
        """Record this plan's launch shapes and concurrent modes under the GPU
        model (name and SM count) and each class (kind, rank, block, padding
        kind) in the JSON file `path` (merged with what it holds)."""
        import json
        try:
            with open(path) as fh:
                tab = json.load(fh)
        except (OSError, ValueError):
            tab = {}
        dev = tab.setdefault(self._device_key(), {"classes": {}, "concurrent": {}})
        for c in self.classes():
            dev["classes"][self._class_key(c)] = {"warps": c["warps"], "ctas_per_sm": c["ctas_per_sm"]}
            dev["concurrent"][str(c["kind"])] = bool(c["concurrent"])
        tmp = path + ".tmp"
        with open(tmp, "w") as fh:
            json.dump(tab, fh, indent=1, sort_keys=True)
        os.replace(tmp, path)

    def load_shapes(self, path: str) -> bool:
        """Apply recorded shapes (save_shapes) when the file holds every class
        of this plan for this GPU model; False (nothing applied) otherwise."""
        import json
        try:
            with open(path) as fh:
                dev = json.load(fh).get(self._device_key())
        except (OSError, ValueError):
            return False
        if not dev:
            return False
        cls = self.classes()
        keys = [self._class_key(c) for c in cls]
        if any(k not in dev.get("classes", {}) for k in keys):
            return False
        for i, k in enumerate(keys):
            sh = dev["classes"][k]
            self.set_shape(i, int(sh["warps"]), int(sh["ctas_per_sm"]))
        conc = set(bool(v) for v in dev.get("concurrent", {}).values())
        if len(conc) == 1:  # one setter serves both sequences: apply only an agreed mode
            self.set_concurrent(conc.pop())
        return True

    def close(self):
        """Release the plan (vsz_batch_destroy)."""
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().vsz_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- entropy stage
HUFF_CHUNK = 1024            # VSZ_HUFF_CHUNK
HUFF_MAX_SYMBOLS = 8192      # VSZ_HUFF_MAX_SYMBOLS


class HuffmanBook:
    """Canonical Huffman codebook of a device histogram (vsz_huffman_book)."""

    def __init__(self, hist, nsym: int | None = None, stream=None):
        import torch
        self.nsym = int(nsym if nsym is not None else hist.numel())
        _need(hist, "hist", 4, self.nsym)
        nb = int(lib().vsz_huffman_book_bytes(self.nsym))
        if nb == 0:
            raise VszError(2 if self.nsym > HUFF_MAX_SYMBOLS else 1, "vsz_huffman_book_bytes")
        self.buf = torch.empty(nb, dtype=torch.uint8, device=hist.device)
        _check(lib().vsz_huffman_book(_ptr(hist), self.nsym, _ptr(self.buf), nb, _stream_handle(stream)),
               "vsz_huffman_book")

    def read(self, stream=None):
        """(lengths uint8[nsym], codewords uint64[nsym], longest length) on the host."""
        import numpy as np
        ln = np.zeros(self.nsym, np.uint8)
        cw = np.zeros(self.nsym, np.uint64)
        mx = ctypes.c_uint32(0)
        _check(lib().vsz_huffman_book_read(_ptr(self.buf), self.nsym, ln.ctypes.data, cw.ctypes.data,
                                           ctypes.byref(mx), _stream_handle(stream)), "vsz_huffman_book_read")
        return ln, cw, int(mx.value)


def shutdown() -> None:
    """vsz_shutdown: switch tracing off, destroy the library's own CUDA
    events and clear its cached launch parameters (for use after a device
    reset).  No library call may be in flight."""
    _check(lib().vsz_shutdown(), "vsz_shutdown")


def huffman_encode(sym, n: int, book: HuffmanBook, words=None, stream=None, index=None):
    """Encode n uint16 symbols (a CUDA tensor viewed as int16/uint16).
    Returns (words, chunk_off, status) as CUDA tensors; status is read by
    the caller (bit 1: a symbol without a codeword, bit 2: words too short).
    With index (an int16 CUDA tensor of 32 entries per chunk, or True to
    allocate one) the decode index is written too (vsz_huffman_encode_indexed;
    bit 16: a chunk too long to index) and (words, chunk_off, status, index)
    is returned."""
    import torch
    nc = (n + HUFF_CHUNK - 1) // HUFF_CHUNK
    _need(sym, "sym", 2, n)
    if words is not None:
        _need(words, "words", 4, 0)
    if index is not None and index is not True:
        _need(index, "index", 2, 32 * nc)
    off = torch.empty(nc + 1, dtype=torch.int64, device=sym.device)
    if words is None:
        words = torch.empty(max(1, n // 2 + nc + 16), dtype=torch.int32, device=sym.device)  # 16 bits/symbol
    st = torch.empty(1, dtype=torch.int32, device=sym.device)
    wsb = int(lib().vsz_huffman_encode_workspace_size(n))
    ws = torch.empty(wsb, dtype=torch.uint8, device=sym.device)
    if index is None:
        _check(lib().vsz_huffman_encode(_ptr(sym), n, _ptr(book.buf), book.nsym, _ptr(words), words.numel(),
                                        _ptr(off), _ptr(st), _ptr(ws), wsb, _stream_handle(stream)),
               "vsz_huffman_encode")
        return words, off, st
    if index is True:
        index = torch.empty(max(1, 32 * nc), dtype=torch.int16, device=sym.device)
    _check(lib().vsz_huffman_encode_indexed(_ptr(sym), n, _ptr(book.buf), book.nsym, _ptr(words), words.numel(),
                                            _ptr(off), _ptr(index), _ptr(st), _ptr(ws), wsb, _stream_handle(stream)),
           "vsz_huffman_encode_indexed")
    return words, off, st, index


def huffman_decode(words, chunk_off, n: int, book: HuffmanBook, out=None, stream=None):
    """Decode n symbols (vsz_huffman_decode); returns (symbols, status)."""
    import torch
    nc = (n + HUFF_CHUNK - 1) // HUFF_CHUNK
    _need(words, "words", 4, 0)
    _need(chunk_off, "chunk_off", 8, nc + 1)
    if out is not None:
        _need(out, "out", 2, n)
    if out is None:
        out = torch.empty(max(n, 1), dtype=torch.int16, device=words.device)
    st = torch.empty(1, dtype=torch.int32, device=words.device)
    _check(lib().vsz_huffman_decode(_ptr(words), words.numel(), _ptr(chunk_off), n, _ptr(book.buf), book.nsym,
                                    _ptr(out), _ptr(st), _stream_handle(stream)), "vsz_huffman_decode")
    return out, st


def huffman_decode_indexed(words, chunk_off, index, n: int, book: HuffmanBook, out=None, stream=None):
    """Decode n symbols with the decode index (vsz_huffman_decode_indexed):
    a warp per chunk; returns (symbols, status)."""
    import torch
    nc = (n + HUFF_CHUNK - 1) // HUFF_CHUNK
    _need(words, "words", 4, 0)
    _need(chunk_off, "chunk_off", 8, nc + 1)
    _need(index, "index", 2, 32 * nc)
    if out is not None:
        _need(out, "out", 2, n)
    if out is None:
        out = torch.empty(max(n, 1), dtype=torch.int16, device=words.device)
    st = torch.empty(1, dtype=torch.int32, device=words.device)
    _check(lib().vsz_huffman_decode_indexed(_ptr(words), words.numel(), _ptr(chunk_off), _ptr(index), n,
                                            _ptr(book.buf), book.nsym, _ptr(out), _ptr(st), _stream_handle(stream)),
           "vsz_huffman_decode_indexed")
    return out, st
