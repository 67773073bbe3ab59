"""One field split across ranks, one GPU per rank, in slabs of whole blocks.

Blocks are independent (Sec. III-A), so a field splits along dims[0] into
slabs of whole blocks and each rank compresses its slab; no tile ever moves
between GPUs.  Three quantities cross slabs, one exchange each:

1. the value range, for a value-range relative error bound (Sec. II-B): the
   minimum of the slabs' finite minima and the maximum of their maxima; the
   field's eb_abs follows from them exactly as the one-field call resolves it
   (in double: eb times the range, eb itself for an empty or zero range);
2. for a global padding mode (Sec. IV-B-1), the padding value: the slabs'
   sums and counts of q (int64) added, their extremes reduced;
   P = min, max, or the rounded mean floor((2S + m) / (2m));
3. the list lengths: the exclusive prefix over the ranks of the slabs'
   outlier and fixup counts places each slab's lists in the field's
   canonical order (blocks in row-major order), so the concatenation over
   the ranks of the slabs' outputs is the whole field's compression.

The per-rank steps run in the library (vsz_slab_range, vsz_slab_qstats,
vsz_compress_slab, vsz_slab_rebase) through a backend object; the exchanges
are torch.distributed collectives (NCCL between GPUs, gloo on CPU ranks).
This module holds the host logic: the slab bounds, the reductions, the
collectives and the order of the steps.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

PAD_ZERO, PAD_GLOBAL_MIN, PAD_GLOBAL_MAX, PAD_GLOBAL_AVG = 0, 1, 2, 3
EB_ABS, EB_REL = 0, 1


# ---------------------------------------------------------------- host logic
def slab_bounds(dims, block: int, world: int, rank: int) -> tuple:
    """[z0, z1) of rank's slab along dims[0]: the block rows dealt as evenly
    as possible, earlier ranks taking one more when they do not divide."""
    n0 = int(dims[0])
    nbz = -(-n0 // block)
    base, extra = divmod(nbz, world)
    b0 = rank * base + min(rank, extra)
    b1 = b0 + base + (1 if rank < extra else 0)
    return min(n0, b0 * block), min(n0, b1 * block)


def field_eb_abs(eb: float, eb_mode: int, gmin: float, gmax: float, has_range: bool) -> float:
    """The field's absolute error bound from the reduced finite range."""
    if eb_mode == EB_ABS or not has_range:
        return float(eb)
    rng = float(gmax) - float(gmin)
    return float(eb) * rng if rng > 0.0 else float(eb)


def global_pad(mode: int, qsum: int, count: int, qmin: int, qmax: int) -> int:
    """The field's global padding value from the reduced q statistics."""
    if count == 0:
        return 0
    if mode == PAD_GLOBAL_MIN:
        return int(qmin)
    if mode == PAD_GLOBAL_MAX:
        return int(qmax)
    return (2 * int(qsum) + int(count)) // (2 * int(count))  # floor division


def exclusive_prefix(values) -> list:
    out, acc = [], 0
    for v in values:
        out.append(acc)
        acc += int(v)
    return out


def is_global_pad(mode: int) -> bool:
    return mode in (PAD_GLOBAL_MIN, PAD_GLOBAL_MAX, PAD_GLOBAL_AVG)


# ---------------------------------------------------------------- exchanges
class Exchange:
    """The three collectives over torch.distributed (any backend: the
    tensors live on `device`)."""

    def __init__(self, dist, device="cpu", group=None):
        self.dist, self.device, self.group = dist, device, group

    def _t(self, vals, dtype):
        import torch
        return torch.tensor(vals, dtype=dtype, device=self.device)

    def range(self, lo: float, hi: float, has: bool) -> tuple:
        import torch
        inf = float("inf")
        t = self._t([lo if has else inf, -(hi if has else -inf)], torch.float64)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MIN, group=self.group)
        gmin, gmax = float(t[0]), -float(t[1])
        return gmin, gmax, gmin != inf

    def qstats(self, qsum: int, count: int, qmin: int, qmax: int) -> tuple:
        import torch
        s = self._t([qsum, count], torch.int64)
        self.dist.all_reduce(s, op=self.dist.ReduceOp.SUM, group=self.group)
        e = self._t([qmin, -qmax], torch.int64)
        self.dist.all_reduce(e, op=self.dist.ReduceOp.MIN, group=self.group)
        return int(s[0]), int(s[1]), int(e[0]), -int(e[1])

    def offsets(self, n_out: int, n_fix: int) -> tuple:
        """(out_base, fix_base, out_total, fix_total) of this rank."""
        import torch
        world = self.dist.get_world_size(self.group)
        mine = self._t([n_out, n_fix], torch.int64)
        allv = [torch.zeros_like(mine) for _ in range(world)]
        self.dist.all_gather(allv, mine, group=self.group)
        outs = [int(v[0]) for v in allv]
        fixs = [int(v[1]) for v in allv]
        r = self.dist.get_rank(self.group)
        return exclusive_prefix(outs)[r], exclusive_prefix(fixs)[r], sum(outs), sum(fixs)


# ---------------------------------------------------------------- drivers
@dataclass
class SlabJob:
    """One rank's part of a split field."""
    dims: tuple      # the whole field's dims
    block: int
    eb: float
    eb_mode: int
    radius: int
    pad: int
    z0: int
    z1: int

    @property
    def slab_dims(self) -> tuple:
        return (self.z1 - self.z0,) + tuple(int(d) for d in self.dims[1:])

    @property
    def elem_base(self) -> int:
        plane = 1
        for d in self.dims[1:]:
            plane *= int(d)
        return self.z0 * plane


def compress_split(exchange: Exchange, backend, job: SlabJob) -> dict:
    """This rank's slab of a split field, in the field's canonical order.
    `backend` runs the per-rank steps (GpuSlabBackend for a GPU rank).
    Returns {"eb_abs", "pad", "out_base", "fix_base", "n_out", "n_fix",
    "n_out_total", "n_fix_total", "result": the backend's output}."""
    if job.eb_mode == EB_REL:
        lo, hi, has = backend.value_range()
        gmin, gmax, ghas = exchange.range(lo, hi, has)
        eb_abs = field_eb_abs(job.eb, job.eb_mode, gmin, gmax, ghas)
    else:
        eb_abs = float(job.eb)
    P = 0
    if is_global_pad(job.pad):
        S, m, mn, mx = backend.qstats(eb_abs)
        S, m, mn, mx = exchange.qstats(S, m, mn, mx)
        P = global_pad(job.pad, S, m, mn, mx)
    res = backend.compress(eb_abs, P)
    n_out, n_fix = backend.counts(res)
    ob, fb, ot, ft = exchange.offsets(n_out, n_fix)
    backend.rebase(res, job.elem_base, ob)
    return {"eb_abs": eb_abs, "pad": P, "out_base": ob, "fix_base": fb, "n_out": n_out, "n_fix": n_fix,
            "n_out_total": ot, "n_fix_total": ft, "result": res}


def compress_split_local(backends, jobs) -> list:
    """The same steps for every rank of a split field in one process (ranks
    emulated one after another, the reductions done here): for one GPU, or
    for tests."""
    job0 = jobs[0]
    if job0.eb_mode == EB_REL:
        rs = [b.value_range() for b in backends]
        fin = [(lo, hi) for lo, hi, has in rs if has]
        has = bool(fin)
        gmin = min(v[0] for v in fin) if has else 0.0
        gmax = max(v[1] for v in fin) if has else 0.0
        eb_abs = field_eb_abs(job0.eb, job0.eb_mode, gmin, gmax, has)
    else:
        eb_abs = float(job0.eb)
    P = 0
    if is_global_pad(job0.pad):
        st = [b.qstats(eb_abs) for b in backends]
        P = global_pad(job0.pad, sum(s[0] for s in st), sum(s[1] for s in st), min(s[2] for s in st),
                       max(s[3] for s in st))
    results = [b.compress(eb_abs, P) for b in backends]
    counts = [b.counts(r) for b, r in zip(backends, results)]
    obase = exclusive_prefix(c[0] for c in counts)
    fbase = exclusive_prefix(c[1] for c in counts)
    out = []
    for b, r, job, c, ob, fb in zip(backends, results, jobs, counts, obase, fbase):
        b.rebase(r, job.elem_base, ob)
        out.append({"eb_abs": eb_abs, "pad": P, "out_base": ob, "fix_base": fb, "n_out": c[0], "n_fix": c[1],
                    "result": r})
    return out


# ---------------------------------------------------------------- the GPU backend
class GpuSlabBackend:
    """The per-rank steps on this rank's GPU, through the library: x is the
    slab's contiguous float32 CUDA tensor; outputs are a Field of the slab
    (absolute mode with the field's eb_abs) with room for `out_cap` outliers
    and `fix_cap` fixups (default: every value)."""

    def __init__(self, job: SlabJob, x, out_cap: int | None = None, fix_cap: int | None = None):
        import torch
        from . import lib
        if not (getattr(x, "is_cuda", False) and x.dtype == torch.float32 and x.is_contiguous()):
            raise TypeError("x must be a contiguous float32 CUDA tensor")
        need = 1
        for d in job.slab_dims:
            need *= int(d)
        if x.numel() != need:
            raise ValueError(f"x has {x.numel()} values, the slab {tuple(job.slab_dims)} holds {need}")
        self.job, self.x = job, x
        self.L = lib()
        self.st = torch.zeros(4, dtype=torch.int64, device=x.device)  # vsz_slab_stats (32 bytes)
        n = x.numel()
        self.out_cap = out_cap if out_cap is not None else max(1, n)
        self.fix_cap = fix_cap if fix_cap is not None else max(1, n)
        self._stream = None

    def _params(self, eb_abs):
        from . import Params
        return Params(tuple(self.job.slab_dims), self.job.block, float(eb_abs), EB_ABS, self.job.radius, self.job.pad)

    def _stats(self) -> dict:
        raw = self.st.cpu().numpy().tobytes()
        s = _SlabStats.from_buffer_copy(raw)
        return {k: getattr(s, k) for k, _ in _SlabStats._fields_}

    def value_range(self):
        from . import _check, _ptr
        _check(self.L.vsz_slab_range(_ptr(self.x), self.x.numel(), _ptr(self.st), None), "vsz_slab_range")
        s = self._stats()
        return float(s["xmin"]), float(s["xmax"]), bool(s["has_range"])

    def qstats(self, eb_abs):
        from . import _check, _ptr
        p = self._params(eb_abs)
        _check(self.L.vsz_slab_qstats(ctypes.byref(p.c()), _ptr(self.x), _ptr(self.st), None), "vsz_slab_qstats")
        s = self._stats()
        return int(s["qsum"]), self.x.numel(), int(s["qmin"]), int(s["qmax"])

    def compress(self, eb_abs, P):
        from . import Field, _check, _ptr
        f = Field(self._params(eb_abs), out_cap=self.out_cap, fix_cap=self.fix_cap)
        _check(self.L.vsz_compress_slab(ctypes.byref(f._cp), int(P), _ptr(self.x), ctypes.byref(f._cc),
                                        _ptr(f.ws), f.ws_bytes, None), "vsz_compress_slab")
        return f

    def counts(self, f):
        h = f.header()
        if h["status"] != 0:
            from . import VszError
            raise VszError(int(h["status"]), "vsz_compress_slab")
        return int(h["n_out"]), int(h["n_fix"])

    def rebase(self, f, elem_base, out_base):
        from . import _check
        _check(self.L.vsz_slab_rebase(ctypes.byref(f._cp), ctypes.byref(f._cc), int(elem_base), int(out_base), None),
               "vsz_slab_rebase")


class _SlabStats(ctypes.Structure):
    _fields_ = [("xmin", ctypes.c_float), ("xmax", ctypes.c_float), ("has_range", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32), ("qsum", ctypes.c_int64), ("qmin", ctypes.c_int32),
                ("qmax", ctypes.c_int32)]
