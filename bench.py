#!/usr/bin/env python
"""Benchmark of the dual-quantization hot path on GB300.

Headline workload: the mixed stream of fields (one 1D field of 280,953,867
random-walk values, 13 fields of 100x500x500 and 20 of 1800x3600, 2.94 GB of
fp32), value-range relative eb 1e-3 (eb 1e-5 reported beside it), R = 512.
Block size and padding per field come from the learned tuner, launch shapes
from the tile autotuner (both chosen once, before the timed region).  One
step is the compression of the whole stream through one batch plan
(value-range pass, fused prequantization + Lorenzo + post-quantization +
guard per class, outlier compaction), replayed as a CUDA graph.  The metric
is GB/s of fp32 input (the paper's prediction-and-quantization bandwidth)
and its fraction of the HBM roofline; the same stream compressed by plain
per-field launches with the default block and zero padding is reported
beside it, as are reconstruction, the end-to-end call from host memory to
host memory, and the one-field 512^3 step.

    python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Under torchrun every rank compresses its own copy of the stream (fields
are independent, so the path shards with no collective on the data path:
weak scaling); rank 0 prints one JSON line.  `--impl reference` times the
CPU oracle (the plain single-threaded C implementation) on bounded samples
of the same stream instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "dual-quant GB/s fp32 in & %HBM roofline, batched+tuned vs plain at fixed eb"
UNIT = "GB/s"
R = 512
STREAM_DESC = ("mixed stream: 1D 280,953,867 random walk + 13 x 100x500x500 GRF + 20 x 1800x3600 Fourier fields "
               "(735,553,867 values, 2.94 GB fp32), relative eb, R=512")


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    ap.add_argument("--eb", type=float, default=1e-3, help="relative eb of the headline")
    ap.add_argument("--eb-beside", type=float, default=1e-5, help="relative eb reported beside the headline")
    ap.add_argument("--no-sampling", action="store_true", help="skip the paper's sampling autotuner baseline")
    ap.add_argument("--no-one-field", action="store_true", help="skip the one-field 512^3 step")
    ap.add_argument("--size", type=int, default=512, help="edge of the cubic one-field workload")
    ap.add_argument("--field-eb", type=float, default=1e-4, help="relative eb of the one-field step")
    ap.add_argument("--pad", default="zero", help="padding of the one-field step")
    ap.add_argument("--block", type=int, default=8, help="block of the one-field step")
    ap.add_argument("--no-sweep", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-entropy", action="store_true", help="skip the Huffman stage and rate-distortion curve")
    ap.add_argument("--batch-profile", action="store_true",
                    help="only a reduced mixed stream (4 of its 1800x3600 fields, 2 of its 100x500x500 fields and "
                         "the first 20M values of its 1D field), the tuner's classes, eb --eb: a small case for "
                         "ncu captures of the batch kernels")
    ap.add_argument("--entropy-profile", action="store_true",
                    help="only the entropy stage on the codes of the one-field workload (--size, --block, --pad; "
                         "timed at --field-eb): a case for ncu captures of the Huffman kernels")
    ap.add_argument("--field-profile", action="store_true",
                    help="only the one-field step (--size, --block, --field-eb, --pad): a case for ncu captures of "
                         "the one-field kernels")
    return ap.parse_args(argv)


def workload_config(a) -> dict:
    return {
        "workload": f"{STREAM_DESC}; eb {a.eb:g}; block and padding per field from the learned tuner, launch "
                    f"shapes from the tile autotuner; compression of the whole stream per step",
        "values": 280_953_867 + 13 * 100 * 500 * 500 + 20 * 1800 * 3600, "eb_rel": a.eb, "radius": R,
        "l2": "inputs larger than L2 (2.94 GB stream vs 129 MB L2); no flush needed",
        "step": "one batch plan (range pass, one persistent kernel per class, origin pass, compaction) "
                "captured once as a CUDA graph and replayed (value)",
    }


def one_field_config(a) -> dict:
    return {
        "workload": f"NYX-like log-normal fp32 {a.size}^3 (exp of k^-3 GRF, seed 2), block {a.block}^3, "
                    f"R={R}, rel eb {a.field_eb:g}, {a.pad} padding: compress (range + fused "
                    f"prequant/Lorenzo/post-quant + compaction) then reconstruct",
        "field_elems": a.size ** 3, "block": a.block, "radius": R, "eb_rel": a.field_eb, "pad": a.pad,
    }


def measured_peaks() -> tuple[float, str]:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid: str | None):
        self.samples = []
        self.proc = None
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "20"]
        if uuid:
            cmd += ["-i", uuid]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.samples.append((time.time(), parts))

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self, t0: float, t1: float) -> dict | None:
        """Clocks and throttle reasons sampled during [t0, t1] (widened by
        the sampling interval, so that a short timed region still holds
        samples)."""
        if not self.samples:
            return None
        win = [p for (t, p) in self.samples if t0 - 0.05 <= t <= t1 + 0.05] or [p for (_, p) in self.samples]

        def num(v):
            try:
                return float(v)
            except ValueError:
                return None
        sm = sorted(v for v in (num(p[1]) for p in win) if v is not None)
        mx = [num(p[2]) for p in win if num(p[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for p in win for i in range(4) if p[5 + i].lower().startswith("active")})
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(win)}


# ---------------------------------------------------------------- ranks
def rank_field_seed(rank: int) -> int:
    """Each rank compresses its own one-field workload: blocks (and fields)
    are independent, so the path shards with no collective on the data path."""
    return 2 + rank


def max_over_ranks(value: float, dist, device: str) -> float:
    """The slowest rank's time (the job's time); identity without dist."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_gbps(world: int, n_per_rank: int, ms: float) -> float:
    """Whole-job GB/s of fp32 input: all ranks' values over the max time."""
    return world * n_per_rank * 4 / (ms * 1e-3) / 1e9


# ---------------------------------------------------------------- roofline
def algorithmic_bytes(name: str, n: int, nb: int, n_out: int, n_fix: int, block_pad: bool) -> int:
    """Bytes a launch must move at minimum (each input read once, each output
    written once), per the data layout of the path."""
    if name in ("range", "qstats", "batch_range"):
        return 4 * n
    if name.startswith(("lorenzo", "batch_lorenzo")):  # x in; codes, outliers/fixups, block offsets (+ pads) out
        return 4 * n + 2 * n + 8 * (n_out + n_fix) + 4 * nb + (4 * nb if block_pad else 0)
    if name == "compact_move":  # staged entries in and out, block offsets read-modify-write
        return 16 * (n_out + n_fix) + 8 * nb
    if name in ("recon", "batch_recon"):  # codes, outliers, block offsets (+ pads) in; values out
        return 2 * n + 8 * n_out + 4 * (nb + 1) + (4 * nb if block_pad else 0) + 4 * n
    if name in ("fixups", "batch_fixups"):
        return 12 * n_fix
    return 0


# The source files that define each profiled kernel (its body, the headers
# it includes and its launcher): a committed ncu figure holds while these
# files are unchanged.
KERNEL_SOURCES = {
    "k_lorenzo_nd_batch": ("common.cuh", "memops.cuh", "ring.cuh", "compress_nd.cuh", "recon_nd.cuh", "k_rank2.cu",
                           "k_rank3.cu"),
    "k_lorenzo_1d_batch": ("common.cuh", "memops.cuh", "k_rank1.cu"),
    "k_lorenzo_nd": ("common.cuh", "memops.cuh", "ring.cuh", "compress_nd.cuh", "recon_nd.cuh", "k_rank3.cu"),
    "k_recon_nd": ("common.cuh", "memops.cuh", "ring.cuh", "compress_nd.cuh", "recon_nd.cuh", "k_rank3.cu"),
    "k_range": ("common.cuh", "memops.cuh", "stats.cuh", "k_misc.cu"),
}


def kernel_sources_digest(kernel: str | None = None) -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2201_04614_gb300", "csrc")
    files = KERNEL_SOURCES.get(kernel.split("<")[0]) if kernel else None
    for f in sorted(files or (f for f in os.listdir(csrc) if f.endswith((".cu", ".cuh")))):
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel: str, workload: str, units: int | None = None, path: str | None = None) -> int | None:
    """dram bytes per launch from a committed ncu summary, if it was taken on
    the current sources of that kernel.  An entry taken on a smaller case of
    the same kernel records bytes per value instead; it is scaled by `units`
    (the values of a full launch)."""
    path = path or os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            tab = json.load(f)
    except Exception:
        return None
    ent = tab.get(f"{kernel}|{workload}")
    if not ent or ent.get("src_digest") != kernel_sources_digest(kernel):
        return None
    if "dram_bytes_per_value" in ent:
        return int(round(float(ent["dram_bytes_per_value"]) * units)) if units else None
    return int(ent["dram_bytes_per_launch"])


# ---------------------------------------------------------------- CPU oracle
def oracle_rate(x3, a, seconds: float, unit_planes: int = 8, rows: int | None = None):
    """Time the oracle (compress + decompress) on consecutive block-aligned
    slabs of the field until `seconds` of CPU time are spent (at least one).
    Returns (GB/s of fp32 input, elements, slabs, sample description)."""
    import numpy as np
    import oracle
    oracle.build()
    nz, ny, nx = x3.shape
    rows = rows or ny
    pad = oracle.PAD_NAMES[a.pad]
    elems, t_used, k = 0, 0.0, 0
    while True:
        z0 = (k * unit_planes) % nz
        y0 = ((k * unit_planes) // nz * rows) % ny
        sl = np.ascontiguousarray(x3[z0:z0 + unit_planes, y0:y0 + rows, :])
        p = oracle.Params(sl.shape, a.block, a.field_eb, oracle.EB_REL, R, pad)
        t = time.perf_counter()
        c = oracle.compress(p, sl)
        oracle.decompress(p, c)
        t_used += time.perf_counter() - t
        elems += sl.size
        k += 1
        if t_used >= seconds:
            break
    desc = (f"{k} block-aligned slabs of {unit_planes}x{rows}x{nx} of the same field, each compressed "
            f"(own rel-eb range pass) and decompressed by the single-threaded oracle")
    return elems * 4 / t_used / 1e9, elems, k, desc


def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def oracle_rate_parallel(x3, a, seconds: float, threads: int | None = None, unit_planes: int = 8):
    """The same oracle with the field's block-aligned slabs spread over the
    host's hardware threads: thread t takes slabs t, t+P, ... until `seconds`
    of wall time have passed (ctypes releases the GIL inside the C oracle, so
    the threads run in parallel).  Returns (GB/s of fp32 input, threads,
    slabs, sample description)."""
    import numpy as np
    import oracle
    from concurrent.futures import ThreadPoolExecutor
    oracle.build()
    P = threads or os.cpu_count() or 1
    nz, ny, nx = x3.shape
    pad = oracle.PAD_NAMES[a.pad]
    nslab = max(1, nz // unit_planes)
    start = threading.Barrier(P)

    def work(t):
        start.wait()
        t0 = time.perf_counter()
        elems, k, j = 0, 0, t
        while True:
            z0 = (j % nslab) * unit_planes
            sl = np.ascontiguousarray(x3[z0:z0 + unit_planes])
            p = oracle.Params(sl.shape, a.block, a.field_eb, oracle.EB_REL, R, pad)
            c = oracle.compress(p, sl)
            oracle.decompress(p, c)
            elems += sl.size
            k += 1
            j += P
            if time.perf_counter() - t0 >= seconds:
                return elems, k, time.perf_counter() - t0

    with ThreadPoolExecutor(P) as ex:
        res = list(ex.map(work, range(P)))
    elems = sum(r[0] for r in res)
    slabs = sum(r[1] for r in res)
    wall = max(r[2] for r in res)
    desc = (f"{slabs} block-aligned slabs of {unit_planes}x{ny}x{nx} of the same field over {P} threads "
            f"(slabs dealt round-robin), each compressed and decompressed by the oracle")
    return elems * 4 / wall / 1e9, P, slabs, desc


# ---------------------------------------------------------------- the mixed stream on the host
def stream_slab(shape, x, k: int, block: int):
    """The k-th block-aligned slab of one field of the stream (a bounded
    sample for the CPU oracle): 2^20 values of the 1D field, 64 rows of a 2D
    field, 32 planes of a 3D field (multiples of every block of the rank)."""
    import numpy as np
    if len(shape) == 1:
        m = 1 << 20
        s0 = ((k * m) % max(1, shape[0] - m)) // block * block
        return np.ascontiguousarray(x[s0:s0 + m])
    x = x.reshape(shape)
    rows = 64 if len(shape) == 2 else 32
    s0 = ((k * rows) % max(1, shape[0] - rows)) // block * block
    return np.ascontiguousarray(x[s0:s0 + rows])


def oracle_stream_rate(specs_host, eb: float, seconds: float, start: int = 0):
    """Time the oracle's compression (the metric's leg) on block-aligned
    slabs of the stream's fields, taken round-robin over the fields, until
    `seconds` of CPU time are spent (at least one slab).  Each slab is
    compressed in absolute mode with its field's eb_abs (relative eb times
    the field's value range) with the default block and zero padding.
    Returns (GB/s of fp32 input, elements, slabs, sample description)."""
    import oracle
    oracle.build()
    blocks = {1: 256, 2: 16, 3: 8}
    elems, t_used, k = 0, 0.0, 0
    nf = len(specs_host)
    while True:
        name, shape, x, eb_abs = specs_host[(start + k) % nf]
        b = blocks[len(shape)]
        sl = stream_slab(shape, x, (start + k) // nf, b)
        p = oracle.Params(sl.shape, b, eb_abs, oracle.EB_ABS, R, oracle.PAD_ZERO)
        t = time.perf_counter()
        oracle.compress(p, sl)
        t_used += time.perf_counter() - t
        elems += sl.size
        k += 1
        if t_used >= seconds:
            break
    desc = (f"{k} block-aligned slabs of the mixed stream's fields (2^20 values of the 1D field, 64 rows of a "
            f"1800x3600 field, 32 planes of a 100x500x500 field; fields round-robin), each compressed by the "
            f"single-threaded oracle with its field's eb_abs at rel eb {eb:g}, default block, zero padding")
    return elems * 4 / t_used / 1e9, elems, k, desc


def stream_host(eb: float, threads: int | None = None):
    """The mixed stream generated on the host: [(name, shape, x, eb_abs)]."""
    import numpy as np
    import synth
    from concurrent.futures import ThreadPoolExecutor
    specs = synth.cfg5_fields()
    with ThreadPoolExecutor(threads or min(16, os.cpu_count() or 1)) as ex:
        xs = list(ex.map(lambda sp: np.ascontiguousarray(sp[2](), np.float32).reshape(-1), specs))
    out = []
    for (name, shape, _), x in zip(specs, xs):
        fin = x[np.isfinite(x)]
        rng = float(fin.max()) - float(fin.min()) if fin.size else 0.0
        out.append((name, shape, x, eb * rng if rng > 0 else eb))
    return out


def run_reference(a):
    """The oracle, as it stands, on the host cores: each step one bounded
    sample of the mixed stream (compression, the metric's leg)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    specs = stream_host(a.eb)
    # size one step so that warmup + steps take about a minute
    probe, _, _, _ = oracle_stream_rate(specs, a.eb, 0.0)
    per_step = max(1.0, min(8.0, 60.0 / max(1, a.steps + a.warmup)))
    k = 0
    for _ in range(a.warmup):
        _, _, used, _ = oracle_stream_rate(specs, a.eb, per_step, start=k)
        k += used
    t = time.perf_counter()
    elems, slabs = 0, 0
    desc = ""
    for _ in range(a.steps):
        _, e, used, desc = oracle_stream_rate(specs, a.eb, per_step, start=k)
        k += used
        elems += e
        slabs += used
    dt = time.perf_counter() - t
    value = elems * 4 / dt / 1e9
    sample = (f"each step: about {per_step:.1f} s of the oracle's compression on block-aligned slabs of the mixed "
              f"stream ({slabs} slabs in {a.steps} steps); " + desc.split("; ", 1)[-1])
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": a.gpus,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": dt / a.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32/i32",
        "data": "synthetic", "config": workload_config(a),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- the mixed stream on the GPU
def kernel_key(rec) -> tuple:
    return rec["name"], int(rec["ndim"]), int(rec["block"])


def class_key(p) -> tuple:
    """(compression kernel name, rank, block) of a field's batch class: its
    trace name carries the padding kind (none, per block, global or edge)."""
    nm = ("batch_lorenzo_bp" if p.is_block_pad else "batch_lorenzo_gp" if p.pad in (1, 2, 3)
          else ("batch_lorenzo_ep" if len(p.dims) > 1 else "batch_lorenzo_gp") if p.is_edge_pad else "batch_lorenzo")
    return nm, len(p.dims), int(p.block)


def sequence_bytes(fields, heads) -> dict:
    """Algorithmic bytes of one compression of the stream, per kernel key and
    in total (each input read once by the range pass and once by the walk,
    each code, outlier, fixup, block offset and padding value written once;
    the compaction's move of staged entries is not algorithmic)."""
    per = {}
    total = 0
    n_all = 0
    for f, h in zip(fields, heads):
        p = f.p
        n, nb = f.n, f.nb
        by = algorithmic_bytes("batch_lorenzo", n, nb, int(h["n_out"]), int(h["n_fix"]), p.is_block_pad)
        k = class_key(p)
        per[k] = per.get(k, 0) + by
        total += by + 4 * n
        n_all += n
    per[("batch_range", 0, 0)] = 4 * n_all
    return {"per_kernel": per, "total": total}


def make_stream_fields(vsz, T, shapes, classes, eb):
    """One Field per stream field, with room in its lists for every element
    (so that no field overflows)."""
    import numpy as np
    out = []
    for shape, c in zip(shapes, classes):
        b, pad = T.class_params(len(shape), c)
        n = int(np.prod(shape))
        out.append(vsz.Field(vsz.Params.make(shape, b, eb, "rel", R, pad), out_cap=n, fix_cap=max(1 << 16, n // 64)))
    return out


def measure_stream(a, vsz, T, torch, names, shapes, xs, eb, stream, keep_tuned=False, log_fn=log) -> dict:
    """Compression and reconstruction of the stream at one eb: plain
    per-field launches with the default classes (eagerly and as one CUDA
    graph), one autotuned batch plan with the default classes, one with the
    learned tuner's classes, and (unless --no-sampling) one with the block
    sizes of the paper's sampling autotuner.  Per-kernel device times of the
    tuned plan come from a traced loop (CUDA events around every launch).
    With keep_tuned the tuned plan, its fields and outputs are returned
    under "_keep" for the headline's timed region."""
    steps = max(5, min(a.steps, 50))
    n_total = sum(x.numel() for x in xs)
    gb = n_total * 4 / 1e9
    outs = [torch.empty(x.numel(), dtype=torch.float32, device="cuda") for x in xs]

    def timed(fn):
        with torch.cuda.stream(stream):
            for _ in range(3):
                fn()
            stream.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(steps):
                fn()
            e1.record(stream)
            stream.synchronize()
        return e0.elapsed_time(e1) / steps

    def autotuned(fields):
        bt = vsz.Batch(fields, xs, use_graph=True)
        bt.set_outputs(outs)
        torch.cuda.synchronize()
        tt = time.time()
        cls = bt.autotune(stream, reps=3)
        return bt, cls, (time.time() - tt) * 1e3

    def shapes_of(cls):
        return [{k: c[k] for k in ("kind", "ndim", "block", "pad_kind", "warps", "ctas_per_sm", "concurrent",
                                   "ms", "ms_default")} for c in cls if c["tiles"]]

    ms, r = {}, {"eb": eb}
    dflt = [T.default_class(len(sh)) for sh in shapes]
    plain = make_stream_fields(vsz, T, shapes, dflt, eb)

    def plain_step():
        for f, x in zip(plain, xs):
            f.compress(x, stream=stream)
    ms["plain"] = timed(plain_step)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(stream):
        plain_step()
        stream.synchronize()
        with torch.cuda.graph(g, stream=stream):
            plain_step()
    ms["plain_graph"] = timed(g.replay)
    del g
    ms["plain_recon"] = timed(lambda: [f.reconstruct(out=o, stream=stream) for f, o in zip(plain, outs)])
    nout_def = [int(f.header()["n_out"]) for f in plain]
    status = [int(f.header()["status"]) for f in plain]
    bd, cls_def, at_def_ms = autotuned(plain)
    ms["batched_default"] = timed(lambda: bd.submit(stream))
    ms["batched_default_recon"] = timed(lambda: bd.reconstruct(stream))
    bd.close()
    del bd, plain
    torch.cuda.empty_cache()

    # the learned tuner's classes: features, one MLP inference, the guard
    torch.cuda.synchronize()
    tt = time.time()
    picks = T.choose([(vsz.Params.make(sh, 8, eb, "rel", R, "zero"), x) for sh, x in zip(shapes, xs)])
    torch.cuda.synchronize()
    tune_ms = (time.time() - tt) * 1e3
    classes = [p["class"] for p in picks]
    tuned = make_stream_fields(vsz, T, shapes, classes, eb)
    bt, cls_tuned, at_tuned_ms = autotuned(tuned)
    ms["batched_tuned"] = timed(lambda: bt.submit(stream))
    ms["batched_tuned_recon"] = timed(lambda: bt.reconstruct(stream))
    heads = [f.header() for f in tuned]
    nout_tuned = [int(h["n_out"]) for h in heads]
    status += [int(h["status"]) for h in heads]

    # per-kernel device times of the tuned plan's compression and reconstruction,
    # with its class kernels one after another (parallel branches would time
    # each kernel with its neighbours' work inside)
    conc = bt.concurrency()
    bt.set_concurrent_each(False, False)
    vsz.trace_enable(True)
    vsz.trace_read()
    reps = max(3, min(steps, 10))
    with torch.cuda.stream(stream):
        for _ in range(reps):
            bt.submit(stream)
        stream.synchronize()
        recs_c = vsz.trace_read(1 << 20)
        for _ in range(reps):
            bt.reconstruct(stream)
        stream.synchronize()
    recs_r = vsz.trace_read(1 << 20)
    vsz.trace_enable(False)
    bt.set_concurrent_each(*conc)
    r["concurrent"] = {"compress": conc[0], "reconstruct": conc[1]}
    sb = sequence_bytes(tuned, heads)
    kern = {}
    for rec in recs_c:
        k = kernel_key(rec)
        d = kern.setdefault(k, {"launches": 0, "ms": 0.0})
        d["launches"] += 1
        d["ms"] += max(0.0, rec["ms"])
    kernels = {}
    for k, d in kern.items():
        avg = d["ms"] / d["launches"]
        by = sb["per_kernel"].get(k)
        kernels[f"{k[0]}<{k[1]}d,b{k[2]}>"] = {
            "launches_per_step": d["launches"] / reps, "avg_us": avg * 1e3,
            "algorithmic_bytes": by, "GBps": (by / (avg * 1e-3) / 1e9) if (by and avg > 0) else None}
    rkern = {}
    for rec in recs_r:
        k = f"{rec['name']}<{rec['ndim']}d,b{rec['block']}>"
        d = rkern.setdefault(k, {"launches": 0, "ms": 0.0})
        d["launches"] += 1
        d["ms"] += max(0.0, rec["ms"])
    rkernels = {k: {"avg_us": d["ms"] / d["launches"] * 1e3} for k, d in rkern.items()}
    launches_per_step = len(recs_c) / reps
    if not keep_tuned:
        bt.close()
        del bt
        torch.cuda.empty_cache()

    if not a.no_sampling:
        # the paper's own autotuner (Sec. III-D) as the learned tuner's
        # baseline: per field the block size whose dual-quant is fastest on a
        # 5 % sample (zero padding), then the same autotuned batch plan
        torch.cuda.synchronize()
        tt = time.time()
        samp = [T.sampling_autotune(vsz.Params.make(sh, 8, eb, "rel", R, "zero"), x, 0.05, 3)
                for sh, x in zip(shapes, xs)]
        samp_ms = (time.time() - tt) * 1e3
        slots = {1: (32, 64, 128, 256), 2: (8, 16, 32, 64), 3: (8, 16, 32)}
        samp_cls = [3 * slots[len(sh)].index(s["block"]) for sh, s in zip(shapes, samp)]
        sampf = make_stream_fields(vsz, T, shapes, samp_cls, eb)
        bs, _, _ = autotuned(sampf)
        ms["batched_sampling_tuned"] = timed(lambda: bs.submit(stream))
        ms["batched_sampling_tuned_recon"] = timed(lambda: bs.reconstruct(stream))
        bs.close()
        nout_samp = [int(f.header()["n_out"]) for f in sampf]
        status += [int(f.header()["status"]) for f in sampf]
        del bs, sampf
        torch.cuda.empty_cache()
        r["sampling_autotuner"] = {"tune_ms_once": samp_ms, "n_out_total": sum(nout_samp),
                                   "blocks": {nm: s["block"] for nm, s in zip(names, samp)}}
    r.update({f"{k}_GBps": gb / (v * 1e-3) for k, v in ms.items()})
    r["ms"] = ms
    r["tuned_vs_plain"] = ms["plain"] / ms["batched_tuned"]
    r["tuned_vs_batched_default"] = ms["batched_default"] / ms["batched_tuned"]
    r["tune_ms_once"] = tune_ms
    r["autotune_ms_once"] = {"default": at_def_ms, "tuned": at_tuned_ms}
    r["shapes_default_classes"] = shapes_of(cls_def)
    r["shapes_tuned_classes"] = shapes_of(cls_tuned)
    r["classes_tuned"] = {nm: T.class_params(len(sh), c) for nm, sh, c in zip(names, shapes, classes)
                          if c != T.default_class(len(sh))}
    r["guard_fallbacks"] = sum(1 for p in picks if p["class"] != p["predicted"])
    r["n_out_default_total"] = sum(nout_def)
    r["n_out_tuned_total"] = sum(nout_tuned)
    r["fields_n_out_tuned_le_default"] = sum(1 for u, v in zip(nout_tuned, nout_def) if u <= v)
    r["fields"] = len(xs)
    r["status_nonzero"] = sum(1 for v in status if v)
    r["tuned_kernels"] = kernels
    r["tuned_recon_kernels"] = rkernels
    r["tuned_launches_per_step"] = launches_per_step
    r["sequence_bytes"] = sb["total"]
    r["_kern"] = kern
    r["_reps"] = reps
    r["_seq"] = sb
    if keep_tuned:
        r["_keep"] = (bt, tuned, outs, heads)
    log_fn(f"[bench] stream eb={eb:g}: " + json.dumps({k: v for k, v in r.items()
                                                      if k.endswith("GBps") or k.startswith("n_out")
                                                      or k == "status_nonzero"}))
    return r


# ---------------------------------------------------------------- the one-field step (512^3)
def run_one_field(a, vsz, torch, xd, x3, n, stream, timed_loop) -> dict:
    """The one-field step on the NYX-like 512^3 field: compression (range
    pass, fused kernel, compaction) then reconstruction, captured once as a
    CUDA graph and replayed; per-kernel device times from a traced loop, and
    the roofline of its dominant kernel."""
    p = vsz.Params.make(x3.shape, a.block, a.field_eb, "rel", R, a.pad)
    f = vsz.Field(p, out_cap=max(1 << 20, n // 8), fix_cap=max(1 << 16, n // 64))
    xh = torch.empty(n, dtype=torch.float32, device="cuda")

    def step():
        f.compress(xd)
        f.reconstruct(out=xh)

    for _ in range(max(3, a.warmup)):
        step()
    torch.cuda.synchronize()
    h = f.header()
    if h["status"] != 0:
        raise SystemExit(f"compression status {h['status']} (capacity too small?)")
    n_out, n_fix = int(h["n_out"]), int(h["n_fix"])
    gstream = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(gstream):
        step()
        gstream.synchronize()
        with torch.cuda.graph(graph, stream=gstream):
            step()
        for _ in range(max(3, a.warmup)):
            graph.replay()
    gstream.synchronize()
    with torch.cuda.stream(gstream):
        ms_step = timed_loop(graph.replay, gstream)
    ms_eager = timed_loop(step, stream)
    vsz.trace_enable(True)
    vsz.trace_read()
    ms_traced = timed_loop(step, stream)
    vsz.trace_enable(False)
    recs = vsz.trace_read(1 << 20)
    del graph
    per = {}
    for r in recs:
        d = per.setdefault(r["name"], {"launches": 0, "ms": 0.0})
        d["launches"] += 1
        d["ms"] += max(0.0, r["ms"])
    nb, bp = p.nblocks, p.is_block_pad
    peak, peak_kind = measured_peaks()
    kernels, step_bytes = {}, 0
    for name, d in per.items():
        avg = d["ms"] / d["launches"]
        by = algorithmic_bytes(name, n, nb, n_out, n_fix, bp)
        step_bytes += by
        kernels[name] = {"launches": d["launches"], "avg_us": avg * 1e3,
                         "share": d["ms"] / max(1e-9, sum(v["ms"] for v in per.values())),
                         "GBps": (by / (avg * 1e-3) / 1e9) if (by and avg > 0) else None}
    dom = max(("lorenzo", "recon"), key=lambda k: per.get(k, {"ms": 0})["ms"])
    dom_avg_s = per[dom]["ms"] / per[dom]["launches"] * 1e-3
    dom_bytes = algorithmic_bytes(dom, n, nb, n_out, n_fix, bp)
    achieved = dom_bytes / dom_avg_s / 1e9
    gp = a.pad.startswith("global")
    kname = {"lorenzo": f"k_lorenzo_nd<3,{a.block},{str(bp).lower()},{str(gp).lower()}>",
             "recon": f"k_recon_nd<3,{a.block},false>"}[dom]
    wl = f"{a.size}^3 b{a.block} eb{a.field_eb:g} {a.pad}"
    steps = a.steps
    compress_ms = sum(per[k]["ms"] for k in ("begin", "range", "lorenzo", "compact_scan", "compact_move",
                                              "origin_fix") if k in per) / steps
    recon_ms = sum(per[k]["ms"] for k in ("recon", "fixups") if k in per) / steps
    out = {
        "config": one_field_config(a), "GBps": n * 4 / (ms_step * 1e-3) / 1e9, "ms_per_step": ms_step,
        "eager": {"GBps": n * 4 / (ms_eager * 1e-3) / 1e9, "ms_per_step": ms_eager},
        "traced": {"GBps": n * 4 / (ms_traced * 1e-3) / 1e9, "ms_per_step": ms_traced},
        "roofline": {"bound": "hbm", "kernel": kname, "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "bytes_per_launch": dom_bytes,
                     "traffic": profiled_traffic(kname, wl)},
        "step_hbm_frac": step_bytes / (ms_step * 1e-3) / 1e9 / peak, "kernels": kernels,
        "outliers": {"n_out": n_out, "n_fix": n_fix, "frac_out": n_out / n},
        "compress_GBps": n * 4 / (compress_ms * 1e-3) / 1e9, "reconstruct_GBps": n * 4 / (recon_ms * 1e-3) / 1e9,
    }
    del f, xh
    torch.cuda.empty_cache()
    return out


def run_sweep(a, vsz, torch, xd, x3, n) -> list:
    """eb x padding sweep of the one-field workload (separate short runs)."""
    xh = torch.empty(n, dtype=torch.float32, device="cuda")
    # the GPU idled at lower clocks during the host-bound legs before: bring
    # it back to speed before the first configuration is timed
    ps0 = vsz.Params.make(x3.shape, a.block, 1e-2, "rel", R, "zero")
    f0 = vsz.Field(ps0, out_cap=n // 4, fix_cap=max(1 << 16, n // 64))
    for _ in range(50):
        f0.compress(xd)
        f0.reconstruct(out=xh)
    torch.cuda.synchronize()
    del f0
    sweep = []
    for eb in (1e-2, 1e-3, 1e-4, 1e-5):
        for pad in ("zero", "block_avg", "global_avg", "edge_avg"):
            ps = vsz.Params.make(x3.shape, a.block, eb, "rel", R, pad)
            fs = vsz.Field(ps, out_cap=n // 4, fix_cap=max(1 << 16, n // 64))
            for _ in range(3):
                fs.compress(xd)
                fs.reconstruct(out=xh)
            torch.cuda.synchronize()
            k = 20
            c0, c1, r1 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            tc = tr = 0.0
            for _ in range(k):
                c0.record()
                fs.compress(xd)
                c1.record()
                fs.reconstruct(out=xh)
                r1.record()
                r1.synchronize()
                tc += c0.elapsed_time(c1)
                tr += c1.elapsed_time(r1)
            hs = fs.header()
            no, nf = int(hs["n_out"]), int(hs["n_fix"])
            nb = ps.nblocks
            cb = 4 * n + algorithmic_bytes("lorenzo", n, nb, no, nf, ps.is_block_pad)
            rb = algorithmic_bytes("recon", n, nb, no, nf, ps.is_block_pad) + 12 * nf
            peak, _ = measured_peaks()
            sweep.append({"eb": eb, "pad": pad, "compress_GBps": n * 4 / (tc / k * 1e-3) / 1e9,
                          "reconstruct_GBps": n * 4 / (tr / k * 1e-3) / 1e9,
                          "compress_hbm_frac": cb / (tc / k * 1e-3) / 1e9 / peak,
                          "reconstruct_hbm_frac": rb / (tr / k * 1e-3) / 1e9 / peak,
                          "n_out": no, "n_fix": nf, "status": int(hs["status"])})
            del fs
            torch.cuda.empty_cache()
    del xh
    return sweep


# ---------------------------------------------------------------- entropy stage
def run_entropy(a, x3, xd, log_fn=log) -> dict:
    """The entropy stage (Sec. II-B) on the codes of the bench field: code
    histogram, Huffman codebook, encode and decode throughput (CUDA events
    around 20 calls in a row), and the rate-distortion curve: PSNR against total bits per
    value (Huffman stream + outliers + fixups + block offsets + chunk
    offsets + padding table), relative eb 1e-2..1e-5."""
    import numpy as np
    import torch
    import paper_2201_04614_gb300 as vsz

    n = x3.size
    vrange = float(x3.max()) - float(x3.min())
    xh = torch.empty(n, dtype=torch.float32, device="cuda")
    out = {"curve": []}

    def ev_ms(fn, k=20):
        # k calls back to back between two events, so that the device time
        # of a call does not include the host's launch latency
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(k):
            fn()
        e1.record()
        e1.synchronize()
        return e0.elapsed_time(e1) / k

    for eb in (1e-2, 1e-3, 1e-4, 1e-5):
        p = vsz.Params.make(x3.shape, a.block, eb, "rel", R, a.pad)
        f = vsz.Field(p, out_cap=n // 2, fix_cap=max(1 << 16, n // 64))
        f.compress(xd)
        f.reconstruct(out=xh)
        h = f.header()
        nsym = 2 * R
        hist = f.code_histogram()
        book = vsz.HuffmanBook(hist, nsym)
        words, off, st = vsz.huffman_encode(f.codes, n, book)
        nwords = int(off[-1].item())
        dec, st2 = vsz.huffman_decode(words, off, n, book)
        ok = int(st.item()) == 0 and int(st2.item()) == 0 and bool(torch.equal(dec[:n], f.codes[:n]))
        # the same stream with its decode index, decoded a warp per chunk
        words_ix, off_ix, st_ix, index = vsz.huffman_encode(f.codes, n, book, index=True)
        dec_ix, st_dix = vsz.huffman_decode_indexed(words_ix, off_ix, index, n, book)
        ok = ok and int(st_ix.item()) == 0 and int(st_dix.item()) == 0 and bool(torch.equal(dec_ix[:n], f.codes[:n])) \
            and bool(torch.equal(off_ix, off)) and bool(torch.equal(words_ix[:nwords], words[:nwords]))
        nc = off.numel() - 1
        table_bits = 32 * (p.nblocks + 1) + 64 * (nc + 1) + 32 * p.pad_len
        bits = 32 * nwords + 64 * int(h["n_out"]) + 64 * int(h["n_fix"]) + table_bits
        mse = float(((xh.double() - xd.double()) ** 2).mean().item())
        psnr = 20 * math.log10(vrange) - 10 * math.log10(mse) if mse > 0 else float("inf")
        row = {"eb": eb, "bits_per_value": bits / n, "ratio": 32.0 * n / bits, "huffman_bits_per_value": 32 * nwords / n,
               "decode_index_bits_per_value": 512.0 * nc / n,
               "psnr_db": psnr, "n_out": int(h["n_out"]), "n_fix": int(h["n_fix"]), "round_trip_ok": ok}
        if eb == a.field_eb:
            ms_hist = ev_ms(lambda: f.code_histogram(out=hist))
            ms_book = ev_ms(lambda: vsz.HuffmanBook(hist, nsym))
            ms_enc = ev_ms(lambda: vsz.huffman_encode(f.codes, n, book, words=words))
            ms_dec = ev_ms(lambda: vsz.huffman_decode(words, off, n, book, out=dec))
            ms_enc_ix = ev_ms(lambda: vsz.huffman_encode(f.codes, n, book, words=words_ix, index=index))
            ms_dec_ix = ev_ms(lambda: vsz.huffman_decode_indexed(words_ix, off_ix, index, n, book, out=dec_ix))
            # bytes each pass must move: encode reads the codes twice (bit
            # counts, then packing) and writes the stream; decode reads the
            # stream and writes the codes
            enc_bytes, dec_bytes = 4 * n + 4 * nwords, 4 * nwords + 2 * n
            vsz.trace_enable(True)
            vsz.trace_read()
            vsz.huffman_encode(f.codes, n, book, words=words)
            vsz.huffman_decode(words, off, n, book, out=dec)
            vsz.huffman_decode_indexed(words_ix, off_ix, index, n, book, out=dec_ix)
            vsz.trace_enable(False)
            kern = {r["name"]: round(r["ms"] * 1e3, 1) for r in vsz.trace_read(64)}
            row["timing"] = {
                "histogram_us": ms_hist * 1e3, "book_us": ms_book * 1e3,
                "encode_us": ms_enc * 1e3, "decode_us": ms_dec * 1e3,
                "encode_GBps_fp32_in": 4 * n / (ms_enc * 1e-3) / 1e9, "decode_GBps_fp32_out": 4 * n / (ms_dec * 1e-3) / 1e9,
                "encode_hbm_GBps": enc_bytes / (ms_enc * 1e-3) / 1e9, "decode_hbm_GBps": dec_bytes / (ms_dec * 1e-3) / 1e9,
                "encode_indexed_us": ms_enc_ix * 1e3, "decode_indexed_us": ms_dec_ix * 1e3,
                "decode_indexed_hbm_GBps": (dec_bytes + 64 * nc) / (ms_dec_ix * 1e-3) / 1e9,
                "kernels_us_one_call": kern}
        out["curve"].append(row)
        log_fn(f"[bench] entropy eb={eb:g}: {row}")
        del f, book, words, off, dec, words_ix, off_ix, index, dec_ix
        torch.cuda.empty_cache()
    return out


def oracle_stream_rate_parallel(specs_host, eb: float, seconds: float, threads: int | None = None):
    """The same oracle with the stream's slabs spread over the host's
    hardware threads (thread t starts at slab t; ctypes releases the GIL
    inside the C oracle).  Returns (GB/s, threads, slabs, description)."""
    from concurrent.futures import ThreadPoolExecutor
    P = threads or os.cpu_count() or 1
    t0 = time.perf_counter()
    with ThreadPoolExecutor(P) as ex:
        res = list(ex.map(lambda t: oracle_stream_rate(specs_host, eb, seconds, start=1000 * t), range(P)))
    wall = time.perf_counter() - t0
    elems = sum(r[1] for r in res)
    slabs = sum(r[2] for r in res)
    desc = f"{slabs} block-aligned slabs of the mixed stream over {P} threads, compressed by the oracle"
    return elems * 4 / wall / 1e9, P, slabs, desc


def batch_kernel_name(key) -> str:
    name, nd, b = key
    bp = "true" if name.endswith("_bp") else "false"
    gp = "true" if name.endswith(("_gp", "_ep")) else "false"
    ep = ",true" if name.endswith("_ep") else ""
    return f"k_lorenzo_1d_batch<{b},{bp},{gp}>" if nd == 1 else f"k_lorenzo_nd_batch<{nd},{b},{bp},{gp}{ep}>"


def strip_private(d: dict) -> dict:
    return {k: v for k, v in d.items() if not k.startswith("_")}


# ---------------------------------------------------------------- GPU arm
def run_gpu(a):
    import numpy as np
    import torch
    import paper_2201_04614_gb300 as vsz
    from paper_2201_04614_gb300 import tuner as T
    import synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (no CPU fallback)")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    def timed_loop(fn, s):
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for _ in range(a.steps):
            fn()
        e1.record(s)
        barrier()
        return max_over_ranks(e0.elapsed_time(e1), dist, "cuda") / a.steps

    vsz.lib()
    t = time.time()
    specs_host = stream_host(a.eb)
    names = [s[0] for s in specs_host]
    shapes = [s[1] for s in specs_host]
    xs = [torch.from_numpy(s[2]).cuda() for s in specs_host]
    n_total = sum(x.numel() for x in xs)
    log(f"[bench] rank {rank}: mixed stream of {len(xs)} fields, {n_total} values, in {time.time() - t:.1f}s")
    stream = torch.cuda.Stream()
    peak, peak_kind = measured_peaks()

    head = measure_stream(a, vsz, T, torch, names, shapes, xs, a.eb, stream, keep_tuned=True)
    bt, tuned, outs, heads = head.pop("_keep")
    kern, reps, sb = head.pop("_kern"), head.pop("_reps"), head.pop("_seq")

    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(local).uuid)
        if not uuid.startswith("GPU-"):
            uuid = "GPU-" + uuid
    except Exception:
        uuid = None
    sampler = ClockSampler(uuid) if rank == 0 else None
    time.sleep(0.3 if sampler else 0)
    # The headline: K replays of the tuned plan's compression graph.
    with torch.cuda.stream(stream):
        for _ in range(max(3, a.warmup)):
            bt.submit(stream)
    stream.synchronize()
    t0 = time.time()
    with torch.cuda.stream(stream):
        # ncu --nvtx --nvtx-include "vsz_headline/" selects the timed launches
        torch.cuda.nvtx.range_push("vsz_headline")
        ms_step = timed_loop(lambda: bt.submit(stream), stream)
        torch.cuda.nvtx.range_pop()
    t1 = time.time()
    clocks = sampler.summary(t0, t1) if sampler else None
    value = job_gbps(world, n_total, ms_step)
    launches = int(round(head["tuned_launches_per_step"] * a.steps))

    # roofline of the dominant class kernel (device time from the traced loop)
    cls_keys = [k for k in kern if k[0].startswith("batch_lorenzo")]
    dom = max(cls_keys, key=lambda k: kern[k]["ms"])
    dom_avg_s = kern[dom]["ms"] / kern[dom]["launches"] * 1e-3
    dom_bytes = sb["per_kernel"][dom]
    achieved = dom_bytes / dom_avg_s / 1e9
    kname = batch_kernel_name(dom)
    dom_vals = sum(f.n for f in tuned if class_key(f.p) == dom)
    roofline = {"bound": "hbm", "kernel": kname, "achieved": achieved, "peak": peak,
                "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs, copy bandwidth)" if peak_kind == "measured"
                else "fallback 6.8 TB/s", "unit": "GB/s", "frac": achieved / peak, "bytes_per_launch": dom_bytes,
                "values_per_launch": dom_vals,
                "traffic": profiled_traffic(kname, f"stream eb{a.eb:g} tuned", units=dom_vals)}
    step_frac = sb["total"] / (ms_step * 1e-3) / 1e9 / peak
    # the largest single launch of the step by device time (the range pass
    # over every value, for the relative error bound), beside the class kernel
    big = max(kern, key=lambda k: kern[k]["ms"])
    big_s = kern[big]["ms"] / kern[big]["launches"] * 1e-3
    big_bytes = sb["per_kernel"].get(big)
    largest = {"kernel": big[0], "share": kern[big]["ms"] / sum(v["ms"] for v in kern.values()),
               "us": big_s * 1e6, "achieved": big_bytes / big_s / 1e9 if big_bytes else None,
               "frac": big_bytes / big_s / 1e9 / peak if big_bytes else None}

    # e2e through the C ABI from host memory to host memory
    e2e = None
    if not a.no_e2e:
        hx = [torch.from_numpy(s[2]).pin_memory() for s in specs_host]
        caps = [(max(1024, int(h["n_out"])), max(1024, int(h["n_fix"]))) for h in heads]
        hout = bt.host_outputs(caps)
        bt.compress_host(hx, hout, stream)
        ke = max(3, min(a.steps, 10))
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(ke):
            hh = bt.compress_host(hx, hout, stream)
        e1.record(stream)
        e1.synchronize()
        barrier()
        ems = max_over_ranks(e0.elapsed_time(e1) / ke, dist, "cuda")
        d2h = sum(64 + 2 * f.n + 4 * (f.nb + 1) + 4 * f.p.pad_len + 8 * int(h["n_out"]) + 8 * int(h["n_fix"])
                  for f, h in zip(tuned, hh))
        e2e = {"value": job_gbps(world, n_total, ems), "unit": UNIT, "h2d_bytes_per_step": 4 * n_total,
               "d2h_bytes_per_step": d2h, "ms_per_step": ems,
               "what": "per step one vsz_batch_compress_host call: every field's input from page-locked host "
                       "memory to the device, the tuned plan's compression, every field's header, codes, block "
                       "offsets, padding table and exact-length outlier and fixup lists back to page-locked "
                       "host memory",
               "status_nonzero": sum(1 for h in hh if h["status"])}
        # the host link on its own (context for e2e): one 1 GiB copy each way
        # between page-locked memory and the device, on the same stream
        hb = torch.empty(1 << 28, dtype=torch.float32).pin_memory()
        db = torch.empty(1 << 28, dtype=torch.float32, device="cuda")
        link = {}
        for name, (dst, src) in (("h2d_GBps", (db, hb)), ("d2h_GBps", (hb, db))):
            with torch.cuda.stream(stream):
                dst.copy_(src, non_blocking=True)
                e0.record(stream)
                dst.copy_(src, non_blocking=True)
                e1.record(stream)
            e1.synchronize()
            link[name] = (1 << 30) / (e0.elapsed_time(e1) * 1e-3) / 1e9
        e2e["host_link"] = link
        del hb, db, hx, hout
    bt.close()
    del bt, tuned, outs
    torch.cuda.empty_cache()

    beside = measure_stream(a, vsz, T, torch, names, shapes, xs, a.eb_beside, stream)
    beside_kern, beside_seq = beside.pop("_kern"), beside.pop("_seq")
    beside.pop("_reps")
    bcls = [k for k in beside_kern if k[0].startswith("batch_lorenzo")]
    bdom = max(bcls, key=lambda k: beside_kern[k]["ms"])
    bavg = beside_kern[bdom]["ms"] / beside_kern[bdom]["launches"] * 1e-3
    beside["roofline"] = {"kernel": batch_kernel_name(bdom), "achieved": beside_seq["per_kernel"][bdom] / bavg / 1e9,
                          "peak": peak, "frac": beside_seq["per_kernel"][bdom] / bavg / 1e9 / peak}
    beside["step_hbm_frac"] = beside_seq["total"] / (beside["ms"]["batched_tuned"] * 1e-3) / 1e9 / peak
    del xs
    torch.cuda.empty_cache()

    one = sweep = entropy = None
    if not a.no_one_field:
        x3 = synth.lognormal3d(a.size, seed=rank_field_seed(rank))
        n = x3.size
        xd = torch.from_numpy(x3.reshape(-1)).cuda()
        one = run_one_field(a, vsz, torch, xd, x3, n, torch.cuda.current_stream(), timed_loop)
        if not a.no_sweep and rank == 0:
            sweep = run_sweep(a, vsz, torch, xd, x3, n)
        if not a.no_entropy and rank == 0:
            entropy = run_entropy(a, x3, xd)
        del xd

    # CPU baseline: the oracle on a bounded sample (rank 0, N = 1 only)
    cpu = None
    if rank == 0 and world == 1 and a.cpu_seconds > 0:
        v, elems, k, desc = oracle_stream_rate(specs_host, a.eb, a.cpu_seconds)
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc}
        pv, pthreads, _, pdesc = oracle_stream_rate_parallel(specs_host, a.eb, max(2.0, a.cpu_seconds / 2))
        cpu["host_parallel"] = {"value": pv, "unit": UNIT, "cores": pthreads, "cpu_model": cpu_model(),
                                "sample": pdesc}

    if sampler:
        sampler.stop()
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32/i32", "data": "synthetic", "config": workload_config(a),
            "roofline": roofline, "step_hbm_frac": step_frac, "largest_launch": largest, "cpu_baseline": cpu,
            "e2e": e2e,
            "clocks": clocks, "gpu_launches": launches,
            "plain_GBps": head["plain_GBps"], "tuned_vs_plain": head["tuned_vs_plain"],
            "stream": strip_private(head), f"stream_eb_{a.eb_beside:g}": strip_private(beside),
            "one_field": one, "sweep": sweep, "entropy": entropy,
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def run_batch_profile(a):
    """A reduced copy of the mixed stream (its first 4 fields of 1800x3600, its
    first 2 of 100x500x500, and the first 20M values of its 1D field: 96M
    values, 384 MB, larger than L2), the learned tuner's classes at eb --eb,
    one autotuned graph plan; `steps` compressions and reconstructions after
    `warmup`.  Prints one JSON line with the plan's GB/s and the per-class
    kernel times the autotuner measured.  A small case to run under ncu
    captures of the batch kernels (the full stream holds >10 GB on the
    device)."""
    import numpy as np
    import torch
    import paper_2201_04614_gb300 as vsz
    from paper_2201_04614_gb300 import tuner as T
    import synth
    specs = synth.cfg5_fields()
    pick = [s for s in specs if s[0].startswith("cesm2d_")][:4] + \
        [s for s in specs if s[0].startswith("hurricane3d_")][:2] + [s for s in specs if s[0].startswith("hacc1d_")]
    xs, shapes = [], []
    for name, sh, mk in pick:
        x = np.ascontiguousarray(mk(), np.float32).reshape(-1)
        if len(sh) == 1:
            x = np.ascontiguousarray(x[:20_000_000])
            sh = (x.size,)
        xs.append(torch.from_numpy(x).cuda())
        shapes.append(sh)
    picks = T.choose([(vsz.Params.make(sh, 8, a.eb, "rel", R, "zero"), x) for sh, x in zip(shapes, xs)])
    fields = make_stream_fields(vsz, T, shapes, [p["class"] for p in picks], a.eb)
    outs = [torch.empty(x.numel(), dtype=torch.float32, device="cuda") for x in xs]
    stream = torch.cuda.Stream()
    n = sum(x.numel() for x in xs)
    with torch.cuda.stream(stream):
        bt = vsz.Batch(fields, xs, use_graph=True)
        bt.set_outputs(outs)
        cls = bt.autotune(stream, reps=3)
        for _ in range(a.warmup):
            bt.submit(stream)
            bt.reconstruct(stream)
        stream.synchronize()
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        torch.cuda.nvtx.range_push("vsz_steps")  # ncu --nvtx --nvtx-include "vsz_steps/" selects these launches
        e0.record(stream)
        for _ in range(a.steps):
            bt.submit(stream)
        e1.record(stream)
        for _ in range(a.steps):
            bt.reconstruct(stream)
        e2.record(stream)
        torch.cuda.nvtx.range_pop()
        stream.synchronize()
    ms_c, ms_r = e0.elapsed_time(e1) / a.steps, e1.elapsed_time(e2) / a.steps
    heads = [f.header() for f in fields]
    line = {"batch_profile": f"4 x 1800x3600 + 2 x 100x500x500 + the first 20M values of the 1D field of the mixed "
                             f"stream, rel eb {a.eb:g}, the learned tuner's classes, autotuned graph plan",
            "values": n, "steps": a.steps, "compress_ms": ms_c, "reconstruct_ms": ms_r,
            "compress_GBps": n * 4 / ms_c / 1e6, "reconstruct_GBps": n * 4 / ms_r / 1e6,
            "status_nonzero": sum(int(h["status"] != 0) for h in heads),
            "n_out": sum(int(h["n_out"]) for h in heads),
            "classes": [{k: c[k] for k in ("kind", "ndim", "block", "pad_kind", "warps", "ctas_per_sm", "ms",
                                           "ms_default")} for c in cls if c["tiles"]],
            "class_values": {batch_kernel_name(k): v for k, v in
                             _class_values(fields).items()}}
    print(json.dumps(line), flush=True)
    bt.close()


def run_field_profile(a):
    """The one-field step alone on the NYX-like field of edge --size (block
    --block, rel eb --field-eb, padding --pad): `warmup` steps, then `steps`
    compressions and `steps` reconstructions inside the NVTX range
    "vsz_steps".  Prints one JSON line with the compression and
    reconstruction GB/s and the outlier counts."""
    import torch
    import paper_2201_04614_gb300 as vsz
    import synth
    x3 = synth.lognormal3d(a.size, seed=rank_field_seed(0))
    n = x3.size
    xd = torch.from_numpy(x3.reshape(-1)).cuda()
    p = vsz.Params.make(x3.shape, a.block, a.field_eb, "rel", R, a.pad)
    f = vsz.Field(p, out_cap=max(1 << 20, n // 4), fix_cap=max(1 << 16, n // 64))
    xh = torch.empty(n, dtype=torch.float32, device="cuda")
    for _ in range(a.warmup):
        f.compress(xd)
        f.reconstruct(out=xh)
    torch.cuda.synchronize()
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    torch.cuda.nvtx.range_push("vsz_steps")
    e0.record()
    for _ in range(a.steps):
        f.compress(xd)
    e1.record()
    for _ in range(a.steps):
        f.reconstruct(out=xh)
    e2.record()
    torch.cuda.nvtx.range_pop()
    e2.synchronize()
    h = f.header()
    ms_c, ms_r = e0.elapsed_time(e1) / a.steps, e1.elapsed_time(e2) / a.steps
    print(json.dumps({"field_profile": f"{a.size}^3 NYX-like, block {a.block}, rel eb {a.field_eb:g}, {a.pad}",
                      "values": n, "steps": a.steps, "compress_ms": ms_c, "reconstruct_ms": ms_r,
                      "compress_GBps": n * 4 / ms_c / 1e6, "reconstruct_GBps": n * 4 / ms_r / 1e6,
                      "n_out": int(h["n_out"]), "n_fix": int(h["n_fix"]), "status": int(h["status"])}), flush=True)


def _class_values(fields) -> dict:
    out = {}
    for f in fields:
        k = class_key(f.p)
        out[k] = out.get(k, 0) + f.n
    return out


def main():
    a = parse_args()
    if a.batch_profile:
        run_batch_profile(a)
        return
    if a.field_profile:
        run_field_profile(a)
        return
    if a.entropy_profile:
        import torch
        import synth
        x3 = synth.lognormal3d(a.size, seed=rank_field_seed(0))
        xd = torch.from_numpy(x3.reshape(-1)).cuda()
        print(json.dumps({"entropy_profile": f"{a.size}^3 NYX-like, block {a.block}, {a.pad}",
                          **run_entropy(a, x3, xd)}), flush=True)
        return
    if a.impl == "reference":
        run_reference(a)
    else:
        run_gpu(a)


if __name__ == "__main__":
    main()
