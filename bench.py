#!/usr/bin/env python
"""Benchmark of the dual-quantization hot path on GB300.

Workload: one NYX-like fp32 field of 512^3 values (exp of a seeded Gaussian
random field with a k^-3 spectrum), blocks of 8^3, radius R = 512, value-range
relative eb = 1e-4, zero padding.  One step is the whole path over the field:
compression (on-device eb resolution from the value range, fused
prequantization + Lorenzo + post-quantization + guard, outlier compaction)
followed by reconstruction.  The metric is GB/s of fp32 input per step.

    python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Under torchrun every rank compresses its own 512^3 field (blocks are
independent, so the path shards with no collective on the data path: weak
scaling); rank 0 prints one JSON line.  `--impl reference` times the CPU
oracle (the plain single-threaded C implementation) on bounded samples of
the same workload instead.
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


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    ap.add_argument("--size", type=int, default=512, help="edge of the cubic field")
    ap.add_argument("--eb", type=float, default=1e-4)
    ap.add_argument("--pad", default="zero")
    ap.add_argument("--block", type=int, default=8)
    ap.add_argument("--radius", type=int, default=512)
    ap.add_argument("--no-sweep", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-batch", action="store_true", help="skip the batched+tuned vs plain comparison")
    ap.add_argument("--batch-steps", type=int, default=20)
    ap.add_argument("--no-entropy", action="store_true", help="skip the Huffman stage and rate-distortion curve")
    ap.add_argument("--batch-profile", action="store_true",
                    help="only a reduced mixed batch (6 CESM-shaped 2D, 2 Hurricane-shaped 3D and one 10M 1D "
                         "field, default classes, eb 1e-4): a small case for ncu captures of the batch kernels")
    return ap.parse_args()


def workload_config(a) -> dict:
    return {
        "workload": f"NYX-like log-normal fp32 {a.size}^3 (exp of k^-3 GRF, seed 2), block {a.block}^3, "
                    f"R={a.radius}, rel eb {a.eb:g}, {a.pad} padding: compress (range + fused "
                    f"prequant/Lorenzo/post-quant + compaction) then reconstruct",
        "field_elems": a.size ** 3, "block": a.block, "radius": a.radius, "eb_rel": a.eb, "pad": a.pad,
        "l2": "inputs larger than L2 (512 MiB field vs 129 MB L2); no flush needed",
        "step": "compress + reconstruct through the library's calls, captured once as a CUDA graph and "
                "replayed (value); eager and traced loops of the same steps are reported beside it",
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
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "100"]
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
        if not self.samples:
            return None
        win = [p for (t, p) in self.samples if t0 <= t <= t1] or [p for (_, p) in self.samples]

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
    """Each rank compresses its own field: blocks (and fields) are
    independent, so the path shards with no collective on the data path."""
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
    if name == "range" or name == "qstats":
        return 4 * n
    if name == "lorenzo":   # x in; codes, staged outliers/fixups, block offsets (+ pads) out
        return 4 * n + 2 * n + 8 * (n_out + n_fix) + 4 * nb + (4 * nb if block_pad else 0)
    if name == "compact_move":  # staged entries in and out, block offsets read-modify-write
        return 16 * (n_out + n_fix) + 8 * nb
    if name == "recon":     # codes, outliers, block offsets (+ pads) in; values out
        return 2 * n + 8 * n_out + 4 * (nb + 1) + (4 * nb if block_pad else 0) + 4 * n
    if name == "fixups":
        return 12 * n_fix
    return 0


# The source files that define each profiled kernel (its body, the headers
# it includes and its launcher): a committed ncu figure holds while these
# files are unchanged.
KERNEL_SOURCES = {
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


def profiled_traffic(kernel: str, workload: str) -> int | None:
    """dram bytes per launch from a committed ncu summary, if it was taken on
    the current sources of that kernel."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            tab = json.load(f)
    except Exception:
        return None
    ent = tab.get(f"{kernel}|{workload}")
    if not ent or ent.get("src_digest") != kernel_sources_digest(kernel):
        return None
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
    done, elems, t_used, k = 0, 0, 0.0, 0
    while True:
        z0 = (k * unit_planes) % nz
        y0 = ((k * unit_planes) // nz * rows) % ny
        sl = np.ascontiguousarray(x3[z0:z0 + unit_planes, y0:y0 + rows, :])
        p = oracle.Params(sl.shape, a.block, a.eb, oracle.EB_REL, a.radius, pad)
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
            p = oracle.Params(sl.shape, a.block, a.eb, oracle.EB_REL, a.radius, pad)
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


def run_reference(a):
    """The oracle, as it stands, on the host cores: each step one bounded
    sample of the workload."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import numpy as np
    import synth
    x3 = synth.cfg2_field(a.size)
    # size one step so that warmup + steps take about a minute
    probe, _, _, _ = oracle_rate(x3, a, 0.0, 8, 64)
    unit_s = (8 * 64 * x3.shape[2] * 4 / 1e9) / probe
    per_step_units = max(1, min(64, int(60.0 / max(1, a.steps + a.warmup) / unit_s)))
    rows = min(x3.shape[1], 64 * per_step_units)
    for _ in range(a.warmup):
        oracle_rate(x3, a, 0.0, 8, rows)
    t = time.perf_counter()
    elems = 0
    for _ in range(a.steps):
        _, e, _, desc = oracle_rate(x3, a, 0.0, 8, rows)
        elems += e
    dt = time.perf_counter() - t
    value = elems * 4 / dt / 1e9
    sample = (f"each step: one block-aligned slab of 8x{rows}x{x3.shape[2]} of the {a.size}^3 field, "
              f"compressed and decompressed by the single-threaded oracle")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": a.gpus,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": dt / a.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32/i32",
        "data": "synthetic", "config": workload_config(a),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- batched + tuned vs plain
def run_batch_compare(a, log_fn=log) -> dict:
    """The mixed stream of fields (one 1D field of 280,953,867 random-walk
    values, 13 fields of 100x500x500, 20 of 1800x3600; relative eb 1e-3 and
    1e-5, R = 512).  Compression: plain per-field launches with the default
    class (block 256 / 8 / 16, zero padding), the same launches replayed as
    one CUDA graph, one batch plan with the default classes (default launch
    shapes, then autotuned shapes), and one batch plan with the tuner's
    classes and autotuned shapes.  Reconstruction: plain per-field launches
    and the batch plans.  Outlier counts per field for the tuner's and the
    default classes.  Every list has room for every element, so no field
    overflows (status 0)."""
    import numpy as np
    import torch
    import paper_2201_04614_gb300 as vsz
    from paper_2201_04614_gb300 import tuner as T
    import synth

    t0 = time.time()
    specs = synth.cfg5_fields()
    xs, shapes, names = [], [], []
    for name, shape, maker in specs:
        xs.append(torch.from_numpy(np.ascontiguousarray(maker(), np.float32).reshape(-1)).cuda())
        shapes.append(shape)
        names.append(name)
    n_total = sum(x.numel() for x in xs)
    log_fn(f"[bench] batch stream: {len(xs)} fields, {n_total} values, generated in {time.time() - t0:.1f}s")
    steps = max(5, min(a.batch_steps, 50))
    stream = torch.cuda.Stream()
    outs = [torch.empty(x.numel(), dtype=torch.float32, device="cuda") for x in xs]

    def timed(fn):
        with torch.cuda.stream(stream):
            for _ in range(3):
                fn()
            stream.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(steps):
                fn()
            e1.record(stream)
            stream.synchronize()
        return e0.elapsed_time(e1) / steps

    def make_fields(classes, eb):
        out = []
        for shape, c in zip(shapes, classes):
            b, pad = T.class_params(len(shape), c)
            n = int(np.prod(shape))
            out.append(vsz.Field(vsz.Params.make(shape, b, eb, "rel", 512, pad), out_cap=n, fix_cap=max(1 << 16, n // 64)))
        return out

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

    res = {"workload": "1D 280,953,867 random walk + 13 x 100x500x500 GRF + 20 x 1800x3600 Fourier fields "
                       "(2.94 GB fp32), relative eb, R=512", "values": n_total, "steps": steps, "by_eb": {}}
    gb = n_total * 4 / 1e9
    for eb in (1e-3, 1e-5):
        r = {}
        dflt = [T.default_class(len(sh)) for sh in shapes]
        plain = make_fields(dflt, eb)

        def plain_step():
            for f, x in zip(plain, xs):
                f.compress(x)
        r["plain"] = timed(plain_step)
        # the same per-field launches captured once into a CUDA graph
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(stream):
            plain_step()
            stream.synchronize()
            with torch.cuda.graph(g, stream=stream):
                plain_step()
        r["plain_graph"] = timed(g.replay)
        del g

        def plain_recon():
            for f, o in zip(plain, outs):
                f.reconstruct(out=o)
        r["plain_recon"] = timed(plain_recon)
        nout_def = [int(f.header()["n_out"]) for f in plain]
        st_def = [int(f.header()["status"]) for f in plain]
        bd = vsz.Batch(plain, xs, use_graph=True)
        bd.set_outputs(outs)
        r["batched_default"] = timed(lambda: bd.submit(stream))
        r["batched_default_recon"] = timed(lambda: bd.reconstruct(stream))
        bd.close()
        del bd
        bda, cls_def, at_def_ms = autotuned(plain)
        r["batched_default_autotuned"] = timed(lambda: bda.submit(stream))
        r["batched_default_autotuned_recon"] = timed(lambda: bda.reconstruct(stream))
        bda.close()
        del bda
        # the tuner's classes: features, one MLP inference, guard (timed on its own)
        torch.cuda.synchronize()
        tt = time.time()
        picks = T.choose([(vsz.Params.make(sh, 8, eb, "rel", 512, "zero"), x) for sh, x in zip(shapes, xs)])
        torch.cuda.synchronize()
        tune_ms = (time.time() - tt) * 1e3
        classes = [p["class"] for p in picks]
        tuned = make_fields(classes, eb)
        bt, cls_tuned, at_tuned_ms = autotuned(tuned)
        r["batched_tuned"] = timed(lambda: bt.submit(stream))
        r["batched_tuned_recon"] = timed(lambda: bt.reconstruct(stream))
        bt.close()
        nout_tuned = [int(f.header()["n_out"]) for f in tuned]
        st_tuned = [int(f.header()["status"]) for f in tuned]
        del bt
        # the paper's own autotuner (Sec. III-D) as the baseline of the learned
        # one: per field, the block size whose dual-quant is fastest on a 5 %
        # sample (zero padding), then the same batch plan with autotuned shapes
        torch.cuda.synchronize()
        tt = time.time()
        samp = [T.sampling_autotune(vsz.Params.make(sh, 8, eb, "rel", 512, "zero"), x, 0.05, 3)
                for sh, x in zip(shapes, xs)]
        samp_ms = (time.time() - tt) * 1e3
        slots = {1: (32, 64, 128, 256), 2: (8, 16, 32, 64), 3: (8, 16, 32)}
        samp_cls = [3 * slots[len(sh)].index(r["block"]) for sh, r in zip(shapes, samp)]
        sampf = make_fields(samp_cls, eb)
        bs, cls_samp, at_samp_ms = autotuned(sampf)
        r["batched_sampling_tuned"] = timed(lambda: bs.submit(stream))
        r["batched_sampling_tuned_recon"] = timed(lambda: bs.reconstruct(stream))
        bs.close()
        del bs
        nout_samp = [int(f.header()["n_out"]) for f in sampf]
        st_samp = [int(f.header()["status"]) for f in sampf]
        res["by_eb"][f"{eb:g}"] = {
            **{f"{k}_GBps": gb / (v * 1e-3) for k, v in r.items()},
            "ms": r,
            "tune_ms_once": tune_ms, "autotune_ms_once": {"default": at_def_ms, "tuned": at_tuned_ms},
            "shapes_default_classes": shapes_of(cls_def), "shapes_tuned_classes": shapes_of(cls_tuned),
            "classes_tuned": {nm: T.class_params(len(sh), c) for nm, sh, c in zip(names, shapes, classes)
                              if c != T.default_class(len(sh))},
            "guard_fallbacks": sum(1 for p in picks if p["class"] != p["predicted"]),
            "n_out_default_total": sum(nout_def), "n_out_tuned_total": sum(nout_tuned),
            "fields_n_out_tuned_le_default": sum(1 for u, v in zip(nout_tuned, nout_def) if u <= v),
            "sampling_autotuner": {"tune_ms_once": samp_ms, "n_out_total": sum(nout_samp),
                                   "blocks": {nm: rr["block"] for nm, rr in zip(names, samp)}},
            "fields": len(xs), "status_nonzero": sum(1 for v in st_def + st_tuned + st_samp if v),
        }
        log_fn(f"[bench] batch eb={eb:g}: " + json.dumps({k: v for k, v in res["by_eb"][f"{eb:g}"].items()
                                                          if k.endswith("GBps") or k.startswith("n_out")
                                                          or k == "status_nonzero"}))
        del plain, tuned, sampf
        torch.cuda.empty_cache()
    del xs, outs
    torch.cuda.empty_cache()
    return res


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
        p = vsz.Params.make(x3.shape, a.block, eb, "rel", a.radius, a.pad)
        f = vsz.Field(p, out_cap=n // 2, fix_cap=max(1 << 16, n // 64))
        f.compress(xd)
        f.reconstruct(out=xh)
        h = f.header()
        nsym = 2 * a.radius
        hist = f.code_histogram()
        book = vsz.HuffmanBook(hist, nsym)
        words, off, st = vsz.huffman_encode(f.codes, n, book)
        nwords = int(off[-1].item())
        dec, st2 = vsz.huffman_decode(words, off, n, book)
        ok = int(st.item()) == 0 and int(st2.item()) == 0 and bool(torch.equal(dec[:n], f.codes[:n]))
        nc = off.numel() - 1
        table_bits = 32 * (p.nblocks + 1) + 64 * (nc + 1) + 32 * p.pad_len
        bits = 32 * nwords + 64 * int(h["n_out"]) + 64 * int(h["n_fix"]) + table_bits
        mse = float(((xh.double() - xd.double()) ** 2).mean().item())
        psnr = 20 * math.log10(vrange) - 10 * math.log10(mse) if mse > 0 else float("inf")
        row = {"eb": eb, "bits_per_value": bits / n, "ratio": 32.0 * n / bits, "huffman_bits_per_value": 32 * nwords / n,
               "psnr_db": psnr, "n_out": int(h["n_out"]), "n_fix": int(h["n_fix"]), "round_trip_ok": ok}
        if eb == a.eb:
            ms_hist = ev_ms(lambda: f.code_histogram(out=hist))
            ms_book = ev_ms(lambda: vsz.HuffmanBook(hist, nsym))
            ms_enc = ev_ms(lambda: vsz.huffman_encode(f.codes, n, book, words=words))
            ms_dec = ev_ms(lambda: vsz.huffman_decode(words, off, n, book, out=dec))
            # bytes each pass must move: encode reads the codes twice (bit
            # counts, then packing) and writes the stream; decode reads the
            # stream and writes the codes
            enc_bytes, dec_bytes = 4 * n + 4 * nwords, 4 * nwords + 2 * n
            vsz.trace_enable(True)
            vsz.trace_read()
            vsz.huffman_encode(f.codes, n, book, words=words)
            vsz.huffman_decode(words, off, n, book, out=dec)
            vsz.trace_enable(False)
            kern = {r["name"]: round(r["ms"] * 1e3, 1) for r in vsz.trace_read(64)}
            row["timing"] = {
                "histogram_us": ms_hist * 1e3, "book_us": ms_book * 1e3,
                "encode_us": ms_enc * 1e3, "decode_us": ms_dec * 1e3,
                "encode_GBps_fp32_in": 4 * n / (ms_enc * 1e-3) / 1e9, "decode_GBps_fp32_out": 4 * n / (ms_dec * 1e-3) / 1e9,
                "encode_hbm_GBps": enc_bytes / (ms_enc * 1e-3) / 1e9, "decode_hbm_GBps": dec_bytes / (ms_dec * 1e-3) / 1e9,
                "kernels_us_one_call": kern}
        out["curve"].append(row)
        log_fn(f"[bench] entropy eb={eb:g}: {row}")
        del f, book, words, off, dec
        torch.cuda.empty_cache()
    return out


# ---------------------------------------------------------------- GPU arm
def run_gpu(a):
    import numpy as np
    import torch
    import paper_2201_04614_gb300 as vsz
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

    vsz.lib()
    t = time.time()
    x3 = synth.lognormal3d(a.size, seed=rank_field_seed(rank))
    log(f"[bench] rank {rank}: generated {a.size}^3 field in {time.time() - t:.1f}s")
    n = x3.size
    p = vsz.Params.make(x3.shape, a.block, a.eb, "rel", a.radius, a.pad)
    f = vsz.Field(p, out_cap=max(1 << 20, n // 8), fix_cap=max(1 << 16, n // 64))
    xd = torch.from_numpy(x3.reshape(-1)).cuda()
    xh = torch.empty(n, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

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

    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(local).uuid)
        if not uuid.startswith("GPU-"):
            uuid = "GPU-" + uuid
    except Exception:
        uuid = None
    sampler = ClockSampler(uuid) if rank == 0 else None
    time.sleep(0.3 if sampler else 0)

    # The step captured once as a CUDA graph (the library's calls are
    # asynchronous and capturable) and replayed K times: the headline.
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

    t0 = time.time()
    with torch.cuda.stream(gstream):
        ms_step = timed_loop(graph.replay, gstream)
    t1 = time.time()
    value = job_gbps(world, n, ms_step)
    # the same steps as eager API calls (no events inside)
    ms_eager = timed_loop(step, stream)
    # and again with events around every launch: the per-kernel durations
    vsz.trace_enable(True)
    vsz.trace_read()
    ms_traced = timed_loop(step, stream)
    vsz.trace_enable(False)
    recs = vsz.trace_read(1 << 20)
    del graph

    # per-kernel device times, and the roofline of the dominant kernel
    per = {}
    for r in recs:
        d = per.setdefault(r["name"], {"launches": 0, "ms": 0.0})
        d["launches"] += 1
        d["ms"] += max(0.0, r["ms"])
    nb = p.nblocks
    bp = p.is_block_pad
    peak, peak_kind = measured_peaks()
    kernels = {}
    step_bytes = 0
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
    wl = f"{a.size}^3 b{a.block} eb{a.eb:g} {a.pad}"
    roofline = {"bound": "hbm", "kernel": kname, "achieved": achieved, "peak": peak,
                "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs, copy bandwidth)" if peak_kind == "measured"
                else "fallback 6.8 TB/s", "unit": "GB/s", "frac": achieved / peak,
                "bytes_per_launch": dom_bytes, "traffic": profiled_traffic(kname, wl)}
    step_frac = step_bytes / (ms_step * 1e-3) / 1e9 / peak
    clocks = sampler.summary(t0, t1) if sampler else None

    # e2e through the public API with host buffers, pipelined across steps:
    # every step copies its input in from pinned host memory, compresses,
    # reconstructs and copies its whole result out (codes, block offsets,
    # outlier and fixup lists, header, x_hat); two sets of device and host
    # buffers let step k's copies out overlap step k+1's copy in and compute
    # (one stream per direction, one for compute)
    e2e = None
    if not a.no_e2e:
        hx = torch.from_numpy(x3.reshape(-1)).pin_memory()
        fe = [f, vsz.Field(p, out_cap=f.out_cap, fix_cap=f.fix_cap)]
        xds, xhs = [xd, torch.empty_like(xd)], [xh, torch.empty_like(xh)]
        pin = lambda t: torch.empty(t.numel(), dtype=t.dtype).pin_memory()
        hcodes = [pin(fe[0].codes), pin(fe[0].codes)]
        hblk = [pin(fe[0].blk_off), pin(fe[0].blk_off)]
        hoi = [pin(fe[0].out_idx), pin(fe[0].out_idx)]
        hod = [pin(fe[0].out_delta), pin(fe[0].out_delta)]
        hfi = [pin(fe[0].fix_idx), pin(fe[0].fix_idx)]
        hfb = [pin(fe[0].fix_bits), pin(fe[0].fix_bits)]
        hxh = [pin(xh), pin(xh)]
        s_in, s_cmp, s_out = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
        ev_in = [torch.cuda.Event(), torch.cuda.Event()]
        ev_cmp = [torch.cuda.Event(), torch.cuda.Event()]
        ev_out = [torch.cuda.Event(), torch.cuda.Event()]
        for evs in (ev_cmp, ev_out):
            for ev in evs:
                ev.record(s_out)
        ke = max(3, min(a.steps, 20))
        d2h = []

        def enqueue_in_compute(k):
            b = k % 2
            s_in.wait_event(ev_cmp[b])  # the input buffer's last reader is done
            with torch.cuda.stream(s_in):
                xds[b].copy_(hx, non_blocking=True)
            ev_in[b].record(s_in)
            s_cmp.wait_event(ev_in[b])
            s_cmp.wait_event(ev_out[b])  # the result buffers' last copies out are done
            fe[b].compress(xds[b], stream=s_cmp)
            fe[b].reconstruct(out=xhs[b], stream=s_cmp)
            ev_cmp[b].record(s_cmp)

        def enqueue_out(k):
            b = k % 2
            s_out.wait_event(ev_cmp[b])
            hd = fe[b].header(stream=s_out)  # the list lengths (synchronizes the out stream)
            no, nf = int(hd["n_out"]), int(hd["n_fix"])
            with torch.cuda.stream(s_out):
                hcodes[b].copy_(fe[b].codes, non_blocking=True)
                hblk[b].copy_(fe[b].blk_off, non_blocking=True)
                hoi[b][:no].copy_(fe[b].out_idx[:no], non_blocking=True)
                hod[b][:no].copy_(fe[b].out_delta[:no], non_blocking=True)
                hfi[b][:nf].copy_(fe[b].fix_idx[:nf], non_blocking=True)
                hfb[b][:nf].copy_(fe[b].fix_bits[:nf], non_blocking=True)
                hxh[b].copy_(xhs[b], non_blocking=True)
            ev_out[b].record(s_out)
            d2h.append(64 + 2 * n + 4 * (nb + 1) + 8 * no + 8 * nf + 4 * n)

        def run(steps):
            enqueue_in_compute(0)
            for k in range(steps):
                if k + 1 < steps:
                    enqueue_in_compute(k + 1)
                enqueue_out(k)
            s_out.synchronize()

        run(2)
        barrier()
        d2h.clear()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(s_in)
        run(ke)
        e1.record(s_out)
        e1.synchronize()
        barrier()
        ems = max_over_ranks(e0.elapsed_time(e1) / ke, dist, "cuda")
        e2e = {"value": job_gbps(world, n, ems), "unit": UNIT, "h2d_bytes_per_step": 4 * n,
               "d2h_bytes_per_step": int(sum(d2h) / len(d2h)), "ms_per_step": ems,
               "what": "per step: pinned host x -> device, compress, reconstruct, header + codes + blk_off + "
                       "outlier and fixup lists + x_hat -> pinned host; steps pipelined on three streams "
                       "(copy in, compute, copy out) with double buffers"}
        del hx, fe, xds, xhs, hcodes, hblk, hoi, hod, hfi, hfb, hxh

    # eb x padding sweep (separate short runs, outside the timed region)
    sweep = None
    if not a.no_sweep and rank == 0:
        sweep = []
        # the GPU idled at lower clocks during the host-bound legs before:
        # bring it back to speed before the first configuration is timed
        ps0 = vsz.Params.make(x3.shape, a.block, 1e-2, "rel", a.radius, "zero")
        f0 = vsz.Field(ps0, out_cap=n // 4, fix_cap=max(1 << 16, n // 64))
        for _ in range(50):
            f0.compress(xd)
            f0.reconstruct(out=xh)
        torch.cuda.synchronize()
        del f0
        for eb in (1e-2, 1e-3, 1e-4, 1e-5):
            for pad in ("zero", "block_avg", "global_avg", "edge_avg"):
                ps = vsz.Params.make(x3.shape, a.block, eb, "rel", a.radius, pad)
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
                sweep.append({"eb": eb, "pad": pad, "compress_GBps": n * 4 / (tc / k * 1e-3) / 1e9,
                              "reconstruct_GBps": n * 4 / (tr / k * 1e-3) / 1e9,
                              "n_out": int(hs["n_out"]), "n_fix": int(hs["n_fix"]), "status": int(hs["status"])})
                del fs
                torch.cuda.empty_cache()

    entropy = None
    if not a.no_entropy and rank == 0:
        entropy = run_entropy(a, x3, xd)

    batched = None
    if not a.no_batch and rank == 0:
        del xh
        torch.cuda.empty_cache()
        batched = run_batch_compare(a)

    # CPU baseline: the oracle on a bounded sample (rank 0, N = 1 only)
    cpu = None
    if rank == 0 and world == 1 and a.cpu_seconds > 0:
        v, elems, k, desc = oracle_rate(x3, a, a.cpu_seconds)
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc}
        pv, pthreads, _, pdesc = oracle_rate_parallel(x3, a, max(2.0, a.cpu_seconds / 2))
        cpu["host_parallel"] = {"value": pv, "unit": UNIT, "cores": pthreads, "cpu_model": cpu_model(),
                                "sample": pdesc}

    if sampler:
        sampler.stop()
    launches = sum(d["launches"] for d in per.values())
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "eager": {"GBps": job_gbps(world, n, ms_eager), "ms_per_step": ms_eager},
            "traced": {"GBps": job_gbps(world, n, ms_traced), "ms_per_step": ms_traced,
                       "what": "the same eager steps with two CUDA events around every launch; "
                               "the kernels' durations and the roofline come from this loop"},
            "vs_baseline": None, "dtype": "f32/i32", "data": "synthetic", "config": workload_config(a),
            "roofline": roofline, "step_hbm_frac": step_frac, "cpu_baseline": cpu, "e2e": e2e,
            "clocks": clocks, "gpu_launches": launches, "kernels": kernels,
            "outliers": {"n_out": n_out, "n_fix": n_fix, "frac_out": n_out / n},
            "compress_GBps": n * 4 / (sum(per[k]["ms"] for k in ("begin", "range", "lorenzo", "compact_scan",
                                                                  "compact_move") if k in per)
                                      / a.steps * 1e-3) / 1e9,
            "reconstruct_GBps": n * 4 / (sum(per[k]["ms"] for k in ("recon", "fixups") if k in per)
                                         / a.steps * 1e-3) / 1e9,
            "sweep": sweep, "entropy": entropy, "batched": batched,
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def run_batch_profile(a):
    """A reduced copy of the 96-field mixed batch (the first 6 of its 1800x3600
    fields, the first 2 of its 100x500x500 fields and the first of its 10M 1D
    fields: 98,880,000 values, 396 MB, larger than L2), default classes, rel eb
    1e-4, one autotuned graph plan; `steps` compressions and reconstructions
    after `warmup`.  Prints one JSON line with the per-class kernel times the
    autotuner measured and the plan's GB/s.  A small case to run under ncu
    captures of the batch kernels (the full batches hold >10 GB on the
    device)."""
    import numpy as np
    import torch
    import paper_2201_04614_gb300 as vsz
    import synth
    specs = synth.cfg3_fields()
    pick = [s for s in specs if s[0].startswith("cesm2d_")][:6] + \
        [s for s in specs if s[0].startswith("hurricane3d_")][:2] + [s for s in specs if s[0].startswith("hacc1d_")][:1]
    blocks = {1: 256, 2: 16, 3: 8}
    xs = [torch.from_numpy(np.ascontiguousarray(mk(), np.float32).reshape(-1)).cuda() for _, _, mk in pick]
    fields = [vsz.Field(vsz.Params.make(sh, blocks[len(sh)], 1e-4, "rel", 512, "zero"), out_cap=x.numel(),
                        fix_cap=max(1 << 16, x.numel() // 64)) for (_, sh, _), x in zip(pick, xs)]
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
        e0.record(stream)
        for _ in range(a.steps):
            bt.submit(stream)
        e1.record(stream)
        for _ in range(a.steps):
            bt.reconstruct(stream)
        e2.record(stream)
        stream.synchronize()
    ms_c, ms_r = e0.elapsed_time(e1) / a.steps, e1.elapsed_time(e2) / a.steps
    bad = sum(int(f.header()["status"] != 0) for f in fields)
    line = {"batch_profile": "6 x 1800x3600 + 2 x 100x500x500 + 1 x 10M of the mixed batch, rel eb 1e-4, zero "
                             "padding, default blocks, autotuned graph plan",
            "values": n, "steps": a.steps, "compress_ms": ms_c, "reconstruct_ms": ms_r,
            "compress_GBps": n * 4 / ms_c / 1e6, "reconstruct_GBps": n * 4 / ms_r / 1e6, "status_nonzero": bad,
            "classes": [{k: c[k] for k in ("kind", "ndim", "block", "warps", "ctas_per_sm", "ms", "ms_default")}
                        for c in cls if c["tiles"]]}
    print(json.dumps(line), flush=True)
    bt.close()


def main():
    a = parse_args()
    if a.batch_profile:
        run_batch_profile(a)
        return
    if a.impl == "reference":
        run_reference(a)
    else:
        run_gpu(a)


if __name__ == "__main__":
    main()
