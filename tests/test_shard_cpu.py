"""A field split across ranks (paper_2201_04614_gb300.shard), on CPU ranks.

Blocks are independent (Sec. III-A), so slabs of whole blocks along dims[0]
compress independently once three quantities are exchanged: the value range
(relative eb, Sec. II-B), the q statistics of a global padding mode
(Sec. IV-B-1), and the list lengths, whose exclusive prefix places each
slab's lists.  Here every rank's per-slab steps run in the CPU oracle (a
backend object with the oracle's slab compression), the exchanges are gloo
collectives between two spawned ranks, and the concatenation of the ranks'
outputs must equal the oracle's whole-field compression bit for bit for
zero, block-average, global-average, global-minimum and edge padding, with
NaN and Inf in one slab.  The same host logic with the reductions done in
one process (compress_split_local) is checked over three emulated ranks.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import oracle  # noqa: E402
import synth  # noqa: E402
from paper_2201_04614_gb300 import shard  # noqa: E402

R = 16
CASES = [((27, 12, 20), 4, "zero"), ((27, 12, 20), 4, "block_avg"), ((27, 12, 20), 4, "global_avg"),
         ((50, 40), 8, "global_min"), ((50, 40), 8, "global_avg"), ((50, 40), 8, "edge_avg"),
         ((19, 9, 11), 4, "edge_min")]


def _field(dims):
    if len(dims) == 2:
        x = synth.fourier2d(dims[0], dims[1], seed=7, value_range=30.0, offset=-4.0)
    else:
        x = np.exp(synth.grf3d(dims, 8)).astype(np.float32) * np.float32(20.0)
    x = np.ascontiguousarray(x, np.float32)
    flat = x.reshape(-1)
    flat[-5] = np.nan  # non-finite values in the last slab: outside the range, kept as fixups
    flat[-17] = np.inf
    return x


class OracleSlab:
    """The per-rank steps of one slab in the CPU oracle."""

    def __init__(self, job, x):
        self.job, self.x = job, np.ascontiguousarray(x, np.float32).reshape(-1)

    def _p(self, eb_abs):
        return oracle.Params(self.job.slab_dims, self.job.block, eb_abs, oracle.EB_ABS, self.job.radius, self.job.pad)

    def value_range(self):
        fin = self.x[np.isfinite(self.x)]
        return (float(fin.min()), float(fin.max()), True) if fin.size else (0.0, 0.0, False)

    def qstats(self, eb_abs):
        e = oracle.resolve_eb(self._p(eb_abs), self.x)
        q = oracle.prequant(self.x, e.inv2eb).astype(np.int64)
        return int(q.sum()), int(q.size), int(q.min()), int(q.max())

    def compress(self, eb_abs, P):
        return oracle.compress_given_pad(self._p(eb_abs), self.x, P)

    def counts(self, c):
        return len(c.out_idx), len(c.fix_idx)

    def rebase(self, c, elem_base, out_base):
        c.out_idx = c.out_idx + np.uint32(elem_base)
        c.fix_idx = c.fix_idx + np.uint32(elem_base)
        c.blk_off = c.blk_off + np.uint32(out_base)


def _job(dims, block, pad, world, rank):
    z0, z1 = shard.slab_bounds(dims, block, world, rank)
    return shard.SlabJob(tuple(dims), block, 1e-3, shard.EB_REL, R, oracle.PAD_NAMES[pad], z0, z1)


def _concat(parts):
    """The field's outputs from the ranks' slab outputs, in rank order."""
    return {
        "codes": np.concatenate([c.codes for c in parts]),
        "blk_off": np.concatenate([c.blk_off[:-1] for c in parts] + [parts[-1].blk_off[-1:]]),
        "out_idx": np.concatenate([c.out_idx for c in parts]),
        "out_delta": np.concatenate([c.out_delta for c in parts]),
        "fix_idx": np.concatenate([c.fix_idx for c in parts]),
        "fix_bits": np.concatenate([c.fix_bits for c in parts]),
        "pad": np.concatenate([c.pad for c in parts]),
    }


def _check_against_whole(dims, block, pad, parts, eb_abs):
    x = _field(dims)
    po = oracle.Params(dims, block, 1e-3, oracle.EB_REL, R, oracle.PAD_NAMES[pad])
    c = oracle.compress(po, x)
    assert eb_abs == c.eb.eb_abs
    got = _concat(parts)
    for k in ("codes", "blk_off", "out_idx", "out_delta", "fix_idx", "fix_bits"):
        assert np.array_equal(got[k], getattr(c, k)), (dims, pad, k)
    if po.is_block_pad or po.is_edge_pad:
        assert np.array_equal(got["pad"], c.pad), (dims, pad)
    assert len(c.out_idx) > 0 and len(c.fix_idx) >= 2  # the lists are exercised


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ex = shard.Exchange(dist, "cpu")
        for i, (dims, block, pad) in enumerate(CASES):
            job = _job(dims, block, pad, world, rank)
            x = _field(dims)
            r = shard.compress_split(ex, OracleSlab(job, x[job.z0:job.z1]), job)
            gathered = [None] * world
            dist.all_gather_object(gathered, (r["result"], r["eb_abs"], r["pad"], r["out_base"], r["n_out_total"]))
            if rank == 0:
                try:
                    _check_against_whole(dims, block, pad, [g[0] for g in gathered], r["eb_abs"])
                    assert [g[4] for g in gathered] == [sum(len(g[0].out_idx) for g in gathered)] * world
                    out[i] = "ok"
                except AssertionError as e:  # reported to the parent
                    out[i] = f"fail: {e!r}"
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_equal_the_whole_field():
    world = 2
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res == {i: "ok" for i in range(len(CASES))}, res


@pytest.mark.parametrize("dims,block,pad", CASES)
def test_three_emulated_ranks_equal_the_whole_field(dims, block, pad):
    world = 3
    x = _field(dims)
    jobs = [_job(dims, block, pad, world, r) for r in range(world)]
    backends = [OracleSlab(j, x[j.z0:j.z1]) for j in jobs]
    res = shard.compress_split_local(backends, jobs)
    _check_against_whole(dims, block, pad, [r["result"] for r in res], res[0]["eb_abs"])


def test_slab_bounds_and_reductions():
    # whole blocks, every row covered once, earlier ranks take the extra block
    for n0, b, w in ((27, 4, 2), (27, 4, 3), (8, 8, 3), (100, 8, 7), (1, 4, 2)):
        bounds = [shard.slab_bounds((n0, 5), b, w, r) for r in range(w)]
        assert bounds[0][0] == 0 and bounds[-1][1] == n0
        assert all(bounds[i][1] == bounds[i + 1][0] for i in range(w - 1))
        assert all(z0 % b == 0 or z0 == n0 for z0, _ in bounds)  # empty slabs sit at the end
        sizes = [-(-(z1 - z0) // b) for z0, z1 in bounds]
        assert max(sizes) - min(sizes) <= 1 and sizes == sorted(sizes, reverse=True)
    # value-range relative eb (reading R1): eb * range in double, eb for a zero or empty range
    assert shard.field_eb_abs(1e-3, shard.EB_REL, -2.5, 7.5, True) == 1e-3 * 10.0
    assert shard.field_eb_abs(1e-3, shard.EB_REL, 3.0, 3.0, True) == 1e-3
    assert shard.field_eb_abs(1e-3, shard.EB_REL, 0.0, 0.0, False) == 1e-3
    assert shard.field_eb_abs(0.25, shard.EB_ABS, -9.0, 9.0, True) == 0.25
    # rounded mean half up with floor division (reading R3), min and max
    assert shard.global_pad(shard.PAD_GLOBAL_AVG, 5, 2, 0, 9) == 3      # 2.5 -> 3
    assert shard.global_pad(shard.PAD_GLOBAL_AVG, -5, 2, 0, 9) == -2    # -2.5 -> -2
    assert shard.global_pad(shard.PAD_GLOBAL_AVG, -7, 3, 0, 9) == -2    # -2.33 -> -2
    assert shard.global_pad(shard.PAD_GLOBAL_MIN, 0, 4, -3, 9) == -3
    assert shard.global_pad(shard.PAD_GLOBAL_MAX, 0, 4, -3, 9) == 9
    assert shard.global_pad(shard.PAD_GLOBAL_AVG, 0, 0, 0, 0) == 0
    assert shard.exclusive_prefix([3, 0, 5, 1]) == [0, 3, 3, 8]
