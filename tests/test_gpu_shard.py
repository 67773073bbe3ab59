"""The per-rank steps of a field split across GPUs, on one GPU: three
emulated ranks run vsz_slab_range, vsz_slab_qstats, vsz_compress_slab and
vsz_slab_rebase (through paper_2201_04614_gb300.shard.GpuSlabBackend) one
after another, the reductions between them done in the process
(compress_split_local); the concatenation of the slabs' outputs must equal
the oracle's whole-field compression bit for bit (Sec. III-A: blocks are
independent), and each slab's own reconstruction the oracle's values."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle  # noqa: E402
from paper_2201_04614_gb300 import shard  # noqa: E402

R = 64
CASES = [((45, 30, 70), 8, "zero"), ((45, 30, 70), 8, "block_avg"), ((45, 30, 70), 8, "global_avg"),
         ((200, 390), 16, "global_max"), ((200, 390), 16, "edge_avg"), ((33, 17, 20), 4, "global_avg"),
         ((1000, 33), 32, "block_min")]


def _field(dims):
    if len(dims) == 2:
        x = synth.fourier2d(dims[0], dims[1], seed=11, value_range=50.0, offset=3.0)
    else:
        x = np.exp(synth.grf3d(dims, 12)).astype(np.float32) * np.float32(7.0)
    x = np.ascontiguousarray(x, np.float32)
    flat = x.reshape(-1)
    flat[-3] = np.nan
    flat[11] = -np.inf
    return x


@pytest.mark.parametrize("dims,block,pad", CASES)
@pytest.mark.parametrize("eb", [1e-3, 1e-5])
def test_split_field_equals_whole_field(dims, block, pad, eb):
    world = 3
    x = _field(dims)
    jobs = []
    for r in range(world):
        z0, z1 = shard.slab_bounds(dims, block, world, r)
        jobs.append(shard.SlabJob(tuple(dims), block, eb, shard.EB_REL, R, oracle.PAD_NAMES[pad], z0, z1))
    backends = [shard.GpuSlabBackend(j, torch.from_numpy(np.ascontiguousarray(x[j.z0:j.z1]).reshape(-1)).cuda())
                for j in jobs]
    res = shard.compress_split_local(backends, jobs)
    fields = [r["result"] for r in res]
    host = [f.to_host() for f in fields]
    po = oracle.Params(dims, block, eb, oracle.EB_REL, R, oracle.PAD_NAMES[pad])
    c = oracle.compress(po, x)
    assert res[0]["eb_abs"] == c.eb.eb_abs
    got = {
        "codes": np.concatenate([h["codes"] for h in host]),
        "blk_off": np.concatenate([h["blk_off"][:-1] for h in host] + [host[-1]["blk_off"][-1:]]),
        "out_idx": np.concatenate([h["out_idx"] for h in host]),
        "out_delta": np.concatenate([h["out_delta"] for h in host]),
        "fix_idx": np.concatenate([h["fix_idx"] for h in host]),
        "fix_bits": np.concatenate([h["fix_bits"] for h in host]),
    }
    for k in got:
        assert np.array_equal(got[k], getattr(c, k)), k
    if po.is_block_pad or po.is_edge_pad:
        assert np.array_equal(np.concatenate([h["pad"] for h in host]), c.pad)
    if pad.startswith("global"):
        assert all(int(h["header"]["pad_global"]) == int(c.pad[0]) for h in host)
    assert len(c.out_idx) > 0 and len(c.fix_idx) >= 2
    # the first slab (element and list bases 0, so its rebased lists are
    # still its own) reconstructs on its own, from its header's eb and P, to
    # the oracle's values
    xo = oracle.decompress(po, c).view(np.uint32)
    n0 = fields[0].n
    assert np.array_equal(fields[0].reconstruct()[:n0].cpu().numpy().view(np.uint32), xo[:n0])
