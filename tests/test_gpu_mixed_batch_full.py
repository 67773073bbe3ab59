"""GPU parity of the batch path at full size, in the launch configuration the
batch plans run in (one plan, autotuned launch shapes, replayed as a CUDA
graph; compression, then reconstruction of every field):

* the mixed batch: 79 CESM-shaped 2D fields (1800x3600, per-field range
  log-uniform in [1e-3, 1e3]), 13 Hurricane-shaped 3D fields (100x500x500)
  and 4 HACC-like 1D fields of 10M random-walk values, 876,920,000 values
  (3.5 GB); relative eb 1e-4, R = 512, zero padding, the default blocks
  (16x16, 8^3, 256);
* the mixed stream: one 1D field of 280,953,867 random-walk values, 13 fields
  of 100x500x500 and 20 of 1800x3600, 735,553,867 values (2.94 GB); relative
  eb 1e-3 and 1e-5, R = 512, block size and padding per field from the
  learned tuner.

Every field is compared bit for bit with the oracle (Sec. III-A: codes,
block offsets, outliers and fixups in canonical order, the resolved error
bound, and the decompressed values).  The oracle runs on the host's hardware
threads, one field per task (ctypes releases the interpreter lock inside the
C oracle)."""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle  # noqa: E402
import paper_2201_04614_gb300 as vsz  # noqa: E402
from paper_2201_04614_gb300 import tuner as T  # noqa: E402

R = 512
DEFAULT_BLOCK = {1: 256, 2: 16, 3: 8}
THREADS = min(16, os.cpu_count() or 1)
CASES = {
    "mixed_batch_eb1e-4_default": (synth.cfg3_fields, 1e-4, False,
                                   79 * 1800 * 3600 + 13 * 100 * 500 * 500 + 4 * 10_000_000),
    "mixed_stream_eb1e-3_tuner": (synth.cfg5_fields, 1e-3, True, 280_953_867 + 13 * 100 * 500 * 500 + 20 * 1800 * 3600),
    "mixed_stream_eb1e-5_tuner": (synth.cfg5_fields, 1e-5, True, 280_953_867 + 13 * 100 * 500 * 500 + 20 * 1800 * 3600),
}


@pytest.fixture(scope="module", params=list(CASES))
def batch(request):
    make, eb, use_tuner, total = CASES[request.param]
    specs = make()
    assert sum(int(np.prod(s)) for _, s, _ in specs) == total
    with ThreadPoolExecutor(THREADS) as ex:
        xs_host = list(ex.map(lambda sp: np.ascontiguousarray(sp[2](), np.float32).reshape(-1), specs))
    oracle.build()
    xs = [torch.from_numpy(x).cuda() for x in xs_host]
    shapes = [sh for _, sh, _ in specs]
    if use_tuner:
        picks = T.choose([(vsz.Params.make(sh, 8, eb, "rel", R, "zero"), x) for sh, x in zip(shapes, xs)])
        params = [T.class_params(len(sh), p["class"]) for sh, p in zip(shapes, picks)]
    else:
        params = [(DEFAULT_BLOCK[len(sh)], "zero") for sh in shapes]
    fields, outs = [], []
    for sh, (b, pad), x in zip(shapes, params, xs):
        n = x.numel()
        fields.append(vsz.Field(vsz.Params.make(sh, b, eb, "rel", R, pad), out_cap=n,
                                fix_cap=max(1 << 16, n // 64)))
        outs.append(torch.empty(n, dtype=torch.float32, device="cuda"))
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        bt = vsz.Batch(fields, xs, use_graph=True)
        bt.set_outputs(outs)
        bt.autotune(stream=stream)
        bt.submit()
        bt.reconstruct()
    stream.synchronize()
    yield request.param, specs, eb, params, xs_host, fields, outs
    bt.close()
    del bt, fields, outs, xs
    torch.cuda.empty_cache()


def test_every_field_matches_oracle(batch):
    case, specs, eb, params, xs_host, fields, outs = batch

    def run_oracle(i):
        sh = specs[i][1]
        b, pad = params[i]
        po = oracle.Params(sh, b, eb, oracle.EB_REL, R, oracle.PAD_NAMES[pad])
        c = oracle.compress(po, xs_host[i])
        return c, oracle.decompress(po, c).view(np.uint32)

    with ThreadPoolExecutor(THREADS) as ex:
        for i, (c, xo) in enumerate(ex.map(run_oracle, range(len(specs)))):
            name = (case, specs[i][0], params[i])
            got = fields[i].to_host()
            h = got["header"]
            assert h["status"] == 0 and h["recon_status"] == 0, name
            assert h["eb_abs"] == c.eb.eb_abs, name
            assert np.float32(h["inv2eb"]) == c.eb.inv2eb and np.float32(h["ebx2"]) == c.eb.ebx2, name
            for k in ("codes", "blk_off", "out_idx", "out_delta", "fix_idx", "fix_bits"):
                assert np.array_equal(got[k], getattr(c, k)), (name, k)
            if got["pad"] is not None and got["pad"].size == c.pad.size:  # per-block tables
                assert np.array_equal(got["pad"], c.pad), name
            assert np.array_equal(outs[i].cpu().numpy().view(np.uint32), xo), name
