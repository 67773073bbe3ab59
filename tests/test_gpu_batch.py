"""GPU tests of the batch path (vsz_batch_*): every field's outputs must be
identical to compressing that field alone with vsz_compress, which the
parity tests tie to the oracle."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle  # noqa: E402
import paper_2201_04614_gb300 as vsz  # noqa: E402

KEYS = ("codes", "pad", "blk_off", "out_idx", "out_delta", "fix_idx", "fix_bits")


def field_for(dims, seed):
    if len(dims) == 1:
        return synth.random_walk1d(dims[0], seed)
    if len(dims) == 2:
        return synth.fourier2d(dims[0], dims[1], seed=seed, value_range=20.0, offset=5.0)
    return np.exp(synth.grf3d(dims, seed))


MIX = [((300, 519), 16, 1e-4, "rel", 512, "zero"), ((160, 384), 8, 1e-5, "rel", 64, "block_avg"),
       ((19, 37, 260), 8, 1e-4, "rel", 512, "zero"), ((17, 23, 29), 8, 1e-3, "abs", 32, "global_avg"),
       ((10007,), 256, 1e-5, "rel", 512, "zero"), ((5000,), 32, 1e-4, "rel", 8, "block_max"),
       ((64, 64), 16, 1e-4, "rel", 512, "zero"), ((0,), 16, 1e-3, "rel", 512, "zero"),
       ((3, 1, 5), 4, 1e-2, "rel", 512, "global_min"), ((1, 700), 32, 1e-4, "abs", 2, "block_avg"),
       ((12, 20, 68), 16, 1e-5, "rel", 16, "block_min")]


def _host(f):
    return f.to_host()


def _make(seed_shift=0):
    fields, xs = [], []
    for i, (dims, b, eb, mode, R, pad) in enumerate(MIX):
        x = field_for(dims, seed=50 + i + seed_shift).reshape(-1) if int(np.prod(dims)) else np.zeros(0, np.float32)
        x = np.ascontiguousarray(x, np.float32)
        n = max(1, x.size)
        fields.append(vsz.Field(vsz.Params.make(dims, b, eb, mode, R, pad), out_cap=n, fix_cap=n))
        xs.append(torch.from_numpy(x).cuda())
    return fields, xs


@pytest.mark.parametrize("use_graph", [False, True])
def test_batch_equals_per_field(use_graph):
    fields, xs = _make()
    ref_fields, _ = _make()
    for f, x in zip(ref_fields, xs):
        f.compress(x)
    want = [_host(f) for f in ref_fields]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        b = vsz.Batch(fields, xs, use_graph=use_graph)
        b.submit()
        b.submit()  # a replay must give the same result
    stream.synchronize()
    for i, (f, w) in enumerate(zip(fields, want)):
        got = _host(f)
        for k in KEYS:
            if w[k] is None:
                assert got[k] is None
            else:
                assert np.array_equal(got[k], w[k]), (MIX[i], k)
        for k in ("eb_abs", "inv2eb", "ebx2", "eb_f32", "pad_global", "n_out", "n_fix", "status"):
            assert got["header"][k] == w["header"][k], (MIX[i], k)
    b.close()


def test_batch_replay_with_new_inputs():
    """The plan (and its graph) keeps the input pointers: new values written
    into the same buffers are compressed by the next submit."""
    fields, xs = _make()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        b = vsz.Batch(fields, xs, use_graph=True)
        b.submit()
    stream.synchronize()
    new = []
    for i, (dims, *_rest) in enumerate(MIX):
        if int(np.prod(dims)):
            v = np.ascontiguousarray(field_for(dims, seed=900 + i).reshape(-1), np.float32)
            xs[i].copy_(torch.from_numpy(v))
            new.append(v)
        else:
            new.append(np.zeros(0, np.float32))
    with torch.cuda.stream(stream):
        b.submit()
    stream.synchronize()
    for i, (dims, blk, eb, mode, R, pad) in enumerate(MIX):
        po = oracle.Params(dims, blk, eb, oracle.EB_REL if mode == "rel" else oracle.EB_ABS, R, oracle.PAD_NAMES[pad])
        c = oracle.compress(po, new[i])
        got = fields[i].to_host()
        assert np.array_equal(got["codes"], c.codes), MIX[i]
        assert np.array_equal(got["out_idx"], c.out_idx), MIX[i]
        assert np.array_equal(got["out_delta"], c.out_delta), MIX[i]
        assert np.array_equal(got["fix_idx"], c.fix_idx), MIX[i]
    b.close()
