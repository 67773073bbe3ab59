"""GPU tests of the batch path (vsz_batch_*): every field's outputs must be
identical to compressing (reconstructing) that field alone with vsz_compress
(vsz_reconstruct), which the parity tests tie to the oracle, and the batch
reconstruction is also checked against the oracle's decompression."""
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
       ((12, 20, 68), 16, 1e-5, "rel", 16, "block_min"), ((150, 260), 16, 1e-4, "rel", 512, "edge_avg"),
       ((13, 21, 140), 8, 1e-4, "rel", 64, "edge_min"), ((7000,), 64, 1e-4, "rel", 512, "edge_max")]


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


def _outs(fields):
    return [torch.full((max(1, f.n),), float("nan"), dtype=torch.float32, device="cuda") for f in fields]


def _assert_recon(fields, outs, want, what):
    for i, f in enumerate(fields):
        if f.n:
            got = outs[i][: f.n].cpu().numpy().view(np.uint32)
            assert np.array_equal(got, want[i]), (what, MIX[i])
            assert f.header()["recon_status"] == 0, (what, MIX[i])


@pytest.mark.parametrize("use_graph", [False, True])
def test_batch_reconstruct_equals_per_field_and_oracle(use_graph):
    fields, xs = _make()
    outs = _outs(fields)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        b = vsz.Batch(fields, xs, use_graph=use_graph)
        b.set_outputs(outs)
        b.submit()
        b.reconstruct()
        b.reconstruct()  # a replay gives the same values
    stream.synchronize()
    kinds = [c["kind"] for c in b.classes()]
    assert 0 in kinds and 1 in kinds
    want = []
    for i, f in enumerate(fields):
        if not f.n:
            want.append(None)
            continue
        single = f.reconstruct().cpu().numpy().view(np.uint32)
        dims, blk, eb, mode, R, pad = MIX[i]
        po = oracle.Params(dims, blk, eb, oracle.EB_REL if mode == "rel" else oracle.EB_ABS, R, oracle.PAD_NAMES[pad])
        x = xs[i].cpu().numpy()
        xo = oracle.decompress(po, oracle.compress(po, x)).view(np.uint32)
        assert np.array_equal(single, xo), MIX[i]
        want.append(xo)
    _assert_recon(fields, outs, want, "batch")
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


def _scramble(fields):
    for f in fields:
        for t in (f.codes, f.blk_off, f.out_idx, f.out_delta, f.fix_idx, f.fix_bits, f.pad):
            if t is not None:
                t.fill_(-7)


def _assert_same(fields, want, what):
    for i, (f, w) in enumerate(zip(fields, want)):
        got = _host(f)
        for k in KEYS:
            if w[k] is not None:
                assert np.array_equal(got[k], w[k]), (what, MIX[i], k)
        for k in ("pad_global", "n_out", "n_fix", "status"):
            assert got["header"][k] == w["header"][k], (what, MIX[i], k)


def test_launch_shapes_and_autotune_change_no_result():
    """Every launch shape of the class kernels (warps per CTA, CTAs per SM),
    the concurrent mode and the autotuner's choice give the same outputs."""
    fields, xs = _make()
    outs = _outs(fields)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        b = vsz.Batch(fields, xs, use_graph=True)
        b.set_outputs(outs)
        b.submit()
        b.reconstruct()
    stream.synchronize()
    want = [_host(f) for f in fields]
    rwant = [o[: f.n].cpu().numpy().view(np.uint32).copy() if f.n else None for f, o in zip(fields, outs)]
    cls = b.classes()
    comp = [c for c in cls if c["kind"] == 0]
    assert len(comp) >= 6 and sum(c["nfields"] for c in comp) == len(MIX)
    assert sum(c["nfields"] for c in cls if c["kind"] == 1) == sum(1 for f in fields if f.n)
    assert {(c["ndim"], c["pad_kind"]) for c in comp} >= {(1, 0), (2, 1), (3, 2)}

    def run_and_check(what):
        _scramble(fields)
        for o in outs:
            o.fill_(float("nan"))
        with torch.cuda.stream(stream):
            b.submit()
            b.reconstruct()
        stream.synchronize()
        _assert_same(fields, want, what)
        _assert_recon(fields, outs, rwant, what)

    for warps, ctas in ((2, 1), (8, 0), (4, 2), (8, 1), (2, 0)):
        for c in range(len(cls)):
            try:
                b.set_shape(c, warps, ctas)
            except vsz.VszError as e:  # shared memory of 8 warps of 3D blocks of 32
                assert e.status == 2 and warps == 8
        run_and_check((warps, ctas))
    for c in range(len(cls)):
        b.set_shape(c, 0, 0)
    b.set_concurrent(True)
    for _ in range(2):  # capture, then replay
        run_and_check("concurrent")
    tuned = b.autotune(stream, reps=2)
    assert len(tuned) == len(cls)
    for c in tuned:
        if c["tiles"]:
            assert c["warps"] in (0, 2, 4, 8) and c["ctas_per_sm"] >= 0
            assert 0 < c["ms"] <= c["ms_default"]
    for _ in range(2):
        run_and_check("autotuned")
    with pytest.raises(vsz.VszError):
        b.set_shape(0, 3, 0)
    with pytest.raises(vsz.VszError):
        b.set_shape(len(cls), 4, 0)
    b.close()


def test_autotune_cache_round_trip(tmp_path):
    """Shapes found by the autotuner are recorded per GPU model and class, and
    a later plan with the same classes takes them without searching."""
    fields, xs = _make()
    outs = _outs(fields)
    cache = str(tmp_path / "shapes.json")
    stream = torch.cuda.Stream()
    b1 = vsz.Batch(fields, xs, use_graph=True)
    b1.set_outputs(outs)
    tuned = b1.autotune(stream, reps=1, cache=cache)
    assert all(c["ms"] > 0 for c in tuned if c["tiles"])  # searched: timings recorded
    b2 = vsz.Batch(fields, xs, use_graph=True)
    b2.set_outputs(outs)
    loaded = b2.autotune(stream, reps=1, cache=cache)
    assert all(c["ms"] == 0 for c in loaded)  # not searched again
    assert [(c["warps"], c["ctas_per_sm"]) for c in loaded] == [(c["warps"], c["ctas_per_sm"]) for c in tuned]
    with torch.cuda.stream(stream):
        b1.submit()
    stream.synchronize()
    want = [_host(f) for f in fields]
    _scramble(fields)
    with torch.cuda.stream(stream):
        b2.submit()
    stream.synchronize()
    _assert_same(fields, want, "cached shapes")
    b1.close()
    b2.close()


def test_allocation_failure_injection():
    """Each device allocation that batch creation and vsz_batch_set_outputs
    make for their tables can fail (injected on the host): the call raises
    VSZ_ERR_CUDA after releasing what it had allocated, the library stays
    usable, and a plan built afterwards gives the per-field results."""
    L = vsz.lib()
    fields, xs = _make()
    ref_fields, _ = _make()
    for f, x in zip(ref_fields, xs):
        f.compress(x)
    want = [_host(f) for f in ref_fields]
    failed = 0
    try:
        for k in range(1, 200):
            assert L.vsz_debug_fail_alloc(k) == 0
            try:
                b = vsz.Batch(fields, xs, use_graph=False)
            except vsz.VszError as e:
                assert e.status == 4
                failed += 1
                continue
            break
        else:
            raise AssertionError("creation never succeeded")
        assert failed >= 1
        outs = _outs(fields)
        failed_out = 0
        for k in range(1, 200):
            assert L.vsz_debug_fail_alloc(k) == 0
            try:
                b.set_outputs(outs)
            except vsz.VszError as e:
                assert e.status == 4
                failed_out += 1
                continue
            break
        assert failed_out >= 1
    finally:
        assert L.vsz_debug_fail_alloc(0) == 0
    b.submit()
    b.reconstruct()
    torch.cuda.synchronize()
    for i, (f, w) in enumerate(zip(fields, want)):
        got = _host(f)
        for key in ("codes", "blk_off", "out_idx", "out_delta"):
            assert np.array_equal(got[key], w[key]), (MIX[i], key)
        if f.n:
            single = f.reconstruct().cpu().numpy().view(np.uint32)
            assert np.array_equal(outs[i][: f.n].cpu().numpy().view(np.uint32), single), MIX[i]
    b.close()


@pytest.mark.parametrize("use_graph", [False, True])
def test_compress_host_equals_device_outputs(use_graph):
    """vsz_batch_compress_host: host inputs in, host outputs out, identical to
    what the plan leaves in device memory, with the lists at their exact
    lengths; twice in a row, the second time from different host inputs."""
    fields, xs = _make()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        b = vsz.Batch(fields, xs, use_graph=use_graph)
    hout = b.host_outputs()
    for shift in (0, 7):
        hx = [torch.from_numpy(np.ascontiguousarray(
            (field_for(dims, seed=50 + i + shift).reshape(-1) if int(np.prod(dims)) else np.zeros(0)), np.float32))
            .pin_memory() for i, (dims, *_rest) in enumerate(MIX)]
        heads = b.compress_host(hx, hout, stream)
        ref, _ = _make(seed_shift=shift)
        for f, x in zip(ref, hx):
            f.compress(x.cuda())
        for i, (f, o, h) in enumerate(zip(ref, hout, heads)):
            w = f.to_host()
            no, nf = int(w["header"]["n_out"]), int(w["header"]["n_fix"])
            assert h["n_out"] == no and h["n_fix"] == nf and h["status"] == 0, MIX[i]
            assert h["eb_abs"] == w["header"]["eb_abs"], MIX[i]
            assert np.array_equal(o["codes"].numpy()[: f.n].view(np.uint16), w["codes"]), MIX[i]
            assert np.array_equal(o["blk_off"].numpy()[: f.nb + 1].view(np.uint32), w["blk_off"]), MIX[i]
            if w["pad"] is not None and f.p.pad_len:
                assert np.array_equal(o["pad"].numpy()[: w["pad"].size], w["pad"]), MIX[i]
            assert np.array_equal(o["out_idx"].numpy()[:no].view(np.uint32), w["out_idx"]), MIX[i]
            assert np.array_equal(o["out_delta"].numpy()[:no], w["out_delta"]), MIX[i]
            assert np.array_equal(o["fix_idx"].numpy()[:nf].view(np.uint32), w["fix_idx"]), MIX[i]
            assert np.array_equal(o["fix_bits"].numpy()[:nf].view(np.uint32), w["fix_bits"]), MIX[i]
    b.close()
