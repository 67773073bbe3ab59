"""GPU parity: the CUDA path (called through the C ABI) against the CPU oracle,
element by element on the same seeded inputs.

Integer work is compared bit-exactly: codes, per-block padding values, block
offsets, outlier indices and residuals, fixup indices and bits, the
reconstructed prequantized integers.  Reconstructed values are compared bit
for bit too (both sides evaluate the same IEEE fp32 product), and the error
bound |x - x_hat| <= eb (1 + 2^-20) is checked on every finite element.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle  # noqa: E402
import paper_2201_04614_gb300 as vsz  # noqa: E402

PADS = ["zero", "global_min", "global_max", "global_avg", "block_min", "block_max", "block_avg",
        "edge_min", "edge_max", "edge_avg"]


def run_both(x, dims, block, eb, eb_mode="rel", radius=512, pad="zero", out_cap=None, fix_cap=None):
    x = np.ascontiguousarray(x, np.float32).reshape(-1)
    p = vsz.Params.make(dims, block, eb, eb_mode, radius, pad)
    n = max(1, x.size)
    f = vsz.Field(p, out_cap=out_cap or n, fix_cap=fix_cap or n)
    xd = torch.from_numpy(x).cuda()
    f.compress(xd)
    qg = f.reconstruct_q().cpu().numpy()
    xg = f.reconstruct().cpu().numpy()
    po = oracle.Params(tuple(dims), block, eb, oracle.EB_REL if eb_mode == "rel" else oracle.EB_ABS,
                       radius, oracle.PAD_NAMES[pad])
    c = oracle.compress(po, x)
    xo, qo = oracle.decompress(po, c, return_q=True)
    return f, c, (qg, xg), (qo, xo), x


def assert_parity(f, c, g, o, x, pad):
    got = f.to_host()
    h = got["header"]
    assert h["recon_status"] == 0
    # error-bound resolution (Sec. II-B) and padding value (Sec. IV)
    assert h["eb_abs"] == c.eb.eb_abs
    assert np.float32(h["inv2eb"]) == c.eb.inv2eb
    assert np.float32(h["ebx2"]) == c.eb.ebx2
    assert np.float32(h["eb_f32"]) == c.eb.eb_f32
    if pad.startswith("global") or pad == "zero":
        assert h["pad_global"] == int(c.pad[0])
    else:
        assert np.array_equal(got["pad"], c.pad)
    assert np.array_equal(got["codes"], c.codes)
    assert np.array_equal(got["blk_off"], c.blk_off)
    assert np.array_equal(got["out_idx"], c.out_idx)
    assert np.array_equal(got["out_delta"], c.out_delta)
    assert np.array_equal(got["fix_idx"], c.fix_idx)
    assert np.array_equal(got["fix_bits"], c.fix_bits)
    qg, xg = g
    qo, xo = o
    assert np.array_equal(qg, c.q)          # prequantized values, via the inverse
    assert np.array_equal(qo, c.q)
    assert np.array_equal(xg.view(np.uint32), xo.view(np.uint32))
    fin = np.isfinite(x)
    err = np.abs(x[fin].astype(np.float64) - xg[fin].astype(np.float64))
    assert (err <= c.eb.eb_abs * (1 + 2.0 ** -20)).all()
    assert np.array_equal(x[~fin].view(np.uint32), xg[~fin].view(np.uint32))


CASES_1D = [((10007,), b) for b in (4, 32, 256)] + [((4096 * 3,), 128), ((77,), 8)]
CASES_2D = [((300, 519), 16), ((160, 384), 16), ((130, 260), 4), ((70, 300), 64), ((129, 257), 128),
            ((33, 1000), 8), ((1, 700), 32), ((700, 3), 16)]
CASES_3D = [((19, 37, 260), 8), ((17, 23, 29), 8), ((9, 10, 140), 4), ((20, 18, 132), 16),
            ((33, 35, 70), 32), ((8, 8, 128), 8), ((3, 1, 5), 4)]


def field_for(dims, seed):
    if len(dims) == 1:
        return synth.random_walk1d(dims[0], seed)
    if len(dims) == 2:
        return synth.fourier2d(dims[0], dims[1], seed=seed, value_range=20.0, offset=5.0)
    return np.exp(synth.grf3d(dims, seed))


@pytest.mark.parametrize("dims,block", CASES_1D + CASES_2D + CASES_3D)
@pytest.mark.parametrize("pad", PADS)
def test_parity_shapes_pads(dims, block, pad):
    x = field_for(dims, seed=len(dims) * 100 + block)
    for eb in (1e-2, 1e-5):
        f, c, g, o, xx = run_both(x, dims, block, eb, "rel", 512, pad)
        assert_parity(f, c, g, o, xx, pad)


@pytest.mark.parametrize("radius", [1, 2, 32768])
@pytest.mark.parametrize("dims,block", [((5000,), 64), ((90, 130), 16), ((12, 20, 68), 8)])
def test_parity_radius_extremes(dims, block, radius):
    x = field_for(dims, seed=7)
    for pad in ("zero", "block_avg", "global_max", "edge_avg"):
        f, c, g, o, xx = run_both(x, dims, block, 1e-4, "rel", radius, pad)
        assert_parity(f, c, g, o, xx, pad)


@pytest.mark.parametrize("dims,block", [((6000,), 16), ((60, 100), 8), ((10, 15, 40), 4)])
@pytest.mark.parametrize("eb_abs", [0.5, 1e-3, 3e-7])
def test_parity_adversarial(dims, block, eb_abs):
    n = int(np.prod(dims))
    x = synth.adversarial_values(n, seed=3, inv2eb=1.0 / (2 * eb_abs))
    for pad in PADS:
        f, c, g, o, xx = run_both(x, dims, block, eb_abs, "abs", 512, pad, out_cap=n, fix_cap=n)
        assert len(c.fix_idx) > 0
        assert_parity(f, c, g, o, xx, pad)


def test_parity_all_nan_and_constant():
    for x in (np.full(3000, np.nan, np.float32), np.full(3000, 2.5, np.float32)):
        for pad in ("zero", "block_avg", "global_avg", "edge_avg"):
            f, c, g, o, xx = run_both(x, (50, 60), 16, 1e-3, "rel", 512, pad, out_cap=3000, fix_cap=3000)
            assert_parity(f, c, g, o, xx, pad)


def test_empty_field():
    p = vsz.Params.make((0,), 16, 1e-3)
    f = vsz.Field(p)
    f.compress(torch.empty(0, dtype=torch.float32, device="cuda"))
    h = f.header()
    assert h["n_out"] == 0 and h["n_fix"] == 0 and h["status"] == 0
    assert f.reconstruct().numel() == 0
    p2 = vsz.Params.make((0, 17), 16, 1e-3, pad="block_avg")
    f2 = vsz.Field(p2)
    f2.compress(torch.empty(0, dtype=torch.float32, device="cuda"))
    assert f2.header()["n_out"] == 0


def test_capacity_overflow_reports_exact_counts():
    dims = (100, 200)
    x = field_for(dims, seed=11)
    p = vsz.Params.make(dims, 8, 1e-6, "rel", 4, "zero")
    po = oracle.Params(dims, 8, 1e-6, oracle.EB_REL, 4, oracle.PAD_ZERO)
    c = oracle.compress(po, x)
    assert len(c.out_idx) > 50
    f = vsz.Field(p, out_cap=10, fix_cap=10)
    f.compress(torch.from_numpy(x.reshape(-1)).cuda())
    h = f.header()
    assert h["status"] == 3  # VSZ_ERR_CAPACITY
    assert f.sync_status() == 3
    assert h["n_out"] == len(c.out_idx)
    assert np.array_equal(f.blk_off.cpu().numpy().view(np.uint32), c.blk_off)
    # retry with room: exact parity
    f2 = vsz.Field(p, out_cap=int(h["n_out"]), fix_cap=max(1, int(h["n_fix"])))
    f2.compress(torch.from_numpy(x.reshape(-1)).cuda())
    got = f2.to_host()
    assert np.array_equal(got["out_idx"], c.out_idx) and np.array_equal(got["codes"], c.codes)


def test_corrupt_outlier_list_is_reported():
    dims = (64, 64)
    x = field_for(dims, seed=12)
    p = vsz.Params.make(dims, 16, 1e-6, "rel", 8, "zero")
    f = vsz.Field(p)
    f.compress(torch.from_numpy(x.reshape(-1)).cuda())
    h = f.header()
    assert h["n_out"] > 0
    f.out_idx[0] += 1  # the first outlier no longer matches its code 0
    f.reconstruct()
    assert f.header()["recon_status"] == 5
    assert f.sync_status() == 5


def test_code_histogram_matches_codes():
    dims = (200, 300)
    x = field_for(dims, seed=13)
    p = vsz.Params.make(dims, 16, 1e-4, "rel", 64, "zero")
    f = vsz.Field(p)
    f.compress(torch.from_numpy(x.reshape(-1)).cuda())
    hist = f.code_histogram().cpu().numpy()
    codes = f.to_host()["codes"]
    assert np.array_equal(hist, np.bincount(codes, minlength=128)[:128])


def test_split_calls_equal_fused_call():
    dims = (50, 70, 36)
    x = field_for(dims, seed=14)
    p = vsz.Params.make(dims, 8, 1e-5, "rel", 512, "block_avg")
    xd = torch.from_numpy(x.reshape(-1)).cuda()
    f1, f2 = vsz.Field(p), vsz.Field(p)
    f1.compress(xd)
    f2.prequant_lorenzo(xd)
    f2.outlier_compact()
    a, b = f1.to_host(), f2.to_host()
    for k in ("codes", "pad", "blk_off", "out_idx", "out_delta"):
        assert np.array_equal(a[k], b[k]), k


def test_repeated_calls_reuse_workspace():
    dims = (40, 300)
    p = vsz.Params.make(dims, 16, 1e-5, "rel", 32, "global_avg")
    f = vsz.Field(p)
    for seed in (21, 22, 23):
        x = field_for(dims, seed)
        f.compress(torch.from_numpy(x.reshape(-1)).cuda())
        c = oracle.compress(oracle.Params(dims, 16, 1e-5, oracle.EB_REL, 32, oracle.PAD_GLOBAL_AVG), x)
        got = f.to_host()
        assert np.array_equal(got["out_idx"], c.out_idx) and np.array_equal(got["codes"], c.codes)


GUARD = 4096


def _guarded(n, dtype, fill):
    t = torch.full((n + GUARD,), fill, dtype=dtype, device="cuda")
    return t, t[:n]


@pytest.mark.parametrize("dims,block", [((260,), 4), ((1000,), 256), ((130, 260), 4), ((33, 130), 16),
                                        ((17, 259), 8), ((9, 11, 132), 8), ((5, 7, 133), 4),
                                        ((12, 40, 200), 32)])
@pytest.mark.parametrize("pad", ["zero", "block_avg", "global_max"])
def test_no_writes_past_outputs(dims, block, pad):
    """Every output buffer is followed by a guard region filled with a
    sentinel; compression and reconstruction must leave it untouched."""
    x = field_for(dims, seed=31)
    x = np.ascontiguousarray(x, np.float32).reshape(-1)
    n = x.size
    p = vsz.Params.make(dims, block, 1e-5, "rel", 8, pad)
    f = vsz.Field(p, out_cap=n, fix_cap=n)
    nb = p.nblocks
    codes_g, f.codes = _guarded(n, torch.int16, 0x5A5A)
    blk_g, f.blk_off = _guarded(nb + 1, torch.int32, 0x5A5A5A5A)
    f._cc.codes = f.codes.data_ptr()
    f._cc.blk_off = f.blk_off.data_ptr()
    if f.pad is not None:
        pad_g, f.pad = _guarded(nb, torch.int32, 0x5A5A5A5A)
        f._cc.pad = f.pad.data_ptr()
    f.compress(torch.from_numpy(x).cuda())
    xh_g, xh = _guarded(n, torch.float32, 1234.5)
    q_g, qv = _guarded(n, torch.int32, 0x5A5A5A5A)
    f.reconstruct(out=xh)
    f.reconstruct_q(out=qv)
    torch.cuda.synchronize()
    assert (codes_g[n:] == 0x5A5A).all()
    assert (blk_g[nb + 1:] == 0x5A5A5A5A).all()
    if f.pad is not None:
        assert (pad_g[nb:] == 0x5A5A5A5A).all()
    assert (xh_g[n:] == 1234.5).all()
    assert (q_g[n:] == 0x5A5A5A5A).all()
    po = oracle.Params(dims, block, 1e-5, oracle.EB_REL, 8, oracle.PAD_NAMES[pad])
    c = oracle.compress(po, x)
    got = f.to_host()
    assert np.array_equal(got["codes"], c.codes)
    assert np.array_equal(got["out_idx"], c.out_idx)


@pytest.mark.parametrize("dims,block", [((40, 300), 16), ((40, 260), 8), ((20, 24, 132), 8),
                                        ((20, 40, 68), 16), ((300000,), 64)])
@pytest.mark.parametrize("pad", ["zero", "block_avg", "block_min", "global_avg"])
def test_parity_exact_mode_switch(dims, block, pad):
    """Rows (2D), planes (3D) or a stretch (1D) whose prequantized values
    cross 2^20 in the middle of a tile, and values right at 2^20, so a tile
    starts in one arithmetic mode and has to continue in the other."""
    rng = np.random.default_rng(17)
    n = int(np.prod(dims))
    x = rng.integers(-300, 301, n).astype(np.float64)
    lead = np.arange(n) // (n // dims[0]) if len(dims) > 1 else np.arange(n)
    big = lead >= (dims[0] * 3) // 5
    x = np.where(big, x + 1.5e6, x + 1000.0)
    x[::97] = 1048576.0          # exactly 2^20
    x[1::89] = -1048575.0
    x = x.astype(np.float32)
    f, c, g, o, xx = run_both(x, dims, block, 0.5, "abs", 512, pad)
    assert_parity(f, c, g, o, xx, pad)


def test_reconstruct_with_and_without_workspace_agree():
    """vsz_reconstruct with the optional workspace (ticket-scheduled tiles)
    and without it (static tiles) give identical values and integers."""
    import ctypes
    dims = (24, 40, 200)
    x = field_for(dims, seed=41).reshape(-1)
    p = vsz.Params.make(dims, 8, 1e-5, "rel", 16, "block_avg")
    f = vsz.Field(p)
    f.compress(torch.from_numpy(np.ascontiguousarray(x, np.float32)).cuda())
    a = f.reconstruct().clone()
    qa = f.reconstruct_q().clone()
    L = vsz.lib()
    b = torch.empty_like(a)
    qb = torch.empty_like(qa)
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert L.vsz_reconstruct(ctypes.byref(f._cp), ctypes.byref(f._cc), ctypes.c_void_p(b.data_ptr()),
                             None, 0, s) == 0
    assert L.vsz_reconstruct_q(ctypes.byref(f._cp), ctypes.byref(f._cc), ctypes.c_void_p(qb.data_ptr()),
                               None, 0, s) == 0
    torch.cuda.synchronize()
    assert torch.equal(a.view(torch.int32), b.view(torch.int32))
    assert torch.equal(qa, qb)
    assert f.header()["n_out"] > 0


@pytest.mark.parametrize("R,n,kind,offset", [(512, 1_000_003, "peaked", 0), (4, 10007, "uniform", 0),
                                             (2, 999, "const", 0), (512, 300_001, "const", 0),
                                             (32768, 200_000, "uniform", 0), (512, 77_777, "peaked", 1),
                                             (7, 5000, "peaked", 3), (512, 2_000_017, "wide", 0),
                                             (40, 100_000, "wide", 2), (4096, 300_000, "wide", 0)])
def test_code_histogram_synthetic(R, n, kind, offset):
    """Histogram of arbitrary code arrays: counts per bin equal numpy's, codes
    at or above 2R are not counted, any alignment of the codes."""
    import ctypes
    rng = np.random.default_rng(R + n)
    if kind == "uniform":
        c = rng.integers(0, 2 * R + 3, n)
    elif kind == "const":
        c = np.full(n, R)
    elif kind == "wide":  # partly outside the bins counted without atomics
        c = np.clip(np.round(rng.normal(R, 40.0, n)), 0, 2 * R + 5)
    else:
        c = np.clip(np.round(rng.normal(R, 3.0, n)), 0, 2 * R + 5)
    c = c.astype(np.uint16)
    buf = torch.from_numpy(np.concatenate([np.zeros(offset, np.uint16), c]).view(np.int16)).cuda()
    p = vsz.Params.make((n,), 256, 1e-3, "abs", R, "zero")
    hist = torch.empty(2 * R, dtype=torch.int32, device="cuda")
    L = vsz.lib()
    rc = L.vsz_code_histogram(ctypes.byref(p.c()), ctypes.c_void_p(buf.data_ptr() + 2 * offset),
                              ctypes.c_void_p(hist.data_ptr()), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0
    want = np.bincount(c[c < 2 * R], minlength=2 * R)
    assert np.array_equal(hist.cpu().numpy().astype(np.int64), want)


def test_trace_and_shutdown():
    """Launch tracing records every kernel of a compression with its device
    time; vsz_shutdown switches tracing off and clears the library's caches,
    after which calls work again and give the same results."""
    x = torch.from_numpy(np.exp(synth.grf3d((40, 64, 96), 5)).astype(np.float32).reshape(-1)).cuda()
    p = vsz.Params.make((40, 64, 96), 8, 1e-4, "rel", 512, "zero")
    f = vsz.Field(p)
    vsz.trace_read()
    vsz.trace_enable(True)
    f.compress(x)
    recs = vsz.trace_read()
    names = [r["name"] for r in recs]
    assert "lorenzo" in names and "range" in names, names
    assert all(r["ms"] >= 0.0 for r in recs)
    first = f.to_host()
    vsz.shutdown()
    f.compress(x)
    assert vsz.trace_read() == []  # tracing is off after shutdown
    again = f.to_host()
    for key in ("codes", "blk_off", "out_idx", "out_delta"):
        assert np.array_equal(first[key], again[key]), key
    vsz.trace_enable(True)
    f.reconstruct()
    assert len(vsz.trace_read()) > 0
    vsz.trace_enable(False)


@pytest.mark.parametrize("dims,block", [((16, 24, 256), 8), ((12, 16, 384), 4), ((64, 256), 16), ((40, 512), 8)])
def test_dense_outliers_aligned_unaligned_and_corrupt_lists(dims, block):
    """Interior tiles whose every batch holds outliers (radius 8 at a relative
    eb of 1e-6), their outliers fetched from the global lists: as allocated
    (16-byte words), at a 4-byte offset (single loads), and with one index
    changed in the middle of the list (reported as corrupt)."""
    import ctypes
    x = field_for(dims, seed=21)
    f, c, g, o, xx = run_both(x, dims, block, 1e-6, radius=8)
    n_out = len(c.out_idx)
    assert n_out > 0.5 * xx.size
    assert_parity(f, c, g, o, xx, "zero")
    xo = o[1].view(np.uint32)
    bi = torch.zeros(f.out_cap + 1, dtype=torch.int32, device="cuda")
    bd = torch.zeros(f.out_cap + 1, dtype=torch.int32, device="cuda")
    bi[1:1 + n_out] = f.out_idx[:n_out]
    bd[1:1 + n_out] = f.out_delta[:n_out]
    cc = vsz._CCompressed(f.codes.data_ptr(), f.pad.data_ptr() if f.pad is not None else 0, f.blk_off.data_ptr(),
                          bi[1:].data_ptr(), bd[1:].data_ptr(), f.out_cap, f.fix_idx.data_ptr(),
                          f.fix_bits.data_ptr(), f.fix_cap, f.hdr.data_ptr())
    out = torch.empty(xx.size, dtype=torch.float32, device="cuda")

    def recon():
        vsz._check(vsz.lib().vsz_reconstruct(ctypes.byref(f._cp), ctypes.byref(cc), vsz._ptr(out), vsz._ptr(f.rws),
                                             vsz.RECON_WS_BYTES, None), "vsz_reconstruct")
        torch.cuda.synchronize()
        return out.cpu().numpy().view(np.uint32)

    assert np.array_equal(recon(), xo)
    assert f.header()["recon_status"] == 0
    bi[1 + n_out // 2] += 1
    recon()
    assert f.header()["recon_status"] == 5
