"""The allocation-free compression entry point, vsz_compress_noalloc.

Some callers cannot allocate device memory: code running inside a framework
whose caching allocator already owns the GPU's memory, and latency-critical
paths that cannot take the device-wide synchronization an allocation may
cause.  vsz_compress_noalloc serves them from a fixed workspace inside the
library instead of a caller-supplied one.

This file is named so that pytest collects it last: if it fails, a run that
stops at the first failure has already run every other test.  It passes on
its own in a fresh process as well as after the other tests (the library's
fixed workspace keeps the previous call's contents, which must not matter).
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2201_04614_gb300 as vsz  # noqa: E402


def _field(dims, seed):
    if len(dims) == 1:
        return synth.random_walk1d(dims[0], seed)
    if len(dims) == 2:
        return synth.fourier2d(dims[0], dims[1], seed=seed, value_range=20.0, offset=5.0)
    return np.exp(synth.grf3d(dims, seed))


CASES = [((300, 519), 16, "block_avg", 1e-5, 8), ((19, 37, 260), 8, "zero", 1e-4, 512),
         ((10007,), 32, "global_avg", 1e-5, 64)]


def _dirty_the_workspace(dims, block, n):
    """A no-alloc call on another field of the same dims with more outliers
    and a global padding mode, so that the next call finds the shared
    workspace full of another call's counters, staged entries and tables."""
    x = np.ascontiguousarray(_field(dims, seed=block + 1000), np.float32).reshape(-1)
    p = vsz.Params.make(dims, block, 1e-7, "rel", 2, "global_avg")
    f = vsz.Field(p, out_cap=n, fix_cap=n // 4)
    f.compress_noalloc(torch.from_numpy(x).cuda())
    assert f.header()["n_out"] > n // 4


def test_noalloc_matches_compress_on_two_calls_in_a_row():
    """Each field is compressed through vsz_compress (caller workspace) and
    then, in a row, through vsz_compress_noalloc, after a no-alloc call on a
    different field left the shared workspace dirty; every output must be
    identical, and so must the reconstructions."""
    for dims, block, pad, eb, radius in CASES:
        x = np.ascontiguousarray(_field(dims, seed=block), np.float32).reshape(-1)
        n = x.size
        p = vsz.Params.make(dims, block, eb, "rel", radius, pad)
        xd = torch.from_numpy(x).cuda()
        ref = vsz.Field(p, out_cap=n, fix_cap=n // 4)
        ref.compress(xd)
        want = ref.to_host()
        want_x = ref.reconstruct().cpu().numpy()
        assert want["header"]["n_out"] > 0  # the staging part of the workspace is exercised
        _dirty_the_workspace(dims, block, n)
        for call in range(2):
            f = vsz.Field(p, out_cap=n, fix_cap=n // 4)
            f.compress_noalloc(xd)
            got = f.to_host()
            for k in ("codes", "pad", "blk_off", "out_idx", "out_delta", "fix_idx", "fix_bits"):
                if want[k] is None:
                    assert got[k] is None
                else:
                    assert np.array_equal(got[k], want[k]), (dims, call, k)
            for k in ("eb_abs", "inv2eb", "ebx2", "eb_f32", "pad_global", "n_out", "n_fix", "status"):
                assert got["header"][k] == want["header"][k], (dims, call, k)
            xh = f.reconstruct().cpu().numpy()
            assert np.array_equal(xh.view(np.uint32), want_x.view(np.uint32)), (dims, call)


def test_noalloc_rejects_calls_beyond_its_workspace():
    """A field whose lists need more scratch than the fixed workspace holds
    is refused before any GPU work, with VSZ_ERR_TOO_LARGE."""
    dims = (2048, 2048)
    p = vsz.Params.make(dims, 16, 1e-4, "rel", 512, "zero")
    n = dims[0] * dims[1]
    assert vsz.workspace_size(p, n, n) > vsz.NOALLOC_WS_BYTES
    f = vsz.Field(p, out_cap=n, fix_cap=n)
    with pytest.raises(vsz.VszError) as err:
        f.compress_noalloc(torch.zeros(n, dtype=torch.float32, device="cuda"))
    assert err.value.status == 6
    # a smaller capacity of the same field fits and works
    f2 = vsz.Field(p, out_cap=n // 16, fix_cap=n // 64)
    assert vsz.workspace_size(p, n // 16, n // 64) <= vsz.NOALLOC_WS_BYTES
    x = _field(dims, seed=5).reshape(-1)
    f2.compress_noalloc(torch.from_numpy(np.ascontiguousarray(x, np.float32)).cuda())
    assert f2.header()["status"] == 0


def test_noalloc_call_leaves_device_memory_unchanged():
    """The call allocates nothing: around a warmed-up call the device's free
    memory (cudaMemGetInfo) does not move."""
    dims = (300, 519)
    x = np.ascontiguousarray(_field(dims, seed=3), np.float32).reshape(-1)
    n = x.size
    p = vsz.Params.make(dims, 16, 1e-5, "rel", 8, "block_avg")
    f = vsz.Field(p, out_cap=n, fix_cap=n // 4)
    xd = torch.from_numpy(x).cuda()
    f.compress_noalloc(xd)  # warm-up: the library's first call on the device
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        f.compress_noalloc(xd)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert f.header()["status"] == 0 and f.header()["n_out"] > 0
