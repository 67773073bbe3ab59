"""The tile chain that places each tile's outliers and fixups in canonical
order (Sec. III-A) without a compaction pass: a decoupled look-back over
the tiles of a field, with a bounded wait.

Through vsz_debug_chain (the same device code as the compression kernels):
every tile must receive the exact exclusive sums of the tiles before it,
over windows of 32 tiles and more; a tile that never publishes makes the
tiles after it give up after the wait limit (no hang), report it, and the
GPU keeps answering.  The compression path is covered by the parity tests,
which compare the lists written by the chain with the oracle's."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2201_04614_gb300 as vsz  # noqa: E402


def _aggs(n, seed):
    rng = np.random.default_rng(seed)
    o = rng.integers(0, 5000, n).astype(np.int32)
    f = rng.integers(0, 3, n).astype(np.int32)
    o[rng.random(n) < 0.3] = 0
    return o, f


@pytest.mark.parametrize("n", [1, 2, 31, 33, 300, 4099])
def test_chain_gives_exact_exclusive_sums(n):
    o, f = _aggs(n, n)
    r = vsz.debug_chain(torch.from_numpy(o).cuda(), torch.from_numpy(f).cuda())
    assert r["timeouts"] == 0
    ex_o = np.concatenate([[0], np.cumsum(o.astype(np.int64))[:-1]])
    ex_f = np.concatenate([[0], np.cumsum(f.astype(np.int64))[:-1]])
    assert np.array_equal(r["ex_o"].numpy(), ex_o)
    assert np.array_equal(r["ex_f"].numpy(), ex_f)


def test_withheld_tile_times_out_and_the_gpu_still_answers():
    n, k = 300, 5
    o, f = _aggs(n, 7)
    # a 2 ms limit: the tiles after tile 5 find no flag there and give up
    r = vsz.debug_chain(torch.from_numpy(o).cuda(), torch.from_numpy(f).cuda(), withhold=k, wait_ns=2_000_000)
    assert r["timeouts"] >= 1
    ex_o = np.concatenate([[0], np.cumsum(o.astype(np.int64))[:-1]])
    assert np.array_equal(r["ex_o"].numpy()[:k], ex_o[:k])  # the tiles before it are exact
    # the context is intact: the full chain runs again, exactly
    r2 = vsz.debug_chain(torch.from_numpy(o).cuda(), torch.from_numpy(f).cuda())
    assert r2["timeouts"] == 0 and np.array_equal(r2["ex_o"].numpy(), ex_o)
    assert float(torch.ones(4, device="cuda").sum().item()) == 4.0


def test_chain_argument_checks():
    a = torch.zeros(4, dtype=torch.int32, device="cuda")
    L = vsz.lib()
    st = torch.zeros(8, dtype=torch.int64, device="cuda")
    assert L.vsz_debug_chain(vsz._ptr(a), vsz._ptr(a), 0, -1, 1000, vsz._ptr(st), vsz._ptr(st), vsz._ptr(a), None) == 1
    assert L.vsz_debug_chain(vsz._ptr(a), vsz._ptr(a), 4, -1, 0, vsz._ptr(st), vsz._ptr(st), vsz._ptr(a), None) == 1
    assert L.vsz_debug_chain(None, vsz._ptr(a), 4, -1, 1000, vsz._ptr(st), vsz._ptr(st), vsz._ptr(a), None) == 1
