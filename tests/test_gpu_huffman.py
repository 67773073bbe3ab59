"""GPU parity of the entropy stage (Sec. II-B): codebook, bitstream and
decoding through the C ABI against the oracle's canonical Huffman coder,
bit for bit."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle  # noqa: E402
import paper_2201_04614_gb300 as vsz  # noqa: E402


def _fib(k):
    f = [1, 1]
    while len(f) < k:
        f.append(f[-1] + f[-2])
    return f


def _hists():
    rng = np.random.default_rng(9)
    out = [("textbook", np.array([45, 13, 12, 16, 9, 5, 0, 0], np.uint32)),
           ("lone", np.array([0, 0, 0, 77], np.uint32)),
           ("fibonacci40", np.array(_fib(40), np.uint32)),
           ("equal", np.full(64, 5, np.uint32)),
           ("random1024", rng.integers(0, 5000, 1024).astype(np.uint32)),
           ("sparse8192", (rng.random(8192) < 0.05) * rng.integers(1, 1 << 20, 8192)),
           ("peaked1024", (1e7 * np.exp(-np.abs(np.arange(1024) - 512) / 3.0)).astype(np.uint32))]
    return [(k, np.asarray(h, np.uint32)) for k, h in out]


@pytest.mark.parametrize("name,hist", _hists(), ids=lambda v: v if isinstance(v, str) else "")
def test_book_matches_oracle(name, hist):
    book = vsz.HuffmanBook(torch.from_numpy(hist.view(np.int32)).cuda(), hist.size)
    ln, cw, mx = book.read()
    lo, co = oracle.huffman_book(hist)
    assert np.array_equal(ln, lo), name
    assert np.array_equal(cw, co), name
    assert mx == int(lo.max())


def _dq_codes(dims, block, eb, R, seed):
    x = synth.fourier2d(*dims, seed=seed, value_range=10.0, offset=1.0) if len(dims) == 2 else \
        np.exp(synth.grf3d(dims, seed))
    f = vsz.Field(vsz.Params.make(dims, block, eb, "rel", R, "zero"))
    f.compress(torch.from_numpy(np.ascontiguousarray(x, np.float32).reshape(-1)).cuda())
    return f.codes[: f.n], f.n, 2 * R


def _streams():
    rng = np.random.default_rng(4)
    out = []
    for dims, block, eb, R in [((300, 519), 16, 1e-4, 512), ((19, 37, 260), 8, 1e-5, 512),
                               ((64, 64), 16, 1e-2, 4096), ((1, 5), 4, 1e-3, 2)]:
        out.append(("dq", dims, block, eb, R))
    for n, nsym in [(4096 * 3 + 5, 300), (1, 4), (4096, 2), (70001, 1024)]:
        out.append(("rand", n, nsym, int(rng.integers(0, 1 << 30)), 0))
    return out


@pytest.mark.parametrize("case", _streams(), ids=lambda c: f"{c[0]}-{c[1]}")
def test_stream_matches_oracle_and_round_trips(case):
    if case[0] == "dq":
        _, dims, block, eb, R = case
        sym_t, n, nsym = _dq_codes(dims, block, eb, R, seed=3)
        sym = sym_t.cpu().numpy().view(np.uint16)
    else:
        _, n, nsym, seed, _ = case
        rng = np.random.default_rng(seed)
        sym = np.minimum(rng.geometric(0.3, n) - 1, nsym - 1).astype(np.uint16)
        sym_t = torch.from_numpy(sym.view(np.int16)).cuda()
    hist = np.bincount(sym, minlength=nsym).astype(np.uint32)
    book = vsz.HuffmanBook(torch.from_numpy(hist.view(np.int32)).cuda(), nsym)
    words, off, st = vsz.huffman_encode(sym_t, n, book)
    assert int(st.item()) == 0
    lo, co = oracle.huffman_book(hist)
    ow, ooff = oracle.huffman_encode(sym, lo, co)
    goff = off.cpu().numpy().view(np.uint64)
    assert np.array_equal(goff, ooff)
    assert np.array_equal(words[: int(goff[-1])].cpu().numpy().view(np.uint32), ow)
    dec, st2 = vsz.huffman_decode(words, off, n, book)
    assert int(st2.item()) == 0
    assert np.array_equal(dec[:n].cpu().numpy().view(np.uint16), sym)


def test_capacity_and_bad_symbols():
    rng = np.random.default_rng(1)
    n, nsym = 20000, 64
    sym = rng.integers(0, nsym, n).astype(np.uint16)
    hist = np.bincount(sym, minlength=nsym).astype(np.uint32)
    book = vsz.HuffmanBook(torch.from_numpy(hist.view(np.int32)).cuda(), nsym)
    sym_t = torch.from_numpy(sym.view(np.int16)).cuda()
    small = torch.zeros(100, dtype=torch.int32, device="cuda")
    words, off, st = vsz.huffman_encode(sym_t, n, book, words=small)
    assert int(st.item()) & 2
    lo, co = oracle.huffman_book(hist)
    assert np.array_equal(off.cpu().numpy().view(np.uint64), oracle.huffman_encode(sym, lo, co)[1])
    bad = sym.copy()
    bad[123] = nsym - 1
    hist2 = hist.copy()
    hist2[nsym - 1] = 0
    book2 = vsz.HuffmanBook(torch.from_numpy(hist2.view(np.int32)).cuda(), nsym)
    _, _, st = vsz.huffman_encode(torch.from_numpy(bad.view(np.int16)).cuda(), n, book2)
    assert int(st.item()) & 1


def test_limits():
    with pytest.raises(vsz.VszError) as e:
        vsz.HuffmanBook(torch.zeros(16384, dtype=torch.int32, device="cuda"), 16384)
    assert e.value.status == 2
    hist = torch.tensor([3, 1], dtype=torch.int32, device="cuda")
    book = vsz.HuffmanBook(hist, 2)
    words, off, st = vsz.huffman_encode(torch.zeros(0, dtype=torch.int16, device="cuda"), 0, book)
    assert int(st.item()) == 0 and int(off[0].item()) == 0


def _round_trip(sym, nsym, weights, sym_shift=0, words_shift=0, out_shift=0):
    """Encode sym with the book of `weights`, compare with the oracle, decode
    (optionally from views that start 2 or 4 bytes past a 16-byte boundary)."""
    n = sym.size
    book = vsz.HuffmanBook(torch.from_numpy(weights.view(np.int32)).cuda(), nsym)
    lo, co = oracle.huffman_book(weights)
    ow, ooff = oracle.huffman_encode(sym, lo, co)
    base = torch.zeros(n + 8, dtype=torch.int16, device="cuda")
    base[sym_shift: sym_shift + n] = torch.from_numpy(sym.view(np.int16)).cuda()
    cap = torch.zeros(ow.size + 16, dtype=torch.int32, device="cuda")
    words, off, st = vsz.huffman_encode(base[sym_shift: sym_shift + n], n, book, words=cap)
    assert int(st.item()) == 0
    goff = off.cpu().numpy().view(np.uint64)
    assert np.array_equal(goff, ooff)
    assert np.array_equal(words[: int(goff[-1])].cpu().numpy().view(np.uint32), ow)
    wbuf = torch.zeros(words.numel() + 4, dtype=torch.int32, device="cuda")
    wbuf[words_shift: words_shift + words.numel()] = words
    obuf = torch.zeros(n + 8, dtype=torch.int16, device="cuda")
    dec, st2 = vsz.huffman_decode(wbuf[words_shift: words_shift + words.numel()], off, n, book,
                                  out=obuf[out_shift: out_shift + n])
    assert int(st2.item()) == 0
    assert np.array_equal(dec[:n].cpu().numpy().view(np.uint16), sym)
    return words, off, book


@pytest.mark.parametrize("n", [1, 1000, 3 * 1024 + 517])
def test_long_codewords(n):
    # Fibonacci weights give codewords up to 39 bits; symbols drawn uniformly
    # make most codewords longer than the decoder's 12-bit table and many
    # longer than 32 bits (split in the encoder, spanning buffer refills in
    # the decoder)
    weights = np.array(_fib(40), np.uint32)
    sym = np.random.default_rng(n).integers(0, 40, n).astype(np.uint16)
    _round_trip(sym, 40, weights)


@pytest.mark.parametrize("shifts", [(1, 0, 0), (0, 1, 0), (0, 0, 1), (3, 2, 5)])
def test_unaligned_views(shifts):
    rng = np.random.default_rng(17)
    n, nsym = 5 * 1024 + 77, 1024
    sym = np.minimum(rng.geometric(0.05, n) - 1, nsym - 1).astype(np.uint16)
    weights = np.bincount(sym, minlength=nsym).astype(np.uint32)
    _round_trip(sym, nsym, weights, *shifts)


def test_truncated_stream_is_reported():
    rng = np.random.default_rng(5)
    n, nsym = 8 * 1024, 256
    sym = rng.integers(0, nsym, n).astype(np.uint16)
    weights = np.bincount(sym, minlength=nsym).astype(np.uint32)
    words, off, book = _round_trip(sym, nsym, weights)
    total = int(off[-1].item())
    _, st = vsz.huffman_decode(words[: total - 40], off, n, book)
    assert int(st.item()) & 4


# ---------------------------------------------------------------- decode index
def _oracle_index(sym, lens):
    """The oracle's decode index (for chunk c and lane j, the bits of the
    chunk's codes before code 32 j; the chunk's total for lanes past the
    data), as the device stores it: uint16."""
    return oracle.huffman_index(sym, lens).astype(np.uint16)


def _indexed_round_trip(sym, nsym, weights, words_shift=0, out_shift=0):
    n = sym.size
    book = vsz.HuffmanBook(torch.from_numpy(weights.view(np.int32)).cuda(), nsym)
    lo, co = oracle.huffman_book(weights)
    ow, ooff = oracle.huffman_encode(sym, lo, co)
    sym_t = torch.from_numpy(sym.view(np.int16)).cuda()
    cap = torch.zeros(ow.size + 16, dtype=torch.int32, device="cuda")
    words, off, st, index = vsz.huffman_encode(sym_t, n, book, words=cap, index=True)
    assert int(st.item()) == 0
    goff = off.cpu().numpy().view(np.uint64)
    assert np.array_equal(goff, ooff)  # the same stream as without the index
    assert np.array_equal(words[: int(goff[-1])].cpu().numpy().view(np.uint32), ow)
    nc = (n + 1023) // 1024
    assert np.array_equal(index[: 32 * nc].cpu().numpy().view(np.uint16), _oracle_index(sym, lo))
    wbuf = torch.zeros(words.numel() + 4, dtype=torch.int32, device="cuda")
    wbuf[words_shift: words_shift + words.numel()] = words
    obuf = torch.zeros(n + 8, dtype=torch.int16, device="cuda")
    dec, st2 = vsz.huffman_decode_indexed(wbuf[words_shift: words_shift + words.numel()], off, index, n, book,
                                          out=obuf[out_shift: out_shift + n])
    assert int(st2.item()) == 0
    assert np.array_equal(dec[:n].cpu().numpy().view(np.uint16), sym)
    return words, off, index, book


@pytest.mark.parametrize("case", _streams(), ids=lambda c: f"{c[0]}-{c[1]}")
def test_indexed_stream_matches_oracle_and_decodes(case):
    if case[0] == "dq":
        _, dims, block, eb, R = case
        sym_t, n, nsym = _dq_codes(dims, block, eb, R, seed=3)
        sym = sym_t.cpu().numpy().view(np.uint16).copy()
    else:
        _, n, nsym, seed, _ = case
        rng = np.random.default_rng(seed)
        sym = np.minimum(rng.geometric(0.3, n) - 1, nsym - 1).astype(np.uint16)
    hist = np.bincount(sym, minlength=nsym).astype(np.uint32)
    _indexed_round_trip(sym, nsym, hist)


@pytest.mark.parametrize("n", [1, 1000, 3 * 1024 + 517])
def test_indexed_long_codewords(n):
    # codewords up to 39 bits, many longer than the 15-bit table and than 32
    weights = np.array(_fib(40), np.uint32)
    sym = np.random.default_rng(n).integers(0, 40, n).astype(np.uint16)
    _indexed_round_trip(sym, 40, weights)


@pytest.mark.parametrize("shifts", [(1, 0), (0, 1), (2, 5)])
def test_indexed_unaligned_views(shifts):
    rng = np.random.default_rng(17)
    n, nsym = 5 * 1024 + 77, 1024
    sym = np.minimum(rng.geometric(0.05, n) - 1, nsym - 1).astype(np.uint16)
    weights = np.bincount(sym, minlength=nsym).astype(np.uint32)
    _indexed_round_trip(sym, nsym, weights, *shifts)


def test_index_that_does_not_fit_the_stream_is_reported():
    rng = np.random.default_rng(8)
    n, nsym = 6 * 1024, 512
    sym = np.minimum(rng.geometric(0.02, n) - 1, nsym - 1).astype(np.uint16)
    weights = np.bincount(sym, minlength=nsym).astype(np.uint32)
    words, off, index, book = _indexed_round_trip(sym, nsym, weights)
    bad = index.clone()
    bad[2 * 32 + 7] += 5  # lane 6 of chunk 2 then ends short of where lane 7 is said to start
    _, st = vsz.huffman_decode_indexed(words, off, bad, n, book)
    assert int(st.item()) & 4
    total = int(off[-1].item())
    _, st = vsz.huffman_decode_indexed(words[: total - 40], off, index, n, book)
    assert int(st.item()) & 4
