"""Pins for the oracle's entropy stage (Sec. II-B: SZ Huffman-codes the
quantization codes), checked against what the mathematics fixes:

* the textbook example of Cormen et al. (six characters with frequencies
  45, 13, 12, 16, 9, 5 thousand: code lengths 1, 3, 3, 3, 4, 4, cost 224);
* optimality: the coded length equals the minimum cost, computed
  independently as the sum of the weights of every merged node (a heap, no
  tie rule needed), on random, skewed, equal and Fibonacci histograms;
* the Kraft equality sum 2^-len = 1 (a complete prefix code), prefix-freeness
  and the canonical order of the codewords;
* the entropy bound H <= mean length < H + 1;
* the tie rule on equal weights, worked by hand;
* the bitstream against a second packer written with Python bit strings,
  and decoding back to the symbols.
"""
import heapq
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle


def optimal_cost(hist):
    h = [int(v) for v in hist if v > 0]
    if len(h) <= 1:
        return sum(h)  # a lone symbol costs one bit each
    heapq.heapify(h)
    cost = 0
    while len(h) > 1:
        a, b = heapq.heappop(h), heapq.heappop(h)
        cost += a + b
        heapq.heappush(h, a + b)
    return cost


def test_textbook_example():
    hist = np.array([45, 13, 12, 16, 9, 5], np.uint32)
    ln, cw = oracle.huffman_book(hist)
    assert ln.tolist() == [1, 3, 3, 3, 4, 4]
    assert int((hist.astype(np.int64) * ln).sum()) == 224


def test_tie_rule_by_hand():
    # three equal weights: leaves 0 and 1 merge first (leaves in symbol
    # order), then leaf 2 (weight 1) with the merged node (weight 2)
    ln, _ = oracle.huffman_book(np.array([1, 1, 1], np.uint32))
    assert ln.tolist() == [2, 2, 1]
    # weights 2, 1, 1: leaves 1 and 2 merge (weight 2); then leaf 0 and the
    # merged node tie at 2 and the leaf is taken first
    ln, _ = oracle.huffman_book(np.array([2, 1, 1], np.uint32))
    assert ln.tolist() == [1, 2, 2]
    ln, _ = oracle.huffman_book(np.array([7] * 8, np.uint32))
    assert ln.tolist() == [3] * 8


def _hists():
    rng = np.random.default_rng(5)
    out = [np.array([0, 0, 9, 0], np.uint32), np.array([3, 0, 5], np.uint32)]
    fib = [1, 1]
    while len(fib) < 40:
        fib.append(fib[-1] + fib[-2])
    out.append(np.array(fib, np.uint32))                       # deepest tree
    out.append(np.array([2 ** k for k in range(30)], np.uint32))
    for _ in range(12):
        nsym = int(rng.integers(2, 1025))
        kind = rng.integers(0, 3)
        if kind == 0:
            h = rng.integers(0, 1000, nsym)
        elif kind == 1:
            h = (1e6 * np.exp(-np.abs(np.arange(nsym) - nsym / 2) / rng.uniform(1, 50))).astype(np.int64)
        else:
            h = rng.integers(0, 3, nsym) * rng.integers(1, 5)
        out.append(h.astype(np.uint32))
    return out


@pytest.mark.parametrize("hist", _hists())
def test_optimal_complete_canonical(hist):
    ln, cw = oracle.huffman_book(hist)
    used = np.nonzero(hist)[0]
    assert (ln[hist == 0] == 0).all() and (ln[used] > 0).all() and ln.max() <= 64
    cost = int((hist.astype(np.int64) * ln.astype(np.int64)).sum())
    assert cost == optimal_cost(hist)
    if used.size >= 2:
        assert sum(Fraction(1, 2 ** int(ln[s])) for s in used) == 1
        n = int(hist.sum())
        H = -sum(int(hist[s]) / n * math.log2(int(hist[s]) / n) for s in used)
        assert H - 1e-9 <= cost / n < H + 1
    order = sorted(used, key=lambda s: (int(ln[s]), int(s)))
    words = [format(int(cw[s]), "b").zfill(int(ln[s])) for s in order]
    for s, w in zip(order, words):
        assert len(w) == int(ln[s])  # the codeword fits its length
    for i in range(len(words) - 1):
        a, b = words[i], words[i + 1]
        assert int(b, 2) > int(a[: len(b)].ljust(len(b), "0"), 2) or len(b) > len(a)
    for i, a in enumerate(words):  # prefix-free
        for b in words[i + 1:]:
            assert not b.startswith(a)


def pack_python(sym, ln, cw, chunk):
    """A second packer: bit strings per chunk, padded to whole 32-bit words."""
    words, off = [], [0]
    for c0 in range(0, len(sym), chunk):
        bits = "".join(format(int(cw[s]), "b").zfill(int(ln[s])) for s in sym[c0:c0 + chunk])
        bits += "0" * (-len(bits) % 32)
        words += [int(bits[i:i + 32], 2) for i in range(0, len(bits), 32)]
        off.append(len(words))
    return np.array(words, np.uint32), np.array(off, np.uint64)


@pytest.mark.parametrize("n,chunk,nsym,seed", [(1, 4, 4, 0), (999, 64, 16, 1), (5000, 4096, 300, 2),
                                               (20000, 1000, 1024, 3), (4096 * 2 + 3, 4096, 7, 4)])
def test_stream_and_round_trip(n, chunk, nsym, seed):
    rng = np.random.default_rng(seed)
    sym = np.minimum(rng.geometric(0.2, n) - 1 + nsym // 2, nsym - 1).astype(np.uint16)
    hist = np.bincount(sym, minlength=nsym).astype(np.uint32)
    ln, cw = oracle.huffman_book(hist)
    words, off = oracle.huffman_encode(sym, ln, cw, chunk)
    pw, poff = pack_python(sym, ln, cw, chunk)
    assert off.tolist() == poff.tolist()
    assert words.tolist() == pw.tolist()
    assert np.array_equal(oracle.huffman_decode(words, off, n, ln, cw, chunk), sym)


def test_lone_symbol():
    sym = np.full(100, 5, np.uint16)
    hist = np.bincount(sym, minlength=8).astype(np.uint32)
    ln, cw = oracle.huffman_book(hist)
    assert ln.tolist() == [0, 0, 0, 0, 0, 1, 0, 0] and int(cw[5]) == 0
    words, off = oracle.huffman_encode(sym, ln, cw, 64)
    assert off.tolist() == [0, 2, 4] and (words == 0).all()  # 64 bits, then 36 bits: two words each
    assert np.array_equal(oracle.huffman_decode(words, off, 100, ln, cw, 64), sym)


def walk_index(words, off, n, ln, cw, chunk, lanes):
    """The decode index found by reading the packed stream one bit at a time:
    at every (chunk / lanes)-th code of a chunk, the bit reached so far;
    each codeword is recognised by its (length, value) in the codebook, and
    must be the symbol that was encoded (checked by the caller)."""
    table = {(int(ln[s]), int(cw[s])): s for s in range(len(ln)) if ln[s]}
    per = chunk // lanes
    nchunks = (n + chunk - 1) // chunk
    index, decoded = [], []
    for c in range(nchunks):
        base = int(off[c]) * 32

        def bit(k):
            w = int(words[(base + k) // 32])
            return (w >> (31 - (base + k) % 32)) & 1

        pos = 0
        cnt = min(chunk, n - c * chunk)
        for i in range(chunk):
            if i % per == 0:
                index.append(pos)
            if i >= cnt:
                continue
            v, L = 0, 0
            while (L, v) not in table:
                v = (v << 1) | bit(pos + L)
                L += 1
                assert L <= 64
            decoded.append(table[(L, v)])
            pos += L
    return np.array(index, np.int64), np.array(decoded, np.uint16)


@pytest.mark.parametrize("n,chunk,lanes,kind", [(1, 1024, 32, "geo"), (1000, 1024, 32, "geo"),
                                                (3 * 1024 + 517, 1024, 32, "fib"), (2500, 256, 8, "geo"),
                                                (4096, 1024, 32, "lone")])
def test_decode_index_against_a_bit_walk(n, chunk, lanes, kind):
    rng = np.random.default_rng(n)
    if kind == "fib":  # codewords up to 39 bits
        f = [1, 1]
        while len(f) < 40:
            f.append(f[-1] + f[-2])
        hist = np.array(f, np.uint32)
        sym = rng.integers(0, 40, n).astype(np.uint16)
    elif kind == "lone":
        sym = np.full(n, 3, np.uint16)
        hist = np.bincount(sym, minlength=8).astype(np.uint32)
    else:
        sym = np.minimum(rng.geometric(0.1, n) - 1, 299).astype(np.uint16)
        hist = np.bincount(sym, minlength=300).astype(np.uint32)
    ln, cw = oracle.huffman_book(hist)
    words, off = oracle.huffman_encode(sym, ln, cw, chunk)
    want, decoded = walk_index(words, off, n, ln, cw, chunk, lanes)
    assert np.array_equal(decoded, sym)
    got = oracle.huffman_index(sym, ln, chunk, lanes)
    assert got.tolist() == want.tolist()
    # a sub-chunk past the data starts at the chunk's end; the chunk fits its words
    nc = (n + chunk - 1) // chunk
    last = got.reshape(nc, lanes)[-1]
    full = (n - (nc - 1) * chunk + chunk // lanes - 1) // (chunk // lanes)
    assert (last[full:] == int(ln.astype(np.int64)[sym[(nc - 1) * chunk:]].sum())).all()
    assert all(got.reshape(nc, lanes)[c, -1] <= 32 * int(off[c + 1] - off[c]) for c in range(nc))
