"""The binding's buffer checks on the entropy-stage, reconstruction and
tuner calls (host logic, no GPU).

The C ABI takes plain pointers and trusts the sizes it is given, so the
Python binding refuses a buffer that is not a contiguous CUDA tensor of the
right element size, or that is shorter than the call needs, before anything
is allocated or called.  The stand-in tensors below carry only a size and an
element type; their data_ptr() raises, so no call can reach the library with
one of them even if a check were missing.
"""
import pytest

import paper_2201_04614_gb300 as vsz


class FakeCuda:
    """A CUDA tensor's shape and type, without memory."""

    is_cuda = True
    device = "cuda"

    def __init__(self, numel: int, itemsize: int, contiguous: bool = True):
        self._n, self._s, self._c = numel, itemsize, contiguous

    def numel(self):
        return self._n

    def element_size(self):
        return self._s

    def is_contiguous(self):
        return self._c

    def data_ptr(self):
        raise AssertionError("a buffer reached a library call")


class FakeHost(FakeCuda):
    is_cuda = False
    device = "cpu"


class FakeBook:
    nsym = 1024
    buf = FakeCuda(4096, 1)


CH = vsz.HUFF_CHUNK


def test_book_needs_a_histogram_of_nsym_counts():
    with pytest.raises(ValueError):
        vsz.HuffmanBook(FakeCuda(100, 4), 1024)
    with pytest.raises(TypeError):
        vsz.HuffmanBook(FakeCuda(1024, 8), 1024)  # int64 counts
    with pytest.raises(TypeError):
        vsz.HuffmanBook(FakeHost(1024, 4), 1024)


def test_encode_checks_symbols_words_and_index():
    n = 3 * CH + 5  # 4 chunks
    with pytest.raises(ValueError):
        vsz.huffman_encode(FakeCuda(n - 1, 2), n, FakeBook())
    with pytest.raises(TypeError):
        vsz.huffman_encode(FakeCuda(n, 4), n, FakeBook())  # int32 symbols
    with pytest.raises(TypeError):
        vsz.huffman_encode(FakeCuda(n, 2, contiguous=False), n, FakeBook())
    with pytest.raises(TypeError):
        vsz.huffman_encode(FakeCuda(n, 2), n, FakeBook(), words=FakeCuda(100, 2))
    with pytest.raises(ValueError):  # the index needs 32 entries per chunk
        vsz.huffman_encode(FakeCuda(n, 2), n, FakeBook(), words=FakeCuda(100, 4), index=FakeCuda(32 * 4 - 1, 2))
    with pytest.raises(TypeError):
        vsz.huffman_encode(FakeCuda(n, 2), n, FakeBook(), words=FakeCuda(100, 4), index=FakeCuda(32 * 4, 4))


@pytest.mark.parametrize("indexed", [False, True])
def test_decode_checks_offsets_output_and_index(indexed):
    n = 2 * CH + 1  # 3 chunks: 4 offsets, 96 index entries

    def dec(words, off, out=None, index=None):
        if indexed:
            return vsz.huffman_decode_indexed(words, off, index if index is not None else FakeCuda(96, 2), n,
                                              FakeBook(), out=out)
        return vsz.huffman_decode(words, off, n, FakeBook(), out=out)

    with pytest.raises(ValueError):
        dec(FakeCuda(50, 4), FakeCuda(3, 8))
    with pytest.raises(TypeError):
        dec(FakeCuda(50, 4), FakeCuda(4, 4))  # 32-bit offsets
    with pytest.raises(TypeError):
        dec(FakeCuda(50, 2), FakeCuda(4, 8))  # 16-bit words
    with pytest.raises(TypeError):
        dec(FakeHost(50, 4), FakeCuda(4, 8))
    with pytest.raises(ValueError):
        dec(FakeCuda(50, 4), FakeCuda(4, 8), out=FakeCuda(n - 1, 2))
    if indexed:
        with pytest.raises(ValueError):
            dec(FakeCuda(50, 4), FakeCuda(4, 8), index=FakeCuda(95, 2))
        with pytest.raises(TypeError):
            dec(FakeCuda(50, 4), FakeCuda(4, 8), index=FakeCuda(96, 4))


class FieldShape:
    """What Field's reconstruction reads before its buffer check: the size."""

    n = 5000


@pytest.mark.parametrize("method", [vsz.Field.reconstruct, vsz.Field.reconstruct_q])
def test_reconstruction_checks_its_output(method):
    with pytest.raises(ValueError):
        method(FieldShape(), out=FakeCuda(4999, 4))
    with pytest.raises(TypeError):
        method(FieldShape(), out=FakeCuda(5000, 2))
    with pytest.raises(TypeError):
        method(FieldShape(), out=FakeHost(5000, 4))


def test_tuner_sample_arrays_must_cover_the_feature_rows():
    import torch
    from paper_2201_04614_gb300 import tuner as T
    X = torch.zeros(5, T.NFEAT)
    T._rows_check(X, torch.zeros(5), torch.zeros(7))
    with pytest.raises(ValueError):
        T._rows_check(X, torch.zeros(4))
    with pytest.raises(ValueError):
        T._rows_check(torch.zeros(5, T.NFEAT - 1))
    with pytest.raises(ValueError):
        T._rows_check(torch.zeros(5 * T.NFEAT))



def test_slab_backend_needs_the_slab_values():
    import torch
    from paper_2201_04614_gb300 import shard

    class FakeF32(FakeCuda):
        dtype = torch.float32

    job = shard.SlabJob((40, 30, 20), 8, 1e-3, shard.EB_REL, 64, 0, 8, 24)  # 16 planes of 30 x 20
    with pytest.raises(ValueError):
        shard.GpuSlabBackend(job, FakeF32(16 * 30 * 20 - 1, 4))
    with pytest.raises(TypeError):
        shard.GpuSlabBackend(job, torch.zeros(16 * 30 * 20))  # a host tensor
