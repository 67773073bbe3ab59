// k_huffman.cu -- the entropy stage: canonical Huffman coding of the
// quantization codes (Sec. II-B: SZ Huffman-codes the integer codes that the
// dual-quantization produces).
//
// Codebook (one CTA): leaves sorted by (count, symbol) with a bitonic sort in
// shared memory, then the two-queue Huffman merge (ties: the leaf first, so
// equal weights resolve leaves before merged nodes, leaves in symbol order,
// merged nodes in merge order), depths, canonical codewords (symbols sorted
// by (length, symbol) get consecutive codes), and the decoder's tables.
//
// Stream: chunks of VSZ_HUFF_CHUNK symbols, each starting on a 32-bit word,
// bits filling each word from its most significant bit; chunk_off[c] is the
// first word of chunk c.  Encoding: per-chunk bit counts, a scan into word
// offsets, then one CTA per chunk packs its codewords into shared memory and
// stores the words.  Decoding: one thread per chunk walks its bits with a
// 2^11-entry lookup table for short codewords and the canonical ranges for
// longer ones.
#include <climits>

#include "common.cuh"
#include "trace.cuh"

namespace vsz {

constexpr int kLutBits = 11;
constexpr uint32_t kMaxSym = VSZ_HUFF_MAX_SYMBOLS;

// Device codebook layout (one caller buffer).
struct HuffHdr {
    uint32_t nsym, max_len, nused, ok;
};
struct HuffLayout {
    size_t code, len, first, count, base, sorted, lut, total;
};
__host__ __device__ inline HuffLayout huff_layout(uint32_t nsym) {
    HuffLayout L;
    size_t off = 64;
    L.code = off;   off += (size_t)nsym * 8;
    L.first = off;  off += 66 * 8;
    L.count = off;  off += 66 * 4;
    L.base = off;   off += 66 * 4;
    L.lut = off;    off += ((size_t)1 << kLutBits) * 4;
    L.len = off;    off += ((size_t)nsym + 15) & ~(size_t)15;
    L.sorted = off; off += ((size_t)nsym * 2 + 15) & ~(size_t)15;
    L.total = off;
    return L;
}

struct HuffBook {
    const HuffHdr* hdr;
    const uint64_t* code;
    const uint8_t* len;
    const uint64_t* first;
    const uint32_t* count;
    const uint32_t* base;
    const uint16_t* sorted;
    const uint32_t* lut;
};
__host__ __device__ inline HuffBook huff_book(const void* p, uint32_t nsym) {
    const HuffLayout L = huff_layout(nsym);
    const char* b = (const char*)p;
    return HuffBook{(const HuffHdr*)b, (const uint64_t*)(b + L.code), (const uint8_t*)(b + L.len),
                    (const uint64_t*)(b + L.first), (const uint32_t*)(b + L.count),
                    (const uint32_t*)(b + L.base), (const uint16_t*)(b + L.sorted), (const uint32_t*)(b + L.lut)};
}

// ---------------------------------------------------------------- codebook
// Bitonic sort (ascending) of n = 2^k 64-bit keys in shared memory.
__device__ void bitonic_sort(unsigned long long* key, uint32_t n) {
    for (uint32_t size = 2; size <= n; size <<= 1) {
        for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
            for (uint32_t i = threadIdx.x; i < n / 2; i += blockDim.x) {
                const uint32_t lo = 2 * i - (i & (stride - 1));
                const uint32_t hi = lo + stride;
                const bool up = (lo & size) == 0;
                const unsigned long long a = key[lo], b = key[hi];
                if ((a > b) == up) {
                    key[lo] = b;
                    key[hi] = a;
                }
            }
            __syncthreads();
        }
    }
}

__global__ void __launch_bounds__(1024) k_huff_book(const uint32_t* __restrict__ hist, uint32_t nsym, void* book) {
    extern __shared__ __align__(16) unsigned char sm[];
    const HuffLayout L = huff_layout(nsym);
    char* B = (char*)book;
    HuffHdr* hdr = (HuffHdr*)B;
    uint64_t* code = (uint64_t*)(B + L.code);
    uint8_t* len = (uint8_t*)(B + L.len);
    uint64_t* first = (uint64_t*)(B + L.first);
    uint32_t* count = (uint32_t*)(B + L.count);
    uint32_t* base = (uint32_t*)(B + L.base);
    uint16_t* sorted = (uint16_t*)(B + L.sorted);
    uint32_t* lut = (uint32_t*)(B + L.lut);

    uint32_t np = 2;
    while (np < nsym) np <<= 1;
    unsigned long long* key = (unsigned long long*)sm;              // [np]
    unsigned long long* iw = key + np;                              // [np] merged weights
    int32_t* lpar = (int32_t*)(iw + np);                            // [np] parent of each leaf
    int32_t* ipar = lpar + np;                                      // [np] parent of each merged node
    uint8_t* depth = (uint8_t*)(ipar + np);                         // [np] depth of each merged node
    __shared__ uint32_t s_cnt[66];
    __shared__ unsigned long long s_first[66];
    __shared__ uint32_t s_base[66];
    __shared__ uint32_t s_m, s_maxlen, s_ok;

    // leaves: (count, symbol) ascending; unused symbols sort to the end
    for (uint32_t i = threadIdx.x; i < np; i += blockDim.x) {
        const uint32_t c = i < nsym ? hist[i] : 0u;
        key[i] = c ? (((unsigned long long)c << 16) | i) : ~0ull;
    }
    for (uint32_t i = threadIdx.x; i < 66; i += blockDim.x) s_cnt[i] = 0;
    __syncthreads();
    bitonic_sort(key, np);
    if (threadIdx.x == 0) {
        uint32_t k = 0;
        while (k < np && key[k] != ~0ull) ++k;
        s_m = k;
        s_ok = 1;
        // two-queue merge: leaves key[0..m), merged nodes iw[0..m-1)
        uint32_t i = 0, j = 0, made = 0;
        auto pick = [&](unsigned long long* w, int* leaf, uint32_t* idx) {
            const bool take_leaf = i < k && (j >= made || (key[i] >> 16) <= iw[j]);
            if (take_leaf) {
                *w = key[i] >> 16;
                *leaf = 1;
                *idx = i++;
            } else {
                *w = iw[j];
                *leaf = 0;
                *idx = j++;
            }
        };
        for (uint32_t t = 0; k >= 2 && t + 1 < k; ++t) {
            unsigned long long wa, wb;
            int la, lb;
            uint32_t ia, ib;
            pick(&wa, &la, &ia);
            pick(&wb, &lb, &ib);
            iw[made] = wa + wb;
            ipar[made] = -1;
            if (la) lpar[ia] = (int32_t)made; else ipar[ia] = (int32_t)made;
            if (lb) lpar[ib] = (int32_t)made; else ipar[ib] = (int32_t)made;
            ++made;
        }
        // depths: the last merged node is the root; parents come after children
        uint32_t maxlen = 0;
        if (made > 0) {
            depth[made - 1] = 0;
            for (int32_t c = (int32_t)made - 2; c >= 0; --c) {
                const uint32_t d = depth[ipar[c]] + 1u;
                depth[c] = (uint8_t)(d > 255u ? 255u : d);
            }
        }
        for (uint32_t c = 0; c < k; ++c) {
            const uint32_t d = made > 0 ? depth[lpar[c]] + 1u : 1u;
            if (d > 64) s_ok = 0;
            maxlen = max(maxlen, d);
            // reuse iw as the (length, symbol) key of leaf c
            iw[c] = ((unsigned long long)d << 16) | (key[c] & 0xffffu);
        }
        s_maxlen = maxlen;
    }
    __syncthreads();
    const uint32_t mm = s_m;
    // per-symbol lengths; canonical order = sort by (length, symbol)
    for (uint32_t i = threadIdx.x; i < nsym; i += blockDim.x) len[i] = 0;
    for (uint32_t i = threadIdx.x; i < np; i += blockDim.x) key[i] = i < mm ? iw[i] : ~0ull;
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < mm; i += blockDim.x) {
        const uint32_t d = (uint32_t)(key[i] >> 16);
        len[key[i] & 0xffffu] = (uint8_t)(d > 64 ? 64 : d);
        atomicAdd(&s_cnt[d > 64 ? 64 : d], 1u);
    }
    __syncthreads();
    bitonic_sort(key, np);
    if (threadIdx.x == 0) {
        // first codeword of each length (canonical): next = (next + count) << 1
        unsigned long long c = 0;
        uint32_t b = 0;
        for (int l = 1; l <= 64; ++l) {
            c = (c + s_cnt[l - 1]) << 1;  // s_cnt[0] == 0: the first length starts at 0
            s_first[l] = c;
            s_base[l] = b;
            b += s_cnt[l];
        }
        s_first[0] = 0;
        s_base[0] = 0;
        s_first[65] = 0;
        s_base[65] = b;
        s_cnt[65] = 0;
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < nsym; i += blockDim.x) code[i] = 0;
    __syncthreads();
    for (uint32_t r = threadIdx.x; r < mm; r += blockDim.x) {
        const uint32_t l = (uint32_t)(key[r] >> 16), s = (uint32_t)(key[r] & 0xffffu);
        code[s] = s_first[l] + (r - s_base[l]);
        sorted[r] = (uint16_t)s;
    }
    for (uint32_t i = threadIdx.x; i < 66; i += blockDim.x) {
        first[i] = s_first[i];
        count[i] = s_cnt[i];
        base[i] = s_base[i];
    }
    for (uint32_t i = threadIdx.x; i < (1u << kLutBits); i += blockDim.x) lut[i] = 0;
    __syncthreads();
    for (uint32_t r = threadIdx.x; r < mm; r += blockDim.x) {
        const uint32_t l = (uint32_t)(key[r] >> 16), s = (uint32_t)(key[r] & 0xffffu);
        if (l <= (uint32_t)kLutBits) {
            const uint32_t c0 = (uint32_t)(s_first[l] + (r - s_base[l])) << (kLutBits - l);
            const uint32_t c1 = c0 + (1u << (kLutBits - l));
            for (uint32_t e = c0; e < c1; ++e) lut[e] = (l << 16) | s;
        }
    }
    if (threadIdx.x == 0) {
        hdr->nsym = nsym;
        hdr->max_len = s_maxlen;
        hdr->nused = mm;
        hdr->ok = s_ok;
    }
}

// ---------------------------------------------------------------- encoding
constexpr int kHC = VSZ_HUFF_CHUNK;
constexpr int kEncThreads = 256;
constexpr int kPerThread = kHC / kEncThreads;  // 16 symbols per thread

// Words of each chunk (its bits rounded up to 32), into off[c].
__global__ void __launch_bounds__(kEncThreads) k_huff_chunk_words(const uint16_t* __restrict__ sym, uint64_t n,
                                                                   const void* bookp, uint32_t nsym, uint64_t* off,
                                                                   uint32_t* status) {
    __shared__ uint8_t slen[kMaxSym];
    __shared__ unsigned long long red[kEncThreads / 32];
    const HuffBook bk = huff_book(bookp, nsym);
    if (bk.hdr->nsym != nsym) {  // a book built for another alphabet
        if (threadIdx.x == 0) {
            off[blockIdx.x] = 0;
            atomicOr(status, 8u);
        }
        return;
    }
    for (uint32_t i = threadIdx.x; i < nsym; i += blockDim.x) slen[i] = bk.len[i];
    __syncthreads();
    const uint64_t c = blockIdx.x;
    const uint64_t i0 = c * kHC + (uint64_t)threadIdx.x * kPerThread;
    unsigned long long bits = 0;
    bool bad = false;
    for (int k = 0; k < kPerThread; ++k) {
        const uint64_t i = i0 + k;
        if (i < n) {
            const uint32_t s = sym[i];
            const uint32_t l = s < nsym ? slen[s] : 0u;
            bad |= l == 0;
            bits += l;
        }
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(status, 1u);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) bits += __shfl_xor_sync(VSZ_FULL, bits, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = bits;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int w = 0; w < kEncThreads / 32; ++w) t += red[w];
        off[c] = (t + 31) / 32;
    }
}

// Exclusive scan of off[0..nc) in place, total into off[nc]; capacity check.
__global__ void __launch_bounds__(1024) k_huff_scan(uint64_t* off, uint64_t nc, uint64_t word_cap,
                                                    uint32_t* status) {
    __shared__ unsigned long long wsum[32];
    __shared__ unsigned long long carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (uint64_t b0 = 0; b0 < nc; b0 += blockDim.x) {
        const uint64_t i = b0 + threadIdx.x;
        const unsigned long long v = i < nc ? off[i] : 0ull;
        unsigned long long x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(VSZ_FULL, x, o);
            if ((threadIdx.x & 31) >= (unsigned)o) x += y;
        }
        if ((threadIdx.x & 31) == 31) wsum[threadIdx.x >> 5] = x;
        __syncthreads();
        if (threadIdx.x < 32) {
            unsigned long long w = wsum[threadIdx.x];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned long long y = __shfl_up_sync(VSZ_FULL, w, o);
                if (threadIdx.x >= (unsigned)o) w += y;
            }
            wsum[threadIdx.x] = w;
        }
        __syncthreads();
        const unsigned long long before = carry + (threadIdx.x >= 32 ? wsum[(threadIdx.x >> 5) - 1] : 0ull) + x - v;
        if (i < nc) off[i] = before;
        __syncthreads();
        if (threadIdx.x == 0) carry += wsum[31];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        off[nc] = carry;
        if (carry > word_cap) atomicOr(status, 2u);
    }
}

// One CTA per chunk: codeword bits packed into shared memory, then stored.
__global__ void __launch_bounds__(kEncThreads) k_huff_encode(const uint16_t* __restrict__ sym, uint64_t n,
                                                              const void* bookp, uint32_t nsym,
                                                              const uint64_t* __restrict__ off, uint32_t* words,
                                                              uint64_t word_cap) {
    extern __shared__ __align__(16) unsigned char smraw[];
    uint32_t* sw = (uint32_t*)smraw;  // [kHC * 64 / 32] words of the chunk
    __shared__ unsigned long long red[kEncThreads / 32];
    const HuffBook bk = huff_book(bookp, nsym);
    if (bk.hdr->nsym != nsym) return;
    const uint64_t c = blockIdx.x;
    const uint64_t w0 = off[c], nw = min(off[c + 1] - w0, (uint64_t)(kHC * 64 / 32));
    for (uint32_t i = threadIdx.x; i < nw; i += blockDim.x) sw[i] = 0;
    const uint64_t i0 = c * kHC + (uint64_t)threadIdx.x * kPerThread;
    uint16_t s[kPerThread];
    uint32_t mybits = 0;
#pragma unroll
    for (int k = 0; k < kPerThread; ++k) {
        const uint64_t i = i0 + k;
        s[k] = i < n ? sym[i] : (uint16_t)0xffffu;
        mybits += (i < n && s[k] < nsym) ? bk.len[s[k]] : 0u;
    }
    // exclusive scan of the threads' bit counts
    unsigned long long x = mybits;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(VSZ_FULL, x, o);
        if ((threadIdx.x & 31) >= (unsigned)o) x += y;
    }
    if ((threadIdx.x & 31) == 31) red[threadIdx.x >> 5] = x;
    __syncthreads();
    unsigned long long pos = x - mybits;
    for (uint32_t w = 0; w < (threadIdx.x >> 5); ++w) pos += red[w];
#pragma unroll
    for (int k = 0; k < kPerThread; ++k) {
        if (s[k] >= nsym) continue;
        uint32_t rem = bk.len[s[k]];
        const unsigned long long cw = bk.code[s[k]];
        while (rem > 0) {
            const uint32_t wi = (uint32_t)(pos >> 5), o = (uint32_t)(pos & 31);
            const uint32_t take = min(32u - o, rem);
            const uint32_t bits = (uint32_t)((cw >> (rem - take)) & ((take == 32) ? 0xffffffffull : ((1ull << take) - 1)));
            if (wi < nw) atomicOr(&sw[wi], bits << (32 - o - take));
            pos += take;
            rem -= take;
        }
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < nw; i += blockDim.x)
        if (w0 + i < word_cap) words[w0 + i] = sw[i];
}

// ---------------------------------------------------------------- decoding
constexpr int kDecThreads = 128;

__global__ void __launch_bounds__(kDecThreads) k_huff_decode(const uint32_t* __restrict__ words, uint64_t word_cap,
                                                              const uint64_t* __restrict__ off, uint64_t n,
                                                              const void* bookp, uint32_t nsym, uint16_t* out,
                                                              uint32_t* status) {
    __shared__ uint32_t lut[1 << kLutBits];
    __shared__ unsigned long long first[66];
    __shared__ uint32_t cnt[66], base[66];
    extern __shared__ __align__(16) unsigned char smraw[];
    uint16_t* sorted = (uint16_t*)smraw;
    const HuffBook bk = huff_book(bookp, nsym);
    if (bk.hdr->nsym != nsym) {  // a book built for another alphabet
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(status, 8u);
        return;
    }
    const uint32_t nused = min(bk.hdr->nused, nsym), maxlen = min(bk.hdr->max_len, 64u);
    for (uint32_t i = threadIdx.x; i < (1u << kLutBits); i += blockDim.x) lut[i] = bk.lut[i];
    for (uint32_t i = threadIdx.x; i < 66; i += blockDim.x) {
        first[i] = bk.first[i];
        cnt[i] = bk.count[i];
        base[i] = bk.base[i];
    }
    for (uint32_t i = threadIdx.x; i < nused; i += blockDim.x) sorted[i] = bk.sorted[i];
    __syncthreads();
    const uint64_t nc = (n + kHC - 1) / kHC;
    const uint64_t c = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nc) return;
    const uint64_t wb = off[c], we = umin64(off[c + 1], word_cap);
    const uint64_t i0 = c * kHC, i1 = umin64(n, i0 + kHC);
    // 96-bit window of words [wi, wi+3)
    uint64_t wi = 0;
    uint32_t a = 0, b = 0, d = 0;
    auto wd = [&](uint64_t k) -> uint32_t { return wb + k < we ? words[wb + k] : 0u; };
    a = wd(0);
    b = wd(1);
    d = wd(2);
    uint64_t pos = 0;
    const bool vec = (reinterpret_cast<uintptr_t>(out) & 15) == 0;
    uint32_t pk[4] = {0, 0, 0, 0};
    int np = 0;
    bool bad = false;
    for (uint64_t i = i0; i < i1; ++i) {
        const uint64_t w = pos >> 5;
        while (wi < w) {
            a = b;
            b = d;
            ++wi;
            d = wd(wi + 2);
        }
        const uint32_t o = (uint32_t)(pos & 31);
        // 64 bits starting at bit o of word wi
        const unsigned long long top = ((unsigned long long)a << 32) | b;
        const unsigned long long win = o ? (top << o) | ((unsigned long long)d >> (32 - o)) : top;
        uint32_t e = lut[(uint32_t)(win >> (64 - kLutBits))];
        uint32_t l = e >> 16, sv = e & 0xffffu;
        if (l == 0) {
            bool found = false;
            for (uint32_t L = kLutBits + 1; L <= maxlen; ++L) {
                const unsigned long long cw = win >> (64 - L);
                if (cw >= first[L] && cw - first[L] < cnt[L]) {
                    sv = sorted[base[L] + (uint32_t)(cw - first[L])];
                    l = L;
                    found = true;
                    break;
                }
            }
            if (!found) {
                bad = true;
                break;
            }
        }
        pos += l;
        if (vec) {
            const int slot = (int)((i - i0) & 7);
            pk[slot >> 1] |= sv << ((slot & 1) * 16);
            if (slot == 7) {
                *reinterpret_cast<uint4*>(out + i - 7) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                pk[0] = pk[1] = pk[2] = pk[3] = 0;
            }
            np = slot + 1;
        } else {
            out[i] = (uint16_t)sv;
        }
    }
    if (vec && !bad) {
        // tail of a chunk that ends inside an 8-symbol group
        const uint64_t done = (i1 - i0) & ~7ull;
        if (np < 8 && done < (i1 - i0))
            for (uint64_t i = i0 + done; i < i1; ++i) {
                const int slot = (int)((i - i0) & 7);
                out[i] = (uint16_t)((pk[slot >> 1] >> ((slot & 1) * 16)) & 0xffffu);
            }
    }
    if (bad || wb > we || ((pos + 31) >> 5) > we - wb) atomicOr(status, 4u);
}

static size_t dec_sorted_bytes(uint32_t nsym) { return ((size_t)nsym * 2 + 15) & ~(size_t)15; }

}  // namespace vsz

using namespace vsz;

extern "C" {

size_t vsz_huffman_book_bytes(uint32_t nsym) {
    if (nsym == 0 || nsym > kMaxSym) return 0;
    return huff_layout(nsym).total;
}

vsz_status vsz_huffman_book(const uint32_t* d_hist, uint32_t nsym, void* d_book, size_t book_bytes, void* stream) {
    if (nsym == 0) return VSZ_ERR_INVALID_ARG;
    if (nsym > kMaxSym) return VSZ_ERR_UNSUPPORTED;
    if (!d_hist || !d_book || !aligned(d_book, 16) || book_bytes < huff_layout(nsym).total) return VSZ_ERR_INVALID_ARG;
    uint32_t np = 2;
    while (np < nsym) np <<= 1;
    const size_t smem = (size_t)np * (8 + 8 + 4 + 4 + 1);
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = raise_smem_attr((const void*)k_huff_book, smem);
    if (e != cudaSuccess) return cuda_fail(e);
    {
        TraceScope ts("huff_book", s);
        k_huff_book<<<1, 1024, smem, s>>>(d_hist, nsym, d_book);
    }
    e = cudaGetLastError();
    return e == cudaSuccess ? VSZ_OK : cuda_fail(e);
}

vsz_status vsz_huffman_book_read(const void* d_book, uint32_t nsym, uint8_t* h_len, uint64_t* h_code,
                                 uint32_t* h_max_len, void* stream) {
    if (!d_book || nsym == 0 || nsym > kMaxSym) return VSZ_ERR_INVALID_ARG;
    const HuffLayout L = huff_layout(nsym);
    cudaStream_t s = (cudaStream_t)stream;
    HuffHdr h;
    cudaError_t e = cudaMemcpyAsync(&h, d_book, sizeof h, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && h_len)
        e = cudaMemcpyAsync(h_len, (const char*)d_book + L.len, nsym, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && h_code)
        e = cudaMemcpyAsync(h_code, (const char*)d_book + L.code, (size_t)nsym * 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e);
    if (h_max_len) *h_max_len = h.max_len;
    return h.ok ? VSZ_OK : VSZ_ERR_UNSUPPORTED;
}

vsz_status vsz_huffman_encode(const uint16_t* d_sym, uint64_t n, const void* d_book, uint32_t nsym,
                              uint32_t* d_words, uint64_t word_cap, uint64_t* d_chunk_off, uint32_t* d_status,
                              void* stream) {
    if (nsym == 0 || nsym > kMaxSym || !d_book || !d_chunk_off || !d_status) return VSZ_ERR_INVALID_ARG;
    if (n > 0 && (!d_sym || (word_cap > 0 && !d_words))) return VSZ_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const uint64_t nc = (n + kHC - 1) / kHC;
    if (nc >= (1ull << 31)) return VSZ_ERR_INVALID_ARG;
    cudaError_t e = cudaMemsetAsync(d_status, 0, sizeof(uint32_t), s);
    if (e != cudaSuccess) return cuda_fail(e);
    if (nc == 0) {
        e = cudaMemsetAsync(d_chunk_off, 0, sizeof(uint64_t), s);
        return e == cudaSuccess ? VSZ_OK : cuda_fail(e);
    }
    {
        TraceScope ts("huff_chunk_words", s, 0, 0, n);
        k_huff_chunk_words<<<(unsigned)nc, kEncThreads, 0, s>>>(d_sym, n, d_book, nsym, d_chunk_off, d_status);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e);
    }
    {
        TraceScope ts("huff_scan", s, 0, 0, n);
        k_huff_scan<<<1, 1024, 0, s>>>(d_chunk_off, nc, word_cap, d_status);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e);
    }
    const size_t smem = (size_t)kHC * 64 / 32 * 4;  // a chunk of 64-bit codewords at most
    if ((e = raise_smem_attr((const void*)k_huff_encode, smem)) != cudaSuccess) return cuda_fail(e);
    {
        TraceScope ts("huff_encode", s, 0, 0, n);
        k_huff_encode<<<(unsigned)nc, kEncThreads, smem, s>>>(d_sym, n, d_book, nsym, d_chunk_off, d_words, word_cap);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e);
    }
    return VSZ_OK;
}

vsz_status vsz_huffman_decode(const uint32_t* d_words, uint64_t word_cap, const uint64_t* d_chunk_off, uint64_t n,
                              const void* d_book, uint32_t nsym, uint16_t* d_sym, uint32_t* d_status, void* stream) {
    if (nsym == 0 || nsym > kMaxSym || !d_book || !d_chunk_off || !d_status) return VSZ_ERR_INVALID_ARG;
    if (n > 0 && (!d_sym || !d_words)) return VSZ_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(d_status, 0, sizeof(uint32_t), s);
    if (e != cudaSuccess) return cuda_fail(e);
    const uint64_t nc = (n + kHC - 1) / kHC;
    if (nc == 0) return VSZ_OK;
    const size_t smem = dec_sorted_bytes(nsym);
    if ((e = raise_smem_attr((const void*)k_huff_decode, smem)) != cudaSuccess) return cuda_fail(e);
    {
        TraceScope ts("huff_decode", s, 0, 0, n);
        k_huff_decode<<<(unsigned)((nc + kDecThreads - 1) / kDecThreads), kDecThreads, smem, s>>>(
            d_words, word_cap, d_chunk_off, n, d_book, nsym, d_sym, d_status);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e);
    }
    return VSZ_OK;
}

}  // extern "C"
