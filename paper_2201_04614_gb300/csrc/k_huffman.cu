// k_huffman.cu -- the entropy stage: canonical Huffman coding of the
// quantization codes (Sec. II-B: SZ Huffman-codes the integer codes that the
// dual-quantization produces).
//
// Codebook (one CTA): leaves sorted by (count, symbol) with a bitonic sort in
// shared memory, then the two-queue Huffman merge (ties: the leaf first, so
// equal weights resolve leaves before merged nodes, leaves in symbol order,
// merged nodes in merge order), depths, canonical codewords (symbols sorted
// by (length, symbol) get consecutive codes), and the canonical ranges; a
// second, many-CTA kernel fills the decoder's lookup table.
//
// Stream: chunks of VSZ_HUFF_CHUNK symbols, each starting on a 32-bit word,
// bits filling each word from its most significant bit; chunk_off[c] is the
// first word of chunk c.  Encoding: per-chunk bit counts, a scan into word
// offsets, then one warp per chunk (32 symbols per lane) packs its codewords
// into shared memory and stores the words.
// Decoding: one thread per chunk (one CTA per SM) walks its bits with a
// 2^15-entry lookup table in shared memory (two codewords per entry when
// both fit, for alphabets up to 4096 symbols) and the canonical ranges for longer codewords, over a two-word
// window fed by aligned 16-byte loads issued ahead of use.
#include <climits>

#include "common.cuh"
#include "trace.cuh"

namespace vsz {

constexpr int kLutBits = 15;  // the decoder's table: 2^15 entries, 128 KB of shared memory
// Alphabets up to 4096 symbols (R <= 2048) use two-symbol table entries:
// s1 | s2 << 12 | len1 << 24 | len2 << 28, len1 = 0 for a codeword longer
// than the table, len2 = 0 when no second codeword fits in the 15 bits.
// Larger alphabets use one-symbol entries len << 16 | s.
constexpr uint32_t kPairMaxSym = 4096;
constexpr uint32_t kMaxSym = VSZ_HUFF_MAX_SYMBOLS;

// Device codebook layout (one caller buffer).
struct HuffHdr {
    uint32_t nsym, max_len, nused, ok;
};
struct HuffLayout {
    size_t code, len, first, count, base, sorted, lut, total;
};
__host__ __device__ inline HuffLayout huff_layout(uint32_t nsym) {
    auto up = [](size_t v) { return (v + 15) & ~(size_t)15; };  // every table starts on 16 bytes
    HuffLayout L;
    size_t off = 64;
    L.code = off;   off = up(off + (size_t)nsym * 8);
    L.first = off;  off = up(off + 66 * 8);
    L.count = off;  off = up(off + 66 * 4);
    L.base = off;   off = up(off + 66 * 4);
    L.lut = off;    off = up(off + ((size_t)1 << kLutBits) * 4);
    L.len = off;    off = up(off + nsym);
    L.sorted = off; off = up(off + (size_t)nsym * 2);
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

// Bytes of the codebook kernel's sort and tree arrays (25 per padded symbol),
// rounded to 16.
__host__ __device__ inline size_t book_smem_front(uint32_t np) { return ((size_t)np * 25 + 15) & ~(size_t)15; }

__global__ void __launch_bounds__(1024, 1) k_huff_book(const uint32_t* __restrict__ hist, uint32_t nsym, void* book) {
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
    {
        // number of used symbols: the first key that is ~0 (keys are sorted)
        const uint32_t used = (uint32_t)__syncthreads_count(threadIdx.x < np && key[threadIdx.x] != ~0ull);
        uint32_t extra = 0;
        for (uint32_t i = blockDim.x + threadIdx.x; i < np; i += blockDim.x) extra += key[i] != ~0ull ? 1u : 0u;
        if (threadIdx.x == 0) s_m = used;
        __syncthreads();
        if (extra) atomicAdd(&s_m, extra);
        __syncthreads();
    }
    const uint32_t kk = s_m;
    if (threadIdx.x == 0) {
        const uint32_t k = kk;
        s_ok = 1;
        // two-queue merge: leaves key[0..k), merged nodes iw[0..k-1); the
        // first two of both queues stay in registers, so that taking a head
        // never waits for a shared-memory load
        uint32_t i = 0, j = 0, made = 0;
        unsigned long long lw = k > 0 ? key[0] >> 16 : ~0ull, lwn = k > 1 ? key[1] >> 16 : ~0ull;
        unsigned long long mw = ~0ull, mwn = ~0ull;
        for (uint32_t t = 0; k >= 2 && t + 1 < k; ++t) {
            unsigned long long w2 = 0;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const bool take_leaf = i < k && (j >= made || lw <= mw);
                unsigned long long w;
                if (take_leaf) {
                    w = lw;
                    lpar[i] = (int32_t)made;
                    ++i;
                    lw = lwn;
                    lwn = i + 1 < k ? key[i + 1] >> 16 : ~0ull;
                } else {
                    w = mw;
                    ipar[j] = (int32_t)made;
                    ++j;
                    mw = mwn;
                    mwn = j + 1 < made ? iw[j + 1] : ~0ull;
                }
                w2 += w;
            }
            iw[made] = w2;
            if (j == made) mw = w2;           // the merged queue was empty
            else if (j + 1 == made) mwn = w2;  // it held one node
            ++made;
        }
        if (made > 0) ipar[made - 1] = -1;
        s_maxlen = made;  // number of merged nodes (the root is the last)
    }
    __syncthreads();
    {
        // every leaf's length is its number of ancestors (parallel over leaves)
        const uint32_t k = kk, made = s_maxlen;
        uint32_t ml = 0;
        for (uint32_t c = threadIdx.x; c < k; c += blockDim.x) {
            uint32_t d = 1;
            if (made > 0)
                for (int32_t v = lpar[c]; ipar[v] >= 0 && d <= 64; v = ipar[v]) ++d;
            ml = max(ml, d);
            depth[c] = (uint8_t)min(d, 255u);
        }
        __syncthreads();
        if (threadIdx.x == 0) s_maxlen = 0;
        __syncthreads();
        atomicMax(&s_maxlen, ml);
        for (uint32_t c = threadIdx.x; c < k; c += blockDim.x) {
            const uint32_t d = depth[c];
            if (d > 64) atomicAnd(&s_ok, 0u);
            // iw now holds the (length, symbol) key of leaf c
            iw[c] = ((unsigned long long)d << 16) | (key[c] & 0xffffu);
        }
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
    if (threadIdx.x == 0) {
        hdr->nsym = nsym;
        hdr->max_len = s_maxlen;
        hdr->nused = mm;
        hdr->ok = s_ok;
    }
}

// The decoder's table (many CTAs, after k_huff_book): entry p holds the
// codeword that the kLutBits bits p start with (the canonical range of its
// length holds p's prefix), and for small alphabets the codeword after it
// when that one ends within the same bits (bits past them read as 0).
__global__ void __launch_bounds__(256) k_huff_lut(uint32_t nsym, void* book) {
    const HuffLayout L = huff_layout(nsym);
    char* B = (char*)book;
    const uint64_t* first = (const uint64_t*)(B + L.first);
    const uint32_t* count = (const uint32_t*)(B + L.count);
    const uint32_t* base = (const uint32_t*)(B + L.base);
    const uint16_t* sorted = (const uint16_t*)(B + L.sorted);
    uint32_t* lut = (uint32_t*)(B + L.lut);
    __shared__ unsigned long long s_first[kLutBits + 1];
    __shared__ uint32_t s_cnt[kLutBits + 1], s_base[kLutBits + 1];
    if (threadIdx.x <= (unsigned)kLutBits) {
        s_first[threadIdx.x] = first[threadIdx.x];
        s_cnt[threadIdx.x] = count[threadIdx.x];
        s_base[threadIdx.x] = base[threadIdx.x];
    }
    __syncthreads();
    auto one = [&](uint32_t p) -> uint32_t {
        for (uint32_t l = 1; l <= (uint32_t)kLutBits; ++l) {
            const unsigned long long cw = p >> (kLutBits - l);
            if (cw >= s_first[l] && cw - s_first[l] < s_cnt[l])
                return (l << 16) | sorted[s_base[l] + (uint32_t)(cw - s_first[l])];
        }
        return 0u;
    };
    const bool pair = nsym <= kPairMaxSym;
    for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < (1u << kLutBits); p += gridDim.x * blockDim.x) {
        const uint32_t e1 = one(p);
        if (!pair) {
            lut[p] = e1;
            continue;
        }
        const uint32_t l1 = e1 >> 16, s1 = e1 & 0xffffu;
        uint32_t l2 = 0, s2 = 0;
        if (l1 > 0 && l1 < (uint32_t)kLutBits) {
            const uint32_t e2 = one((p << l1) & ((1u << kLutBits) - 1));
            if ((e2 >> 16) > 0 && (e2 >> 16) <= (uint32_t)kLutBits - l1) {
                l2 = e2 >> 16;
                s2 = e2 & 0xffffu;
            }
        }
        lut[p] = l1 ? (s1 | (s2 << 12) | (l1 << 24) | (l2 << 28)) : 0u;
    }
}

// ---------------------------------------------------------------- encoding
constexpr int kHC = VSZ_HUFF_CHUNK;
constexpr int kEncThreads = 128;                // four warps; one warp codes one chunk at a time
constexpr int kLaneSyms = kHC / 32;             // 32 symbols per lane: four 16-byte loads
static_assert(kLaneSyms == 32, "a chunk is 32 lanes of 32 symbols");
constexpr int kChunkWordsMax = kHC * 64 / 32;   // a chunk of 64-bit codewords at most
constexpr uint64_t kEncMaxCtas = 4096;          // persistent CTAs of the encoder (ranges of chunks)

// The 32 symbols of lane `lane` of chunk c (0xffff past the end).
__device__ __forceinline__ void load32(const uint16_t* __restrict__ sym, uint64_t n, uint64_t c, int lane, bool vec,
                                       uint32_t (&v)[kLaneSyms]) {
    const uint64_t i0 = c * kHC + (uint64_t)lane * kLaneSyms;
    if (vec && i0 + kLaneSyms <= n) {
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const uint4 q = *reinterpret_cast<const uint4*>(sym + i0 + 8 * h);
            const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                v[8 * h + 2 * k] = w[k] & 0xffffu;
                v[8 * h + 2 * k + 1] = w[k] >> 16;
            }
        }
    } else {
#pragma unroll
        for (int k = 0; k < kLaneSyms; ++k) v[k] = i0 + k < n ? (uint32_t)sym[i0 + k] : 0xffffu;
    }
}

// The chunks of persistent CTA j of G: a contiguous range.
__device__ __forceinline__ void chunk_range(uint64_t nc, uint32_t G, uint32_t j, uint64_t* c0, uint64_t* c1) {
    const uint64_t per = (nc + G - 1) / G;
    *c0 = umin64(nc, (uint64_t)j * per);
    *c1 = umin64(nc, *c0 + per);
}

// Pass 1: the words of each chunk (its bits rounded up to 32), one warp per
// chunk; then CTA j turns its range's counts into offsets local to the
// range (off[c] = words of its chunks before c) and its total into rt[j].
__global__ void __launch_bounds__(kEncThreads) k_huff_chunk_words(const uint16_t* __restrict__ sym, uint64_t n,
                                                                   const void* bookp, uint32_t nsym, uint64_t* off,
                                                                   unsigned long long* rt, uint32_t* status) {
    __shared__ uint8_t slen[kMaxSym];
    const HuffBook bk = huff_book(bookp, nsym);
    const uint64_t nc = (n + kHC - 1) / kHC;
    uint64_t c0, c1;
    chunk_range(nc, gridDim.x, blockIdx.x, &c0, &c1);
    if (bk.hdr->nsym != nsym) {  // a book built for another alphabet
        for (uint64_t c = c0 + threadIdx.x; c < c1; c += blockDim.x) off[c] = 0;
        if (threadIdx.x == 0) {
            rt[blockIdx.x] = 0;
            atomicOr(status, 8u);
        }
        return;
    }
    for (uint32_t i = threadIdx.x; i < nsym; i += blockDim.x) slen[i] = bk.len[i];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool vec = (reinterpret_cast<uintptr_t>(sym) & 15) == 0;
    bool bad = false;
    for (uint64_t c = c0 + warp; c < c1; c += kEncThreads / 32) {
        uint32_t v[kLaneSyms];
        load32(sym, n, c, lane, vec, v);
        const uint64_t i0 = c * kHC + (uint64_t)lane * kLaneSyms;
        const uint32_t lim = i0 + kLaneSyms <= n ? (uint32_t)kLaneSyms : (uint32_t)(n > i0 ? n - i0 : 0);
        unsigned int bits = 0;
#pragma unroll
        for (int k = 0; k < kLaneSyms; ++k) {
            if ((uint32_t)k < lim) {
                const uint32_t l = v[k] < nsym ? slen[v[k]] : 0u;
                bad |= l == 0;
                bits += l;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) bits += __shfl_xor_sync(VSZ_FULL, bits, o);
        if (lane == 0) off[c] = (bits + 31u) / 32u;
    }
    __syncthreads();
    if (warp == 0) {  // range-local exclusive offsets, in place
        unsigned long long carry = 0;
        for (uint64_t b0 = c0; b0 < c1; b0 += 32) {
            const uint64_t c = b0 + lane;
            const unsigned long long w = c < c1 ? off[c] : 0ull;
            unsigned long long x = w;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned long long y = __shfl_up_sync(VSZ_FULL, x, o);
                if (lane >= o) x += y;
            }
            if (c < c1) off[c] = carry + x - w;
            carry += __shfl_sync(VSZ_FULL, x, 31);
        }
        if (lane == 0) rt[blockIdx.x] = carry;
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(status, 1u);
}

// Pass 2 (one CTA): exclusive scan of the G range totals in place, the
// stream's total into rt[G] and off[nc]; capacity check.
__global__ void __launch_bounds__(1024) k_huff_scan(unsigned long long* rt, uint32_t G, uint64_t* off, uint64_t nc,
                                                    uint64_t word_cap, uint32_t* status) {
    __shared__ unsigned long long wsum[32];
    __shared__ unsigned long long carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (uint32_t b0 = 0; b0 < G; b0 += blockDim.x) {
        const uint32_t i = b0 + threadIdx.x;
        const unsigned long long v = i < G ? rt[i] : 0ull;
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
        const unsigned long long before = carry + ((threadIdx.x >> 5) ? wsum[(threadIdx.x >> 5) - 1] : 0ull) + x - v;
        if (i < G) rt[i] = before;
        __syncthreads();
        if (threadIdx.x == 0) carry += wsum[31];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        rt[G] = carry;
        off[nc] = carry;
        if (carry > word_cap) atomicOr(status, 2u);
    }
}

// Pass 3: CTA j codes its chunks (same ranges as pass 1), one warp per
// chunk: each lane writes its 32 codewords through a 64-bit bit-writer into
// the warp's words in shared memory (the words it shares with its neighbour
// lanes by OR), then the warp stores them and the chunk's final offset
// replaces its local one.  With a decode index, lane j also records the
// chunk-relative bit where its 32 codewords start (index[32 c + j]; a chunk
// of 2^16 bits or more cannot be indexed: status bit 16).
__global__ void __launch_bounds__(kEncThreads) k_huff_encode(const uint16_t* __restrict__ sym, uint64_t n,
                                                              const void* bookp, uint32_t nsym, uint64_t* off,
                                                              const unsigned long long* __restrict__ rt,
                                                              uint32_t* words, uint64_t word_cap, uint16_t* index,
                                                              uint32_t* status) {
    __shared__ uint32_t sw[kEncThreads / 32][kChunkWordsMax];
    extern __shared__ __align__(16) unsigned char smraw[];
    unsigned long long* scode = (unsigned long long*)smraw;  // [nsym]
    uint8_t* slen = (uint8_t*)(scode + nsym);                 // [nsym]
    const HuffBook bk = huff_book(bookp, nsym);
    if (bk.hdr->nsym != nsym) return;
    for (uint32_t i = threadIdx.x; i < nsym; i += blockDim.x) {
        scode[i] = bk.code[i];
        slen[i] = bk.len[i];
    }
    __syncthreads();
    const uint64_t nc = (n + kHC - 1) / kHC;
    uint64_t c0, c1;
    chunk_range(nc, gridDim.x, blockIdx.x, &c0, &c1);
    const unsigned long long base = rt[blockIdx.x];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t* ws = sw[warp];
    const bool vec = (reinterpret_cast<uintptr_t>(sym) & 15) == 0;
    for (uint64_t c = c0 + warp; c < c1; c += kEncThreads / 32) {
        uint32_t v[kLaneSyms];
        load32(sym, n, c, lane, vec, v);
        uint32_t mybits = 0;
#pragma unroll
        for (int k = 0; k < kLaneSyms; ++k) mybits += v[k] < nsym ? slen[v[k]] : 0u;
        uint32_t x = mybits;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(VSZ_FULL, x, o);
            if (lane >= o) x += y;
        }
        const uint32_t total = __shfl_sync(VSZ_FULL, x, 31);
        const uint32_t nw = min((total + 31u) / 32u, (uint32_t)kChunkWordsMax);
        const uint32_t pos = x - mybits;  // this lane's first bit in the chunk
        if (index) {
            index[c * 32 + lane] = (uint16_t)pos;
            if (lane == 31 && total > 0xffffu) atomicOr(status, 16u);
        }
        for (uint32_t i = lane; i < nw; i += 32) ws[i] = 0;
        __syncwarp();
        // bit-writer: acc holds nacc pending bits (nacc < 32 between codes);
        // the lane's first word starts with pos & 31 bits of its neighbour
        unsigned long long acc = 0;
        uint32_t nacc = pos & 31u, wi = pos >> 5;
        auto push = [&](unsigned long long bits, uint32_t len) {  // len <= 32
            acc = (acc << len) | bits;
            nacc += len;
            if (nacc >= 32) {
                nacc -= 32;
                const uint32_t word = (uint32_t)(acc >> nacc);
                if (wi < nw) atomicOr(&ws[wi], word);
                ++wi;
                acc &= nacc ? ((1ull << nacc) - 1) : 0ull;
            }
        };
#pragma unroll
        for (int k = 0; k < kLaneSyms; ++k) {
            if (v[k] >= nsym) continue;
            const uint32_t l = slen[v[k]];
            const unsigned long long cw = scode[v[k]];
            if (l > 32) {
                push(cw >> 32, l - 32);
                push(cw & 0xffffffffull, 32);
            } else if (l) {
                push(cw, l);
            }
        }
        if (nacc > 0 && wi < nw) atomicOr(&ws[wi], (uint32_t)(acc << (32 - nacc)));
        __syncwarp();
        const uint64_t w0 = base + off[c];  // the local offset, read by this warp only
        for (uint32_t i = lane; i < nw; i += 32)
            if (w0 + i < word_cap) words[w0 + i] = ws[i];
        __syncwarp();
        if (lane == 0) off[c] = w0;  // final offset
    }
}

// ---------------------------------------------------------------- decoding
constexpr int kDecMaxThreads = 1024;  // one CTA per SM, one thread per chunk

__global__ void __launch_bounds__(kDecMaxThreads) k_huff_decode(const uint32_t* __restrict__ words, uint64_t word_cap,
                                                              const uint64_t* __restrict__ off, uint64_t n,
                                                              const void* bookp, uint32_t nsym, uint16_t* out,
                                                              uint32_t* status) {
    __shared__ unsigned long long first[66];
    __shared__ uint32_t cnt[66], base[66];
    extern __shared__ __align__(16) unsigned char smraw[];
    uint32_t* lut = (uint32_t*)smraw;                           // [2^kLutBits]
    uint16_t* sorted = (uint16_t*)(lut + (1u << kLutBits));     // [nused]
    const HuffBook bk = huff_book(bookp, nsym);
    if (bk.hdr->nsym != nsym) {  // a book built for another alphabet
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(status, 8u);
        return;
    }
    const uint32_t nused = min(bk.hdr->nused, nsym), maxlen = min(bk.hdr->max_len, 64u);
    for (uint32_t i = threadIdx.x; i < (1u << kLutBits) / 4; i += blockDim.x)
        reinterpret_cast<uint4*>(lut)[i] = __ldg(reinterpret_cast<const uint4*>(bk.lut) + i);
    for (uint32_t i = threadIdx.x; i < 66; i += blockDim.x) {
        first[i] = bk.first[i];
        cnt[i] = bk.count[i];
        base[i] = bk.base[i];
    }
    for (uint32_t i = threadIdx.x; i < nused; i += blockDim.x) sorted[i] = bk.sorted[i];
    __syncthreads();
    const uint64_t nc = (n + kHC - 1) / kHC;
    for (uint64_t c = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t wb = off[c], we = umin64(off[c + 1], word_cap);
    if (wb > we) {
        atomicOr(status, 4u);
        continue;
    }
    const uint64_t i0 = c * kHC;
    const uint32_t m = (uint32_t)(umin64(n, i0 + kHC) - i0);  // symbols of this chunk
    uint16_t* o = out + i0;
    // Words arrive through a two-deep queue of aligned 16-byte loads (the
    // words before wb in the first one are skipped), each used 4..8 words
    // after it was issued.  Words past the chunk's end are read (within
    // word_cap) but never consumed by a valid stream.
    const bool vw = (reinterpret_cast<uintptr_t>(words) & 15) == 0;
    auto ld4 = [&](uint64_t a) -> uint4 {  // a is a multiple of 4
        if (vw && a + 4 <= word_cap) return __ldg(reinterpret_cast<const uint4*>(words + a));
        uint4 r;
        r.x = a < word_cap ? __ldg(words + a) : 0u;
        r.y = a + 1 < word_cap ? __ldg(words + a + 1) : 0u;
        r.z = a + 2 < word_cap ? __ldg(words + a + 2) : 0u;
        r.w = a + 3 < word_cap ? __ldg(words + a + 3) : 0u;
        return r;
    };
    uint64_t na = wb & ~3ull;
    uint4 cur = ld4(na), nxt = ld4(na + 4);
    na += 8;
    uint32_t k = (uint32_t)(wb & 3);  // the next word of cur
    auto sel = [&]() -> uint32_t { return k == 0 ? cur.x : k == 1 ? cur.y : k == 2 ? cur.z : cur.w; };
    auto step_queue = [&]() {
        if (k == 4) {
            cur = nxt;
            nxt = ld4(na);
            na += 4;
            k = 0;
        }
    };
    // The window: the stream's next bit is bit ob (from the top) of w0; w1
    // follows w0 and sel() follows w1.
    uint32_t w0 = sel();
    ++k;
    step_queue();
    uint32_t w1 = sel();
    ++k;
    step_queue();
    uint32_t ob = 0;
    // Output: symbols gather four at a time in a 64-bit register (slot 0 the
    // oldest) and leave in 8-byte stores when out is 8-byte aligned; one
    // store per symbol if not.
    const bool vec = (reinterpret_cast<uintptr_t>(out) & 7) == 0;
    unsigned long long acc = 0;
    uint32_t pend = 0, g = 0;  // symbols in acc; symbols stored
    auto emit = [&](uint32_t val, uint32_t cnt, uint32_t i) {  // cnt symbols, the first in the low half
        if (vec) {
            acc |= (unsigned long long)val << (16 * pend);
            const uint32_t np = pend + cnt;
            if (np >= 4) {
                *reinterpret_cast<unsigned long long*>(o + g) = acc;
                g += 4;
                acc = np == 5 ? (unsigned long long)(val >> 16) : 0ull;
            }
            pend = np >= 4 ? np - 4 : np;
        } else {
            o[i] = (uint16_t)val;
            if (cnt == 2) o[i + 1] = (uint16_t)(val >> 16);
        }
    };
    const bool pair = nsym <= kPairMaxSym;
    bool bad = false;
    uint32_t used = 0;  // bits consumed
    for (uint32_t i = 0; i < m;) {
        const uint32_t e = lut[__funnelshift_l(w1, w0, ob) >> (32 - kLutBits)];
        uint32_t l, sv, l2 = 0, sv2 = 0;
        if (pair) {
            l = (e >> 24) & 15u;
            sv = e & 0xfffu;
            l2 = e >> 28;
            sv2 = (e >> 12) & 0xfffu;
        } else {
            l = e >> 16;
            sv = e & 0xffffu;
        }
        if (l == 0) {  // a codeword longer than the table: the canonical ranges on a 64-bit window
            const uint32_t w2 = sel();
            const unsigned long long win = ((unsigned long long)__funnelshift_l(w1, w0, ob) << 32) |
                                           __funnelshift_l(w2, w1, ob);
            for (uint32_t L = kLutBits + 1; L <= maxlen; ++L) {
                const unsigned long long cw = win >> (64 - L);
                if (cw >= first[L] && cw - first[L] < cnt[L]) {
                    sv = sorted[base[L] + (uint32_t)(cw - first[L])];
                    l = L;
                    break;
                }
            }
            if (l == 0) {
                bad = true;
                break;
            }
            emit(sv, 1, i);
            used += l;
            ob += l;
            while (ob >= 32) {  // at most twice
                w0 = w1;
                w1 = sel();
                ++k;
                step_queue();
                ob -= 32;
            }
            ++i;
            continue;
        }
        if (i + 1 >= m) l2 = 0;  // the chunk's last symbol: what follows is padding
        const uint32_t t = l + l2;  // <= 12
        emit(l2 ? sv | (sv2 << 16) : sv, l2 ? 2u : 1u, i);
        used += t;
        i += l2 ? 2 : 1;
        ob += t;
        const bool adv = ob >= 32;
        const uint32_t wn = sel();
        w0 = adv ? w1 : w0;
        w1 = adv ? wn : w1;
        ob -= adv ? 32u : 0u;
        k += adv ? 1u : 0u;
        step_queue();
    }
    if (vec && !bad) {  // the last 0..3 symbols
        for (uint32_t j = 0; j < pend; ++j) o[g + j] = (uint16_t)(acc >> (16 * j));
    }
    if (bad || ((uint64_t)(used + 31) >> 5) > we - wb) atomicOr(status, 4u);
    }
}

// Indexed decoding: one warp per chunk; lane j decodes the chunk's codes
// 32j..32j+31 starting at the bit index[32 c + j] that the encoder recorded,
// over a two-word window whose words it reads through L1 (the chunk's words
// are shared by its lanes).  Same table and canonical ranges as above.  A
// lane whose codes do not end exactly where the next lane's start (or past
// the chunk's words, for the last lane) reports status bit 4.
__global__ void __launch_bounds__(kDecMaxThreads) k_huff_decode_ix(const uint32_t* __restrict__ words,
                                                                 uint64_t word_cap, const uint64_t* __restrict__ off,
                                                                 const uint16_t* __restrict__ index, uint64_t n,
                                                                 const void* bookp, uint32_t nsym, uint16_t* out,
                                                                 uint32_t* status) {
    __shared__ unsigned long long first[66];
    __shared__ uint32_t cnt[66], base[66];
    extern __shared__ __align__(16) unsigned char smraw[];
    uint32_t* lut = (uint32_t*)smraw;                           // [2^kLutBits]
    uint16_t* sorted = (uint16_t*)(lut + (1u << kLutBits));     // [nused]
    const HuffBook bk = huff_book(bookp, nsym);
    if (bk.hdr->nsym != nsym) {
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(status, 8u);
        return;
    }
    const uint32_t nused = min(bk.hdr->nused, nsym), maxlen = min(bk.hdr->max_len, 64u);
    for (uint32_t i = threadIdx.x; i < (1u << kLutBits) / 4; i += blockDim.x)
        reinterpret_cast<uint4*>(lut)[i] = __ldg(reinterpret_cast<const uint4*>(bk.lut) + i);
    for (uint32_t i = threadIdx.x; i < 66; i += blockDim.x) {
        first[i] = bk.first[i];
        cnt[i] = bk.count[i];
        base[i] = bk.base[i];
    }
    for (uint32_t i = threadIdx.x; i < nused; i += blockDim.x) sorted[i] = bk.sorted[i];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const uint64_t nc = (n + kHC - 1) / kHC;
    const uint64_t nwarps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    const bool vec = (reinterpret_cast<uintptr_t>(out) & 7) == 0;
    const bool pair = nsym <= kPairMaxSym;
    auto rd = [&](uint64_t a) -> uint32_t { return a < word_cap ? __ldg(words + a) : 0u; };
    for (uint64_t c = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); c < nc; c += nwarps) {
        const uint64_t wb = off[c], we = umin64(off[c + 1], word_cap);
        if (wb > we) {
            if (lane == 0) atomicOr(status, 4u);
            continue;
        }
        const uint32_t start = index[c * 32 + lane];
        const uint64_t i0 = c * kHC + (uint64_t)lane * kLaneSyms;
        const uint32_t m = i0 < n ? (uint32_t)umin64(kLaneSyms, n - i0) : 0u;  // this lane's codes
        uint16_t* o = out + i0;
        uint64_t nxt = wb + (start >> 5);
        uint32_t w0 = rd(nxt), w1 = rd(nxt + 1);
        nxt += 2;
        uint32_t ob = start & 31u;
        unsigned long long acc = 0;
        uint32_t pend = 0, g = 0;
        auto emit = [&](uint32_t val, uint32_t k, uint32_t i) {  // k symbols, the first in the low half
            if (vec) {
                acc |= (unsigned long long)val << (16 * pend);
                const uint32_t np = pend + k;
                if (np >= 4) {
                    *reinterpret_cast<unsigned long long*>(o + g) = acc;
                    g += 4;
                    acc = np == 5 ? (unsigned long long)(val >> 16) : 0ull;
                }
                pend = np >= 4 ? np - 4 : np;
            } else {
                o[i] = (uint16_t)val;
                if (k == 2) o[i + 1] = (uint16_t)(val >> 16);
            }
        };
        bool bad = false;
        uint32_t used = 0;
        for (uint32_t i = 0; i < m;) {
            const uint32_t e = lut[__funnelshift_l(w1, w0, ob) >> (32 - kLutBits)];
            uint32_t l, sv, l2 = 0, sv2 = 0;
            if (pair) {
                l = (e >> 24) & 15u;
                sv = e & 0xfffu;
                l2 = e >> 28;
                sv2 = (e >> 12) & 0xfffu;
            } else {
                l = e >> 16;
                sv = e & 0xffffu;
            }
            if (l == 0) {  // a codeword longer than the table: the canonical ranges on a 64-bit window
                const uint32_t w2 = rd(nxt);
                const unsigned long long win = ((unsigned long long)__funnelshift_l(w1, w0, ob) << 32) |
                                               __funnelshift_l(w2, w1, ob);
                for (uint32_t L = kLutBits + 1; L <= maxlen; ++L) {
                    const unsigned long long cw = win >> (64 - L);
                    if (cw >= first[L] && cw - first[L] < cnt[L]) {
                        sv = sorted[base[L] + (uint32_t)(cw - first[L])];
                        l = L;
                        break;
                    }
                }
                if (l == 0) {
                    bad = true;
                    break;
                }
                emit(sv, 1, i);
                used += l;
                ob += l;
                while (ob >= 32) {  // at most twice
                    w0 = w1;
                    w1 = rd(nxt++);
                    ob -= 32;
                }
                ++i;
                continue;
            }
            if (i + 1 >= m) l2 = 0;  // the lane's last code: what follows is the next lane's
            const uint32_t t = l + l2;  // <= 15
            emit(l2 ? sv | (sv2 << 16) : sv, l2 ? 2u : 1u, i);
            used += t;
            i += l2 ? 2 : 1;
            ob += t;
            if (ob >= 32) {
                w0 = w1;
                w1 = rd(nxt++);
                ob -= 32;
            }
        }
        if (vec && !bad)
            for (uint32_t j = 0; j < pend; ++j) o[g + j] = (uint16_t)(acc >> (16 * j));
        const bool ends = lane < 31 ? start + used == (uint32_t)index[c * 32 + lane + 1]
                                    : ((uint64_t)start + used + 31) / 32 <= we - wb;
        if (bad || !ends) atomicOr(status, 4u);
    }
}

static size_t dec_smem_bytes(uint32_t nsym) { return ((size_t)1 << kLutBits) * 4 + (((size_t)nsym * 2 + 15) & ~(size_t)15); }

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
    const size_t smem = book_smem_front(np);
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = raise_smem_attr((const void*)k_huff_book, smem);
    if (e != cudaSuccess) return cuda_fail(e);
    {
        TraceScope ts("huff_book", s);
        k_huff_book<<<1, 1024, smem, s>>>(d_hist, nsym, d_book);
        if ((e = cudaGetLastError()) == cudaSuccess)
            k_huff_lut<<<(1u << kLutBits) / 256, 256, 0, s>>>(nsym, d_book);
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

// One wave of the coding pass: the SMs times the CTAs of k_huff_encode an SM
// holds with the book's tables in shared memory.
static uint32_t encode_ctas(uint64_t nc, size_t smem) {
    const int occ = occupancy((const void*)k_huff_encode, kEncThreads, smem);
    const uint64_t g = umin64(nc, umin64((uint64_t)num_sms() * (uint64_t)(occ > 0 ? occ : 1), kEncMaxCtas));
    return (uint32_t)(g ? g : 1);
}

size_t vsz_huffman_encode_workspace_size(uint64_t n) {
    (void)n;
    return (kEncMaxCtas + 1) * sizeof(unsigned long long);
}

static vsz_status huffman_encode_impl(const uint16_t* d_sym, uint64_t n, const void* d_book, uint32_t nsym,
                                      uint32_t* d_words, uint64_t word_cap, uint64_t* d_chunk_off, uint16_t* d_index,
                                      uint32_t* d_status, void* d_ws, size_t ws_bytes, void* stream) {
    if (nsym == 0 || nsym > kMaxSym || !d_book || !aligned(d_book, 16) || !d_chunk_off || !d_status)
        return VSZ_ERR_INVALID_ARG;
    if (n > 0 && (!d_sym || (word_cap > 0 && !d_words))) return VSZ_ERR_INVALID_ARG;
    if (!d_ws || !aligned(d_ws, 8) || ws_bytes < vsz_huffman_encode_workspace_size(n)) return VSZ_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const uint64_t nc = (n + kHC - 1) / kHC;
    if (nc >= (1ull << 31)) return VSZ_ERR_INVALID_ARG;
    cudaError_t e = cudaMemsetAsync(d_status, 0, sizeof(uint32_t), s);
    if (e != cudaSuccess) return cuda_fail(e);
    if (nc == 0) {
        e = cudaMemsetAsync(d_chunk_off, 0, sizeof(uint64_t), s);
        return e == cudaSuccess ? VSZ_OK : cuda_fail(e);
    }
    unsigned long long* rt = (unsigned long long*)d_ws;
    const size_t smem = (size_t)nsym * 9;  // codeword and length tables
    if ((e = raise_smem_attr((const void*)k_huff_encode, smem)) != cudaSuccess) return cuda_fail(e);
    const uint32_t G = encode_ctas(nc, smem);
    {
        TraceScope ts("huff_chunk_words", s, 0, 0, n);
        k_huff_chunk_words<<<G, kEncThreads, 0, s>>>(d_sym, n, d_book, nsym, d_chunk_off, rt, d_status);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e);
    }
    {
        TraceScope ts("huff_scan", s, 0, 0, n);
        k_huff_scan<<<1, 1024, 0, s>>>(rt, G, d_chunk_off, nc, word_cap, d_status);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e);
    }
    {
        TraceScope ts("huff_encode", s, 0, 0, n);
        k_huff_encode<<<G, kEncThreads, smem, s>>>(d_sym, n, d_book, nsym, d_chunk_off, rt, d_words, word_cap,
                                                   d_index, d_status);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e);
    }
    return VSZ_OK;
}

vsz_status vsz_huffman_encode(const uint16_t* d_sym, uint64_t n, const void* d_book, uint32_t nsym,
                              uint32_t* d_words, uint64_t word_cap, uint64_t* d_chunk_off, uint32_t* d_status,
                              void* d_ws, size_t ws_bytes, void* stream) {
    return huffman_encode_impl(d_sym, n, d_book, nsym, d_words, word_cap, d_chunk_off, nullptr, d_status, d_ws,
                               ws_bytes, stream);
}

vsz_status vsz_huffman_encode_indexed(const uint16_t* d_sym, uint64_t n, const void* d_book, uint32_t nsym,
                                      uint32_t* d_words, uint64_t word_cap, uint64_t* d_chunk_off, uint16_t* d_index,
                                      uint32_t* d_status, void* d_ws, size_t ws_bytes, void* stream) {
    if (n > 0 && !d_index) return VSZ_ERR_INVALID_ARG;
    return huffman_encode_impl(d_sym, n, d_book, nsym, d_words, word_cap, d_chunk_off, d_index, d_status, d_ws,
                               ws_bytes, stream);
}

vsz_status vsz_huffman_decode(const uint32_t* d_words, uint64_t word_cap, const uint64_t* d_chunk_off, uint64_t n,
                              const void* d_book, uint32_t nsym, uint16_t* d_sym, uint32_t* d_status, void* stream) {
    if (nsym == 0 || nsym > kMaxSym || !d_book || !aligned(d_book, 16) || !d_chunk_off || !d_status)
        return VSZ_ERR_INVALID_ARG;
    if (n > 0 && (!d_sym || !d_words)) return VSZ_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(d_status, 0, sizeof(uint32_t), s);
    if (e != cudaSuccess) return cuda_fail(e);
    const uint64_t nc = (n + kHC - 1) / kHC;
    if (nc == 0) return VSZ_OK;
    const size_t smem = dec_smem_bytes(nsym);
    if ((e = raise_smem_attr((const void*)k_huff_decode, smem)) != cudaSuccess) return cuda_fail(e);
    // one CTA per SM (the table fills most of its shared memory), a thread
    // per chunk, threads looping when there are more chunks than that
    const uint64_t sms = (uint64_t)num_sms();
    const uint64_t G = umin64(sms, (nc + 31) / 32);
    const uint64_t T = umin64((uint64_t)kDecMaxThreads, ((nc + G - 1) / G + 31) / 32 * 32);
    {
        TraceScope ts("huff_decode", s, 0, 0, n);
        k_huff_decode<<<(unsigned)G, (unsigned)T, smem, s>>>(
            d_words, word_cap, d_chunk_off, n, d_book, nsym, d_sym, d_status);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e);
    }
    return VSZ_OK;
}

vsz_status vsz_huffman_decode_indexed(const uint32_t* d_words, uint64_t word_cap, const uint64_t* d_chunk_off,
                                      const uint16_t* d_index, uint64_t n, const void* d_book, uint32_t nsym,
                                      uint16_t* d_sym, uint32_t* d_status, void* stream) {
    if (nsym == 0 || nsym > kMaxSym || !d_book || !aligned(d_book, 16) || !d_chunk_off || !d_status)
        return VSZ_ERR_INVALID_ARG;
    if (n > 0 && (!d_sym || !d_words || !d_index)) return VSZ_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(d_status, 0, sizeof(uint32_t), s);
    if (e != cudaSuccess) return cuda_fail(e);
    const uint64_t nc = (n + kHC - 1) / kHC;
    if (nc == 0) return VSZ_OK;
    const size_t smem = dec_smem_bytes(nsym);
    if ((e = raise_smem_attr((const void*)k_huff_decode_ix, smem)) != cudaSuccess) return cuda_fail(e);
    // one CTA of 32 warps per SM (the table fills most of its shared memory),
    // a warp per chunk, warps looping when there are more chunks than that
    const uint64_t G = umin64((uint64_t)num_sms(), (nc + 31) / 32);
    {
        TraceScope ts("huff_decode_ix", s, 0, 0, n);
        k_huff_decode_ix<<<(unsigned)G, kDecMaxThreads, smem, s>>>(d_words, word_cap, d_chunk_off, d_index, n,
                                                                   d_book, nsym, d_sym, d_status);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e);
    }
    return VSZ_OK;
}

}  // extern "C"
