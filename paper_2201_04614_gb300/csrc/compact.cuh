// compact.cuh -- outlier compaction (the second step of compression).
//
// Part 1 scans the per-chunk totals of one field (one CTA); part 2, one CTA
// per chunk of 32 tiles, turns the in-tile block offsets left by the
// compression kernel into global ones and moves each tile's staged outliers
// and fixups, which are contiguous both in staging and in the final lists, to
// their canonical place.  With block-slot staging (2D/3D) part 2 gathers the
// tile's outliers from its blocks' slots instead.  Both bodies serve the single-field kernels
// (k_misc.cu) and the batch kernels (k_batch.cu).
#pragma once

#include <climits>

#include "common.cuh"

namespace vsz {

// Compaction, part 1: exclusive scan of the per-chunk totals (one CTA of 1024 threads).
__device__ __forceinline__ void compact_scan_body(uint4* chunks, uint64_t nchunks, vsz_header* hdr,
                                                  uint32_t* blk_off, uint64_t nb, uint64_t out_cap,
                                                  uint64_t fix_cap) {
    __shared__ unsigned long long so[32], sf[32];
    unsigned long long carry_o = 0, carry_f = 0;
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    for (uint64_t b0 = 0; b0 < nchunks; b0 += blockDim.x) {
        const uint64_t i = b0 + threadIdx.x;
        const uint4 c = i < nchunks ? chunks[i] : make_uint4(0, 0, 0, 0);
        unsigned long long io = c.x, iff = c.y;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const unsigned long long yo = __shfl_up_sync(VSZ_FULL, io, off);
            const unsigned long long yf = __shfl_up_sync(VSZ_FULL, iff, off);
            if (l >= off) { io += yo; iff += yf; }
        }
        if (l == 31) { so[w] = io; sf[w] = iff; }
        __syncthreads();
        if (w == 0) {
            unsigned long long vo = so[l], vf = sf[l];
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const unsigned long long yo = __shfl_up_sync(VSZ_FULL, vo, off);
                const unsigned long long yf = __shfl_up_sync(VSZ_FULL, vf, off);
                if (l >= off) { vo += yo; vf += yf; }
            }
            so[l] = vo;  // inclusive over warps
            sf[l] = vf;
        }
        __syncthreads();
        const unsigned long long wo = w ? so[w - 1] : 0ull, wf = w ? sf[w - 1] : 0ull;
        if (i < nchunks) {
            chunks[i].z = (uint32_t)(carry_o + wo + io - c.x);
            chunks[i].w = (uint32_t)(carry_f + wf + iff - c.y);
        }
        carry_o += so[31];
        carry_f += sf[31];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        hdr->n_out = carry_o;
        hdr->n_fix = carry_f;
        blk_off[nb] = (uint32_t)carry_o;
        if (carry_o > out_cap || carry_f > fix_cap) hdr->status = VSZ_ERR_CAPACITY;
    }
}

// Compaction, part 2: per chunk of tiles (one CTA), the tiles' offsets, the blocks'
// final offsets (in-tile prefix + tile offset) and the move of each tile's
// staged entries to their canonical place.  With a global padding mode, the
// origin pass may have added an outlier at the origin of some blocks: it
// goes first in its block, so the block's staged entries and every later
// block of the tile shift by the number of such origins before them.
__device__ __forceinline__ void compact_chunk_body(uint64_t chunk, const CompressArgs& a) {
    __shared__ uint4 rec[kTilesPerChunk];
    __shared__ uint32_t toff_o[kTilesPerChunk], toff_f[kTilesPerChunk];
    __shared__ uint32_t fw[8][32], fpre[8][32];  // per warp: origin-outlier bits of a tile, prefix popcounts
    const Geom& g = a.g;
    const uint64_t ntiles = g.ntiles, nseg = g.nseg, nbx = g.nbx;
    const uint32_t bpt = g.bpt;
    const uint64_t t0 = chunk * kTilesPerChunk;
    // A chunk with no outliers in it or before it has its block offsets
    // final as the walk left them (in-tile, and zero): only its fixups, if
    // it has any, move.
    const uint4 ch = a.chunks[chunk];  // {outliers, fixups, offset of outliers, offset of fixups}
    const bool outl = (ch.x | ch.z) != 0u;
    if (!outl && ch.y == 0u) return;
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (w == 0) {  // the chunk's tile offsets: chunk offset + exclusive scan of the tile totals
        uint32_t bo = ch.z, bf = ch.w;
        for (int i0 = 0; i0 < kTilesPerChunk; i0 += 32) {
            const uint64_t t = t0 + i0 + l;
            const uint4 r = t < ntiles ? a.tiles[t] : make_uint4(0, 0, 0, 0);
            uint32_t io = r.y, iff = r.w;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const uint32_t yo = __shfl_up_sync(VSZ_FULL, io, off);
                const uint32_t yf = __shfl_up_sync(VSZ_FULL, iff, off);
                if (l >= off) { io += yo; iff += yf; }
            }
            rec[i0 + l] = r;
            toff_o[i0 + l] = bo + io - r.y;
            toff_f[i0 + l] = bf + iff - r.w;
            bo += __shfl_sync(VSZ_FULL, io, 31);
            bf += __shfl_sync(VSZ_FULL, iff, 31);
        }
    }
    __syncthreads();

    const int nt = (int)umin64(kTilesPerChunk, ntiles - t0);
    for (int j = w; j < nt; j += 8) {
        const uint64_t tt = t0 + j;
        const uint4 rr = rec[j];
        const uint32_t to = toff_o[j], tf = toff_f[j];
        const uint64_t s = tt % nseg;
        const uint64_t fb = (tt / nseg) * nbx + s * bpt;
        const uint32_t nblk = (uint32_t)umin64(bpt, nbx - s * bpt);
        if (outl) {
            // origin outliers of this tile's blocks (global padding only)
            uint32_t nflag = 0;
            const uint32_t nwords = (nblk + 31) / 32;
            if (a.oflag) {
                for (uint32_t wd = 0; wd < nwords; ++wd) {
                    const uint32_t k = wd * 32 + l;
                    const uint32_t bits = __ballot_sync(VSZ_FULL, k < nblk && a.oflag[fb + k] != 0);
                    if (l == 0) fw[w][wd] = bits;
                    nflag += __popc(bits);
                }
            }
            const uint32_t staged = rr.y - nflag;
            if (nflag == 0) {
                for (uint32_t k = l; k < nblk; k += 32) a.blk_off[fb + k] += to;
                if (rr.y && (uint64_t)rr.x + rr.y <= a.out_cap && (uint64_t)to + rr.y <= a.out_cap) {
                    uint32_t k = l;
                    for (; k + 96 < rr.y; k += 128) {  // four loads in flight per lane
                        uint2 e[4];
#pragma unroll
                        for (int u = 0; u < 4; ++u) e[u] = a.stage_out[rr.x + k + 32 * u];
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            a.out_idx[to + k + 32 * u] = e[u].x;
                            a.out_delta[to + k + 32 * u] = (int32_t)e[u].y;
                        }
                    }
                    for (; k < rr.y; k += 32) {
                        const uint2 e = a.stage_out[rr.x + k];
                        a.out_idx[to + k] = e.x;
                        a.out_delta[to + k] = (int32_t)e.y;
                    }
                }
            } else {
                __syncwarp();
                {  // exclusive prefix of the words' popcounts (nwords <= 32)
                    const uint32_t c = l < (int)nwords ? __popc(fw[w][l]) : 0u;
                    uint32_t inc = c;
#pragma unroll
                    for (int off = 1; off < 32; off <<= 1) {
                        const uint32_t y = __shfl_up_sync(VSZ_FULL, inc, off);
                        if (l >= off) inc += y;
                    }
                    if (l < (int)nwords) fpre[w][l] = inc - c;
                }
                __syncwarp();
                // flagged origins before block k, and k's own flag
                auto before = [&](uint32_t k) {
                    return fpre[w][k >> 5] + __popc(fw[w][k >> 5] & ((1u << (k & 31)) - 1u));
                };
                const bool fits = (uint64_t)to + rr.y <= a.out_cap;
                for (uint32_t k = l; k < nblk; k += 32) {
                    const uint32_t np = a.blk_off[fb + k] + before(k);
                    a.blk_off[fb + k] = to + np;
                    if (fits && ((fw[w][k >> 5] >> (k & 31)) & 1u)) {
                        uint64_t idx, tile;
                        block_origin(g, fb + k, &idx, &tile);
                        a.out_idx[to + np] = (uint32_t)idx;
                        a.out_delta[to + np] = a.origin[fb + k];
                    }
                }
                if (staged && (uint64_t)rr.x + staged <= a.out_cap && fits) {
                    // block of an entry inside the tile, from its element index
                    const uint32_t nx32 = (uint32_t)g.nx, c0 = (uint32_t)(s * kSegCols), e0 = (uint32_t)(tt * kChunk1D);
                    auto place = [&](uint32_t i, uint2 e) {
                        const uint32_t k = (g.nd == 1 ? e.x - e0 : e.x % nx32 - c0) / g.b;
                        const uint32_t pos = to + i + before(k) + ((fw[w][k >> 5] >> (k & 31)) & 1u);
                        a.out_idx[pos] = e.x;
                        a.out_delta[pos] = (int32_t)e.y;
                    };
                    uint32_t i = l;
                    for (; i + 96 < staged; i += 128) {  // four loads in flight per lane
                        uint2 e[4];
#pragma unroll
                        for (int u = 0; u < 4; ++u) e[u] = a.stage_out[rr.x + i + 32 * u];
#pragma unroll
                        for (int u = 0; u < 4; ++u) place(i + 32 * u, e[u]);
                    }
                    for (; i < staged; i += 32) place(i, a.stage_out[rr.x + i]);
                }
            }
        }
        if (rr.w && (uint64_t)rr.z + rr.w <= a.fix_cap && (uint64_t)tf + rr.w <= a.fix_cap) {
            for (uint32_t k = l; k < rr.w; k += 32) {
                const uint2 e = a.stage_fix[rr.z + k];
                a.fix_idx[tf + k] = e.x;
                a.fix_bits[tf + k] = e.y;
            }
        }
    }
}

// Compaction, part 2, with block-slot staging (2D/3D).  Outliers cluster
// where the field is rough, so one chunk can hold most of a field's
// entries: a chunk is served by up to kSplit CTAs (split 0..kSplit-1), each
// moving an equal share of the chunk's places, and a CTA whose share is
// empty returns at once.  A CTA owns the chunk's tiles whose first place
// falls in its share (the last split also those starting at the chunk's
// end): it writes their blocks' final offsets (blk_off) and places their
// origin outliers (global or edge padding: a block's first entry).  It
// builds in shared memory a table of the blocks that hold entries, for the
// tiles it owns or whose places meet its share, in order: each one's first
// place relative to the chunk (tile offset + the block's in-tile offset
// from the walk + the origin outliers of the tile's earlier blocks) and the
// slot index of that place.  A block's places are its origin outlier, if
// any, then its slot entries, from slot 1 on, or from slot 0 when a
// per-block padding mode put the block's origin there.  A warp moves a
// contiguous run of the share, 32 places at a time: with k0 the block
// holding the window's first place qs, lane j reads the first place of
// block k0+1+j, and since first places strictly increase, the OR over the
// lanes of 1 << (first - qs) (for those inside the window) marks where
// blocks start; place qs+i is in block k0 + the marks at 1..i.  Split 0
// moves the fixups (contiguous per tile in staging and in the list).
constexpr int kSplit = 8;                    // CTAs per chunk at most
constexpr uint32_t kSplitMinEntries = 4096;  // entries a CTA moves at least before the chunk is split further
constexpr int kMoveWindows = 8;              // 32-place windows a warp maps before it moves them

// Splits a chunk of `entries` outliers needs (the per-field launch gives
// every chunk kSplit CTAs; a batch lists the extra ones of its dense chunks).
__host__ __device__ inline uint32_t chunk_splits(uint32_t entries) {
    const uint32_t ns = (entries + kSplitMinEntries - 1) / kSplitMinEntries;
    return ns < 1u ? 1u : ns > (uint32_t)kSplit ? (uint32_t)kSplit : ns;
}

__device__ __forceinline__ void compact_chunk_body_slots(uint64_t chunk, int split, const CompressArgs& a) {
    constexpr int kTab = kTilesPerChunk * 32;          // blocks of a chunk at most (32 per tile)
    constexpr uint64_t kOrig = 1ull << 63;             // source word flag: the block's origin outlier comes first
    __shared__ uint32_t s_first[kTab + 32];            // blocks with entries: first place (then sentinels)
    __shared__ uint64_t s_src[kTab];                   // ... slot index of place 0 (place r: + r)
    __shared__ uint32_t s_toff[kTilesPerChunk + 1], s_tfix[kTilesPerChunk], s_nblk[kTilesPerChunk];
    __shared__ uint64_t s_fb[kTilesPerChunk];          // first block of each tile
    __shared__ uint4 s_rec[kTilesPerChunk];
    __shared__ uint32_t s_wtot[kTab / 32];             // blocks with entries per warp and round
    const Geom& g = a.g;
    const uint32_t bpt = g.bpt, lb = (uint32_t)(__ffs(bpt) - 1);  // blocks per tile: a power of two
    const uint64_t S = block_slot(g.nd, g.b);
    const bool bp = is_block_pad(a.pad_mode);
    const uint64_t t0 = chunk * kTilesPerChunk;
    const int nt = (int)umin64(kTilesPerChunk, g.ntiles - t0);
    const uint4 ch = a.chunks[chunk];  // {outliers, fixups, offset of outliers, offset of fixups}
    const uint32_t E = ch.x;
    const uint32_t ns = chunk_splits(E);
    if (split > 0 && (uint32_t)split >= ns) return;
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (w == 0) {  // tile records, chunk-relative tile offsets, tile geometry
        // (a chunk without entries has tile records of zeros: not read)
        const uint4 r = (l < nt && (E | ch.y) != 0u) ? a.tiles[t0 + l] : make_uint4(0, 0, 0, 0);
        uint32_t io = r.y, iff = r.w;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t yo = __shfl_up_sync(VSZ_FULL, io, off);
            const uint32_t yf = __shfl_up_sync(VSZ_FULL, iff, off);
            if (l >= off) { io += yo; iff += yf; }
        }
        s_rec[l] = r;
        s_toff[l] = io - r.y;
        s_tfix[l] = iff - r.w;
        if (l == 31) s_toff[32] = io;
        const uint64_t tt = t0 + (uint64_t)l;
        const uint64_t row = tt / g.nseg, sg = tt - row * g.nseg;
        s_fb[l] = row * g.nbx + sg * bpt;
        s_nblk[l] = l < nt ? (uint32_t)umin64(bpt, g.nbx - sg * bpt) : 0u;
    }
    __syncthreads();
    // this CTA's share of places, the tiles it owns and the tiles it needs
    const uint32_t q0 = (uint32_t)((uint64_t)E * (uint32_t)split / ns);
    const uint32_t q1 = (uint32_t)((uint64_t)E * ((uint32_t)split + 1) / ns);
    const bool lastsplit = (uint32_t)split + 1 == ns;
    uint32_t owned, needed;
    {
        const uint32_t tj = s_toff[l], tj1 = s_toff[l + 1];
        const bool valid = l < nt;
        const bool own = valid && tj >= q0 && (tj < q1 || lastsplit);
        const bool meets = valid && tj < q1 && tj1 > q0;
        owned = __ballot_sync(VSZ_FULL, own);
        needed = owned | __ballot_sync(VSZ_FULL, meets);
    }
    const uint32_t ja = needed ? (uint32_t)(__ffs(needed) - 1) : 0u;
    const uint32_t jb = needed ? (uint32_t)(31 - __clz(needed)) : 0u;
    const uint32_t ibase = ja << lb, ntab = needed ? (jb - ja + 1u) << lb : 0u;
    // the table: four entries per thread at most, one round of loads; a
    // warp's lanes cover whole tiles (bpt divides 32)
    constexpr int kPer = kTab / 256;
    const uint32_t tmask = bpt >= 32 ? VSZ_FULL : (((1u << bpt) - 1u) << (l & ~(bpt - 1)));  // this lane's tile
    const uint32_t lt = (1u << l) - 1u;
    uint32_t eo[kPer], fl[kPer], s0[kPer];
    uint64_t bk[kPer];
    bool has[kPer];
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
        const uint32_t i = (uint32_t)threadIdx.x + 256u * u;
        const uint32_t j = (ibase + i) >> lb, k = (ibase + i) & (bpt - 1u);
        has[u] = i < ntab && k < s_nblk[j < 32u ? j : 0u];
        bk[u] = s_fb[j < 32u ? j : 0u] + k;
        // a chunk without outliers (E = 0: none staged, no origin outlier)
        // has every in-tile offset zero and no slot to move from
        const bool rd = has[u] && E != 0u;
        eo[u] = rd ? a.blk_in[bk[u]] : 0u;
        fl[u] = (rd && a.oflag && a.oflag[bk[u]] != 0) ? 1u : 0u;
        s0[u] = (bp && rd && a.slots[bk[u] * S].x != 0xffffffffu) ? 1u : 0u;
    }
    uint32_t first[kPer], keep[kPer];
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
        const uint32_t i = (uint32_t)threadIdx.x + 256u * u;
        const uint32_t j = i < ntab ? (ibase + i) >> lb : 0u;
        const uint32_t fls = __ballot_sync(VSZ_FULL, fl[u] != 0u) & tmask & lt;
        first[u] = has[u] ? s_toff[j] + eo[u] + (uint32_t)__popc(fls) : s_toff[j + 1];
        uint32_t nxt = __shfl_down_sync(VSZ_FULL, first[u], 1);
        if ((i & (bpt - 1u)) == bpt - 1u) nxt = s_toff[j + 1];  // the tile's last block: up to the tile's end
        keep[u] = (has[u] && nxt > first[u]) ? 1u : 0u;
        if (has[u] && ((owned >> j) & 1u) && VSZ_IN(bk[u], g.nb, 403)) {
            const uint32_t fin = ch.z + first[u];
            a.blk_off[bk[u]] = fin;
            if (fl[u] && (uint64_t)fin < a.out_cap) {
                uint64_t idx, tile;
                block_origin(g, bk[u], &idx, &tile);
                a.out_idx[fin] = (uint32_t)idx;
                a.out_delta[fin] = a.origin[bk[u]];
            }
        }
        const uint32_t kb = __ballot_sync(VSZ_FULL, keep[u] != 0u);
        if (l == 0) s_wtot[u * 8 + w] = (uint32_t)__popc(kb);
        keep[u] = keep[u] ? (uint32_t)__popc(kb & lt) + 1u : 0u;  // rank among the warp's kept, plus one
    }
    __syncthreads();
    uint32_t nkeep = 0, before[kPer];  // kept blocks in all, before each round of this warp
#pragma unroll
    for (int q = 0; q < kTab / 32; ++q) {
        const uint32_t v = s_wtot[q];
#pragma unroll
        for (int u = 0; u < kPer; ++u)
            if (q == u * 8) before[u] = nkeep;
        nkeep += v;
    }
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
        uint32_t c = before[u];
        for (int q = u * 8; q < u * 8 + w; ++q) c += s_wtot[q];
        if (keep[u]) {
            c += keep[u] - 1u;
            s_first[c] = first[u];
            s_src[c] = (bk[u] * S + (s0[u] ? 0u : 1u) - fl[u]) | (fl[u] ? kOrig : 0ull);
        }
    }
    if (threadIdx.x < 32) s_first[nkeep + threadIdx.x] = 0xffffffffu;  // sentinels past the last block
    __syncthreads();

    // the moves: a contiguous run of the share per warp, whole windows
    const uint32_t per = ((q1 - q0 + 8 * 32 - 1) / (8 * 32)) * 32;
    const uint32_t wq0 = q0 + (uint32_t)w * per, wq1 = min(q1, wq0 + per);
    if (wq0 < wq1 && nkeep > 0) {
        uint32_t k0 = 0;  // the kept block holding place wq0: the last first place <= wq0
#pragma unroll
        for (uint32_t step = kTab / 2; step > 0; step >>= 1)
            if (k0 + step < nkeep && s_first[k0 + step] <= wq0) k0 += step;
        const uint32_t upto = (l == 31) ? VSZ_FULL : ((2u << l) - 1u);  // marks at 1..l
        for (uint32_t qs = wq0; qs < wq1; qs += 32u * kMoveWindows) {
            uint2 e[kMoveWindows];
            uint32_t d[kMoveWindows];
            bool mv[kMoveWindows];
#pragma unroll
            for (int m = 0; m < kMoveWindows; ++m) {
                const uint32_t ws = qs + 32u * m;                 // this window's first place
                const uint32_t dj = s_first[k0 + 1 + l] - ws;     // where block k0+1+l starts, from ws
                const uint32_t marks = __reduce_or_sync(VSZ_FULL, dj < 32u ? (1u << dj) : 0u);
                const uint32_t kq = k0 + (uint32_t)__popc(marks & upto);
                k0 += (uint32_t)__popc(__ballot_sync(VSZ_FULL, dj <= 32u));  // the next window's first block
                const uint32_t q = ws + (uint32_t)l;
                const uint32_t rq = q - s_first[kq];
                const uint64_t sw = s_src[kq];
                const uint64_t src = (sw & ~kOrig) + rq;
                d[m] = ch.z + q;
                mv[m] = q < wq1 && !((sw & kOrig) && rq == 0) && (uint64_t)d[m] < a.out_cap &&
                        VSZ_IN(src, g.nb * S, 401);
                if (mv[m]) e[m] = a.slots[src];
            }
#pragma unroll
            for (int m = 0; m < kMoveWindows; ++m) {
                if (mv[m] && VSZ_IN((uint64_t)d[m], a.out_cap, 402)) {
                    a.out_idx[d[m]] = e[m].x;
                    a.out_delta[d[m]] = (int32_t)e[m].y;
                }
            }
        }
    }

    if (split == 0 && ch.y) {  // fixups: tile by tile, contiguous in staging and in the list
        for (int j = w; j < nt; j += 8) {
            const uint4 rr = s_rec[j];
            const uint32_t tf = ch.w + s_tfix[j];
            if (rr.w && (uint64_t)rr.z + rr.w <= a.fix_cap && (uint64_t)tf + rr.w <= a.fix_cap) {
                for (uint32_t k = l; k < rr.w; k += 32) {
                    const uint2 fe = a.stage_fix[rr.z + k];
                    a.fix_idx[tf + k] = fe.x;
                    a.fix_bits[tf + k] = fe.y;
                }
            }
        }
    }
}

// The origin pass of a global padding mode, for block `blk`: the residual
// of the block origin q - P, its code, and whether it is an outlier (then
// counted in its tile and chunk before the compaction).
// q0: the block origin's q, a.origin[blk] (loaded ahead by the caller, so
// that a thread can have several blocks' loads in flight).
__device__ __forceinline__ void origin_fix_block(const CompressArgs& a, uint64_t blk, int32_t q0, int32_t P) {
    uint64_t idx, tile;
    block_origin(a.g, blk, &idx, &tile);
    const int32_t d = (int32_t)((uint32_t)q0 - (uint32_t)P);
    const uint32_t c = code_of(d, a.R);
    a.codes[idx] = (uint16_t)c;
    const bool out = c == 0u;
    a.oflag[blk] = out ? 1 : 0;
    if (out) {
        a.origin[blk] = d;
        atomicAdd(&a.tiles[tile].y, 1u);
        atomicAdd(&a.chunks[tile / kTilesPerChunk].x, 1u);
    }
}

// Edge granularity (Sec. IV-B-3): per block and axis k, the min / max /
// rounded mean of q over the block's face at local coordinate 0 along k,
// into a.pad[blk * nd + k] (k = 0 the slowest axis).  2D/3D: one warp per
// tile (a 128-column segment of a row of blocks, as the compression walk):
// lane l holds columns 4l..4l+3, b/4 lanes share a block; rows on a y or z
// face are read whole, other rows only at each block's column 0.  1D: the
// face of a block is its first element; a warp's unit is 32 blocks.
__device__ __forceinline__ void edge_stats_unit(const CompressArgs& a, uint64_t t, int lane) {
    const Geom& g = a.g;
    const float inv2eb = a.hdr->inv2eb;
    const int kind = a.pad_mode - VSZ_PAD_EDGE_MIN;  // 0 min, 1 max, 2 mean
    if (g.nd == 1) {
        const uint64_t b = t * 32 + (uint64_t)lane;
        if (b < g.nb) a.pad[b] = prequant(a.x[b * g.b], inv2eb);
        return;
    }
    // the compression walk gathered the faces itself (fp32 mode proved for
    // the whole field by the range pass)
    if (a.wsh->fp32_ok != 0u) return;
    const int nd = g.nd;
    const uint64_t B = g.b;
    const int G = (int)(B / 4);
    const int glane = lane & (G - 1);
    const uint64_t grp = (uint64_t)(lane / G);
    const uint64_t nx = g.nx, plane = g.ny * g.nx;
    const uint64_t sg = t % g.nseg, rb = t / g.nseg;
    const uint64_t by = rb % g.nby, bz = rb / g.nby;
    const uint64_t x0 = sg * kSegCols + (uint64_t)lane * 4;
    const uint64_t bx = (sg * kSegCols) / B + grp;
    const int valid = x0 < nx ? (int)umin64(4, nx - x0) : 0;
    const int ylen = (int)umin64(B, g.ny - by * B);
    const int zlen = nd == 3 ? (int)umin64(B, g.nz - bz * B) : 1;
    const uint64_t base = (nd == 3 ? bz * B * plane : 0) + by * B * nx + x0;
    // faces: 0 = x (axis nd-1), 1 = y (axis nd-2), 2 = z (axis 0 of 3D)
    long long sm[3] = {0, 0, 0};
    int mn[3] = {INT_MAX, INT_MAX, INT_MAX}, mx[3] = {INT_MIN, INT_MIN, INT_MIN};
    auto take = [&](int f, int32_t v) {
        sm[f] += v;
        mn[f] = min(mn[f], v);
        mx[f] = max(mx[f], v);
    };
    // Face rows (every row of the first plane, the first row of the other
    // planes) carry the y and z faces: the lane's 4 values, eight rows'
    // loads issued before any is used.  The other rows carry only the x face:
    // one value on the block's first lane, 32 rows' loads at a time.
    const bool vec4 = valid == 4 && (reinterpret_cast<uintptr_t>(a.x) & 15) == 0 && (nx & 3) == 0;
    auto row_ptr = [&](int lz, int ly) { return a.x + base + (uint64_t)lz * plane + (uint64_t)ly * nx; };
    if (valid > 0) {
        const int nface = nd == 3 ? ylen + zlen - 1 : 1;  // face row i: plane 0 row i, then plane i-ylen+1 row 0
        constexpr int RF = 8;
        for (int i0 = 0; i0 < nface; i0 += RF) {
            float v[RF][4];
#pragma unroll
            for (int r = 0; r < RF; ++r) {
                const int i = i0 + r;
                const int lz = i < ylen ? 0 : i - ylen + 1, ly = i < ylen ? i : 0;
                v[r][0] = v[r][1] = v[r][2] = v[r][3] = 0.0f;
                if (i < nface) {
                    const float* row = row_ptr(lz, ly);
                    if (vec4) {
                        const float4 f = __ldg(reinterpret_cast<const float4*>(row));
                        v[r][0] = f.x;
                        v[r][1] = f.y;
                        v[r][2] = f.z;
                        v[r][3] = f.w;
                    } else {
#pragma unroll
                        for (int k = 0; k < 4; ++k)
                            if (k < valid) v[r][k] = __ldg(row + k);
                    }
                }
            }
#pragma unroll
            for (int r = 0; r < RF; ++r) {
                const int i = i0 + r;
                if (i >= nface) continue;
                const int lz = i < ylen ? 0 : i - ylen + 1, ly = i < ylen ? i : 0;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    if (k >= valid) continue;
                    const int32_t q = prequant(v[r][k], inv2eb);
                    if (k == 0 && glane == 0) take(0, q);
                    if (ly == 0) take(1, q);
                    if (nd == 3 && lz == 0) take(2, q);
                }
            }
        }
        // the remaining rows: planes lz >= 1 (3D) or 0 (2D), rows ly >= 1
        if (glane == 0) {
            const int z1 = nd == 3 ? 1 : 0;
            const int nrest = (zlen - z1) * (ylen - 1);
            constexpr int RX = 32;
            for (int i0 = 0; i0 < nrest; i0 += RX) {
                float v[RX];
#pragma unroll
                for (int r = 0; r < RX; ++r) {
                    const int i = i0 + r;
                    const int lz = z1 + i / (ylen - 1), ly = 1 + i % (ylen - 1);
                    v[r] = i < nrest ? __ldg(row_ptr(lz, ly)) : 0.0f;
                }
#pragma unroll
                for (int r = 0; r < RX; ++r)
                    if (i0 + r < nrest) take(0, prequant(v[r], inv2eb));
            }
        }
    }
    for (int off = 1; off < G; off <<= 1) {  // the y and z faces span the block's lanes
#pragma unroll
        for (int f = 1; f < 3; ++f) {
            sm[f] += __shfl_xor_sync(VSZ_FULL, sm[f], off);
            mn[f] = min(mn[f], __shfl_xor_sync(VSZ_FULL, mn[f], off));
            mx[f] = max(mx[f], __shfl_xor_sync(VSZ_FULL, mx[f], off));
        }
    }
    if (glane == 0 && bx < g.nbx) {
        const uint64_t blk = (bz * g.nby + by) * g.nbx + bx;
        const long long xw = (long long)umin64(B, nx - bx * B);
        const long long cnt[3] = {(long long)ylen * zlen, xw * zlen, xw * ylen};
        for (int f = 0; f < nd; ++f) {
            const int32_t v = kind == 0 ? mn[f] : kind == 1 ? mx[f] : rounded_mean(sm[f], cnt[f]);
            a.pad[blk * (uint64_t)nd + (uint64_t)(nd - 1 - f)] = v;
        }
    }
}

// Units of the face-statistics pass: tiles (2D/3D) or groups of 32 blocks (1D).
__host__ __device__ inline uint64_t edge_units(const Geom& g) { return g.nd == 1 ? (g.nb + 31) / 32 : g.ntiles; }

}  // namespace vsz
