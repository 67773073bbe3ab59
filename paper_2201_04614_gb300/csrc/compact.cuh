// compact.cuh -- outlier compaction (the second step of compression).
//
// Part 1 scans the per-chunk totals of one field (one CTA); part 2, one CTA
// per chunk of 32 tiles, turns the in-tile block offsets left by the
// compression kernel into global ones and moves each tile's staged outliers
// and fixups, which are contiguous both in staging and in the final lists, to
// their canonical place.  Both bodies serve the single-field kernels
// (k_misc.cu) and the batch kernels (k_batch.cu).
#pragma once

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
// staged entries to their canonical place.
__device__ __forceinline__ void compact_chunk_body(uint64_t chunk, const uint4* __restrict__ tiles,
                                                   const uint4* __restrict__ chunks, uint64_t ntiles, uint64_t nseg,
                                                   uint64_t nbx, uint32_t bpt, uint32_t* blk_off,
                                                   const uint2* __restrict__ stage_out,
                                                   const uint2* __restrict__ stage_fix, uint32_t* out_idx,
                                                   int32_t* out_delta, uint64_t out_cap, uint32_t* fix_idx,
                                                   uint32_t* fix_bits, uint64_t fix_cap) {
    __shared__ uint4 rec[kTilesPerChunk];
    __shared__ uint32_t toff_o[kTilesPerChunk], toff_f[kTilesPerChunk];
    const uint64_t t0 = chunk * kTilesPerChunk;
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (w == 0) {  // the chunk's tile offsets: chunk offset + exclusive scan of the tile totals
        uint32_t bo = chunks[chunk].z, bf = chunks[chunk].w;
        for (int i0 = 0; i0 < kTilesPerChunk; i0 += 32) {
            const uint64_t t = t0 + i0 + l;
            const uint4 r = t < ntiles ? tiles[t] : make_uint4(0, 0, 0, 0);
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
        const uint64_t nblk = umin64(bpt, nbx - s * bpt);
        for (uint64_t k = l; k < nblk; k += 32) blk_off[fb + k] += to;
        if (rr.y && (uint64_t)rr.x + rr.y <= out_cap && (uint64_t)to + rr.y <= out_cap) {
            for (uint32_t k = l; k < rr.y; k += 32) {
                const uint2 e = stage_out[rr.x + k];
                out_idx[to + k] = e.x;
                out_delta[to + k] = (int32_t)e.y;
            }
        }
        if (rr.w && (uint64_t)rr.z + rr.w <= fix_cap && (uint64_t)tf + rr.w <= fix_cap) {
            for (uint32_t k = l; k < rr.w; k += 32) {
                const uint2 e = stage_fix[rr.z + k];
                fix_idx[tf + k] = e.x;
                fix_bits[tf + k] = e.y;
            }
        }
    }
}

}  // namespace vsz
