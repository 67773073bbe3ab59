// k_misc.cu -- error-bound resolution, global statistics, outlier
// compaction, fixup scatter and code histogram.
#include <climits>

#include "common.cuh"
#include "memops.cuh"
#include "compact.cuh"
#include "stats.cuh"
#include "misc.cuh"

namespace vsz {

__global__ void k_begin(WsHeader* wsh, uint4* chunks, uint64_t nchunks, vsz_header* hdr, double eb, int rel) {
    pdl_prologue();
    const uint64_t i0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (uint64_t i = i0; i < nchunks; i += (uint64_t)gridDim.x * blockDim.x) chunks[i] = make_uint4(0, 0, 0, 0);
    if (i0 == 0) {
        wsh->stage_out = 0;
        wsh->stage_fix = 0;
        wsh->qsum = 0;
        wsh->xmin_ord = 0xffffffffu;
        wsh->xmax_ord = 0u;
        wsh->qmin = INT_MAX;
        wsh->qmax = INT_MIN;
        wsh->done0 = 0;
        wsh->done1 = 0;
        wsh->nonfinite = 0;
        wsh->fp32_ok = 0;
        wsh->ticket = 0;
        hdr->pad_global = 0;
        hdr->status = 0;
        hdr->recon_status = 0;
        hdr->reserved = 0;
        hdr->n_out = 0;
        hdr->n_fix = 0;
        if (!rel) resolve_eb(hdr, eb, false, false, 0.0f, 0.0f);
    }
}

// Finite min/max of x; the last block resolves the relative error bound.
__global__ void __launch_bounds__(256) k_range(const float* __restrict__ x, uint64_t n, WsHeader* wsh,
                                               vsz_header* hdr, double eb, int vec) {
    pdl_prologue();
    __shared__ unsigned int smu[32];
    __shared__ bool last;
    unsigned int lo = 0xffffffffu, hi = 0u;
    bool nf = false;
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t nth = (uint64_t)gridDim.x * blockDim.x;
    auto take = [&](float v) {
        if (isfinite(v)) {
            const unsigned u = float_to_ord(v);
            lo = min(lo, u);
            hi = max(hi, u);
        } else {
            nf = true;
        }
    };
    if (vec) {
        // four 16-byte loads in flight per thread, each coalesced across the grid
        const uint64_t n4 = n / 4;
        uint64_t i = tid;
        for (; i + 3 * nth < n4; i += 4 * nth) {
            float4 v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) v[u] = ld_stream_f4(x + 4 * (i + u * nth));
#pragma unroll
            for (int u = 0; u < 4; ++u) { take(v[u].x); take(v[u].y); take(v[u].z); take(v[u].w); }
        }
        for (; i < n4; i += nth) {
            const float4 v = ld_stream_f4(x + 4 * i);
            take(v.x); take(v.y); take(v.z); take(v.w);
        }
        for (uint64_t k = 4 * n4 + tid; k < n; k += nth) take(x[k]);
    } else {
        for (uint64_t i = tid; i < n; i += nth) take(x[i]);
    }
    nf = __syncthreads_or(nf) != 0;
    lo = block_reduce(lo, OpMin(), smu, 0xffffffffu);
    hi = block_reduce(hi, OpMax(), smu, 0u);
    if (threadIdx.x == 0) {
        if (nf) atomicOr(&wsh->nonfinite, 1u);
        if (lo != 0xffffffffu) {
            atomicMin(&wsh->xmin_ord, lo);
            atomicMax(&wsh->xmax_ord, hi);
        }
        __threadfence();
        last = atomicAdd(&wsh->done0, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        finish_range(wsh, hdr, eb);
    }
}

// Compaction of one field (bodies in compact.cuh).
__global__ void __launch_bounds__(1024) k_compact_scan(uint4* chunks, uint64_t nchunks, vsz_header* hdr,
                                                       uint32_t* blk_off, uint64_t nb, uint64_t out_cap,
                                                       uint64_t fix_cap) {
    pdl_prologue();
    compact_scan_body(chunks, nchunks, hdr, blk_off, nb, out_cap, fix_cap);
}

__global__ void __launch_bounds__(256) k_compact(const CompressArgs a) {
    pdl_prologue();
    if (a.slots) compact_chunk_body_slots(blockIdx.x, (int)blockIdx.y, a);
    else compact_chunk_body(blockIdx.x, a);
}

// Origin pass of a global padding mode (one field): every block origin's
// residual q - P and its code, P from the field's header.
// Four blocks per thread per round, their origin loads issued first.
constexpr int kOriginUnroll = 4;

__global__ void __launch_bounds__(256) k_origin_fix(const CompressArgs a) {
    pdl_prologue();
    const int32_t P = global_pad_value(a);
    if (blockIdx.x == 0 && threadIdx.x == 0) const_cast<vsz_header*>(a.hdr)->pad_global = P;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t b0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; b0 < a.g.nb; b0 += kOriginUnroll * stride) {
        int32_t q0[kOriginUnroll];
#pragma unroll
        for (int u = 0; u < kOriginUnroll; ++u) {
            const uint64_t b = b0 + u * stride;
            q0[u] = b < a.g.nb ? a.origin[b] : 0;
        }
#pragma unroll
        for (int u = 0; u < kOriginUnroll; ++u) {
            const uint64_t b = b0 + u * stride;
            if (b < a.g.nb) origin_fix_block(a, b, q0[u], P);
        }
    }
}

__global__ void __launch_bounds__(256) k_edge_stats(const CompressArgs a) {
    pdl_prologue();
    const uint64_t nwarps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    const uint64_t units = edge_units(a.g);
    for (uint64_t t = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); t < units; t += nwarps)
        edge_stats_unit(a, t, threadIdx.x & 31);
}

// Origin pass of an edge padding mode: every block origin's residual from
// its block's per-axis scalars.
__global__ void __launch_bounds__(256) k_origin_fix_edge(const CompressArgs a) {
    pdl_prologue();
    const int nd = a.g.nd;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t b0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; b0 < a.g.nb; b0 += kOriginUnroll * stride) {
        int32_t q0[kOriginUnroll], sc[kOriginUnroll][3];
#pragma unroll
        for (int u = 0; u < kOriginUnroll; ++u) {
            const uint64_t b = b0 + u * stride;
            const bool in = b < a.g.nb;
            q0[u] = in ? a.origin[b] : 0;
#pragma unroll
            for (int k = 0; k < 3; ++k) sc[u][k] = (in && k < nd) ? a.pad[b * (uint64_t)nd + k] : 0;
        }
#pragma unroll
        for (int u = 0; u < kOriginUnroll; ++u) {
            const uint64_t b = b0 + u * stride;
            if (b < a.g.nb) origin_fix_block(a, b, q0[u], edge_origin_pred_r(sc[u][0], sc[u][1], sc[u][2], nd));
        }
    }
}

// Fixups restore their values verbatim after the inverse.
__global__ void __launch_bounds__(256) k_fixups(const vsz_header* hdr, const uint32_t* __restrict__ fix_idx,
                                                const uint32_t* __restrict__ fix_bits, uint64_t fix_cap,
                                                float* xhat, uint64_t n) {
    pdl_prologue();
    const uint64_t cnt = umin64(hdr->n_fix, fix_cap);
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t j = fix_idx[i];
        if (j < n) xhat[j] = __uint_as_float(fix_bits[i]);
    }
}

// Code histogram.  Codes cluster around R (small residuals): the kHistWin
// bins from R - kHistWin/2 count in lane-private 16-bit counters in shared
// memory, two bins to a 32-bit word (column `lane` of the warp's table, so
// a lane's increments need no atomic and never share a bank with another
// lane's); every other code adds with an atomic to the CTA's bins (shared
// memory when they fit, else global).  At the end each warp sums its
// table's columns into the bins.  The launch gives every thread at most
// kHistMaxPerThread codes, so no 16-bit counter overflows.
constexpr int kHistWin = 64;
constexpr int kHistThreads = 256;
constexpr uint64_t kHistMaxPerThread = 60000;
__global__ void __launch_bounds__(kHistThreads) k_histogram(const uint16_t* __restrict__ codes, uint64_t n,
                                                            uint32_t* hist, uint32_t nbins, int use_smem) {
    extern __shared__ uint32_t sm[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t* tab = sm + (size_t)warp * (kHistWin / 2) * 32;   // [kHistWin/2][32] of this warp
    uint32_t* sh = sm + (size_t)(kHistThreads / 32) * (kHistWin / 2) * 32;  // [nbins] when use_smem
#pragma unroll
    for (int k = 0; k < kHistWin / 2; ++k) tab[k * 32 + lane] = 0;
    if (use_smem)
        for (uint32_t i = threadIdx.x; i < nbins; i += blockDim.x) sh[i] = 0;
    __syncthreads();
    const uint32_t R = nbins / 2, base = R >= kHistWin / 2 ? R - kHistWin / 2 : 0;
    auto put = [&](uint32_t c, uint32_t k) { if (use_smem) atomicAdd(&sh[c], k); else atomicAdd(&hist[c], k); };
    auto add = [&](uint32_t c) {
        const uint32_t k = c - base;
        if (k < (uint32_t)kHistWin && c < nbins) tab[(k >> 1) * 32 + lane] += 1u << ((k & 1u) * 16);
        else if (c < nbins) put(c, 1u);
    };
    auto add8 = [&](const uint4 v) {
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            add(w[k] & 0xffffu);
            add(w[k] >> 16);
        }
    };
    const uint64_t nth = (uint64_t)gridDim.x * blockDim.x, tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool vec = (reinterpret_cast<uintptr_t>(codes) & 15) == 0;
    const uint64_t n8 = vec ? n / 8 : 0;
    uint64_t j = tid;
    for (; j + 3 * nth < n8; j += 4 * nth) {  // four 16-byte loads in flight
        uint4 v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = *reinterpret_cast<const uint4*>(codes + 8 * (j + u * nth));
#pragma unroll
        for (int u = 0; u < 4; ++u) add8(v[u]);
    }
    for (; j < n8; j += nth) add8(*reinterpret_cast<const uint4*>(codes + 8 * j));
    for (uint64_t i = 8 * n8 + tid; i < n; i += nth) add(codes[i]);
    __syncwarp();
    // bin base + k (k = lane, lane + 32): the sum of its half-words over the
    // warp's 32 columns, read in a rotated order so that the lanes hit 32 banks
#pragma unroll
    for (int h = 0; h < kHistWin / 32; ++h) {
        const uint32_t k = (uint32_t)(h * 32 + lane);
        uint32_t sum = 0;
#pragma unroll 8
        for (int c = 0; c < 32; ++c) sum += (tab[(k >> 1) * 32 + ((c + lane) & 31)] >> ((k & 1u) * 16)) & 0xffffu;
        if (sum && base + k < nbins) put(base + k, sum);
    }
    if (use_smem) {
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < nbins; i += blockDim.x)
            if (sh[i]) atomicAdd(&hist[i], sh[i]);
    }
}

// ---------------------------------------------------------------------------
// Launch helpers used by api.cu.

cudaError_t launch_begin(WsHeader* wsh, uint4* chunks, uint64_t nchunks, vsz_header* hdr, double eb, bool rel,
                         cudaStream_t s) {
    const int grid = (int)umin64(64, (nchunks + 255) / 256 + 1);
    return launch_pdl(k_begin, grid, 256, 0, s, wsh, chunks, nchunks, hdr, eb, rel ? 1 : 0);
}

cudaError_t launch_range(const float* x, uint64_t n, WsHeader* wsh, vsz_header* hdr, double eb, bool vec,
                         cudaStream_t s) {
    const int grid = grid_for((const void*)k_range, 256, 0, 256 * 16, n);
    return launch_pdl(k_range, grid, 256, 0, s, x, n, wsh, hdr, eb, vec ? 1 : 0);
}

cudaError_t launch_compact_scan(const Geom& g, uint4* chunks, vsz_header* hdr, uint32_t* blk_off,
                                uint64_t out_cap, uint64_t fix_cap, cudaStream_t s) {
    return launch_pdl(k_compact_scan, 1, 1024, 0, s, chunks, g.nchunks, hdr, blk_off, g.nb, out_cap, fix_cap);
}

cudaError_t launch_compact_move(const CompressArgs& a, cudaStream_t s) {
    if (a.g.nchunks == 0) return cudaSuccess;
    // block slots: kSplit CTAs per chunk (blockIdx.y), those past the
    // chunk's share return at once
    return launch_pdl(k_compact, dim3((unsigned)a.g.nchunks, a.slots ? kSplit : 1), 256, 0, s, a);
}

cudaError_t launch_origin_fix(const CompressArgs& a, cudaStream_t s) {
    if (is_edge_pad(a.pad_mode)) {
        if (a.g.nb == 0) return cudaSuccess;
        const uint64_t items = (edge_units(a.g) + 7) / 8;
        const int gs = grid_for((const void*)k_edge_stats, 256, 0, 1, items);
        cudaError_t e = launch_pdl(k_edge_stats, gs, 256, 0, s, a);
        if (e != cudaSuccess) return e;
        const int go = grid_for((const void*)k_origin_fix_edge, 256, 0, 256 * kOriginUnroll, a.g.nb);
        return launch_pdl(k_origin_fix_edge, go, 256, 0, s, a);
    }
    const int grid = grid_for((const void*)k_origin_fix, 256, 0, 256 * kOriginUnroll, a.g.nb ? a.g.nb : 1);
    return launch_pdl(k_origin_fix, grid, 256, 0, s, a);
}

cudaError_t launch_fixups(const vsz_header* hdr, const uint32_t* fix_idx, const uint32_t* fix_bits,
                          uint64_t fix_cap, float* xhat, uint64_t n, cudaStream_t s) {
    const int grid = (int)umin64((uint64_t)num_sms(), (fix_cap + 255) / 256);
    if (grid == 0) return cudaSuccess;
    return launch_pdl(k_fixups, grid, 256, 0, s, hdr, fix_idx, fix_bits, fix_cap, xhat, n);
}

cudaError_t launch_histogram(const uint16_t* codes, uint64_t n, uint32_t* hist, uint32_t nbins, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(hist, 0, (size_t)nbins * 4, s);
    if (e != cudaSuccess || n == 0) return e;
    const size_t tab = (size_t)(kHistThreads / 32) * (kHistWin / 2) * 32 * 4;  // the warps' window tables
    const int use_smem = (size_t)nbins * 4 <= 96 * 1024;
    const size_t smem = tab + (use_smem ? (size_t)nbins * 4 : 0);
    if ((e = raise_smem_attr((const void*)k_histogram, smem)) != cudaSuccess) return e;
    const int occ = occupancy((const void*)k_histogram, kHistThreads, smem);
    const uint64_t want = (n + (uint64_t)kHistThreads * 128 - 1) / ((uint64_t)kHistThreads * 128);
    uint64_t grid = umin64(want, (uint64_t)num_sms() * (uint64_t)(occ > 0 ? occ : 1));
    const uint64_t least = (n + kHistThreads * kHistMaxPerThread - 1) / (kHistThreads * kHistMaxPerThread);
    if (grid < least) grid = least;  // at most kHistMaxPerThread codes per thread (16-bit counters)
    if (grid > 0x7fffffffull) return cudaErrorInvalidValue;
    k_histogram<<<(unsigned)grid, kHistThreads, smem, s>>>(codes, n, hist, nbins, use_smem);
    return cudaGetLastError();
}

}  // namespace vsz
