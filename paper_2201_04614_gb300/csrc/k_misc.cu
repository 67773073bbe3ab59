// k_misc.cu -- error-bound resolution, global statistics, outlier
// compaction, fixup scatter and code histogram.
#include <climits>

#include "common.cuh"
#include "memops.cuh"
#include "misc.cuh"

namespace vsz {

// ---------------------------------------------------------------------------
// Error-bound resolution (Sec. II-B), on the device so that relative mode
// needs no host round trip: eb_abs = eb, or eb * (max - min) over the finite
// values (eb itself when that range is zero or empty); 1/(2 eb_abs) and
// 2 eb_abs are formed in double and rounded once to float; the guard's bound
// is eb_abs rounded toward zero.
__device__ void resolve_eb(vsz_header* h, double eb, bool rel, bool has, float xmin, float xmax) {
    double eb_abs = eb;
    if (rel && has) {
        const double range = __dsub_rn((double)xmax, (double)xmin);
        if (range > 0.0) eb_abs = __dmul_rn(eb, range);
    }
    h->eb_abs = eb_abs;
    h->inv2eb = __double2float_rn(__ddiv_rn(1.0, __dmul_rn(2.0, eb_abs)));
    h->ebx2 = __double2float_rn(__dmul_rn(2.0, eb_abs));
    h->eb_f32 = __double2float_rz(eb_abs);
    h->has_range = has ? 1u : 0u;
    h->xmin = has ? xmin : 0.0f;
    h->xmax = has ? xmax : 0.0f;
}

__global__ void k_begin(WsHeader* wsh, uint4* chunks, uint64_t nchunks, vsz_header* hdr, double eb, int rel) {
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
        wsh->has_finite = 0;
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

// Block-wide reductions through shared memory (blockDim.x == 256).
template <typename T, typename Op>
__device__ __forceinline__ T block_reduce(T v, Op op, T* sm, T identity) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v = op(v, __shfl_xor_sync(VSZ_FULL, v, off));
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sm[w] = v;
    __syncthreads();
    if (w == 0) {
        v = (l < (int)(blockDim.x >> 5)) ? sm[l] : identity;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v = op(v, __shfl_xor_sync(VSZ_FULL, v, off));
    }
    return v;  // valid in warp 0
}

struct OpMin { template <class T> __device__ T operator()(T a, T b) const { return a < b ? a : b; } };
struct OpMax { template <class T> __device__ T operator()(T a, T b) const { return a > b ? a : b; } };
struct OpAdd { template <class T> __device__ T operator()(T a, T b) const { return a + b; } };

// Finite min/max of x; the last block resolves the relative error bound.
__global__ void __launch_bounds__(256) k_range(const float* __restrict__ x, uint64_t n, WsHeader* wsh,
                                               vsz_header* hdr, double eb, int vec) {
    __shared__ unsigned int smu[32];
    __shared__ bool last;
    unsigned int lo = 0xffffffffu, hi = 0u;
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t nth = (uint64_t)gridDim.x * blockDim.x;
    if (vec) {
        const uint64_t n4 = n / 4;
        for (uint64_t i = tid; i < n4; i += nth) {
            const float4 v = ld_stream_f4(x + 4 * i);
            const float a[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (isfinite(a[k])) { const unsigned u = float_to_ord(a[k]); lo = min(lo, u); hi = max(hi, u); }
        }
        for (uint64_t i = 4 * n4 + tid; i < n; i += nth)
            if (isfinite(x[i])) { const unsigned u = float_to_ord(x[i]); lo = min(lo, u); hi = max(hi, u); }
    } else {
        for (uint64_t i = tid; i < n; i += nth)
            if (isfinite(x[i])) { const unsigned u = float_to_ord(x[i]); lo = min(lo, u); hi = max(hi, u); }
    }
    lo = block_reduce(lo, OpMin(), smu, 0xffffffffu);
    hi = block_reduce(hi, OpMax(), smu, 0u);
    if (threadIdx.x == 0) {
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
        const unsigned l = atomicAdd(&wsh->xmin_ord, 0u);
        const unsigned h = atomicAdd(&wsh->xmax_ord, 0u);
        const bool has = l != 0xffffffffu;
        resolve_eb(hdr, eb, true, has, has ? ord_to_float(l) : 0.0f, has ? ord_to_float(h) : 0.0f);
    }
}

// Global min / max / sum of q (Sec. IV-B-1); the last block sets P.
__global__ void __launch_bounds__(256) k_qstats(const float* __restrict__ x, uint64_t n, WsHeader* wsh,
                                                vsz_header* hdr, int pad_mode, int vec) {
    __shared__ int smi[32];
    __shared__ long long sml[32];
    __shared__ bool last;
    const float inv2eb = hdr->inv2eb;
    int qlo = INT_MAX, qhi = INT_MIN;
    long long qs = 0;
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t nth = (uint64_t)gridDim.x * blockDim.x;
    if (vec) {
        const uint64_t n4 = n / 4;
        for (uint64_t i = tid; i < n4; i += nth) {
            const float4 v = ld_stream_f4(x + 4 * i);
            const float a[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int q = prequant(a[k], inv2eb);
                qlo = min(qlo, q); qhi = max(qhi, q); qs += q;
            }
        }
        for (uint64_t i = 4 * n4 + tid; i < n; i += nth) {
            const int q = prequant(x[i], inv2eb);
            qlo = min(qlo, q); qhi = max(qhi, q); qs += q;
        }
    } else {
        for (uint64_t i = tid; i < n; i += nth) {
            const int q = prequant(x[i], inv2eb);
            qlo = min(qlo, q); qhi = max(qhi, q); qs += q;
        }
    }
    qlo = block_reduce(qlo, OpMin(), smi, INT_MAX);
    qhi = block_reduce(qhi, OpMax(), smi, INT_MIN);
    qs = block_reduce(qs, OpAdd(), sml, 0ll);
    if (threadIdx.x == 0) {
        atomicMin(&wsh->qmin, qlo);
        atomicMax(&wsh->qmax, qhi);
        atomicAdd(&wsh->qsum, (unsigned long long)qs);
        __threadfence();
        last = atomicAdd(&wsh->done1, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        const int l = atomicAdd(&wsh->qmin, 0);
        const int h = atomicAdd(&wsh->qmax, 0);
        const long long S = (long long)atomicAdd(&wsh->qsum, 0ull);
        int32_t P = 0;
        if (n > 0) {
            P = pad_mode == VSZ_PAD_GLOBAL_MIN ? l
              : pad_mode == VSZ_PAD_GLOBAL_MAX ? h
              : rounded_mean(S, (long long)n);
        }
        hdr->pad_global = P;
    }
}

// ---------------------------------------------------------------------------
// Compaction, part 1: exclusive scan of the per-chunk totals (one CTA).
__global__ void __launch_bounds__(1024) k_compact_scan(uint4* chunks, uint64_t nchunks, vsz_header* hdr,
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
__global__ void __launch_bounds__(256) k_compact(const uint4* __restrict__ tiles, const uint4* __restrict__ chunks,
                                                 uint64_t ntiles, uint64_t nseg, uint64_t nbx, uint32_t bpt,
                                                 uint32_t* blk_off, const uint2* __restrict__ stage_out,
                                                 const uint2* __restrict__ stage_fix, uint32_t* out_idx,
                                                 int32_t* out_delta, uint64_t out_cap, uint32_t* fix_idx,
                                                 uint32_t* fix_bits, uint64_t fix_cap) {
    __shared__ uint4 rec[kTilesPerChunk];
    __shared__ uint32_t toff_o[kTilesPerChunk], toff_f[kTilesPerChunk];
    const uint64_t t0 = (uint64_t)blockIdx.x * kTilesPerChunk;
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (w == 0) {  // the chunk's tile offsets: chunk offset + exclusive scan of the tile totals
        uint32_t bo = chunks[blockIdx.x].z, bf = chunks[blockIdx.x].w;
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

// Fixups restore their values verbatim after the inverse.
__global__ void __launch_bounds__(256) k_fixups(const vsz_header* hdr, const uint32_t* __restrict__ fix_idx,
                                                const uint32_t* __restrict__ fix_bits, uint64_t fix_cap,
                                                float* xhat, uint64_t n) {
    const uint64_t cnt = umin64(hdr->n_fix, fix_cap);
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t j = fix_idx[i];
        if (j < n) xhat[j] = __uint_as_float(fix_bits[i]);
    }
}

// Code histogram: per-CTA shared-memory bins when they fit, else global.
__global__ void __launch_bounds__(256) k_histogram(const uint16_t* __restrict__ codes, uint64_t n,
                                                   uint32_t* hist, uint32_t nbins, int use_smem) {
    extern __shared__ uint32_t sh[];
    if (use_smem) {
        for (uint32_t i = threadIdx.x; i < nbins; i += blockDim.x) sh[i] = 0;
        __syncthreads();
    }
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t c = codes[i];
        if (c < nbins) {
            if (use_smem) atomicAdd(&sh[c], 1u);
            else atomicAdd(&hist[c], 1u);
        }
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
    k_begin<<<grid, 256, 0, s>>>(wsh, chunks, nchunks, hdr, eb, rel ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_range(const float* x, uint64_t n, WsHeader* wsh, vsz_header* hdr, double eb, bool vec,
                         cudaStream_t s) {
    const int grid = grid_for((const void*)k_range, 256, 0, 256 * 16, n);
    k_range<<<grid, 256, 0, s>>>(x, n, wsh, hdr, eb, vec ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_qstats(const float* x, uint64_t n, WsHeader* wsh, vsz_header* hdr, int pad_mode, bool vec,
                          cudaStream_t s) {
    const int grid = grid_for((const void*)k_qstats, 256, 0, 256 * 16, n);
    k_qstats<<<grid, 256, 0, s>>>(x, n, wsh, hdr, pad_mode, vec ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_compact_scan(const Geom& g, uint4* chunks, vsz_header* hdr, uint32_t* blk_off,
                                uint64_t out_cap, uint64_t fix_cap, cudaStream_t s) {
    k_compact_scan<<<1, 1024, 0, s>>>(chunks, g.nchunks, hdr, blk_off, g.nb, out_cap, fix_cap);
    return cudaGetLastError();
}

cudaError_t launch_compact_move(const Geom& g, const uint4* tiles, const uint4* chunks, uint32_t* blk_off,
                                const uint2* stage_out, const uint2* stage_fix, uint32_t* out_idx,
                                int32_t* out_delta, uint64_t out_cap, uint32_t* fix_idx, uint32_t* fix_bits,
                                uint64_t fix_cap, cudaStream_t s) {
    if (g.nchunks == 0) return cudaSuccess;
    k_compact<<<(unsigned)g.nchunks, 256, 0, s>>>(tiles, chunks, g.ntiles, g.nseg, g.nbx, g.bpt, blk_off,
                                                  stage_out, stage_fix, out_idx, out_delta, out_cap, fix_idx,
                                                  fix_bits, fix_cap);
    return cudaGetLastError();
}

cudaError_t launch_fixups(const vsz_header* hdr, const uint32_t* fix_idx, const uint32_t* fix_bits,
                          uint64_t fix_cap, float* xhat, uint64_t n, cudaStream_t s) {
    const int grid = (int)umin64((uint64_t)num_sms(), (fix_cap + 255) / 256);
    if (grid == 0) return cudaSuccess;
    k_fixups<<<grid, 256, 0, s>>>(hdr, fix_idx, fix_bits, fix_cap, xhat, n);
    return cudaGetLastError();
}

cudaError_t launch_histogram(const uint16_t* codes, uint64_t n, uint32_t* hist, uint32_t nbins, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(hist, 0, (size_t)nbins * 4, s);
    if (e != cudaSuccess || n == 0) return e;
    const size_t smem = (size_t)nbins * 4;
    const int use_smem = smem <= 96 * 1024;
    if (use_smem && smem > 48 * 1024) {
        e = cudaFuncSetAttribute((const void*)k_histogram, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    const int grid = grid_for((const void*)k_histogram, 256, use_smem ? smem : 0, 256 * 64, n);
    k_histogram<<<grid, 256, use_smem ? smem : 0, s>>>(codes, n, hist, nbins, use_smem);
    return cudaGetLastError();
}

}  // namespace vsz
