// recon_nd.cuh -- inverse dual-quant for 2D and 3D fields (Sec. III-A).
//
// Same tiles and lane layout as the compression walk.  Per row: residuals
// from the codes (code - R), outliers patched from the block's slice of the
// outlier list, P added at the block origin, then the inverse of each
// first-order difference:
//   Sx: inclusive scan inside the lane, then a segmented warp scan across
//       the b/4 lanes of the block (shuffles);
//   Sy: running sum over the block's rows, carried in registers;
//   Sz: running sum over planes at the same row (registers for b <= 8,
//       lane-private shared memory above).
// The walk visits a block's elements in the canonical order (planes, rows,
// then x), so the k-th code 0 met in a block is the block's k-th outlier:
// no search over the outlier list is needed.
#pragma once

#include "compress_nd.cuh"

namespace vsz {

template <int ND, int B, bool QOUT>
__global__ void __launch_bounds__(NdCfg<ND, B>::THREADS)
k_recon_nd(const ReconArgs a) {
    using C = NdCfg<ND, B>;
    constexpr int G = C::G;
    constexpr int U = C::U;
    extern __shared__ int4 zsm[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const Geom& g = a.g;
    const float ebx2 = a.hdr->ebx2;
    const int32_t Pg = a.hdr->pad_global;
    const int32_t R = a.R;
    const bool bp = is_block_pad(a.pad_mode);
    int4* zs = C::ZSMEM ? (zsm + (size_t)wib * B * 32) : nullptr;
    const uint64_t plane = g.ny * g.nx;
    const int glane = lane & (G - 1);
    const bool first = glane == 0;
    const int src = lane & ~(G - 1);

    for (uint64_t t = (uint64_t)blockIdx.x * C::WARPS + wib; t < g.ntiles;
         t += (uint64_t)gridDim.x * C::WARPS) {
        const uint64_t s = t % g.nseg;
        const uint64_t rb = t / g.nseg;
        const uint64_t by = rb % g.nby;
        const uint64_t bz = rb / g.nby;
        const uint64_t x0 = s * kSegCols + (uint64_t)lane * 4;
        const uint64_t bx = (s * kSegCols) / B + (uint64_t)(lane / G);
        const bool bexists = bx < g.nbx;
        const int valid = x0 < g.nx ? (int)umin64(4, g.nx - x0) : 0;
        const int ylen = (int)umin64(B, g.ny - by * B);
        const int zlen = ND == 3 ? (int)umin64(B, g.nz - bz * B) : 1;
        const uint64_t blk = (bz * g.nby + by) * g.nbx + bx;
        const bool vec = a.vec && valid == 4;
        const uint64_t tile_base = (ND == 3 ? bz * B * plane : 0) + by * B * g.nx + x0;

        uint32_t lo = 0, hi = 0;
        int32_t P = Pg;
        if (first && bexists) {
            lo = a.blk_off[blk];
            hi = a.blk_off[blk + 1];
            if (bp) P = a.pad[blk];
        }
        lo = __shfl_sync(VSZ_FULL, lo, src);
        hi = __shfl_sync(VSZ_FULL, hi, src);
        P = __shfl_sync(VSZ_FULL, P, src);
        const bool anyout = __any_sync(VSZ_FULL, hi > lo);
        uint32_t rank = lo;

        int32_t ys[4] = {0, 0, 0, 0};
        int32_t zr[(ND == 3 && !C::ZSMEM) ? B : 1][4];

        for (int lz = 0; lz < zlen; ++lz) {
            const uint64_t zoff = tile_base + (uint64_t)lz * plane;
#pragma unroll((ND == 3 && !C::ZSMEM) ? B : 1)
            for (int ly0 = 0; ly0 < ((ND == 3 && !C::ZSMEM) ? B : ylen); ly0 += U) {
                uint32_t cr[U][4];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int ly = ly0 + u;
                    if (ly < ylen) {
                        load4c(a.codes + zoff + (uint64_t)ly * g.nx, valid, vec, cr[u]);
                    } else {
#pragma unroll
                        for (int k = 0; k < 4; ++k) cr[u][k] = 0u;
                    }
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int ly = ly0 + u;
                    if (ly >= ylen) break;
                    const uint64_t roff = zoff + (uint64_t)ly * g.nx;
                    int32_t d[4];
                    uint32_t zm = 0;
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        d[k] = (k < valid) ? (int32_t)cr[u][k] - R : 0;
                        if (k < valid && cr[u][k] == 0u) zm |= 1u << k;
                    }
                    if (anyout && __any_sync(VSZ_FULL, zm != 0)) {
                        const uint32_t cz = __popc(zm);
                        uint32_t iz = cz;
#pragma unroll
                        for (int off = 1; off < G; off <<= 1) {
                            const uint32_t y = __shfl_up_sync(VSZ_FULL, iz, off);
                            if (glane >= off) iz += y;
                        }
                        const uint32_t gtot = __shfl_sync(VSZ_FULL, iz, src + G - 1);
                        uint32_t r = rank + (iz - cz);
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            if (zm & (1u << k)) {
                                if (r < hi && r < a.out_cap && a.out_idx[r] == (uint32_t)(roff + k)) {
                                    d[k] = a.out_delta[r];
                                } else {
                                    atomicMax(&a.hdr->recon_status, (unsigned)VSZ_ERR_CORRUPT);
                                    d[k] = 0;
                                }
                                ++r;
                            }
                        }
                        rank += gtot;
                    }
                    if (first && ly == 0 && lz == 0) d[0] = wadd(d[0], P);
                    // Sx
                    d[1] = wadd(d[1], d[0]);
                    d[2] = wadd(d[2], d[1]);
                    d[3] = wadd(d[3], d[2]);
                    {
                        const uint32_t tot = (uint32_t)d[3];
                        uint32_t inc = tot;
#pragma unroll
                        for (int off = 1; off < G; off <<= 1) {
                            const uint32_t y = __shfl_up_sync(VSZ_FULL, inc, off);
                            if (glane >= off) inc += y;
                        }
                        const int32_t ex = (int32_t)(inc - tot);
#pragma unroll
                        for (int k = 0; k < 4; ++k) d[k] = wadd(d[k], ex);
                    }
                    // Sy
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        if (ly > 0) d[k] = wadd(d[k], ys[k]);
                        ys[k] = d[k];
                    }
                    // Sz
                    if (ND == 3) {
                        if (C::ZSMEM) {
                            int4& stz = zs[ly * 32 + lane];
                            if (lz > 0) {
                                const int4 pv = stz;
                                d[0] = wadd(d[0], pv.x); d[1] = wadd(d[1], pv.y);
                                d[2] = wadd(d[2], pv.z); d[3] = wadd(d[3], pv.w);
                            }
                            stz = make_int4(d[0], d[1], d[2], d[3]);
                        } else {
                            const int yi = (ND == 3 && !C::ZSMEM) ? ly : 0;
#pragma unroll
                            for (int k = 0; k < 4; ++k) {
                                if (lz > 0) d[k] = wadd(d[k], zr[yi][k]);
                                zr[yi][k] = d[k];
                            }
                        }
                    }
                    if (QOUT) {
                        int32_t* o = reinterpret_cast<int32_t*>(a.out) + roff;
                        if (vec) {
                            *reinterpret_cast<int4*>(o) = make_int4(d[0], d[1], d[2], d[3]);
                        } else {
#pragma unroll
                            for (int k = 0; k < 4; ++k)
                                if (k < valid) o[k] = d[k];
                        }
                    } else {
                        float v[4];
#pragma unroll
                        for (int k = 0; k < 4; ++k) v[k] = __fmul_rn(q2f(d[k]), ebx2);
                        float* o = reinterpret_cast<float*>(a.out) + roff;
                        if (vec) {
                            *reinterpret_cast<float4*>(o) = make_float4(v[0], v[1], v[2], v[3]);
                        } else {
#pragma unroll
                            for (int k = 0; k < 4; ++k)
                                if (k < valid) o[k] = v[k];
                        }
                    }
                }
            }
        }
    }
}

// Host-side launch helpers for one rank, instantiated by k_rank2.cu / k_rank3.cu.
template <int ND, int B>
cudaError_t launch_nd_compress(const CompressArgs& a, cudaStream_t s) {
    using C = NdCfg<ND, B>;
    const bool bp = is_block_pad(a.pad_mode);
    const void* k = bp ? (const void*)k_lorenzo_nd<ND, B, true> : (const void*)k_lorenzo_nd<ND, B, false>;
    if (C::SMEM > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
        if (e != cudaSuccess) return e;
    }
    const int grid = grid_for(k, C::THREADS, C::SMEM, C::WARPS, a.g.ntiles);
    if (bp) k_lorenzo_nd<ND, B, true><<<grid, C::THREADS, C::SMEM, s>>>(a);
    else k_lorenzo_nd<ND, B, false><<<grid, C::THREADS, C::SMEM, s>>>(a);
    return cudaGetLastError();
}

template <int ND, int B>
cudaError_t launch_nd_recon(const ReconArgs& a, bool q_out, cudaStream_t s) {
    using C = NdCfg<ND, B>;
    const void* k = q_out ? (const void*)k_recon_nd<ND, B, true> : (const void*)k_recon_nd<ND, B, false>;
    if (C::SMEM > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
        if (e != cudaSuccess) return e;
    }
    const int grid = grid_for(k, C::THREADS, C::SMEM, C::WARPS, a.g.ntiles);
    if (q_out) k_recon_nd<ND, B, true><<<grid, C::THREADS, C::SMEM, s>>>(a);
    else k_recon_nd<ND, B, false><<<grid, C::THREADS, C::SMEM, s>>>(a);
    return cudaGetLastError();
}

}  // namespace vsz
