// recon_nd.cuh -- inverse dual-quant for 2D and 3D fields (Sec. III-A).
//
// Same tiles and lane layout as the compression walk; the codes stream
// through a lane-private cp.async ring (8 bytes per lane and row).  Per row:
// residuals from the codes (code - R), outliers patched from the block's
// slice of the outlier list, P added at the block origin, then the inverse of
// each first-order difference:
//   Sx: inclusive scan inside the lane, then a segmented warp scan across
//       the b/4 lanes of the block (shuffles);
//   Sy: running sum over the block's rows (registers, zeroed per plane);
//   Sz: running sum over planes at the same row, in lane-private shared
//       memory (zeroed per tile).
// The walk visits a block's elements in canonical order (planes, rows, then
// x), so the k-th code 0 met in a block is the block's k-th outlier: no
// search over the outlier list is needed.
#pragma once

#include "compress_nd.cuh"

namespace vsz {

template <int ND, int B, bool QOUT>
__global__ void __launch_bounds__(NdCfg<ND, B>::THREADS)
k_recon_nd(const ReconArgs a) {
    using C = NdCfg<ND, B>;
    constexpr int G = C::G;
    constexpr int S = C::S;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    unsigned char* wsm = smem_raw + (size_t)wib * C::WARP_R;
    unsigned char* ring = wsm;
    int4* zs = reinterpret_cast<int4*>(wsm + C::RING_R);
    const uint32_t ring_lane = smem_addr(ring) + lane * 8;

    const Geom& g = a.g;
    const float ebx2 = a.hdr->ebx2;
    const int32_t Pg = a.hdr->pad_global;
    const int32_t R = a.R;
    const bool bp = is_block_pad(a.pad_mode);
    const uint64_t nx = g.nx;
    const uint64_t plane = g.ny * g.nx;
    const int glane = lane & (G - 1);
    const bool first = glane == 0;
    const int src = lane & ~(G - 1);
    const bool vec = a.vec != 0;

    for (uint64_t t = (uint64_t)blockIdx.x * C::WARPS + wib; t < g.ntiles;
         t += (uint64_t)gridDim.x * C::WARPS) {
        const uint64_t s = t % g.nseg;
        const uint64_t rb = t / g.nseg;
        const uint64_t by = rb % g.nby;
        const uint64_t bz = rb / g.nby;
        const uint64_t x0 = s * kSegCols + (uint64_t)lane * 4;
        const uint64_t bx = (s * kSegCols) / B + (uint64_t)(lane / G);
        const bool bexists = bx < g.nbx;
        const int valid = x0 < nx ? (int)umin64(4, nx - x0) : 0;
        const uint32_t vmask = (1u << valid) - 1u;
        const int ylen = (int)umin64(B, g.ny - by * B);
        const int zlen = ND == 3 ? (int)umin64(B, g.nz - bz * B) : 1;
        const int nrows = zlen * ylen;
        const uint64_t blk = (bz * g.nby + by) * g.nbx + bx;
        const uint64_t tile_base = (ND == 3 ? bz * B * plane : 0) + by * B * nx + x0;

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

        auto issue = [&](const RowCursor& ic, int row) {
            if (!vec) return;
            const uint32_t dst = ring_lane + (uint32_t)((row & (S - 1)) * 32 * 8);
            const uint16_t* p = valid ? a.codes + ic.off : a.codes;
            cp_async8(dst, p, valid ? 8u : 0u);
        };

        int32_t ys[4] = {0, 0, 0, 0};
        int32_t zr[C::ZREG ? B : 1][4];
        if (C::ZREG) {
#pragma unroll
            for (int i = 0; i < (C::ZREG ? B : 1); ++i)
#pragma unroll
                for (int k = 0; k < 4; ++k) zr[i][k] = 0;
        }
        if (C::ZSMEM)
            for (int ly = 0; ly < ylen; ++ly) zs[ly * 32 + lane] = make_int4(0, 0, 0, 0);

        RowCursor ic{tile_base, 0, 0};
#pragma unroll
        for (int i = 0; i < S - 1; ++i) {
            if (i < nrows) {
                issue(ic, i);
                ic.next(ylen, nx, plane);
            }
            cp_async_commit();
        }
        RowCursor rc{tile_base, 0, 0};
        int row = 0;

        auto do_row = [&](int ly, int zi) {
            if (row + S - 1 < nrows) {
                issue(ic, row + S - 1);
                ic.next(ylen, nx, plane);
            }
            cp_async_commit();
            uint32_t c[4];
            if (vec) {
                cp_async_wait<S - 1>();
                const uint2 u = *reinterpret_cast<const uint2*>(ring + ((row & (S - 1)) * 32 + lane) * 8);
                c[0] = u.x & 0xffffu; c[1] = u.x >> 16; c[2] = u.y & 0xffffu; c[3] = u.y >> 16;
            } else {
                load4c(a.codes + rc.off, valid, false, c);
            }
            int32_t d[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) d[k] = (int32_t)c[k] - R;
            if (anyout) {
                uint32_t zm = 0;
#pragma unroll
                for (int k = 0; k < 4; ++k) zm |= (c[k] == 0u ? 1u : 0u) << k;
                zm &= vmask;
                if (__any_sync(VSZ_FULL, zm != 0u)) {
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
                            if (r < hi && r < a.out_cap && a.out_idx[r] == (uint32_t)(rc.off + k)) {
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
            }
            if (row == 0 && first) d[0] = wadd(d[0], P);
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
                d[k] = wadd(d[k], ys[k]);
                ys[k] = d[k];
            }
            // Sz
            if (ND == 3) {
                if (C::ZSMEM) {
                    int4& stz = zs[ly * 32 + lane];
                    const int4 pv = stz;
                    d[0] = wadd(d[0], pv.x); d[1] = wadd(d[1], pv.y);
                    d[2] = wadd(d[2], pv.z); d[3] = wadd(d[3], pv.w);
                    stz = make_int4(d[0], d[1], d[2], d[3]);
                } else {
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        d[k] = wadd(d[k], zr[zi][k]);
                        zr[zi][k] = d[k];
                    }
                }
            }
            const bool full = vec && valid == 4;
            if (QOUT) {
                int32_t* o = reinterpret_cast<int32_t*>(a.out) + rc.off;
                if (full) {
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
                float* o = reinterpret_cast<float*>(a.out) + rc.off;
                if (full) {
                    *reinterpret_cast<float4*>(o) = make_float4(v[0], v[1], v[2], v[3]);
                } else {
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        if (k < valid) o[k] = v[k];
                }
            }
            rc.next(ylen, nx, plane);
            ++row;
        };

        for (int lz = 0; lz < zlen; ++lz) {
#pragma unroll
            for (int k = 0; k < 4; ++k) ys[k] = 0;
            if (C::ZREG) {
#pragma unroll
                for (int ly = 0; ly < (C::ZREG ? B : 1); ++ly)
                    if (ly < ylen) do_row(ly, ly);
            } else {
                for (int ly = 0; ly < ylen; ++ly) do_row(ly, 0);
            }
        }
        cp_async_wait<0>();
    }
}

// Host-side launch helpers for one rank, instantiated by k_rank2.cu / k_rank3.cu.
template <int ND, int B>
cudaError_t launch_nd_compress(const CompressArgs& a, cudaStream_t s) {
    using C = NdCfg<ND, B>;
    const bool bp = is_block_pad(a.pad_mode);
    const void* k = bp ? (const void*)k_lorenzo_nd<ND, B, true> : (const void*)k_lorenzo_nd<ND, B, false>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM_C);
    if (e != cudaSuccess) return e;
    const int grid = grid_for(k, C::THREADS, C::SMEM_C, C::WARPS, a.g.ntiles);
    if (bp) k_lorenzo_nd<ND, B, true><<<grid, C::THREADS, C::SMEM_C, s>>>(a);
    else k_lorenzo_nd<ND, B, false><<<grid, C::THREADS, C::SMEM_C, s>>>(a);
    return cudaGetLastError();
}

template <int ND, int B>
cudaError_t launch_nd_recon(const ReconArgs& a, bool q_out, cudaStream_t s) {
    using C = NdCfg<ND, B>;
    const void* k = q_out ? (const void*)k_recon_nd<ND, B, true> : (const void*)k_recon_nd<ND, B, false>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM_R);
    if (e != cudaSuccess) return e;
    const int grid = grid_for(k, C::THREADS, C::SMEM_R, C::WARPS, a.g.ntiles);
    if (q_out) k_recon_nd<ND, B, true><<<grid, C::THREADS, C::SMEM_R, s>>>(a);
    else k_recon_nd<ND, B, false><<<grid, C::THREADS, C::SMEM_R, s>>>(a);
    return cudaGetLastError();
}

}  // namespace vsz
