// compress_nd.cuh -- fused prequant + blockwise Lorenzo + post-quant + guard
// for 2D and 3D fields (Sec. III-A, Alg. 2; padding Sec. IV).
//
// One warp owns one tile: a 128-column segment along x of one row of blocks
// (2D: b rows; 3D: b*b rows, z outer, y inner).  Lane l owns columns
// 4l..4l+3, so b/4 consecutive lanes cover one block along x.  Walking the
// rows in order, the first-order Lorenzo residual is the mixed difference
// delta = Dz Dy Dx q, where a difference at a block's low face is the
// identity (the neighbour outside the block is the padding value, which
// cancels everywhere except at the block origin, delta_origin = q - P):
//   Dx: within the lane, and from lane l-1 by shuffle;
//   Dy: against the previous row's Dx result, carried in registers;
//   Dz: against the previous plane's Dy result at the same row (registers
//       for b <= 8, lane-private shared memory above).
// Every input byte is read once from HBM; codes are written once.
//
// Outliers and fixups are counted per block during the walk.  A tile with
// any reserves one contiguous staging range (one atomic per tile) and then
// re-derives its entries block by block in canonical order (row-major inside
// the block) from the P-padded neighbourhood of each element, which the
// compaction kernel later moves to their final place.
#pragma once

#include <climits>

#include "common.cuh"
#include "memops.cuh"

namespace vsz {

template <int ND, int B>
struct NdCfg {
    static_assert(B >= 4 && B <= 128 && (B & (B - 1)) == 0, "block edge");
    static constexpr int G = B / 4;                        // lanes per block along x
    static constexpr bool ZSMEM = (ND == 3) && (B >= 16);  // z state in shared memory
    static constexpr int WARPS = ZSMEM ? 4 : 8;
    static constexpr int THREADS = WARPS * 32;
    static constexpr int U = (B < 8) ? B : 8;              // rows loaded per batch
    static constexpr size_t SMEM = ZSMEM ? (size_t)WARPS * B * 32 * sizeof(int4) : 0;
};

__device__ __forceinline__ int32_t wsub(int32_t a, int32_t b) { return (int32_t)((uint32_t)a - (uint32_t)b); }
__device__ __forceinline__ int32_t wadd(int32_t a, int32_t b) { return (int32_t)((uint32_t)a + (uint32_t)b); }

// Canonical-order emission of one block's outliers and fixups into staging.
// The residual is evaluated in its P-padded form: the signed sum of q over
// the 2^ND corners of the unit cube below the element, with P for corners
// outside the block.
template <int ND>
__device__ __noinline__ void emit_block_nd(const float* __restrict__ x, uint2* __restrict__ stage_out,
                                           uint2* __restrict__ stage_fix, uint64_t out_cap,
                                           uint64_t fix_cap, uint64_t nx, uint64_t ny, int32_t R,
                                           uint64_t oz, uint64_t oy, uint64_t ox,
                                           uint32_t zlen, uint32_t ylen, uint32_t xlen, int32_t P,
                                           uint64_t ko, uint64_t kf, int lane, float inv2eb, float ebx2,
                                           float ebf) {
    const uint32_t m = zlen * ylen * xlen;
    for (uint32_t i0 = 0; i0 < m; i0 += 32) {
        const uint32_t i = i0 + (uint32_t)lane;
        bool iso = false, isf = false;
        int32_t d = 0;
        uint32_t idx = 0;
        float xv = 0.0f;
        if (i < m) {
            const uint32_t lx = i % xlen;
            const uint32_t rest = i / xlen;
            const uint32_t ly = rest % ylen;
            const uint32_t lz = rest / ylen;
            uint32_t acc = 0;
            int32_t q0 = 0;
#pragma unroll
            for (int dz = 0; dz < (ND == 3 ? 2 : 1); ++dz)
#pragma unroll
                for (int dy = 0; dy < 2; ++dy)
#pragma unroll
                    for (int dx = 0; dx < 2; ++dx) {
                        int32_t qv;
                        if (lz < (uint32_t)dz || ly < (uint32_t)dy || lx < (uint32_t)dx) {
                            qv = P;
                        } else {
                            const uint64_t e = ((oz + lz - dz) * ny + (oy + ly - dy)) * nx + (ox + lx - dx);
                            qv = prequant(x[e], inv2eb);
                        }
                        if (dz + dy + dx == 0) q0 = qv;
                        acc = ((dz + dy + dx) & 1) ? acc - (uint32_t)qv : acc + (uint32_t)qv;
                    }
            d = (int32_t)acc;
            idx = (uint32_t)(((oz + lz) * ny + (oy + ly)) * nx + (ox + lx));
            xv = x[idx];
            iso = code_of(d, R) == 0u;
            isf = needs_fixup(xv, q0, ebx2, ebf);
        }
        const uint32_t mo = __ballot_sync(VSZ_FULL, iso);
        const uint32_t mf = __ballot_sync(VSZ_FULL, isf);
        const uint32_t lt = lanemask_lt();
        if (iso) {
            const uint64_t pos = ko + __popc(mo & lt);
            if (pos < out_cap) stage_out[pos] = make_uint2(idx, (uint32_t)d);
        }
        if (isf) {
            const uint64_t pos = kf + __popc(mf & lt);
            if (pos < fix_cap) stage_fix[pos] = make_uint2(idx, __float_as_uint(xv));
        }
        ko += __popc(mo);
        kf += __popc(mf);
    }
}

template <int ND, int B, bool BP>
__global__ void __launch_bounds__(NdCfg<ND, B>::THREADS)
k_lorenzo_nd(const CompressArgs a) {
    using C = NdCfg<ND, B>;
    constexpr int G = C::G;
    constexpr int U = C::U;
    extern __shared__ int4 zsm[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const Geom& g = a.g;
    const float inv2eb = a.hdr->inv2eb;
    const float ebx2 = a.hdr->ebx2;
    const float ebf = a.hdr->eb_f32;
    const int32_t Pg = a.hdr->pad_global;
    const int32_t R = a.R;
    int4* zs = C::ZSMEM ? (zsm + (size_t)wib * B * 32) : nullptr;
    const uint64_t plane = g.ny * g.nx;
    const int glane = lane & (G - 1);
    const bool first = glane == 0;

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

        int32_t prev1[4] = {0, 0, 0, 0};
        int32_t zr[(ND == 3 && !C::ZSMEM) ? B : 1][4];
        uint32_t cnt_out = 0, cnt_fix = 0;
        int32_t smin = INT_MAX, smax = INT_MIN;
        long long ssum = 0;
        int32_t qcorner = 0;
        uint32_t r0c01 = 0, r0c23 = 0;
        const int32_t P = BP ? 0 : Pg;

        for (int lz = 0; lz < zlen; ++lz) {
            const uint64_t zoff = tile_base + (uint64_t)lz * plane;
#pragma unroll((ND == 3 && !C::ZSMEM) ? B : 1)
            for (int ly0 = 0; ly0 < ((ND == 3 && !C::ZSMEM) ? B : ylen); ly0 += U) {
                float xr[U][4];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int ly = ly0 + u;
                    if (ly < ylen) {
                        load4f(a.x + zoff + (uint64_t)ly * g.nx, valid, vec, xr[u]);
                    } else {
#pragma unroll
                        for (int k = 0; k < 4; ++k) xr[u][k] = 0.0f;
                    }
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int ly = ly0 + u;
                    if (ly >= ylen) break;
                    int32_t q[4];
#pragma unroll
                    for (int k = 0; k < 4; ++k) q[k] = prequant(xr[u][k], inv2eb);
                    int32_t left = __shfl_up_sync(VSZ_FULL, q[3], 1);
                    if (first) left = 0;
                    int32_t r[4];
                    r[0] = wsub(q[0], left);
                    r[1] = wsub(q[1], q[0]);
                    r[2] = wsub(q[2], q[1]);
                    r[3] = wsub(q[3], q[2]);
                    // Dy
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const int32_t r1 = r[k];
                        if (ly > 0) r[k] = wsub(r1, prev1[k]);
                        prev1[k] = r1;
                    }
                    // Dz
                    if (ND == 3) {
                        if (C::ZSMEM) {
                            int4& st = zs[ly * 32 + lane];
                            int4 pv = st;
                            if (lz > 0) {
                                const int32_t r0 = r[0], r1v = r[1], r2v = r[2], r3v = r[3];
                                r[0] = wsub(r0, pv.x); r[1] = wsub(r1v, pv.y);
                                r[2] = wsub(r2v, pv.z); r[3] = wsub(r3v, pv.w);
                                st = make_int4(r0, r1v, r2v, r3v);
                            } else {
                                st = make_int4(r[0], r[1], r[2], r[3]);
                            }
                        } else {
                            const int yi = (ND == 3 && !C::ZSMEM) ? ly : 0;
#pragma unroll
                            for (int k = 0; k < 4; ++k) {
                                const int32_t r2 = r[k];
                                if (lz > 0) r[k] = wsub(r2, zr[yi][k]);
                                zr[yi][k] = r2;
                            }
                        }
                    }
                    const bool corner = first && ly == 0 && lz == 0;
                    if (corner) {
                        if (BP) qcorner = q[0];
                        else r[0] = wsub(r[0], P);
                    }
                    uint32_t c[4];
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        c[k] = code_of(r[k], R);
                        if (k < valid) {
                            if (!(BP && corner && k == 0)) cnt_out += (c[k] == 0u);
                            cnt_fix += needs_fixup(xr[u][k], q[k], ebx2, ebf) ? 1u : 0u;
                            if (BP) {
                                smin = min(smin, q[k]);
                                smax = max(smax, q[k]);
                                ssum += q[k];
                            }
                        }
                    }
                    const uint32_t c01 = c[0] | (c[1] << 16), c23 = c[2] | (c[3] << 16);
                    if (BP && ly == 0 && lz == 0) {
                        r0c01 = c01;
                        r0c23 = c23;
                    } else {
                        store4c(a.codes + zoff + (uint64_t)ly * g.nx, valid, vec, c01, c23);
                    }
                }
            }
        }

        // Per-block padding value (Sec. IV-B-2) and the deferred block origin.
        int32_t Pb = P;
        if (BP) {
#pragma unroll
            for (int off = 1; off < G; off <<= 1) {
                smin = min(smin, __shfl_xor_sync(VSZ_FULL, smin, off));
                smax = max(smax, __shfl_xor_sync(VSZ_FULL, smax, off));
                ssum += __shfl_xor_sync(VSZ_FULL, ssum, off);
            }
            const long long xlen = bexists ? (long long)umin64(B, g.nx - bx * B) : 1;
            const long long m = (long long)zlen * ylen * xlen;
            Pb = a.pad_mode == VSZ_PAD_BLOCK_MIN ? smin
               : a.pad_mode == VSZ_PAD_BLOCK_MAX ? smax
               : rounded_mean(ssum, m);
            if (first && bexists) {
                a.pad[blk] = Pb;
                const uint32_t cc = code_of(wsub(qcorner, Pb), R);
                cnt_out += (cc == 0u);
                r0c01 = (r0c01 & 0xffff0000u) | cc;
            }
            store4c(a.codes + tile_base, valid, vec, r0c01, r0c23);
        }

        // Per-block counts, in-tile exclusive offsets (blk_off), tile totals.
        uint32_t bo = cnt_out, bf = cnt_fix;
#pragma unroll
        for (int off = 1; off < G; off <<= 1) {
            bo += __shfl_xor_sync(VSZ_FULL, bo, off);
            bf += __shfl_xor_sync(VSZ_FULL, bf, off);
        }
        const uint32_t vo = (first && bexists) ? bo : 0u;
        const uint32_t vf = (first && bexists) ? bf : 0u;
        uint32_t io = vo, iff = vf;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t yo = __shfl_up_sync(VSZ_FULL, io, off);
            const uint32_t yf = __shfl_up_sync(VSZ_FULL, iff, off);
            if (lane >= off) { io += yo; iff += yf; }
        }
        const uint32_t eo = io - vo, ef = iff - vf;
        const uint32_t tot_out = __shfl_sync(VSZ_FULL, io, 31);
        const uint32_t tot_fix = __shfl_sync(VSZ_FULL, iff, 31);
        if (first && bexists) a.blk_off[blk] = eo;

        unsigned long long base_out = 0, base_fix = 0;
        if (tot_out | tot_fix) {
            if (lane == 0) {
                if (tot_out) base_out = atomicAdd(&a.wsh->stage_out, (unsigned long long)tot_out);
                if (tot_fix) base_fix = atomicAdd(&a.wsh->stage_fix, (unsigned long long)tot_fix);
                uint4* ch = a.chunks + t / kTilesPerChunk;
                if (tot_out) atomicAdd(&ch->x, tot_out);
                if (tot_fix) atomicAdd(&ch->y, tot_fix);
            }
            base_out = __shfl_sync(VSZ_FULL, base_out, 0);
            base_fix = __shfl_sync(VSZ_FULL, base_fix, 0);
        }
        if (lane == 0)
            a.tiles[t] = make_uint4((uint32_t)base_out, tot_out, (uint32_t)base_fix, tot_fix);

        if (tot_out | tot_fix) {
            uint32_t need = __ballot_sync(VSZ_FULL, first && bexists && (bo | bf));
            while (need) {
                const int l0 = __ffs(need) - 1;
                need &= need - 1;
                const uint32_t eoj = __shfl_sync(VSZ_FULL, eo, l0);
                const uint32_t efj = __shfl_sync(VSZ_FULL, ef, l0);
                const int32_t Pj = BP ? __shfl_sync(VSZ_FULL, Pb, l0) : P;
                const uint64_t bxj = (s * kSegCols) / B + (uint64_t)(l0 / G);
                const uint32_t xlen = (uint32_t)umin64(B, g.nx - bxj * B);
                emit_block_nd<ND>(a.x, a.stage_out, a.stage_fix, a.out_cap, a.fix_cap, g.nx, g.ny, R,
                                  ND == 3 ? bz * B : 0, by * B, bxj * B, (uint32_t)zlen, (uint32_t)ylen,
                                  xlen, Pj, base_out + eoj, base_fix + efj, lane, inv2eb, ebx2, ebf);
            }
        }
    }
}

}  // namespace vsz
