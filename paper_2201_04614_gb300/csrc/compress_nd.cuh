// compress_nd.cuh -- fused prequant + blockwise Lorenzo + post-quant + guard
// for 2D and 3D fields (Sec. III-A, Alg. 2; padding Sec. IV).
//
// One warp owns one tile: a 128-column segment along x of one row of blocks
// (2D: b rows; 3D: b*b rows, z outer, y inner).  Lane l owns columns
// 4l..4l+3, so b/4 consecutive lanes cover one block along x.  Rows stream
// through a lane-private cp.async ring in shared memory (S-1 rows in flight
// per warp while one is processed).  Walking the rows in order, the
// first-order Lorenzo residual is the mixed difference delta = Dz Dy Dx q,
// where a difference at a block's low face is the identity: the neighbour
// outside the block is the padding value P, which cancels everywhere except
// at the block origin, delta_origin = q - P:
//   Dx: within the lane, and from lane l-1 by shuffle;
//   Dy: against the previous row's Dx result (registers, zeroed per plane);
//   Dz: against the previous plane's Dy result at the same row, kept in
//       lane-private shared memory (zeroed per tile).
// Every input byte is read once from HBM and every code written once.
//
// Outliers and fixups met during the walk are appended to a per-warp stash
// in shared memory (walk order).  At the end of the tile one atomic reserves
// the tile's staging range and the stash is scattered into canonical order
// (blocks in row-major order, row-major inside a block) with a counting
// sort keyed by block: inside one block the walk order is already the
// canonical order.  A tile whose stash overflows re-derives its entries
// block by block from the input instead.
#pragma once

#include <climits>

#include "common.cuh"
#include "memops.cuh"
#include "ring.cuh"

namespace vsz {

template <int ND, int B>
struct NdCfg {
    static_assert(B >= 4 && B <= 128 && (B & (B - 1)) == 0, "block edge");
    static constexpr int G = B / 4;                         // lanes per block along x
    static constexpr bool ZSMEM = (ND == 3);                // z state in shared memory
    static constexpr bool ZREG = false;                     // (registers: kept for experiments)
    static constexpr int WARPS = ZSMEM ? 4 : 8;
    static constexpr int THREADS = WARPS * 32;
    static constexpr int S = 8;                             // ring depth (rows)
    static constexpr int STASH = 256;                       // stash entries per warp
    // per-warp shared memory, compression: ring | stash | tables | z state
    static constexpr size_t RING_C = (size_t)S * 32 * 16;
    static constexpr size_t STASH_B = (size_t)STASH * 8;
    static constexpr size_t TAB_B = 128 * 4;
    static constexpr size_t ZS_B = ZSMEM ? (size_t)B * 32 * 16 : 0;
    static constexpr size_t WARP_C = RING_C + STASH_B + TAB_B + ZS_B;
    static constexpr size_t SMEM_C = WARP_C * WARPS;
    // per-warp shared memory, reconstruction: ring of codes | z state
    static constexpr size_t RING_R = (size_t)S * 32 * 8;
    static constexpr size_t WARP_R = RING_R + ZS_B;
    static constexpr size_t SMEM_R = WARP_R * WARPS;
};

__device__ __forceinline__ int32_t wsub(int32_t a, int32_t b) { return (int32_t)((uint32_t)a - (uint32_t)b); }
__device__ __forceinline__ int32_t wadd(int32_t a, int32_t b) { return (int32_t)((uint32_t)a + (uint32_t)b); }

// Canonical-order emission of one block's outliers and fixups into staging,
// re-deriving every element from the input (the stash-overflow path).  The
// residual is evaluated in its P-padded form: the signed sum of q over the
// 2^ND corners of the unit cube below the element, with P for corners
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

// Stash key: [31] fixup? | [30:26] block within the tile | [25:7] row | [6:0] column.
__device__ __forceinline__ uint32_t stash_key(uint32_t fix, uint32_t g, uint32_t row, uint32_t col) {
    return (fix << 31) | (g << 26) | (row << 7) | col;
}

template <int ND, int B, bool BP>
__global__ void __launch_bounds__(NdCfg<ND, B>::THREADS)
k_lorenzo_nd(const CompressArgs a) {
    using C = NdCfg<ND, B>;
    constexpr int G = C::G;
    constexpr int S = C::S;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    unsigned char* wsm = smem_raw + (size_t)wib * C::WARP_C;
    unsigned char* ring = wsm;
    uint2* stash = reinterpret_cast<uint2*>(wsm + C::RING_C);
    uint32_t* pre_out = reinterpret_cast<uint32_t*>(wsm + C::RING_C + C::STASH_B);
    uint32_t* pre_fix = pre_out + 32;
    uint32_t* run = pre_out + 64;  // 64 counters: [fix][group]
    int4* zs = reinterpret_cast<int4*>(wsm + C::RING_C + C::STASH_B + C::TAB_B);
    const uint32_t ring_lane = smem_addr(ring) + lane * 16;

    const Geom& g = a.g;
    const float inv2eb = a.hdr->inv2eb;
    const float ebx2 = a.hdr->ebx2;
    const float ebf = a.hdr->eb_f32;
    const int32_t Pg = a.hdr->pad_global;
    const int32_t R = a.R;
    const uint64_t nx = g.nx;
    const uint64_t plane = g.ny * g.nx;
    const int glane = lane & (G - 1);
    const bool first = glane == 0;
    const uint32_t grp = (uint32_t)(lane / G);
    const uint32_t lt = lanemask_lt();
    const bool vec = a.vec != 0;

    for (uint64_t t = (uint64_t)blockIdx.x * C::WARPS + wib; t < g.ntiles;
         t += (uint64_t)gridDim.x * C::WARPS) {
        const uint64_t s = t % g.nseg;
        const uint64_t rb = t / g.nseg;
        const uint64_t by = rb % g.nby;
        const uint64_t bz = rb / g.nby;
        const uint64_t x0 = s * kSegCols + (uint64_t)lane * 4;
        const uint64_t bx = (s * kSegCols) / B + grp;
        const bool bexists = bx < g.nbx;
        const int valid = x0 < nx ? (int)umin64(4, nx - x0) : 0;
        const uint32_t vmask = (1u << valid) - 1u;
        const bool vst = vec && valid == 4;  // this lane's 4 codes are stored as one 8-byte word
        const int ylen = (int)umin64(B, g.ny - by * B);
        const int zlen = ND == 3 ? (int)umin64(B, g.nz - bz * B) : 1;
        const int nrows = zlen * ylen;
        const uint64_t blk = (bz * g.nby + by) * g.nbx + bx;
        const uint64_t tile_base = (ND == 3 ? bz * B * plane : 0) + by * B * nx + x0;
        const float* xsrc = a.x;

        // issue the copy of one row into its ring slot
        auto issue = [&](const RowCursor& ic, int row) {
            const uint32_t dst = ring_lane + (uint32_t)((row & (S - 1)) * 32 * 16);
            if (vec) {
                const float* src = valid ? xsrc + ic.off : xsrc;
                cp_async16(dst, src, valid ? 16u : 0u);
            } else {
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const float* src = (k < valid) ? xsrc + ic.off + k : xsrc;
                    cp_async4(dst + 4 * k, src, (k < valid) ? 4u : 0u);
                }
            }
        };

        int32_t prev1[4] = {0, 0, 0, 0};
        int32_t zr[C::ZREG ? B : 1][4];
        if (C::ZREG) {
#pragma unroll
            for (int i = 0; i < (C::ZREG ? B : 1); ++i)
#pragma unroll
                for (int k = 0; k < 4; ++k) zr[i][k] = 0;
        }
        if (C::ZSMEM)
            for (int ly = 0; ly < ylen; ++ly) zs[ly * 32 + lane] = make_int4(0, 0, 0, 0);
        uint32_t cnt_out = 0, cnt_fix = 0, nst = 0;
        int32_t smin = INT_MAX, smax = INT_MIN;
        long long ssum = 0;
        int32_t qcorner = 0;
        uint32_t r0c01 = 0, r0c23 = 0;
        const int32_t P = BP ? 0 : Pg;

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
            cp_async_wait<S - 1>();
            const float4 v = *reinterpret_cast<const float4*>(ring + ((row & (S - 1)) * 32 + lane) * 16);
            const float xv[4] = {v.x, v.y, v.z, v.w};
            int32_t q[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) q[k] = prequant(xv[k], inv2eb);
            int32_t left = __shfl_up_sync(VSZ_FULL, q[3], 1);
            if (first) left = 0;
            int32_t d[4];
            d[0] = wsub(q[0], left);
            d[1] = wsub(q[1], q[0]);
            d[2] = wsub(q[2], q[1]);
            d[3] = wsub(q[3], q[2]);
#pragma unroll
            for (int k = 0; k < 4; ++k) {  // Dy
                const int32_t r1 = d[k];
                d[k] = wsub(r1, prev1[k]);
                prev1[k] = r1;
            }
            if (ND == 3) {  // Dz
                if (C::ZSMEM) {
                    int4& st = zs[ly * 32 + lane];
                    const int4 pv = st;
                    st = make_int4(d[0], d[1], d[2], d[3]);
                    d[0] = wsub(d[0], pv.x); d[1] = wsub(d[1], pv.y);
                    d[2] = wsub(d[2], pv.z); d[3] = wsub(d[3], pv.w);
                } else {
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const int32_t r2 = d[k];
                        d[k] = wsub(r2, zr[zi][k]);
                        zr[zi][k] = r2;
                    }
                }
            }
            const bool row0 = row == 0;
            if (row0 && first) {
                if (BP) qcorner = q[0];
                else d[0] = wsub(d[0], P);
            }
            uint32_t c[4], om = 0, fm = 0;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                c[k] = code_of(d[k], R);
                om |= (c[k] == 0u ? 1u : 0u) << k;
                fm |= (needs_fixup(xv[k], q[k], ebx2, ebf) ? 1u : 0u) << k;
                if (BP && k < valid) {
                    smin = min(smin, q[k]);
                    smax = max(smax, q[k]);
                    ssum += q[k];
                }
            }
            om &= vmask;
            fm &= vmask;
            if (BP && row0 && first) om &= ~1u;  // the origin waits for P
            cnt_out += __popc(om);
            cnt_fix += __popc(fm);
            const uint32_t c01 = c[0] | (c[1] << 16), c23 = c[2] | (c[3] << 16);
            if (BP && row0) {
                r0c01 = c01;
                r0c23 = c23;
            } else {
                store4c(a.codes + rc.off, valid, vst, c01, c23);
            }
            if (__any_sync(VSZ_FULL, (om | fm) != 0u)) {
                const uint32_t cl = __popc(om) + __popc(fm);
                uint32_t incl = cl;
#pragma unroll
                for (int off = 1; off < 32; off <<= 1) {
                    const uint32_t y = __shfl_up_sync(VSZ_FULL, incl, off);
                    if (lane >= off) incl += y;
                }
                uint32_t pos = nst + incl - cl;
                const uint32_t total = __shfl_sync(VSZ_FULL, incl, 31);
                if (nst + total <= (uint32_t)C::STASH) {
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        if (om & (1u << k))
                            stash[pos++] = make_uint2(stash_key(0, grp, row, lane * 4 + k), (uint32_t)d[k]);
                        if (fm & (1u << k))
                            stash[pos++] = make_uint2(stash_key(1, grp, row, lane * 4 + k), __float_as_uint(xv[k]));
                    }
                }
                nst += total;
            }
            rc.next(ylen, nx, plane);
            ++row;
        };

        for (int lz = 0; lz < zlen; ++lz) {
#pragma unroll
            for (int k = 0; k < 4; ++k) prev1[k] = 0;
            if (C::ZREG) {
#pragma unroll
                for (int ly = 0; ly < (C::ZREG ? B : 1); ++ly)
                    if (ly < ylen) do_row(ly, ly);
            } else {
                for (int ly = 0; ly < ylen; ++ly) do_row(ly, 0);
            }
        }
        cp_async_wait<0>();

        // Per-block padding value (Sec. IV-B-2) and the deferred block origin.
        int32_t Pb = P;
        uint32_t corner_out = 0;
        int32_t dcorner = 0;
        if (BP) {
#pragma unroll
            for (int off = 1; off < G; off <<= 1) {
                smin = min(smin, __shfl_xor_sync(VSZ_FULL, smin, off));
                smax = max(smax, __shfl_xor_sync(VSZ_FULL, smax, off));
                ssum += __shfl_xor_sync(VSZ_FULL, ssum, off);
            }
            const long long xlen = bexists ? (long long)umin64(B, nx - bx * B) : 1;
            const long long m = (long long)zlen * ylen * xlen;
            Pb = a.pad_mode == VSZ_PAD_BLOCK_MIN ? smin
               : a.pad_mode == VSZ_PAD_BLOCK_MAX ? smax
               : rounded_mean(ssum, m);
            if (first && bexists) {
                a.pad[blk] = Pb;
                dcorner = wsub(qcorner, Pb);
                const uint32_t cc = code_of(dcorner, R);
                corner_out = (cc == 0u) ? 1u : 0u;
                cnt_out += corner_out;
                r0c01 = (r0c01 & 0xffff0000u) | cc;
            }
            store4c(a.codes + tile_base, valid, vst, r0c01, r0c23);
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

        if ((tot_out | tot_fix) && nst <= (uint32_t)C::STASH) {
            // Counting sort of the stash into canonical order.
            if (first) {
                pre_out[grp] = (uint32_t)base_out + eo + corner_out;
                pre_fix[grp] = (uint32_t)base_fix + ef;
                if (BP && corner_out) {
                    const uint64_t pos = base_out + eo;
                    if (pos < a.out_cap) a.stage_out[pos] = make_uint2((uint32_t)tile_base, (uint32_t)dcorner);
                }
            }
            run[lane] = 0;
            run[lane + 32] = 0;
            __syncwarp();
            const uint64_t row_base = (ND == 3 ? bz * B * plane : 0) + by * B * nx + s * kSegCols;
            for (uint32_t j0 = 0; j0 < nst; j0 += 32) {
                const uint32_t j = j0 + lane;
                const bool act = j < nst;
                const uint2 e = act ? stash[j] : make_uint2(0, 0);
                const uint32_t bucket = act ? (e.x >> 26) : (64u + lane);
                const uint32_t peers = __match_any_sync(VSZ_FULL, bucket);
                const uint32_t rank = __popc(peers & lt);
                uint32_t cnt0 = 0;
                if (act) {
                    const uint32_t isfix = e.x >> 31;
                    const uint32_t gb = (e.x >> 26) & 31u;
                    const uint32_t rowi = (e.x >> 7) & 0x7ffffu;
                    const uint32_t col = e.x & 127u;
                    cnt0 = run[bucket];
                    const uint32_t lzr = rowi / (uint32_t)ylen, lyr = rowi % (uint32_t)ylen;
                    const uint32_t idx = (uint32_t)(row_base + (uint64_t)lzr * plane + (uint64_t)lyr * nx + col);
                    const uint64_t pos = (uint64_t)(isfix ? pre_fix[gb] : pre_out[gb]) + cnt0 + rank;
                    if (isfix) {
                        if (pos < a.fix_cap) a.stage_fix[pos] = make_uint2(idx, e.y);
                    } else {
                        if (pos < a.out_cap) a.stage_out[pos] = make_uint2(idx, e.y);
                    }
                }
                __syncwarp();
                if (act && (peers >> lane) == 1u) run[bucket] = cnt0 + rank + 1;  // last peer updates
                __syncwarp();
            }
        } else if (tot_out | tot_fix) {
            // Stash overflow: re-derive the entries block by block.
            uint32_t need = __ballot_sync(VSZ_FULL, first && bexists && (bo | bf));
            while (need) {
                const int l0 = __ffs(need) - 1;
                need &= need - 1;
                const uint32_t eoj = __shfl_sync(VSZ_FULL, eo, l0);
                const uint32_t efj = __shfl_sync(VSZ_FULL, ef, l0);
                const int32_t Pj = BP ? __shfl_sync(VSZ_FULL, Pb, l0) : P;
                const uint64_t bxj = (s * kSegCols) / B + (uint64_t)(l0 / G);
                const uint32_t xlen = (uint32_t)umin64(B, nx - bxj * B);
                emit_block_nd<ND>(a.x, a.stage_out, a.stage_fix, a.out_cap, a.fix_cap, nx, g.ny, R,
                                  ND == 3 ? bz * B : 0, by * B, bxj * B, (uint32_t)zlen, (uint32_t)ylen,
                                  xlen, Pj, base_out + eoj, base_fix + efj, lane, inv2eb, ebx2, ebf);
            }
        }
        __syncwarp();
    }
}

}  // namespace vsz
