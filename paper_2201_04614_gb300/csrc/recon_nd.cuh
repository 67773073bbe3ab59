// recon_nd.cuh -- inverse dual-quant for 2D and 3D fields (Sec. III-A).
//
// Same tiles, lane layout and batches of rows as the compression walk; the
// codes stream through a lane-private, multi-stage cp.async ring (8 bytes
// per lane and row).  Per row:
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
// search over the outlier list is needed.  A batch is first checked for
// code 0 as a whole; only batches that contain one take the patching path.
#pragma once

#include <type_traits>

#include "compress_nd.cuh"

namespace vsz {

// Codes 1 (residual 1 - R, never an outlier), which a lane past a field's
// last column copies instead of codes in the lean reconstruction walk, so
// that the walk's outlier tests need no mask (global memory, never written).
__device__ __align__(16) uint16_t kOneCodes[8] = {1, 1, 1, 1, 1, 1, 1, 1};

// The inverse of one tile t of one field, by one warp whose shared memory
// slice is wsm.
template <int ND, int B, bool QOUT>
__device__ __forceinline__ void nd_recon_tile(const ReconArgs& a, const uint64_t t, unsigned char* wsm,
                                              const int lane) {
    using C = NdCfg<ND, B>;
    constexpr int G = C::G;
    constexpr int U = C::U;
    int4* zs = reinterpret_cast<int4*>(wsm + C::RING_R);
    uint32_t* const oc_idx0 = reinterpret_cast<uint32_t*>(wsm + C::RING_R + C::ZS_B);
    // interior tiles of 3D blocks up to 8 keep their z sums in registers, so
    // their outlier cache may also take the z-state area in front of it
    constexpr bool ZREG_R = ND == 3 && B <= 8;
    constexpr uint32_t OCAP_BIG = (uint32_t)((C::ZS_B + C::OC_B - C::PS_RAW) / 8);  // ps takes the end
    const uint2* ring_rd = reinterpret_cast<const uint2*>(wsm) + lane;  // slot (h*U + u)*32
    const uint32_t ring_wr = smem_addr(wsm) + lane * 8;

    const Geom& g = a.g;
    const float ebx2 = a.hdr->ebx2;
    const int32_t Pg = a.hdr->pad_global;
    // every finite value had |x * inv2eb| < 2^20 (the range recorded by a
    // relative-mode compression), so every q of a finite value converts to
    // float exactly by the bias trick; non-finite values are fixups
    const float inv2eb_h = a.hdr->inv2eb;
    const bool fastcvt = a.hdr->has_range != 0u && fabsf(__fmul_rn(a.hdr->xmin, inv2eb_h)) < 1048576.0f &&
                         fabsf(__fmul_rn(a.hdr->xmax, inv2eb_h)) < 1048576.0f;
    const int32_t R = a.R;
    const bool bp = is_block_pad(a.pad_mode);
    const bool ep = is_edge_pad(a.pad_mode);
    const uint64_t nx = g.nx;
    const uint64_t plane = g.ny * g.nx;
    const int glane = lane & (G - 1);
    const bool first = glane == 0;
    const int src = lane & ~(G - 1);
    const bool vec = a.vec != 0;

    const uint64_t s = t % g.nseg;
    const uint64_t rb = t / g.nseg;
    const uint64_t by = rb % g.nby;
    const uint64_t bz = rb / g.nby;
    const uint64_t x0 = s * kSegCols + (uint64_t)lane * 4;
    const uint64_t bx = (s * kSegCols) / B + (uint64_t)(lane / G);
    const bool bexists = bx < g.nbx;
    const int valid = x0 < nx ? (int)umin64(4, nx - x0) : 0;
    const uint32_t vmask = (1u << valid) - 1u;
    const bool full = vec && valid == 4;
    const int ylen = (int)umin64(B, g.ny - by * B);
    const int zlen = ND == 3 ? (int)umin64(B, g.nz - bz * B) : 1;
    const int nbpp = (ylen + U - 1) / U;
    const int nbatch = zlen * nbpp;
    const uint64_t blk = (bz * g.nby + by) * g.nbx + bx;
    const uint64_t tile_base = (ND == 3 ? bz * B * plane : 0) + by * B * nx + x0;

    uint32_t lo = 0, hi = 0;
    int32_t P = Pg;
    if (first && bexists) {
        lo = a.blk_off[blk];
        hi = a.blk_off[blk + 1];
        if (bp) P = a.pad[blk];
        else if (ep) P = edge_origin_pred(a.pad + blk * ND, ND);
    }
    lo = __shfl_sync(VSZ_FULL, lo, src);
    hi = __shfl_sync(VSZ_FULL, hi, src);
    P = __shfl_sync(VSZ_FULL, P, src);
    const bool anyout = __any_sync(VSZ_FULL, hi > lo);
    uint32_t rank = lo;

    // The tile's blocks are consecutive in canonical order, so its outliers
    // are one slice of the list: bring it into shared memory with the first
    // batch when it is short enough.
    uint32_t lo_t = 0;
    bool cached = false;
    // interior tile: b rows and (3D) b planes, every lane 4 columns or (the
    // field's last segment, nx a multiple of 4) none
    const bool interior = vec && ylen == B && (ND == 2 || zlen == B);
    const uint32_t ocap = ZREG_R && interior ? OCAP_BIG : (uint32_t)C::OCAP;
    uint32_t* const oc_idx = ZREG_R && interior ? reinterpret_cast<uint32_t*>(zs) : oc_idx0;
    int32_t* const oc_del = reinterpret_cast<int32_t*>(oc_idx + ocap);
    if (anyout) {
        const uint64_t fb = (bz * g.nby + by) * g.nbx + (s * kSegCols) / B;
        const uint64_t nblk = umin64(kSegCols / B, g.nbx - (s * kSegCols) / B);
        uint32_t hi_t = 0;
        if (lane == 0) {
            lo_t = a.blk_off[fb];
            hi_t = a.blk_off[fb + nblk];
        }
        lo_t = __shfl_sync(VSZ_FULL, lo_t, 0);
        hi_t = __shfl_sync(VSZ_FULL, hi_t, 0);
        cached = hi_t >= lo_t && hi_t - lo_t <= ocap && (uint64_t)hi_t <= a.out_cap;
        if (cached) {
            const uint32_t sidx = smem_addr(oc_idx), sdel = smem_addr(oc_del);
            for (uint32_t i = lane; i < hi_t - lo_t; i += 32) {
                cp_async4(sidx + 4 * i, a.out_idx + lo_t + i, 4u);
                cp_async4(sdel + 4 * i, a.out_delta + lo_t + i, 4u);
            }
        }
    }

    // Outliers of one batch of an interior tile (every code 0 of its U rows),
    // fetched at once: the k-th code 0 met in a block (planes, rows, then x)
    // is the block's k-th outlier, so each one's rank is the block's running
    // rank plus the code-0 counts of the earlier rows of the batch, of the
    // block's earlier lanes in its row, and of the lane's earlier columns.
    // The residuals land in ps (per lane and row), from where the row walk
    // takes them; a tile whose outliers are cached in shared memory reads
    // them from there, four at a time.
    int4* const ps = reinterpret_cast<int4*>(wsm + C::RING_R + C::ZS_B + C::OC_B - (ZREG_R ? C::PS_RAW : 0)) + lane;
    auto patch_batch = [&](const uint2 (&cw)[U], uint32_t base, uint32_t nx32) {
        uint32_t zm = 0;  // bit u*4 + k: code 0 at row u, column k
#pragma unroll
        for (int u = 0; u < U; ++u) {
            zm |= (((cw[u].x & 0xffffu) == 0u) ? 1u : 0u) << (4 * u);
            zm |= (((cw[u].x >> 16) == 0u) ? 2u : 0u) << (4 * u);
            zm |= (((cw[u].y & 0xffffu) == 0u) ? 4u : 0u) << (4 * u);
            zm |= (((cw[u].y >> 16) == 0u) ? 8u : 0u) << (4 * u);
        }
        // code-0 counts per row, one byte each (at most 4 per lane, 4G per block)
        uint32_t pk = 0;
#pragma unroll
        for (int u = 0; u < U; ++u) pk |= (uint32_t)__popc((zm >> (4 * u)) & 0xfu) << (8 * u);
        uint32_t inc = pk;
#pragma unroll
        for (int off = 1; off < G; off <<= 1) {
            const uint32_t y = __shfl_up_sync(VSZ_FULL, inc, off);
            if (glane >= off) inc += y;
        }
        const uint32_t tot = __shfl_sync(VSZ_FULL, inc, src + G - 1);  // the block's count per row
        const uint32_t excl = inc - pk;                                  // earlier lanes of the block, per row
        uint32_t rowpre[U];                                              // earlier rows of the batch
        rowpre[0] = rank;
#pragma unroll
        for (int u = 1; u < U; ++u) rowpre[u] = rowpre[u - 1] + ((tot >> (8 * (u - 1))) & 0xffu);
        auto rank_of = [&](uint32_t jq) {
            const uint32_t u = jq >> 2, k = jq & 3u;
            uint32_t rb = rowpre[0];
#pragma unroll
            for (int w = 1; w < U; ++w) rb = u == (uint32_t)w ? rowpre[w] : rb;
            return rb + ((excl >> (8 * u)) & 0xffu) + (uint32_t)__popc((zm >> (4 * u)) & ((1u << k) - 1u));
        };
        if (!cached) {
            // Outliers from the global lists: every one of the batch copied
            // into shared memory at once (index beside residual, in the cache
            // area this tile leaves unused), then one wait: a batch costs one
            // memory latency however many outliers it holds.  The wait also
            // completes the ring's prefetched batches, which stay valid.
            int32_t* const pi = reinterpret_cast<int32_t*>(reinterpret_cast<int4*>(oc_idx) + lane);
            int32_t* const pd = reinterpret_cast<int32_t*>(ps);
            const uint32_t spi = smem_addr(pi), spd = smem_addr(pd);
            uint32_t m = zm;
#pragma unroll 1
            while (m) {
                const uint32_t jq = (uint32_t)(__ffs(m) - 1);
                m &= m - 1u;
                const uint32_t r = rank_of(jq);
                const uint32_t off = (jq >> 2) * 32 * 16 + (jq & 3u) * 4;  // row u of the lane's column, entry k
                if (r < hi && r < a.out_cap) {
                    cp_async4(spi + off, a.out_idx + r, 4u);
                    cp_async4(spd + off, a.out_delta + r, 4u);
                } else {
                    pi[off / 4] = -1;  // no such outlier: reported below
                }
            }
            cp_async_commit();
            cp_async_wait<0>();
            m = zm;
#pragma unroll 1
            while (m) {
                const uint32_t jq = (uint32_t)(__ffs(m) - 1);
                m &= m - 1u;
                const uint32_t off = (jq >> 2) * 32 * 4 + (jq & 3u);  // in 4-byte words
                if ((uint32_t)pi[off] != base + (jq >> 2) * nx32 + (jq & 3u)) {
                    atomicMax(&a.hdr->recon_status, (unsigned)VSZ_ERR_CORRUPT);
                    pd[off] = 0;
                }
            }
            rank = rowpre[U - 1] + ((tot >> (8 * (U - 1))) & 0xffu);
            return;
        }
        uint32_t m = zm;
#pragma unroll 1
        while (m) {
            uint32_t jj[4], rr[4], oi[4];
            int32_t od[4];
            bool v[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                v[q] = m != 0u;
                jj[q] = v[q] ? (uint32_t)(__ffs(m) - 1) : 0u;
                m &= m - 1u;
                rr[q] = rank_of(jj[q]);
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const bool in = v[q] && rr[q] < hi && rr[q] < a.out_cap;
                oi[q] = ~0u;
                od[q] = 0;
                if (in && (!cached || VSZ_IN(rr[q] - lo_t, ocap, 203))) {
                    oi[q] = cached ? oc_idx[rr[q] - lo_t] : a.out_idx[rr[q]];
                    od[q] = cached ? oc_del[rr[q] - lo_t] : a.out_delta[rr[q]];
                }
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (!v[q]) continue;
                const uint32_t u = jj[q] >> 2, k = jj[q] & 3u;
                int32_t val = od[q];
                if (oi[q] != base + u * nx32 + k) {
                    atomicMax(&a.hdr->recon_status, (unsigned)VSZ_ERR_CORRUPT);
                    val = 0;
                }
                reinterpret_cast<int32_t*>(ps + u * 32)[k] = val;
            }
        }
        rank = rowpre[U - 1] + ((tot >> (8 * (U - 1))) & 0xffu);
    };

    // copy the codes of batch (lz, j) into ring half h (vector path only)
    auto issue_batch = [&](int lz, int j, int h) {
        if (vec) {
            const uint64_t off0 = tile_base + (uint64_t)lz * plane + (uint64_t)(j * U) * nx;
            const uint32_t dst0 = ring_wr + (uint32_t)(h * U * 32 * 8);
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (j * U + u < ylen) {
                    const uint64_t off = off0 + (uint64_t)u * nx;
                    cp_async8(dst0 + u * 32 * 8, valid ? a.codes + off : a.codes, valid ? 8u : 0u);
                }
            }
        }
        cp_async_commit();
    };

    if (interior) {
        // Lean walk of an interior tile: compile-time trip counts, 32-bit
        // offsets, and P carried in the running-sum state (the z sums of
        // 3D blocks start from P, the y sums of 2D blocks), which adds P
        // to every element of the block exactly as adding it to the
        // origin's residual before the sums does.  3D blocks of up to 8
        // keep their z sums in registers (the rows of a plane unrolled).
        constexpr int BPP = B / U;
        constexpr int NPL = ND == 3 ? B : 1;
        constexpr bool ZREG = ND == 3 && B <= 8;
        constexpr int NB = NPL * BPP;
        const uint32_t nx32 = (uint32_t)nx, pl32 = (uint32_t)plane;
        const uint16_t* cl = a.codes + tile_base;
        auto issue_fast = [&](int kb, int st) {
            const uint16_t* src0 = cl + (uint32_t)(kb / BPP) * pl32 + (uint32_t)((kb % BPP) * U) * nx32;
            const uint32_t dst0 = ring_wr + (uint32_t)(st * U * 32 * 8);
#pragma unroll
            for (int u = 0; u < U; ++u)  // a lane past the field's last column copies codes 1 (no outlier)
                cp_async8(dst0 + u * 32 * 8, valid ? src0 + (uint32_t)u * nx32 : kOneCodes, 8u);
            cp_async_commit();
        };
#pragma unroll
        for (int st = 0; st < C::NSR - 1; ++st) {
            if (st < NB) issue_fast(st, st);
            else cp_async_commit();
        }
        int32_t zr[ZREG ? B : 1][4];
#pragma unroll
        for (int ly = 0; ly < (ZREG ? B : 1); ++ly)
#pragma unroll
            for (int k = 0; k < 4; ++k) zr[ly][k] = P;
        if (ND == 3 && !ZREG) {
#pragma unroll 4
            for (int ly = 0; ly < B; ++ly) zs[ly * 32 + lane] = make_int4(P, P, P, P);
        }
        int32_t ys[4];
        int h = 0, kb = 0;
        for (int lz = 0; lz < NPL; ++lz) {
#pragma unroll
            for (int k = 0; k < 4; ++k) ys[k] = ND == 3 ? 0 : P;
#pragma unroll(ZREG ? BPP : 1)
            for (int jb = 0; jb < BPP; ++jb, ++kb) {
                if (kb + C::NSR - 1 < NB) issue_fast(kb + C::NSR - 1, (kb + C::NSR - 1) % C::NSR);
                else cp_async_commit();
                cp_async_wait<C::NSR - 1>();
                if (cached && kb == 0) __syncwarp();  // every lane's share of the outlier slice has landed
                const uint32_t boff = (uint32_t)lz * pl32 + (uint32_t)(jb * U) * nx32;
                const uint2* rr = ring_rd + h * U * 32;
                uint2 cw[U];
                uint32_t hz = 0;
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    cw[u] = rr[u * 32];
                    hz |= ((cw[u].x - 0x00010001u) & ~cw[u].x & 0x80008000u) |
                          ((cw[u].y - 0x00010001u) & ~cw[u].y & 0x80008000u);
                }
                const bool patch = anyout && __any_sync(VSZ_FULL, hz != 0u);
                if (patch) patch_batch(cw, (uint32_t)tile_base + boff, nx32);
                // one copy of the row code (the patch test is a uniform
                // branch), which keeps the unrolled plane loop small
                auto lrow = [&](int u) {
                    const uint32_t c[4] = {cw[u].x & 0xffffu, cw[u].x >> 16, cw[u].y & 0xffffu, cw[u].y >> 16};
                    int32_t d[4];
#pragma unroll
                    for (int k = 0; k < 4; ++k) d[k] = (int32_t)c[k] - R;
                    if (patch) {  // the outliers' residuals, fetched for the whole batch
                        const int4 pv = ps[u * 32];
                        d[0] = c[0] ? d[0] : pv.x;
                        d[1] = c[1] ? d[1] : pv.y;
                        d[2] = c[2] ? d[2] : pv.z;
                        d[3] = c[3] ? d[3] : pv.w;
                    }
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
                    if (ZREG) {
                        const int ly = ZREG ? jb * U + u : 0;
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            d[k] = wadd(d[k], zr[ly][k]);
                            zr[ly][k] = d[k];
                        }
                    } else if (ND == 3) {
                        int4& stz = zs[(jb * U + u) * 32 + lane];
                        const int4 pv = stz;
                        d[0] = wadd(d[0], pv.x); d[1] = wadd(d[1], pv.y);
                        d[2] = wadd(d[2], pv.z); d[3] = wadd(d[3], pv.w);
                        stz = make_int4(d[0], d[1], d[2], d[3]);
                    }
                    const uint32_t ro = boff + (uint32_t)u * nx32;
                    if (QOUT) {
                        if (valid && VSZ_IN(tile_base + ro + 3, g.n, 201))
                        st_out4(reinterpret_cast<int4*>(reinterpret_cast<int32_t*>(a.out) + tile_base + ro),
                                make_int4(d[0], d[1], d[2], d[3]));
                    } else {
                        int4 vv;
                        if (fastcvt) {  // (float)q by the 1.5 * 2^23 bias, exact for |q| < 2^22
                            vv.x = __float_as_int(__fmul_rn(__fsub_rn(__int_as_float(d[0] + 0x4B400000), 12582912.0f), ebx2));
                            vv.y = __float_as_int(__fmul_rn(__fsub_rn(__int_as_float(d[1] + 0x4B400000), 12582912.0f), ebx2));
                            vv.z = __float_as_int(__fmul_rn(__fsub_rn(__int_as_float(d[2] + 0x4B400000), 12582912.0f), ebx2));
                            vv.w = __float_as_int(__fmul_rn(__fsub_rn(__int_as_float(d[3] + 0x4B400000), 12582912.0f), ebx2));
                        } else {
                            vv.x = __float_as_int(__fmul_rn(q2f(d[0]), ebx2));
                            vv.y = __float_as_int(__fmul_rn(q2f(d[1]), ebx2));
                            vv.z = __float_as_int(__fmul_rn(q2f(d[2]), ebx2));
                            vv.w = __float_as_int(__fmul_rn(q2f(d[3]), ebx2));
                        }
                        if (valid && VSZ_IN(tile_base + ro + 3, g.n, 202))
                            st_out4(reinterpret_cast<int4*>(reinterpret_cast<float*>(a.out) + tile_base + ro), vv);
                    }
                };
#pragma unroll
                for (int u = 0; u < U; ++u) lrow(u);
                h = h + 1 == C::NSR ? 0 : h + 1;
            }
        }
        cp_async_wait<0>();
        return;
    }

    int32_t ys[4] = {0, 0, 0, 0};
    if (C::ZSMEM)
        for (int ly = 0; ly < ylen; ++ly) zs[ly * 32 + lane] = make_int4(0, 0, 0, 0);

    int ilz = 0, ij = 0;  // next batch to issue
#pragma unroll
    for (int st = 0; st < C::NSR - 1; ++st) {
        if (st < nbatch) {
            issue_batch(ilz, ij, st);
            if (++ij == nbpp) { ij = 0; ++ilz; }
        } else {
            cp_async_commit();
        }
    }
    int lz = 0, j = 0, h = 0, hs = C::NSR - 1;
    for (int kb = 0; kb < nbatch; ++kb) {
        int nj = j + 1, nlz = lz;
        if (nj == nbpp) { nj = 0; ++nlz; }
        if (kb + C::NSR - 1 < nbatch) {
            issue_batch(ilz, ij, hs);
            if (++ij == nbpp) { ij = 0; ++ilz; }
        } else {
            cp_async_commit();
        }
        cp_async_wait<C::NSR - 1>();
        if (cached && kb == 0) __syncwarp();  // every lane's share of the outlier slice has landed
        if (j == 0) {
#pragma unroll
            for (int k = 0; k < 4; ++k) ys[k] = 0;
        }
        const uint64_t boff = tile_base + (uint64_t)lz * plane + (uint64_t)(j * U) * nx;
        const bool b0 = kb == 0;
        // Codes of the batch; rows past the edge read as "no outlier".
        uint2 cw[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (j * U + u < ylen) {
                if (vec) {
                    cw[u] = ring_rd[(h * U + u) * 32];
                } else {
                    uint32_t c4[4];
                    load4c(a.codes + boff + (uint64_t)u * nx, valid, false, c4);
                    const uint32_t rr = (uint32_t)R;
                    cw[u] = make_uint2((valid > 0 ? c4[0] : rr) | ((valid > 1 ? c4[1] : rr) << 16),
                                       (valid > 2 ? c4[2] : rr) | ((valid > 3 ? c4[3] : rr) << 16));
                }
            } else {
                cw[u] = make_uint2(0x00010001u, 0x00010001u);
            }
        }
        // Does any code 0 (an outlier) occur in this batch?
        uint32_t hz = 0;
#pragma unroll
        for (int u = 0; u < U; ++u)
            hz |= ((cw[u].x - 0x00010001u) & ~cw[u].x & 0x80008000u) |
                  ((cw[u].y - 0x00010001u) & ~cw[u].y & 0x80008000u);
        const bool patch = anyout && __any_sync(VSZ_FULL, valid > 0 && hz != 0u);

        auto row = [&](auto patch_tag, int u) {
            constexpr bool PATCH = decltype(patch_tag)::value;
            const int ly = j * U + u;
            const uint64_t roff = boff + (uint64_t)u * nx;
            const uint32_t c[4] = {cw[u].x & 0xffffu, cw[u].x >> 16, cw[u].y & 0xffffu, cw[u].y >> 16};
            int32_t d[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) d[k] = (int32_t)c[k] - R;
            if (PATCH) {
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
                            const bool in = r < hi && r < a.out_cap;
                            const uint32_t oi = !in ? ~0u : cached ? oc_idx[r - lo_t] : a.out_idx[r];
                            if (in && oi == (uint32_t)(roff + k)) {
                                d[k] = cached ? oc_del[r - lo_t] : a.out_delta[r];
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
            if (b0 && u == 0 && first) d[0] = wadd(d[0], P);
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
            if (C::ZSMEM) {
                int4& stz = zs[ly * 32 + lane];
                const int4 pv = stz;
                d[0] = wadd(d[0], pv.x); d[1] = wadd(d[1], pv.y);
                d[2] = wadd(d[2], pv.z); d[3] = wadd(d[3], pv.w);
                stz = make_int4(d[0], d[1], d[2], d[3]);
            }
            if (valid > 0 && !VSZ_IN(roff + valid - 1, g.n, 204)) {
                // (bounds-checking build only) an output row past the field
            } else if (QOUT) {
                int32_t* o = reinterpret_cast<int32_t*>(a.out) + roff;
                if (full) {
                    *reinterpret_cast<int4*>(o) = make_int4(d[0], d[1], d[2], d[3]);
                } else {
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        if (k < valid) o[k] = d[k];
                }
            } else {
                float vv[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) vv[k] = __fmul_rn(q2f(d[k]), ebx2);
                float* o = reinterpret_cast<float*>(a.out) + roff;
                if (full) {
                    *reinterpret_cast<float4*>(o) = make_float4(vv[0], vv[1], vv[2], vv[3]);
                } else {
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        if (k < valid) o[k] = vv[k];
                }
            }
        };
        if (patch) {
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (j * U + u < ylen) row(std::true_type{}, u);
        } else {
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (j * U + u < ylen) row(std::false_type{}, u);
        }
        h = h + 1 == C::NSR ? 0 : h + 1;
        hs = hs + 1 == C::NSR ? 0 : hs + 1;
        lz = nlz;
        j = nj;
    }
    cp_async_wait<0>();
}

// One field: tiles from the ticket when there is one (evens out tiles with
// many outliers), else a static grid stride.
template <int ND, int B, bool QOUT>
__global__ void __launch_bounds__(NdCfg<ND, B>::THREADS, NdCfg<ND, B>::MINB_R)
k_recon_nd(const ReconArgs a) {
    pdl_prologue();
    using C = NdCfg<ND, B>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    unsigned char* wsm = smem_raw + (size_t)wib * C::WARP_R;
    uint64_t tnext = (uint64_t)blockIdx.x * C::WARPS + wib;
    for (;;) {
        uint64_t t = tnext;
        if (a.ticket) {
            unsigned int tk = 0;
            if (lane == 0) tk = atomicAdd(a.ticket, 1u);
            t = __shfl_sync(VSZ_FULL, tk, 0);
        }
        tnext += (uint64_t)gridDim.x * C::WARPS;
        if (t >= a.g.ntiles) break;
        nd_recon_tile<ND, B, QOUT>(a, t, wsm, lane);
    }
}

// Many fields of one class (rank, block edge): one queue over the tiles of
// all of them (tile_prefix as for the batch compression); any warps per CTA
// up to 8.
template <int ND, int B>
__global__ void __launch_bounds__(NdBatchBounds<ND, B>::MAXT, NdBatchBounds<ND, B>::MINB_R)
k_recon_nd_batch(const ReconArgs* __restrict__ fields, const uint64_t* __restrict__ tile_prefix, int nfields,
                 unsigned long long* ticket) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    unsigned char* wsm = smem_raw + (size_t)(threadIdx.x >> 5) * NdCfg<ND, B>::WARP_R;
    const uint64_t total = tile_prefix[nfields];
    for (;;) {
        unsigned long long tk = 0;
        if (lane == 0) tk = atomicAdd(ticket, 1ull);
        const uint64_t gt = __shfl_sync(VSZ_FULL, tk, 0);
        if (gt >= total) break;
        int lo = 0, hi = nfields - 1;  // last field whose first tile is <= gt
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (tile_prefix[mid] <= gt) lo = mid; else hi = mid - 1;
        }
        nd_recon_tile<ND, B, false>(fields[lo], gt - tile_prefix[lo], wsm, lane);
    }
}

// Host-side launch helpers for one rank, instantiated by k_rank2.cu / k_rank3.cu.
template <int ND, int B, bool BP, bool GP, bool EP = false>
cudaError_t launch_nd_compress_k(const CompressArgs& a, cudaStream_t s) {
    using C = NdCfg<ND, B>;
    const void* k = (const void*)k_lorenzo_nd<ND, B, BP, GP, EP>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM_C);
    if (e != cudaSuccess) return e;
    const int grid = grid_for(k, C::THREADS, C::SMEM_C, C::WARPS, a.g.ntiles);
    return launch_pdl(k_lorenzo_nd<ND, B, BP, GP, EP>, grid, C::THREADS, C::SMEM_C, s, a);
}

template <int ND, int B>
cudaError_t launch_nd_compress(const CompressArgs& a, cudaStream_t s) {
    if (is_block_pad(a.pad_mode)) return launch_nd_compress_k<ND, B, true, false>(a, s);
    if (is_edge_pad(a.pad_mode)) return launch_nd_compress_k<ND, B, false, true, true>(a, s);
    if (defers_origin(a.pad_mode)) return launch_nd_compress_k<ND, B, false, true>(a, s);
    return launch_nd_compress_k<ND, B, false, false>(a, s);
}

template <int ND, int B, bool BP, bool GP, bool EP = false>
cudaError_t launch_nd_compress_batch_k(const CompressArgs* fields, const uint64_t* tile_prefix, int nfields,
                                       uint64_t total_tiles, unsigned long long* ticket, LaunchShape sh,
                                       cudaStream_t s, int* occ) {
    using C = NdCfg<ND, B>;
    const void* k = (const void*)k_lorenzo_nd_batch<ND, B, BP, GP, EP>;
    const int warps = sh.warps > 0 ? sh.warps : C::WARPS;
    if (warps * 32 > NdBatchBounds<ND, B>::MAXT) {
        if (occ) *occ = 0;
        return occ ? cudaSuccess : cudaErrorInvalidValue;
    }
    const size_t smem = C::WARP_C * (size_t)warps;
    cudaError_t e = raise_smem_attr(k, smem);
    if (occ) {
        *occ = e == cudaSuccess ? occupancy(k, warps * 32, smem) : 0;
        return cudaSuccess;
    }
    if (e != cudaSuccess) return e;
    const int grid = grid_shape(k, warps * 32, smem, (uint64_t)warps, total_tiles, sh.ctas);
    k_lorenzo_nd_batch<ND, B, BP, GP, EP><<<grid, warps * 32, smem, s>>>(fields, tile_prefix, nfields, ticket);
    return cudaGetLastError();
}

// pk: 0 zero padding, 1 per-block padding, 2 global padding, 3 edge padding
template <int ND, int B>
cudaError_t launch_nd_compress_batch(int pk, const CompressArgs* fields, const uint64_t* tile_prefix, int nfields,
                                     uint64_t total_tiles, unsigned long long* ticket, LaunchShape sh,
                                     cudaStream_t s, int* occ) {
    if (pk == 1)
        return launch_nd_compress_batch_k<ND, B, true, false>(fields, tile_prefix, nfields, total_tiles, ticket, sh, s, occ);
    if (pk == 3)
        return launch_nd_compress_batch_k<ND, B, false, true, true>(fields, tile_prefix, nfields, total_tiles, ticket, sh,
                                                                    s, occ);
    if (pk == 2)
        return launch_nd_compress_batch_k<ND, B, false, true>(fields, tile_prefix, nfields, total_tiles, ticket, sh, s, occ);
    return launch_nd_compress_batch_k<ND, B, false, false>(fields, tile_prefix, nfields, total_tiles, ticket, sh, s, occ);
}

template <int ND, int B>
cudaError_t launch_nd_recon(const ReconArgs& a, bool q_out, cudaStream_t s) {
    using C = NdCfg<ND, B>;
    const void* k = q_out ? (const void*)k_recon_nd<ND, B, true> : (const void*)k_recon_nd<ND, B, false>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM_R);
    if (e != cudaSuccess) return e;
    const int grid = grid_for(k, C::THREADS, C::SMEM_R, C::WARPS, a.g.ntiles);
    return q_out ? launch_pdl(k_recon_nd<ND, B, true>, grid, C::THREADS, C::SMEM_R, s, a)
                 : launch_pdl(k_recon_nd<ND, B, false>, grid, C::THREADS, C::SMEM_R, s, a);
}

template <int ND, int B>
cudaError_t launch_nd_recon_batch(const ReconArgs* fields, const uint64_t* tile_prefix, int nfields,
                                  uint64_t total_tiles, unsigned long long* ticket, LaunchShape sh, cudaStream_t s,
                                  int* occ) {
    using C = NdCfg<ND, B>;
    const void* k = (const void*)k_recon_nd_batch<ND, B>;
    const int warps = sh.warps > 0 ? sh.warps : C::WARPS;
    if (warps * 32 > NdBatchBounds<ND, B>::MAXT) {
        if (occ) *occ = 0;
        return occ ? cudaSuccess : cudaErrorInvalidValue;
    }
    const size_t smem = C::WARP_R * (size_t)warps;
    cudaError_t e = raise_smem_attr(k, smem);
    if (occ) {
        *occ = e == cudaSuccess ? occupancy(k, warps * 32, smem) : 0;
        return cudaSuccess;
    }
    if (e != cudaSuccess) return e;
    const int grid = grid_shape(k, warps * 32, smem, (uint64_t)warps, total_tiles, sh.ctas);
    k_recon_nd_batch<ND, B><<<grid, warps * 32, smem, s>>>(fields, tile_prefix, nfields, ticket);
    return cudaGetLastError();
}

}  // namespace vsz
