// compress_nd.cuh -- fused prequant + blockwise Lorenzo + post-quant + guard
// for 2D and 3D fields (Sec. III-A, Alg. 2; padding Sec. IV).
//
// One warp owns one tile: a 128-column segment along x of one row of blocks
// (2D: b rows; 3D: b*b rows, z outer, y inner).  Lane l owns columns
// 4l..4l+3, so b/4 consecutive lanes cover one block along x.  Rows arrive in
// batches of U = min(b, 4) rows of one plane through an NS-stage lane-private
// cp.async ring in shared memory (each lane copies and reads only its own 16
// bytes per row, so one cp.async group per batch is all the synchronization
// needed; NS - 1 batches are in flight while one is processed).  Walking the rows in order, the first-order
// Lorenzo residual is the mixed difference delta = Dz Dy Dx q, where a
// difference at a block's low face is the identity: the neighbour outside
// the block is the padding value P, which cancels everywhere except at the
// block origin, delta_origin = q - P:
//   Dx: within the lane, and from lane l-1 by shuffle;
//   Dy: against the previous row's Dx result (registers, zeroed per plane);
//   Dz: against the previous plane's Dy result at the same row, kept in
//       lane-private shared memory (zeroed per tile).
// Two exact arithmetic modes compute the same integers.  While every
// |x * inv2eb| of a batch is below 2^20 (proved for the whole field by the
// range pass of relative mode, else checked per batch; NaN fails both
// checks), rounding, differences, the code and the guard run on the fp32
// pipe: the rounded values are integers below 2^20 and every difference an
// integer below 2^24, so each fp32 operation is exact.  Otherwise the tile
// continues in int32 (wrapping) arithmetic, its carried state converted.
// The fp32 mode's code is the low half of fl(d + R + 2^23), which is d + R
// when |d| < R; the lean walk of interior tiles stores it with the
// outliers' codes already zeroed (a select on |d| < R), the general walk
// stores it raw and rewrites the codes of flagged rows that hold an outlier.
// Every input byte is read once from HBM and every code written once.
//
// The pass over a batch is branch-free: each row's residuals go to a
// lane-private history and two flag bits per row mark rows that may hold an
// outlier or a fixup.  After the batch, flagged rows are re-examined exactly
// (the guard only for rows flagged for it).  Inside one block the walk order
// is the canonical order (blocks in row-major order, row-major inside a
// block), so:
//  - with block-slot staging (a workspace of vsz_workspace_size_dense), each
//    outlier goes straight to its block's slot at 1 + its rank in the block
//    (a scan over the block's b/4 lanes); fixups go to a per-warp stash;
//  - otherwise outliers and fixups both go to the stash (walk order).
// At the end of the tile one atomic reserves the tile's staging range of
// what the stash holds, and the stash is scattered into canonical order with
// a counting sort keyed by block.  A tile whose stash overflows counts only
// from then on and is walked a second time (int32 arithmetic, no code
// stores, no guard when the tile has no fixup), which writes each stashed
// kind straight to its canonical place from per-block running ranks.  Tiles
// are handed out by an atomic ticket, so warps that finish early take more.
#pragma once

#include <climits>

#include "common.cuh"
#include "memops.cuh"
#include "ring.cuh"

// Tile-shape knobs (compile time): rows per batch, warps per CTA, the
// resident CTAs per SM that the register allocation must allow, and the
// stash entries per warp.
#ifndef VSZ_ND_ROWS
#define VSZ_ND_ROWS 4
#endif
#ifndef VSZ_ND_WARPS
#define VSZ_ND_WARPS 4
#endif
#ifndef VSZ_ND_MINB_C
#define VSZ_ND_MINB_C 4
#endif
#ifndef VSZ_ND_MINB_R
#define VSZ_ND_MINB_R 5
#endif
#ifndef VSZ_ND_STASH
#define VSZ_ND_STASH 256
#endif
#ifndef VSZ_ND_STAGES
#define VSZ_ND_STAGES 2
#endif
#ifndef VSZ_ND_STASH3_8
#define VSZ_ND_STASH3_8 384
#endif
#ifndef VSZ_ND_STAGES_R
#define VSZ_ND_STAGES_R 6
#endif

namespace vsz {

template <int ND, int B>
struct NdCfg {
    static_assert(B >= 4 && B <= 128 && (B & (B - 1)) == 0, "block edge");
    static constexpr int G = B / 4;                               // lanes per block along x
    static constexpr int U = B < VSZ_ND_ROWS ? B : VSZ_ND_ROWS;   // rows per batch
    static constexpr bool ZSMEM = (ND == 3);                      // z state in shared memory
    static constexpr int WARPS = VSZ_ND_WARPS;
    static constexpr int THREADS = WARPS * 32;
    static constexpr int MINB_C = ZSMEM && B >= 32 ? 2 : VSZ_ND_MINB_C;  // caps registers
    static constexpr int MINB_R = VSZ_ND_MINB_R;
    // stash entries per warp: a 3D tile holds 8192 (b 8) or 32768 (b 16)
    // values, so those take what shared memory has left at the same
    // resident CTAs per SM (4 and 3); 2D tiles (at most 4096) keep the default
    static constexpr int STASH = (ND == 3 && B == 8) ? VSZ_ND_STASH3_8 : (ND == 3 && B == 16) ? 512 : VSZ_ND_STASH;
    static constexpr size_t ZS_B = ZSMEM ? (size_t)B * 32 * 16 : 0;
    // ring stages: the z state of 3D blocks of 32 leaves room for two
    static constexpr int NS = ZS_B > 8192 ? 2 : VSZ_ND_STAGES;
    static constexpr int NSR = ZS_B > 8192 ? 2 : VSZ_ND_STAGES_R;
    // per-warp shared memory, compression: ring | stash | tables | z state
    static constexpr size_t RING_C = (size_t)NS * U * 32 * 16;
    static constexpr size_t STASH_B = (size_t)STASH * 8;
    static constexpr size_t TAB_B = 128 * 4;
    static constexpr size_t HIST_B = (size_t)U * 32 * 16;  // residuals of the current batch
    static constexpr size_t CNT_B = 2 * 32 * 4;            // per lane: outliers, fixups
    static constexpr size_t WARP_C = RING_C + STASH_B + TAB_B + ZS_B + HIST_B + CNT_B;
    static constexpr size_t SMEM_C = WARP_C * WARPS;
    // per-warp shared memory, reconstruction: ring of codes | z state | outliers of the tile
    static constexpr int OCAP = 256;
    static constexpr size_t RING_R = (size_t)NSR * U * 32 * 8;
    static constexpr size_t OC_B = (size_t)OCAP * 8;
    // the outliers' residuals of the current batch of an interior tile: 3D
    // blocks up to 8 keep them in the z-state area (their z sums are in
    // registers), every other shape in an area of its own
    static constexpr size_t PS_RAW = (size_t)U * 32 * 16;
    static constexpr size_t PS_B = (ND == 3 && B <= 8) ? 0 : PS_RAW;
    static constexpr size_t WARP_R = RING_R + ZS_B + OC_B + PS_B;
    static constexpr size_t SMEM_R = WARP_R * WARPS;
    // staging entries per block in the block-slot layout
    static constexpr uint64_t SLOT = block_slot(ND, B);
};

__device__ __forceinline__ int32_t wsub(int32_t a, int32_t b) { return (int32_t)((uint32_t)a - (uint32_t)b); }
__device__ __forceinline__ int32_t wadd(int32_t a, int32_t b) { return (int32_t)((uint32_t)a + (uint32_t)b); }

// Stash key: [31] fixup? | [30:26] block within the tile | [25:7] row | [6:0] column.
__device__ __forceinline__ uint32_t stash_key(uint32_t fix, uint32_t g, uint32_t row, uint32_t col) {
    return (fix << 31) | (g << 26) | (row << 7) | col;
}

// All the work of one tile t of one field: the walk(s), the per-block
// padding and counts, and the tile's staged outliers and fixups.  BP: a
// per-block padding mode; GP: a global padding mode, whose value is known
// only once every tile has been walked, so block origins are deferred to
// the origin pass (their q and the tile's q statistics are recorded here).
template <int ND, int B, bool BP, bool GP, bool EP = false>
__device__ __forceinline__ void nd_compress_tile(const CompressArgs& a, uint64_t t, unsigned char* wsm, int lane) {
    using C = NdCfg<ND, B>;
    constexpr int G = C::G;
    constexpr int U = C::U;
    constexpr float kSafe = 1048576.0f;     // 2^20
    constexpr float kMagic = 12582912.0f;   // 1.5 * 2^23: adding it rounds |p| < 2^22 to an integer
    uint2* stash = reinterpret_cast<uint2*>(wsm + C::RING_C);
    uint32_t* pre_out = reinterpret_cast<uint32_t*>(wsm + C::RING_C + C::STASH_B);
    uint32_t* pre_fix = pre_out + 32;
    uint32_t* run = pre_out + 64;  // 64 counters: [fix][group]
    int4* zs = reinterpret_cast<int4*>(wsm + C::RING_C + C::STASH_B + C::TAB_B);
    int4* dh = reinterpret_cast<int4*>(wsm + C::RING_C + C::STASH_B + C::TAB_B + C::ZS_B) + lane;
    // counters the rare path updates, kept in shared memory (lane-private) so
    // that they hold no register through the walk
    uint32_t* const cnt = reinterpret_cast<uint32_t*>(wsm + C::RING_C + C::STASH_B + C::TAB_B + C::ZS_B + C::HIST_B) + lane;
    cnt[0] = 0;   // outliers of this lane's columns
    cnt[32] = 0;  // fixups of this lane's columns
    const float4* ring_rd = reinterpret_cast<const float4*>(wsm) + lane;  // slot (h*U + u)*32
    const uint32_t ring_wr = smem_addr(wsm) + lane * 16;

    const Geom& g = a.g;
    const float inv2eb = a.hdr->inv2eb;
    const float ebx2 = a.hdr->ebx2;
    const float ebf = a.hdr->eb_f32;
    const int32_t Pg = a.hdr->pad_global;
    const int32_t R = a.R;
    const float Rf = (float)R;
    const float RB = (float)(R + 8388608);  // R + 2^23
    const uint64_t nx = g.nx;
    const uint64_t plane = g.ny * g.nx;
    const int glane = lane & (G - 1);
    const bool first = glane == 0;
    const int src = lane & ~(G - 1);
    const uint32_t grp = (uint32_t)(lane / G);
    const uint32_t lt = lanemask_lt();
    const bool vec = a.vec != 0;
    // the fp32 mode needs the global padding value itself to be small
    const bool pg_small = BP || GP || (Pg >= -(1 << 20) && Pg <= (1 << 20));
    const float Pgf = (float)(BP || GP ? 0 : Pg);
    // a range pass that proved every |x * inv2eb| < 2^20 (and no NaN/Inf)
    // lets the fp32 mode skip its per-batch check
    const bool fast = pg_small && a.wsh->fp32_ok != 0u;

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
    const int nbpp = (ylen + U - 1) / U;  // batches per plane
    const int nbatch = zlen * nbpp;
    const uint64_t blk = (bz * g.nby + by) * g.nbx + bx;
    const uint64_t tile_base = (ND == 3 ? bz * B * plane : 0) + by * B * nx + x0;
    const float* xsrc = a.x;
    // interior tile: b rows and (3D) b planes, every lane 4 columns or (the
    // field's last segment, nx a multiple of 4) none; a short segment takes
    // the lean walk only with zero padding, whose walk keeps no statistic
    // that lanes past the field would enter
    const bool interior = vec && ylen == B && (ND == 2 || zlen == B) &&
                          (s * kSegCols + kSegCols <= nx || (!BP && !GP && !EP));

    // copy the rows of batch (lz, j) into ring half h
    auto issue_batch = [&](int lz, int j, int h) {
        const uint64_t off0 = tile_base + (uint64_t)lz * plane + (uint64_t)(j * U) * nx;
        const uint32_t dst0 = ring_wr + (uint32_t)(h * U * 32 * 16);
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (j * U + u < ylen) {
                const uint64_t off = off0 + (uint64_t)u * nx;
                const uint32_t dst = dst0 + u * 32 * 16;
                if (vec) {
                    cp_async16(dst, valid ? xsrc + off : xsrc, valid ? 16u : 0u);
                } else {
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        cp_async4(dst + 4 * k, (k < valid) ? xsrc + off + k : xsrc, (k < valid) ? 4u : 0u);
                }
            }
        }
        cp_async_commit();
    };

    // results of the first pass that the second pass needs
    uint32_t nst = 0;
    int32_t Pb = BP || GP ? 0 : Pg;
    uint32_t eo_g = 0, ef_g = 0;
    unsigned long long base_out = 0, base_fix = 0;
    int32_t qcorner = 0;
    uint32_t r0c01 = 0, r0c23 = 0;
    int32_t smin = INT_MAX, smax = INT_MIN;
    float sminf = __int_as_float(0x7f800000), smaxf = -__int_as_float(0x7f800000);
    // an average padding needs only the sum of q
    const bool need_mm = (BP || GP) && a.pad_mode != VSZ_PAD_GLOBAL_AVG && a.pad_mode != VSZ_PAD_BLOCK_AVG;
    long long ssum = 0;
    // Edge padding (Sec. IV-B-3): the min / max / sum of q over each block's
    // faces (x: local x = 0, y: local y = 0, z: local z = 0), gathered by the
    // walk when the range pass proved the fp32 mode for the whole field (then
    // every |q| < 2^20 and a lane's face sums fit in 32 bits); otherwise the
    // face-statistics pass computes them from x.
    const bool efs = EP && fast;
    const int ekind = EP ? a.pad_mode - VSZ_PAD_EDGE_MIN : 0;  // 0 min, 1 max, 2 mean
    const int32_t eid = ekind == 0 ? INT_MAX : ekind == 1 ? INT_MIN : 0;
    int32_t efx = eid, efy = eid, efz = eid;
    auto etake = [&](int32_t& acc, int32_t v) {
        acc = ekind == 0 ? min(acc, v) : ekind == 1 ? max(acc, v) : acc + v;
    };
    // nv of a row's 4 values (exact integers below 2^20 as floats)
    auto etake_row = [&](int32_t& acc, const float (&r)[4], int nv) {
        float m = ekind == 0 ? __int_as_float(0x7f800000) : ekind == 1 ? -__int_as_float(0x7f800000) : 0.0f;
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (k < nv) m = ekind == 0 ? fminf(m, r[k]) : ekind == 1 ? fmaxf(m, r[k]) : __fadd_rn(m, r[k]);
        if (nv > 0) etake(acc, __float2int_rn(m));
    };

    // Rare path of one batch: exact masks of the flagged rows; counts and
    // stash entries (first walk) or direct canonical writes (second walk).
    // Rows of a batch stored raw by the fp32 mode get their outliers' codes
    // zeroed here.
    uint32_t run_o = 0, run_f = 0;  // running ranks inside this lane's block (second walk)
    // block slots of the staging area (2D/3D, when the workspace holds
    // them): block k's outliers at slots[k * S + 1 ...] in walk order, which
    // inside a block is the canonical order; slot 0 holds the origin of a
    // per-block padding mode
    uint2* const slots = a.slots;
    uint2* const myslot = slots ? slots + (bexists ? blk : 0) * (uint64_t)C::SLOT : nullptr;
    uint32_t seg_o = 0;             // outliers of this lane's block in its slot (first walk)
    bool ovf = false;               // the stash overflowed: count only, then walk again
    bool nofix = false;             // second walk of a tile without fixups: no guard checks
    // entries go to the staging area, which the compaction moves from
    auto put_out = [&](uint64_t pos, uint32_t idx, uint32_t d) {
        if (pos < a.out_cap) a.stage_out[pos] = make_uint2(idx, d);
    };
    auto put_fix = [&](uint64_t pos, uint32_t idx, uint32_t bits) {
        if (pos < a.fix_cap) a.stage_fix[pos] = make_uint2(idx, bits);
    };
    auto rare_rows = [&](uint32_t rows, uint32_t rows_f, int h, uint64_t boff, int j, int lz, bool b0, bool imode,
                         bool raw, bool emit) {
        while (rows) {
            const int u = __ffs(rows) - 1;
            rows &= rows - 1;
            const int ly = j * U + u;
            const int4 dv = dh[u * 32];
            int32_t d[4];
            if (imode) {
                d[0] = dv.x; d[1] = dv.y; d[2] = dv.z; d[3] = dv.w;
            } else {
                d[0] = __float2int_rn(__int_as_float(dv.x)); d[1] = __float2int_rn(__int_as_float(dv.y));
                d[2] = __float2int_rn(__int_as_float(dv.z)); d[3] = __float2int_rn(__int_as_float(dv.w));
            }
            const float4 v = ring_rd[(h * U + u) * 32];
            const float xv[4] = {v.x, v.y, v.z, v.w};
            uint32_t om = 0, fm = 0;
#pragma unroll
            for (int k = 0; k < 4; ++k) om |= (code_of(d[k], R) == 0u ? 1u : 0u) << k;
            if ((rows_f >> u) & 1u) {  // warp-uniform: some lane of this row may need a fixup
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    fm |= (needs_fixup(xv[k], prequant(xv[k], inv2eb), ebx2, ebf) ? 1u : 0u) << k;
            }
            om &= vmask;
            fm &= vmask;
            if (raw && om) {  // fp32 mode stored raw codes: zero the outliers' codes
                uint32_t c[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) c[k] = ((om >> k) & 1u) ? 0u : ((uint32_t)(d[k] + R) & 0xffffu);
                const uint32_t c01 = c[0] | (c[1] << 16), c23 = c[2] | (c[3] << 16);
                if (BP && b0 && u == 0) {
                    r0c01 = c01;
                    r0c23 = c23;
                } else {
                    if (valid == 0 || VSZ_IN(boff + (uint64_t)u * nx + valid - 1, g.n, 101))
                        store4c(a.codes + boff + (uint64_t)u * nx, valid, vst, c01, c23);
                }
            }
            if (((BP && !emit) || GP) && b0 && u == 0 && first) om &= ~1u;  // the origin waits for P
            const uint32_t co = __popc(om), cf = __popc(fm);
            if (!emit) {
                cnt[0] += co;
                cnt[32] += cf;
                if (slots && __any_sync(VSZ_FULL, om != 0u)) {
                    // outliers to the block's slot: rank among the block's lanes
                    uint32_t io = co;
#pragma unroll
                    for (int off = 1; off < G; off <<= 1) {
                        const uint32_t y = __shfl_up_sync(VSZ_FULL, io, off);
                        if (glane >= off) io += y;
                    }
                    uint32_t pos = seg_o + io - co;
                    const uint32_t idx0 = (uint32_t)(boff + (uint64_t)u * nx);
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        if (om & (1u << k)) {
                            if (VSZ_IN((uint64_t)(myslot - slots) + 1 + pos, g.nb * C::SLOT, 102))
                                myslot[1 + pos] = make_uint2(idx0 + k, (uint32_t)d[k]);
                            ++pos;
                        }
                    }
                    seg_o += __shfl_sync(VSZ_FULL, io, src + G - 1);
                }
                // the stash overflowed: the tile is walked again for what the
                // stash holds, and counts are all this walk still needs
                if (ovf) continue;
                const uint32_t oms = slots ? 0u : om;  // outliers that go to the stash
                const uint32_t cl = __popc(oms) + cf;
                if (__any_sync(VSZ_FULL, cl != 0u)) {
                    uint32_t incl = cl;
#pragma unroll
                    for (int off = 1; off < 32; off <<= 1) {
                        const uint32_t y = __shfl_up_sync(VSZ_FULL, incl, off);
                        if (lane >= off) incl += y;
                    }
                    uint32_t pos = nst + incl - cl;
                    const uint32_t total = __shfl_sync(VSZ_FULL, incl, 31);
                    if (nst + total <= (uint32_t)C::STASH) {
                        const uint32_t row = (uint32_t)(lz * ylen + ly);
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            if (oms & (1u << k))
                                stash[pos++] = make_uint2(stash_key(0, grp, row, lane * 4 + k), (uint32_t)d[k]);
                            if (fm & (1u << k))
                                stash[pos++] = make_uint2(stash_key(1, grp, row, lane * 4 + k), __float_as_uint(xv[k]));
                        }
                    }
                    nst += total;
                    ovf = ovf || nst > (uint32_t)C::STASH;
                }
            } else {
                // ranks inside the block: earlier rows, then earlier lanes of this row
                uint32_t io = co, iff = cf;
#pragma unroll
                for (int off = 1; off < G; off <<= 1) {
                    const uint32_t yo = __shfl_up_sync(VSZ_FULL, io, off);
                    const uint32_t yf = __shfl_up_sync(VSZ_FULL, iff, off);
                    if (glane >= off) { io += yo; iff += yf; }
                }
                uint64_t po = base_out + eo_g + run_o + (io - co);
                uint64_t pq = base_fix + ef_g + run_f + (iff - cf);
                const uint32_t idx0 = (uint32_t)(boff + (uint64_t)u * nx);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    if (om & (1u << k)) {  // (with block slots the first walk placed them)
                        if (!slots) put_out(po, idx0 + k, (uint32_t)d[k]);
                        ++po;
                    }
                    if (fm & (1u << k)) {
                        put_fix(pq, idx0 + k, __float_as_uint(xv[k]));
                        ++pq;
                    }
                }
                run_o += __shfl_sync(VSZ_FULL, io, src + G - 1);
                run_f += __shfl_sync(VSZ_FULL, iff, src + G - 1);
            }
        }
    };

    for (int pass = 0; pass < 2; ++pass) {
        const bool emit = pass == 1;  // second walk: write entries, no codes
        // carried state: fp32 mode uses pf / float bits in zs, int mode p1 / ints in zs
        float pf[4] = {0.f, 0.f, 0.f, 0.f};
        int32_t p1[4] = {0, 0, 0, 0};
        if (C::ZSMEM)
            for (int ly = 0; ly < ylen; ++ly) zs[ly * 32 + lane] = make_int4(0, 0, 0, 0);
        bool imode = emit || !pg_small;
        run_o = 0;
        run_f = 0;

        if (!emit && fast && interior) {
            // Lean first walk of an interior tile in fp32 mode: compile-time
            // trip counts, 32-bit offsets, no per-row bounds or mode checks.
            constexpr int BPP = B / U;                       // batches per plane
            constexpr int NB = (ND == 3 ? B : 1) * BPP;      // batches per tile
            const uint32_t nx32 = (uint32_t)nx, pl32 = (uint32_t)plane;
            // a lane past the field's last column copies nothing (zeros)
            // from the field's start: its source and size, once per tile
            const float* xl = valid ? a.x + tile_base : a.x;
            const uint32_t xsz = valid ? 16u : 0u;
            uint16_t* cl = a.codes + tile_base;
            auto off32 = [&](int kb) -> uint32_t {
                return (uint32_t)(kb / BPP) * pl32 + (uint32_t)((kb % BPP) * U) * nx32;
            };
            auto issue_fast = [&](int kb, int st) {
                const float* src0 = xl + off32(kb);
                const uint32_t dst0 = ring_wr + (uint32_t)(st * U * 32 * 16);
#pragma unroll
                for (int u = 0; u < U; ++u) cp_async16(dst0 + u * 32 * 16, src0 + (uint32_t)u * nx32, xsz);
                cp_async_commit();
            };
#pragma unroll
            for (int st = 0; st < C::NS - 1; ++st) {
                if (st < NB) issue_fast(st, st);
                else cp_async_commit();
            }
            // the padding value only enters at the tile's origin: preload it
            // into the carried difference state (3D: plane state of row 0;
            // 2D: row state)
            if (!BP && !GP && first) {
                if (ND == 3) zs[lane] = make_int4(__float_as_int(Pgf), 0, 0, 0);
                else pf[0] = Pgf;
            }
            int h = 0;
            int32_t lsum = 0;
            for (int kb = 0; kb < NB; ++kb) {
                const int jb = kb % BPP;
                if (kb + C::NS - 1 < NB) issue_fast(kb + C::NS - 1, (kb + C::NS - 1) % C::NS);
                else cp_async_commit();
                cp_async_wait<C::NS - 1>();
                if (ND == 3 && jb == 0) {
#pragma unroll
                    for (int k = 0; k < 4; ++k) pf[k] = 0.f;
                }
                const float4* rr = ring_rd + h * U * 32;
                uint16_t* crow = cl + off32(kb);
                int4* zrow = zs + jb * U * 32 + lane;
                uint32_t fmask = 0;
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const float4 v = rr[u * 32];
                    const float xv[4] = {v.x, v.y, v.z, v.w};
                    float rp[4], d[4];
#pragma unroll
                    for (int k = 0; k < 4; ++k) rp[k] = __fsub_rn(__fadd_rn(__fmul_rn(xv[k], inv2eb), kMagic), kMagic);
                    float left = __shfl_up_sync(VSZ_FULL, rp[3], 1);
                    if (first) left = 0.f;
                    d[0] = __fsub_rn(rp[0], left);
                    d[1] = __fsub_rn(rp[1], rp[0]);
                    d[2] = __fsub_rn(rp[2], rp[1]);
                    d[3] = __fsub_rn(rp[3], rp[2]);
#pragma unroll
                    for (int k = 0; k < 4; ++k) {  // Dy
                        const float r1 = d[k];
                        d[k] = __fsub_rn(r1, pf[k]);
                        pf[k] = r1;
                    }
                    if (ND == 3) {  // Dz
                        const int4 pv = zrow[u * 32];
                        zrow[u * 32] = make_int4(__float_as_int(d[0]), __float_as_int(d[1]), __float_as_int(d[2]),
                                                 __float_as_int(d[3]));
                        d[0] = __fsub_rn(d[0], __int_as_float(pv.x)); d[1] = __fsub_rn(d[1], __int_as_float(pv.y));
                        d[2] = __fsub_rn(d[2], __int_as_float(pv.z)); d[3] = __fsub_rn(d[3], __int_as_float(pv.w));
                    }
                    dh[u * 32] = make_int4(__float_as_int(d[0]), __float_as_int(d[1]), __float_as_int(d[2]),
                                           __float_as_int(d[3]));
                    uint32_t cb[4];
                    bool fo = false, ff = false;
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        // an outlier's code is 0 from the first store on
                        const bool in = fabsf(d[k]) < Rf;
                        cb[k] = in ? __float_as_uint(__fadd_rn(d[k], RB)) : 0u;
                        const float xh = __fmul_rn(rp[k], ebx2);
                        fo |= !in;
                        ff |= !(fabsf(__fsub_rn(xv[k], xh)) <= ebf);
                    }
                    if (EP && efs) {
                        if (first) etake(efx, __float2int_rn(rp[0]));    // local x = 0: every row
                        if (jb == 0 && u == 0) etake_row(efy, rp, 4);    // local y = 0
                        if (ND == 3 && kb < BPP) etake_row(efz, rp, 4);  // local z = 0: the first plane
                    }
                    if (BP || (GP && !EP)) {
                        if (need_mm) {
                            sminf = fminf(sminf, fminf(fminf(rp[0], rp[1]), fminf(rp[2], rp[3])));
                            smaxf = fmaxf(smaxf, fmaxf(fmaxf(rp[0], rp[1]), fmaxf(rp[2], rp[3])));
                        }
                        // the row sum is an integer below 2^22: exact in fp32, converted by the
                        // 1.5 * 2^23 bias; a batch's sum stays below 2^24
                        const float rs = __fadd_rn(__fadd_rn(__fadd_rn(rp[0], rp[1]), rp[2]), rp[3]);
                        lsum += __float_as_int(__fadd_rn(rs, kMagic)) - 0x4B400000;
                    }
                    fmask |= (fo ? (1u << u) : 0u) | (ff ? (0x100u << u) : 0u);
                    const uint32_t c01 = __byte_perm(cb[0], cb[1], 0x5410), c23 = __byte_perm(cb[2], cb[3], 0x5410);
                    if (BP && u == 0 && kb == 0) {
                        r0c01 = c01;
                        r0c23 = c23;
                    }
                    if (valid && VSZ_IN(tile_base + off32(kb) + (uint64_t)u * nx + 3, g.n, 103))
                        *reinterpret_cast<uint2*>(crow + (uint32_t)u * nx32) = make_uint2(c01, c23);
                }
                if ((BP || GP) && kb == 0) qcorner = __float2int_rn(__int_as_float(dh[0].x));
                const uint32_t rows = __reduce_or_sync(VSZ_FULL, valid ? fmask : 0u);
                if (rows)  // codes already final: no rewrite
                    rare_rows((rows | (rows >> 8)) & 0xffu, rows >> 8, h, tile_base + off32(kb), jb, kb / BPP, kb == 0,
                              false, false, false);
                h = h + 1 == C::NS ? 0 : h + 1;
                if (BP || (GP && !EP)) {
                    ssum += lsum;
                    lsum = 0;
                }
            }
        } else {
        // NS-stage ring: batches kb+1 .. kb+NS-1 are in flight while batch kb is processed
        int ilz = 0, ij = 0;  // next batch to issue
#pragma unroll
        for (int st = 0; st < C::NS - 1; ++st) {
            if (st < nbatch) {
                issue_batch(ilz, ij, st);
                if (++ij == nbpp) { ij = 0; ++ilz; }
            } else {
                cp_async_commit();
            }
        }
        int lz = 0, j = 0, h = 0, hi = C::NS - 1;
        for (int kb = 0; kb < nbatch; ++kb) {
            int nj = j + 1, nlz = lz;
            if (nj == nbpp) { nj = 0; ++nlz; }
            if (kb + C::NS - 1 < nbatch) {
                issue_batch(ilz, ij, hi);
                if (++ij == nbpp) { ij = 0; ++ilz; }
            } else {
                cp_async_commit();
            }
            cp_async_wait<C::NS - 1>();
            if (j == 0) {
#pragma unroll
                for (int k = 0; k < 4; ++k) { pf[k] = 0.f; p1[k] = 0; }
            }
            const uint64_t boff = tile_base + (uint64_t)lz * plane + (uint64_t)(j * U) * nx;
            const bool b0 = kb == 0;
            float xr[U][4], pr[U][4];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const float4 v = (j * U + u < ylen) ? ring_rd[(h * U + u) * 32] : make_float4(0.f, 0.f, 0.f, 0.f);
                xr[u][0] = v.x; xr[u][1] = v.y; xr[u][2] = v.z; xr[u][3] = v.w;
#pragma unroll
                for (int k = 0; k < 4; ++k) pr[u][k] = __fmul_rn(xr[u][k], inv2eb);
            }
            bool unsafe = false;
            if (!imode && !fast) {
                // |p0|+|p1|+|p2|+|p3| < 2^20 bounds every |p| (NaN fails it)
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const float sa = __fadd_rn(__fadd_rn(fabsf(pr[u][0]), fabsf(pr[u][1])),
                                               __fadd_rn(fabsf(pr[u][2]), fabsf(pr[u][3])));
                    unsafe |= !(sa < kSafe);
                }
                unsafe = __any_sync(VSZ_FULL, unsafe);
            }
            const bool raw = !imode && !unsafe;  // codes of this batch stored raw, outliers fixed below
            if (unsafe) {
                // switch this tile to int32 arithmetic; the carried state is exact
                imode = true;
#pragma unroll
                for (int k = 0; k < 4; ++k) p1[k] = __float2int_rn(pf[k]);
                if (C::ZSMEM)
                    for (int ly = 0; ly < ylen; ++ly) {
                        const int4 w = zs[ly * 32 + lane];
                        zs[ly * 32 + lane] = make_int4(__float2int_rn(__int_as_float(w.x)), __float2int_rn(__int_as_float(w.y)),
                                                       __float2int_rn(__int_as_float(w.z)), __float2int_rn(__int_as_float(w.w)));
                    }
            }
            // Branch-free pass over the batch: codes out, residuals to the
            // history, one flag bit per row that may hold an outlier or fixup.
            uint32_t fmask = 0;
            if (!imode) {
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int ly = j * U + u;
                    if (ly >= ylen) break;
                    float rp[4], d[4];
#pragma unroll
                    for (int k = 0; k < 4; ++k) rp[k] = __fsub_rn(__fadd_rn(pr[u][k], kMagic), kMagic);
                    float left = __shfl_up_sync(VSZ_FULL, rp[3], 1);
                    if (first) left = 0.f;
                    d[0] = __fsub_rn(rp[0], left);
                    d[1] = __fsub_rn(rp[1], rp[0]);
                    d[2] = __fsub_rn(rp[2], rp[1]);
                    d[3] = __fsub_rn(rp[3], rp[2]);
#pragma unroll
                    for (int k = 0; k < 4; ++k) {  // Dy
                        const float r1 = d[k];
                        d[k] = __fsub_rn(r1, pf[k]);
                        pf[k] = r1;
                    }
                    if (C::ZSMEM) {  // Dz
                        int4& st = zs[ly * 32 + lane];
                        const int4 pv = st;
                        st = make_int4(__float_as_int(d[0]), __float_as_int(d[1]), __float_as_int(d[2]), __float_as_int(d[3]));
                        d[0] = __fsub_rn(d[0], __int_as_float(pv.x)); d[1] = __fsub_rn(d[1], __int_as_float(pv.y));
                        d[2] = __fsub_rn(d[2], __int_as_float(pv.z)); d[3] = __fsub_rn(d[3], __int_as_float(pv.w));
                    }
                    if (u == 0 && b0 && first) {
                        if (BP || GP) qcorner = __float2int_rn(rp[0]);
                        else d[0] = __fsub_rn(d[0], Pgf);
                    }
                    dh[u * 32] = make_int4(__float_as_int(d[0]), __float_as_int(d[1]), __float_as_int(d[2]), __float_as_int(d[3]));
                    // raw codes: the low 16 bits of fl(d + R + 2^23) are d + R
                    // whenever |d| < R; outlier rows are rewritten below
                    uint32_t cb[4];
                    bool fo = false, ff = false;
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        cb[k] = __float_as_uint(__fadd_rn(d[k], RB));
                        const float xh = __fmul_rn(rp[k], ebx2);
                        fo |= !(fabsf(d[k]) < Rf);
                        ff |= !(fabsf(__fsub_rn(xr[u][k], xh)) <= ebf);
                    }
                    if (EP && efs && valid > 0) {
                        if (first) etake(efx, __float2int_rn(rp[0]));
                        if (ly == 0) etake_row(efy, rp, valid);
                        if (ND == 3 && lz == 0) etake_row(efz, rp, valid);
                    }
                    if (BP || (GP && !EP)) {
                        float rs = 0.f;
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            if (k < valid) {
                                sminf = fminf(sminf, rp[k]);
                                smaxf = fmaxf(smaxf, rp[k]);
                            }
                            rs = __fadd_rn(rs, rp[k]);  // zero-filled past the edge; exact below 2^22
                        }
                        ssum += __float2int_rn(rs);
                    }
                    fmask |= (fo ? (1u << u) : 0u) | (ff ? (0x100u << u) : 0u);
                    const uint32_t c01 = __byte_perm(cb[0], cb[1], 0x5410), c23 = __byte_perm(cb[2], cb[3], 0x5410);
                    if (BP && b0 && u == 0) {
                        r0c01 = c01;
                        r0c23 = c23;
                    } else if (valid == 0 || VSZ_IN(boff + (uint64_t)u * nx + valid - 1, g.n, 109)) {
                        store4c(a.codes + boff + (uint64_t)u * nx, valid, vst, c01, c23);
                    }
                }
            } else {
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int ly = j * U + u;
                    if (ly >= ylen) break;
                    int32_t q[4];
#pragma unroll
                    for (int k = 0; k < 4; ++k) q[k] = prequant(xr[u][k], inv2eb);
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
                        d[k] = wsub(r1, p1[k]);
                        p1[k] = r1;
                    }
                    if (C::ZSMEM) {  // Dz
                        int4& st = zs[ly * 32 + lane];
                        const int4 pv = st;
                        st = make_int4(d[0], d[1], d[2], d[3]);
                        d[0] = wsub(d[0], pv.x); d[1] = wsub(d[1], pv.y);
                        d[2] = wsub(d[2], pv.z); d[3] = wsub(d[3], pv.w);
                    }
                    if (u == 0 && b0 && first) {
                        if ((BP || GP) && !emit) qcorner = q[0];
                        else d[0] = wsub(d[0], Pb);
                    }
                    dh[u * 32] = make_int4(d[0], d[1], d[2], d[3]);
                    uint32_t c[4];
                    bool fo = false, ff = false;
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        c[k] = code_of(d[k], R);
                        fo |= c[k] == 0u;
                        if (!nofix) ff |= needs_fixup(xr[u][k], q[k], ebx2, ebf);
                        if ((BP || (GP && !EP)) && !emit && k < valid) {
                            smin = min(smin, q[k]);
                            smax = max(smax, q[k]);
                            ssum += q[k];
                        }
                    }
                    fmask |= (fo ? (1u << u) : 0u) | (ff ? (0x100u << u) : 0u);
                    if (!emit) {
                        const uint32_t c01 = c[0] | (c[1] << 16), c23 = c[2] | (c[3] << 16);
                        if (BP && b0 && u == 0) {
                            r0c01 = c01;
                            r0c23 = c23;
                        } else if (valid == 0 || VSZ_IN(boff + (uint64_t)u * nx + valid - 1, g.n, 110)) {
                            store4c(a.codes + boff + (uint64_t)u * nx, valid, vst, c01, c23);
                        }
                    }
                }
            }
            // Rare path: rows that may hold an outlier or a fixup.
            const uint32_t rows = __reduce_or_sync(VSZ_FULL, valid ? fmask : 0u);
            if (rows) rare_rows((rows | (rows >> 8)) & 0xffu, rows >> 8, h, boff, j, lz, b0, imode, raw, emit);
            h = h + 1 == C::NS ? 0 : h + 1;
            hi = hi + 1 == C::NS ? 0 : hi + 1;
            lz = nlz;
            j = nj;
        }
        }
        cp_async_wait<0>();
        if (emit) break;

        // Per-block padding value (Sec. IV-B-2) and the deferred block origin.
        uint32_t corner_out = 0;
        int32_t dcorner = 0;
        if (BP) {
            // fp32-mode extremes are exact integers; +-inf saturate to the identities
            smin = min(smin, __float2int_rn(sminf));
            smax = max(smax, __float2int_rn(smaxf));
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
                if (VSZ_IN(blk, g.nb, 104)) a.pad[blk] = Pb;
                dcorner = wsub(qcorner, Pb);
                const uint32_t cc = code_of(dcorner, R);
                corner_out = (cc == 0u) ? 1u : 0u;
                cnt[0] += corner_out;
                r0c01 = (r0c01 & 0xffff0000u) | cc;
                // block slots: slot 0 holds the origin outlier, or a marker
                // index that no element has
                if (slots && VSZ_IN(blk, g.nb, 105)) myslot[0] = corner_out ? make_uint2((uint32_t)tile_base, (uint32_t)dcorner)
                                                  : make_uint2(0xffffffffu, 0u);
            }
            if (valid == 0 || VSZ_IN(tile_base + valid - 1, g.n, 106)) store4c(a.codes + tile_base, valid, vst, r0c01, r0c23);
        }

        if (GP && !EP) {
            // the tile's q statistics for the global padding value
            smin = min(smin, __float2int_rn(sminf));
            smax = max(smax, __float2int_rn(smaxf));
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                smin = min(smin, __shfl_xor_sync(VSZ_FULL, smin, off));
                smax = max(smax, __shfl_xor_sync(VSZ_FULL, smax, off));
                ssum += __shfl_xor_sync(VSZ_FULL, ssum, off);
            }
            if (lane == 0) global_stats_add(a, smin, smax, ssum);
        }
        // the block origins wait for the padding value in the origin table
        if (GP && first && bexists && VSZ_IN(blk, g.nb, 107)) a.origin[blk] = qcorner;
        if (EP && efs) {
            // each block's face scalars: its G lanes reduced, then the
            // minimum, maximum or rounded mean (counts of in-field elements)
#pragma unroll
            for (int off = 1; off < G; off <<= 1) {
                etake(efx, __shfl_xor_sync(VSZ_FULL, efx, off));
                etake(efy, __shfl_xor_sync(VSZ_FULL, efy, off));
                if (ND == 3) etake(efz, __shfl_xor_sync(VSZ_FULL, efz, off));
            }
            if (first && bexists && VSZ_IN(blk * ND + ND - 1, g.nb * ND, 112)) {
                const long long xl = (long long)umin64(B, nx - bx * B), yl = ylen, zl = zlen;
                auto fin = [&](int32_t acc, long long cnt) {
                    return ekind == 2 ? rounded_mean((long long)acc, cnt) : acc;
                };
                int32_t* pd = a.pad + blk * ND;
                if (ND == 3) {
                    pd[0] = fin(efz, yl * xl);
                    pd[1] = fin(efy, zl * xl);
                    pd[2] = fin(efx, zl * yl);
                } else {
                    pd[0] = fin(efy, xl);
                    pd[1] = fin(efx, yl);
                }
            }
        }

        // Per-block counts, in-tile exclusive offsets (blk_off), tile totals.
        uint32_t bo = cnt[0], bf = cnt[32];
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
        eo_g = __shfl_sync(VSZ_FULL, eo, src);
        ef_g = __shfl_sync(VSZ_FULL, ef, src);
        const uint32_t tot_out = __shfl_sync(VSZ_FULL, io, 31);
        const uint32_t tot_fix = __shfl_sync(VSZ_FULL, iff, 31);
        if (first && bexists && VSZ_IN(blk, g.nb + 1, 108)) a.blk_in[blk] = eo;

        if (tot_out | tot_fix) {
            if (lane == 0) {
                if (tot_out && !slots) base_out = atomicAdd(&a.wsh->stage_out, (unsigned long long)tot_out);
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
        if (!(tot_out | tot_fix)) break;
        nofix = tot_fix == 0u;
        if (ovf) continue;  // stash or segment overflow: second walk

        // Counting sort of the stash into canonical order.
        if (first) {
            pre_out[grp] = (uint32_t)base_out + eo + corner_out;
            pre_fix[grp] = (uint32_t)base_fix + ef;
            if (BP && corner_out && !slots) put_out(base_out + eo, (uint32_t)tile_base, (uint32_t)dcorner);
        }
        run[lane] = 0;
        run[lane + 32] = 0;
        __syncwarp();
        const uint64_t row_base = (ND == 3 ? bz * B * plane : 0) + by * B * nx + s * kSegCols;
        for (uint32_t j0 = 0; j0 < nst; j0 += 32) {
            const uint32_t jj = j0 + lane;
            const bool act = jj < nst;
            const uint2 e = act ? stash[jj] : make_uint2(0, 0);
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
                if (isfix) put_fix(pos, idx, e.y);
                else put_out(pos, idx, e.y);
            }
            __syncwarp();
            if (act && (peers >> lane) == 1u) run[bucket] = cnt0 + rank + 1;  // last peer updates
            __syncwarp();
        }
        break;
    }
    __syncwarp();
}

// One field: tiles handed out by the field's own ticket.
template <int ND, int B, bool BP, bool GP, bool EP = false>
__global__ void __launch_bounds__(NdCfg<ND, B>::THREADS, NdCfg<ND, B>::MINB_C)
k_lorenzo_nd(const CompressArgs a) {
    pdl_prologue();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    unsigned char* wsm = smem_raw + (size_t)(threadIdx.x >> 5) * NdCfg<ND, B>::WARP_C;
    for (;;) {
        unsigned long long tk = 0;
        if (lane == 0) tk = atomicAdd(&a.wsh->ticket, 1ull);
        const uint64_t t = __shfl_sync(VSZ_FULL, tk, 0);
        if (t >= a.g.ntiles) break;
        nd_compress_tile<ND, B, BP, GP, EP>(a, t, wsm, lane);
    }
}

// Block-size bounds of the batch kernels: up to 8 warps per CTA, chosen at
// launch, under the register cap of the one-field kernel (the same threads
// per SM times registers per thread).
template <int ND, int B>
struct NdBatchBounds {
    static constexpr int MAXT = 256;
    static constexpr int PER_SM = NdCfg<ND, B>::THREADS * NdCfg<ND, B>::MINB_C;
    static constexpr int MINB = PER_SM / MAXT > 0 ? PER_SM / MAXT : 1;
    static constexpr int MINB_R = NdCfg<ND, B>::THREADS * NdCfg<ND, B>::MINB_R / MAXT > 0
                                      ? NdCfg<ND, B>::THREADS * NdCfg<ND, B>::MINB_R / MAXT : 1;
};

// Many fields of one class (rank, block edge, padding kind): one queue over
// the tiles of all of them.  tile_prefix[f] is the first global tile of field
// f, tile_prefix[nfields] the total.  Any warps per CTA up to 8.
template <int ND, int B, bool BP, bool GP, bool EP = false>
__global__ void __launch_bounds__(NdBatchBounds<ND, B>::MAXT, NdBatchBounds<ND, B>::MINB)
k_lorenzo_nd_batch(const CompressArgs* __restrict__ fields, const uint64_t* __restrict__ tile_prefix, int nfields,
                   unsigned long long* ticket) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    unsigned char* wsm = smem_raw + (size_t)(threadIdx.x >> 5) * NdCfg<ND, B>::WARP_C;
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
        nd_compress_tile<ND, B, BP, GP, EP>(fields[lo], gt - tile_prefix[lo], wsm, lane);
    }
}

}  // namespace vsz
