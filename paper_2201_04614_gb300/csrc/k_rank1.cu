// k_rank1.cu -- 1D dual-quant: fused compression and the inverse.
//
// A warp-tile is a chunk of 4096 consecutive elements processed in steps of
// 32*EPL elements (each lane owns EPL consecutive values: 4, or 8 for b=256).
// The step width is a multiple of the block length b, so every block lies
// inside one step and a step needs nothing from its neighbours: the 1D
// Lorenzo residual is q[i] - q[i-1] inside a block and q - P at its first
// element (Sec. III-A), and the inverse is a segmented inclusive prefix sum
// over the b/EPL lanes of each block.
#include <climits>

#include "common.cuh"
#include "memops.cuh"

namespace vsz {

template <int B>
struct Cfg1 {
    static_assert(B >= 4 && B <= 256 && (B & (B - 1)) == 0, "block length");
    static constexpr int EPL = B >= 256 ? 8 : 4;
    static constexpr int SPAN = 32 * EPL;
    static constexpr int STEPS = kChunk1D / SPAN;
    static constexpr int G = B / EPL;  // lanes per block
    static constexpr int WARPS = 8;
};

__device__ __forceinline__ int32_t wsub1(int32_t a, int32_t b) { return (int32_t)((uint32_t)a - (uint32_t)b); }

template <int EPL>
__device__ __forceinline__ void load_epl(const float* __restrict__ p, int valid, bool vec, float (&v)[EPL]) {
    if (vec) {
#pragma unroll
        for (int h = 0; h < EPL / 4; ++h) {
            const float4 f = ld_stream_f4(p + 4 * h);
            v[4 * h + 0] = f.x; v[4 * h + 1] = f.y; v[4 * h + 2] = f.z; v[4 * h + 3] = f.w;
        }
    } else {
#pragma unroll
        for (int k = 0; k < EPL; ++k) v[k] = (k < valid) ? p[k] : 0.0f;
    }
}

// One step of 32*EPL elements: prequant, padding value, residual, codes.
// GP (a global padding mode): the residual at each block origin is left as
// q itself; the origin pass settles it once the field's statistics are known.
template <int B, bool BP, bool GP>
struct Step1 {
    static constexpr int EPL = Cfg1<B>::EPL;
    static constexpr int G = Cfg1<B>::G;
    float x[EPL];
    int32_t d[EPL];
    int32_t q[EPL];
    int32_t P;
    int valid;

    __device__ __forceinline__ void run(const CompressArgs& a, uint64_t base, int lane, float inv2eb, int32_t Pg) {
        const uint64_t n = a.g.n;
        valid = base < n ? (int)umin64(EPL, n - base) : 0;
        load_epl<EPL>(a.x + base, valid, a.vec && valid == EPL, x);
#pragma unroll
        for (int k = 0; k < EPL; ++k) q[k] = prequant(x[k], inv2eb);
        const int glane = lane & (G - 1);
        P = GP ? 0 : Pg;
        if (BP) {
            int32_t smin = INT_MAX, smax = INT_MIN;
            long long ssum = 0;
#pragma unroll
            for (int k = 0; k < EPL; ++k)
                if (k < valid) { smin = min(smin, q[k]); smax = max(smax, q[k]); ssum += q[k]; }
#pragma unroll
            for (int off = 1; off < G; off <<= 1) {
                smin = min(smin, __shfl_xor_sync(VSZ_FULL, smin, off));
                smax = max(smax, __shfl_xor_sync(VSZ_FULL, smax, off));
                ssum += __shfl_xor_sync(VSZ_FULL, ssum, off);
            }
            const uint64_t bstart = base - (uint64_t)glane * EPL;
            const long long m = bstart < n ? (long long)umin64(B, n - bstart) : 1;
            P = a.pad_mode == VSZ_PAD_BLOCK_MIN ? smin
              : a.pad_mode == VSZ_PAD_BLOCK_MAX ? smax
              : rounded_mean(ssum, m);
        }
        const int32_t left = __shfl_up_sync(VSZ_FULL, q[EPL - 1], 1);
        d[0] = wsub1(q[0], glane == 0 ? P : left);
#pragma unroll
        for (int k = 1; k < EPL; ++k) d[k] = wsub1(q[k], q[k - 1]);
    }
};

// Outliers a warp keeps in shared memory while it walks a tile, in linear
// (= canonical) order; a tile with more, or with a step that needs the
// integer path, writes its lists by walking its steps with entries again.
constexpr int kStash1 = 512;
constexpr int kStash1F = 128;  // fixups (rounding at the quantization boundaries)

// All the work of one 4096-element tile t of a 1D field.
template <int B, bool BP, bool GP>
__device__ __forceinline__ void compress_1d_tile(const CompressArgs& a, uint64_t t, int lane,
                                                 uint2* __restrict__ stash, uint2* __restrict__ fstash,
                                                 int2* __restrict__ mm) {
    using C = Cfg1<B>;
    constexpr int EPL = C::EPL, G = C::G, SPAN = C::SPAN;
    const float inv2eb = a.hdr->inv2eb;
    const float ebx2 = a.hdr->ebx2;
    const float ebf = a.hdr->eb_f32;
    const int32_t Pg = a.hdr->pad_global;
    const int32_t R = a.R;
    const uint64_t n = a.g.n;
    const int glane = lane & (G - 1);
    const uint64_t start = t * kChunk1D;
    uint32_t run_out = 0, run_fix = 0, stepmask = 0;
    uint32_t nst = 0;   // outliers met by fp32 steps (stashed while they fit)
    uint32_t nfst = 0;  // fixups met by fp32 steps (stashed while they fit)
    bool slow = false;  // a step took the integer path
    int32_t gsum = 0;  // a lane's sum of q over the tile's fp32 steps: at most 128 values of |q| < 2^20
    // The value-range pass proved every |x * inv2eb| < 2^20 and no NaN/Inf:
    // full steps then run in exact fp32 -- rounding by the 1.5 * 2^23 bias,
    // differences of integers below 2^21, the code as the low half of
    // d + R + 2^23 -- with the outliers' codes zeroed and the outliers kept
    // in the warp's stash; only steps whose warp holds a fixup take the
    // integer path below.
    constexpr float kMagic = 12582912.0f;
    const bool fast = a.wsh->fp32_ok != 0u && a.vec != 0 && (BP || GP || (Pg >= -(1 << 20) && Pg <= (1 << 20)));
    const float Rf = (float)R, RB = (float)(R + 8388608), Pgf = (float)Pg;
    const bool need_mm = GP && a.pad_mode != VSZ_PAD_GLOBAL_AVG;
    if (need_mm) mm[lane] = make_int2(INT_MAX, INT_MIN);  // q extremes of the tile (global min or max)
    // The next full step's values are loaded before this step's work, so a
    // warp keeps two steps of loads in flight (the code stores in between
    // would otherwise hold the next loads back: the compiler cannot prove
    // that they do not alias the input).  Whenever a step takes the fp32
    // path, xn holds its values: the step before it was full too, and loaded it.
    float xn[EPL];
    if (fast && start + SPAN <= n) load_epl<EPL>(a.x + start + (uint64_t)lane * EPL, EPL, true, xn);
#pragma unroll 1
    for (int st = 0; st < C::STEPS; ++st) {
        const uint64_t s0 = start + (uint64_t)st * SPAN;
        if (s0 >= n) break;
        const uint64_t base = s0 + (uint64_t)lane * EPL;
        if (fast && s0 + SPAN <= n) {
            float xv[EPL], rp[EPL];
#pragma unroll
            for (int k = 0; k < EPL; ++k) xv[k] = xn[k];
            if (st + 1 < C::STEPS && s0 + 2 * SPAN <= n) load_epl<EPL>(a.x + base + SPAN, EPL, true, xn);
#pragma unroll
            for (int k = 0; k < EPL; ++k) rp[k] = __fsub_rn(__fadd_rn(__fmul_rn(xv[k], inv2eb), kMagic), kMagic);
            const bool origin = glane == 0;  // this lane's first value opens a block
            float Pf = GP ? 0.0f : Pgf;
            int32_t Pb = 0;
            if (BP) {  // block statistic over the block's G lanes (full step: whole blocks)
                float mn = rp[0], mx = rp[0], ls = rp[0];
#pragma unroll
                for (int k = 1; k < EPL; ++k) {
                    mn = fminf(mn, rp[k]);
                    mx = fmaxf(mx, rp[k]);
                    ls = __fadd_rn(ls, rp[k]);  // |sum| < 2^23: exact
                }
                int32_t smin = __float2int_rn(mn), smax = __float2int_rn(mx);
                int32_t ssum = __float2int_rn(ls);  // at most 256 values of |q| < 2^20
#pragma unroll
                for (int off = 1; off < G; off <<= 1) {
                    smin = min(smin, __shfl_xor_sync(VSZ_FULL, smin, off));
                    smax = max(smax, __shfl_xor_sync(VSZ_FULL, smax, off));
                    ssum += __shfl_xor_sync(VSZ_FULL, ssum, off);
                }
                Pb = a.pad_mode == VSZ_PAD_BLOCK_MIN ? smin : a.pad_mode == VSZ_PAD_BLOCK_MAX ? smax
                                                                : rounded_mean((long long)ssum, (long long)B);
                Pf = (float)Pb;  // |Pb| < 2^20: exact
            }
            const float left = __shfl_up_sync(VSZ_FULL, rp[EPL - 1], 1);
            float d[EPL];
            d[0] = __fsub_rn(rp[0], origin ? Pf : left);
#pragma unroll
            for (int k = 1; k < EPL; ++k) d[k] = __fsub_rn(rp[k], rp[k - 1]);
            uint32_t cb[EPL];
            uint32_t om = 0, fm = 0;
#pragma unroll
            for (int k = 0; k < EPL; ++k) {
                cb[k] = __float_as_uint(__fadd_rn(d[k], RB)) & 0xffffu;
                // an outlier (the origin of a global padding mode waits for the origin pass)
                const bool out = !(fabsf(d[k]) < Rf) && !(GP && k == 0 && origin);
                om |= out ? (1u << k) : 0u;
                fm |= !(fabsf(__fsub_rn(xv[k], __fmul_rn(rp[k], ebx2))) <= ebf) ? (1u << k) : 0u;
            }
            {
                if (__any_sync(VSZ_FULL, fm != 0u)) {
                    // fixups (no NaN or Inf here: rounding at a quantization
                    // boundary), kept in order beside the outliers
                    const uint32_t cf = __popc(fm);
                    uint32_t iff = cf;
#pragma unroll
                    for (int off = 1; off < 32; off <<= 1) {
                        const uint32_t y = __shfl_up_sync(VSZ_FULL, iff, off);
                        if (lane >= off) iff += y;
                    }
                    uint32_t pos = nfst + iff - cf;
#pragma unroll
                    for (int k = 0; k < EPL; ++k) {
                        if (fm & (1u << k)) {
                            if (pos < (uint32_t)kStash1F) fstash[pos] = make_uint2((uint32_t)(base + k), __float_as_uint(xv[k]));
                            ++pos;
                        }
                    }
                    const uint32_t sf = __shfl_sync(VSZ_FULL, iff, 31);
                    nfst += sf;
                    run_fix += sf;
                    stepmask |= 1u << st;  // walked again if the stashes cannot serve the tile
                }
                uint32_t ex = 0, so = 0;  // outliers of earlier lanes of the step, of the step
                if (__any_sync(VSZ_FULL, om != 0u)) {
                    const uint32_t co = __popc(om);
                    uint32_t io = co;
#pragma unroll
                    for (int off = 1; off < 32; off <<= 1) {
                        const uint32_t y = __shfl_up_sync(VSZ_FULL, io, off);
                        if (lane >= off) io += y;
                    }
                    so = __shfl_sync(VSZ_FULL, io, 31);
                    ex = io - co;
                    uint32_t pos = nst + ex;
#pragma unroll
                    for (int k = 0; k < EPL; ++k) {
                        if (om & (1u << k)) {
                            cb[k] = 0u;
                            if (pos < (uint32_t)kStash1)
                                stash[pos] = make_uint2((uint32_t)(base + k), (uint32_t)__float2int_rn(d[k]));
                            ++pos;
                        }
                    }
                    nst += so;
                    stepmask |= 1u << st;  // walked again if the stash cannot serve the tile
                }
                uint16_t* cp = a.codes + base;
                if (!VSZ_IN(base + EPL - 1, n, 301)) {
                    // (bounds-checking build only) a step past the field
                } else if (EPL == 4) {
                    *reinterpret_cast<uint2*>(cp) = make_uint2(cb[0] | (cb[1] << 16), cb[2] | (cb[3 % EPL] << 16));
                } else {
                    *reinterpret_cast<uint4*>(cp) =
                        make_uint4(cb[0] | (cb[1] << 16), cb[2] | (cb[3 % EPL] << 16), cb[4 % EPL] | (cb[5 % EPL] << 16),
                                   cb[6 % EPL] | (cb[7 % EPL] << 16));
                }
                if (origin && VSZ_IN(base / B, a.g.nb, 302)) {
                    const uint64_t blk = base / B;
                    a.blk_off[blk] = run_out + ex;
                    if (BP) a.pad[blk] = Pb;
                    if (GP) a.origin[blk] = __float2int_rn(rp[0]);
                }
                run_out += so;
                if (GP) {
                    float ls = rp[0];
#pragma unroll
                    for (int k = 1; k < EPL; ++k) ls = __fadd_rn(ls, rp[k]);
                    gsum += __float2int_rn(ls);
                    if (need_mm) {  // a min or max mode: the lane's extremes in shared memory
                        float mn = rp[0], mx = rp[0];
#pragma unroll
                        for (int k = 1; k < EPL; ++k) {
                            mn = fminf(mn, rp[k]);
                            mx = fmaxf(mx, rp[k]);
                        }
                        const int2 e = mm[lane];
                        mm[lane] = make_int2(min(e.x, __float2int_rn(mn)), max(e.y, __float2int_rn(mx)));
                    }
                }
                continue;
            }
        }
        slow = true;
        Step1<B, BP, GP> S;
        S.run(a, base, lane, inv2eb, Pg);
        uint32_t co = 0, cf = 0;
        uint32_t c[EPL];
#pragma unroll
        for (int k = 0; k < EPL; ++k) {
            c[k] = code_of(S.d[k], R);
            if (k < S.valid) {
                co += (c[k] == 0u && !(GP && k == 0 && glane == 0));
                cf += needs_fixup(S.x[k], S.q[k], ebx2, ebf) ? 1u : 0u;
                if (GP && need_mm) {
                    const int2 e = mm[lane];
                    mm[lane] = make_int2(min(e.x, S.q[k]), max(e.y, S.q[k]));
                }
            }
        }
        if (GP) {  // an integer step's q are unbounded: its sum goes to the field at once
            long long ss = 0;
#pragma unroll
            for (int k = 0; k < EPL; ++k) ss += k < S.valid ? (long long)S.q[k] : 0ll;
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) ss += __shfl_xor_sync(VSZ_FULL, ss, off);
            if (lane == 0) global_stats_add(a, INT_MAX, INT_MIN, ss);
        }
        // in-step exclusive prefix of outliers -> per-block offsets
        uint32_t io = co, iff = cf;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t yo = __shfl_up_sync(VSZ_FULL, io, off);
            const uint32_t yf = __shfl_up_sync(VSZ_FULL, iff, off);
            if (lane >= off) { io += yo; iff += yf; }
        }
        const uint32_t so = __shfl_sync(VSZ_FULL, io, 31);
        const uint32_t sf = __shfl_sync(VSZ_FULL, iff, 31);
        if (glane == 0 && base < n) {
            const uint64_t blk = base / B;
            a.blk_off[blk] = run_out + (io - co);
            if (BP) a.pad[blk] = S.P;
            if (GP) a.origin[blk] = S.q[0];
        }
        run_out += so;
        run_fix += sf;
        if (so | sf) stepmask |= 1u << st;
        // codes
        uint16_t* cp = a.codes + base;
        if (a.vec && S.valid == EPL) {
            if (EPL == 4) {
                *reinterpret_cast<uint2*>(cp) = make_uint2(c[0] | (c[1] << 16), c[2] | (c[3] << 16));
            } else {
                *reinterpret_cast<uint4*>(cp) = make_uint4(c[0] | (c[1] << 16), c[2] | (c[3] << 16),
                                                           c[4 % EPL] | (c[5 % EPL] << 16),
                                                           c[6 % EPL] | (c[7 % EPL] << 16));
            }
        } else {
#pragma unroll
            for (int k = 0; k < EPL; ++k)
                if (k < S.valid) cp[k] = (uint16_t)c[k];
        }
    }

    if (GP) {
        long long gs = gsum;
        int32_t gmin = INT_MAX, gmax = INT_MIN;
        if (need_mm) {
            const int2 e = mm[lane];
            gmin = e.x;
            gmax = e.y;
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            if (need_mm) {
                gmin = min(gmin, __shfl_xor_sync(VSZ_FULL, gmin, off));
                gmax = max(gmax, __shfl_xor_sync(VSZ_FULL, gmax, off));
            }
            gs += __shfl_xor_sync(VSZ_FULL, gs, off);
        }
        if (lane == 0) global_stats_add(a, gmin, gmax, gs);
    }
    unsigned long long base_out = 0, base_fix = 0;
    if (run_out | run_fix) {
        if (lane == 0) {
            if (run_out) base_out = atomicAdd(&a.wsh->stage_out, (unsigned long long)run_out);
            if (run_fix) base_fix = atomicAdd(&a.wsh->stage_fix, (unsigned long long)run_fix);
            uint4* ch = a.chunks + t / kTilesPerChunk;
            if (run_out) atomicAdd(&ch->x, run_out);
            if (run_fix) atomicAdd(&ch->y, run_fix);
        }
        base_out = __shfl_sync(VSZ_FULL, base_out, 0);
        base_fix = __shfl_sync(VSZ_FULL, base_fix, 0);
    }
    if (lane == 0) a.tiles[t] = make_uint4((uint32_t)base_out, run_out, (uint32_t)base_fix, run_fix);
    // entries go to the staging area, which the compaction moves from
    auto put_out = [&](uint64_t pos, uint2 e) {
        if (pos < a.out_cap) a.stage_out[pos] = e;
    };
    auto put_fix = [&](uint64_t pos, uint2 e) {
        if (pos < a.fix_cap) a.stage_fix[pos] = e;
    };

    if (!slow && nst <= (uint32_t)kStash1 && nfst <= (uint32_t)kStash1F) {
        // every entry comes from an fp32 step, stashed in order
        __syncwarp();
        for (uint32_t j = lane; j < nst; j += 32) put_out(base_out + j, stash[j]);
        for (uint32_t j = lane; j < nfst; j += 32) put_fix(base_fix + j, fstash[j]);
        __syncwarp();
        return;
    }
    // Emission in linear (= canonical) order, only for steps with entries.
    uint64_t ko = base_out, kf = base_fix;
    while (stepmask) {
        const int st = __ffs(stepmask) - 1;
        stepmask &= stepmask - 1;
        const uint64_t base = start + (uint64_t)st * SPAN + (uint64_t)lane * EPL;
        Step1<B, BP, GP> S;
        S.run(a, base, lane, inv2eb, Pg);
        uint32_t mo = 0, mf = 0;  // per-element flags of this lane
#pragma unroll
        for (int k = 0; k < EPL; ++k) {
            if (k < S.valid) {
                if (code_of(S.d[k], R) == 0u && !(GP && k == 0 && glane == 0)) mo |= 1u << k;
                if (needs_fixup(S.x[k], S.q[k], ebx2, ebf)) mf |= 1u << k;
            }
        }
        uint32_t io = __popc(mo), iff = __popc(mf);
        const uint32_t co = io, cf = iff;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t yo = __shfl_up_sync(VSZ_FULL, io, off);
            const uint32_t yf = __shfl_up_sync(VSZ_FULL, iff, off);
            if (lane >= off) { io += yo; iff += yf; }
        }
        uint64_t po = ko + (io - co), pf = kf + (iff - cf);
#pragma unroll
        for (int k = 0; k < EPL; ++k) {
            if (mo & (1u << k)) {
                put_out(po, make_uint2((uint32_t)(base + k), (uint32_t)S.d[k]));
                ++po;
            }
            if (mf & (1u << k)) {
                put_fix(pf, make_uint2((uint32_t)(base + k), __float_as_uint(S.x[k])));
                ++pf;
            }
        }
        ko += __shfl_sync(VSZ_FULL, io, 31);
        kf += __shfl_sync(VSZ_FULL, iff, 31);
    }
}

// One field: tiles handed out by the field's own ticket.
template <int B, bool BP, bool GP>
__global__ void __launch_bounds__(256, 4) k_lorenzo_1d(const CompressArgs a) {
    pdl_prologue();
    __shared__ uint2 stash[8][kStash1];
    __shared__ uint2 fstash[8][kStash1F];
    __shared__ int2 mm[8][32];
    const int lane = threadIdx.x & 31;
    for (;;) {
        unsigned long long tk = 0;
        if (lane == 0) tk = atomicAdd(&a.wsh->ticket, 1ull);
        const uint64_t t = __shfl_sync(VSZ_FULL, tk, 0);
        if (t >= a.g.ntiles) break;
        compress_1d_tile<B, BP, GP>(a, t, lane, stash[threadIdx.x >> 5], fstash[threadIdx.x >> 5],
                                    mm[threadIdx.x >> 5]);
    }
}

// Many 1D fields with the same block length and padding kind: one queue
// over all their tiles (tile_prefix as for the 2D/3D batch kernel).
template <int B, bool BP, bool GP>
__global__ void __launch_bounds__(256, 4) k_lorenzo_1d_batch(const CompressArgs* __restrict__ fields,
                                                          const uint64_t* __restrict__ tile_prefix, int nfields,
                                                          unsigned long long* ticket) {
    __shared__ uint2 stash[8][kStash1];
    __shared__ uint2 fstash[8][kStash1F];
    __shared__ int2 mm[8][32];
    const int lane = threadIdx.x & 31;
    const uint64_t total = tile_prefix[nfields];
    for (;;) {
        unsigned long long tk = 0;
        if (lane == 0) tk = atomicAdd(ticket, 1ull);
        const uint64_t gt = __shfl_sync(VSZ_FULL, tk, 0);
        if (gt >= total) break;
        int lo = 0, hi = nfields - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (tile_prefix[mid] <= gt) lo = mid; else hi = mid - 1;
        }
        compress_1d_tile<B, BP, GP>(fields[lo], gt - tile_prefix[lo], lane, stash[threadIdx.x >> 5],
                                    fstash[threadIdx.x >> 5], mm[threadIdx.x >> 5]);
    }
}

// ---------------------------------------------------------------------------
// Inverse: codes -> residuals (outliers patched by their rank inside the
// block), block origin += P, segmented inclusive scan, x_hat = q * ebx2.
// One step st (32*EPL elements) of one field; ebx2 and Pg from its header.
template <int B, bool QOUT>
__device__ __forceinline__ void recon_1d_step(const ReconArgs& a, const uint64_t st, const int lane,
                                              const float ebx2, const int32_t Pg) {
    using C = Cfg1<B>;
    constexpr int EPL = C::EPL, G = C::G, SPAN = C::SPAN;
    const int32_t R = a.R;
    const uint64_t n = a.g.n;
    const int glane = lane & (G - 1);
    const bool bp = is_block_pad(a.pad_mode) || is_edge_pad(a.pad_mode);  // 1D edge: one scalar per block
    {
        const uint64_t base = st * SPAN + (uint64_t)lane * EPL;
        const int valid = base < n ? (int)umin64(EPL, n - base) : 0;
        const bool vec = a.vec && valid == EPL;
        uint32_t c[EPL];
        if (vec) {
            if (EPL == 4) {
                const uint2 u = ld_stream_u2(a.codes + base);
                c[0] = u.x & 0xffffu; c[1] = u.x >> 16; c[2 % EPL] = u.y & 0xffffu; c[3 % EPL] = u.y >> 16;
            } else {
                const uint4 u = ld_stream_u4(a.codes + base);
                c[0] = u.x & 0xffffu; c[1] = u.x >> 16; c[2] = u.y & 0xffffu; c[3] = u.y >> 16;
                c[4 % EPL] = u.z & 0xffffu; c[5 % EPL] = u.z >> 16; c[6 % EPL] = u.w & 0xffffu; c[7 % EPL] = u.w >> 16;
            }
        } else {
#pragma unroll
            for (int k = 0; k < EPL; ++k) c[k] = (k < valid) ? (uint32_t)a.codes[base + k] : (uint32_t)R;
        }
        int32_t d[EPL];
        uint32_t zm = 0;
#pragma unroll
        for (int k = 0; k < EPL; ++k) {
            d[k] = (int32_t)c[k] - R;
            if (k < valid && c[k] == 0u) zm |= 1u << k;
        }
        const uint64_t blk = base / B;
        if (__any_sync(VSZ_FULL, zm != 0)) {
            // rank of each outlier inside its block = zeros before it
            uint32_t iz = __popc(zm);
            const uint32_t cz = iz;
#pragma unroll
            for (int off = 1; off < G; off <<= 1) {
                const uint32_t y = __shfl_up_sync(VSZ_FULL, iz, off);
                if (glane >= off) iz += y;
            }
            if (zm) {
                const uint32_t lo = a.blk_off[blk], hi = a.blk_off[blk + 1];
                uint32_t r = lo + (iz - cz);
#pragma unroll
                for (int k = 0; k < EPL; ++k) {
                    if (zm & (1u << k)) {
                        if (r < hi && r < a.out_cap && a.out_idx[r] == (uint32_t)(base + k)) {
                            d[k] = a.out_delta[r];
                        } else {
                            atomicMax(&a.hdr->recon_status, (unsigned)VSZ_ERR_CORRUPT);
                            d[k] = 0;
                        }
                        ++r;
                    }
                }
            }
        }
        if (glane == 0 && valid > 0) {
            const int32_t P = bp ? a.pad[blk] : Pg;
            d[0] = (int32_t)((uint32_t)d[0] + (uint32_t)P);
        }
        // inclusive scan: in lane, then segmented across the block's lanes
#pragma unroll
        for (int k = 1; k < EPL; ++k) d[k] = (int32_t)((uint32_t)d[k] + (uint32_t)d[k - 1]);
        uint32_t tot = (uint32_t)d[EPL - 1], inc = tot;
#pragma unroll
        for (int off = 1; off < G; off <<= 1) {
            const uint32_t y = __shfl_up_sync(VSZ_FULL, inc, off);
            if (glane >= off) inc += y;
        }
        const uint32_t ex = inc - tot;
#pragma unroll
        for (int k = 0; k < EPL; ++k) d[k] = (int32_t)((uint32_t)d[k] + ex);

        if (QOUT) {
            int32_t* o = reinterpret_cast<int32_t*>(a.out) + base;
            if (vec) {
#pragma unroll
                for (int h = 0; h < EPL / 4; ++h)
                    *reinterpret_cast<int4*>(o + 4 * h) = make_int4(d[4 * h], d[4 * h + 1], d[4 * h + 2], d[4 * h + 3]);
            } else {
#pragma unroll
                for (int k = 0; k < EPL; ++k)
                    if (k < valid) o[k] = d[k];
            }
        } else {
            float* o = reinterpret_cast<float*>(a.out) + base;
            float v[EPL];
#pragma unroll
            for (int k = 0; k < EPL; ++k) v[k] = __fmul_rn(q2f(d[k]), ebx2);
            if (vec) {
#pragma unroll
                for (int h = 0; h < EPL / 4; ++h)
                    *reinterpret_cast<float4*>(o + 4 * h) = make_float4(v[4 * h], v[4 * h + 1], v[4 * h + 2], v[4 * h + 3]);
            } else {
#pragma unroll
                for (int k = 0; k < EPL; ++k)
                    if (k < valid) o[k] = v[k];
            }
        }
    }
}

template <int B, bool QOUT>
__global__ void __launch_bounds__(256) k_recon_1d(const ReconArgs a) {
    pdl_prologue();
    using C = Cfg1<B>;
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const float ebx2 = a.hdr->ebx2;
    const int32_t Pg = a.hdr->pad_global;
    const uint64_t nsteps = (a.g.n + C::SPAN - 1) / C::SPAN;
    for (uint64_t st = (uint64_t)blockIdx.x * C::WARPS + wib; st < nsteps; st += (uint64_t)gridDim.x * C::WARPS)
        recon_1d_step<B, QOUT>(a, st, lane, ebx2, Pg);
}

// Many 1D fields with the same block length: one queue over their tiles of
// kChunk1D values (tile_prefix as for the batch compression).
template <int B>
__global__ void __launch_bounds__(256) k_recon_1d_batch(const ReconArgs* __restrict__ fields,
                                                        const uint64_t* __restrict__ tile_prefix, int nfields,
                                                        unsigned long long* ticket) {
    using C = Cfg1<B>;
    const int lane = threadIdx.x & 31;
    const uint64_t total = tile_prefix[nfields];
    for (;;) {
        unsigned long long tk = 0;
        if (lane == 0) tk = atomicAdd(ticket, 1ull);
        const uint64_t gt = __shfl_sync(VSZ_FULL, tk, 0);
        if (gt >= total) break;
        int lo = 0, hi = nfields - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (tile_prefix[mid] <= gt) lo = mid; else hi = mid - 1;
        }
        const ReconArgs& a = fields[lo];
        const float ebx2 = a.hdr->ebx2;
        const int32_t Pg = a.hdr->pad_global;
        const uint64_t st0 = (gt - tile_prefix[lo]) * C::STEPS;
        const uint64_t nsteps = (a.g.n + C::SPAN - 1) / C::SPAN;
        const uint64_t st1 = umin64(nsteps, st0 + C::STEPS);
        for (uint64_t st = st0; st < st1; ++st) recon_1d_step<B, false>(a, st, lane, ebx2, Pg);
    }
}

// ---------------------------------------------------------------------------
template <int B, bool BP, bool GP>
static cudaError_t launch_c1_k(const CompressArgs& a, cudaStream_t s) {
    const void* k = (const void*)k_lorenzo_1d<B, BP, GP>;
    const int grid = grid_for(k, 256, 0, Cfg1<B>::WARPS, a.g.ntiles);
    return launch_pdl(k_lorenzo_1d<B, BP, GP>, grid, 256, 0, s, a);
}

template <int B>
static cudaError_t launch_c1(const CompressArgs& a, cudaStream_t s) {
    if (is_block_pad(a.pad_mode)) return launch_c1_k<B, true, false>(a, s);
    if (defers_origin(a.pad_mode)) return launch_c1_k<B, false, true>(a, s);
    return launch_c1_k<B, false, false>(a, s);
}

template <int B, bool BP, bool GP>
static cudaError_t launch_c1_batch_k(const CompressArgs* fields, const uint64_t* tile_prefix, int nfields,
                                     uint64_t total_tiles, unsigned long long* ticket, LaunchShape sh,
                                     cudaStream_t s, int* occ) {
    const void* k = (const void*)k_lorenzo_1d_batch<B, BP, GP>;
    const int warps = sh.warps > 0 ? sh.warps : Cfg1<B>::WARPS;
    if (warps > 8) {
        if (occ) *occ = 0;
        return occ ? cudaSuccess : cudaErrorInvalidValue;
    }
    if (occ) {
        *occ = occupancy(k, warps * 32, 0);
        return cudaSuccess;
    }
    const int grid = grid_shape(k, warps * 32, 0, (uint64_t)warps, total_tiles, sh.ctas);
    k_lorenzo_1d_batch<B, BP, GP><<<grid, warps * 32, 0, s>>>(fields, tile_prefix, nfields, ticket);
    return cudaGetLastError();
}

// pk: 0 zero padding, 1 per-block padding, 2 global padding, 3 edge padding
template <int B>
static cudaError_t launch_c1_batch(int pk, const CompressArgs* fields, const uint64_t* tile_prefix, int nfields,
                                   uint64_t total_tiles, unsigned long long* ticket, LaunchShape sh, cudaStream_t s,
                                   int* occ) {
    if (pk == 1) return launch_c1_batch_k<B, true, false>(fields, tile_prefix, nfields, total_tiles, ticket, sh, s, occ);
    if (pk == 2 || pk == 3)  // global or edge padding (a 1D block's face is its first value)
        return launch_c1_batch_k<B, false, true>(fields, tile_prefix, nfields, total_tiles, ticket, sh, s, occ);
    return launch_c1_batch_k<B, false, false>(fields, tile_prefix, nfields, total_tiles, ticket, sh, s, occ);
}

template <int B>
static cudaError_t launch_r1_batch(const ReconArgs* fields, const uint64_t* tile_prefix, int nfields,
                                   uint64_t total_tiles, unsigned long long* ticket, LaunchShape sh, cudaStream_t s,
                                   int* occ) {
    const void* k = (const void*)k_recon_1d_batch<B>;
    const int warps = sh.warps > 0 ? sh.warps : Cfg1<B>::WARPS;
    if (warps > 8) {
        if (occ) *occ = 0;
        return occ ? cudaSuccess : cudaErrorInvalidValue;
    }
    if (occ) {
        *occ = occupancy(k, warps * 32, 0);
        return cudaSuccess;
    }
    const int grid = grid_shape(k, warps * 32, 0, (uint64_t)warps, total_tiles, sh.ctas);
    k_recon_1d_batch<B><<<grid, warps * 32, 0, s>>>(fields, tile_prefix, nfields, ticket);
    return cudaGetLastError();
}

template <int B>
static cudaError_t launch_r1(const ReconArgs& a, bool q_out, cudaStream_t s) {
    const uint64_t nsteps = (a.g.n + Cfg1<B>::SPAN - 1) / Cfg1<B>::SPAN;
    const void* k = q_out ? (const void*)k_recon_1d<B, true> : (const void*)k_recon_1d<B, false>;
    const int grid = grid_for(k, 256, 0, 8, nsteps);
    return q_out ? launch_pdl(k_recon_1d<B, true>, grid, 256, 0, s, a) : launch_pdl(k_recon_1d<B, false>, grid, 256, 0, s, a);
}

cudaError_t launch_lorenzo_1d(const CompressArgs& a, cudaStream_t s) {
    switch (a.g.b) {
    case 4: return launch_c1<4>(a, s);
    case 8: return launch_c1<8>(a, s);
    case 16: return launch_c1<16>(a, s);
    case 32: return launch_c1<32>(a, s);
    case 64: return launch_c1<64>(a, s);
    case 128: return launch_c1<128>(a, s);
    case 256: return launch_c1<256>(a, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_lorenzo_batch_1d(uint32_t b, int pk, const CompressArgs* fields, const uint64_t* tile_prefix,
                                    int nfields, uint64_t total_tiles, unsigned long long* ticket, LaunchShape sh,
                                    cudaStream_t s, int* occ) {
    switch (b) {
    case 4: return launch_c1_batch<4>(pk, fields, tile_prefix, nfields, total_tiles, ticket, sh, s, occ);
    case 8: return launch_c1_batch<8>(pk, fields, tile_prefix, nfields, total_tiles, ticket, sh, s, occ);
    case 16: return launch_c1_batch<16>(pk, fields, tile_prefix, nfields, total_tiles, ticket, sh, s, occ);
    case 32: return launch_c1_batch<32>(pk, fields, tile_prefix, nfields, total_tiles, ticket, sh, s, occ);
    case 64: return launch_c1_batch<64>(pk, fields, tile_prefix, nfields, total_tiles, ticket, sh, s, occ);
    case 128: return launch_c1_batch<128>(pk, fields, tile_prefix, nfields, total_tiles, ticket, sh, s, occ);
    case 256: return launch_c1_batch<256>(pk, fields, tile_prefix, nfields, total_tiles, ticket, sh, s, occ);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_recon_1d(const ReconArgs& a, bool q_out, cudaStream_t s) {
    switch (a.g.b) {
    case 4: return launch_r1<4>(a, q_out, s);
    case 8: return launch_r1<8>(a, q_out, s);
    case 16: return launch_r1<16>(a, q_out, s);
    case 32: return launch_r1<32>(a, q_out, s);
    case 64: return launch_r1<64>(a, q_out, s);
    case 128: return launch_r1<128>(a, q_out, s);
    case 256: return launch_r1<256>(a, q_out, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_recon_batch_1d(uint32_t b, const ReconArgs* fields, const uint64_t* tile_prefix, int nfields,
                                  uint64_t total_tiles, unsigned long long* ticket, LaunchShape sh, cudaStream_t s,
                                  int* occ) {
    switch (b) {
    case 4: return launch_r1_batch<4>(fields, tile_prefix, nfields, total_tiles, ticket, sh, s, occ);
    case 8: return launch_r1_batch<8>(fields, tile_prefix, nfields, total_tiles, ticket, sh, s, occ);
    case 16: return launch_r1_batch<16>(fields, tile_prefix, nfields, total_tiles, ticket, sh, s, occ);
    case 32: return launch_r1_batch<32>(fields, tile_prefix, nfields, total_tiles, ticket, sh, s, occ);
    case 64: return launch_r1_batch<64>(fields, tile_prefix, nfields, total_tiles, ticket, sh, s, occ);
    case 128: return launch_r1_batch<128>(fields, tile_prefix, nfields, total_tiles, ticket, sh, s, occ);
    case 256: return launch_r1_batch<256>(fields, tile_prefix, nfields, total_tiles, ticket, sh, s, occ);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace vsz
