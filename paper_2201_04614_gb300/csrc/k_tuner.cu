// k_tuner.cu -- the learned tuner of block size and padding mode.
//
// The paper tunes the block size (Sec. III-D) with a sampling autotuner and
// studies padding values (Sec. IV) by hand; this library learns both from
// cheap field statistics instead.  Here: the sampled features of a field,
// the exhaustive class sweep that labels training fields with the estimated
// compressed size of every class (codes after entropy coding, Sec. II-B,
// plus outliers, fixups and padding scalars), the MLP's inference, gradient
// and Adam kernels, and the outlier-count guard that falls back to the
// default class.  All fp32/fp64 CUDA-core code: the network is far too small
// for tensor cores to matter.
#include <cmath>
#include <cstring>

#include "common.cuh"
#include "misc.cuh"
#include "stats.cuh"
#include "trace.cuh"

namespace vsz {

constexpr int kNF = VSZ_TUNER_NFEAT;
constexpr int kNC = VSZ_TUNER_NCLASS;
constexpr int kH = VSZ_TUNER_HIDDEN;
constexpr int kNP = VSZ_TUNER_NPARAM;
constexpr int oW1 = 0, ob1 = oW1 + kH * kNF, oW2 = ob1 + kH, ob2 = oW2 + kH * kH, oW3 = ob2 + kH,
              ob3 = oW3 + kNC * kH;
static_assert(ob3 + kNC == kNP, "parameter layout");
constexpr uint64_t kSampleMax = 32768;
constexpr uint64_t kHashMul = 2654435761ull;

// Block sizes of the class slots per rank (0 = slot not allowed).
__host__ __device__ inline uint32_t class_block(int nd, int slot) {
    const uint32_t t1[4] = {32, 64, 128, 256}, t2[4] = {8, 16, 32, 64}, t3[4] = {8, 16, 32, 0};
    if (slot < 0 || slot > 3) return 0;
    return nd == 1 ? t1[slot] : nd == 2 ? t2[slot] : nd == 3 ? t3[slot] : 0;
}
__host__ __device__ inline int class_pad(int padslot) {
    return padslot == 0 ? VSZ_PAD_ZERO : padslot == 1 ? VSZ_PAD_GLOBAL_AVG : VSZ_PAD_BLOCK_AVG;
}

// ---------------------------------------------------------------- features

struct FeatAcc {
    unsigned int xmin_ord, xmax_ord;
    unsigned long long cnt, qbig;
    unsigned long long gcnt[3];
    double sum, sq;
    double gsum[3];
};

struct FeatGeom {
    uint64_t n, S;
    uint64_t stride[3], ext[3];  // axis a: x (fastest) first
    int nd;
    int R;
    double eb;
    int rel;
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(VSZ_FULL, v, off);
    return v;
}
__device__ __forceinline__ unsigned long long warp_sum(unsigned long long v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(VSZ_FULL, v, off);
    return v;
}

__global__ void k_feat_init(FeatAcc* acc) {
    if (threadIdx.x == 0) {
        std::memset(acc, 0, sizeof(FeatAcc));
        acc->xmin_ord = 0xffffffffu;
        acc->xmax_ord = 0u;
    }
}

// Pass 1 over the samples: finite range, sum, and forward differences per axis.
__global__ void __launch_bounds__(256) k_feat_pass1(const float* __restrict__ x, FeatGeom fg, FeatAcc* acc) {
    unsigned int lo = 0xffffffffu, hi = 0u;
    unsigned long long cnt = 0, gc[3] = {0, 0, 0};
    double sum = 0.0, gs[3] = {0.0, 0.0, 0.0};
    for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < fg.S;
         k += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t j = (k * kHashMul) % fg.n;
        const float v = x[j];
        if (isfinite(v)) {
            const unsigned u = float_to_ord(v);
            lo = min(lo, u);
            hi = max(hi, u);
            sum += (double)v;
            ++cnt;
        }
        for (int a = 0; a < fg.nd; ++a) {
            const uint64_t c = (j / fg.stride[a]) % fg.ext[a];
            if (c + 1 < fg.ext[a]) {
                const double d = __dsub_rn((double)x[j + fg.stride[a]], (double)v);
                if (isfinite(d)) {
                    gs[a] += fabs(d);
                    ++gc[a];
                }
            }
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        lo = min(lo, __shfl_xor_sync(VSZ_FULL, lo, off));
        hi = max(hi, __shfl_xor_sync(VSZ_FULL, hi, off));
    }
    sum = warp_sum(sum);
    cnt = warp_sum(cnt);
    for (int a = 0; a < 3; ++a) {
        gs[a] = warp_sum(gs[a]);
        gc[a] = warp_sum(gc[a]);
    }
    if ((threadIdx.x & 31) == 0) {
        if (cnt) {
            atomicMin(&acc->xmin_ord, lo);
            atomicMax(&acc->xmax_ord, hi);
            atomicAdd(&acc->sum, sum);
            atomicAdd(&acc->cnt, cnt);
        }
        for (int a = 0; a < 3; ++a)
            if (gc[a]) {
                atomicAdd(&acc->gsum[a], gs[a]);
                atomicAdd(&acc->gcnt[a], gc[a]);
            }
    }
}

struct FeatScalars {
    double lo, hi, rng, eb_abs, mean;
    float inv2eb;
};

__device__ __forceinline__ FeatScalars feat_scalars(const FeatAcc* acc, const FeatGeom& fg) {
    FeatScalars s;
    const bool has = acc->cnt > 0;
    s.lo = has ? (double)ord_to_float(acc->xmin_ord) : 0.0;
    s.hi = has ? (double)ord_to_float(acc->xmax_ord) : 0.0;
    s.rng = __dsub_rn(s.hi, s.lo);
    s.eb_abs = (fg.rel && s.rng > 0.0) ? __dmul_rn(fg.eb, s.rng) : fg.eb;
    s.mean = has ? __ddiv_rn(acc->sum, (double)acc->cnt) : 0.0;
    s.inv2eb = __double2float_rn(__ddiv_rn(1.0, __dmul_rn(2.0, s.eb_abs)));
    return s;
}

// Pass 2: squared deviations from the mean, and samples with |q| >= R.
__global__ void __launch_bounds__(256) k_feat_pass2(const float* __restrict__ x, FeatGeom fg, FeatAcc* acc) {
    const FeatScalars sc = feat_scalars(acc, fg);
    double sq = 0.0;
    unsigned long long big = 0;
    for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < fg.S;
         k += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t j = (k * kHashMul) % fg.n;
        const float v = x[j];
        if (isfinite(v)) {
            const double d = __dsub_rn((double)v, sc.mean);
            sq += d * d;
            const int32_t q = prequant(v, sc.inv2eb);
            big += (q >= fg.R || q <= -fg.R) ? 1ull : 0ull;
        }
    }
    sq = warp_sum(sq);
    big = warp_sum(big);
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&acc->sq, sq);
        atomicAdd(&acc->qbig, big);
    }
}

__global__ void k_feat_finish(const FeatAcc* acc, FeatGeom fg, double* f64, float* f32) {
    if (threadIdx.x != 0) return;
    double f[kNF];
    for (int i = 0; i < kNF; ++i) f[i] = 0.0;
    f[fg.nd - 1] = 1.0;
    f[11] = log2((double)fg.R);
    if (fg.n > 0) {
        f[3] = log10((double)fg.n);
        if (acc->cnt > 0) {
            const FeatScalars sc = feat_scalars(acc, fg);
            const double cnt = (double)acc->cnt;
            for (int a = 0; a < fg.nd; ++a) {
                const double g = acc->gcnt[a] ? acc->gsum[a] / (double)acc->gcnt[a] : 0.0;
                f[5 + a] = log1p(g / sc.eb_abs);
            }
            if (sc.rng > 0.0) {
                f[4] = log10(sc.rng / sc.eb_abs);
                f[8] = fabs(sc.mean) / sc.rng;
                f[9] = sqrt(acc->sq / cnt) / sc.rng;
            }
            f[10] = (double)acc->qbig / cnt;
        }
    }
    for (int i = 0; i < kNF; ++i) {
        if (f64) f64[i] = f[i];
        if (f32) f32[i] = (float)f[i];
    }
}

static bool feat_geom(const Geom& g, const vsz_params* p, FeatGeom* fg) {
    std::memset(fg, 0, sizeof *fg);
    fg->n = g.n;
    fg->S = g.n < kSampleMax ? g.n : kSampleMax;
    fg->nd = g.nd;
    fg->R = (int)p->radius;
    fg->eb = p->eb;
    fg->rel = p->eb_mode == VSZ_EB_REL;
    const uint64_t e[3] = {g.nx, g.ny, g.nz};
    uint64_t s = 1;
    for (int a = 0; a < 3; ++a) {
        fg->stride[a] = s;
        fg->ext[a] = e[a];
        s *= e[a];
    }
    return true;
}

// ---------------------------------------------------------------- sweep

// Shannon entropy of the code histogram and the estimated size of a class.
__global__ void __launch_bounds__(1024) k_class_cost(const uint32_t* __restrict__ hist, uint32_t nbins, uint64_t n,
                                                     const vsz_header* hdr, double npad, double* cost) {
    __shared__ double sm[32];
    double h = 0.0;
    const double dn = (double)n;
    for (uint32_t i = threadIdx.x; i < nbins; i += blockDim.x) {
        const uint32_t c = hist[i];
        if (c) {
            const double p = (double)c / dn;
            h -= p * log2(p);
        }
    }
    h = warp_sum(h);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sm[w] = h;
    __syncthreads();
    if (w == 0) {
        h = l < (int)(blockDim.x >> 5) ? sm[l] : 0.0;
        h = warp_sum(h);
        if (l == 0)
            *cost = dn * h / 8.0 + 8.0 * (double)hdr->n_out + 8.0 * (double)hdr->n_fix + 4.0 * npad;
    }
}

__global__ void k_set_double(double* p, double v) {
    if (threadIdx.x == 0) *p = v;
}

__global__ void k_set_u64(uint64_t* p, uint64_t v) {
    if (threadIdx.x == 0) *p = v;
}

__global__ void k_copy_nout(const vsz_header* hdr, uint64_t* dst) {
    if (threadIdx.x == 0) *dst = hdr->n_out;
}

// Buffers of one count-only compression (no outlier lists): the codes, the
// per-block tables and the compression workspace.
struct CountBufs {
    size_t off_hdr, off_hist, off_codes, off_pad, off_blk, off_cws, total;
    size_t cws_bytes;
};

static CountBufs count_bufs(uint64_t n, uint64_t nb_max, uint32_t R, size_t cws_bytes, size_t extra_front) {
    CountBufs b;
    size_t off = align256(extra_front);
    b.off_hdr = off;
    off = align256(off + sizeof(vsz_header));
    b.off_hist = off;
    off = align256(off + (size_t)2 * R * 4);
    b.off_codes = off;
    off = align256(off + n * 2);
    b.off_pad = off;
    off = align256(off + (nb_max + 1) * 4);
    b.off_blk = off;
    off = align256(off + (nb_max + 1) * 4);
    b.off_cws = off;
    b.cws_bytes = cws_bytes;
    off = align256(off + cws_bytes);
    b.total = off;
    return b;
}

// Count-only compression of one class: exact n_out / n_fix in the header
// (the lists themselves are not kept: their capacities are zero).
static vsz_status count_class(const vsz_params* pc, const float* d_x, char* ws, const CountBufs& B, cudaStream_t s) {
    vsz_compressed c;
    std::memset(&c, 0, sizeof c);
    c.codes = (uint16_t*)(ws + B.off_codes);
    c.pad = (int32_t*)(ws + B.off_pad);
    c.blk_off = (uint32_t*)(ws + B.off_blk);
    c.hdr = (vsz_header*)(ws + B.off_hdr);
    vsz_status st = vsz_prequant_lorenzo(pc, d_x, &c, ws + B.off_cws, B.cws_bytes, s);
    if (st != VSZ_OK) return st;
    return vsz_outlier_compact(pc, &c, ws + B.off_cws, B.cws_bytes, s);
}

static vsz_params class_params_of(const vsz_params* p, int c) {
    vsz_params pc = *p;
    pc.block = class_block(p->ndim, c / 3);
    pc.pad = class_pad(c % 3);
    return pc;
}

static vsz_status sweep_bufs(const vsz_params* p, CountBufs* out) {
    if (!p || p->ndim < 1 || p->ndim > 3) return VSZ_ERR_INVALID_ARG;
    vsz_status st;
    uint64_t nb_max = 0;
    size_t cws = 0;
    uint64_t n = 0;
    for (int c = 0; c < kNC; ++c) {
        if (!class_block(p->ndim, c / 3)) continue;
        const vsz_params pc = class_params_of(p, c);
        Geom gc;
        if ((st = make_geom(&pc, &gc)) != VSZ_OK) return st;
        n = gc.n;
        nb_max = gc.nb > nb_max ? gc.nb : nb_max;
        const size_t w = ws_layout(gc, 0, 0).total;
        cws = w > cws ? w : cws;
    }
    *out = count_bufs(n, nb_max, p->radius, cws, 0);
    return VSZ_OK;
}

// ---------------------------------------------------------------- guard sample

struct GuardGeom {
    bool whole;
    int nd;
    uint64_t K, E0, Ey;       // regions, extent along dims[0], extent along y (3D)
    uint64_t m0, my;          // aligned slots along dims[0] and y
    uint64_t dims[3];         // stacked sub-field dims (C-order)
    uint64_t nsub;
    uint64_t ny, nx;          // source extents
};

// min_slots: fewer aligned slots along dims[0] than this samples the whole
// field; frac < 0: the guard's K (about 2 % of the field), else K regions
// holding about frac of the elements.
static GuardGeom region_geom(const Geom& g, const vsz_params* p, uint64_t min_slots, double frac) {
    GuardGeom G;
    std::memset(&G, 0, sizeof G);
    G.nd = g.nd;
    const uint64_t L = g.nd == 1 ? 256 : g.nd == 2 ? 64 : 32;
    G.E0 = g.nd == 1 ? 65536 : L;
    const uint64_t d0 = p->dims[0];
    G.whole = g.n <= (1ull << 20) || d0 < min_slots * G.E0;
    G.ny = g.ny;
    G.nx = g.nx;
    if (G.whole) {
        for (int k = 0; k < 3; ++k) G.dims[k] = p->dims[k];
        G.nsub = g.n;
        G.K = 1;
        return G;
    }
    G.Ey = g.nd == 3 ? (g.ny <= L ? g.ny : L) : 1;
    const uint64_t r = g.nd == 1 ? G.E0 : g.nd == 2 ? G.E0 * g.nx : G.E0 * G.Ey * g.nx;
    G.m0 = d0 / G.E0;
    G.my = g.nd == 3 ? (g.ny <= L ? 1 : g.ny / L) : 1;
    uint64_t K = g.n / (50 * r);
    if (frac >= 0.0) {
        const double kd = frac * (double)g.n / (double)r;
        K = kd < 1.0 ? 1 : (uint64_t)(kd + 0.5);
    }
    if (K < 1) K = 1;
    if (K > G.m0) K = G.m0;
    G.K = K;
    G.dims[0] = K * G.E0;
    if (g.nd == 2) G.dims[1] = g.nx;
    if (g.nd == 3) {
        G.dims[1] = G.Ey;
        G.dims[2] = g.nx;
    }
    G.nsub = K * r;
    return G;
}

static GuardGeom guard_geom(const Geom& g, const vsz_params* p) { return region_geom(g, p, 4, -1.0); }

// Gather of the guard's sample regions into one stacked field.
__global__ void __launch_bounds__(256) k_gather_sample(const float* __restrict__ x, float* __restrict__ out,
                                                       GuardGeom G) {
    for (uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; s < G.nsub;
         s += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t src;
        if (G.nd == 1) {
            const uint64_t i = s / G.E0, o = s % G.E0;
            src = (i * G.m0 / G.K) * G.E0 + o;
        } else if (G.nd == 2) {
            const uint64_t row = s / G.nx, col = s % G.nx;
            const uint64_t i = row / G.E0, lr = row % G.E0;
            src = ((i * G.m0 / G.K) * G.E0 + lr) * G.nx + col;
        } else {
            const uint64_t col = s % G.nx;
            const uint64_t ky = (s / G.nx) % G.Ey;
            const uint64_t kz = s / (G.nx * G.Ey);
            const uint64_t i = kz / G.E0, lz = kz % G.E0;
            const uint64_t z = (i * G.m0 / G.K) * G.E0 + lz;
            const uint64_t y = (i * G.my / G.K) * G.Ey + ky;
            src = (z * G.ny + y) * G.nx + col;
        }
        out[s] = x[src];
    }
}

// ---------------------------------------------------------------- network

// Forward pass of one sample by a CTA of 128 threads; the parameters are in
// shared memory.  Leaves xt, h1, h2 and the masked logits z in shared memory.
struct MlpSmem {
    float th[kNP];
    float mu[kNF], sg[kNF];
    float xt[kNF], h1[kH], h2[kH], z[kNC];
    float dz[kNC], d2[kH], d1[kH];
    float loss;
};

__device__ __forceinline__ void mlp_load(MlpSmem& S, const float* theta, const float* norm) {
    for (int i = threadIdx.x; i < kNP; i += blockDim.x) S.th[i] = theta[i];
    for (int i = threadIdx.x; i < kNF; i += blockDim.x) {
        S.mu[i] = norm[i];
        S.sg[i] = norm[kNF + i];
    }
    __syncthreads();
}

__device__ __forceinline__ void mlp_fwd(MlpSmem& S, const float* xrow, uint32_t mask) {
    const int t = threadIdx.x;
    if (t < kNF) S.xt[t] = __fdiv_rn(__fsub_rn(xrow[t], S.mu[t]), S.sg[t]);
    __syncthreads();
    if (t < kH) {
        float a = S.th[ob1 + t];
        for (int k = 0; k < kNF; ++k) a = __fadd_rn(a, __fmul_rn(S.th[oW1 + t * kNF + k], S.xt[k]));
        S.h1[t] = fmaxf(a, 0.0f);
    }
    __syncthreads();
    if (t < kH) {
        float a = S.th[ob2 + t];
        for (int i = 0; i < kH; ++i) a = __fadd_rn(a, __fmul_rn(S.th[oW2 + t * kH + i], S.h1[i]));
        S.h2[t] = fmaxf(a, 0.0f);
    }
    __syncthreads();
    if (t < kNC) {
        float a = S.th[ob3 + t];
        for (int j = 0; j < kH; ++j) a = __fadd_rn(a, __fmul_rn(S.th[oW3 + t * kH + j], S.h2[j]));
        S.z[t] = ((mask >> t) & 1u) ? a : -INFINITY;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(128) k_mlp_forward(const float* __restrict__ theta, const float* __restrict__ norm,
                                                     const float* __restrict__ X, const uint32_t* __restrict__ mask,
                                                     int n, float* logits, int32_t* cls) {
    __shared__ MlpSmem S;
    mlp_load(S, theta, norm);
    for (int s = blockIdx.x; s < n; s += gridDim.x) {
        mlp_fwd(S, X + (size_t)s * kNF, mask[s]);
        if (threadIdx.x < kNC && logits) logits[(size_t)s * kNC + threadIdx.x] = S.z[threadIdx.x];
        if (threadIdx.x == 0 && cls) {
            int best = 0;
            for (int c = 1; c < kNC; ++c)
                if (S.z[c] > S.z[best]) best = c;
            cls[s] = best;
        }
        __syncthreads();
    }
}

constexpr int kSPC = 16;  // samples per CTA in the gradient kernel

// Per-CTA sums of the per-sample cross-entropy gradients over a chunk of the
// minibatch (backpropagation through the three layers).  Every gradient
// entry is owned by one thread (entry e -> thread e mod 128), so the sums
// are deterministic.  partial[cta][kNP] receives the chunk's loss sum.
__global__ void __launch_bounds__(128) k_mlp_grad(const float* __restrict__ theta, const float* __restrict__ norm,
                                                  const float* __restrict__ X, const int32_t* __restrict__ y,
                                                  const uint32_t* __restrict__ mask, const int32_t* __restrict__ idx,
                                                  int batch, float* __restrict__ partial) {
    __shared__ MlpSmem S;
    mlp_load(S, theta, norm);
    const int t = threadIdx.x;
    constexpr int R1 = (kH * kNF + 127) / 128, R2 = (kH * kH) / 128, R3 = (kNC * kH + 127) / 128;
    float g1[R1], g2[R2], g3[R3];
    float gb1 = 0.f, gb2 = 0.f, gb3 = 0.f, lsum = 0.f;
#pragma unroll
    for (int r = 0; r < R1; ++r) g1[r] = 0.f;
#pragma unroll
    for (int r = 0; r < R2; ++r) g2[r] = 0.f;
#pragma unroll
    for (int r = 0; r < R3; ++r) g3[r] = 0.f;
    const int b0 = blockIdx.x * kSPC;
    const int b1 = min(batch, b0 + kSPC);
    for (int b = b0; b < b1; ++b) {
        const int s = idx ? idx[b] : b;
        const uint32_t m = mask[s];
        const int ys = y[s];
        mlp_fwd(S, X + (size_t)s * kNF, m);
        if (t == 0) {  // masked softmax cross-entropy: dL/dz = p - onehot(y)
            float mx = -INFINITY;
            for (int c = 0; c < kNC; ++c) mx = fmaxf(mx, S.z[c]);
            float e[kNC], sum = 0.f;
            for (int c = 0; c < kNC; ++c) {
                e[c] = ((m >> c) & 1u) ? expf(__fsub_rn(S.z[c], mx)) : 0.f;
                sum = __fadd_rn(sum, e[c]);
            }
            for (int c = 0; c < kNC; ++c) S.dz[c] = __fsub_rn(__fdiv_rn(e[c], sum), c == ys ? 1.f : 0.f);
            S.loss = __fsub_rn(logf(sum), __fsub_rn(S.z[ys], mx));
        }
        __syncthreads();
        lsum = __fadd_rn(lsum, S.loss);
#pragma unroll
        for (int r = 0; r < R3; ++r) {
            const int e = t + 128 * r;
            if (e < kNC * kH) g3[r] = __fadd_rn(g3[r], __fmul_rn(S.dz[e / kH], S.h2[e % kH]));
        }
        if (t < kNC) gb3 = __fadd_rn(gb3, S.dz[t]);
        if (t < kH) {
            float a = 0.f;
            for (int c = 0; c < kNC; ++c) a = __fadd_rn(a, __fmul_rn(S.th[oW3 + c * kH + t], S.dz[c]));
            S.d2[t] = S.h2[t] > 0.f ? a : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < R2; ++r) {
            const int e = t + 128 * r;
            g2[r] = __fadd_rn(g2[r], __fmul_rn(S.d2[e / kH], S.h1[e % kH]));
        }
        if (t < kH) {
            gb2 = __fadd_rn(gb2, S.d2[t]);
            float a = 0.f;
            for (int j = 0; j < kH; ++j) a = __fadd_rn(a, __fmul_rn(S.th[oW2 + j * kH + t], S.d2[j]));
            S.d1[t] = S.h1[t] > 0.f ? a : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < R1; ++r) {
            const int e = t + 128 * r;
            if (e < kH * kNF) g1[r] = __fadd_rn(g1[r], __fmul_rn(S.d1[e / kNF], S.xt[e % kNF]));
        }
        if (t < kH) gb1 = __fadd_rn(gb1, S.d1[t]);
        __syncthreads();
    }
    float* out = partial + (size_t)blockIdx.x * (kNP + 1);
#pragma unroll
    for (int r = 0; r < R1; ++r) {
        const int e = t + 128 * r;
        if (e < kH * kNF) out[oW1 + e] = g1[r];
    }
#pragma unroll
    for (int r = 0; r < R2; ++r) out[oW2 + t + 128 * r] = g2[r];
#pragma unroll
    for (int r = 0; r < R3; ++r) {
        const int e = t + 128 * r;
        if (e < kNC * kH) out[oW3 + e] = g3[r];
    }
    if (t < kH) {
        out[ob1 + t] = gb1;
        out[ob2 + t] = gb2;
    }
    if (t < kNC) out[ob3 + t] = gb3;
    if (t == 0) out[kNP] = lsum;
}

// Sum of the per-CTA partials in CTA order, divided by the batch size.
__global__ void __launch_bounds__(256) k_mlp_reduce(const float* __restrict__ partial, int nparts, int batch,
                                                    float* grad, float* loss) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i > kNP) return;
    float a = 0.f;
    for (int c = 0; c < nparts; ++c) a = __fadd_rn(a, partial[(size_t)c * (kNP + 1) + i]);
    const float v = __fdiv_rn(a, (float)batch);
    if (i < kNP) grad[i] = v;
    else if (loss) *loss = v;
}

// Adam (Kingma & Ba, 2015) with bias corrections c1 = 1/(1-beta1^t), c2 = 1/(1-beta2^t).
__global__ void __launch_bounds__(256) k_adam(float* theta, const float* __restrict__ grad, float* m, float* v, int n,
                                              float lr, float beta1, float beta2, float eps, float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float g = grad[i];
    const float mi = __fadd_rn(__fmul_rn(beta1, m[i]), __fmul_rn(__fsub_rn(1.f, beta1), g));
    const float vi = __fadd_rn(__fmul_rn(beta2, v[i]), __fmul_rn(__fsub_rn(1.f, beta2), __fmul_rn(g, g)));
    m[i] = mi;
    v[i] = vi;
    const float mh = __fmul_rn(mi, c1), vh = __fmul_rn(vi, c2);
    theta[i] = __fsub_rn(theta[i], __fdiv_rn(__fmul_rn(lr, mh), __fadd_rn(__fsqrt_rn(vh), eps)));
}

}  // namespace vsz

using namespace vsz;

extern "C" {

size_t vsz_tuner_features_workspace_size(void) { return 256; }

vsz_status vsz_tuner_features(const vsz_params* p, const float* d_x, double* d_feat, float* d_feat32, void* d_ws,
                              size_t ws_bytes, void* stream) {
    if (!p || p->ndim < 1 || p->ndim > 3) return VSZ_ERR_INVALID_ARG;
    Geom g;
    vsz_params q = *p;
    q.block = 8;  // the features do not depend on the block edge
    vsz_status st = make_geom(&q, &g);
    if (st != VSZ_OK) return st;
    if ((!d_feat && !d_feat32) || !d_ws || ws_bytes < sizeof(FeatAcc) || !aligned(d_ws, 16)) return VSZ_ERR_INVALID_ARG;
    if (g.n > 0 && !d_x) return VSZ_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    FeatGeom fg;
    feat_geom(g, p, &fg);
    FeatAcc* acc = (FeatAcc*)d_ws;
    TraceScope ts("features", s, g.nd, 0, g.n);
    k_feat_init<<<1, 32, 0, s>>>(acc);
    if (fg.S > 0) {
        const int grid = (int)((fg.S + 255) / 256);
        k_feat_pass1<<<grid, 256, 0, s>>>(d_x, fg, acc);
        k_feat_pass2<<<grid, 256, 0, s>>>(d_x, fg, acc);
    }
    k_feat_finish<<<1, 32, 0, s>>>(acc, fg, d_feat, d_feat32);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? VSZ_OK : cuda_fail(e);
}

size_t vsz_tuner_sweep_workspace_size(const vsz_params* p) {
    CountBufs b;
    return sweep_bufs(p, &b) == VSZ_OK ? b.total : 0;
}

vsz_status vsz_tuner_sweep(const vsz_params* p, const float* d_x, double* d_cost, uint64_t* d_nout, void* d_ws,
                           size_t ws_bytes, void* stream) {
    CountBufs B;
    vsz_status st = sweep_bufs(p, &B);
    if (st != VSZ_OK) return st;
    if (!d_cost || !d_ws || ws_bytes < B.total || !aligned(d_ws, 256)) return VSZ_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    char* ws = (char*)d_ws;
    for (int c = 0; c < kNC; ++c) {
        if (!class_block(p->ndim, c / 3)) {
            k_set_double<<<1, 32, 0, s>>>(d_cost + c, INFINITY);
            if (d_nout) k_set_u64<<<1, 32, 0, s>>>(d_nout + c, ~0ull);
            continue;
        }
        const vsz_params pc = class_params_of(p, c);
        if ((st = count_class(&pc, d_x, ws, B, s)) != VSZ_OK) return st;
        if ((st = vsz_code_histogram(&pc, (const uint16_t*)(ws + B.off_codes), (uint32_t*)(ws + B.off_hist), s)) !=
            VSZ_OK)
            return st;
        Geom gc;
        make_geom(&pc, &gc);
        const double npad = pc.pad == VSZ_PAD_BLOCK_AVG ? (double)gc.nb : pc.pad == VSZ_PAD_GLOBAL_AVG ? 1.0 : 0.0;
        TraceScope ts("class_cost", s, gc.nd, gc.b, gc.n);
        k_class_cost<<<1, 1024, 0, s>>>((const uint32_t*)(ws + B.off_hist), 2u * p->radius, gc.n,
                                        (const vsz_header*)(ws + B.off_hdr), npad, d_cost + c);
        if (d_nout) k_copy_nout<<<1, 32, 0, s>>>((const vsz_header*)(ws + B.off_hdr), d_nout + c);
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? VSZ_OK : cuda_fail(e);
}

vsz_status vsz_tuner_guard_sample_dims(const vsz_params* p, uint64_t* sub_dims) {
    Geom g;
    vsz_params q = *p;
    q.block = 8;
    vsz_status st = make_geom(&q, &g);
    if (st != VSZ_OK) return st;
    if (!sub_dims) return VSZ_ERR_INVALID_ARG;
    const GuardGeom G = guard_geom(g, p);
    for (int k = 0; k < 3; ++k) sub_dims[k] = k < p->ndim ? G.dims[k] : 0;
    return VSZ_OK;
}

static vsz_status guard_layout(const vsz_params* p, int ca, int cb, GuardGeom* G, vsz_params* pa, vsz_params* pb,
                               CountBufs* B) {
    if (!p || p->ndim < 1 || p->ndim > 3) return VSZ_ERR_INVALID_ARG;
    if (ca < 0 || ca >= kNC || cb < 0 || cb >= kNC) return VSZ_ERR_INVALID_ARG;
    if (!class_block(p->ndim, ca / 3) || !class_block(p->ndim, cb / 3)) return VSZ_ERR_INVALID_ARG;
    Geom g;
    vsz_params q = *p;
    q.block = 8;
    vsz_status st = make_geom(&q, &g);
    if (st != VSZ_OK) return st;
    *G = guard_geom(g, p);
    vsz_params sub = *p;
    for (int k = 0; k < 3; ++k) sub.dims[k] = k < p->ndim ? G->dims[k] : 0;
    *pa = class_params_of(&sub, ca);
    *pb = class_params_of(&sub, cb);
    Geom ga, gb;
    if ((st = make_geom(pa, &ga)) != VSZ_OK) return st;
    if ((st = make_geom(pb, &gb)) != VSZ_OK) return st;
    const uint64_t nb = ga.nb > gb.nb ? ga.nb : gb.nb;
    const size_t wa = ws_layout(ga, 0, 0).total, wb = ws_layout(gb, 0, 0).total;
    const size_t front = G->whole ? 0 : (size_t)G->nsub * 4;
    *B = count_bufs(ga.n, nb, p->radius, wa > wb ? wa : wb, front);
    return VSZ_OK;
}

size_t vsz_tuner_guard_workspace_size(const vsz_params* p, int class_a, int class_b) {
    GuardGeom G;
    vsz_params pa, pb;
    CountBufs B;
    return guard_layout(p, class_a, class_b, &G, &pa, &pb, &B) == VSZ_OK ? B.total : 0;
}

vsz_status vsz_tuner_guard(const vsz_params* p, const float* d_x, int class_a, int class_b, uint64_t* d_nout,
                           double* d_cost, void* d_ws, size_t ws_bytes, void* stream) {
    GuardGeom G;
    vsz_params pa, pb;
    CountBufs B;
    vsz_status st = guard_layout(p, class_a, class_b, &G, &pa, &pb, &B);
    if (st != VSZ_OK) return st;
    if (!d_nout || !d_ws || ws_bytes < B.total || !aligned(d_ws, 256)) return VSZ_ERR_INVALID_ARG;
    if (G.nsub > 0 && !d_x) return VSZ_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    char* ws = (char*)d_ws;
    const float* src = d_x;
    if (!G.whole) {
        float* sub = (float*)ws;
        TraceScope ts("guard_gather", s, G.nd, 0, G.nsub);
        const int grid = grid_for((const void*)k_gather_sample, 256, 0, 256 * 8, G.nsub);
        k_gather_sample<<<grid, 256, 0, s>>>(d_x, sub, G);
        src = sub;
    }
    const vsz_params* pc[2] = {&pa, &pb};
    for (int k = 0; k < 2; ++k) {
        if ((st = count_class(pc[k], src, ws, B, s)) != VSZ_OK) return st;
        k_copy_nout<<<1, 32, 0, s>>>((const vsz_header*)(ws + B.off_hdr), d_nout + k);
        if (d_cost) {  // the class's estimated size on the sample, as the sweep computes it
            if ((st = vsz_code_histogram(pc[k], (const uint16_t*)(ws + B.off_codes), (uint32_t*)(ws + B.off_hist),
                                         s)) != VSZ_OK)
                return st;
            Geom gc;
            make_geom(pc[k], &gc);
            const double npad =
                pc[k]->pad == VSZ_PAD_BLOCK_AVG ? (double)gc.nb : pc[k]->pad == VSZ_PAD_GLOBAL_AVG ? 1.0 : 0.0;
            k_class_cost<<<1, 1024, 0, s>>>((const uint32_t*)(ws + B.off_hist), 2u * p->radius, gc.n,
                                            (const vsz_header*)(ws + B.off_hdr), npad, d_cost + k);
        }
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? VSZ_OK : cuda_fail(e);
}

// ---------------------------------------------------------------- sampling autotuner
// The paper's autotuner (Sec. III-D, Sec. V-E): time the dual-quant of every
// configuration on a fixed fraction of the field's blocks, several times,
// and keep the configuration with the best mean.  The sample is K regions
// spread evenly along dims[0] (as for the guard), aligned to every candidate
// block, stacked into one field: about sample_frac of the elements.
static GuardGeom sample_geom(const Geom& g, const vsz_params* p, double frac) {
    return region_geom(g, p, 1, frac);
}

static vsz_status sampling_layout(const vsz_params* p, double frac, GuardGeom* G, CountBufs* B) {
    if (!p || p->ndim < 1 || p->ndim > 3 || !(frac > 0.0) || frac > 1.0) return VSZ_ERR_INVALID_ARG;
    Geom g;
    vsz_params q = *p;
    q.block = 8;
    vsz_status st = make_geom(&q, &g);
    if (st != VSZ_OK) return st;
    *G = sample_geom(g, p, frac);
    vsz_params sub = *p;
    for (int k = 0; k < 3; ++k) sub.dims[k] = k < p->ndim ? G->dims[k] : 0;
    uint64_t nb_max = 0;
    size_t cws = 0;
    for (int slot = 0; slot < 4; ++slot) {
        const uint32_t b = class_block(p->ndim, slot);
        if (!b) continue;
        vsz_params pc = sub;
        pc.block = b;
        Geom gc;
        if ((st = make_geom(&pc, &gc)) != VSZ_OK) return st;
        nb_max = gc.nb > nb_max ? gc.nb : nb_max;
        const size_t w = ws_layout(gc, 0, 0).total;
        cws = w > cws ? w : cws;
    }
    const size_t front = G->whole ? 0 : (size_t)G->nsub * 4;
    *B = count_bufs(G->nsub, nb_max, p->radius, cws, front);
    return VSZ_OK;
}

size_t vsz_sampling_autotune_workspace_size(const vsz_params* p, double sample_frac) {
    GuardGeom G;
    CountBufs B;
    return sampling_layout(p, sample_frac, &G, &B) == VSZ_OK ? B.total : 0;
}

vsz_status vsz_sampling_autotune(const vsz_params* p, const float* d_x, double sample_frac, int iters,
                                 uint32_t* h_best_block, float* h_ms, uint64_t* h_sample_elems, void* d_ws,
                                 size_t ws_bytes, void* stream) {
    GuardGeom G;
    CountBufs B;
    vsz_status st = sampling_layout(p, sample_frac, &G, &B);
    if (st != VSZ_OK) return st;
    if (iters < 1 || iters > 100 || !h_best_block || !d_ws || ws_bytes < B.total || !aligned(d_ws, 256))
        return VSZ_ERR_INVALID_ARG;
    if (G.nsub > 0 && !d_x) return VSZ_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(s, &cs);
    if (e != cudaSuccess) return cuda_fail(e);
    if (cs != cudaStreamCaptureStatusNone) return VSZ_ERR_INVALID_ARG;
    char* ws = (char*)d_ws;
    const float* src = d_x;
    if (!G.whole) {
        float* sub = (float*)ws;
        TraceScope ts("sample_gather", s, G.nd, 0, G.nsub);
        const int grid = grid_for((const void*)k_gather_sample, 256, 0, 256 * 8, G.nsub);
        k_gather_sample<<<grid, 256, 0, s>>>(d_x, sub, G);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e);
        src = sub;
    }
    if (h_sample_elems) *h_sample_elems = G.nsub;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if ((e = cudaEventCreate(&e0)) != cudaSuccess) return cuda_fail(e);
    if ((e = cudaEventCreate(&e1)) != cudaSuccess) {
        cudaEventDestroy(e0);
        return cuda_fail(e);
    }
    vsz_compressed c;
    std::memset(&c, 0, sizeof c);
    c.codes = (uint16_t*)(ws + B.off_codes);
    c.pad = (int32_t*)(ws + B.off_pad);
    c.blk_off = (uint32_t*)(ws + B.off_blk);
    c.hdr = (vsz_header*)(ws + B.off_hdr);
    float best = INFINITY;
    uint32_t best_b = 0;
    for (int slot = 0; slot < 4 && st == VSZ_OK; ++slot) {
        const uint32_t b = class_block(p->ndim, slot);
        if (h_ms) h_ms[slot] = -1.0f;
        if (!b) continue;
        vsz_params pc = *p;
        for (int k = 0; k < 3; ++k) pc.dims[k] = k < p->ndim ? G.dims[k] : 0;
        pc.block = b;
        // one warm-up, then `iters` timed runs of the dual-quant on the sample
        if ((st = vsz_prequant_lorenzo(&pc, src, &c, ws + B.off_cws, B.cws_bytes, s)) != VSZ_OK) break;
        if ((e = cudaEventRecord(e0, s)) != cudaSuccess) { st = cuda_fail(e); break; }
        for (int it = 0; it < iters && st == VSZ_OK; ++it)
            st = vsz_prequant_lorenzo(&pc, src, &c, ws + B.off_cws, B.cws_bytes, s);
        if (st != VSZ_OK) break;
        if ((e = cudaEventRecord(e1, s)) != cudaSuccess || (e = cudaEventSynchronize(e1)) != cudaSuccess) {
            st = cuda_fail(e);
            break;
        }
        float ms = 0.0f;
        if ((e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) { st = cuda_fail(e); break; }
        ms /= (float)iters;
        if (h_ms) h_ms[slot] = ms;
        if (ms < best) {
            best = ms;
            best_b = b;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st == VSZ_OK) *h_best_block = best_b;
    return st;
}

vsz_status vsz_mlp_forward(const float* d_theta, const float* d_norm, const float* d_X, const uint32_t* d_mask, int n,
                           float* d_logits, int32_t* d_class, void* stream) {
    if (n < 0 || !d_theta || !d_norm || (n > 0 && (!d_X || !d_mask)) || (!d_logits && !d_class))
        return VSZ_ERR_INVALID_ARG;
    if (n == 0) return VSZ_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const int grid = n < 4 * num_sms() ? n : 4 * num_sms();
    TraceScope ts("mlp_forward", s, 0, 0, (uint64_t)n);
    k_mlp_forward<<<grid, 128, 0, s>>>(d_theta, d_norm, d_X, d_mask, n, d_logits, d_class);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? VSZ_OK : cuda_fail(e);
}

size_t vsz_mlp_grad_workspace_size(int batch) {
    if (batch <= 0) return 0;
    const size_t parts = (size_t)(batch + kSPC - 1) / kSPC;
    return parts * (kNP + 1) * sizeof(float);
}

vsz_status vsz_mlp_grad(const float* d_theta, const float* d_norm, const float* d_X, const int32_t* d_y,
                        const uint32_t* d_mask, const int32_t* d_idx, int batch, float* d_grad, float* d_loss,
                        void* d_ws, size_t ws_bytes, void* stream) {
    if (batch <= 0 || !d_theta || !d_norm || !d_X || !d_y || !d_mask || !d_grad) return VSZ_ERR_INVALID_ARG;
    if (!d_ws || ws_bytes < vsz_mlp_grad_workspace_size(batch) || !aligned(d_ws, 16)) return VSZ_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int parts = (batch + kSPC - 1) / kSPC;
    float* partial = (float*)d_ws;
    {
        TraceScope ts("mlp_grad", s, 0, 0, (uint64_t)batch);
        k_mlp_grad<<<parts, 128, 0, s>>>(d_theta, d_norm, d_X, d_y, d_mask, d_idx, batch, partial);
    }
    {
        TraceScope ts("mlp_reduce", s, 0, 0, (uint64_t)batch);
        k_mlp_reduce<<<(kNP + 1 + 255) / 256, 256, 0, s>>>(partial, parts, batch, d_grad, d_loss);
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? VSZ_OK : cuda_fail(e);
}

vsz_status vsz_mlp_adam(float* d_theta, const float* d_grad, float* d_m, float* d_v, int nparam, float lr, float beta1,
                        float beta2, float eps, int step, void* stream) {
    if (nparam <= 0 || !d_theta || !d_grad || !d_m || !d_v || step < 1) return VSZ_ERR_INVALID_ARG;
    if (!(beta1 >= 0.f && beta1 < 1.f && beta2 >= 0.f && beta2 < 1.f && eps > 0.f && lr >= 0.f))
        return VSZ_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const float c1 = (float)(1.0 / (1.0 - std::pow((double)beta1, (double)step)));
    const float c2 = (float)(1.0 / (1.0 - std::pow((double)beta2, (double)step)));
    TraceScope ts("adam", s, 0, 0, (uint64_t)nparam);
    k_adam<<<(nparam + 255) / 256, 256, 0, s>>>(d_theta, d_grad, d_m, d_v, nparam, lr, beta1, beta2, eps, c1, c2);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? VSZ_OK : cuda_fail(e);
}

}  // extern "C"
