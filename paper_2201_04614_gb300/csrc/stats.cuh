// stats.cuh -- error-bound resolution and block-wide reductions shared by
// the single-field and batch statistics kernels.
#pragma once

#include "common.cuh"

namespace vsz {

// Error-bound resolution (Sec. II-B), on the device so that relative mode
// needs no host round trip: eb_abs = eb, or eb * (max - min) over the finite
// values (eb itself when that range is zero or empty); 1/(2 eb_abs) and
// 2 eb_abs are formed in double and rounded once to float; the guard's bound
// is eb_abs rounded toward zero.
__device__ __forceinline__ void resolve_eb(vsz_header* h, double eb, bool rel, bool has, float xmin, float xmax) {
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

// After a range pass: resolve the relative error bound and record whether
// the whole field qualifies for the exact fp32 arithmetic of the compression
// walk (no NaN/Inf and every |fl(x * inv2eb)| < 2^20).  The product is
// monotone in x, so the extremes of x bound it for every element.
__device__ __forceinline__ void finish_range(WsHeader* w, vsz_header* h, double eb) {
    const unsigned l = atomicAdd(&w->xmin_ord, 0u);
    const unsigned u = atomicAdd(&w->xmax_ord, 0u);
    const bool has = l != 0xffffffffu;
    const float lo = has ? ord_to_float(l) : 0.0f, hi = has ? ord_to_float(u) : 0.0f;
    resolve_eb(h, eb, true, has, lo, hi);
    const float inv2eb = h->inv2eb;
    const bool small = fabsf(__fmul_rn(lo, inv2eb)) < 1048576.0f && fabsf(__fmul_rn(hi, inv2eb)) < 1048576.0f;
    w->fp32_ok = (has && atomicAdd(&w->nonfinite, 0u) == 0u && small) ? 1u : 0u;
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

}  // namespace vsz
