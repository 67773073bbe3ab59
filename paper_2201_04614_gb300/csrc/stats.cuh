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
