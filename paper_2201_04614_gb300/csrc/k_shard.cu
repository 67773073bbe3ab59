// k_shard.cu -- the per-rank steps of a field split across GPUs.
//
// Blocks are independent (Sec. III-A), so a field splits along dims[0] into
// slabs of whole blocks, one per rank, and each rank compresses its slab.
// Only three quantities cross slabs, each reduced over the ranks by the
// caller's collective between these calls:
//  - the finite value range, for a value-range relative error bound
//    (Sec. II-B): vsz_slab_range gives each slab's;
//  - the padding value of a global padding mode (Sec. IV-B-1): vsz_slab_qstats
//    gives each slab's sum, count and extremes of q under the field's eb;
//  - the lengths of the outlier and fixup lists, whose exclusive prefix over
//    the ranks places each slab's lists in the field's canonical order:
//    vsz_slab_rebase shifts a slab's indices and block offsets there.
// vsz_compress_slab compresses a slab with the field's eb and padding value.
#include <climits>

#include "common.cuh"
#include "memops.cuh"
#include "misc.cuh"
#include "stats.cuh"
#include "trace.cuh"

namespace vsz {

// Order-preserving encodings of the range while it is reduced, then the floats.
__global__ void k_slab_init(vsz_slab_stats* st, int range, int q) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (range) {
        reinterpret_cast<unsigned int*>(&st->xmin)[0] = 0xffffffffu;
        reinterpret_cast<unsigned int*>(&st->xmax)[0] = 0u;
        st->has_range = 0;
    }
    if (q) {
        st->qsum = 0;
        st->qmin = INT_MAX;
        st->qmax = INT_MIN;
    }
}

__global__ void __launch_bounds__(256) k_slab_range(const float* __restrict__ x, uint64_t n, vsz_slab_stats* st) {
    __shared__ unsigned int smu[32];
    unsigned int lo = 0xffffffffu, hi = 0u;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const float v = x[i];
        if (isfinite(v)) {
            const unsigned u = float_to_ord(v);
            lo = min(lo, u);
            hi = max(hi, u);
        }
    }
    lo = block_reduce(lo, OpMin(), smu, 0xffffffffu);
    hi = block_reduce(hi, OpMax(), smu, 0u);
    if (threadIdx.x == 0 && lo != 0xffffffffu) {
        atomicMin(reinterpret_cast<unsigned int*>(&st->xmin), lo);
        atomicMax(reinterpret_cast<unsigned int*>(&st->xmax), hi);
    }
}

__global__ void k_slab_range_final(vsz_slab_stats* st) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const unsigned int lo = reinterpret_cast<unsigned int*>(&st->xmin)[0];
    const unsigned int hi = reinterpret_cast<unsigned int*>(&st->xmax)[0];
    if (lo == 0xffffffffu) {  // no finite value
        st->xmin = 0.0f;
        st->xmax = 0.0f;
        st->has_range = 0;
    } else {
        st->xmin = ord_to_float(lo);
        st->xmax = ord_to_float(hi);
        st->has_range = 1;
    }
}

// Sum and extremes of q = rint(x * inv2eb) over every value (NaN gives 0,
// infinities saturate), as a global padding mode takes them.
__global__ void __launch_bounds__(256) k_slab_qstats(const float* __restrict__ x, uint64_t n, double eb_abs,
                                                     vsz_slab_stats* st) {
    // inv2eb exactly as the compression resolves it from eb_abs (reading R1)
    const float inv2eb = __double2float_rn(__ddiv_rn(1.0, __dmul_rn(2.0, eb_abs)));
    __shared__ long long sms[32];
    __shared__ int smi[32], sma[32];
    long long sm = 0;
    int mn = INT_MAX, mx = INT_MIN;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const int32_t q = prequant(x[i], inv2eb);
        sm += q;
        mn = min(mn, q);
        mx = max(mx, q);
    }
    sm = block_reduce(sm, OpAdd(), sms, 0ll);
    mn = block_reduce(mn, OpMin(), smi, INT_MAX);
    mx = block_reduce(mx, OpMax(), sma, INT_MIN);
    if (threadIdx.x == 0) {
        atomicAdd(reinterpret_cast<unsigned long long*>(&st->qsum), (unsigned long long)sm);
        atomicMin(&st->qmin, mn);
        atomicMax(&st->qmax, mx);
    }
}

// A slab's lists and block offsets moved to the field's canonical place.
__global__ void __launch_bounds__(256) k_slab_rebase(const vsz_header* hdr, uint32_t* out_idx, uint64_t out_cap,
                                                     uint32_t* fix_idx, uint64_t fix_cap, uint32_t* blk_off,
                                                     uint64_t nb, uint32_t elem_base, uint32_t out_base) {
    const uint64_t no = umin64(hdr->n_out, out_cap), nf = umin64(hdr->n_fix, fix_cap);
    const uint64_t step = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t i0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (uint64_t i = i0; i < no; i += step) out_idx[i] += elem_base;
    for (uint64_t i = i0; i < nf; i += step) fix_idx[i] += elem_base;
    for (uint64_t i = i0; i <= nb; i += step) blk_off[i] += out_base;
}

}  // namespace vsz

using namespace vsz;

extern "C" {

vsz_status vsz_slab_range(const float* d_x, uint64_t n, vsz_slab_stats* d_st, void* stream) {
    if (!d_st || (n > 0 && !d_x)) return VSZ_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    k_slab_init<<<1, 32, 0, s>>>(d_st, 1, 0);
    if (n > 0) {
        TraceScope ts("slab_range", s, 0, 0, n);
        const int grid = grid_for((const void*)k_slab_range, 256, 0, 256 * 16, n);
        k_slab_range<<<grid, 256, 0, s>>>(d_x, n, d_st);
    }
    k_slab_range_final<<<1, 32, 0, s>>>(d_st);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? VSZ_OK : cuda_fail(e);
}

vsz_status vsz_slab_qstats(const vsz_params* p, const float* d_x, vsz_slab_stats* d_st, void* stream) {
    Geom g;
    vsz_status st = make_geom(p, &g);
    if (st != VSZ_OK) return st;
    if (p->eb_mode != VSZ_EB_ABS || !d_st || (g.n > 0 && !d_x)) return VSZ_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    k_slab_init<<<1, 32, 0, s>>>(d_st, 0, 1);
    if (g.n > 0) {
        TraceScope ts("slab_qstats", s, g.nd, g.b, g.n);
        const int grid = grid_for((const void*)k_slab_qstats, 256, 0, 256 * 16, g.n);
        k_slab_qstats<<<grid, 256, 0, s>>>(d_x, g.n, p->eb, d_st);
    }
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? VSZ_OK : cuda_fail(e);
}

vsz_status vsz_slab_rebase(const vsz_params* p, const vsz_compressed* c, uint64_t elem_base, uint64_t out_base,
                           void* stream) {
    Geom g;
    vsz_status st = make_geom(p, &g);
    if (st != VSZ_OK) return st;
    if ((st = check_compressed(g, p, c)) != VSZ_OK) return st;
    if (elem_base >= (1ull << 32) || out_base >= (1ull << 32)) return VSZ_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    TraceScope ts("slab_rebase", s, g.nd, g.b, g.n);
    uint64_t work = c->out_cap > c->fix_cap ? c->out_cap : c->fix_cap;
    if (work < g.nb + 1) work = g.nb + 1;
    if (work > (1ull << 26)) work = 1ull << 26;
    const int grid = grid_for((const void*)k_slab_rebase, 256, 0, 256 * 8, work);
    k_slab_rebase<<<grid, 256, 0, s>>>(c->hdr, c->out_idx, c->out_cap, c->fix_idx, c->fix_cap, c->blk_off, g.nb,
                                       (uint32_t)elem_base, (uint32_t)out_base);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? VSZ_OK : cuda_fail(e);
}

}  // extern "C"
