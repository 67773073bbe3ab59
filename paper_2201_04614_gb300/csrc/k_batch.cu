// k_batch.cu -- many fields compressed together (vsz_batch_*).
//
// A batch is planned once: every field's geometry and workspace region, its
// class (rank, block edge, per-block padding or not), and device tables of
// per-field descriptors and prefix sums of work items.  Submitting it runs a
// fixed sequence of launches, whatever the number of fields:
//   k_batch_begin         one CTA per field: workspace and header set-up;
//   k_batch_range         value range of every relative-eb field, items of
//                         1M elements; the last item of a field resolves eb;
//   k_lorenzo_*_batch     per class, one persistent kernel drawing tiles of
//                         all the class's fields from one ticket;
//   k_batch_edge_stats    face statistics of every edge-padding field;
//   k_batch_origin_fix    block origins of every global- or edge-padding
//                         field, once its padding values are known;
//   k_batch_compact_scan  one CTA per field: chunk offsets and totals;
//   k_batch_compact_move  one CTA per chunk of any field: final placement.
// Reconstruction of the batch (once output buffers are set) is a second
// fixed sequence: one persistent inverse kernel per class (rank, block edge)
// drawing tiles of all the class's fields from one queue, then one fixup
// kernel over every field.  Each sequence can be captured into a CUDA graph
// once and replayed.
#include <algorithm>
#include <climits>
#include <cstring>
#include <map>
#include <tuple>
#include <vector>

#include "common.cuh"
#include "compact.cuh"
#include "misc.cuh"
#include "memops.cuh"
#include "stats.cuh"
#include "trace.cuh"

namespace vsz {

constexpr uint64_t kItemElems = 1ull << 18;  // elements per statistics work item
constexpr int kMaxClasses = 28;               // tickets in the batch header, per sequence
constexpr size_t kBatchHeader = 512;          // compression tickets, then reconstruction tickets
constexpr size_t kReconTickets = 256;         // byte offset of the reconstruction tickets
constexpr int kSplitCount = 60;               // header word: extra compaction items listed by the scan
static_assert(kReconTickets / 8 + kMaxClasses <= kSplitCount && (kSplitCount + 1) * 8 <= kBatchHeader,
              "batch header words");

struct BatchField {
    CompressArgs a;     // the field's pointers, geometry and workspace
    double eb;          // user error bound
    int32_t rel;        // value-range relative bound
    int32_t gpad;       // a global padding mode (its block origins wait for the origin pass)
    int32_t epad;       // an edge padding mode (the same, with per-block face scalars)
};

// Index of the last entry of prefix[0..n) that is <= v (prefix[0] == 0).
__device__ __forceinline__ int find_field(const uint64_t* __restrict__ prefix, int n, uint64_t v) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (prefix[mid] <= v) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// blockIdx.x: the field; blockIdx.y strides over its chunk sums; CTA (f, 0)
// sets the headers.
__global__ void __launch_bounds__(256) k_batch_begin(const BatchField* __restrict__ F,
                                                     unsigned long long* tickets) {
    const BatchField& b = F[blockIdx.x];
    const CompressArgs& a = b.a;
    const uint64_t i0 = (uint64_t)blockIdx.y * blockDim.x + threadIdx.x, stride = (uint64_t)gridDim.y * blockDim.x;
    for (uint64_t i = i0; i < a.g.nchunks; i += stride) a.chunks[i] = make_uint4(0, 0, 0, 0);
    if (blockIdx.y != 0) return;
    if (threadIdx.x == 0) {
        WsHeader* w = a.wsh;
        w->stage_out = 0;
        w->stage_fix = 0;
        w->qsum = 0;
        w->xmin_ord = 0xffffffffu;
        w->xmax_ord = 0u;
        w->qmin = INT_MAX;
        w->qmax = INT_MIN;
        w->done0 = 0;
        w->done1 = 0;
        w->nonfinite = 0;
        w->fp32_ok = 0;
        w->ticket = 0;
        vsz_header* h = const_cast<vsz_header*>(a.hdr);
        h->pad_global = 0;
        h->status = 0;
        h->recon_status = 0;
        h->reserved = 0;
        h->n_out = 0;
        h->n_fix = 0;
        if (!b.rel) resolve_eb(h, b.eb, false, false, 0.0f, 0.0f);
    }
    if (blockIdx.x == 0 && threadIdx.x < kMaxClasses) tickets[threadIdx.x] = 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) tickets[kSplitCount] = 0;
}

// Finite min/max of every relative-eb field; items of kItemElems elements.
__global__ void __launch_bounds__(256) k_batch_range(const BatchField* __restrict__ F, int nf,
                                                     const uint64_t* __restrict__ prefix, uint64_t nitems) {
    __shared__ unsigned int smu[32];
    __shared__ bool last;
    for (uint64_t item = blockIdx.x; item < nitems; item += gridDim.x) {
        const int f = find_field(prefix, nf, item);
        const BatchField& b = F[f];
        const uint64_t n = b.a.g.n;
        const uint64_t i0 = (item - prefix[f]) * kItemElems, i1 = umin64(n, i0 + kItemElems);
        const float* x = b.a.x;
        unsigned int lo = 0xffffffffu, hi = 0u;
        bool nf = false;
        auto take = [&](float v) {
            if (isfinite(v)) {
                const unsigned u = float_to_ord(v);
                lo = min(lo, u);
                hi = max(hi, u);
            } else {
                nf = true;
            }
        };
        if (b.a.vec) {
            // four 16-byte loads in flight per thread
            uint64_t i = i0 + 4 * threadIdx.x;
            for (; i + 12 * blockDim.x + 3 < i1; i += 16 * blockDim.x) {
                float4 v[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) v[u] = ld_stream_f4(x + i + 4 * u * blockDim.x);
#pragma unroll
                for (int u = 0; u < 4; ++u) { take(v[u].x); take(v[u].y); take(v[u].z); take(v[u].w); }
            }
            for (; i + 3 < i1; i += 4 * blockDim.x) {
                const float4 v = ld_stream_f4(x + i);
                take(v.x); take(v.y); take(v.z); take(v.w);
            }
            for (uint64_t k = i0 + ((i1 - i0) & ~3ull) + threadIdx.x; k < i1; k += blockDim.x) take(x[k]);
        } else {
            for (uint64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) take(x[i]);
        }
        nf = __syncthreads_or(nf) != 0;
        lo = block_reduce(lo, OpMin(), smu, 0xffffffffu);
        hi = block_reduce(hi, OpMax(), smu, 0u);
        if (threadIdx.x == 0) {
            WsHeader* w = b.a.wsh;
            if (nf) atomicOr(&w->nonfinite, 1u);
            if (lo != 0xffffffffu) {
                atomicMin(&w->xmin_ord, lo);
                atomicMax(&w->xmax_ord, hi);
            }
            __threadfence();
            last = atomicAdd(&w->done0, 1u) == (unsigned)(prefix[f + 1] - prefix[f] - 1);
            if (last) {
                __threadfence();
                finish_range(w, const_cast<vsz_header*>(b.a.hdr), b.eb);
            }
        }
        __syncthreads();
    }
}

// Global padding value of every global-padding field (one CTA per field).

// Face statistics of every edge-padding field: items are warp units (tiles,
// or 32 blocks in 1D), one warp each.
__global__ void __launch_bounds__(256) k_batch_edge_stats(const BatchField* __restrict__ F, int nf,
                                                          const uint64_t* __restrict__ prefix, uint64_t nitems) {
    const uint64_t nwarps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    for (uint64_t item = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); item < nitems;
         item += nwarps) {
        const int f = find_field(prefix, nf, item);
        edge_stats_unit(F[f].a, item - prefix[f], threadIdx.x & 31);
    }
}

// Origin pass of every global- or edge-padding field: items are blocks.
// Each warp takes 32 consecutive blocks: one search for the field of the
// first, then a step forward for lanes past that field's end.
// A warp takes kObWarp consecutive items (blocks of the class's global- or
// edge-padding fields, in field order), eight per lane: the field, its
// padding value and geometry once, then every lane's origin loads (and an
// edge field's face scalars) in flight together.  A range that runs into
// the next field goes item by item.
constexpr int kObLane = 8;
constexpr uint64_t kObWarp = 32 * kObLane;

__global__ void __launch_bounds__(256) k_batch_origin_fix(const BatchField* __restrict__ F, int nf,
                                                          const uint64_t* __restrict__ prefix, uint64_t nitems) {
    const int lane = threadIdx.x & 31;
    const uint64_t nwarps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    for (uint64_t w0 = ((uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * kObWarp; w0 < nitems;
         w0 += nwarps * kObWarp) {
        int f = 0;
        if (lane == 0) f = find_field(prefix, nf, w0);
        f = __shfl_sync(VSZ_FULL, f, 0);
        const uint64_t fb = prefix[f], fe = prefix[f + 1];
        if (w0 + kObWarp <= fe) {
            const CompressArgs& a = F[f].a;
            const bool ep = F[f].epad != 0;
            const int nd = a.g.nd;
            const int32_t Pg = ep ? 0 : global_pad_value(a);
            int32_t q0[kObLane], sc[kObLane][3];
#pragma unroll
            for (int u = 0; u < kObLane; ++u) {
                const uint64_t blk = w0 + (uint64_t)(u * 32 + lane) - fb;
                q0[u] = a.origin[blk];
#pragma unroll
                for (int k = 0; k < 3; ++k) sc[u][k] = (ep && k < nd) ? a.pad[blk * (uint64_t)nd + k] : 0;
            }
#pragma unroll
            for (int u = 0; u < kObLane; ++u) {
                const uint64_t blk = w0 + (uint64_t)(u * 32 + lane) - fb;
                if (!ep && blk == 0) const_cast<vsz_header*>(a.hdr)->pad_global = Pg;
                origin_fix_block(a, blk, q0[u], ep ? edge_origin_pred_r(sc[u][0], sc[u][1], sc[u][2], nd) : Pg);
            }
            continue;
        }
        for (int u = 0; u < kObLane; ++u) {
            const uint64_t item = w0 + (uint64_t)(u * 32 + lane);
            if (item >= nitems) break;
            int g = f;
            while (item >= prefix[g + 1]) ++g;
            const CompressArgs& a = F[g].a;
            const uint64_t blk = item - prefix[g];
            const int nd = a.g.nd;
            int32_t P;
            if (F[g].epad) {
                P = edge_origin_pred(a.pad + blk * (uint64_t)nd, nd);
            } else {
                P = global_pad_value(a);
                if (blk == 0) const_cast<vsz_header*>(a.hdr)->pad_global = P;
            }
            origin_fix_block(a, blk, a.origin[blk], P);
        }
    }
}

// One CTA per field: the chunk offsets and totals, then (a block-slot
// field) the extra compaction items of its dense chunks, {field, chunk *
// kSplit + split} for splits 1.., appended to `list`.
__global__ void __launch_bounds__(1024) k_batch_compact_scan(const BatchField* __restrict__ F, uint2* list,
                                                             unsigned long long* count) {
    const CompressArgs& a = F[blockIdx.x].a;
    compact_scan_body(a.chunks, a.g.nchunks, const_cast<vsz_header*>(a.hdr), a.blk_off, a.g.nb, a.out_cap,
                      a.fix_cap);
    if (!a.slots || !list) return;
    for (uint64_t c = threadIdx.x; c < a.g.nchunks; c += blockDim.x) {
        const uint32_t ns = chunk_splits(a.chunks[c].x);
        if (ns > 1) {
            const unsigned long long base = atomicAdd(count, (unsigned long long)(ns - 1));
            for (uint32_t sp = 1; sp < ns; ++sp)
                list[base + sp - 1] = make_uint2(blockIdx.x, (uint32_t)(c * kSplit + sp));
        }
    }
}

// Items: first the extra splits the scan listed (the heavy ones), then
// split 0 of every chunk of every field.
__global__ void __launch_bounds__(256, 3) k_batch_compact_move(const BatchField* __restrict__ F, int nf,
                                                            const uint64_t* __restrict__ prefix,
                                                            uint64_t nchunks, const uint2* __restrict__ list,
                                                            const unsigned long long* __restrict__ count) {
    const uint64_t nx = list ? *count : 0;
    for (uint64_t item = blockIdx.x; item < nx + nchunks; item += gridDim.x) {
        if (item < nx) {
            const uint2 it = list[item];
            compact_chunk_body_slots(it.y / kSplit, (int)(it.y % kSplit), F[it.x].a);
        } else {
            const uint64_t c = item - nx;
            const int f = find_field(prefix, nf, c);
            const CompressArgs& a = F[f].a;
            if (a.slots) compact_chunk_body_slots(c - prefix[f], 0, a);
            else compact_chunk_body(c - prefix[f], a);
        }
        __syncthreads();
    }
}

// Fixups of every field of a batch (blockIdx.x: field; blockIdx.y strides
// over its list): the verbatim values of the error-bound guard.
struct BatchFix {
    const vsz_header* hdr;
    const uint32_t* fix_idx;
    const uint32_t* fix_bits;
    uint64_t fix_cap;
    float* out;
    uint64_t n;
};

__global__ void __launch_bounds__(256) k_batch_fixups(const BatchFix* __restrict__ F) {
    const BatchFix& f = F[blockIdx.x];
    if (!f.out) return;
    const uint64_t cnt = umin64(f.hdr->n_fix, f.fix_cap);
    for (uint64_t i = (uint64_t)blockIdx.y * blockDim.x + threadIdx.x; i < cnt; i += (uint64_t)gridDim.y * blockDim.x) {
        const uint32_t j = f.fix_idx[i];
        if (j < f.n) f.out[j] = __uint_as_float(f.fix_bits[i]);
    }
}

}  // namespace vsz

// ---------------------------------------------------------------------------
// Host side.

using namespace vsz;

struct BatchClass {
    int nd;
    uint32_t b;
    int pk;                        // 0 zero, 1 per-block, 2 global, 3 edge padding (compression)
    int kind = 0;                  // 0 compression, 1 reconstruction
    std::vector<int> fields;       // indices into the batch
    CompressArgs* d_args = nullptr;
    ReconArgs* d_rargs = nullptr;
    uint64_t* d_prefix = nullptr;
    uint64_t total_tiles = 0;
    // a global or edge padding class: its fields' descriptors and the
    // prefixes of their blocks and face-statistics units (the origin pass
    // and edge statistics run on the class's own branch, after its kernel)
    BatchField* d_bfields = nullptr;
    uint64_t* d_ob_prefix = nullptr;
    uint64_t* d_edge_prefix = nullptr;
    uint64_t origin_items = 0, edge_items = 0;
    LaunchShape shape;             // launch shape of the class kernel (autotuned or set)
    float ms_best = 0.0f, ms_default = 0.0f;  // autotuner measurements
};

struct vsz_batch_st {
    int n = 0;
    std::vector<vsz_field_job> jobs;
    std::vector<BatchField> fields;
    std::vector<BatchClass> classes;
    BatchField* d_fields = nullptr;
    uint64_t* d_range_prefix = nullptr;
    uint64_t* d_chunk_prefix = nullptr;
    uint2* d_split = nullptr;            // extra compaction items of dense chunks (filled by the scan)
    uint64_t split_cap = 0;
    uint64_t range_items = 0, chunks = 0;
    unsigned begin_y = 1;                // CTAs per field of the begin kernel
    unsigned long long* tickets = nullptr;  // in the caller's workspace
    bool use_graph = false;
    cudaGraphExec_t exec = nullptr;
    bool concurrent = false;             // class kernels as parallel branches
    std::vector<cudaStream_t> side;      // one per class after the first (concurrent mode)
    std::vector<cudaEvent_t> ev;         // fork event, then one join event per side stream
    // reconstruction (after vsz_batch_set_outputs)
    std::vector<BatchClass> rclasses;
    BatchFix* d_fix = nullptr;
    bool rconcurrent = false;
    cudaGraphExec_t rexec = nullptr;
};

// Class of a job: (rank, block edge, padding kind 0 zero / 1 per block / 2 global / 3 edge).
using ClassKey = std::tuple<int, uint32_t, int>;
static ClassKey class_key(const vsz_field_job& j, const Geom& g) {
    const int32_t m = j.params.pad;
    return std::make_tuple(g.nd, g.b, is_block_pad(m) ? 1 : is_global_pad(m) ? 2 : is_edge_pad(m) ? 3 : 0);
}

// Workspace of a batch: the header, then every field's workspace (2D/3D
// fields with block-slot staging).
static size_t batch_layout(const vsz_field_job* jobs, int n, std::vector<size_t>* offs, std::vector<Geom>* geoms) {
    size_t off = kBatchHeader;  // batch header: class tickets
    for (int i = 0; i < n; ++i) {
        Geom g;
        if (make_geom(&jobs[i].params, &g) != VSZ_OK) return 0;
        const WsLayout L = ws_layout(g, jobs[i].out.out_cap, jobs[i].out.fix_cap, true);
        if (offs) offs->push_back(off);
        if (geoms) geoms->push_back(g);
        off = align256(off + L.total);
    }
    return off;
}

static void free_recon(vsz_batch_st* b) {
    if (b->rexec) cudaGraphExecDestroy(b->rexec);
    b->rexec = nullptr;
    for (BatchClass& c : b->rclasses) {
        if (c.d_rargs) cudaFree(c.d_rargs);
        if (c.d_prefix) cudaFree(c.d_prefix);
    }
    b->rclasses.clear();
    if (b->d_fix) cudaFree(b->d_fix);
    b->d_fix = nullptr;
}

static void free_batch(vsz_batch_st* b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    free_recon(b);  // also the reconstruction graph
    for (cudaStream_t t : b->side) cudaStreamDestroy(t);
    for (cudaEvent_t e : b->ev) cudaEventDestroy(e);
    for (BatchClass& c : b->classes) {
        if (c.d_args) cudaFree(c.d_args);
        if (c.d_prefix) cudaFree(c.d_prefix);
        if (c.d_bfields) cudaFree(c.d_bfields);
        if (c.d_ob_prefix) cudaFree(c.d_ob_prefix);
        if (c.d_edge_prefix) cudaFree(c.d_edge_prefix);
    }
    if (b->d_fields) cudaFree(b->d_fields);
    if (b->d_range_prefix) cudaFree(b->d_range_prefix);
    if (b->d_chunk_prefix) cudaFree(b->d_chunk_prefix);
    if (b->d_split) cudaFree(b->d_split);
    delete b;
}

template <typename T>
static cudaError_t upload(T** dst, const std::vector<T>& v) {
    cudaError_t e = lib_malloc((void**)dst, sizeof(T) * (v.empty() ? 1 : v.size()));
    if (e != cudaSuccess) return e;
    if (!v.empty()) e = cudaMemcpy(*dst, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice);
    return e;
}

// Side streams and fork/join events of the concurrent mode (created once).
static cudaError_t ensure_side_streams(vsz_batch_st* b) {
    const size_t nc = std::max(b->classes.size(), b->rclasses.size());
    const size_t want = nc ? nc - 1 : 0;
    while (b->side.size() < want) {
        cudaStream_t t = nullptr;
        const cudaError_t e = cudaStreamCreateWithFlags(&t, cudaStreamNonBlocking);
        if (e != cudaSuccess) return e;
        b->side.push_back(t);
    }
    while (b->ev.size() < want + 1) {
        cudaEvent_t v = nullptr;
        const cudaError_t e = cudaEventCreateWithFlags(&v, cudaEventDisableTiming);
        if (e != cudaSuccess) return e;
        b->ev.push_back(v);
    }
    return cudaSuccess;
}

static unsigned long long* recon_tickets(vsz_batch_st* b) {
    return (unsigned long long*)((char*)b->tickets + kReconTickets);
}

static cudaError_t launch_rclass(vsz_batch_st* b, size_t c, cudaStream_t s) {
    BatchClass& k = b->rclasses[c];
    TraceScope ts("batch_recon", s, k.nd, k.b);
    unsigned long long* t = recon_tickets(b) + c;
    return k.nd == 1 ? launch_recon_batch_1d(k.b, k.d_rargs, k.d_prefix, (int)k.fields.size(), k.total_tiles, t,
                                             k.shape, s)
         : k.nd == 2 ? launch_recon_batch_2d(k.b, k.d_rargs, k.d_prefix, (int)k.fields.size(), k.total_tiles, t,
                                             k.shape, s)
                     : launch_recon_batch_3d(k.b, k.d_rargs, k.d_prefix, (int)k.fields.size(), k.total_tiles, t,
                                             k.shape, s);
}

// The deferred block origins of a global or edge padding class, once its
// kernel is done: face statistics of its edge-padding fields, then the
// origin pass over its fields' blocks (on the class's stream).
static cudaError_t launch_class_origins(vsz_batch_st* b, size_t c, cudaStream_t s) {
    const BatchClass& k = b->classes[c];
    const int nf = (int)k.fields.size();
    if (k.edge_items) {
        TraceScope ts("batch_edge_stats", s, k.nd, k.b);
        const int grid = grid_for((const void*)k_batch_edge_stats, 256, 0, 8, k.edge_items);
        k_batch_edge_stats<<<grid, 256, 0, s>>>(k.d_bfields, nf, k.d_edge_prefix, k.edge_items);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (k.origin_items) {
        TraceScope ts("batch_origin_fix", s, k.nd, k.b);
        const int grid = grid_for((const void*)k_batch_origin_fix, 256, 0, 8 * kObWarp, k.origin_items);
        k_batch_origin_fix<<<grid, 256, 0, s>>>(k.d_bfields, nf, k.d_ob_prefix, k.origin_items);
        return cudaGetLastError();
    }
    return cudaSuccess;
}

static cudaError_t launch_class(vsz_batch_st* b, size_t c, cudaStream_t s) {
    BatchClass& k = b->classes[c];
    TraceScope ts(k.pk == 1 ? "batch_lorenzo_bp" : k.pk == 2 ? "batch_lorenzo_gp" : k.pk == 3 ? "batch_lorenzo_ep"
                                                                                             : "batch_lorenzo",
                  s, k.nd, k.b);
    return k.nd == 1 ? launch_lorenzo_batch_1d(k.b, k.pk, k.d_args, k.d_prefix, (int)k.fields.size(), k.total_tiles,
                                               b->tickets + c, k.shape, s)
         : k.nd == 2 ? launch_lorenzo_batch_2d(k.b, k.pk, k.d_args, k.d_prefix, (int)k.fields.size(), k.total_tiles,
                                               b->tickets + c, k.shape, s)
                     : launch_lorenzo_batch_3d(k.b, k.pk, k.d_args, k.d_prefix, (int)k.fields.size(), k.total_tiles,
                                               b->tickets + c, k.shape, s);
}

// Optional events around one class kernel (the autotuner's measurement).
struct ClassTimer {
    int kind = 0;  // 0 compression, 1 reconstruction
    int cls = -1;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
};

// The class kernels of one sequence (kind 0: compression, 1: reconstruction),
// one after another, or as parallel branches forked from `s` and joined back.
static vsz_status run_classes(vsz_batch_st* b, int kind, cudaStream_t s, const ClassTimer* tm) {
    std::vector<BatchClass>& cls = kind ? b->rclasses : b->classes;
    const bool conc = kind ? b->rconcurrent : b->concurrent;
    auto launch = [&](size_t c, cudaStream_t t) { return kind ? launch_rclass(b, c, t) : launch_class(b, c, t); };
    auto post = [&](size_t c, cudaStream_t t) { return kind ? cudaSuccess : launch_class_origins(b, c, t); };
    cudaError_t e;
    std::vector<size_t> run;
    for (size_t c = 0; c < cls.size(); ++c)
        if (cls[c].total_tiles) run.push_back(c);
    if (conc && run.size() > 1 && !tm) {
        // the first class on `s`, every other on its own side stream
        if ((e = ensure_side_streams(b)) != cudaSuccess) return cuda_fail(e);
        if ((e = cudaEventRecord(b->ev[0], s)) != cudaSuccess) return cuda_fail(e);
        for (size_t i = 1; i < run.size(); ++i)
            if ((e = cudaStreamWaitEvent(b->side[i - 1], b->ev[0], 0)) != cudaSuccess) return cuda_fail(e);
        for (size_t i = 0; i < run.size(); ++i) {
            if ((e = launch(run[i], i == 0 ? s : b->side[i - 1])) != cudaSuccess) return cuda_fail(e);
            if ((e = post(run[i], i == 0 ? s : b->side[i - 1])) != cudaSuccess) return cuda_fail(e);
        }
        for (size_t i = 1; i < run.size(); ++i) {
            if ((e = cudaEventRecord(b->ev[i], b->side[i - 1])) != cudaSuccess) return cuda_fail(e);
            if ((e = cudaStreamWaitEvent(s, b->ev[i], 0)) != cudaSuccess) return cuda_fail(e);
        }
        return VSZ_OK;
    }
    for (size_t c : run) {
        const bool timed = tm && tm->kind == kind && tm->cls == (int)c;
        if (timed && (e = cudaEventRecord(tm->e0, s)) != cudaSuccess) return cuda_fail(e);
        if ((e = launch(c, s)) != cudaSuccess) return cuda_fail(e);
        if (timed && (e = cudaEventRecord(tm->e1, s)) != cudaSuccess) return cuda_fail(e);
        if ((e = post(c, s)) != cudaSuccess) return cuda_fail(e);
    }
    return VSZ_OK;
}

static vsz_status launch_recon_sequence(vsz_batch_st* b, cudaStream_t s, const ClassTimer* tm = nullptr) {
    cudaError_t e = cudaMemsetAsync(recon_tickets(b), 0, kMaxClasses * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return cuda_fail(e);
    const vsz_status st = run_classes(b, 1, s, tm);
    if (st != VSZ_OK) return st;
    TraceScope ts("batch_fixups", s);
    // enough CTAs per field for its list capacity (fields with few fixups
    // leave most of them idle at once)
    uint64_t fcap = 0;
    for (const vsz_field_job& j : b->jobs) fcap = j.out.fix_cap > fcap ? j.out.fix_cap : fcap;
    const unsigned fy = (unsigned)umin64(256, umin64(65535, (fcap + 2047) / 2048 + 1));
    k_batch_fixups<<<dim3((unsigned)b->n, fy), 256, 0, s>>>(b->d_fix);
    return (e = cudaGetLastError()) == cudaSuccess ? VSZ_OK : cuda_fail(e);
}

static vsz_status launch_sequence(vsz_batch_st* b, cudaStream_t s, const ClassTimer* tm = nullptr) {
    cudaError_t e;
    {
        TraceScope ts("batch_begin", s);
        k_batch_begin<<<dim3((unsigned)b->n, b->begin_y), 256, 0, s>>>(b->d_fields, b->tickets);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return cuda_fail(e);
    if (b->range_items) {
        TraceScope ts("batch_range", s);
        const int grid = grid_for((const void*)k_batch_range, 256, 0, 1, b->range_items);
        k_batch_range<<<grid, 256, 0, s>>>(b->d_fields, b->n, b->d_range_prefix, b->range_items);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e);
    }
    {
        // forked after the range pass, joined before the compaction (each
        // global or edge padding class runs its origin pass on its branch)
        const vsz_status st = run_classes(b, 0, s, tm);
        if (st != VSZ_OK) return st;
    }
    {
        TraceScope ts("batch_compact_scan", s);
        k_batch_compact_scan<<<b->n, 1024, 0, s>>>(b->d_fields, b->d_split, b->tickets + kSplitCount);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e);
    }
    if (b->chunks) {
        TraceScope ts("batch_compact_move", s);
        const int grid = grid_for((const void*)k_batch_compact_move, 256, 0, 1, b->chunks + b->split_cap);
        k_batch_compact_move<<<grid, 256, 0, s>>>(b->d_fields, b->n, b->d_chunk_prefix, b->chunks, b->d_split,
                                                  b->tickets + kSplitCount);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e);
    }
    return VSZ_OK;
}

extern "C" {

size_t vsz_batch_workspace_size(const vsz_field_job* jobs, int njobs) {
    if (!jobs || njobs <= 0) return 0;
    return batch_layout(jobs, njobs, nullptr, nullptr);
}

vsz_status vsz_batch_create(const vsz_field_job* jobs, int njobs, void* d_ws, size_t ws_bytes, int use_graph,
                            vsz_batch* out) {
    if (!jobs || njobs <= 0 || !out || !d_ws || !aligned(d_ws, 256)) return VSZ_ERR_INVALID_ARG;
    *out = nullptr;
    std::vector<size_t> offs;
    std::vector<Geom> geoms;
    for (int i = 0; i < njobs; ++i) {
        Geom g;
        vsz_status st = make_geom(&jobs[i].params, &g);
        if (st != VSZ_OK) return st;
        if ((st = check_compressed(g, &jobs[i].params, &jobs[i].out)) != VSZ_OK) return st;
        if (g.n > 0 && !jobs[i].d_x) return VSZ_ERR_INVALID_ARG;
    }
    const size_t need = batch_layout(jobs, njobs, &offs, &geoms);
    if (!need || ws_bytes < need) return VSZ_ERR_INVALID_ARG;

    vsz_batch_st* b = new vsz_batch_st();
    b->n = njobs;
    b->jobs.assign(jobs, jobs + njobs);
    b->use_graph = use_graph != 0;
    char* ws = (char*)d_ws;
    b->tickets = (unsigned long long*)ws;
    std::vector<uint64_t> rp(1, 0), cp(1, 0);
    std::map<ClassKey, int> cls;
    for (int i = 0; i < njobs; ++i) {
        const vsz_field_job& j = jobs[i];
        const Geom& g = geoms[i];
        const WsLayout L = ws_layout(g, j.out.out_cap, j.out.fix_cap, true);
        char* fw = ws + offs[i];
        BatchField bf;
        std::memset(&bf, 0, sizeof bf);
        CompressArgs& a = bf.a;
        a.x = j.d_x;
        a.codes = j.out.codes;
        a.pad = j.out.pad;
        a.blk_off = j.out.blk_off;
        a.hdr = j.out.hdr;
        a.wsh = (WsHeader*)fw;
        a.tiles = (uint4*)(fw + L.tiles);
        a.chunks = (uint4*)(fw + L.chunks);
        a.stage_out = (uint2*)(fw + L.stage_out);
        a.stage_fix = (uint2*)(fw + L.stage_fix);
        if (defers_origin(j.params.pad)) {
            a.origin = (int32_t*)(fw + L.origin);
            a.oflag = (uint8_t*)(fw + L.oflag);
        }
        a.out_idx = j.out.out_idx;
        a.out_delta = j.out.out_delta;
        a.fix_idx = j.out.fix_idx;
        a.fix_bits = j.out.fix_bits;
        a.out_cap = j.out.out_cap;
        a.fix_cap = j.out.fix_cap;
        a.g = g;
        a.R = (int32_t)j.params.radius;
        a.pad_mode = j.params.pad;
        a.vec = (aligned(j.d_x, 16) && aligned(j.out.codes, 16) && (g.nd == 1 || g.nx % 4 == 0)) ? 1 : 0;
        bf.eb = j.params.eb;
        bf.rel = j.params.eb_mode == VSZ_EB_REL;
        bf.gpad = is_global_pad(j.params.pad) ? 1 : 0;
        bf.epad = is_edge_pad(j.params.pad) ? 1 : 0;
        a.blk_in = a.blk_off;
        if (g.nd >= 2) {  // block-slot staging
            a.slots = a.stage_out;
            a.blk_in = (uint32_t*)(fw + L.blkin);
        }
        b->fields.push_back(bf);
        const uint64_t items = (g.n + kItemElems - 1) / kItemElems;
        rp.push_back(rp.back() + (bf.rel ? (items ? items : 1) : 0));
        cp.push_back(cp.back() + g.nchunks);
        b->begin_y = (unsigned)umax64(b->begin_y, umin64(16, (g.nchunks + 4095) / 4096));
        const ClassKey key = class_key(j, g);
        const int pk = std::get<2>(key);
        auto it = cls.find(key);
        if (it == cls.end()) {
            BatchClass c;
            c.nd = g.nd;
            c.b = g.b;
            c.pk = pk;
            b->classes.push_back(c);
            it = cls.emplace(key, (int)b->classes.size() - 1).first;
        }
        b->classes[it->second].fields.push_back(i);
    }
    if ((int)b->classes.size() > kMaxClasses) { free_batch(b); return VSZ_ERR_UNSUPPORTED; }
    b->range_items = rp.back();
    b->chunks = cp.back();
    cudaError_t e = upload(&b->d_fields, b->fields);
    if (e == cudaSuccess) e = upload(&b->d_range_prefix, rp);
    if (e == cudaSuccess) e = upload(&b->d_chunk_prefix, cp);
    for (const BatchField& bf : b->fields)
        if (bf.a.slots) b->split_cap += bf.a.g.nchunks * (kSplit - 1);
    if (e == cudaSuccess && b->split_cap) e = lib_malloc((void**)&b->d_split, sizeof(uint2) * b->split_cap);
    for (BatchClass& c : b->classes) {
        if (e != cudaSuccess) break;
        std::vector<CompressArgs> args;
        std::vector<BatchField> bfs;
        std::vector<uint64_t> pre(1, 0), qp(1, 0), ep(1, 0);
        for (int i : c.fields) {
            const BatchField& bf = b->fields[i];
            args.push_back(bf.a);
            bfs.push_back(bf);
            pre.push_back(pre.back() + bf.a.g.ntiles);
            qp.push_back(qp.back() + (bf.gpad || bf.epad ? bf.a.g.nb : 0));
            ep.push_back(ep.back() + (bf.epad ? edge_units(bf.a.g) : 0));
        }
        c.total_tiles = pre.back();
        c.origin_items = qp.back();
        c.edge_items = ep.back();
        e = upload(&c.d_args, args);
        if (e == cudaSuccess) e = upload(&c.d_prefix, pre);
        if (e == cudaSuccess && c.origin_items) e = upload(&c.d_bfields, bfs);
        if (e == cudaSuccess && c.origin_items) e = upload(&c.d_ob_prefix, qp);
        if (e == cudaSuccess && c.edge_items) e = upload(&c.d_edge_prefix, ep);
    }
    if (e != cudaSuccess) {
        free_batch(b);
        return cuda_fail(e);
    }
    *out = b;
    return VSZ_OK;
}

vsz_status vsz_batch_submit(vsz_batch b, void* stream) {
    if (!b) return VSZ_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (!b->use_graph || s == nullptr || s == cudaStreamLegacy || Tracer::get().on()) return launch_sequence(b, s);
    if (!b->exec) {
        cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_fail(e);
        const vsz_status st = launch_sequence(b, s);
        cudaGraph_t graph = nullptr;
        e = cudaStreamEndCapture(s, &graph);
        if (st != VSZ_OK) {
            if (graph) cudaGraphDestroy(graph);
            return st;
        }
        if (e != cudaSuccess) return cuda_fail(e);
        e = cudaGraphInstantiate(&b->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            b->exec = nullptr;
            return cuda_fail(e);
        }
    }
    const cudaError_t e = cudaGraphLaunch(b->exec, s);
    return e == cudaSuccess ? VSZ_OK : cuda_fail(e);
}

vsz_status vsz_batch_set_outputs(vsz_batch b, float* const* h_xhat) {
    if (!b || !h_xhat) return VSZ_ERR_INVALID_ARG;
    for (int i = 0; i < b->n; ++i)
        if (b->fields[i].a.g.n > 0 && !h_xhat[i]) return VSZ_ERR_INVALID_ARG;
    free_recon(b);
    std::map<std::pair<int, uint32_t>, int> cls;
    std::vector<BatchFix> fix((size_t)b->n);
    std::vector<ReconArgs> ra((size_t)b->n);
    for (int i = 0; i < b->n; ++i) {
        const vsz_field_job& j = b->jobs[i];
        const Geom& g = b->fields[i].a.g;
        ReconArgs& a = ra[i];
        std::memset(&a, 0, sizeof a);
        a.codes = j.out.codes;
        a.pad = j.out.pad;
        a.blk_off = j.out.blk_off;
        a.out_idx = j.out.out_idx;
        a.out_delta = j.out.out_delta;
        a.out_cap = j.out.out_cap;
        a.ticket = nullptr;
        a.hdr = j.out.hdr;
        a.out = h_xhat[i];
        a.g = g;
        a.R = (int32_t)j.params.radius;
        a.pad_mode = j.params.pad;
        a.vec = (aligned(j.out.codes, 16) && aligned(h_xhat[i], 16) && (g.nd == 1 || g.nx % 4 == 0)) ? 1 : 0;
        fix[i] = BatchFix{j.out.hdr, j.out.fix_idx, j.out.fix_bits, j.out.fix_cap,
                          g.n > 0 && j.out.fix_cap > 0 ? h_xhat[i] : nullptr, g.n};
        if (!g.ntiles) continue;
        const auto key = std::make_pair(g.nd, g.b);
        auto it = cls.find(key);
        if (it == cls.end()) {
            BatchClass c;
            c.nd = g.nd;
            c.b = g.b;
            c.pk = 0;
            c.kind = 1;
            b->rclasses.push_back(c);
            it = cls.emplace(key, (int)b->rclasses.size() - 1).first;
        }
        b->rclasses[it->second].fields.push_back(i);
    }
    cudaError_t e = upload(&b->d_fix, fix);
    for (BatchClass& c : b->rclasses) {
        if (e != cudaSuccess) break;
        std::vector<ReconArgs> args;
        std::vector<uint64_t> pre(1, 0);
        for (int i : c.fields) {
            args.push_back(ra[i]);
            pre.push_back(pre.back() + ra[i].g.ntiles);
        }
        c.total_tiles = pre.back();
        e = upload(&c.d_rargs, args);
        if (e == cudaSuccess) e = upload(&c.d_prefix, pre);
    }
    if (e != cudaSuccess) {
        free_recon(b);
        return cuda_fail(e);
    }
    return VSZ_OK;
}

vsz_status vsz_batch_reconstruct(vsz_batch b, void* stream) {
    if (!b || !b->d_fix) return VSZ_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (!b->use_graph || s == nullptr || s == cudaStreamLegacy || Tracer::get().on())
        return launch_recon_sequence(b, s);
    if (!b->rexec) {
        cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_fail(e);
        const vsz_status st = launch_recon_sequence(b, s);
        cudaGraph_t graph = nullptr;
        e = cudaStreamEndCapture(s, &graph);
        if (st != VSZ_OK) {
            if (graph) cudaGraphDestroy(graph);
            return st;
        }
        if (e != cudaSuccess) return cuda_fail(e);
        e = cudaGraphInstantiate(&b->rexec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            b->rexec = nullptr;
            return cuda_fail(e);
        }
    }
    const cudaError_t e = cudaGraphLaunch(b->rexec, s);
    return e == cudaSuccess ? VSZ_OK : cuda_fail(e);
}

int vsz_batch_num_classes(vsz_batch b) { return b ? (int)(b->classes.size() + b->rclasses.size()) : 0; }

// Class c of the combined list: compression classes, then reconstruction ones.
static BatchClass* class_at(vsz_batch_st* b, int c) {
    if (!b || c < 0) return nullptr;
    if ((size_t)c < b->classes.size()) return &b->classes[c];
    c -= (int)b->classes.size();
    return (size_t)c < b->rclasses.size() ? &b->rclasses[c] : nullptr;
}

vsz_status vsz_batch_get_class(vsz_batch b, int c, vsz_batch_class* out) {
    const BatchClass* k = class_at(b, c);
    if (!k || !out) return VSZ_ERR_INVALID_ARG;
    std::memset(out, 0, sizeof *out);
    out->ndim = k->nd;
    out->block = k->b;
    out->pad_kind = k->pk;
    out->nfields = (int32_t)k->fields.size();
    out->tiles = k->total_tiles;
    out->warps = k->shape.warps;
    out->ctas_per_sm = k->shape.ctas;
    out->ms = k->ms_best;
    out->ms_default = k->ms_default;
    out->concurrent = (k->kind ? b->rconcurrent : b->concurrent) ? 1 : 0;
    out->kind = k->kind;
    return VSZ_OK;
}

static void drop_graphs(vsz_batch_st* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
    if (b->rexec) cudaGraphExecDestroy(b->rexec);
    b->rexec = nullptr;
}

static int class_occupancy(const BatchClass& k, int warps) {
    int occ = 0;
    const LaunchShape sh{warps, 0};
    cudaError_t e;
    if (k.kind == 0)
        e = k.nd == 1 ? launch_lorenzo_batch_1d(k.b, k.pk, nullptr, nullptr, 0, 0, nullptr, sh, nullptr, &occ)
          : k.nd == 2 ? launch_lorenzo_batch_2d(k.b, k.pk, nullptr, nullptr, 0, 0, nullptr, sh, nullptr, &occ)
                      : launch_lorenzo_batch_3d(k.b, k.pk, nullptr, nullptr, 0, 0, nullptr, sh, nullptr, &occ);
    else
        e = k.nd == 1 ? launch_recon_batch_1d(k.b, nullptr, nullptr, 0, 0, nullptr, sh, nullptr, &occ)
          : k.nd == 2 ? launch_recon_batch_2d(k.b, nullptr, nullptr, 0, 0, nullptr, sh, nullptr, &occ)
                      : launch_recon_batch_3d(k.b, nullptr, nullptr, 0, 0, nullptr, sh, nullptr, &occ);
    return e == cudaSuccess ? occ : 0;
}

vsz_status vsz_batch_set_shape(vsz_batch b, int c, int warps, int ctas_per_sm) {
    BatchClass* k = class_at(b, c);
    if (!k) return VSZ_ERR_INVALID_ARG;
    if (!(warps == 0 || warps == 2 || warps == 4 || warps == 8) || ctas_per_sm < 0 || ctas_per_sm > 64)
        return VSZ_ERR_INVALID_ARG;
    if (class_occupancy(*k, warps) < 1) return VSZ_ERR_UNSUPPORTED;
    k->shape = LaunchShape{warps, ctas_per_sm};
    drop_graphs(b);
    return VSZ_OK;
}

vsz_status vsz_batch_set_concurrent(vsz_batch b, int on) {
    if (!b) return VSZ_ERR_INVALID_ARG;
    b->concurrent = b->rconcurrent = on != 0;
    drop_graphs(b);
    return VSZ_OK;
}

vsz_status vsz_batch_set_concurrent_each(vsz_batch b, int compress_on, int reconstruct_on) {
    if (!b) return VSZ_ERR_INVALID_ARG;
    b->concurrent = compress_on != 0;
    b->rconcurrent = reconstruct_on != 0;
    drop_graphs(b);
    return VSZ_OK;
}

vsz_status vsz_batch_autotune(vsz_batch b, void* stream, int reps) {
    if (!b || reps < 1 || reps > 50) return VSZ_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(s, &cs);
    if (e != cudaSuccess) return cuda_fail(e);
    if (cs != cudaStreamCaptureStatusNone) return VSZ_ERR_INVALID_ARG;
    drop_graphs(b);
    ClassTimer tm;
    if ((e = cudaEventCreate(&tm.e0)) != cudaSuccess) return cuda_fail(e);
    if ((e = cudaEventCreate(&tm.e1)) != cudaSuccess) {
        cudaEventDestroy(tm.e0);
        return cuda_fail(e);
    }
    // median device time of `reps` runs of a sequence (kind 0 compression,
    // 1 reconstruction), with events around class `cls` or, when cls < 0,
    // around the whole sequence
    // A whole sequence (cls < 0) of a graph plan is timed as the plan runs
    // it: its graph is captured again for the current shapes and replayed.
    const bool graphs = b->use_graph && s != nullptr && s != cudaStreamLegacy && !Tracer::get().on();
    auto measure = [&](int kind, int cls, float* ms) -> vsz_status {
        std::vector<float> t;
        if (cls < 0 && graphs) {
            drop_graphs(b);
            const vsz_status sw = kind ? vsz_batch_reconstruct(b, s) : vsz_batch_submit(b, s);  // builds the graph
            if (sw != VSZ_OK) return sw;
            for (int r = 0; r < reps; ++r) {
                cudaError_t e2 = cudaEventRecord(tm.e0, s);
                if (e2 != cudaSuccess) return cuda_fail(e2);
                const vsz_status st2 = kind ? vsz_batch_reconstruct(b, s) : vsz_batch_submit(b, s);
                if (st2 != VSZ_OK) return st2;
                if ((e2 = cudaEventRecord(tm.e1, s)) != cudaSuccess) return cuda_fail(e2);
                if ((e2 = cudaEventSynchronize(tm.e1)) != cudaSuccess) return cuda_fail(e2);
                float v = 0.0f;
                if ((e2 = cudaEventElapsedTime(&v, tm.e0, tm.e1)) != cudaSuccess) return cuda_fail(e2);
                t.push_back(v);
            }
            drop_graphs(b);
            std::sort(t.begin(), t.end());
            *ms = t[t.size() / 2];
            return VSZ_OK;
        }
        for (int r = 0; r < reps; ++r) {
            tm.kind = kind;
            tm.cls = cls;
            cudaError_t e2 = cudaSuccess;
            if (cls < 0 && (e2 = cudaEventRecord(tm.e0, s)) != cudaSuccess) return cuda_fail(e2);
            const ClassTimer* tp = cls < 0 ? nullptr : &tm;
            const vsz_status st2 = kind ? launch_recon_sequence(b, s, tp) : launch_sequence(b, s, tp);
            if (st2 != VSZ_OK) return st2;
            if (cls < 0 && (e2 = cudaEventRecord(tm.e1, s)) != cudaSuccess) return cuda_fail(e2);
            if ((e2 = cudaEventSynchronize(tm.e1)) != cudaSuccess) return cuda_fail(e2);
            float v = 0.0f;
            if ((e2 = cudaEventElapsedTime(&v, tm.e0, tm.e1)) != cudaSuccess) return cuda_fail(e2);
            t.push_back(v);
        }
        std::sort(t.begin(), t.end());
        *ms = t[t.size() / 2];
        return VSZ_OK;
    };
    const bool conc0 = b->concurrent, rconc0 = b->rconcurrent;
    b->concurrent = b->rconcurrent = false;
    vsz_status st = launch_sequence(b, s);  // warm-up; the compressed data the inverse reads
    for (int kind = 0; kind < 2 && st == VSZ_OK; ++kind) {
        std::vector<BatchClass>& cls = kind ? b->rclasses : b->classes;
        if (cls.empty() || (kind && !b->d_fix)) continue;  // no outputs set: nothing to reconstruct
        for (size_t c = 0; st == VSZ_OK && c < cls.size(); ++c) {
            BatchClass& k = cls[c];
            if (!k.total_tiles) continue;
            k.shape = LaunchShape{};
            float best = 0.0f;
            if ((st = measure(kind, (int)c, &best)) != VSZ_OK) break;
            k.ms_default = best;
            LaunchShape pick{};
            for (int w : {2, 4, 8}) {
                const int occ = class_occupancy(k, w);
                if (occ < 1) continue;
                std::vector<int> cands = {1, 2, 4, occ};
                std::sort(cands.begin(), cands.end());
                cands.erase(std::unique(cands.begin(), cands.end()), cands.end());
                for (int ct : cands) {
                    if (ct > occ) continue;
                    k.shape = LaunchShape{w, ct};
                    float ms = 0.0f;
                    if ((st = measure(kind, (int)c, &ms)) != VSZ_OK) break;
                    if (ms < best) {
                        best = ms;
                        pick = k.shape;
                    }
                }
                if (st != VSZ_OK) break;
            }
            k.shape = pick;
            k.ms_best = best;
        }
        if (st != VSZ_OK) break;
        // Events around one class kernel break its overlap with its
        // neighbours in the sequence, so keep the tuned shapes only if the
        // whole sequence is faster with them than with the default ones.
        bool changed = false;
        for (const BatchClass& k : cls) changed |= k.shape.warps != 0 || k.shape.ctas != 0;
        if (changed) {
            std::vector<LaunchShape> tuned;
            for (const BatchClass& k : cls) tuned.push_back(k.shape);
            float t_tuned = 0.0f, t_def = 0.0f;
            if ((st = measure(kind, -1, &t_tuned)) != VSZ_OK) break;
            for (BatchClass& k : cls) k.shape = LaunchShape{};
            if ((st = measure(kind, -1, &t_def)) != VSZ_OK) break;
            if (t_tuned < t_def) {
                for (size_t c = 0; c < cls.size(); ++c) cls[c].shape = tuned[c];
            } else {
                for (BatchClass& k : cls) k.ms_best = k.ms_default;
            }
        }
        int active = 0;
        for (const BatchClass& k : cls) active += k.total_tiles ? 1 : 0;
        if (active > 1) {
            bool& flag = kind ? b->rconcurrent : b->concurrent;
            float ser = 0.0f, con = 0.0f;
            flag = false;
            if ((st = measure(kind, -1, &ser)) != VSZ_OK) break;
            flag = true;
            if ((st = measure(kind, -1, &con)) != VSZ_OK) break;
            flag = con < ser;
        }
    }
    if (st != VSZ_OK) {
        b->concurrent = conc0;
        b->rconcurrent = rconc0;
    }
    drop_graphs(b);
    cudaEventDestroy(tm.e0);
    cudaEventDestroy(tm.e1);
    return st;
}

vsz_status vsz_batch_compress_host(vsz_batch b, const float* const* h_x, vsz_host_field* h_out, void* stream) {
    if (!b || !h_x || !h_out) return VSZ_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    for (int i = 0; i < b->n; ++i) {
        const Geom& g = b->fields[i].a.g;
        const vsz_host_field& o = h_out[i];
        const int32_t pm = b->jobs[i].params.pad;
        const bool table = (is_block_pad(pm) || is_edge_pad(pm)) && g.nb > 0;
        if (!o.hdr || (g.n > 0 && (!h_x[i] || !o.codes)) || !o.blk_off || (table && !o.pad) ||
            (o.out_cap && (!o.out_idx || !o.out_delta)) || (o.fix_cap && (!o.fix_idx || !o.fix_bits)))
            return VSZ_ERR_INVALID_ARG;
    }
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < b->n && e == cudaSuccess; ++i) {
        const uint64_t n = b->fields[i].a.g.n;
        if (n) e = cudaMemcpyAsync((void*)b->jobs[i].d_x, h_x[i], n * sizeof(float), cudaMemcpyHostToDevice, s);
    }
    if (e != cudaSuccess) return cuda_fail(e);
    const vsz_status st = vsz_batch_submit(b, stream);
    if (st != VSZ_OK) return st;
    // headers first, then the dense outputs, which stay in flight while the
    // host waits for the headers' list lengths
    for (int i = 0; i < b->n && e == cudaSuccess; ++i)
        e = cudaMemcpyAsync(h_out[i].hdr, b->jobs[i].out.hdr, sizeof(vsz_header), cudaMemcpyDeviceToHost, s);
    for (int i = 0; i < b->n && e == cudaSuccess; ++i) {
        const Geom& g = b->fields[i].a.g;
        const vsz_compressed& c = b->jobs[i].out;
        const int32_t pm = b->jobs[i].params.pad;
        if (g.n) e = cudaMemcpyAsync(h_out[i].codes, c.codes, g.n * sizeof(uint16_t), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(h_out[i].blk_off, c.blk_off, (g.nb + 1) * sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
        const uint64_t plen = is_block_pad(pm) ? g.nb : is_edge_pad(pm) ? g.nb * (uint64_t)g.nd : 0;
        if (e == cudaSuccess && plen)
            e = cudaMemcpyAsync(h_out[i].pad, c.pad, plen * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    for (int i = 0; i < b->n && e == cudaSuccess; ++i) {
        const vsz_compressed& c = b->jobs[i].out;
        const vsz_host_field& o = h_out[i];
        const uint64_t no = std::min(o.hdr->n_out, std::min(c.out_cap, o.out_cap));
        const uint64_t nf = std::min(o.hdr->n_fix, std::min(c.fix_cap, o.fix_cap));
        if (no) e = cudaMemcpyAsync(o.out_idx, c.out_idx, no * sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
        if (no && e == cudaSuccess)
            e = cudaMemcpyAsync(o.out_delta, c.out_delta, no * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
        if (nf && e == cudaSuccess)
            e = cudaMemcpyAsync(o.fix_idx, c.fix_idx, nf * sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
        if (nf && e == cudaSuccess)
            e = cudaMemcpyAsync(o.fix_bits, c.fix_bits, nf * sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e == cudaSuccess ? VSZ_OK : cuda_fail(e);
}

vsz_status vsz_batch_destroy(vsz_batch b) {
    if (!b) return VSZ_ERR_INVALID_ARG;
    free_batch(b);
    return VSZ_OK;
}

}  // extern "C"
