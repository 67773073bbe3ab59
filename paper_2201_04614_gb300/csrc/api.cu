// api.cu -- host implementation of the vsz.h C ABI.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <map>
#include <mutex>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "common.cuh"
#include "misc.cuh"
#include "trace.cuh"

namespace vsz {

// Per-device and per-kernel caches of launch parameters (vsz_shutdown
// clears them, so that the library works again after a device reset).
namespace {
std::mutex g_cache_mu;
int g_num_sms[64] = {0};
std::unordered_map<const void*, int> g_grid_occ;                     // grid_for
std::map<std::tuple<const void*, int, size_t>, int> g_occ;           // occupancy
std::map<std::pair<int, const void*>, size_t> g_smem_attr;           // raise_smem_attr
void* g_noalloc_addr[64] = {nullptr};                                 // noalloc_workspace
}  // namespace

// Failure injection for tests: the k-th library device allocation from the
// call of vsz_debug_fail_alloc(k) fails as if the device were out of memory.
static std::atomic<int> g_fail_alloc{0};

cudaError_t lib_malloc(void** p, size_t bytes) {
    int k = g_fail_alloc.load();
    while (k > 0 && !g_fail_alloc.compare_exchange_weak(k, k - 1)) {
    }
    if (k == 1) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}

static void reset_launch_caches() {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    for (int& v : g_num_sms) v = 0;
    g_grid_occ.clear();
    g_occ.clear();
    g_smem_attr.clear();
    for (void*& p : g_noalloc_addr) p = nullptr;
}

#ifdef VSZ_DEBUG_BOUNDS
std::vector<unsigned int (*)()>& bounds_readers() {
    static std::vector<unsigned int (*)()> v;  // one reader per translation unit
    return v;
}
void register_bounds_reader(unsigned int (*reader)()) { bounds_readers().push_back(reader); }
#endif

int num_sms() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 148;
    std::lock_guard<std::mutex> lk(g_cache_mu);
    if (!g_num_sms[dev]) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 148;
        g_num_sms[dev] = v;
    }
    return g_num_sms[dev];
}

// CTAs for a grid-stride kernel: enough to cover `work` at `per_cta` items
// each, capped at the number of CTAs that are resident at once.
int grid_for(const void* kernel, int threads, size_t smem, uint64_t per_cta, uint64_t work) {
    int occ = 0;
    {
        std::lock_guard<std::mutex> lk(g_cache_mu);
        auto it = g_grid_occ.find(kernel);
        if (it != g_grid_occ.end()) {
            occ = it->second;
        } else {
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, threads, smem) != cudaSuccess || occ < 1)
                occ = 1;
            g_grid_occ[kernel] = occ;
        }
    }
    const uint64_t want = (work + per_cta - 1) / (per_cta ? per_cta : 1);
    const uint64_t cap = (uint64_t)num_sms() * (uint64_t)occ;
    uint64_t g = want < cap ? want : cap;
    if (g < 1) g = 1;
    return (int)g;
}

int occupancy(const void* kernel, int threads, size_t smem) {
    const auto key = std::make_tuple(kernel, threads, smem);
    std::lock_guard<std::mutex> lk(g_cache_mu);
    auto it = g_occ.find(key);
    if (it != g_occ.end()) return it->second;
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, threads, smem) != cudaSuccess) {
        (void)cudaGetLastError();
        occ = 0;
    }
    g_occ[key] = occ;
    return occ;
}

int grid_shape(const void* kernel, int threads, size_t smem, uint64_t per_cta, uint64_t work, int ctas) {
    int occ = occupancy(kernel, threads, smem);
    if (occ < 1) occ = 1;
    if (ctas > 0 && ctas < occ) occ = ctas;
    const uint64_t want = (work + per_cta - 1) / (per_cta ? per_cta : 1);
    const uint64_t cap = (uint64_t)num_sms() * (uint64_t)occ;
    uint64_t g = want < cap ? want : cap;
    if (g < 1) g = 1;
    return (int)g;
}

cudaError_t raise_smem_attr(const void* kernel, size_t bytes) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    int optin = 0;
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    if (bytes > (size_t)optin) return cudaErrorInvalidValue;
    std::lock_guard<std::mutex> lk(g_cache_mu);
    size_t& cur = g_smem_attr[std::make_pair(dev, kernel)];
    if (bytes <= cur) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) cur = bytes;
    return e;
}

static thread_local char g_last_err[256] = "";

vsz_status cuda_fail(cudaError_t e) {
    std::snprintf(g_last_err, sizeof g_last_err, "%s: %s", cudaGetErrorName(e), cudaGetErrorString(e));
    return VSZ_ERR_CUDA;
}

static bool pow2(uint32_t v) { return v && !(v & (v - 1)); }

// Validate parameters and derive the geometry and tiling of a field.
vsz_status make_geom(const vsz_params* p, Geom* g) {
    if (!p) return VSZ_ERR_INVALID_ARG;
    if (p->ndim == 4) return VSZ_ERR_UNSUPPORTED;
    if (p->ndim < 1 || p->ndim > 3) return VSZ_ERR_INVALID_ARG;
    if (!(p->eb > 0.0) || !std::isfinite(p->eb)) return VSZ_ERR_INVALID_ARG;
    if (p->eb_mode != VSZ_EB_ABS && p->eb_mode != VSZ_EB_REL) return VSZ_ERR_INVALID_ARG;
    if (p->radius < 1 || p->radius > 32768) return VSZ_ERR_INVALID_ARG;
    if (p->pad < VSZ_PAD_ZERO || p->pad > VSZ_PAD_EDGE_AVG) return VSZ_ERR_INVALID_ARG;
    if (p->block < 1) return VSZ_ERR_INVALID_ARG;
    const uint32_t bmax = p->ndim == 1 ? 256u : p->ndim == 2 ? 128u : 32u;
    if (!pow2(p->block) || p->block < 4 || p->block > bmax) return VSZ_ERR_UNSUPPORTED;
    uint64_t n = 1;
    for (int k = 0; k < p->ndim; ++k) {
        const uint64_t d = p->dims[k];
        if (d >= (1ull << 32)) return VSZ_ERR_INVALID_ARG;
        n *= d;
        if (n >= (1ull << 32)) return VSZ_ERR_INVALID_ARG;
    }
    std::memset(g, 0, sizeof *g);
    g->nd = p->ndim;
    g->b = p->block;
    g->n = n;
    const uint64_t b = p->block;
    g->nz = p->ndim == 3 ? p->dims[0] : 1;
    g->ny = p->ndim == 3 ? p->dims[1] : p->ndim == 2 ? p->dims[0] : 1;
    g->nx = p->dims[p->ndim - 1];
    g->nbx = (g->nx + b - 1) / b;
    g->nby = p->ndim >= 2 ? (g->ny + b - 1) / b : 1;
    g->nbz = p->ndim == 3 ? (g->nz + b - 1) / b : 1;
    g->nb = n ? g->nbx * g->nby * g->nbz : 0;
    if (n == 0) {
        g->nseg = 0;
        g->ntiles = 0;
        g->bpt = p->ndim == 1 ? (uint32_t)(kChunk1D / b) : (uint32_t)(kSegCols / b);
    } else if (p->ndim == 1) {
        g->ntiles = (n + kChunk1D - 1) / kChunk1D;
        g->nseg = g->ntiles;
        g->bpt = (uint32_t)(kChunk1D / b);
    } else {
        g->nseg = (g->nx + kSegCols - 1) / kSegCols;
        g->ntiles = g->nseg * g->nby * g->nbz;
        g->bpt = (uint32_t)(kSegCols / b);
    }
    g->nchunks = (g->ntiles + kTilesPerChunk - 1) / kTilesPerChunk;
    return VSZ_OK;
}

bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

vsz_status check_compressed(const Geom& g, const vsz_params* p, const vsz_compressed* c) {
    if (!c || !c->hdr || !c->blk_off) return VSZ_ERR_INVALID_ARG;
    if (!aligned(c->hdr, 8)) return VSZ_ERR_INVALID_ARG;
    if (g.n > 0 && !c->codes) return VSZ_ERR_INVALID_ARG;
    if ((is_block_pad(p->pad) || is_edge_pad(p->pad)) && g.nb > 0 && !c->pad) return VSZ_ERR_INVALID_ARG;
    if (c->out_cap > 0 && (!c->out_idx || !c->out_delta)) return VSZ_ERR_INVALID_ARG;
    if (c->fix_cap > 0 && (!c->fix_idx || !c->fix_bits)) return VSZ_ERR_INVALID_ARG;
    if (c->out_cap >= (1ull << 32) || c->fix_cap >= (1ull << 32)) return VSZ_ERR_INVALID_ARG;
    return VSZ_OK;
}

// Fixed workspace of vsz_compress_noalloc: part of the library's device
// image, so it exists on every GPU that loads the library, until exit.
static __device__ __align__(256) unsigned char g_noalloc_ws[VSZ_NOALLOC_WS_BYTES];

// Device address of g_noalloc_ws on the current device, looked up once per
// device.  In host code the array's name is only a host-side stand-in, so
// kernels must get this address, never the name.
static vsz_status noalloc_workspace(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e);
    if (dev < 0 || dev >= 64) return VSZ_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_cache_mu);
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_ws);
        if (e != cudaSuccess) return cuda_fail(e);
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return VSZ_OK;
}

}  // namespace vsz

using namespace vsz;

extern "C" {

const char* vsz_status_string(vsz_status s) {
    switch (s) {
    case VSZ_OK: return "VSZ_OK";
    case VSZ_ERR_INVALID_ARG: return "VSZ_ERR_INVALID_ARG";
    case VSZ_ERR_UNSUPPORTED: return "VSZ_ERR_UNSUPPORTED";
    case VSZ_ERR_CAPACITY: return "VSZ_ERR_CAPACITY";
    case VSZ_ERR_CUDA: return "VSZ_ERR_CUDA";
    case VSZ_ERR_CORRUPT: return "VSZ_ERR_CORRUPT";
    case VSZ_ERR_TOO_LARGE: return "VSZ_ERR_TOO_LARGE";
    default: return "VSZ_ERR_UNKNOWN";
    }
}

const char* vsz_last_cuda_error(void) { return g_last_err; }

vsz_status vsz_debug_bounds_word(uint32_t* out) {
    if (!out) return VSZ_ERR_INVALID_ARG;
#ifdef VSZ_DEBUG_BOUNDS
    uint32_t v = 0;
    std::vector<unsigned int (*)()> rs;
    {
        std::lock_guard<std::mutex> lk(g_cache_mu);
        rs = bounds_readers();
    }
    for (auto r : rs) {
        const uint32_t w = r();
        if (!v) v = w;
    }
    *out = v;
    return VSZ_OK;
#else
    *out = 0;
    return VSZ_ERR_UNSUPPORTED;
#endif
}

int vsz_abi_version(void) { return VSZ_ABI_VERSION; }

vsz_status vsz_validate(const vsz_params* p) {
    Geom g;
    return make_geom(p, &g);
}

uint64_t vsz_num_elems(const vsz_params* p) {
    Geom g;
    return make_geom(p, &g) == VSZ_OK ? g.n : 0;
}

uint64_t vsz_num_blocks(const vsz_params* p) {
    Geom g;
    return make_geom(p, &g) == VSZ_OK ? g.nb : 0;
}

size_t vsz_workspace_size(const vsz_params* p, uint64_t out_cap, uint64_t fix_cap) {
    Geom g;
    if (make_geom(p, &g) != VSZ_OK) return 0;
    return ws_layout(g, out_cap, fix_cap).total;
}

size_t vsz_workspace_size_dense(const vsz_params* p, uint64_t out_cap, uint64_t fix_cap) {
    Geom g;
    if (make_geom(p, &g) != VSZ_OK) return 0;
    return ws_layout(g, out_cap, fix_cap, true).total;
}


}  // extern "C"

namespace vsz {
// The workspace layout a call uses: block-slot staging for 2D/3D fields when
// the workspace holds it (vsz_workspace_size_dense), else the plain one.
static WsLayout layout_for(const Geom& g, const vsz_compressed* c, size_t ws_bytes, bool* slots) {
    if (g.nd >= 2) {
        const WsLayout Ls = ws_layout(g, c->out_cap, c->fix_cap, true);
        if (ws_bytes >= Ls.total) {
            *slots = true;
            return Ls;
        }
    }
    *slots = false;
    return ws_layout(g, c->out_cap, c->fix_cap);
}

// Kernel arguments of one field's compression over its workspace.
static CompressArgs compress_args(const Geom& g, const vsz_params* p, const float* d_x, const vsz_compressed* c,
                                  char* ws, const WsLayout& L, bool slots) {
    CompressArgs a;
    std::memset(&a, 0, sizeof a);
    a.x = d_x;
    a.codes = c->codes;
    a.pad = c->pad;
    a.blk_off = c->blk_off;
    a.hdr = c->hdr;
    a.wsh = (WsHeader*)ws;
    a.tiles = (uint4*)(ws + L.tiles);
    a.chunks = (uint4*)(ws + L.chunks);
    a.stage_out = (uint2*)(ws + L.stage_out);
    a.stage_fix = (uint2*)(ws + L.stage_fix);
    if (defers_origin(p->pad)) {
        a.origin = (int32_t*)(ws + L.origin);
        a.oflag = (uint8_t*)(ws + L.oflag);
    }
    a.out_idx = c->out_idx;
    a.out_delta = c->out_delta;
    a.fix_idx = c->fix_idx;
    a.fix_bits = c->fix_bits;
    a.out_cap = c->out_cap;
    a.fix_cap = c->fix_cap;
    a.g = g;
    a.R = (int32_t)p->radius;
    a.pad_mode = p->pad;
    a.vec = (aligned(d_x, 16) && aligned(c->codes, 16) && (g.nd == 1 || g.nx % 4 == 0)) ? 1 : 0;
    a.blk_in = c->blk_off;
    if (slots) {
        a.slots = a.stage_out;
        a.blk_in = (uint32_t*)(ws + L.blkin);
    }
    return a;
}
}  // namespace vsz

extern "C" {

static vsz_status prequant_lorenzo_impl(const vsz_params* p, const float* d_x, vsz_compressed* c, void* d_ws,
                                        size_t ws_bytes, void* stream, const int32_t* given_pad) {
    Geom g;
    vsz_status st = make_geom(p, &g);
    if (st != VSZ_OK) return st;
    if ((st = check_compressed(g, p, c)) != VSZ_OK) return st;
    if (g.n > 0 && !d_x) return VSZ_ERR_INVALID_ARG;
    bool slots = false;
    const WsLayout L = layout_for(g, c, ws_bytes, &slots);
    if (!d_ws || ws_bytes < L.total || !aligned(d_ws, 256)) return VSZ_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    char* ws = (char*)d_ws;
    WsHeader* wsh = (WsHeader*)ws;
    uint4* chunks = (uint4*)(ws + L.chunks);
    const bool rel = p->eb_mode == VSZ_EB_REL;
    const bool xvec = aligned(d_x, 16);

    cudaError_t e;
    {
        TraceScope ts("begin", s, g.nd, g.b, g.n);
        e = launch_begin(wsh, chunks, g.nchunks, c->hdr, p->eb, rel, s);
    }
    if (e != cudaSuccess) return cuda_fail(e);
    if (rel) {
        TraceScope ts("range", s, g.nd, g.b, g.n);
        e = launch_range(d_x, g.n, wsh, c->hdr, p->eb, xvec, s);
        if (e != cudaSuccess) return cuda_fail(e);
    }
    if (g.ntiles == 0) return VSZ_OK;

    CompressArgs a = compress_args(g, p, d_x, c, ws, L, slots);
    if (given_pad) {
        a.has_gpad = 1;
        a.gpad = *given_pad;
    }
    {
        TraceScope ts("lorenzo", s, g.nd, g.b, g.n);
        e = g.nd == 1 ? launch_lorenzo_1d(a, s) : g.nd == 2 ? launch_lorenzo_2d(a, s) : launch_lorenzo_3d(a, s);
    }
    if (e != cudaSuccess) return cuda_fail(e);
    if (defers_origin(p->pad)) {
        // the global padding value is known once every tile is walked; edge
        // scalars come from a face-statistics pass
        TraceScope ts("origin_fix", s, g.nd, g.b, g.n);
        e = launch_origin_fix(a, s);
        if (e != cudaSuccess) return cuda_fail(e);
    }
    return VSZ_OK;
}

vsz_status vsz_prequant_lorenzo(const vsz_params* p, const float* d_x, vsz_compressed* c, void* d_ws,
                                size_t ws_bytes, void* stream) {
    return prequant_lorenzo_impl(p, d_x, c, d_ws, ws_bytes, stream, nullptr);
}

vsz_status vsz_compress_slab(const vsz_params* p, int32_t pad_value, const float* d_x, vsz_compressed* c,
                             void* d_ws, size_t ws_bytes, void* stream) {
    if (!p || p->eb_mode != VSZ_EB_ABS) return VSZ_ERR_INVALID_ARG;
    vsz_status st = prequant_lorenzo_impl(p, d_x, c, d_ws, ws_bytes, stream, &pad_value);
    if (st != VSZ_OK) return st;
    return vsz_outlier_compact(p, c, d_ws, ws_bytes, stream);
}

vsz_status vsz_outlier_compact(const vsz_params* p, vsz_compressed* c, void* d_ws, size_t ws_bytes,
                               void* stream) {
    Geom g;
    vsz_status st = make_geom(p, &g);
    if (st != VSZ_OK) return st;
    if ((st = check_compressed(g, p, c)) != VSZ_OK) return st;
    bool slots = false;
    const WsLayout L = layout_for(g, c, ws_bytes, &slots);
    if (!d_ws || ws_bytes < L.total || !aligned(d_ws, 256)) return VSZ_ERR_INVALID_ARG;
    char* ws = (char*)d_ws;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e;
    {
        TraceScope ts("compact_scan", s, g.nd, g.b, g.n);
        e = launch_compact_scan(g, (uint4*)(ws + L.chunks), c->hdr, c->blk_off, c->out_cap, c->fix_cap, s);
    }
    if (e != cudaSuccess) return cuda_fail(e);
    if (g.nchunks > 0) {
        TraceScope ts("compact_move", s, g.nd, g.b, g.n);
        e = launch_compact_move(compress_args(g, p, nullptr, c, ws, L, slots), s);
    }
    if (e != cudaSuccess) return cuda_fail(e);
    return VSZ_OK;
}

vsz_status vsz_compress(const vsz_params* p, const float* d_x, vsz_compressed* c, void* d_ws, size_t ws_bytes,
                        void* stream) {
    vsz_status st = vsz_prequant_lorenzo(p, d_x, c, d_ws, ws_bytes, stream);
    if (st != VSZ_OK) return st;
    return vsz_outlier_compact(p, c, d_ws, ws_bytes, stream);
}

vsz_status vsz_compress_noalloc(const vsz_params* p, const float* d_x, vsz_compressed* c, void* stream) {
    Geom g;
    vsz_status st = make_geom(p, &g);
    if (st != VSZ_OK) return st;
    if ((st = check_compressed(g, p, c)) != VSZ_OK) return st;
    const size_t need = ws_layout(g, c->out_cap, c->fix_cap).total;
    if (need > (size_t)VSZ_NOALLOC_WS_BYTES) return VSZ_ERR_TOO_LARGE;
    void* ws = nullptr;
    if ((st = noalloc_workspace(&ws)) != VSZ_OK) return st;
    // k_begin, the first kernel of the call, re-zeroes the cursors, counters
    // and chunk sums this call relies on; the rest is written before it is read.
    return vsz_compress(p, d_x, c, ws, VSZ_NOALLOC_WS_BYTES, stream);
}

static vsz_status reconstruct_impl(const vsz_params* p, const vsz_compressed* c, void* out, bool q_out,
                                   void* d_ws, size_t ws_bytes, void* stream) {
    Geom g;
    vsz_status st = make_geom(p, &g);
    if (st != VSZ_OK) return st;
    if ((st = check_compressed(g, p, c)) != VSZ_OK) return st;
    if (g.n > 0 && !out) return VSZ_ERR_INVALID_ARG;
    if (d_ws && (ws_bytes < VSZ_RECON_WS_BYTES || !aligned(d_ws, 16))) return VSZ_ERR_INVALID_ARG;
    if (g.n == 0) return VSZ_OK;
    cudaStream_t s = (cudaStream_t)stream;
    ReconArgs a;
    std::memset(&a, 0, sizeof a);
    a.codes = c->codes;
    a.pad = c->pad;
    a.blk_off = c->blk_off;
    a.out_idx = c->out_idx;
    a.out_delta = c->out_delta;
    a.out_cap = c->out_cap;
    a.ticket = (d_ws && g.nd > 1) ? (unsigned int*)d_ws : nullptr;
    a.hdr = c->hdr;
    a.out = out;
    a.g = g;
    a.R = (int32_t)p->radius;
    a.pad_mode = p->pad;
    a.vec = (aligned(c->codes, 16) && aligned(out, 16) && (g.nd == 1 || g.nx % 4 == 0)) ? 1 : 0;
    cudaError_t e;
    if (a.ticket) {
        e = cudaMemsetAsync(a.ticket, 0, sizeof(unsigned int), s);
        if (e != cudaSuccess) return cuda_fail(e);
    }
    {
        TraceScope ts(q_out ? "recon_q" : "recon", s, g.nd, g.b, g.n);
        e = g.nd == 1 ? launch_recon_1d(a, q_out, s)
          : g.nd == 2 ? launch_recon_2d(a, q_out, s)
                      : launch_recon_3d(a, q_out, s);
    }
    if (e != cudaSuccess) return cuda_fail(e);
    if (!q_out && c->fix_cap > 0) {
        TraceScope ts("fixups", s, g.nd, g.b, g.n);
        e = launch_fixups(c->hdr, c->fix_idx, c->fix_bits, c->fix_cap, (float*)out, g.n, s);
        if (e != cudaSuccess) return cuda_fail(e);
    }
    return VSZ_OK;
}

vsz_status vsz_reconstruct(const vsz_params* p, const vsz_compressed* c, float* d_xhat, void* d_ws,
                           size_t ws_bytes, void* stream) {
    return reconstruct_impl(p, c, d_xhat, false, d_ws, ws_bytes, stream);
}

vsz_status vsz_reconstruct_q(const vsz_params* p, const vsz_compressed* c, int32_t* d_q, void* d_ws,
                             size_t ws_bytes, void* stream) {
    return reconstruct_impl(p, c, d_q, true, d_ws, ws_bytes, stream);
}

vsz_status vsz_code_histogram(const vsz_params* p, const uint16_t* d_codes, uint32_t* d_hist, void* stream) {
    Geom g;
    vsz_status st = make_geom(p, &g);
    if (st != VSZ_OK) return st;
    if (!d_hist || (g.n > 0 && !d_codes)) return VSZ_ERR_INVALID_ARG;
    cudaError_t e;
    {
        TraceScope ts("histogram", (cudaStream_t)stream, g.nd, g.b, g.n);
        e = launch_histogram(d_codes, g.n, d_hist, 2u * p->radius, (cudaStream_t)stream);
    }
    if (e != cudaSuccess) return cuda_fail(e);
    return VSZ_OK;
}

vsz_status vsz_debug_fail_alloc(int k) {
    if (k < 0) return VSZ_ERR_INVALID_ARG;
    g_fail_alloc.store(k);
    return VSZ_OK;
}

vsz_status vsz_shutdown(void) {
    Tracer::get().shutdown();
    reset_launch_caches();
    return VSZ_OK;
}

vsz_status vsz_trace_enable(int on) {
    Tracer::get().enable(on != 0);
    return VSZ_OK;
}

int vsz_trace_read(vsz_trace_record* h_out, int max_records) {
    return Tracer::get().read(h_out, h_out ? max_records : 0);
}

vsz_status vsz_read_header(const vsz_compressed* c, vsz_header* h_out, void* stream) {
    if (!c || !c->hdr || !h_out) return VSZ_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(h_out, c->hdr, sizeof(vsz_header), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return cuda_fail(e);
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e);
    return VSZ_OK;
}

vsz_status vsz_sync_status(const vsz_compressed* c, void* stream) {
    vsz_header h;
    const vsz_status st = vsz_read_header(c, &h, stream);
    if (st != VSZ_OK) return st;
    const uint32_t v = h.status > h.recon_status ? h.status : h.recon_status;
    return (vsz_status)v;
}

}  // extern "C"
