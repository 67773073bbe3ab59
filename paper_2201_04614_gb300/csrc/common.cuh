// common.cuh -- internal definitions shared by the libvsz kernels and host code.
//
// Geometry, workspace layout and the device arithmetic of the dual-quant
// (prequantization, int->float, guard).  Nothing here is visible through the
// C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "vsz.h"

#define VSZ_FULL 0xffffffffu

namespace vsz {

// Tiling.  2D/3D: a warp-tile is one 128-column segment along x of one row
// of blocks (all b rows of the block row in 2D, all b*b rows of the block
// slab in 3D); every lane owns 4 consecutive columns.  1D: a warp-tile is a
// chunk of 4096 consecutive elements.  A tile always holds whole blocks along
// x, so its blocks are consecutive in the canonical block order.
constexpr int kSegCols = 128;
constexpr int kChunk1D = 4096;
constexpr int kTilesPerChunk = 32;   // tiles per compaction chunk (one CTA each)

// Block-slot staging of the 2D/3D compression: when the workspace holds
// it, the staging area has one slot of b^nd + 1 entries per block, and the
// walk writes each outlier straight into its block's slot (position 1 + its
// rank in the block; slot 0 holds the origin of a per-block padding mode).
// No outlier needs a stash, a sort or a second walk, however dense they are;
// the compaction moves each slot's entries to their final place.
__host__ __device__ constexpr uint64_t block_slot(int nd, uint32_t b) {
    return (nd == 3 ? (uint64_t)b * b * b : (uint64_t)b * b) + 1;
}

struct Geom {
    int32_t nd;
    uint32_t b;
    uint64_t n;
    uint64_t nx, ny, nz;     // nz = ny = 1 for lower ranks
    uint64_t nbx, nby, nbz;  // blocks per axis
    uint64_t nb;
    uint64_t nseg;           // tiles per row of blocks (1D: all tiles)
    uint64_t ntiles;
    uint32_t bpt;            // blocks per tile (interior)
    uint64_t nchunks;
};

// Workspace header (first 256 bytes of the workspace).
struct WsHeader {
    unsigned long long stage_out;  // staging cursors
    unsigned long long stage_fix;
    unsigned long long qsum;       // sum of q, two's complement (global padding)
    unsigned int xmin_ord, xmax_ord;  // order-preserving encodings of finite min/max
    int qmin, qmax;                // extremes of q (global min / max padding)
    unsigned int done0, done1;     // last-block counters
    unsigned int nonfinite;        // a range pass met a NaN or Inf
    unsigned int fp32_ok;          // every |x * inv2eb| < 2^20 and no NaN/Inf (relative mode only)
    unsigned long long ticket;     // dynamic tile scheduling of the compression kernel
};
static_assert(sizeof(WsHeader) <= 256, "ws header");


struct WsLayout {
    size_t tiles;      // uint4 per tile {stage_base_out, tot_out, stage_base_fix, tot_fix}
    size_t chunks;     // uint4 per chunk {sum_out, sum_fix, off_out, off_fix}
    size_t origin;     // int32 per block: q at the block origin, then its residual (global padding)
    size_t oflag;      // uint8 per block: the origin is an outlier (global padding)
    size_t blkin;      // uint32 per block: in-tile offsets from the walk (block slots only)
    size_t stage_out;  // uint2 per outlier {idx, delta}
    size_t stage_fix;  // uint2 per fixup {idx, bits}
    size_t total;
};

inline size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

// slots: the staging area of outliers laid out as block slots (2D/3D only).
inline WsLayout ws_layout(const Geom& g, uint64_t out_cap, uint64_t fix_cap, bool slots = false) {
    if (slots && g.nd >= 2) {
        const uint64_t need = g.nb * block_slot(g.nd, g.b);
        if (out_cap < need) out_cap = need;
    }
    WsLayout L;
    size_t off = 256;
    L.tiles = off;
    off = align256(off + g.ntiles * 16);
    L.chunks = off;
    off = align256(off + g.nchunks * 16);
    L.origin = off;
    off = align256(off + g.nb * 4);
    L.oflag = off;
    off = align256(off + g.nb);
    L.blkin = off;
    if (slots && g.nd >= 2) off = align256(off + g.nb * 4);
    L.stage_out = off;
    off = align256(off + out_cap * 8);
    L.stage_fix = off;
    off = align256(off + fix_cap * 8);
    L.total = off;
    return L;
}

// ---- bounds-checking build ----------------------------------------------------
// Built with -DVSZ_DEBUG_BOUNDS, the kernels check the index of each of their
// writes to the field-sized buffers (codes, values, lists, slots, tables)
// and of their reads of the slots and outlier caches against the buffer's
// length; an access that would fall outside is skipped and its site number
// recorded in a device word (first site wins; nothing traps).  Every
// translation unit has its own word and registers a reader at load time;
// vsz_debug_bounds_word() reads and clears them all.  In the normal build the
// checks compile away.
#ifdef VSZ_DEBUG_BOUNDS
static __device__ unsigned int g_bounds_err;
__device__ __forceinline__ bool in_bounds(uint64_t i, uint64_t n, unsigned int site) {
    if (i < n) return true;
    atomicCAS(&g_bounds_err, 0u, site);
    return false;
}
#define VSZ_IN(i, n, site) (::vsz::in_bounds((uint64_t)(i), (uint64_t)(n), (site)))
void register_bounds_reader(unsigned int (*reader)());
static unsigned int read_and_clear_bounds_word() {
    unsigned int v = 0, z = 0;
    if (cudaMemcpyFromSymbol(&v, g_bounds_err, sizeof v) != cudaSuccess) return 0xffffffffu;
    cudaMemcpyToSymbol(g_bounds_err, &z, sizeof z);
    return v;
}
struct BoundsReaderReg {
    BoundsReaderReg() { register_bounds_reader(&read_and_clear_bounds_word); }
};
static BoundsReaderReg g_bounds_reader_reg;
#else
#define VSZ_IN(i, n, site) true
#endif

// ---- device arithmetic ------------------------------------------------------

__host__ __device__ __forceinline__ uint64_t umin64(uint64_t a, uint64_t b) { return a < b ? a : b; }
__host__ __device__ __forceinline__ uint64_t umax64(uint64_t a, uint64_t b) { return a > b ? a : b; }

// Prequantization q = rint(x * inv2eb) (Sec. III-A): one fp32 product, then
// the conversion instruction with round-to-nearest-even, which saturates to
// the int32 range and maps NaN to 0.  Branch-free.
__device__ __forceinline__ int32_t prequant(float x, float inv2eb) {
    const float p = __fmul_rn(x, inv2eb);
    int32_t q;
    asm("cvt.rni.sat.s32.f32 %0, %1;" : "=r"(q) : "f"(p));
    return q;
}

// (float)q, round to nearest even.
__device__ __forceinline__ float q2f(int32_t q) {
    float f;
    asm("cvt.rn.f32.s32 %0, %1;" : "=f"(f) : "r"(q));
    return f;
}

// Error-bound guard (fixup test): true when x_hat = fl(fl(q) * ebx2) misses
// |x - x_hat| <= eb_f32, and for every NaN or Inf x.
__device__ __forceinline__ bool needs_fixup(float x, int32_t q, float ebx2, float eb_f32) {
    const float xh = __fmul_rn(q2f(q), ebx2);
    return !(fabsf(__fsub_rn(x, xh)) <= eb_f32);
}

// Code of a residual: delta + R when -R < delta < R, else 0 (outlier).
__device__ __forceinline__ uint32_t code_of(int32_t d, int32_t R) {
    return (d > -R && d < R) ? (uint32_t)(d + R) : 0u;
}

// Rounded mean of the q values of a block: floor((2S + m) / (2m)), computed
// without overflow as floor(S/m) plus one when the remainder is >= m/2.
__device__ __forceinline__ int32_t rounded_mean(long long S, long long m) {
    long long qt = S / m;
    long long r = S - qt * m;
    if (r < 0) { qt -= 1; r += m; }
    return (int32_t)(qt + ((2 * r >= m) ? 1 : 0));
}

// Edge granularity (Sec. IV-B-3): the block origin's prediction from the
// block's per-axis scalars Pk[0..nd): the inclusion-exclusion sum over the
// non-empty sets S of axes of (-1)^(|S|+1) times the rounded mean of the
// scalars in S (the value of a neighbour outside along exactly the axes in
// S), modulo 2^32.  Every other residual does not depend on the scalars.
__device__ __forceinline__ int32_t edge_origin_pred(const int32_t* __restrict__ Pk, int nd) {
    uint32_t acc = 0;
    for (unsigned S = 1; S < (1u << nd); ++S) {
        long long sum = 0;
        int m = 0;
        for (int k = 0; k < nd; ++k)
            if ((S >> k) & 1u) {
                sum += Pk[k];
                ++m;
            }
        const uint32_t v = (uint32_t)rounded_mean(sum, m);
        acc = (__popc(S) & 1) ? acc + v : acc - v;
    }
    return (int32_t)acc;
}
// The same prediction from the scalars in registers (p2 unused below 3D,
// p1 in 1D): the subsets S of {0, .., nd-1} unrolled, no indexed array.
__device__ __forceinline__ int32_t edge_origin_pred_r(int32_t p0, int32_t p1, int32_t p2, int nd) {
    uint32_t acc = 0;
#pragma unroll
    for (unsigned S = 1; S < 8u; ++S) {
        if (S < (1u << nd)) {
            long long sum = 0;
            int m = 0;
            if (S & 1u) { sum += p0; ++m; }
            if (S & 2u) { sum += p1; ++m; }
            if (S & 4u) { sum += p2; ++m; }
            const uint32_t v = (uint32_t)rounded_mean(sum, m);
            acc = (__popc(S) & 1) ? acc + v : acc - v;
        }
    }
    return (int32_t)acc;
}

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Order-preserving uint encoding of a float (for atomic min/max).
__device__ __forceinline__ unsigned int float_to_ord(float f) {
    unsigned int u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float ord_to_float(unsigned int u) {
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

// ---- kernel argument blocks --------------------------------------------------

struct CompressArgs {
    const float* x;
    uint16_t* codes;
    int32_t* pad;          // [nb] block modes
    uint32_t* blk_off;     // [nb+1]
    uint32_t* blk_in;      // [nb] in-tile exclusive prefixes from the walk: blk_off itself, or (block
                           // slots) a workspace table, which the compaction reads while it writes blk_off
    const vsz_header* hdr;
    WsHeader* wsh;
    uint4* tiles;
    uint4* chunks;
    uint2* stage_out;
    uint2* stage_fix;
    int32_t* origin;       // [nb] block-origin q / residual (global padding modes)
    uint8_t* oflag;        // [nb] origin-outlier flags (global padding modes)
    uint32_t* out_idx;     // final lists (used by the batch compaction)
    int32_t* out_delta;
    uint32_t* fix_idx;
    uint32_t* fix_bits;
    uint64_t out_cap, fix_cap;
    Geom g;
    int32_t R;
    int32_t pad_mode;
    int32_t vec;           // 16-byte vector path allowed
    uint2* slots;          // block-slot staging (2D/3D: stage_out laid out as nb slots), or nullptr
    int32_t has_gpad;      // a global padding value given by the caller (a slab of a split field)
    int32_t gpad;
};

struct ReconArgs {
    const uint16_t* codes;
    const int32_t* pad;
    const uint32_t* blk_off;
    const uint32_t* out_idx;
    const int32_t* out_delta;
    uint64_t out_cap;      // entries readable in out_idx / out_delta
    unsigned int* ticket;  // zeroed tile counter (dynamic scheduling) or nullptr (static)
    vsz_header* hdr;
    void* out;             // float* (values) or int32_t* (q)
    Geom g;
    int32_t R;
    int32_t pad_mode;
    int32_t vec;
};

__host__ __device__ inline bool is_block_pad(int m) {
    return m == VSZ_PAD_BLOCK_MIN || m == VSZ_PAD_BLOCK_MAX || m == VSZ_PAD_BLOCK_AVG;
}
__host__ __device__ inline bool is_global_pad(int m) {
    return m == VSZ_PAD_GLOBAL_MIN || m == VSZ_PAD_GLOBAL_MAX || m == VSZ_PAD_GLOBAL_AVG;
}
__host__ __device__ inline bool is_edge_pad(int m) {
    return m == VSZ_PAD_EDGE_MIN || m == VSZ_PAD_EDGE_MAX || m == VSZ_PAD_EDGE_AVG;
}
// Modes whose padding is known only after the walk: the walk leaves the block
// origins to an origin pass (global statistics, or per-block face statistics).
__host__ __device__ inline bool defers_origin(int m) { return is_global_pad(m) || is_edge_pad(m); }

// Element index of the origin of block `blk` and the tile holding it.
__host__ __device__ inline void block_origin(const Geom& g, uint64_t blk, uint64_t* idx, uint64_t* tile) {
    if (g.nd == 1) {
        *idx = blk * g.b;
        *tile = (blk * g.b) / kChunk1D;
        return;
    }
    // block counts are below 2^32: 32-bit divisions
    const uint32_t b32 = (uint32_t)blk, nbx = (uint32_t)g.nbx, nby = (uint32_t)g.nby;
    const uint32_t r32 = b32 / nbx;
    const uint64_t bx = b32 - r32 * nbx, r = r32;
    const uint64_t bz = r32 / nby, by = r32 - (uint32_t)bz * nby;
    *idx = (bz * g.b * g.ny + by * g.b) * g.nx + bx * g.b;
    *tile = r * g.nseg + (bx * g.b) / kSegCols;
}

// A tile's q statistics into its field's global-padding accumulators
// (workspace header, zeroed by the first kernel of the call): the sum, and
// the extremes for a min or max mode.  Integer sums and extremes do not
// depend on the order of the tiles.
__device__ __forceinline__ void global_stats_add(const CompressArgs& a, int32_t qmin, int32_t qmax, long long qsum) {
    atomicAdd(&a.wsh->qsum, (unsigned long long)qsum);
    if (a.pad_mode == VSZ_PAD_GLOBAL_MIN) atomicMin(&a.wsh->qmin, qmin);
    if (a.pad_mode == VSZ_PAD_GLOBAL_MAX) atomicMax(&a.wsh->qmax, qmax);
}

// The global padding value (Sec. IV-B-1) once every tile is added: the
// minimum, the maximum, or the rounded mean of q over the field.
__device__ __forceinline__ int32_t global_pad_value(const CompressArgs& a) {
    if (a.has_gpad) return a.gpad;  // the whole field's, for one slab of it
    if (a.g.n == 0) return 0;
    return a.pad_mode == VSZ_PAD_GLOBAL_MIN ? a.wsh->qmin
         : a.pad_mode == VSZ_PAD_GLOBAL_MAX ? a.wsh->qmax
         : rounded_mean((long long)a.wsh->qsum, (long long)a.g.n);
}

// Programmatic dependent launch.  Every kernel of the one-field sequence
// (begin, range, compression, origin pass, compaction, reconstruction,
// fixups) starts with pdl_prologue(): it lets the next kernel in the stream
// launch (its CTAs take the SM slots this grid frees as it drains) and then
// waits until the previous kernel has completed and its writes are visible,
// before touching anything.  Since a grid only launches once every CTA of its
// predecessor has started, a waiting grid never holds resources its
// predecessor still needs.  Outside such a launch both instructions are
// no-ops.
__device__ __forceinline__ void pdl_prologue() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args... args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr{};
    attr.id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr.val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// Host launchers implemented in the per-rank translation units.
cudaError_t launch_lorenzo_1d(const CompressArgs& a, cudaStream_t s);
cudaError_t launch_lorenzo_2d(const CompressArgs& a, cudaStream_t s);
cudaError_t launch_lorenzo_3d(const CompressArgs& a, cudaStream_t s);
cudaError_t launch_recon_1d(const ReconArgs& a, bool q_out, cudaStream_t s);
cudaError_t launch_recon_2d(const ReconArgs& a, bool q_out, cudaStream_t s);
cudaError_t launch_recon_3d(const ReconArgs& a, bool q_out, cudaStream_t s);

// Launch shape of a persistent batch kernel, the knobs of the batch
// autotuner: warps per CTA (0 = the kernel's default) and resident CTAs per
// SM (0 = as many as fit).  Tiles are claimed per warp from a ticket, so the
// shape changes only how the work is spread, never a result.
struct LaunchShape {
    int warps = 0;
    int ctas = 0;
};

// Batch launchers.  With occ != nullptr nothing is launched: *occ receives
// the CTAs per SM that fit with sh.warps (0 if the shape cannot launch).
cudaError_t launch_lorenzo_batch_1d(uint32_t b, int pk, const CompressArgs* fields, const uint64_t* tile_prefix,
                                    int nfields, uint64_t total_tiles, unsigned long long* ticket, LaunchShape sh,
                                    cudaStream_t s, int* occ = nullptr);
cudaError_t launch_lorenzo_batch_2d(uint32_t b, int pk, const CompressArgs* fields, const uint64_t* tile_prefix,
                                    int nfields, uint64_t total_tiles, unsigned long long* ticket, LaunchShape sh,
                                    cudaStream_t s, int* occ = nullptr);
cudaError_t launch_lorenzo_batch_3d(uint32_t b, int pk, const CompressArgs* fields, const uint64_t* tile_prefix,
                                    int nfields, uint64_t total_tiles, unsigned long long* ticket, LaunchShape sh,
                                    cudaStream_t s, int* occ = nullptr);

cudaError_t launch_recon_batch_1d(uint32_t b, const ReconArgs* fields, const uint64_t* tile_prefix, int nfields,
                                  uint64_t total_tiles, unsigned long long* ticket, LaunchShape sh, cudaStream_t s,
                                  int* occ = nullptr);
cudaError_t launch_recon_batch_2d(uint32_t b, const ReconArgs* fields, const uint64_t* tile_prefix, int nfields,
                                  uint64_t total_tiles, unsigned long long* ticket, LaunchShape sh, cudaStream_t s,
                                  int* occ = nullptr);
cudaError_t launch_recon_batch_3d(uint32_t b, const ReconArgs* fields, const uint64_t* tile_prefix, int nfields,
                                  uint64_t total_tiles, unsigned long long* ticket, LaunchShape sh, cudaStream_t s,
                                  int* occ = nullptr);

int num_sms();

int grid_for(const void* kernel, int threads, size_t smem, uint64_t work_items_per_cta, uint64_t work);
// Resident CTAs per SM of `kernel` at this block size and dynamic shared
// memory (0 if it cannot launch), cached per (kernel, threads, smem).
int occupancy(const void* kernel, int threads, size_t smem);
// As grid_for, with at most `ctas` resident CTAs per SM (0 = no cap).
int grid_shape(const void* kernel, int threads, size_t smem, uint64_t per_cta, uint64_t work, int ctas);
// Raise the kernel's dynamic shared memory limit to at least `bytes`
// (never lowers it, so graphs captured with a larger shape stay valid).
cudaError_t raise_smem_attr(const void* kernel, size_t bytes);

// Host helpers of the C ABI (api.cu).
vsz_status make_geom(const vsz_params* p, Geom* g);
vsz_status check_compressed(const Geom& g, const vsz_params* p, const vsz_compressed* c);
vsz_status cuda_fail(cudaError_t e);
bool aligned(const void* p, size_t a);

}  // namespace vsz
