/*
 * vsz.h -- C ABI of the GB300 dual-quantization library (libvsz.so).
 *
 * The library implements the prediction-and-quantization step of SZ as the
 * paper "SIMD Lossy Compression for Scientific Data" (arXiv 2201.04614)
 * restates it (dual-quantization, Sec. III-A, Alg. 2), with the paper's
 * error-bound modes (Sec. II-B) and padding values (Sec. IV), and its inverse.
 * Every step runs in the library's own CUDA kernels for sm_103a.
 *
 * Conventions for every call:
 *  - Fields are fp32, C-order: dims[0] is the slowest axis, dims[ndim-1] the
 *    fastest (x).  Blocks are b^ndim boxes; blocks at the + edges are
 *    truncated.  Blocks are numbered in row-major order over the block grid.
 *  - "d_" pointers are device pointers; "h_" pointers are host pointers.
 *  - The caller owns every buffer.  The library allocates nothing on the
 *    compression and reconstruction paths (the batch API caches one small
 *    descriptor table per handle, freed by vsz_batch_destroy).
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  All calls are asynchronous on it unless stated otherwise, and
 *    none synchronizes the device, so sequences of calls can be captured
 *    into a CUDA graph.
 *  - Errors are returned as a vsz_status; nothing aborts, traps or throws.
 *    Errors that only the device can see (capacity overflow, inconsistent
 *    outlier data) are recorded in the vsz_header in device memory and are
 *    read with vsz_read_header().
 */
#ifndef VSZ_H
#define VSZ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define VSZ_ABI_VERSION 1

#if defined(__GNUC__)
#define VSZ_API __attribute__((visibility("default")))
#else
#define VSZ_API
#endif

typedef enum {
    VSZ_OK = 0,
    VSZ_ERR_INVALID_ARG = 1,  /* a NULL pointer, a bad size or parameter */
    VSZ_ERR_UNSUPPORTED = 2,  /* valid for the method, not built (e.g. ndim 4) */
    VSZ_ERR_CAPACITY = 3,     /* outlier or fixup lists longer than the caller's capacity */
    VSZ_ERR_CUDA = 4,         /* a CUDA launch or runtime call failed */
    VSZ_ERR_CORRUPT = 5,      /* reconstruction met a code 0 with no matching outlier */
    VSZ_ERR_TOO_LARGE = 6     /* the call needs more scratch than vsz_compress_noalloc's fixed workspace */
} vsz_status;

/* Sec. II-B: absolute, or value-range relative (eb * (max - min)). */
typedef enum { VSZ_EB_ABS = 0, VSZ_EB_REL = 1 } vsz_eb_mode;

/* Sec. IV: padding value standing in for every Lorenzo neighbour outside a
 * block: zero (cuSZ), or the min / max / average of the prequantized data,
 * over the whole field (global, Sec. IV-B-1), per block (Sec. IV-B-2), or
 * per block and axis (edge, Sec. IV-B-3).
 * Edge granularity keeps ndim scalars per block: the scalar of axis k is the
 * statistic of the block's face at local coordinate 0 along k (k = 0 the
 * slowest axis), and a neighbour outside along several axes takes the
 * rounded mean of their scalars (the paper leaves those corners open).  With
 * the first-order Lorenzo predictor such a layer changes only the residual
 * of the block origin: it is q minus the inclusion-exclusion sum, over the
 * non-empty sets S of axes, of (-1)^(|S|+1) times the value of S. */
typedef enum {
    VSZ_PAD_ZERO = 0,
    VSZ_PAD_GLOBAL_MIN = 1,
    VSZ_PAD_GLOBAL_MAX = 2,
    VSZ_PAD_GLOBAL_AVG = 3,
    VSZ_PAD_BLOCK_MIN = 4,
    VSZ_PAD_BLOCK_MAX = 5,
    VSZ_PAD_BLOCK_AVG = 6,
    VSZ_PAD_EDGE_MIN = 7,
    VSZ_PAD_EDGE_MAX = 8,
    VSZ_PAD_EDGE_AVG = 9
} vsz_pad_mode;

/* The paper's statement of the problem: field dims, block size, error bound
 * and its mode, quantization radius, padding mode. */
typedef struct {
    int32_t  ndim;       /* 1, 2 or 3 (4D is VSZ_ERR_UNSUPPORTED) */
    uint64_t dims[3];    /* C-order extents, dims[0] slowest; product < 2^32 */
    uint32_t block;      /* block edge b, a power of two: 1D 4..256, 2D 4..128, 3D 4..32 */
    double   eb;         /* error bound, finite and > 0 */
    int32_t  eb_mode;    /* vsz_eb_mode */
    uint32_t radius;     /* R, 1..32768: codes are delta+R in [1, 2R-1], 0 = outlier */
    int32_t  pad;        /* vsz_pad_mode */
} vsz_params;

/* Per-field header in device memory (caller-allocated, sizeof(vsz_header)
 * bytes, 8-byte aligned).  Compression writes it; reconstruction reads the
 * scalars it needs from it, so no host round trip is needed between them. */
typedef struct {
    double   eb_abs;       /* absolute error bound used (Sec. II-B) */
    float    inv2eb;       /* (float)(1 / (2 eb_abs)), rounded once */
    float    ebx2;         /* (float)(2 eb_abs) */
    float    eb_f32;       /* largest float <= eb_abs: the guard's bound */
    float    xmin, xmax;   /* finite range of the input (valid if has_range) */
    int32_t  pad_global;   /* P for ZERO and GLOBAL_* modes (q domain) */
    uint32_t has_range;
    uint32_t status;       /* 0, or a vsz_status raised by compression */
    uint32_t recon_status; /* 0, or a vsz_status raised by reconstruction */
    uint32_t reserved;
    uint64_t n_out;        /* outliers: exact count, even on overflow */
    uint64_t n_fix;        /* fixups: exact count, even on overflow */
} vsz_header;

/* A compressed field: caller-owned device buffers. */
typedef struct {
    uint16_t*   codes;     /* [n] quantization codes, field layout */
    int32_t*    pad;       /* [nb] per-block padding values (BLOCK_* modes), [nb * ndim] (EDGE_* modes);
                              else may be NULL */
    uint32_t*   blk_off;   /* [nb+1] outlier offsets per block, canonical order */
    uint32_t*   out_idx;   /* [out_cap] global linear index of each outlier */
    int32_t*    out_delta; /* [out_cap] its residual delta */
    uint64_t    out_cap;
    uint32_t*   fix_idx;   /* [fix_cap] index of each fixup (value kept verbatim) */
    uint32_t*   fix_bits;  /* [fix_cap] raw fp32 bits of x */
    uint64_t    fix_cap;
    vsz_header* hdr;       /* device header */
} vsz_compressed;

/* Human-readable name of a status.  Never NULL. */
VSZ_API const char* vsz_status_string(vsz_status s);

/* Text of the last CUDA error that made a call on this host thread return
 * VSZ_ERR_CUDA ("" if none).  Never NULL; valid until the next failing call. */
VSZ_API const char* vsz_last_cuda_error(void);

/* VSZ_ABI_VERSION of the loaded library. */
VSZ_API int vsz_abi_version(void);

/* Host-side check of a parameter set: VSZ_OK, VSZ_ERR_INVALID_ARG or
 * VSZ_ERR_UNSUPPORTED.  No GPU work. */
VSZ_API vsz_status vsz_validate(const vsz_params* p);

/* Number of elements and of blocks of the field (0 if p is invalid). */
VSZ_API uint64_t vsz_num_elems(const vsz_params* p);
VSZ_API uint64_t vsz_num_blocks(const vsz_params* p);

/* Bytes of device workspace that vsz_prequant_lorenzo / vsz_outlier_compact
 * need for this field when the caller's lists hold out_cap outliers and
 * fix_cap fixups (0 if p is invalid).  The workspace is caller-owned, must
 * be 256-byte aligned, and must not be shared by calls in flight at once. */
VSZ_API size_t vsz_workspace_size(const vsz_params* p, uint64_t out_cap, uint64_t fix_cap);

/* Bytes of a workspace whose outlier staging is laid out in block slots
 * (2D/3D fields; the same as vsz_workspace_size for 1D fields): one slot of
 * b^ndim + 1 entries per block, so the staging holds at least
 * nb * (b^ndim + 1) entries whatever out_cap is.  With such a workspace the
 * compression writes every outlier straight into its block's slot, in
 * canonical order, and never walks a tile twice for its outliers however
 * dense they are (at tight error bounds most residuals can be outliers;
 * Sec. V-H counts them per padding mode).  Results are identical with either
 * size; vsz_prequant_lorenzo and vsz_outlier_compact use the slot layout when
 * ws_bytes is at least this large. */
VSZ_API size_t vsz_workspace_size_dense(const vsz_params* p, uint64_t out_cap, uint64_t fix_cap);

/*
 * Compression, step 1 (Sec. III-A, Alg. 2; Sec. IV; Sec. II-B): error-bound
 * resolution, prequantization q = rint(x * inv2eb), padding value, blockwise
 * first-order Lorenzo prediction, post-quantization into uint16 codes, and
 * the fp32 error-bound guard.  Writes c->codes, c->pad (block modes),
 * c->hdr (scalars), and leaves per-tile outlier and fixup lists staged in
 * the workspace.  For VSZ_EB_REL the value range is reduced on the device;
 * no host synchronization happens.
 *   p         field and method parameters (host)
 *   d_x       [n] fp32 input (device), 16-byte aligned for the vector path
 *   c         output buffers (host struct of device pointers)
 *   d_ws      workspace of at least vsz_workspace_size(p, c->out_cap, c->fix_cap) bytes
 * Returns VSZ_ERR_INVALID_ARG / VSZ_ERR_UNSUPPORTED before any GPU work on
 * bad input, VSZ_ERR_CUDA if a launch fails.
 */
VSZ_API vsz_status vsz_prequant_lorenzo(const vsz_params* p, const float* d_x, vsz_compressed* c,
                                void* d_ws, size_t ws_bytes, void* stream);

/*
 * Compression, step 2: outlier compaction.  Places the staged outliers and
 * fixups in canonical order (blocks in row-major block order, elements
 * row-major inside each block) in c->out_idx/out_delta and c->fix_idx/
 * fix_bits, writes c->blk_off[0..nb] and c->hdr->n_out / n_fix.  If a list
 * is longer than its capacity, the counts and blk_off are still exact, the
 * lists are truncated and c->hdr->status = VSZ_ERR_CAPACITY; retry with
 * larger buffers.  Must follow vsz_prequant_lorenzo on the same workspace.
 */
VSZ_API vsz_status vsz_outlier_compact(const vsz_params* p, vsz_compressed* c,
                               void* d_ws, size_t ws_bytes, void* stream);

/* Both compression steps in order. */
VSZ_API vsz_status vsz_compress(const vsz_params* p, const float* d_x, vsz_compressed* c,
                        void* d_ws, size_t ws_bytes, void* stream);

/* Bytes of the fixed workspace that vsz_compress_noalloc uses (16 MiB). */
#define VSZ_NOALLOC_WS_BYTES (16u << 20)

/*
 * vsz_compress without a caller-supplied workspace and without allocating
 * (the paper has no counterpart: this is a deployment aid).  Some callers
 * cannot allocate device memory: code running inside a framework whose
 * caching allocator already owns the GPU's memory, where a cudaMalloc of its
 * own fails or makes the framework release its caches, and latency-critical
 * paths that cannot accept the device-wide synchronization a cudaMalloc or
 * cudaFree may cause.  They pass inputs and outputs exactly as for
 * vsz_compress; the scratch is a fixed VSZ_NOALLOC_WS_BYTES array in the
 * library's own device memory, which every GPU that loads the library holds
 * until the process exits.  The call allocates nothing (no cudaMalloc, no
 * cudaFree, no allocating library routine).
 *  - Size limit: if vsz_workspace_size(p, c->out_cap, c->fix_cap) exceeds
 *    VSZ_NOALLOC_WS_BYTES the call returns VSZ_ERR_TOO_LARGE before any GPU
 *    work (use vsz_compress with your own workspace, or smaller capacities).
 *  - The first call on a device looks up the array's device address (once
 *    per device, with that device current); make that first call before any
 *    stream capture.
 *  - All calls share the one array, and it keeps the last call's contents;
 *    each call clears the parts that must start at zero itself.  Calls whose
 *    GPU work overlaps (on different streams, or from several host threads
 *    without ordering) race on it: order them on one stream.
 */
VSZ_API vsz_status vsz_compress_noalloc(const vsz_params* p, const float* d_x, vsz_compressed* c,
                                        void* stream);

/* ------------------------------------------------------------------------ */
/* One field split across GPUs: the per-rank steps.                        */
/* ------------------------------------------------------------------------ */
/*
 * Blocks are independent (Sec. III-A), so a field splits along dims[0] into
 * slabs of whole blocks (every slab but the last a multiple of the block
 * edge b along dims[0]), one per rank.  Three quantities cross slabs; the
 * caller reduces each over the ranks with its own collective (the Python
 * module paper_2201_04614_gb300.shard does it with torch.distributed):
 *  1. relative eb (Sec. II-B): vsz_slab_range per slab, then the min of the
 *     minima and the max of the maxima; the field's eb_abs is eb times their
 *     difference in double (eb itself if it is 0 or no slab has a finite
 *     value), exactly as the one-field call resolves it;
 *  2. a global padding mode (Sec. IV-B-1): vsz_slab_qstats per slab under
 *     the field's eb_abs, then the sums and counts added and the extremes
 *     reduced; P = min, max, or floor((2S + m) / (2m)) of the totals;
 *  3. vsz_compress_slab per slab with eb_abs and P, then the exclusive prefix
 *     over the ranks of the slabs' n_out (from their headers), and
 *     vsz_slab_rebase, which moves each slab's lists into the field's
 *     canonical order: the concatenation over the ranks of the slabs' codes,
 *     outlier lists, fixup lists, padding tables and blk_off[0..nb_slab) (then
 *     the last slab's blk_off[nb_slab]) is the whole field's compression.
 */
typedef struct {
    float    xmin, xmax;  /* finite range of the slab (valid if has_range) */
    uint32_t has_range;   /* the slab holds a finite value */
    uint32_t reserved;
    int64_t  qsum;        /* sum of q = rint(x * inv2eb) over every value (NaN gives 0) */
    int32_t  qmin, qmax;  /* extremes of q */
} vsz_slab_stats;

/* Finite min/max of the slab's n values into d_st->xmin/xmax/has_range
 * (device struct, caller-owned). */
VSZ_API vsz_status vsz_slab_range(const float* d_x, uint64_t n, vsz_slab_stats* d_st, void* stream);

/* Sum and extremes of q over the slab (p: the slab, absolute mode with the
 * field's eb_abs) into d_st->qsum/qmin/qmax. */
VSZ_API vsz_status vsz_slab_qstats(const vsz_params* p, const float* d_x, vsz_slab_stats* d_st, void* stream);

/* vsz_compress of one slab: p in absolute mode with the field's eb_abs (it
 * resolves to the same inv2eb, ebx2 and eb_f32); pad_value is the field's P
 * for a global padding mode and is ignored by the other modes.  Indices and
 * block offsets are the slab's own until vsz_slab_rebase. */
VSZ_API vsz_status vsz_compress_slab(const vsz_params* p, int32_t pad_value, const float* d_x, vsz_compressed* c,
                                     void* d_ws, size_t ws_bytes, void* stream);

/* Adds elem_base (the slab's first element in the field) to the slab's
 * outlier and fixup indices and out_base (the outliers of the earlier slabs)
 * to its blk_off[0..nb_slab]; the list lengths come from c->hdr. */
VSZ_API vsz_status vsz_slab_rebase(const vsz_params* p, const vsz_compressed* c, uint64_t elem_base,
                                   uint64_t out_base, void* stream);

/* ------------------------------------------------------------------------ */
/* Batches: many fields of uneven rank and size compressed together.        */
/* ------------------------------------------------------------------------ */

/* One field of a batch: its parameters, its fp32 input and its output
 * buffers, exactly as for vsz_compress. */
typedef struct {
    vsz_params     params;
    const float*   d_x;
    vsz_compressed out;
} vsz_field_job;

/* Opaque batch plan. */
typedef struct vsz_batch_st* vsz_batch;

/* Workspace bytes for a batch (0 if a job is invalid). */
VSZ_API size_t vsz_batch_workspace_size(const vsz_field_job* jobs, int njobs);

/*
 * Plan a batch (the batching pattern of this build; the paper processes one
 * field at a time with OpenMP over its blocks, Sec. III-F).  Fields are
 * grouped by class (rank, block edge, per-block padding or not); compressing
 * the batch then takes a fixed number of launches whatever the number of
 * fields: one initialisation, one value-range pass over every relative-eb
 * field, one global-statistics pass over every global-padding field, one
 * face-statistics pass over every edge-padding field, one
 * persistent compression kernel per class whose warps draw tiles of all the
 * class's fields from one queue, and two compaction kernels.  Results are
 * identical to vsz_compress on each field.  The plan keeps the jobs' pointers;
 * their buffers must outlive it.  The plan allocates its descriptor tables on
 * the device (freed by vsz_batch_destroy); d_ws (caller-owned, 256-byte
 * aligned) holds every field's compression workspace.  use_graph != 0
 * captures the launch sequence into a CUDA graph on the first submit and
 * replays it afterwards (not on the legacy default stream).
 */
VSZ_API vsz_status vsz_batch_create(const vsz_field_job* jobs, int njobs, void* d_ws, size_t ws_bytes,
                                    int use_graph, vsz_batch* out);

/* Compress every field of the batch, asynchronously on `stream`. */
VSZ_API vsz_status vsz_batch_submit(vsz_batch b, void* stream);

/* Free the plan (waits for nothing; do not destroy a plan with work in flight). */
VSZ_API vsz_status vsz_batch_destroy(vsz_batch b);

/*
 * Launch shapes of a batch and their autotuner (the batching pattern's tile
 * autotuner; the paper tunes only block size and vector length, by timing,
 * Sec. III-D).  Each class kernel is persistent: its warps claim tiles (a
 * 128-column segment of a row of blocks; 4096 values in 1D) from the
 * class's queue.  What is tuned is how that queue is served: warps per CTA
 * (2, 4 or 8), resident CTAs per SM, and whether the class kernels run one
 * after another or as parallel branches (so one class's tail overlaps the
 * next).  No shape changes any result.
 */
typedef struct {
    int32_t  ndim;
    uint32_t block;
    int32_t  pad_kind;     /* 0 zero, 1 per-block, 2 global, 3 edge padding (2, 3: origins deferred) */
    int32_t  nfields;      /* fields in the class */
    uint64_t tiles;        /* tiles of all of them */
    int32_t  warps;        /* warps per CTA of the class kernel (0 = default: 4, or 8 in 1D) */
    int32_t  ctas_per_sm;  /* resident CTAs per SM (0 = as many as fit) */
    float    ms;           /* last autotune: median device time of the class kernel with the chosen shape */
    float    ms_default;   /* last autotune: the same with the default shape (0 if never tuned) */
    int32_t  concurrent;   /* the plan runs this sequence's class kernels as parallel branches */
    int32_t  kind;         /* 0 compression class, 1 reconstruction class */
} vsz_batch_class;

/* Number of classes of a plan (0 if b is NULL), and one class's description.
 * Classes 0..k-1 are the compression classes (rank, block edge, padding
 * kind); after vsz_batch_set_outputs, the reconstruction classes (rank,
 * block edge) follow. */
VSZ_API int vsz_batch_num_classes(vsz_batch b);
VSZ_API vsz_status vsz_batch_get_class(vsz_batch b, int c, vsz_batch_class* out);

/* Set class c's launch shape (either kind): warps in {0, 2, 4, 8} (0 = default), ctas_per_sm
 * in 0..64 (0 = as many as fit; larger values are capped at what fits).
 * VSZ_ERR_UNSUPPORTED if the shape cannot launch (shared memory).  Drops
 * the cached graph (re-captured by the next submit). */
VSZ_API vsz_status vsz_batch_set_shape(vsz_batch b, int c, int warps, int ctas_per_sm);

/* Run the class kernels one after another (0) or as parallel branches (1):
 * in compression forked after the value-range pass and joined before the
 * origin pass, in reconstruction joined before the fixups.  Both sequences.
 * Drops the cached graphs. */
VSZ_API vsz_status vsz_batch_set_concurrent(vsz_batch b, int on);
/* As vsz_batch_set_concurrent, for the compression and the reconstruction
 * sequence separately (the autotuner may choose differently for each). */
VSZ_API vsz_status vsz_batch_set_concurrent_each(vsz_batch b, int compress_on, int reconstruct_on);

/*
 * Autotune the plan on its own inputs: for each class (compression, and
 * reconstruction when outputs are set), run its whole sequence `reps` times
 * (1..50) per candidate shape (warps 2, 4, 8 x CTAs per SM 1, 2, 4 and the
 * most that fit) and keep the shape with the smallest median device time of
 * the class kernel (the default shape unless another is faster); keep those
 * shapes only if the whole sequence runs faster with them than with the
 * default ones; then time each sequence serial and concurrent and keep the
 * faster.  Synchronous: it
 * waits for its own runs on `stream`, which must not be capturing
 * (VSZ_ERR_INVALID_ARG).  It compresses (and reconstructs) the batch many
 * times, with the same results each time, and drops the cached graphs.
 * Read the choices and times with vsz_batch_get_class.
 */
VSZ_API vsz_status vsz_batch_autotune(vsz_batch b, void* stream, int reps);

/*
 * Batch decompression (the inverse of Sec. III-A for every field of the
 * plan; the paper leaves decompression sequential).  vsz_batch_set_outputs
 * records one fp32 output per job (h_xhat: host array of njobs device
 * pointers, each [n_i] floats, 16-byte aligned for the vector path; NULL
 * allowed where n_i = 0), groups the fields by (rank, block edge) and
 * uploads one descriptor table per class (freed by vsz_batch_destroy or the
 * next vsz_batch_set_outputs).  vsz_batch_reconstruct then runs a fixed
 * sequence whatever the number of fields: one persistent inverse kernel per
 * class whose warps draw tiles of all the class's fields from one queue,
 * and one fixup kernel over every field.  It reads what the last
 * compression of the plan wrote (codes, lists, headers) and gives each
 * field exactly what vsz_reconstruct gives it.  Captured into a CUDA graph
 * on the first call and replayed, as vsz_batch_submit.  Errors only the
 * device sees go to each field's header (recon_status).
 */
VSZ_API vsz_status vsz_batch_set_outputs(vsz_batch b, float* const* h_xhat);
VSZ_API vsz_status vsz_batch_reconstruct(vsz_batch b, void* stream);

/* Host copies of one field's compressed output, for
 * vsz_batch_compress_host: the layout of vsz_compressed, in host memory
 * (page-locked memory keeps the copies at the host link's full speed). */
typedef struct {
    uint16_t*   codes;     /* [n] */
    int32_t*    pad;       /* [nb] (BLOCK_* modes), [nb * ndim] (EDGE_* modes); may be NULL otherwise */
    uint32_t*   blk_off;   /* [nb+1] */
    uint32_t*   out_idx;   /* [out_cap] */
    int32_t*    out_delta; /* [out_cap] */
    uint64_t    out_cap;
    uint32_t*   fix_idx;   /* [fix_cap] */
    uint32_t*   fix_bits;  /* [fix_cap] */
    uint64_t    fix_cap;
    vsz_header* hdr;       /* the field's header */
} vsz_host_field;

/*
 * Compression of a whole batch from host memory to host memory (the
 * dual-quant of Sec. III-A on every field of the plan, end to end): copies
 * each field's input h_x[i] ([n_i] floats in host memory) into the job's
 * device input d_x, runs the plan's compression exactly as
 * vsz_batch_submit (graph replay when the plan uses one), then copies each
 * field's header, codes, block offsets, padding table and its outlier and
 * fixup lists back into h_out[i].  The lists are copied at their exact
 * lengths, min(count, capacity) of both the device list and the host one;
 * the header carries the counts and any device-recorded status.  Blocking:
 * returns once the host buffers hold the result (it synchronizes `stream`
 * twice: after the headers, to learn the list lengths, and at the end).
 * h_x, h_out: host arrays of njobs entries.  Returns VSZ_ERR_INVALID_ARG on
 * a NULL buffer where the field needs one, VSZ_ERR_CUDA if a copy or a
 * launch fails; capacity overflow is reported in h_out[i].hdr->status.
 */
VSZ_API vsz_status vsz_batch_compress_host(vsz_batch b, const float* const* h_x, vsz_host_field* h_out,
                                           void* stream);

/* Bytes of the optional reconstruction workspace. */
#define VSZ_RECON_WS_BYTES 256

/*
 * Decompression (Sec. III-A: the inverse of the dual-quant): residuals from
 * the codes and the outlier lists, per-block inclusive prefix sums along x,
 * y and z, q = e + P, x_hat = (float)q * ebx2, then fixups restore their
 * values verbatim.  Reads the scalars from c->hdr.  |x - x_hat| <= eb(1+2^-20)
 * for every finite x; NaN/Inf come back bit for bit.  A code 0 without a
 * matching outlier sets c->hdr->recon_status = VSZ_ERR_CORRUPT.
 *   d_xhat    [n] fp32 output (device)
 *   d_ws      optional workspace of VSZ_RECON_WS_BYTES (device, 16-byte
 *             aligned) or NULL.  With it, tiles are handed to warps by an
 *             atomic ticket, which evens out tiles that hold many outliers;
 *             without it, tiles are assigned statically.  Calls in flight at
 *             the same time need distinct workspaces.
 */
VSZ_API vsz_status vsz_reconstruct(const vsz_params* p, const vsz_compressed* c, float* d_xhat,
                                   void* d_ws, size_t ws_bytes, void* stream);

/* Same inverse, writing the reconstructed prequantized integers q (int32[n])
 * instead of values (no fixups applied).  Used to verify that the inverse
 * reproduces the prequantization exactly. */
VSZ_API vsz_status vsz_reconstruct_q(const vsz_params* p, const vsz_compressed* c, int32_t* d_q,
                                     void* d_ws, size_t ws_bytes, void* stream);

/*
 * Code statistics (the learned tuner's labels): d_hist[0..2R-1] receives the
 * number of elements with each code (code 0 = outliers); codes at or above
 * 2R (not dual-quant codes) are not counted.  d_hist must hold 2R uint32
 * and is overwritten.  d_codes may have any 2-byte alignment.  Shannon
 * entropy of the codes follows from it on the host.
 */
VSZ_API vsz_status vsz_code_histogram(const vsz_params* p, const uint16_t* d_codes, uint32_t* d_hist,
                              void* stream);

/* ------------------------------------------------------------------------ */
/* Entropy stage: canonical Huffman coding of the quantization codes.       */
/* ------------------------------------------------------------------------ */
/*
 * Sec. II-B: SZ follows the prediction and quantization with Huffman coding
 * of the integer codes.  Symbols are the codes 0..nsym-1 (nsym = 2R for
 * dual-quant codes).  The codebook is a Huffman code of the symbols'
 * histogram (vsz_code_histogram), built by repeatedly merging the two
 * lightest nodes; among equal weights leaves come before merged nodes,
 * leaves in symbol order, merged nodes in the order they were made.
 * Codewords are canonical: symbols sorted by (length, symbol) get
 * consecutive codes.  A lone symbol gets length 1.  Lengths never exceed 64
 * for counts below 2^32.
 * The stream is cut into chunks of VSZ_HUFF_CHUNK symbols; each chunk starts
 * on a 32-bit word and fills words from the most significant bit down (the
 * unused tail bits are zero); chunk_off[c] is the first word of chunk c and
 * chunk_off[nchunks] the total, so chunks encode and decode independently.
 */
#define VSZ_HUFF_CHUNK 1024
#define VSZ_HUFF_MAX_SYMBOLS 8192   /* codebooks for R <= 4096 */

/* Bytes of a device codebook for nsym symbols (0 if nsym is 0 or above
 * VSZ_HUFF_MAX_SYMBOLS). */
VSZ_API size_t vsz_huffman_book_bytes(uint32_t nsym);

/* Build the codebook of d_hist[nsym] (uint32 counts, device) into d_book
 * (device, 16-byte aligned, vsz_huffman_book_bytes(nsym) bytes; opaque):
 * one CTA builds the tree, lengths and codewords, a second kernel the
 * decoder's lookup table.  VSZ_ERR_UNSUPPORTED if nsym > VSZ_HUFF_MAX_SYMBOLS. */
VSZ_API vsz_status vsz_huffman_book(const uint32_t* d_hist, uint32_t nsym, void* d_book, size_t book_bytes,
                                    void* stream);

/* Copy a codebook's lengths (h_len[nsym], 0 = unused symbol), codewords
 * (h_code[nsym], right-aligned) and longest length to the host; any of them
 * may be NULL.  Synchronizes the stream. */
VSZ_API vsz_status vsz_huffman_book_read(const void* d_book, uint32_t nsym, uint8_t* h_len, uint64_t* h_code,
                                         uint32_t* h_max_len, void* stream);

/* Bytes of the encoder's workspace (device, 8-byte aligned, caller-owned;
 * not shared by calls in flight at once). */
VSZ_API size_t vsz_huffman_encode_workspace_size(uint64_t n);

/* Encode d_sym[n] (uint16 symbols < nsym, device) into d_words (uint32,
 * word_cap words) and d_chunk_off[ceil(n / VSZ_HUFF_CHUNK) + 1] (uint64);
 * d_book as vsz_huffman_book wrote it (16-byte aligned, else
 * VSZ_ERR_INVALID_ARG).  *d_status (device uint32) receives bit 1 if a symbol has no codeword and
 * bit 2 if the stream is longer than word_cap words (the offsets are still
 * exact, so the caller can retry with chunk_off[nchunks] words). */
VSZ_API vsz_status vsz_huffman_encode(const uint16_t* d_sym, uint64_t n, const void* d_book, uint32_t nsym,
                                      uint32_t* d_words, uint64_t word_cap, uint64_t* d_chunk_off,
                                      uint32_t* d_status, void* d_ws, size_t ws_bytes, void* stream);

/* Decode n symbols from d_words (word_cap words readable) / d_chunk_off into
 * d_sym (uint16, device) with d_book (16-byte aligned, else
 * VSZ_ERR_INVALID_ARG).  *d_status receives bit 4 if a chunk holds no
 * valid codeword where one is expected or runs past its words (or past
 * word_cap).  Both calls set bit 8 if d_book was built for another nsym. */
VSZ_API vsz_status vsz_huffman_decode(const uint32_t* d_words, uint64_t word_cap, const uint64_t* d_chunk_off,
                                      uint64_t n, const void* d_book, uint32_t nsym, uint16_t* d_sym,
                                      uint32_t* d_status, void* stream);

/* Decode index (Sec. II-B's Huffman stage, decoded in parallel): the same
 * stream as vsz_huffman_encode (bit for bit), plus d_index[32 * nchunks]
 * (uint16, device): entry 32 c + j is the bit, relative to the start of
 * chunk c, where its codes 32 j .. 32 j + 31 begin (the chunk's total bits
 * for lanes past the end of the data).  The index is 64 bytes per chunk of
 * 1024 codes and is not part of the stream: it lets vsz_huffman_decode_indexed
 * give each chunk to a warp.  *d_status as vsz_huffman_encode, plus bit 16 if
 * a chunk holds 2^16 bits or more (its index entries are then truncated and
 * the stream must be decoded with vsz_huffman_decode).  VSZ_ERR_INVALID_ARG
 * as vsz_huffman_encode, or if d_index is NULL with n > 0. */
VSZ_API vsz_status vsz_huffman_encode_indexed(const uint16_t* d_sym, uint64_t n, const void* d_book, uint32_t nsym,
                                              uint32_t* d_words, uint64_t word_cap, uint64_t* d_chunk_off,
                                              uint16_t* d_index, uint32_t* d_status, void* d_ws, size_t ws_bytes,
                                              void* stream);

/* Decode n codes as vsz_huffman_decode, with the decode index of
 * vsz_huffman_encode_indexed: one warp per chunk, each lane decoding its 32
 * codes from its own starting bit.  Same outputs and status bits; bit 4 also
 * if a lane's codes do not end where the next lane's begin (a stream or an
 * index that do not belong together). */
VSZ_API vsz_status vsz_huffman_decode_indexed(const uint32_t* d_words, uint64_t word_cap, const uint64_t* d_chunk_off,
                                              const uint16_t* d_index, uint64_t n, const void* d_book, uint32_t nsym,
                                              uint16_t* d_sym, uint32_t* d_status, void* stream);

/* ------------------------------------------------------------------------ */
/* Learned tuner of block size and padding mode.                            */
/* ------------------------------------------------------------------------ */
/*
 * The paper picks the block size with a sampling autotuner (Sec. III-D,
 * Sec. V-E) and compares padding values by hand (Sec. IV, Sec. V-H).  This
 * library instead maps cheap sampled statistics of a field to a class
 * (block size x padding mode) with a small MLP, trained on the GPU with the
 * kernels below on labels from an exhaustive GPU sweep.  No call here
 * changes any integer result of compression: a class is only a vsz_params.
 *
 * Classes: c = 3 * slot + padslot; padslot 0 zero, 1 global average,
 * 2 block average (Sec. IV-B); block slots 1D {32, 64, 128, 256},
 * 2D {8, 16, 32, 64}, 3D {8, 16, 32} (slot 3 not allowed in 3D).
 */
#define VSZ_TUNER_NFEAT 12
#define VSZ_TUNER_NCLASS 12
#define VSZ_TUNER_HIDDEN 64
/* flat fp32 parameters: W1[64x12] b1[64] W2[64x64] b2[64] W3[12x64] b3[12], row-major */
#define VSZ_TUNER_NPARAM 5772

/* Bytes of workspace vsz_tuner_features needs (device, 16-byte aligned). */
VSZ_API size_t vsz_tuner_features_workspace_size(void);

/*
 * The 12 tuner features of a field, from S = min(n, 32768) samples at
 * linear indices (k * 2654435761) mod n: ndim one-hot (3); log10 n;
 * log10(range / eb_abs); log1p(mean |forward difference| / eb_abs) along x,
 * y, z (0 for absent axes); |mean| / range; std / range; the fraction of
 * samples with |q| >= R (under zero padding a block origin's residual is
 * q itself, Sec. IV-A); log2 R.  Statistics cover the finite samples; range
 * is theirs; eb_abs = eb, or eb * range in relative mode (Sec. II-B).
 * p->block and p->pad are ignored.
 *   d_feat    [12] double (device) or NULL;  d_feat32  [12] float or NULL
 */
VSZ_API vsz_status vsz_tuner_features(const vsz_params* p, const float* d_x, double* d_feat, float* d_feat32,
                                      void* d_ws, size_t ws_bytes, void* stream);

/* Bytes of workspace vsz_tuner_sweep needs (0 if p is invalid). */
VSZ_API size_t vsz_tuner_sweep_workspace_size(const vsz_params* p);

/*
 * Exhaustive sweep (the tuner's labels): compresses the field with every
 * allowed class (counting outliers and fixups exactly, keeping no lists),
 * takes the 2R-bin code histogram and writes the estimated size in bytes of
 * each class, n * H / 8 + 8 n_out + 8 n_fix + 4 * (padding scalars), with H
 * the Shannon entropy of the codes in bits per element (the Huffman stage
 * that follows the quantization, Sec. II-B), to d_cost[c]; +inf for classes
 * the rank does not allow.  p->block and p->pad are ignored.
 *   d_cost    [12] double (device)
 *   d_nout    [12] uint64 (device) or NULL: each class's outlier count
 *             (UINT64_MAX for classes not allowed)
 *   d_ws      workspace of vsz_tuner_sweep_workspace_size(p) bytes, 256-byte aligned
 */
VSZ_API vsz_status vsz_tuner_sweep(const vsz_params* p, const float* d_x, double* d_cost, uint64_t* d_nout,
                                   void* d_ws, size_t ws_bytes, void* stream);

/*
 * Guard of a tuned class: the exact outlier counts of classes a and b on a
 * fixed sample of the field (d_nout[0], d_nout[1], device uint64).  The
 * sample is the whole field when n <= 2^20 or dims[0] < 4 E0; otherwise K =
 * max(1, min(m0, floor(n / (50 r)))) regions (about 2% of the field) stacked
 * along dims[0] into one field and compressed with the same eb, eb mode and
 * R.  With L = 256 (1D), 64 (2D), 32 (3D): E0 = 65536 (1D) or L; region i
 * starts along dims[0] at floor(i * m0 / K) * E0, m0 = floor(dims[0] / E0);
 * a region is E0 values (1D), E0 rows (2D), or E0 planes of Ey = min(ny, L)
 * rows starting at row floor(i * my / K) * Ey, my = max(1, floor(ny / L))
 * (3D); r is a region's element count.  Regions are aligned to every
 * class's blocks, so each sampled block is a block of the field.  In
 * relative mode the error bound is relative to the sample's own range.
 * d_cost (device double[2], or NULL): the two classes' estimated sizes on
 * the sample, computed as vsz_tuner_sweep computes a class's cost.
 */
VSZ_API size_t vsz_tuner_guard_workspace_size(const vsz_params* p, int class_a, int class_b);
VSZ_API vsz_status vsz_tuner_guard(const vsz_params* p, const float* d_x, int class_a, int class_b,
                                   uint64_t* d_nout, double* d_cost, void* d_ws, size_t ws_bytes, void* stream);

/* Dims of the guard's stacked sample (host, no GPU work): sub_dims[0..2]. */
VSZ_API vsz_status vsz_tuner_guard_sample_dims(const vsz_params* p, uint64_t* sub_dims);

/*
 * The paper's own autotuner (Sec. III-D, Sec. V-E), kept as a baseline for
 * the learned tuner and the batch tile autotuner: an exhaustive search that
 * times the dual-quant (vsz_prequant_lorenzo) of every block size of the
 * rank (1D 32..256, 2D 8..64, 3D 8..32; the padding mode is p->pad) on a
 * sample of about sample_frac (0 < f <= 1) of the field's blocks, once to
 * warm up and then `iters` times (1..100), and keeps the block size with the
 * smallest mean time.  The sample is K regions spread evenly along dims[0]
 * and aligned to every candidate block (the guard's layout, with K from the
 * fraction); fields of at most 2^20 values, or shorter along dims[0] than
 * one region, are sampled whole.  On the GPU
 * the vector width the paper also tunes is fixed (16-byte lanes).
 * Synchronous (waits for its timing events; not under stream capture).
 *   h_best_block  the chosen block size (host)
 *   h_ms          [4] host, mean ms per block slot (-1 for slots the rank lacks), or NULL
 *   h_sample_elems  elements in the sample (host), or NULL
 *   d_ws          vsz_sampling_autotune_workspace_size(p, sample_frac) bytes, 256-byte aligned
 */
VSZ_API size_t vsz_sampling_autotune_workspace_size(const vsz_params* p, double sample_frac);
VSZ_API vsz_status vsz_sampling_autotune(const vsz_params* p, const float* d_x, double sample_frac, int iters,
                                         uint32_t* h_best_block, float* h_ms, uint64_t* h_sample_elems,
                                         void* d_ws, size_t ws_bytes, void* stream);

/*
 * MLP inference: for n samples X[n][12] (fp32, device) with allowed-class
 * bit masks d_mask[n], the logits z = W3 relu(W2 relu(W1 xt + b1) + b2) + b3
 * with xt = (x - mu) / sigma (d_norm = mu[12] then sigma[12]); masked
 * classes get -inf.  d_logits [n][12] and/or d_class [n] (the most probable
 * allowed class, ties to the lowest index) may be NULL.
 */
VSZ_API vsz_status vsz_mlp_forward(const float* d_theta, const float* d_norm, const float* d_X,
                                   const uint32_t* d_mask, int n, float* d_logits, int32_t* d_class,
                                   void* stream);

/* Bytes of workspace vsz_mlp_grad needs for a minibatch of `batch` samples. */
VSZ_API size_t vsz_mlp_grad_workspace_size(int batch);

/*
 * Mean masked-softmax cross-entropy over a minibatch and its gradient with
 * respect to the flat parameters (backpropagation).  The minibatch is the
 * samples d_idx[0..batch-1] (or 0..batch-1 when d_idx is NULL) of X / d_y /
 * d_mask.  Writes d_grad[VSZ_TUNER_NPARAM] and, if non-NULL, *d_loss.
 * Deterministic: every sum runs in a fixed order.
 */
VSZ_API vsz_status vsz_mlp_grad(const float* d_theta, const float* d_norm, const float* d_X, const int32_t* d_y,
                                const uint32_t* d_mask, const int32_t* d_idx, int batch, float* d_grad,
                                float* d_loss, void* d_ws, size_t ws_bytes, void* stream);

/* One Adam step (Kingma & Ba, 2015) at step >= 1 on nparam parameters, with
 * first and second moment buffers d_m, d_v (zero before step 1). */
VSZ_API vsz_status vsz_mlp_adam(float* d_theta, const float* d_grad, float* d_m, float* d_v, int nparam,
                                float lr, float beta1, float beta2, float eps, int step, void* stream);

/* One traced kernel launch. */
typedef struct {
    char     name[24];  /* kernel: begin, range, qstats, lorenzo, compact_scan, compact_move, recon, fixups, histogram */
    int32_t  ndim;      /* field rank (0 if not field-specific) */
    uint32_t block;     /* block edge (0 if not field-specific) */
    uint64_t n;         /* elements of the field */
    float    ms;        /* device time between the events around the launch (-1 if unknown) */
    uint32_t reserved;
} vsz_trace_record;

/* Launch tracing (profiling aid, no counterpart in the paper's method): when
 * on, every kernel the library launches is bracketed by two CUDA events on
 * its stream.  Off by default.  Not meant for streams under graph capture. */
VSZ_API vsz_status vsz_trace_enable(int on);

/* Waits for every traced launch since the last read, writes up to
 * max_records of them (oldest first) to h_out (host, may be NULL), clears
 * the list and returns how many launches were traced. */
VSZ_API int vsz_trace_read(vsz_trace_record* h_out, int max_records);

/* Copy the device header to the host and wait for it (synchronizes the
 * stream). */
VSZ_API vsz_status vsz_read_header(const vsz_compressed* c, vsz_header* h_out, void* stream);

/* The error the device recorded for this field, after the stream's work so
 * far: VSZ_OK, VSZ_ERR_CAPACITY (lists longer than their capacities; the
 * counts are exact) or VSZ_ERR_CORRUPT (reconstruction met a code 0 without
 * its outlier) -- the larger of the header's status and recon_status.
 * Synchronizes the stream; a failing copy returns VSZ_ERR_CUDA. */
VSZ_API vsz_status vsz_sync_status(const vsz_compressed* c, void* stream);

/* Failure injection for tests (host side; no kernel is involved): the k-th
 * device allocation the library makes for itself from now on (the tables
 * of vsz_batch_create and vsz_batch_set_outputs) fails as if the device
 * were out of memory, and the call that made it returns VSZ_ERR_CUDA after
 * releasing what it had allocated.  k = 0 switches it off; negative k is
 * VSZ_ERR_INVALID_ARG. */
VSZ_API vsz_status vsz_debug_fail_alloc(int k);

/* Bounds-checking build (compiled with -DVSZ_DEBUG_BOUNDS; a checking aid,
 * since no memory checker is available on every machine): the kernels check
 * the index of each write to a field-sized buffer (codes, values, lists,
 * block slots, tables) and of each read of the block slots and outlier
 * caches; an access out of its buffer is skipped and the site recorded.
 * Reads the first recorded site number (0 if none) into *out and clears it.
 * The normal build checks nothing and returns VSZ_ERR_UNSUPPORTED with 0. */
VSZ_API vsz_status vsz_debug_bounds_word(uint32_t* out);

/* Release what the library holds itself: tracing is switched off, pending
 * trace records are dropped and the recorder's CUDA events destroyed, and
 * the per-device and per-kernel caches of launch parameters (SM counts,
 * occupancies, shared-memory limits already raised) are cleared, so that the
 * library works again after the caller resets the device.  Buffers and batch
 * plans are the caller's (vsz_batch_destroy releases a plan).  Call it with
 * no library call in flight on any thread; later calls rebuild the caches.
 * Always VSZ_OK. */
VSZ_API vsz_status vsz_shutdown(void);

#ifdef __cplusplus
}
#endif
#endif /* VSZ_H */
