/*
 * oracle.h -- plain, single-threaded CPU dual-quantization oracle.
 *
 * TEST INFRASTRUCTURE ONLY.  This file and oracle.c define what the
 * dual-quantization hot path computes, written straight from the paper
 * (SIMD Lossy Compression for Scientific Data, arXiv 2201.04614) so that a
 * reader can check it against the text.  Only the tests, the smoke check and
 * the CPU-baseline leg of the benchmark may load it.  It shares no code,
 * header, table or helper with the CUDA library under
 * paper_2201_04614_gb300/, and neither side includes the other.
 *
 * Conventions (the paper's notation where it has one):
 *   d      input value (fp32)                       -- Sec. III-A
 *   eb     user error bound, absolute or value-range relative -- Sec. II-B
 *   d°     prequantized value, kept as int32 q      -- Sec. III-A, Alg. 2
 *   δ°     post-quantization residual (delta)       -- Sec. III-A
 *   P      block padding value (q domain)           -- Sec. IV
 * Fields are C-order: dims[0] is the slowest axis, dims[ndim-1] the fastest
 * (x).  Blocks are b^ndim boxes; blocks at the + edges are truncated.
 */
#ifndef VSZ_ORACLE_H
#define VSZ_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { VSZO_EB_ABS = 0, VSZO_EB_REL = 1 };
enum {
    VSZO_PAD_ZERO = 0,
    VSZO_PAD_GLOBAL_MIN = 1,
    VSZO_PAD_GLOBAL_MAX = 2,
    VSZO_PAD_GLOBAL_AVG = 3,
    VSZO_PAD_BLOCK_MIN = 4,
    VSZO_PAD_BLOCK_MAX = 5,
    VSZO_PAD_BLOCK_AVG = 6,
    VSZO_PAD_EDGE_MIN = 7,
    VSZO_PAD_EDGE_MAX = 8,
    VSZO_PAD_EDGE_AVG = 9
};
enum { VSZO_OK = 0, VSZO_ERR_ARG = 1, VSZO_ERR_DATA = 2 };

typedef struct {
    int32_t  ndim;       /* 1, 2 or 3 */
    uint64_t dims[3];    /* dims[0..ndim-1], C-order */
    uint32_t block;      /* block edge b >= 1 */
    double   eb;         /* user error bound, > 0 */
    int32_t  eb_mode;    /* VSZO_EB_ABS or VSZO_EB_REL */
    uint32_t radius;     /* R, 1..32768 */
    int32_t  pad;        /* VSZO_PAD_* */
} vszo_params;

typedef struct {
    double  eb_abs;      /* absolute error bound actually used */
    float   inv2eb;      /* (float)(1 / (2 eb_abs)) */
    float   ebx2;        /* (float)(2 eb_abs) */
    float   eb_f32;      /* largest float <= eb_abs */
    float   xmin, xmax;  /* finite range (valid when has_range) */
    int32_t has_range;
} vszo_eb;

/* Number of elements and of blocks of a field. */
uint64_t vszo_num_elems(const vszo_params* p);
uint64_t vszo_num_blocks(const vszo_params* p);

/* Error-bound resolution, Sec. II-B. */
int vszo_resolve_eb(const vszo_params* p, const float* x, vszo_eb* out);

/* Prequantization d° = round(d / (2 eb)), Sec. III-A / Alg. 2. */
void vszo_prequant(const float* x, uint64_t n, float inv2eb, int32_t* q);

/* Padding values, Sec. IV-A/B.  pad receives 1 value for ZERO and GLOBAL_*
 * modes, one value per block (canonical block order) for BLOCK_* modes, and
 * ndim values per block for EDGE_* modes (Sec. IV-B-3): pad[blk*ndim + k]
 * is the statistic of the block's face at local coordinate 0 along axis k
 * (k = 0 the slowest axis). */
int vszo_pad_values(const vszo_params* p, const int32_t* q, int32_t* pad);

/* Lorenzo residuals δ° for every element (field layout), Sec. III-A. */
int vszo_lorenzo_delta(const vszo_params* p, const int32_t* q,
                       const int32_t* pad, int32_t* delta);

/* Whole compression-side dual-quant.  Array sizes: codes[n], q_out[n] (may be
 * NULL), pad[nb] (EDGE_*: [nb*ndim]; else [1]), blk_off[nb+1], out_idx/out_delta[n],
 * fix_idx/fix_bits[n].  Outliers and fixups are written in canonical order:
 * blocks in row-major block order, elements row-major inside a block. */
int vszo_compress(const vszo_params* p, const float* x, vszo_eb* eb,
                  uint16_t* codes, int32_t* q_out, int32_t* pad,
                  uint32_t* blk_off, uint32_t* out_idx, int32_t* out_delta,
                  uint64_t* n_out, uint32_t* fix_idx, uint32_t* fix_bits,
                  uint64_t* n_fix);

/* One whole-block slab of a field split along dims[0]: p in absolute mode
 * with the field's eb_abs; P the field's padding value for a global mode. */
int vszo_compress_given_pad(const vszo_params* p, const float* x, int32_t P, vszo_eb* eb,
                            uint16_t* codes, int32_t* pad, uint32_t* blk_off,
                            uint32_t* out_idx, int32_t* out_delta, uint64_t* n_out,
                            uint32_t* fix_idx, uint32_t* fix_bits, uint64_t* n_fix);

/* Decompression (inverse dual-quant).  q_out (may be NULL) receives the
 * reconstructed prequantized integers, xhat[n] the values. */
int vszo_decompress(const vszo_params* p, const vszo_eb* eb,
                    const uint16_t* codes, const int32_t* pad,
                    const uint32_t* blk_off, const uint32_t* out_idx,
                    const int32_t* out_delta, uint64_t n_out,
                    const uint32_t* fix_idx, const uint32_t* fix_bits,
                    uint64_t n_fix, int32_t* q_out, float* xhat);

/* Entropy stage (Sec. II-B): canonical Huffman code of the quantization
 * codes.  lengths: len[s] in 0..64 (0 = unused symbol); codes: canonical
 * codewords (right-aligned).  encode/decode: chunks of `chunk` symbols,
 * each starting on a 32-bit word, MSB first; chunk_off[nchunks + 1] word
 * offsets. */
int vszo_huffman_lengths(const uint32_t* hist, uint32_t nsym, uint8_t* len);
int vszo_huffman_codes(const uint8_t* len, uint32_t nsym, uint64_t* code);
int vszo_huffman_encode(const uint16_t* sym, uint64_t n, const uint8_t* len, const uint64_t* code,
                        uint32_t nsym, uint32_t chunk, uint32_t* words, uint64_t* chunk_off);
int vszo_huffman_decode(const uint32_t* words, const uint64_t* chunk_off, uint64_t n, const uint8_t* len,
                        const uint64_t* code, uint32_t nsym, uint32_t chunk, uint16_t* sym);

#ifdef __cplusplus
}
#endif
#endif /* VSZ_ORACLE_H */
