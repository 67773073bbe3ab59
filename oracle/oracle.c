/*
 * oracle.c -- plain, single-threaded CPU dual-quantization oracle.
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h).  Written from the paper's text:
 *   Sec. II-B   error-bound modes: absolute and value-range relative;
 *   Sec. III-A  dual-quantization (Alg. 2): prequantize every value, predict
 *               the prequantized values with a Lorenzo predictor inside each
 *               block, post-quantize the residual into an integer code, keep
 *               out-of-range residuals aside; decompression reverses it;
 *   Sec. IV     padding values (zero, min, max, average; global, block or
 *               edge granularity).
 * Where the paper is silent (rounding, tie-breaking, the sentinel, the
 * outlier payload and order, the average's rounding, the fp32 guard), the
 * readings below are the ones the design notes list; each is marked
 * "reading:" where it is applied.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off (no -ffast-math), so that every
 * float expression is one IEEE single-precision operation as written.
 * No blocking, fusion or reordering: blocks are visited in row-major block
 * order and elements in row-major order inside each block.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ */
/* Field and block geometry                                            */
/* ------------------------------------------------------------------ */

typedef struct {
    int      d;          /* ndim */
    uint64_t n[3];       /* extents, n[0] slowest */
    uint64_t nb[3];      /* blocks per axis */
    uint64_t stride[3];  /* element strides, stride[d-1] == 1 */
    uint32_t b;          /* block edge */
} geom;

static int make_geom(const vszo_params* p, geom* g)
{
    if (!p || p->ndim < 1 || p->ndim > 3 || p->block < 1) return VSZO_ERR_ARG;
    g->d = p->ndim;
    g->b = p->block;
    for (int k = 0; k < g->d; ++k) {
        g->n[k] = p->dims[k];
        g->nb[k] = (p->dims[k] + p->block - 1) / p->block;
    }
    g->stride[g->d - 1] = 1;
    for (int k = g->d - 2; k >= 0; --k) g->stride[k] = g->stride[k + 1] * g->n[k + 1];
    return VSZO_OK;
}

uint64_t vszo_num_elems(const vszo_params* p)
{
    uint64_t n = 1;
    for (int k = 0; k < p->ndim; ++k) n *= p->dims[k];
    return n;
}

uint64_t vszo_num_blocks(const vszo_params* p)
{
    uint64_t nb = 1;
    for (int k = 0; k < p->ndim; ++k) nb *= (p->dims[k] + p->block - 1) / p->block;
    return nb;
}

/* Block number `blk` (row-major over the block grid) -> origin and extent. */
static void block_box(const geom* g, uint64_t blk, uint64_t org[3], uint64_t ext[3])
{
    for (int k = g->d - 1; k >= 0; --k) {
        uint64_t bi = blk % g->nb[k];
        blk /= g->nb[k];
        org[k] = bi * g->b;
        ext[k] = g->n[k] - org[k] < g->b ? g->n[k] - org[k] : g->b;
    }
}

/* Local coordinate l (row-major inside a box of extent ext) of local index i. */
static void local_coord(const geom* g, uint64_t i, const uint64_t ext[3], uint64_t l[3])
{
    for (int k = g->d - 1; k >= 0; --k) {
        l[k] = i % ext[k];
        i /= ext[k];
    }
}

static uint64_t box_size(const geom* g, const uint64_t ext[3])
{
    uint64_t m = 1;
    for (int k = 0; k < g->d; ++k) m *= ext[k];
    return m;
}

static uint64_t lin_index(const geom* g, const uint64_t org[3], const uint64_t l[3])
{
    uint64_t idx = 0;
    for (int k = 0; k < g->d; ++k) idx += (org[k] + l[k]) * g->stride[k];
    return idx;
}

/* ------------------------------------------------------------------ */
/* Sec. II-B: error-bound resolution                                   */
/* ------------------------------------------------------------------ */

int vszo_resolve_eb(const vszo_params* p, const float* x, vszo_eb* out)
{
    if (!p || !out || !(p->eb > 0.0) || !isfinite(p->eb)) return VSZO_ERR_ARG;
    uint64_t n = vszo_num_elems(p);
    memset(out, 0, sizeof(*out));

    /* Value range over the finite values (reading: NaN and +-Inf carry no
     * range information). */
    for (uint64_t i = 0; i < n; ++i) {
        float v = x[i];
        if (!isfinite(v)) continue;
        if (!out->has_range) {
            out->xmin = out->xmax = v;
            out->has_range = 1;
        } else {
            if (v < out->xmin) out->xmin = v;
            if (v > out->xmax) out->xmax = v;
        }
    }

    if (p->eb_mode == VSZO_EB_ABS) {
        out->eb_abs = p->eb;
    } else if (p->eb_mode == VSZO_EB_REL) {
        /* Value-range relative bound: eb times (max - min), in double.
         * reading: a field with no finite values or a zero range falls
         * back to eb itself. */
        double range = out->has_range ? (double)out->xmax - (double)out->xmin : 0.0;
        out->eb_abs = range > 0.0 ? p->eb * range : p->eb;
    } else {
        return VSZO_ERR_ARG;
    }

    /* reading: 1/(2 eb) and 2 eb are formed once in double and rounded once
     * to float; the comparison bound eb_f32 is the largest float that does
     * not exceed eb_abs. */
    out->inv2eb = (float)(1.0 / (2.0 * out->eb_abs));
    out->ebx2 = (float)(2.0 * out->eb_abs);
    float f = (float)out->eb_abs;
    if ((double)f > out->eb_abs) f = nextafterf(f, 0.0f);
    out->eb_f32 = f;
    return VSZO_OK;
}

/* ------------------------------------------------------------------ */
/* Sec. III-A / Alg. 2: prequantization                                */
/* ------------------------------------------------------------------ */

/* d° = round(d / (2 eb)), so that |d - 2 d° eb| <= eb.
 * reading: the quotient is one fp32 product d * inv2eb; it is rounded to
 * the nearest integer with ties to even (the default IEEE rounding mode),
 * converted to int32 with saturation, and NaN maps to 0. */
static int32_t prequant_one(float d, float inv2eb)
{
    float prod = d * inv2eb;
    if (isnan(prod)) return 0;
    float r = nearbyintf(prod);
    if (r >= 2147483648.0f) return INT32_MAX;
    if (r <= -2147483648.0f) return INT32_MIN;
    return (int32_t)r;
}

void vszo_prequant(const float* x, uint64_t n, float inv2eb, int32_t* q)
{
    for (uint64_t i = 0; i < n; ++i) q[i] = prequant_one(x[i], inv2eb);
}

/* ------------------------------------------------------------------ */
/* Sec. IV: padding value, in the prequantized (q) domain              */
/* ------------------------------------------------------------------ */

/* reading: the average is the exact integer mean rounded half up,
 * floor((2S + m) / (2m)) with S = sum of q (exact) and m = count. */
static int32_t rounded_mean(__int128 sum, uint64_t m)
{
    if (m == 0) return 0;
    __int128 num = 2 * sum + (__int128)m;
    __int128 den = 2 * (__int128)m;
    __int128 fl = num / den;                  /* C division truncates toward 0 */
    if ((num % den != 0) && (num < 0)) fl -= 1; /* make it a floor */
    return (int32_t)fl;
}

static int is_block_mode(int pad)
{
    return pad == VSZO_PAD_BLOCK_MIN || pad == VSZO_PAD_BLOCK_MAX || pad == VSZO_PAD_BLOCK_AVG;
}

static int is_edge_mode(int pad)
{
    return pad == VSZO_PAD_EDGE_MIN || pad == VSZO_PAD_EDGE_MAX || pad == VSZO_PAD_EDGE_AVG;
}

/* Min, max or rounded mean of the listed q values. */
static int32_t statistic(int kind_min_max_avg, const int32_t* vals, uint64_t m)
{
    if (m == 0) return 0;
    int32_t lo = vals[0], hi = vals[0];
    __int128 s = 0;
    for (uint64_t i = 0; i < m; ++i) {
        if (vals[i] < lo) lo = vals[i];
        if (vals[i] > hi) hi = vals[i];
        s += vals[i];
    }
    if (kind_min_max_avg == 0) return lo;
    if (kind_min_max_avg == 1) return hi;
    return rounded_mean(s, m);
}

int vszo_pad_values(const vszo_params* p, const int32_t* q, int32_t* pad)
{
    geom g;
    if (make_geom(p, &g)) return VSZO_ERR_ARG;
    uint64_t n = vszo_num_elems(p);
    switch (p->pad) {
    case VSZO_PAD_ZERO: /* cuSZ's default: borders are predicted from zeros */
        pad[0] = 0;
        return VSZO_OK;
    case VSZO_PAD_GLOBAL_MIN: /* Sec. IV-B-1: one scalar for the whole field */
        pad[0] = statistic(0, q, n);
        return VSZO_OK;
    case VSZO_PAD_GLOBAL_MAX:
        pad[0] = statistic(1, q, n);
        return VSZO_OK;
    case VSZO_PAD_GLOBAL_AVG:
        pad[0] = statistic(2, q, n);
        return VSZO_OK;
    case VSZO_PAD_BLOCK_MIN: /* Sec. IV-B-2: one scalar per block */
    case VSZO_PAD_BLOCK_MAX:
    case VSZO_PAD_BLOCK_AVG: {
        int kind = p->pad - VSZO_PAD_BLOCK_MIN;
        uint64_t nb = vszo_num_blocks(p);
        int32_t* tmp = (int32_t*)malloc(sizeof(int32_t) * (size_t)(g.b) *
                                        (g.d > 1 ? g.b : 1) * (g.d > 2 ? g.b : 1));
        if (!tmp) return VSZO_ERR_ARG;
        for (uint64_t blk = 0; blk < nb; ++blk) {
            uint64_t org[3], ext[3], l[3];
            block_box(&g, blk, org, ext);
            uint64_t m = box_size(&g, ext); /* reading: in-field elements only */
            for (uint64_t i = 0; i < m; ++i) {
                local_coord(&g, i, ext, l);
                tmp[i] = q[lin_index(&g, org, l)];
            }
            pad[blk] = statistic(kind, tmp, m);
        }
        free(tmp);
        return VSZO_OK;
    }
    case VSZO_PAD_EDGE_MIN: /* Sec. IV-B-3: one scalar per set of border values */
    case VSZO_PAD_EDGE_MAX:
    case VSZO_PAD_EDGE_AVG: {
        /* reading: the border values of a block along axis k are its
         * in-field elements at local coordinate 0 along k (those whose
         * predecessor along k lies outside the block); the scalar is their
         * min, max or rounded mean.  nb * ndim scalars in all. */
        int kind = p->pad - VSZO_PAD_EDGE_MIN;
        uint64_t nb = vszo_num_blocks(p);
        int32_t* tmp = (int32_t*)malloc(sizeof(int32_t) * (size_t)(g.b) *
                                        (g.d > 1 ? g.b : 1) * (g.d > 2 ? g.b : 1));
        if (!tmp) return VSZO_ERR_ARG;
        for (uint64_t blk = 0; blk < nb; ++blk) {
            uint64_t org[3], ext[3], l[3];
            block_box(&g, blk, org, ext);
            uint64_t m = box_size(&g, ext);
            for (int k = 0; k < g.d; ++k) {
                uint64_t c = 0;
                for (uint64_t i = 0; i < m; ++i) {
                    local_coord(&g, i, ext, l);
                    if (l[k] == 0) tmp[c++] = q[lin_index(&g, org, l)];
                }
                pad[blk * (uint64_t)g.d + (uint64_t)k] = statistic(kind, tmp, c);
            }
        }
        free(tmp);
        return VSZO_OK;
    }
    default:
        return VSZO_ERR_ARG;
    }
}

/* ------------------------------------------------------------------ */
/* Sec. III-A: blockwise first-order Lorenzo prediction                */
/* ------------------------------------------------------------------ */

/* Lorenzo residual of one element.  With e = q - P inside the block and
 * e = 0 outside it (reading: every neighbour outside the block takes the
 * padding value P, i.e. the shifted value e is zero there), the first-order
 * Lorenzo predictor is the signed sum over the 2^d - 1 neighbours at offsets
 * s in {0,1}^d \ {0}:
 *     pred = sum_{s != 0} (-1)^(|s|+1) e[l - s],
 * and the residual is  delta = e[l] - pred = sum_{s} (-1)^|s| e[l - s].
 * 1D: e[i] - e[i-1]; 2D: e - e_left - e_up + e_upleft; 3D: seven terms.
 * Integer arithmetic wraps modulo 2^32 (reading). */
static int32_t lorenzo_residual(const geom* g, const int32_t* q, int32_t P,
                                const uint64_t org[3], const uint64_t l[3])
{
    uint32_t acc = 0;
    for (unsigned s = 0; s < (1u << g->d); ++s) {
        uint64_t nbr[3];
        int inside = 1, parity = 0;
        for (int k = 0; k < g->d; ++k) {
            unsigned sk = (s >> (g->d - 1 - k)) & 1u;
            parity ^= (int)sk;
            if (sk && l[k] == 0) inside = 0;
            nbr[k] = l[k] - (sk ? 1 : 0);
        }
        uint32_t e = inside ? (uint32_t)q[lin_index(g, org, nbr)] - (uint32_t)P : 0u;
        acc = parity ? acc - e : acc + e;
    }
    return (int32_t)acc;
}

static int32_t block_pad(const vszo_params* p, const int32_t* pad, uint64_t blk)
{
    return is_block_mode(p->pad) ? pad[blk] : pad[0];
}

/* Edge granularity (Sec. IV-B-3): the value standing in for a neighbour
 * outside the block.  A neighbour outside along exactly one axis k takes
 * that axis's scalar Pk.  reading (the paper leaves the corners open): a
 * neighbour outside along a set S of several axes takes the rounded mean of
 * the scalars of the axes in S. */
static int32_t edge_value(int d, const int32_t* Pk, unsigned outside)
{
    __int128 sum = 0;
    uint64_t m = 0;
    for (int k = 0; k < d; ++k)
        if (outside & (1u << k)) {
            sum += Pk[k];
            ++m;
        }
    return rounded_mean(sum, m);
}

/* Lorenzo residual under edge padding: the same signed sum over the 2^d
 * neighbours at offsets s in {0,1}^d, on raw values, with every neighbour
 * outside the block replaced by its edge value:
 *     delta = sum_{s} (-1)^|s| v[l - s]. */
static int32_t lorenzo_residual_edge(const geom* g, const int32_t* q, const int32_t* Pk,
                                     const uint64_t org[3], const uint64_t l[3])
{
    uint32_t acc = 0;
    for (unsigned s = 0; s < (1u << g->d); ++s) {
        uint64_t nbr[3];
        unsigned outside = 0;
        int parity = 0;
        for (int k = 0; k < g->d; ++k) {
            unsigned sk = (s >> (g->d - 1 - k)) & 1u;
            parity ^= (int)sk;
            if (sk && l[k] == 0) outside |= 1u << k;
            nbr[k] = l[k] - (sk ? 1 : 0);
        }
        uint32_t v = outside ? (uint32_t)edge_value(g->d, Pk, outside) : (uint32_t)q[lin_index(g, org, nbr)];
        acc = parity ? acc - v : acc + v;
    }
    return (int32_t)acc;
}

/* Residual of one element under any padding mode. */
static int32_t residual(const vszo_params* p, const geom* g, const int32_t* q, const int32_t* pad,
                        uint64_t blk, const uint64_t org[3], const uint64_t l[3])
{
    if (is_edge_mode(p->pad)) return lorenzo_residual_edge(g, q, pad + blk * (uint64_t)g->d, org, l);
    return lorenzo_residual(g, q, block_pad(p, pad, blk), org, l);
}

int vszo_lorenzo_delta(const vszo_params* p, const int32_t* q, const int32_t* pad,
                       int32_t* delta)
{
    geom g;
    if (make_geom(p, &g)) return VSZO_ERR_ARG;
    uint64_t nb = vszo_num_blocks(p);
    for (uint64_t blk = 0; blk < nb; ++blk) {
        uint64_t org[3], ext[3], l[3];
        block_box(&g, blk, org, ext);
        uint64_t m = box_size(&g, ext);
        for (uint64_t i = 0; i < m; ++i) {
            local_coord(&g, i, ext, l);
            delta[lin_index(&g, org, l)] = residual(p, &g, q, pad, blk, org, l);
        }
    }
    return VSZO_OK;
}

/* ------------------------------------------------------------------ */
/* Whole compression side: prequant, Lorenzo, post-quant, outliers     */
/* ------------------------------------------------------------------ */

static uint32_t float_bits(float v)
{
    uint32_t u;
    memcpy(&u, &v, sizeof u);
    return u;
}

static float bits_float(uint32_t u)
{
    float v;
    memcpy(&v, &u, sizeof v);
    return v;
}

static int compress_impl(const vszo_params* p, const float* x, vszo_eb* eb,
                         uint16_t* codes, int32_t* q_out, int32_t* pad,
                         uint32_t* blk_off, uint32_t* out_idx, int32_t* out_delta,
                         uint64_t* n_out, uint32_t* fix_idx, uint32_t* fix_bits,
                         uint64_t* n_fix, const int32_t* global_pad);

int vszo_compress(const vszo_params* p, const float* x, vszo_eb* eb,
                  uint16_t* codes, int32_t* q_out, int32_t* pad,
                  uint32_t* blk_off, uint32_t* out_idx, int32_t* out_delta,
                  uint64_t* n_out, uint32_t* fix_idx, uint32_t* fix_bits,
                  uint64_t* n_fix)
{
    return compress_impl(p, x, eb, codes, q_out, pad, blk_off, out_idx, out_delta, n_out,
                         fix_idx, fix_bits, n_fix, NULL);
}

/* One slab of a field split across ranks along dims[0] in whole blocks:
 * blocks are independent (Sec. III-A), so the slab's compression is the
 * whole field's restricted to the slab, once the two field-wide quantities
 * it depends on are given: the error bound (pass p in absolute mode with the
 * field's eb_abs, which resolves to the same inv2eb, ebx2 and eb_f32) and,
 * for a global padding mode (Sec. IV-B-1), the field's padding value P,
 * which stands in for the slab's own.  Every other mode ignores P. */
int vszo_compress_given_pad(const vszo_params* p, const float* x, int32_t P, vszo_eb* eb,
                            uint16_t* codes, int32_t* pad, uint32_t* blk_off,
                            uint32_t* out_idx, int32_t* out_delta, uint64_t* n_out,
                            uint32_t* fix_idx, uint32_t* fix_bits, uint64_t* n_fix)
{
    return compress_impl(p, x, eb, codes, NULL, pad, blk_off, out_idx, out_delta, n_out,
                         fix_idx, fix_bits, n_fix, &P);
}

static int compress_impl(const vszo_params* p, const float* x, vszo_eb* eb,
                         uint16_t* codes, int32_t* q_out, int32_t* pad,
                         uint32_t* blk_off, uint32_t* out_idx, int32_t* out_delta,
                         uint64_t* n_out, uint32_t* fix_idx, uint32_t* fix_bits,
                         uint64_t* n_fix, const int32_t* global_pad)
{
    geom g;
    if (make_geom(p, &g)) return VSZO_ERR_ARG;
    if (p->radius < 1 || p->radius > 32768) return VSZO_ERR_ARG;
    uint64_t n = vszo_num_elems(p);
    if (n >= ((uint64_t)1 << 32)) return VSZO_ERR_ARG;
    int rc = vszo_resolve_eb(p, x, eb);
    if (rc) return rc;

    /* Alg. 2, prequantization of every datum into D°. */
    int32_t* q = (int32_t*)malloc(sizeof(int32_t) * (n ? n : 1));
    if (!q) return VSZO_ERR_ARG;
    vszo_prequant(x, n, eb->inv2eb, q);
    if (q_out) memcpy(q_out, q, sizeof(int32_t) * n);

    /* Sec. IV: the padding value(s). */
    rc = vszo_pad_values(p, q, pad);
    if (rc) { free(q); return rc; }
    if (global_pad && (p->pad == VSZO_PAD_GLOBAL_MIN || p->pad == VSZO_PAD_GLOBAL_MAX ||
                       p->pad == VSZO_PAD_GLOBAL_AVG))
        pad[0] = *global_pad;

    const int32_t R = (int32_t)p->radius;
    uint64_t nb = vszo_num_blocks(p);
    uint64_t no = 0, nf = 0;
    for (uint64_t blk = 0; blk < nb; ++blk) {
        uint64_t org[3], ext[3], l[3];
        block_box(&g, blk, org, ext);
        blk_off[blk] = (uint32_t)no;
        uint64_t m = box_size(&g, ext);
        for (uint64_t i = 0; i < m; ++i) {
            local_coord(&g, i, ext, l);
            uint64_t idx = lin_index(&g, org, l);
            /* Post-quantization: delta = d° - prediction (Sec. III-A).
             * reading: a residual with |delta| < R becomes the uint16 code
             * delta + R in [1, 2R-1]; otherwise the code is 0 and the pair
             * (index, delta) is kept aside as an outlier. */
            int32_t delta = residual(p, &g, q, pad, blk, org, l);
            if (delta > -R && delta < R) {
                codes[idx] = (uint16_t)(delta + R);
            } else {
                codes[idx] = 0;
                out_idx[no] = (uint32_t)idx;
                out_delta[no] = delta;
                ++no;
            }
            /* reading: fp32 rounding of d * inv2eb and q * 2eb can break the
             * bound; a value whose reconstruction q * ebx2 misses it (and
             * every NaN or Inf) is kept verbatim as a fixup, as the paper
             * keeps unpredictable data verbatim (Sec. III-A). */
            float xh = (float)q[idx] * eb->ebx2;
            if (!(fabsf(x[idx] - xh) <= eb->eb_f32)) {
                fix_idx[nf] = (uint32_t)idx;
                fix_bits[nf] = float_bits(x[idx]);
                ++nf;
            }
        }
    }
    blk_off[nb] = (uint32_t)no;
    *n_out = no;
    *n_fix = nf;
    free(q);
    return VSZO_OK;
}

/* ------------------------------------------------------------------ */
/* Decompression: the inverse of the dual-quant                        */
/* ------------------------------------------------------------------ */

/* Sec. III-A: decompression reverses the quantization.  The residual of the
 * first-order Lorenzo predictor is the mixed first difference of e along
 * every axis of the block, so e is recovered by an inclusive cumulative sum
 * along x, then y, then z inside the block (wrapping modulo 2^32); then
 * q = e + P and x_hat = (float)q * ebx2; fixups override. */
int vszo_decompress(const vszo_params* p, const vszo_eb* eb,
                    const uint16_t* codes, const int32_t* pad,
                    const uint32_t* blk_off, const uint32_t* out_idx,
                    const int32_t* out_delta, uint64_t n_out,
                    const uint32_t* fix_idx, const uint32_t* fix_bits,
                    uint64_t n_fix, int32_t* q_out, float* xhat)
{
    geom g;
    if (make_geom(p, &g)) return VSZO_ERR_ARG;
    const int32_t R = (int32_t)p->radius;
    uint64_t n = vszo_num_elems(p);
    uint64_t nb = vszo_num_blocks(p);
    size_t cap = (size_t)g.b * (g.d > 1 ? g.b : 1) * (g.d > 2 ? g.b : 1);
    uint32_t* e = (uint32_t*)malloc(sizeof(uint32_t) * cap);
    if (!e) return VSZO_ERR_ARG;
    int rc = VSZO_OK;

    for (uint64_t blk = 0; blk < nb && rc == VSZO_OK; ++blk) {
        uint64_t org[3], ext[3], l[3];
        block_box(&g, blk, org, ext);
        int32_t P = block_pad(p, pad, blk);
        uint64_t m = box_size(&g, ext);
        uint64_t lo = blk_off[blk], hi = blk_off[blk + 1];
        if (hi < lo || hi > n_out) { rc = VSZO_ERR_DATA; break; }

        /* Residuals: from the code, or from this block's outlier list. */
        for (uint64_t i = 0; i < m; ++i) {
            local_coord(&g, i, ext, l);
            uint64_t idx = lin_index(&g, org, l);
            if (codes[idx] != 0) {
                e[i] = (uint32_t)((int32_t)codes[idx] - R);
            } else {
                uint64_t j = lo;
                while (j < hi && out_idx[j] != idx) ++j;
                if (j == hi) { rc = VSZO_ERR_DATA; break; }
                e[i] = (uint32_t)out_delta[j];
            }
        }
        if (rc) break;

        if (is_edge_mode(p->pad)) {
            /* Edge granularity: invert delta = sum_s (-1)^|s| v[l - s]
             * element by element in row-major order, where every in-block
             * neighbour l - s (s != 0) is already reconstructed:
             *     q[l] = delta[l] - sum_{s != 0} (-1)^|s| v[l - s]. */
            const int32_t* Pk = pad + blk * (uint64_t)g.d;
            for (uint64_t i = 0; i < m; ++i) {
                local_coord(&g, i, ext, l);
                uint32_t acc = e[i];
                for (unsigned s = 1; s < (1u << g.d); ++s) {
                    uint64_t nbr[3];
                    unsigned outside = 0;
                    int parity = 0;
                    for (int k = 0; k < g.d; ++k) {
                        unsigned sk = (s >> (g.d - 1 - k)) & 1u;
                        parity ^= (int)sk;
                        if (sk && l[k] == 0) outside |= 1u << k;
                        nbr[k] = l[k] - (sk ? 1 : 0);
                    }
                    uint32_t v;
                    if (outside) {
                        v = (uint32_t)edge_value(g.d, Pk, outside);
                    } else {
                        uint64_t j = 0; /* local row-major index of the neighbour */
                        for (int k = 0; k < g.d; ++k) j = j * ext[k] + nbr[k];
                        v = e[j];
                    }
                    acc = parity ? acc + v : acc - v;
                }
                e[i] = acc;
            }
            for (uint64_t i = 0; i < m; ++i) {
                local_coord(&g, i, ext, l);
                uint64_t idx = lin_index(&g, org, l);
                int32_t qv = (int32_t)e[i];
                if (q_out) q_out[idx] = qv;
                xhat[idx] = (float)qv * eb->ebx2;
            }
            continue;
        }

        /* Inclusive cumulative sums along each axis, fastest axis first.
         * Visiting the box in row-major order, the element one step back
         * along axis a has already been summed. */
        for (int a = g.d - 1; a >= 0; --a) {
            uint64_t step = 1;
            for (int k = g.d - 1; k > a; --k) step *= ext[k];
            for (uint64_t i = 0; i < m; ++i) {
                local_coord(&g, i, ext, l);
                if (l[a] > 0) e[i] += e[i - step];
            }
        }

        for (uint64_t i = 0; i < m; ++i) {
            local_coord(&g, i, ext, l);
            uint64_t idx = lin_index(&g, org, l);
            int32_t qv = (int32_t)(e[i] + (uint32_t)P);
            if (q_out) q_out[idx] = qv;
            xhat[idx] = (float)qv * eb->ebx2;
        }
    }
    free(e);
    if (rc) return rc;

    for (uint64_t k = 0; k < n_fix; ++k) {
        if (fix_idx[k] >= n) return VSZO_ERR_DATA;
        xhat[fix_idx[k]] = bits_float(fix_bits[k]);
    }
    return VSZO_OK;
}

/* ------------------------------------------------------------------ */
/* Entropy stage: canonical Huffman coding of the quantization codes   */
/* ------------------------------------------------------------------ */

/* Sec. II-B: SZ entropy-codes the quantization codes with Huffman coding.
 * reading: the code is a plain Huffman code built from the code histogram
 * by repeatedly merging the two lightest nodes; among nodes of equal weight
 * leaves come before merged nodes, leaves in symbol order, merged nodes in
 * the order they were made.  A leaf's length is its depth (a lone symbol
 * gets length 1).  Codewords are canonical: symbols sorted by (length,
 * symbol) get consecutive codes, each shifted left when the length grows. */
int vszo_huffman_lengths(const uint32_t* hist, uint32_t nsym, uint8_t* len)
{
    /* nodes 0..nsym-1 are the leaves, nsym.. the merged nodes */
    uint64_t* w = (uint64_t*)malloc(sizeof(uint64_t) * 2 * (size_t)nsym);
    int32_t* parent = (int32_t*)malloc(sizeof(int32_t) * 2 * (size_t)nsym);
    uint8_t* alive = (uint8_t*)malloc(2 * (size_t)nsym);
    if (!w || !parent || !alive) { free(w); free(parent); free(alive); return VSZO_ERR_ARG; }
    uint32_t live = 0, next = nsym;
    for (uint32_t s = 0; s < nsym; ++s) {
        w[s] = hist[s];
        parent[s] = -1;
        alive[s] = hist[s] > 0;
        live += alive[s];
        len[s] = 0;
    }
    if (live == 1) {
        for (uint32_t s = 0; s < nsym; ++s) if (alive[s]) len[s] = 1;
    }
    while (live > 1) {
        /* the two lightest live nodes; node ids order the ties as the
         * reading says (leaves < merged; symbols ascending; merge order) */
        int64_t a = -1, b = -1;
        for (uint32_t i = 0; i < next; ++i) {
            if (!alive[i]) continue;
            if (a < 0 || w[i] < w[a]) { b = a; a = i; }
            else if (b < 0 || w[i] < w[b]) { b = i; }
        }
        w[next] = w[a] + w[b];
        parent[next] = -1;
        alive[next] = 1;
        parent[a] = (int32_t)next;
        parent[b] = (int32_t)next;
        alive[a] = alive[b] = 0;
        ++next;
        --live;
    }
    if (next > nsym) {
        for (uint32_t s = 0; s < nsym; ++s) {
            if (hist[s] == 0) continue;
            uint32_t d = 0;
            for (int32_t v = (int32_t)s; parent[v] >= 0; v = parent[v]) ++d;
            if (d > 64) { free(w); free(parent); free(alive); return VSZO_ERR_ARG; }
            len[s] = (uint8_t)d;
        }
    }
    free(w);
    free(parent);
    free(alive);
    return VSZO_OK;
}

int vszo_huffman_codes(const uint8_t* len, uint32_t nsym, uint64_t* code)
{
    uint64_t c = 0;
    int prev = 0, first = 1;
    for (int L = 1; L <= 64; ++L) {
        for (uint32_t s = 0; s < nsym; ++s) {
            if (len[s] != L) continue;
            if (first) { c = 0; first = 0; }
            else { c = (c + 1) << (L - prev); }
            prev = L;
            code[s] = c;
        }
    }
    for (uint32_t s = 0; s < nsym; ++s) if (len[s] == 0) code[s] = 0;
    return VSZO_OK;
}

/* reading: the stream is cut into chunks of `chunk` symbols; each chunk
 * starts on a 32-bit word boundary and its bits fill words from the most
 * significant bit down; chunk_off[c] is the first word of chunk c and
 * chunk_off[nchunks] the total.  A chunk's unused tail bits are zero. */
int vszo_huffman_encode(const uint16_t* sym, uint64_t n, const uint8_t* len, const uint64_t* code,
                        uint32_t nsym, uint32_t chunk, uint32_t* words, uint64_t* chunk_off)
{
    uint64_t nchunks = (n + chunk - 1) / chunk, wpos = 0;
    for (uint64_t c = 0; c < nchunks; ++c) {
        chunk_off[c] = wpos;
        uint64_t bit = 0; /* bits written in this chunk */
        uint64_t i1 = (c + 1) * chunk < n ? (c + 1) * chunk : n;
        for (uint64_t i = c * chunk; i < i1; ++i) {
            uint32_t s = sym[i];
            if (s >= nsym || len[s] == 0) return VSZO_ERR_DATA;
            for (int k = len[s] - 1; k >= 0; --k) {
                uint64_t wi = wpos + bit / 32;
                if (bit % 32 == 0) words[wi] = 0;
                if ((code[s] >> k) & 1u) words[wi] |= 1u << (31 - bit % 32);
                ++bit;
            }
        }
        wpos += (bit + 31) / 32;
    }
    chunk_off[nchunks] = wpos;
    return VSZO_OK;
}

/* Decoding reads bits one at a time and matches the accumulated prefix
 * against every symbol's (length, codeword); the code is prefix-free, so
 * the first match is the symbol. */
int vszo_huffman_decode(const uint32_t* words, const uint64_t* chunk_off, uint64_t n, const uint8_t* len,
                        const uint64_t* code, uint32_t nsym, uint32_t chunk, uint16_t* sym)
{
    uint64_t nchunks = (n + chunk - 1) / chunk;
    for (uint64_t c = 0; c < nchunks; ++c) {
        uint64_t bit = 0, wbase = chunk_off[c], wend = chunk_off[c + 1];
        uint64_t i1 = (c + 1) * chunk < n ? (c + 1) * chunk : n;
        for (uint64_t i = c * chunk; i < i1; ++i) {
            uint64_t acc = 0;
            int L = 0, found = 0;
            while (!found) {
                if (L == 64 || wbase + bit / 32 >= wend) return VSZO_ERR_DATA;
                acc = (acc << 1) | ((words[wbase + bit / 32] >> (31 - bit % 32)) & 1u);
                ++bit;
                ++L;
                for (uint32_t s = 0; s < nsym; ++s) {
                    if (len[s] == L && code[s] == acc) { sym[i] = (uint16_t)s; found = 1; break; }
                }
            }
        }
    }
    return VSZO_OK;
}
