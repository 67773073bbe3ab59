"""Pins for the CPU oracle: it is checked against what the paper and the
mathematics fix, never against itself.

* hand-worked blocks (tests/golden/lorenzo_handworked.json, derived by hand);
* IEEE definitions of the prequantization (exact rational rounding);
* closed forms of the first-order Lorenzo residual (linear, bilinear and
  two-coordinate fields, constant fields under each padding);
* an independent formulation of the residual (the P-padded block differenced
  axis by axis) on brute-force sweeps of tiny shapes, with outlier counts and
  the canonical outlier order recounted directly;
* the round-trip guarantee |x - x_hat| <= eb (Sec. III-A) with the fp32 guard,
  checked in exact rational arithmetic, and NaN/Inf surviving bit for bit.
"""
import itertools
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "lorenzo_handworked.json")
I32_MIN, I32_MAX = -(2 ** 31), 2 ** 31 - 1


# ---------------------------------------------------------------- helpers
def exact_prequant(x: np.float32, inv2eb: np.float32) -> int:
    """Round-half-even of the IEEE single product, saturated; NaN -> 0."""
    with np.errstate(all="ignore"):
        p = np.float32(x) * np.float32(inv2eb)
    if np.isnan(p):
        return 0
    if np.isinf(p):
        return I32_MAX if p > 0 else I32_MIN
    r = round(Fraction(float(p)))  # Fraction rounds half to even
    return max(I32_MIN, min(I32_MAX, r))


def to_i32(a):
    a = np.asarray(a, dtype=np.int64) & 0xFFFFFFFF
    return a.astype(np.uint32).view(np.int32)


def block_slices(dims, b):
    grids = [range(0, d, b) for d in dims]
    for org in itertools.product(*grids):
        yield tuple(slice(o, min(o + b, d)) for o, d in zip(org, dims))


def separable_delta(q, dims, b, pads, block_mode):
    """Residual by a second formulation: pad each block on its low side with
    P and take first differences along every axis in turn."""
    qf = np.asarray(q, np.int64).reshape(dims)
    out = np.zeros(dims, np.int64)
    for k, sl in enumerate(block_slices(dims, b)):
        P = int(pads[k] if block_mode else pads[0])
        box = np.pad(qf[sl], [(1, 0)] * len(dims), mode="constant", constant_values=P)
        for ax in range(len(dims)):
            box = np.diff(box, axis=ax)
        out[sl] = box
    return to_i32(out.reshape(-1))


def canonical_order(dims, b):
    """Linear indices of the field in block-major, row-major-in-block order."""
    idx = np.arange(int(np.prod(dims))).reshape(dims)
    order = []
    for sl in block_slices(dims, b):
        order.append(idx[sl].reshape(-1))
    return np.concatenate(order) if order else np.zeros(0, np.int64)


def block_stat(q, dims, b, kind):
    qf = np.asarray(q, np.int64).reshape(dims)
    vals = []
    for sl in block_slices(dims, b):
        v = qf[sl].reshape(-1)
        if kind == "min":
            vals.append(int(v.min()))
        elif kind == "max":
            vals.append(int(v.max()))
        else:
            vals.append(math.floor(Fraction(int(v.sum()), v.size) + Fraction(1, 2)))
    return np.array(vals, np.int64)


# ------------------------------------------------------- hand-worked blocks
def load_golden():
    with open(GOLDEN) as f:
        return json.load(f)["cases"]


@pytest.mark.parametrize("case", load_golden(), ids=lambda c: c["name"])
def test_handworked_lorenzo(orc, case):
    p = orc.Params(tuple(case["dims"]), case["block"], 0.5, orc.EB_ABS, case["radius"],
                   orc.PAD_NAMES[case["pad"]])
    q = np.array(case["q"], np.int32)
    pads = orc.pad_values(p, q)
    assert pads.tolist() == case["P"]
    assert orc.lorenzo_delta(p, q, pads).tolist() == case["delta"]
    # With eb = 0.5 absolute, inv2eb = 1: x = q prequantizes to itself.
    c = orc.compress(p, q.astype(np.float32))
    assert c.q.tolist() == case["q"]
    d = np.array(case["delta"])
    R = case["radius"]
    exp_codes = np.where(np.abs(d) < R, d + R, 0)
    assert c.codes.astype(int).tolist() == exp_codes.tolist()
    if "codes" in case:
        assert c.codes.tolist() == case["codes"]
        assert c.out_idx.tolist() == case["out_idx"]
        assert c.out_delta.tolist() == case["out_delta"]
        assert c.blk_off.tolist() == case["blk_off"]
    xh, qh = orc.decompress(p, c, return_q=True)
    assert qh.tolist() == case["q"]


# ------------------------------------------------------- prequantization
@pytest.mark.parametrize("inv2eb", [0.5, 1.0, 3.0, 1.0 / 3.0, 1234.5678, 5e-4, 7.25e6])
def test_prequant_matches_exact_rounding(orc, inv2eb):
    rng = np.random.default_rng(7)
    x = np.concatenate([rng.normal(0, 1e3, 4000), rng.uniform(-10, 10, 4000),
                        rng.normal(0, 1e7, 500)]).astype(np.float32)
    q = orc.prequant(x, inv2eb)
    exp = [exact_prequant(v, np.float32(inv2eb)) for v in x]
    assert q.tolist() == exp


def test_prequant_ties_window(orc):
    """Every float within 6 ulps of each odd integer 2k+1, halved exactly by
    inv2eb = 0.5: exact ties must round to even."""
    xs = []
    for k in range(-60, 60):
        c = np.float32(2 * k + 1)
        v = c
        for _ in range(6):
            v = np.nextafter(v, np.float32(np.inf))
        hi = v
        v = c
        for _ in range(6):
            v = np.nextafter(v, np.float32(-np.inf))
        v0 = v
        while v0 <= hi:
            xs.append(v0)
            v0 = np.nextafter(v0, np.float32(np.inf))
    x = np.array(xs, np.float32)
    q = orc.prequant(x, 0.5)
    for xv, qv in zip(x, q):
        half = Fraction(float(xv)) / 2
        assert qv == round(half)
        assert abs(half - qv) <= Fraction(1, 2)  # |d - 2 d° eb| <= eb, Sec. III-A


def test_prequant_saturation_and_nan(orc):
    x = np.array([np.nan, np.inf, -np.inf, 3e9, -3e9, -2147483648.0, 2147483520.0,
                  2147483648.0, 0.0, -0.0, 0.49999997, -0.5, 0.5, 1.5, 2.5], np.float32)
    q = orc.prequant(x, 1.0)
    assert q.tolist() == [0, I32_MAX, I32_MIN, I32_MAX, I32_MIN, I32_MIN, 2147483520,
                          I32_MAX, 0, 0, 0, 0, 0, 2, 2]


# ------------------------------------------------------- error bound
def test_eb_resolution(orc):
    x = np.array([3.0, -1.5, np.nan, 7.25, np.inf, 2.0], np.float32)
    pa = orc.Params((6,), 4, 1e-3, orc.EB_ABS)
    ea = orc.resolve_eb(pa, x)
    assert ea.eb_abs == 1e-3
    pr = orc.Params((6,), 4, 1e-3, orc.EB_REL)
    er = orc.resolve_eb(pr, x)
    # Sec. II-B value-range relative: eb times (max - min) of the finite data.
    assert er.xmin == np.float32(-1.5) and er.xmax == np.float32(7.25)
    assert er.eb_abs == 1e-3 * (7.25 - (-1.5))
    for e in (ea, er):
        ex = Fraction(e.eb_abs)
        # eb_f32 is the largest float not above eb_abs
        assert Fraction(float(e.eb_f32)) <= ex
        assert Fraction(float(np.nextafter(e.eb_f32, np.float32(np.inf)))) > ex
        # inv2eb and ebx2 are correctly rounded (within half an ulp)
        t = 1 / (2 * ex)
        ulp = Fraction(float(np.spacing(e.inv2eb)))
        assert abs(Fraction(float(e.inv2eb)) - t) <= ulp / 2
        t2 = 2 * ex
        ulp2 = Fraction(float(np.spacing(e.ebx2)))
        assert abs(Fraction(float(e.ebx2)) - t2) <= ulp2 / 2


def test_eb_resolution_degenerate_range(orc):
    p = orc.Params((5,), 4, 1e-2, orc.EB_REL)
    assert orc.resolve_eb(p, np.full(5, 3.5, np.float32)).eb_abs == 1e-2
    assert orc.resolve_eb(p, np.full(5, np.nan, np.float32)).eb_abs == 1e-2
    with pytest.raises(ValueError):
        orc.resolve_eb(orc.Params((5,), 4, -1.0, orc.EB_ABS), np.zeros(5, np.float32))


# ------------------------------------------------------- closed forms
def _abs_half(dims, b, pad=0, R=512):
    import oracle
    return oracle.Params(tuple(dims), b, 0.5, oracle.EB_ABS, R, pad)


@pytest.mark.parametrize("b", [2, 3, 4, 5, 8])
def test_closed_form_linear_2d(orc, b):
    """q = a + s*i + t*j: the mixed difference vanishes inside a block, the
    first row of a block sees only the x-difference t, the first column only
    the y-difference s, and the block origin gets q - P."""
    ny, nx, a, s, t = 13, 11, 7, -3, 5
    i, j = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    q = (a + s * i + t * j).astype(np.int32)
    p = _abs_half((ny, nx), b)
    d = orc.lorenzo_delta(p, q, np.zeros(1, np.int32)).reshape(ny, nx)
    li, lj = i % b, j % b
    exp = np.where((li > 0) & (lj > 0), 0,
                   np.where((li == 0) & (lj > 0), t, np.where((li > 0) & (lj == 0), s, q)))
    assert (d == exp).all()


def test_closed_form_bilinear_2d(orc):
    ny, nx, c, b = 12, 12, 3, 4
    i, j = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    q = (c * i * j).astype(np.int32)
    d = orc.lorenzo_delta(_abs_half((ny, nx), b), q, np.zeros(1, np.int32)).reshape(ny, nx)
    inner = ((i % b) > 0) & ((j % b) > 0)
    assert (d[inner] == c).all()


def test_closed_form_two_coordinate_3d(orc):
    """In 3D the mixed difference of any sum of functions of at most two
    coordinates is zero, so every residual off the block's low faces is 0."""
    rng = np.random.default_rng(3)
    nz, ny, nx, b = 7, 9, 10, 4
    fzy = rng.integers(-50, 50, (nz, ny))
    fyx = rng.integers(-50, 50, (ny, nx))
    fzx = rng.integers(-50, 50, (nz, nx))
    q = (fzy[:, :, None] + fyx[None, :, :] + fzx[:, None, :]).astype(np.int32)
    d = orc.lorenzo_delta(_abs_half((nz, ny, nx), b), q, np.zeros(1, np.int32))
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    inner = ((z % b) > 0) & ((y % b) > 0) & ((x % b) > 0)
    assert (d.reshape(nz, ny, nx)[inner] == 0).all()


@pytest.mark.parametrize("dims,b", [((37,), 8), ((10, 13), 4), ((5, 6, 7), 3)])
def test_constant_field_padding(orc, dims, b):
    """Sec. V-H: on a constant field zero padding leaves exactly one non-zero
    residual per block (its origin, delta = q), so n_out = nb when |q| >= R;
    block- or global-average padding removes every outlier."""
    R = 16
    val = 40.0  # q = 40 with inv2eb = 1
    x = np.full(dims, val, np.float32)
    pz = _abs_half(dims, b, orc.PAD_ZERO, R)
    cz = orc.compress(pz, x)
    nb = pz.nblocks
    assert len(cz.out_idx) == nb and (cz.out_delta == 40).all()
    idx = np.arange(int(np.prod(dims))).reshape(dims)
    origins = [int(idx[sl].reshape(-1)[0]) for sl in block_slices(dims, b)]
    assert cz.out_idx.tolist() == origins
    for mode in (orc.PAD_BLOCK_AVG, orc.PAD_GLOBAL_AVG, orc.PAD_BLOCK_MIN, orc.PAD_GLOBAL_MAX):
        c = orc.compress(_abs_half(dims, b, mode, R), x)
        assert len(c.out_idx) == 0
        assert (c.codes == R).all()


# ------------------------------------------------------- padding values
def test_pad_values_exact(orc):
    rng = np.random.default_rng(11)
    for dims, b in [((17,), 4), ((9, 11), 3), ((5, 7, 6), 2), ((8,), 8)]:
        q = rng.integers(-1000, 1000, int(np.prod(dims))).astype(np.int32)
        for kind, mode in (("min", orc.PAD_BLOCK_MIN), ("max", orc.PAD_BLOCK_MAX),
                           ("avg", orc.PAD_BLOCK_AVG)):
            pads = orc.pad_values(_abs_half(dims, b, mode), q)
            assert pads.tolist() == block_stat(q, dims, b, kind).tolist()
        n = q.size
        assert orc.pad_values(_abs_half(dims, b, orc.PAD_GLOBAL_MIN), q)[0] == q.min()
        assert orc.pad_values(_abs_half(dims, b, orc.PAD_GLOBAL_MAX), q)[0] == q.max()
        g = math.floor(Fraction(int(q.astype(np.int64).sum()), n) + Fraction(1, 2))
        assert orc.pad_values(_abs_half(dims, b, orc.PAD_GLOBAL_AVG), q)[0] == g


@pytest.mark.parametrize("vals,exp", [([0, 1], 1), ([-1, 0], 0), ([-2, -1], -1),
                                      ([1, 2, 2], 2), ([-3, -3, -2], -3),
                                      ([I32_MAX, I32_MAX], I32_MAX),
                                      ([I32_MIN, I32_MIN, I32_MIN], I32_MIN)])
def test_average_rounds_half_up(orc, vals, exp):
    q = np.array(vals, np.int32)
    assert orc.pad_values(_abs_half((len(vals),), 64, orc.PAD_GLOBAL_AVG), q)[0] == exp


# ------------------------------------------------------- brute force
def _tiny_cases():
    rng = np.random.default_rng(2024)
    cases = []
    for ndim in (1, 2, 3):
        for _ in range(14 if ndim < 3 else 10):
            dims = tuple(int(v) for v in rng.integers(1, 10, ndim))
            b = int(rng.integers(1, 9))
            pad = int(rng.integers(0, 7))
            R = int(rng.choice([1, 2, 3, 512]))
            cases.append((dims, b, pad, R, int(rng.integers(0, 1 << 30))))
    return cases


@pytest.mark.parametrize("dims,b,pad,R,seed", _tiny_cases())
def test_brute_force_tiny(orc, dims, b, pad, R, seed):
    rng = np.random.default_rng(seed)
    n = int(np.prod(dims))
    # integers near +-R, a slow walk, and occasional spikes; eb = 0.5 abs
    walk = np.cumsum(rng.integers(-R - 1, R + 2, n)) + rng.integers(-3 * R, 3 * R)
    spikes = rng.random(n) < 0.1
    walk = np.where(spikes, walk + rng.integers(-5 * R, 5 * R + 1, n), walk)
    x = walk.astype(np.float32)
    p = _abs_half(dims, b, pad, R)
    c = orc.compress(p, x)
    assert (c.q == x.astype(np.int64)).all()
    block_mode = pad >= orc.PAD_BLOCK_MIN
    d = separable_delta(c.q, dims, b, c.pad, block_mode)
    is_out = np.abs(d.astype(np.int64)) >= R
    exp_codes = np.where(is_out, 0, d.astype(np.int64) + R)
    assert (c.codes.astype(np.int64) == exp_codes).all()
    # outliers: exactly the |delta| >= R positions, in canonical order
    canon = canonical_order(dims, b)
    exp_idx = canon[is_out[canon]]
    assert c.out_idx.tolist() == exp_idx.tolist()
    assert c.out_delta.tolist() == d[exp_idx].tolist()
    # per-block offsets count the outliers of each block
    counts = [int(is_out[np.arange(n).reshape(dims)[sl]].sum()) for sl in block_slices(dims, b)]
    assert c.blk_off.tolist() == np.concatenate([[0], np.cumsum(counts)]).tolist()
    # integer identity of the inverse, then the value
    xh, qh = orc.decompress(p, c, return_q=True)
    assert (qh == c.q).all()
    assert len(c.fix_idx) == 0
    assert (xh == x).all()


# ------------------------------------------------------- round trip / guard
def _check_bound(x, xh, eb_abs, fix_idx):
    """|x - x_hat| <= eb (1 + 2^-20) in exact arithmetic for finite x; NaN and
    Inf reproduced bit for bit."""
    tol = Fraction(eb_abs) * (1 + Fraction(1, 2 ** 20))
    xb, hb = x.view(np.uint32), xh.view(np.uint32)
    for i in range(x.size):
        if not np.isfinite(x[i]):
            assert xb[i] == hb[i]
            continue
        assert abs(Fraction(float(x[i])) - Fraction(float(xh[i]))) <= tol, i


def _check_fixups_minimal(c, x):
    """Every fixup is needed: without it the reconstruction q*ebx2 would
    miss the bound (or x is not finite)."""
    with np.errstate(all="ignore"):
        for i in c.fix_idx:
            xh = np.float32(np.float32(c.q[i]) * c.eb.ebx2)
            bad = (not np.isfinite(x[i])) or Fraction(abs(float(np.float32(x[i] - xh)))) > Fraction(float(c.eb.eb_f32))
            assert bad, i


@pytest.mark.parametrize("dims,b", [((300,), 16), ((23, 29), 8), ((9, 10, 11), 4), ((64, 64), 16)])
@pytest.mark.parametrize("eb", [1e-2, 1e-4, 1e-6])
def test_round_trip_bound_smooth(orc, dims, b, eb):
    x = synth.grf3d(dims, seed=5, slope=-3.0) * np.float32(100.0) + np.float32(50.0)
    for pad in (orc.PAD_ZERO, orc.PAD_BLOCK_AVG, orc.PAD_GLOBAL_MAX):
        p = orc.Params(dims, b, eb, orc.EB_REL, 512, pad)
        c = orc.compress(p, x)
        xh, qh = orc.decompress(p, c, return_q=True)
        assert (qh == c.q).all()
        _check_bound(x.reshape(-1), xh, c.eb.eb_abs, c.fix_idx)
        _check_fixups_minimal(c, x.reshape(-1))


@pytest.mark.parametrize("eb_abs", [0.5, 1e-3, 3e-7])
def test_round_trip_adversarial(orc, eb_abs):
    x = synth.adversarial_values(3000, seed=9, inv2eb=1.0 / (2 * eb_abs))
    for dims, b in [((3000,), 32), ((50, 60), 8), ((10, 15, 20), 4)]:
        for pad in (orc.PAD_ZERO, orc.PAD_GLOBAL_AVG, orc.PAD_BLOCK_MAX):
            p = orc.Params(dims, b, eb_abs, orc.EB_ABS, 512, pad)
            c = orc.compress(p, x)
            xh, qh = orc.decompress(p, c, return_q=True)
            assert (qh == c.q).all()
            _check_bound(x, xh, eb_abs, c.fix_idx)
            _check_fixups_minimal(c, x)
            nonfinite = np.flatnonzero(~np.isfinite(x))
            assert set(nonfinite.tolist()) <= set(c.fix_idx.tolist())


def test_decompress_rejects_missing_outlier(orc):
    p = _abs_half((8,), 4, orc.PAD_ZERO, 2)
    x = np.array([0, 9, 9, 9, 0, 0, 0, 0], np.float32)
    c = orc.compress(p, x)
    assert len(c.out_idx) >= 1
    c.out_idx = c.out_idx[:0]
    c.out_delta = c.out_delta[:0]
    c.blk_off = np.zeros_like(c.blk_off)
    with pytest.raises(ValueError):
        orc.decompress(p, c)


def test_padding_trend_unpinned(orc):
    """Sec. V-H reports fewer outliers with average padding; the size of the
    gain depends on the data (parity unpinned), so only the direction is
    checked on a field far from zero."""
    x = synth.fourier2d(256, 256, seed=4, value_range=10.0, offset=1000.0)
    nz = len(orc.compress(orc.Params((256, 256), 16, 1e-4, orc.EB_REL, 512, orc.PAD_ZERO), x).out_idx)
    na = len(orc.compress(orc.Params((256, 256), 16, 1e-4, orc.EB_REL, 512, orc.PAD_BLOCK_AVG), x).out_idx)
    assert na <= nz


# ------------------------------------------------------- edge granularity (Sec. IV-B-3)
def half_up_mean(vals):
    return math.floor(Fraction(int(sum(int(v) for v in vals)), len(vals)) + Fraction(1, 2))


def face_stats(q, dims, b, kind):
    """Per block and axis k (k = 0 slowest): the statistic of the block's
    in-field elements at local coordinate 0 along k."""
    qf = np.asarray(q, np.int64).reshape(dims)
    out = []
    for sl in block_slices(dims, b):
        box = qf[sl]
        for k in range(len(dims)):
            face = np.take(box, 0, axis=k).reshape(-1)
            out.append(int(face.min()) if kind == "min" else int(face.max()) if kind == "max"
                       else half_up_mean(face))
    return out


def edge_padded_delta(q, dims, b, pads):
    """Second formulation of the edge-padded residual: surround each block on
    its low sides with a layer whose cells outside along the axis set S hold
    the half-up mean of those axes' scalars, then take first differences
    along every axis in turn."""
    qf = np.asarray(q, np.int64).reshape(dims)
    d = len(dims)
    out = np.zeros(dims, np.int64)
    for bi, sl in enumerate(block_slices(dims, b)):
        Pk = [int(v) for v in pads[bi * d:(bi + 1) * d]]
        ext = tuple(s.stop - s.start for s in sl)
        box = np.zeros(tuple(e + 1 for e in ext), np.int64)
        for cell in itertools.product(*[range(e + 1) for e in ext]):
            S = [k for k in range(d) if cell[k] == 0]
            box[cell] = half_up_mean([Pk[k] for k in S]) if S else qf[sl][tuple(c - 1 for c in cell)]
        for ax in range(d):
            box = np.diff(box, axis=ax)
        out[sl] = box
    return to_i32(out.reshape(-1))


def origin_mask(dims, b):
    m = np.zeros(dims, bool)
    for sl in block_slices(dims, b):
        m[tuple(s.start for s in sl)] = True
    return m.reshape(-1)


def _edge_cases():
    rng = np.random.default_rng(77)
    out = []
    for ndim in (1, 2, 3):
        for _ in range(8):
            dims = tuple(int(v) for v in rng.integers(1, 10 if ndim < 3 else 8, ndim))
            out.append((dims, int(rng.integers(1, 7)), int(rng.integers(0, 1 << 30))))
    return out


@pytest.mark.parametrize("dims,b,seed", _edge_cases())
def test_edge_pad_values_and_residuals(orc, dims, b, seed):
    """Face statistics recomputed directly; residuals by the padded-layer
    formulation; and the consequence of first-order Lorenzo that a padding
    layer constant on each face changes only the block origin's residual:
    every other residual equals the zero-padding one, and the origin's is
    q - (sum over non-empty axis sets S of (-1)^(|S|+1) V(S))."""
    rng = np.random.default_rng(seed)
    n = int(np.prod(dims))
    q = rng.integers(-5000, 5000, n).astype(np.int32)
    pz = _abs_half(dims, b, orc.PAD_ZERO)
    dz = orc.lorenzo_delta(pz, q, np.zeros(1, np.int32))
    org = origin_mask(dims, b)
    for kind, mode in (("min", orc.PAD_EDGE_MIN), ("max", orc.PAD_EDGE_MAX), ("avg", orc.PAD_EDGE_AVG)):
        p = _abs_half(dims, b, mode)
        pads = orc.pad_values(p, q)
        assert pads.tolist() == face_stats(q, dims, b, kind)
        de = orc.lorenzo_delta(p, q, pads)
        assert de.tolist() == edge_padded_delta(q, dims, b, pads).tolist()
        assert (de[~org] == dz[~org]).all()
        d = len(dims)
        for bi, sl in enumerate(block_slices(dims, b)):
            Pk = [int(v) for v in pads[bi * d:(bi + 1) * d]]
            pred = sum((-1) ** (r + 1) * half_up_mean([Pk[k] for k in S])
                       for r in range(1, d + 1) for S in itertools.combinations(range(d), r))
            i0 = int(np.ravel_multi_index(tuple(s.start for s in sl), dims))
            assert int(de[i0]) == int(to_i32([int(q[i0]) - pred])[0])


@pytest.mark.parametrize("dims,b,seed", _edge_cases()[::2])
@pytest.mark.parametrize("R", [1, 3, 512])
def test_edge_round_trip_tiny(orc, dims, b, seed, R):
    """Codes, outliers and blk_off from the residuals; the inverse (element by
    element in row-major order) gives q back exactly."""
    rng = np.random.default_rng(seed + R)
    n = int(np.prod(dims))
    x = (np.cumsum(rng.integers(-R - 1, R + 2, n)) + rng.integers(-3 * R, 3 * R)).astype(np.float32)
    for mode in (orc.PAD_EDGE_MIN, orc.PAD_EDGE_MAX, orc.PAD_EDGE_AVG):
        p = _abs_half(dims, b, mode, R)
        c = orc.compress(p, x)
        assert len(c.pad) == max(1, p.nblocks * len(dims))
        d = edge_padded_delta(c.q, dims, b, c.pad)
        is_out = np.abs(d.astype(np.int64)) >= R
        assert (c.codes.astype(np.int64) == np.where(is_out, 0, d.astype(np.int64) + R)).all()
        canon = canonical_order(dims, b)
        assert c.out_idx.tolist() == canon[is_out[canon]].tolist()
        xh, qh = orc.decompress(p, c, return_q=True)
        assert (qh == c.q).all() and (xh == x).all()


@pytest.mark.parametrize("dims,b", [((37,), 8), ((10, 13), 4), ((5, 6, 7), 3)])
def test_edge_constant_field(orc, dims, b):
    """On a constant field every face scalar and corner value equals q, the
    inclusion-exclusion sum at the origin is q, and no residual is left."""
    x = np.full(dims, 40.0, np.float32)
    for mode in (orc.PAD_EDGE_MIN, orc.PAD_EDGE_MAX, orc.PAD_EDGE_AVG):
        c = orc.compress(_abs_half(dims, b, mode, 16), x)
        assert len(c.out_idx) == 0 and (c.codes == 16).all() and (c.pad == 40).all()
