"""Plain CPU oracle of the learned tuner (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module.  It is numpy in float64 and shares no
code with the CUDA library.  The tuner chooses the block size and padding mode
of the dual-quantization (Sec. III-D block sizes, Sec. IV padding values) from
cheap sampled statistics of a field; its labels are the estimated size of the
quantization codes after the entropy stage (Sec. II-B: Huffman coding follows
the quantization) plus the sparse outliers (Sec. V-H counts them).

Definitions (the CUDA side computes the same quantities in its own kernels):

* sample points: k = 0..S-1 with S = min(n, 32768), linear index
  j_k = (k * 2654435761) mod n (a multiplicative hash, exact in integers);
* features (12): ndim one-hot (3); log10 n; log10(range / eb_abs);
  log1p(mean |d/dx| / eb_abs), log1p(mean |d/dy| / eb_abs),
  log1p(mean |d/dz| / eb_abs) (0 for absent axes; x is the fastest axis; the
  forward difference x[j + stride] - x[j] is taken where the neighbour is
  inside the field); |mean| / range; std / range (population); the fraction
  of samples with |q| >= R, q = rint(fl32(x * inv2eb)) (under zero padding a
  block origin's residual is q itself); log2 R.  Statistics run over the
  finite sampled values; range = max - min of them; eb_abs = eb (absolute)
  or eb * range (relative; eb when the range is 0); inv2eb =
  fl32(1 / (2 eb_abs)).  Ratios with a zero range are 0;
* classes: c = 3 * slot + padslot, padslot 0 = zero, 1 = global average,
  2 = block average; block slots 1D {32, 64, 128, 256}, 2D {8, 16, 32, 64},
  3D {8, 16, 32} (slot 3 masked);
* cost of a class (bytes): n * H / 8 + 8 n_out + 8 n_fix + 4 * (number of
  padding scalars), H the Shannon entropy (bits per element) of the 2R-bin
  code histogram (code 0 = outlier included), padding scalars nb for block
  modes, 1 for the global one, 0 for zero padding.  The label is the cheapest
  allowed class, ties to the lowest index;
* network: x~ = (x - mu) / sigma; h1 = relu(W1 x~ + b1) (64); h2 = relu(W2 h1
  + b2) (64); z = W3 h2 + b3 (12); softmax over the allowed classes; loss =
  mean cross-entropy.  Flat parameter layout W1[64x12], b1[64], W2[64x64],
  b2[64], W3[12x64], b3[12] (row-major, 5772 floats).  Gradients by the chain
  rule (backpropagation); Adam as Kingma & Ba (2015), bias-corrected.

Pins (tests/test_oracle_tuner.py): closed-form features of ramps, constants
and two-valued fields; entropies of uniform and two-point histograms; costs
recounted from the compression oracle on constant fields; a hand-worked
forward pass with non-zero weights in every layer, mu != 0, sigma != 1 and a
negative pre-activation in each hidden layer (tests/golden/
tuner_forward_handworked.json), which fixes the flat parameter layout too;
the gradient against central finite differences; Adam's first steps in
closed form, and a second step under a changed gradient.
"""
from __future__ import annotations

import math

import numpy as np

from . import Params, compress, EB_ABS, EB_REL, PAD_ZERO, PAD_GLOBAL_AVG, PAD_BLOCK_AVG

NFEAT = 12
NCLASS = 12
HID = 64
SAMPLE_MAX = 32768
HASH_MUL = 2654435761
PAD_SLOTS = (PAD_ZERO, PAD_GLOBAL_AVG, PAD_BLOCK_AVG)
BLOCKS = {1: (32, 64, 128, 256), 2: (8, 16, 32, 64), 3: (8, 16, 32)}
DEFAULT_BLOCK = {1: 256, 2: 16, 3: 8}

# flat parameter layout
SHAPES = [("W1", (HID, NFEAT)), ("b1", (HID,)), ("W2", (HID, HID)), ("b2", (HID,)),
          ("W3", (NCLASS, HID)), ("b3", (NCLASS,))]
NPARAM = sum(int(np.prod(s)) for _, s in SHAPES)


# ---------------------------------------------------------------- classes
def class_params(ndim: int, c: int):
    """(block, pad mode) of class c for a field of this rank, or None if the
    class is not allowed."""
    slot, ps = divmod(c, 3)
    blocks = BLOCKS[ndim]
    if slot >= len(blocks):
        return None
    return blocks[slot], PAD_SLOTS[ps]


def class_mask(ndim: int) -> int:
    """Bit c set when class c is allowed for this rank."""
    m = 0
    for c in range(NCLASS):
        if class_params(ndim, c) is not None:
            m |= 1 << c
    return m


def default_class(ndim: int) -> int:
    return 3 * BLOCKS[ndim].index(DEFAULT_BLOCK[ndim]) + 0


# ---------------------------------------------------------------- features
def sample_indices(n: int) -> np.ndarray:
    S = min(n, SAMPLE_MAX)
    k = np.arange(S, dtype=np.uint64)
    return ((k * np.uint64(HASH_MUL)) % np.uint64(max(n, 1))).astype(np.int64)


def features(x, dims, eb: float, eb_mode: int, radius: int) -> np.ndarray:
    """The 12 features of a field (float64)."""
    dims = tuple(int(d) for d in dims)
    nd = len(dims)
    x = np.ascontiguousarray(x, np.float32).reshape(-1)
    n = x.size
    f = np.zeros(NFEAT, np.float64)
    f[nd - 1] = 1.0
    f[11] = math.log2(radius)
    if n == 0:
        return f
    f[3] = math.log10(n)
    j = sample_indices(n)
    xs = x[j].astype(np.float64)
    fin = np.isfinite(xs)
    v = xs[fin]
    if v.size == 0:
        return f
    lo, hi = float(v.min()), float(v.max())
    rng = hi - lo
    eb_abs = eb if eb_mode == EB_ABS else (eb * rng if rng > 0 else eb)
    # strides of the axes, x (fastest) first
    strides, extents = [], []
    s = 1
    for d in reversed(dims):
        strides.append(s)
        extents.append(d)
        s *= d
    for a in range(nd):
        st, ext = strides[a], extents[a]
        coord = (j // st) % ext
        ok = coord + 1 < ext
        jj = j[ok]
        d = x[jj + st].astype(np.float64) - x[jj].astype(np.float64)
        d = np.abs(d[np.isfinite(d)])
        g = float(d.sum() / d.size) if d.size else 0.0
        f[5 + a] = math.log1p(g / eb_abs)
    f[4] = math.log10(rng / eb_abs) if rng > 0 else 0.0
    mean = float(v.sum() / v.size)
    var = float(((v - mean) ** 2).sum() / v.size)
    f[8] = abs(mean) / rng if rng > 0 else 0.0
    f[9] = math.sqrt(var) / rng if rng > 0 else 0.0
    inv2eb = np.float32(1.0 / (2.0 * eb_abs))
    with np.errstate(all="ignore"):
        p = v.astype(np.float32) * inv2eb          # one fp32 product
    q = np.rint(p.astype(np.float64))              # half to even
    f[10] = float(np.count_nonzero(np.abs(q) >= radius)) / v.size
    return f


# ---------------------------------------------------------------- labels
def code_entropy(hist) -> float:
    """Shannon entropy in bits per element of a histogram of codes."""
    h = np.asarray(hist, np.float64)
    n = h.sum()
    if n <= 0:
        return 0.0
    p = h[h > 0] / n
    return float(-(p * np.log2(p)).sum())


def class_cost(x, dims, eb, eb_mode, radius, c):
    """(cost in bytes, n_out, n_fix, entropy) of class c, from the compression
    oracle."""
    nd = len(dims)
    b, pad = class_params(nd, c)
    p = Params(tuple(dims), b, eb, eb_mode, radius, pad)
    r = compress(p, x)
    n = p.n
    hist = np.bincount(r.codes.astype(np.int64), minlength=2 * radius)
    H = code_entropy(hist)
    npad = p.nblocks if pad == PAD_BLOCK_AVG else (1 if pad == PAD_GLOBAL_AVG else 0)
    no, nf = len(r.out_idx), len(r.fix_idx)
    return n * H / 8.0 + 8.0 * no + 8.0 * nf + 4.0 * npad, no, nf, H


def sweep_costs(x, dims, eb, eb_mode, radius) -> np.ndarray:
    """Cost of every class (inf where not allowed)."""
    out = np.full(NCLASS, np.inf)
    for c in range(NCLASS):
        if class_params(len(dims), c) is not None:
            out[c] = class_cost(x, dims, eb, eb_mode, radius, c)[0]
    return out


# Estimated sizes within this fraction of the least count as equal, and the
# padding that costs least to compute wins among them: zero, then per block
# (a table written during the walk), then global (a statistic of the whole
# field and a second pass over the block origins).
SIZE_TOL = 0.005
PAD_RANK = (0, 2, 1)  # by padslot: zero, global average, block average


def label(costs) -> int:
    """The label of a field from its classes' estimated sizes: among the
    classes within SIZE_TOL of the least size, the one with the cheapest
    padding (PAD_RANK), then the smaller size, then the lower index."""
    costs = np.asarray(costs, np.float64)
    lo = float(np.min(costs))
    best = None
    for c in range(costs.size):
        if not (costs[c] <= lo * (1.0 + SIZE_TOL)):
            continue
        key = (PAD_RANK[c % 3], float(costs[c]), c)
        if best is None or key < best[0]:
            best = (key, c)
    return best[1]


# ---------------------------------------------------------------- network
def unflatten(theta) -> dict:
    theta = np.asarray(theta, np.float64)
    out, o = {}, 0
    for name, shp in SHAPES:
        k = int(np.prod(shp))
        out[name] = theta[o:o + k].reshape(shp)
        o += k
    return out


def flatten(parts: dict) -> np.ndarray:
    return np.concatenate([np.asarray(parts[name], np.float64).reshape(-1) for name, _ in SHAPES])


def forward(theta, mu, sigma, X, masks):
    """Logits z (masked classes set to -inf), probabilities p and the
    intermediate activations, for samples X[B, 12] with class masks[B]."""
    P = unflatten(theta)
    X = np.asarray(X, np.float64)
    xt = (X - np.asarray(mu, np.float64)) / np.asarray(sigma, np.float64)
    a1 = xt @ P["W1"].T + P["b1"]
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ P["W2"].T + P["b2"]
    h2 = np.maximum(a2, 0.0)
    z = h2 @ P["W3"].T + P["b3"]
    allowed = ((np.asarray(masks, np.int64)[:, None] >> np.arange(NCLASS)) & 1).astype(bool)
    zm = np.where(allowed, z, -np.inf)
    m = zm.max(axis=1, keepdims=True)
    e = np.where(allowed, np.exp(zm - m), 0.0)
    p = e / e.sum(axis=1, keepdims=True)
    return zm, p, (xt, a1, h1, a2, h2)


def loss(theta, mu, sigma, X, y, masks) -> float:
    _, p, _ = forward(theta, mu, sigma, X, masks)
    y = np.asarray(y, np.int64)
    return float(-np.log(p[np.arange(len(y)), y]).mean())


def loss_grad(theta, mu, sigma, X, y, masks):
    """Mean cross-entropy and its gradient by the chain rule."""
    P = unflatten(theta)
    _, p, (xt, a1, h1, a2, h2) = forward(theta, mu, sigma, X, masks)
    y = np.asarray(y, np.int64)
    B = len(y)
    L = float(-np.log(p[np.arange(B), y]).mean())
    dz = p.copy()
    dz[np.arange(B), y] -= 1.0
    dz /= B
    g = {"W3": dz.T @ h2, "b3": dz.sum(0)}
    dh2 = dz @ P["W3"]
    da2 = dh2 * (a2 > 0)
    g["W2"] = da2.T @ h1
    g["b2"] = da2.sum(0)
    dh1 = da2 @ P["W2"]
    da1 = dh1 * (a1 > 0)
    g["W1"] = da1.T @ xt
    g["b1"] = da1.sum(0)
    return L, flatten(g)


def adam_step(theta, grad, m, v, t: int, lr: float, beta1: float = 0.9, beta2: float = 0.999,
              eps: float = 1e-8):
    """One Adam update (Kingma & Ba, 2015) at step t >= 1; returns
    (theta, m, v)."""
    theta = np.asarray(theta, np.float64)
    g = np.asarray(grad, np.float64)
    m = beta1 * np.asarray(m, np.float64) + (1 - beta1) * g
    v = beta2 * np.asarray(v, np.float64) + (1 - beta2) * g * g
    mh = m / (1 - beta1 ** t)
    vh = v / (1 - beta2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def predict(theta, mu, sigma, X, masks) -> np.ndarray:
    """Most probable allowed class per sample, ties to the lowest index."""
    zm, _, _ = forward(theta, mu, sigma, X, masks)
    out = []
    for row in zm:
        best = 0
        for c in range(1, row.size):
            if row[c] > row[best]:
                best = c
        out.append(best)
    return np.array(out, np.int64)
