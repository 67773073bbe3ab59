"""Pins for the tuner oracle (oracle/tuner.py), checked against closed forms
and independent formulations, never against itself:

* the sample hash is a permutation of the field when n <= 32768, so sampled
  statistics are full-field statistics there;
* features of ramps, planes, constants and two-valued fields in closed form
  (derived by hand in each test);
* entropies of uniform and two-point histograms;
* class costs of constant fields from the closed-form outlier counts of
  first-order Lorenzo (one nonzero residual per block, at its origin);
* a hand-worked forward pass (tests/golden/tuner_forward_handworked.json):
  non-zero weights in every layer at their documented flat offsets, mu != 0,
  sigma != 1, a negative pre-activation in each hidden layer, an asymmetric
  W2 and a class removed only by the mask; planted mistakes (transposed W2,
  a dropped ReLU, swapped normalisation) each fail it;
* the gradient against central finite differences of the loss, and its b3
  part against the closed form mean(p - onehot(y));
* Adam's first steps in closed form (Kingma & Ba, 2015), and a second step
  under a changed gradient worked by hand.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from oracle import tuner as T


def test_sample_is_a_permutation_for_small_fields():
    for n in (1, 2, 7, 1000, 4096, 32768):
        j = T.sample_indices(n)
        assert len(j) == n
        assert np.array_equal(np.sort(j), np.arange(n))
    j = T.sample_indices(10 ** 6)
    assert len(j) == T.SAMPLE_MAX and len(np.unique(j)) == T.SAMPLE_MAX
    assert j.min() >= 0 and j.max() < 10 ** 6


def test_class_table():
    assert T.class_params(2, 0) == (8, oracle.PAD_ZERO)
    assert T.class_params(2, 4) == (16, oracle.PAD_GLOBAL_AVG)
    assert T.class_params(1, 11) == (256, oracle.PAD_BLOCK_AVG)
    assert T.class_params(3, 9) is None and T.class_params(3, 8) == (32, oracle.PAD_BLOCK_AVG)
    assert T.class_mask(3) == 0x1FF and T.class_mask(2) == 0xFFF
    assert T.default_class(1) == 9 and T.default_class(2) == 3 and T.default_class(3) == 0


def test_features_1d_ramp_closed_form():
    # x_i = i/4, i < 1000, absolute eb 1/2 (inv2eb = 1): every sample is used
    n, R = 1000, 64
    x = (np.arange(n) * 0.25).astype(np.float32)
    f = T.features(x, (n,), 0.5, oracle.EB_ABS, R)
    rng = 999 * 0.25
    assert f[0] == 1 and f[1] == 0 and f[2] == 0
    assert f[3] == pytest.approx(3.0)
    assert f[4] == pytest.approx(math.log10(rng / 0.5))
    assert f[5] == pytest.approx(math.log1p(0.25 / 0.5))
    assert f[6] == 0 and f[7] == 0
    assert f[8] == pytest.approx(0.5)                    # mean = rng / 2
    # population std of an n-point ramp of step s: s * sqrt((n^2 - 1) / 12)
    assert f[9] == pytest.approx(0.25 * math.sqrt((n * n - 1) / 12) / rng)
    # q = rint(i / 4) >= 64  <=>  i / 4 >= 63.5 (63.5 rounds to 64, even)  <=>  i >= 254
    assert f[10] == pytest.approx((n - 254) / n)
    assert f[11] == 6.0


@pytest.mark.parametrize("dims", [(40, 50), (12, 20, 30)])
def test_features_plane_gradients(dims):
    # x = a*ix + b*iy (+ c*iz): forward differences are a, b, c exactly
    coefs = (0.5, -2.0, 0.125)
    idx = np.indices(dims)
    x = np.zeros(dims)
    for ax in range(len(dims)):
        x = x + coefs[ax] * idx[len(dims) - 1 - ax]  # axis 0 of coefs is x (fastest)
    x = x.astype(np.float32)
    f = T.features(x, dims, 1e-2, oracle.EB_ABS, 512)
    assert f[len(dims) - 1] == 1
    for ax in range(3):
        want = math.log1p(abs(coefs[ax]) / 1e-2) if ax < len(dims) else 0.0
        assert f[5 + ax] == pytest.approx(want, rel=1e-12)


def test_features_constant_and_two_valued():
    n = 5000
    c = np.full(n, 3.0, np.float32)
    f = T.features(c, (n,), 1e-3, oracle.EB_REL, 512)   # range 0: eb_abs = eb
    assert f[4] == 0 and f[5] == 0 and f[8] == 0 and f[9] == 0
    assert f[10] == 1.0                                  # rint(3 / 2e-3) = 1500 >= 512
    f = T.features(c, (n,), 1.0, oracle.EB_ABS, 512)
    assert f[10] == 0.0                                  # rint(1.5) = 2 < 512
    # half a, half b: mean (a+b)/2, std |a-b|/2, range |a-b|
    a, b = 1.0, 5.0
    x = np.where(np.arange(n) % 2 == 0, a, b).astype(np.float32)
    f = T.features(x, (n,), 1e-2, oracle.EB_REL, 512)
    assert f[8] == pytest.approx(3.0 / 4.0)
    assert f[9] == pytest.approx(0.5)
    assert f[4] == pytest.approx(2.0)                    # log10(1 / 1e-2)
    assert f[5] == pytest.approx(math.log1p(4.0 / (1e-2 * 4.0)))


def test_features_skip_nonfinite():
    x = np.arange(100, dtype=np.float32)
    y = x.copy()
    y[[10, 50]] = np.nan
    y[70] = np.inf
    f = T.features(y, (100,), 1.0, oracle.EB_ABS, 8)
    v = np.delete(x, [10, 50, 70]).astype(np.float64)
    assert f[8] == pytest.approx(abs(v.mean()) / 99.0)
    # differences touching a non-finite value are dropped; the rest are 1
    assert f[5] == pytest.approx(math.log1p(1.0))


def test_entropy_closed_forms():
    assert T.code_entropy([0, 10, 0]) == 0.0
    for k in (2, 3, 8, 1000):
        assert T.code_entropy(np.ones(k)) == pytest.approx(math.log2(k))
    p = 0.1
    assert T.code_entropy([1, 9]) == pytest.approx(-(p * math.log2(p) + (1 - p) * math.log2(1 - p)))
    assert T.code_entropy([]) == 0.0


def test_costs_of_a_constant_field():
    # constant q = 1500 (x = 3, abs eb 1e-3): first-order Lorenzo leaves one
    # nonzero residual per block, q - P at its origin.  Zero padding: nb
    # outliers (|q| >= R), every other code is R.  Block average: P = q, no
    # outlier, one code value, entropy 0; only the nb padding scalars count.
    dims, R = (64, 96), 512
    x = np.full(dims, 3.0, np.float32)
    n = x.size
    for c in range(T.NCLASS):
        b, pad = T.class_params(2, c)
        nb = math.ceil(64 / b) * math.ceil(96 / b)
        cost, no, nf, H = T.class_cost(x, dims, 1e-3, oracle.EB_ABS, R, c)
        assert nf == 0
        if pad == oracle.PAD_BLOCK_AVG:
            assert no == 0 and H == 0.0 and cost == pytest.approx(4.0 * nb)
        elif pad == oracle.PAD_GLOBAL_AVG:
            assert no == 0 and H == 0.0 and cost == pytest.approx(4.0)
        else:
            p = nb / n
            Hw = -(p * math.log2(p) + (1 - p) * math.log2(1 - p))
            assert no == nb and H == pytest.approx(Hw)
            assert cost == pytest.approx(n * Hw / 8 + 8 * nb)
    costs = T.sweep_costs(x, dims, 1e-3, oracle.EB_ABS, R)
    assert T.label(costs) == 1          # global average at block 8: 4 bytes, lowest index of the tie
    assert T.label([3.0, 1.0, 1.0, 0.5, 0.5]) == 3


def test_label_prefers_the_cheaper_padding_within_the_tolerance():
    inf = float("inf")
    # class 1 (global average) is least by 0.2 %: within 0.5 % of it, zero
    # padding (class 0) wins, and block average (class 2) beats global
    assert T.label([100.0, 99.8, 99.9] + [inf] * 9) == 0
    assert T.label([inf, 99.8, 99.9] + [inf] * 9) == 2
    # a gain beyond the tolerance is taken: 1 % less than zero padding
    assert T.label([100.0, 99.0, 99.9] + [inf] * 9) == 1
    # among equal paddings the smaller size, then the lower index
    assert T.label([100.6, 100.0, 200.0, 100.2, 300.0, 300.0] + [inf] * 6) == 3
    assert T.label([100.0, 300.0, 300.0, 100.0] + [inf] * 8) == 0
    assert T.label([100.4, 100.0] + [inf] * 10) == 0  # 0.4 % above the least: equal
    assert T.label([100.6, 100.0] + [inf] * 10) == 1  # 0.6 % above: not


def _rand_problem(seed, B=9):
    rng = np.random.default_rng(seed)
    theta = rng.normal(0, 0.4, T.NPARAM)
    mu = rng.normal(0, 1, T.NFEAT)
    sigma = rng.uniform(0.5, 2.0, T.NFEAT)
    X = rng.normal(0, 1.5, (B, T.NFEAT))
    nds = rng.integers(1, 4, B)
    masks = np.array([T.class_mask(int(d)) for d in nds])
    y = np.array([rng.choice([c for c in range(T.NCLASS) if m >> c & 1]) for m in masks])
    return theta, mu, sigma, X, y, masks


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_gradient_matches_finite_differences(seed):
    theta, mu, sigma, X, y, masks = _rand_problem(seed)
    L, g = T.loss_grad(theta, mu, sigma, X, y, masks)
    assert L == pytest.approx(T.loss(theta, mu, sigma, X, y, masks))
    rng = np.random.default_rng(100 + seed)
    h = 1e-6
    for i in rng.choice(T.NPARAM, 300, replace=False):
        e = np.zeros(T.NPARAM)
        e[i] = h
        fd = (T.loss(theta + e, mu, sigma, X, y, masks) - T.loss(theta - e, mu, sigma, X, y, masks)) / (2 * h)
        assert g[i] == pytest.approx(fd, rel=1e-5, abs=1e-8)
    # classes masked out for every sample get no gradient on their bias
    m3 = np.full(len(y), T.class_mask(3))
    _, g3 = T.loss_grad(theta, mu, sigma, X, y % 9, m3)
    assert np.all(g3[-3:] == 0) and np.any(g3[-12:-3] != 0)


def test_forward_closed_form():
    # all weights zero: the logits are b3, softmax over the allowed classes
    theta = np.zeros(T.NPARAM)
    b3 = np.log(np.arange(1, T.NCLASS + 1, dtype=np.float64))
    theta[-T.NCLASS:] = b3
    masks = np.array([T.class_mask(3), T.class_mask(2)])
    X = np.zeros((2, T.NFEAT))
    _, p, _ = T.forward(theta, np.zeros(T.NFEAT), np.ones(T.NFEAT), X, masks)
    w3 = np.arange(1, 10) / np.arange(1, 10).sum()
    w2 = np.arange(1, 13) / np.arange(1, 13).sum()
    assert np.allclose(p[0, :9], w3) and np.all(p[0, 9:] == 0)
    assert np.allclose(p[1], w2)
    y = np.array([4, 11])
    assert T.loss(theta, np.zeros(12), np.ones(12), X, y, masks) == pytest.approx(
        -(math.log(w3[4]) + math.log(w2[11])) / 2)
    assert list(T.predict(theta, np.zeros(12), np.ones(12), X, masks)) == [8, 11]
    # ties go to the lowest index
    assert list(T.predict(np.zeros(T.NPARAM), np.zeros(12), np.ones(12), X, masks)) == [0, 0]


def test_adam_first_steps_closed_form():
    rng = np.random.default_rng(5)
    th = rng.normal(size=50)
    g = rng.normal(size=50)
    lr, eps = 1e-2, 1e-8
    t1, m, v = T.adam_step(th, g, np.zeros(50), np.zeros(50), 1, lr, eps=eps)
    # step 1: m_hat = g, v_hat = g^2
    assert np.allclose(t1, th - lr * g / (np.abs(g) + eps), rtol=0, atol=1e-15)
    # a constant gradient keeps m_hat = g and v_hat = g^2 at every step
    t2, _, _ = T.adam_step(t1, g, m, v, 2, lr, eps=eps)
    assert np.allclose(t2, t1 - lr * g / (np.abs(g) + eps), rtol=0, atol=1e-14)


# ---------------------------------------------------------------- hand-worked network
GOLDEN_FWD = os.path.join(os.path.dirname(__file__), "golden", "tuner_forward_handworked.json")
# documented flat layout: (offset, columns) of each parameter block
LAYOUT = {"W1": (0, 12), "b1": (768, None), "W2": (832, 64), "b2": (4928, None), "W3": (4992, 64),
          "b3": (5760, None)}


def _golden():
    with open(GOLDEN_FWD) as f:
        gd = json.load(f)
    theta = np.zeros(5772)
    for name, (off, ncol) in LAYOUT.items():
        for ent in gd[name]:
            if ncol is None:
                i, v = ent
                theta[off + i] = v
            else:
                r, c, v = ent
                theta[off + r * ncol + c] = v
    X = np.array([s["x"] for s in gd["samples"]], np.float64)
    masks = np.array([T.class_mask(s["ndim"]) for s in gd["samples"]])
    return gd, theta, np.array(gd["mu"], np.float64), np.array(gd["sigma"], np.float64), X, masks


def _expected_logits(s):
    return np.array([-np.inf if v is None else v for v in s["logits"]], np.float64)


def test_forward_handworked_network():
    """Non-zero weights in every layer, mu != 0 and sigma != 1, a negative
    pre-activation in each hidden layer, an asymmetric W2 and a class that
    only the mask removes (tests/golden/tuner_forward_handworked.json)."""
    gd, theta, mu, sigma, X, masks = _golden()
    assert T.NPARAM == 5772
    zm, p, (xt, a1, h1, a2, h2) = T.forward(theta, mu, sigma, X, masks)
    for i, s in enumerate(gd["samples"]):
        assert np.array_equal(xt[i], np.array(s["xt"], np.float64)), s["name"]
        assert np.array_equal(a1[i, :4], s["a1_head"]) and np.all(a1[i, 4:] == 0), s["name"]
        assert np.array_equal(h1[i, :4], s["h1_head"]) and np.all(h1[i, 4:] == 0), s["name"]
        assert np.array_equal(a2[i, :4], s["a2_head"]) and np.all(a2[i, 4:] == 0), s["name"]
        assert np.array_equal(h2[i, :4], s["h2_head"]) and np.all(h2[i, 4:] == 0), s["name"]
        z = _expected_logits(s)
        assert np.array_equal(zm[i], z), s["name"]
        # softmax of the hand-worked logits over the allowed classes
        e = [math.exp(v) if np.isfinite(v) else 0.0 for v in z]
        assert np.allclose(p[i], np.array(e) / sum(e), rtol=1e-14, atol=0), s["name"]
    assert list(T.predict(theta, mu, sigma, X, masks)) == [s["predicted"] for s in gd["samples"]]
    # the gradient of the mean cross-entropy with respect to b3 is the mean
    # of p - onehot(y) (softmax with cross-entropy, closed form)
    y = np.array([4, 3])
    _, g = T.loss_grad(theta, mu, sigma, X, y, masks)
    onehot = np.zeros((2, T.NCLASS))
    onehot[[0, 1], y] = 1.0
    assert np.allclose(g[-T.NCLASS:], (p - onehot).mean(0), rtol=1e-13, atol=1e-15)


def _forward_variant(theta, mu, sigma, X, masks, mistake):
    """The network of the golden case with one planted mistake, to show that
    the hand-worked case tells each of them apart."""
    P = T.unflatten(theta)
    xt = X * sigma + mu if mistake == "swapped_normalisation" else (X - mu) / sigma
    a1 = xt @ P["W1"].T + P["b1"]
    h1 = a1 if mistake == "no_relu1" else np.maximum(a1, 0.0)
    W2 = P["W2"] if mistake == "w2_transposed" else P["W2"].T
    a2 = h1 @ W2 + P["b2"]
    h2 = a2 if mistake == "no_relu2" else np.maximum(a2, 0.0)
    z = h2 @ P["W3"].T + P["b3"]
    allowed = ((masks[:, None] >> np.arange(T.NCLASS)) & 1).astype(bool)
    return np.where(allowed, z, -np.inf)


@pytest.mark.parametrize("mistake", ["swapped_normalisation", "no_relu1", "w2_transposed", "no_relu2"])
def test_handworked_network_catches_planted_mistakes(mistake):
    gd, theta, mu, sigma, X, masks = _golden()
    want = np.array([_expected_logits(s) for s in gd["samples"]])
    assert np.array_equal(_forward_variant(theta, mu, sigma, X, masks, None), want)
    assert not np.array_equal(_forward_variant(theta, mu, sigma, X, masks, mistake), want)


def test_adam_second_step_with_a_changed_gradient():
    """Two Adam steps with g1 = 2, g2 = -1, lr = 0.1, eps = 0, from theta = 0
    (Kingma & Ba, 2015, Algorithm 1), worked by hand:
      step 1: m = 0.2, v = 0.004, m_hat = 2, v_hat = 4, theta = -0.1 * 2 / 2 = -0.1;
      step 2: m = 0.9 * 0.2 + 0.1 * (-1) = 0.08, v = 0.999 * 0.004 + 0.001 * 1 = 0.004996,
              m_hat = 0.08 / 0.19 = 8/19, v_hat = 0.004996 / 0.001999 = 4996/1999,
              theta = -0.1 - 0.1 * (8/19) / sqrt(4996/1999).
    beta1 and beta2 enter differently under a changing gradient, so a swap
    of the two, or a bias correction with the wrong power, fails."""
    th1, m, v = T.adam_step(np.zeros(1), np.array([2.0]), np.zeros(1), np.zeros(1), 1, 0.1, eps=0.0)
    assert th1[0] == pytest.approx(-0.1, rel=1e-15)
    assert m[0] == pytest.approx(0.2, rel=1e-15) and v[0] == pytest.approx(0.004, rel=1e-14)
    th2, m, v = T.adam_step(th1, np.array([-1.0]), m, v, 2, 0.1, eps=0.0)
    assert m[0] == pytest.approx(0.08, rel=1e-14) and v[0] == pytest.approx(0.004996, rel=1e-14)
    assert th2[0] == pytest.approx(-0.1 - 0.1 * (8 / 19) / math.sqrt(4996 / 1999), rel=1e-14)
