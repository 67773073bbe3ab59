"""GPU parity of the learned tuner (called through the C ABI) against the
tuner oracle (oracle/tuner.py, float64 numpy):

* features: every one of the 12 within 1e-9 relative (fp64 sums in another
  order, and the device's log/log1p within a few ulps);
* sweep: per-class costs within 1e-10 relative (outlier and fixup counts and
  the code histogram are integers, so only the entropy's rounding differs),
  and the same label;
* guard: outlier counts of both classes equal to the compression oracle's on
  the same stacked sample, built here from the rule in include/vsz.h;
* network: logits, loss and gradient of fp32 kernels against float64 within
  1e-5 (relative, norm-wise for the gradient); Adam steps within 1e-5.
"""
import math

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle  # noqa: E402
from oracle import tuner as OT  # noqa: E402
import paper_2201_04614_gb300 as vsz  # noqa: E402
from paper_2201_04614_gb300 import tuner as T  # noqa: E402


def field(dims, seed):
    if len(dims) == 1:
        return synth.random_walk1d(dims[0], seed)
    if len(dims) == 2:
        return synth.fourier2d(dims[0], dims[1], seed=seed, value_range=20.0, offset=5.0)
    return np.exp(synth.grf3d(dims, seed))


FEAT_CASES = [((10007,), 1e-4, "rel", 512), ((300, 519), 1e-3, "rel", 64), ((19, 37, 260), 1e-4, "rel", 512),
              ((100000,), 1e-2, "abs", 8), ((40, 1000), 1e-5, "rel", 32768), ((64, 64, 64), 1e-3, "abs", 128),
              ((5,), 1e-3, "rel", 4)]


@pytest.mark.parametrize("dims,eb,mode,R", FEAT_CASES)
def test_features_match_oracle(dims, eb, mode, R):
    x = field(dims, seed=7).reshape(-1)
    p = vsz.Params.make(dims, 8, eb, mode, R, "zero")
    f64, f32 = T.features(p, torch.from_numpy(x).cuda())
    want = OT.features(x, dims, eb, oracle.EB_REL if mode == "rel" else oracle.EB_ABS, R)
    got = f64.cpu().numpy()
    assert np.allclose(got, want, rtol=1e-9, atol=1e-12), (got, want)
    assert np.array_equal(f32.cpu().numpy(), got.astype(np.float32))


def test_features_with_nonfinite_values():
    x = field((5000,), seed=3)
    x[::97] = np.nan
    x[5::131] = np.inf
    p = vsz.Params.make((5000,), 8, 1e-3, "rel", 512, "zero")
    got = T.features(p, torch.from_numpy(x).cuda())[0].cpu().numpy()
    want = OT.features(x, (5000,), 1e-3, oracle.EB_REL, 512)
    assert np.allclose(got, want, rtol=1e-9, atol=1e-12)


SWEEP_CASES = [((20011,), 1e-4, "rel", 512), ((130, 260), 1e-4, "rel", 512), ((17, 40, 70), 1e-3, "rel", 64),
               ((96, 96), 1e-2, "abs", 16), ((3000,), 1e-5, "rel", 32)]


@pytest.mark.parametrize("dims,eb,mode,R", SWEEP_CASES)
def test_sweep_costs_match_oracle(dims, eb, mode, R):
    x = field(dims, seed=11).reshape(-1)
    p = vsz.Params.make(dims, 8, eb, mode, R, "zero")
    got = T.sweep(p, torch.from_numpy(x).cuda()).cpu().numpy()
    want = OT.sweep_costs(x, dims, eb, oracle.EB_REL if mode == "rel" else oracle.EB_ABS, R)
    fin = np.isfinite(want)
    assert np.array_equal(np.isfinite(got), fin)
    assert np.allclose(got[fin], want[fin], rtol=1e-10, atol=0)
    assert T.label_of(got) == OT.label(want)


def stacked_sample(x, dims):
    """The guard's sample, from the rule documented with vsz_tuner_guard."""
    nd = len(dims)
    L = {1: 256, 2: 64, 3: 32}[nd]
    E0 = 65536 if nd == 1 else L
    n = int(np.prod(dims))
    if n <= 1 << 20 or dims[0] < 4 * E0:
        return x.reshape(dims)
    xf = x.reshape(dims)
    Ey = (dims[1] if dims[1] <= L else L) if nd == 3 else 1
    r = E0 if nd == 1 else E0 * dims[-1] if nd == 2 else E0 * Ey * dims[-1]
    m0 = dims[0] // E0
    my = (1 if dims[1] <= L else dims[1] // L) if nd == 3 else 1
    K = max(1, min(m0, n // (50 * r)))
    parts = []
    for i in range(K):
        z = (i * m0 // K) * E0
        if nd == 3:
            y = (i * my // K) * Ey
            parts.append(xf[z:z + E0, y:y + Ey, :])
        else:
            parts.append(xf[z:z + E0])
    return np.concatenate(parts, axis=0)


@pytest.mark.parametrize("dims,ca,cb", [((2 ** 21 + 300,), 9, 11), ((8_400_000,), 9, 2), ((2048, 1100), 3, 8),
                                        ((8192, 130), 3, 11), ((160, 130, 70), 0, 5), ((512, 256, 16), 0, 8),
                                        ((300, 400), 3, 5), ((300, 200, 30), 0, 2)])
def test_guard_counts_match_oracle(dims, ca, cb):
    x = field(dims, seed=5).reshape(-1)
    p = vsz.Params.make(dims, 8, 1e-4, "rel", 64, "zero")
    sub = stacked_sample(x, dims)
    assert T.guard_sample_dims(p) == sub.shape
    got, cost = T.guard_counts(p, torch.from_numpy(x).cuda(), ca, cb, with_cost=True)
    got, cost = got.cpu().numpy(), cost.cpu().numpy()
    for k, c in enumerate((ca, cb)):
        b, pad = OT.class_params(len(dims), c)
        r = oracle.compress(oracle.Params(sub.shape, b, 1e-4, oracle.EB_REL, 64, pad), sub)
        assert int(got[k]) == len(r.out_idx)
        # the estimated size on the sample, as the sweep's cost of the class
        want = OT.class_cost(sub.reshape(-1), sub.shape, 1e-4, oracle.EB_REL, 64, c)[0]
        assert np.isclose(cost[k], want, rtol=1e-10, atol=0)
    # without sizes the counts are the same
    plain = T.guard_counts(p, torch.from_numpy(x).cuda(), ca, cb).cpu().numpy()
    assert np.array_equal(plain, got)


def _problem(seed, B):
    rng = np.random.default_rng(seed)
    theta = (rng.normal(0, 0.3, T.NPARAM)).astype(np.float32)
    mu = rng.normal(0, 1, T.NFEAT).astype(np.float32)
    sigma = rng.uniform(0.5, 2.0, T.NFEAT).astype(np.float32)
    X = rng.normal(0, 1.5, (B, T.NFEAT)).astype(np.float32)
    nds = rng.integers(1, 4, B)
    masks = np.array([T.class_mask(int(d)) for d in nds], np.uint32)
    y = np.array([rng.choice([c for c in range(T.NCLASS) if m >> c & 1]) for m in masks], np.int32)
    return theta, mu, sigma, X, y, masks


def test_mlp_forward_matches_oracle():
    theta, mu, sigma, X, y, masks = _problem(0, 300)
    net = T.MLP(theta, mu, sigma)
    logits, cls = net.forward(X, masks)
    z, _, _ = OT.forward(theta, mu, sigma, X, masks)
    lg = logits.cpu().numpy()
    fin = np.isfinite(z)
    assert np.array_equal(np.isfinite(lg), fin)
    assert np.allclose(lg[fin], z[fin], rtol=1e-5, atol=1e-5)
    # the class agrees wherever the top two allowed logits are apart
    zs = np.sort(np.where(fin, z, -np.inf), axis=1)
    clear = (zs[:, -1] - zs[:, -2]) > 1e-3
    assert np.array_equal(cls.cpu().numpy()[clear], OT.predict(theta, mu, sigma, X, masks)[clear])


@pytest.mark.parametrize("B,use_idx", [(1, False), (37, False), (256, True), (1000, True)])
def test_mlp_gradient_matches_oracle(B, use_idx):
    theta, mu, sigma, X, y, masks = _problem(B, max(B, 1200))
    idx = np.random.default_rng(B).permutation(len(y))[:B].astype(np.int32) if use_idx else None
    net = T.MLP(theta, mu, sigma)
    loss, g = net.grad(X if use_idx else X[:B], y if use_idx else y[:B], masks if use_idx else masks[:B], idx)
    sel = idx if use_idx else np.arange(B)
    Lw, gw = OT.loss_grad(theta, mu, sigma, X[sel], y[sel], masks[sel])
    assert float(loss.item()) == pytest.approx(Lw, rel=1e-5)
    gg = g.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(gg - gw) <= 1e-5 * np.linalg.norm(gw)


def test_adam_matches_oracle():
    rng = np.random.default_rng(3)
    th = rng.normal(size=T.NPARAM).astype(np.float32)
    net = T.MLP(th)
    L = T._bind()
    m = torch.zeros(T.NPARAM, device="cuda")
    v = torch.zeros(T.NPARAM, device="cuda")
    tw, mw, vw = th.astype(np.float64), np.zeros(T.NPARAM), np.zeros(T.NPARAM)
    for step in range(1, 6):
        g = rng.normal(size=T.NPARAM).astype(np.float32)
        gd = torch.from_numpy(g).cuda()
        rc = L.vsz_mlp_adam(T._ptr(net.theta), T._ptr(gd), T._ptr(m), T._ptr(v), T.NPARAM, 1e-2, 0.9, 0.999, 1e-8,
                            step, T._stream_handle(None))
        assert rc == 0
        tw, mw, vw = OT.adam_step(tw, g, mw, vw, step, 1e-2)
        assert np.allclose(net.theta.cpu().numpy(), tw, rtol=1e-5, atol=1e-6)


def test_training_fits_a_separable_problem():
    # labels that are a fixed function of the features: training must drive
    # the loss down and classify the training set
    rng = np.random.default_rng(9)
    X = rng.normal(size=(2000, T.NFEAT)).astype(np.float32)
    y = (X[:, 0] > 0).astype(np.int32) * 3 + (X[:, 1] > 0).astype(np.int32)
    masks = np.full(2000, T.class_mask(2), np.uint32)
    net = T.MLP(seed=1)
    hist = net.train(X, y, masks, epochs=40, batch=128, lr=3e-3, seed=2)
    assert hist[-1] < 0.25 * hist[0]
    _, cls = net.forward(X, masks)
    assert (cls.cpu().numpy() == y).mean() > 0.95


def test_weights_round_trip(tmp_path):
    net = T.MLP(seed=4, mu=np.arange(12), sigma=np.arange(1, 13))
    path = str(tmp_path / "w.bin")
    net.save(path)
    back = T.MLP.load(path)
    assert torch.equal(back.theta, net.theta) and torch.equal(back.norm, net.norm)
