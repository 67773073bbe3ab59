"""What the trained tuner gains over the method without it (the default block
size and zero padding), on held-out synthetic fields it was not trained on.

For each field the exhaustive GPU sweep gives the estimated compressed size
of every class (its per-class parity with the oracle is tested in
test_gpu_tuner.py).  The committed network must
* choose classes whose mean size is below the default class's;
* get within 1% of the best class's mean size (the sweep's own optimum);
* never end with more outliers than the default on the guard's sample, and
  fall back to the default exactly where the guard's rule says so.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2201_04614_gb300 as vsz  # noqa: E402
from paper_2201_04614_gb300 import tuner as T  # noqa: E402

HELD_OUT = range(20000, 20060)   # training used seeds 10000..14499
MAX_N = 1 << 21


def test_trained_tuner_beats_the_default_on_held_out_fields():
    net = T.MLP.load()
    ratios_pick, ratios_best, n = [], [], 0
    for seed in HELD_OUT:
        x, eb = synth.tuner_field(seed)
        if x.size > MAX_N:
            continue
        dims = x.shape
        p = vsz.Params.make(dims, 8, eb, "rel", 512, "zero")
        xd = torch.from_numpy(np.ascontiguousarray(x.reshape(-1))).cuda()
        costs = T.sweep(p, xd).cpu().numpy()
        pick = T.choose([(p, xd)], mlp=net)[0]
        d = T.default_class(len(dims))
        ratios_pick.append(costs[pick["class"]] / costs[d])
        ratios_best.append(costs[T.label_of(costs)] / costs[d])
        if pick["guard_nout"] is not None:
            got, dflt = pick["guard_nout"]
            # the guard's rule on its own sample: more outliers, or a dearer
            # padding whose size gain ties, give the default class
            assert pick["class"] == T.guard_pick(pick["predicted"], d, pick["guard_nout"], pick["guard_cost"])
            if pick["class"] != d:
                assert got <= dflt
        n += 1
    assert n >= 30
    mean_pick, mean_best = float(np.mean(ratios_pick)), float(np.mean(ratios_best))
    assert mean_pick < 1.0, mean_pick
    assert mean_pick <= mean_best + 0.01, (mean_pick, mean_best)


@pytest.mark.parametrize("dims,frac", [((1800, 3600), 0.05), ((100, 500, 500), 0.05), ((3_000_000,), 0.1),
                                       ((300, 200), 0.5)])
def test_sampling_autotuner(dims, frac):
    """The paper's sampling autotuner: a block size of the rank, the fastest
    of its own timings, on a sample of about the requested fraction (whole
    for small fields)."""
    import numpy as np
    import synth
    from paper_2201_04614_gb300 import tuner as T
    n = int(np.prod(dims))
    if len(dims) == 1:
        x = synth.random_walk1d(n, 3)
    elif len(dims) == 2:
        x = synth.fourier2d(*dims, seed=3, value_range=10.0, offset=2.0)
    else:
        x = np.exp(synth.grf3d(dims, 3))
    xd = torch.from_numpy(np.ascontiguousarray(x, np.float32).reshape(-1)).cuda()
    r = T.sampling_autotune(vsz.Params.make(dims, 8, 1e-4, "rel", 512, "zero"), xd, frac, iters=2)
    allowed = {1: (32, 64, 128, 256), 2: (8, 16, 32, 64), 3: (8, 16, 32)}[len(dims)]
    assert set(r["ms"]) == set(allowed) and all(v > 0 for v in r["ms"].values())
    assert r["block"] == min(r["ms"], key=r["ms"].get)
    if n <= (1 << 20):
        assert r["sample_elems"] == n
    else:
        assert 0 < r["sample_elems"] <= n and r["sample_elems"] < 3 * frac * n + 4 * 65536
