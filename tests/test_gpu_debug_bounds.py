"""The bounds-checking build (-DVSZ_DEBUG_BOUNDS) on the small parity shapes.

A memory checker is not available on every machine, so the library can be
built with its own checks: every write to a field-sized buffer (codes,
values, outlier and fixup lists, block slots, padding and offset tables)
and every read of the block slots and outlier caches checks its index
against the buffer's length, skips an access out of bounds and records its
site.  This test builds that variant, runs ragged 1D/2D/3D shapes in every
padding kind, dense and sparse outliers, the one-field calls and a batch,
in a separate process, and requires results identical to the oracle's and
no recorded site.
"""
import os
import subprocess
import sys
import textwrap

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = textwrap.dedent('''
    import sys
    import numpy as np
    import torch
    sys.path.insert(0, ROOT)
    import oracle, synth
    import paper_2201_04614_gb300 as vsz

    assert vsz.debug_bounds_word() == 0  # the checking build is loaded
    shapes = [((77,), 8), ((5000,), 256), ((129, 257), 16), ((100, 83), 8), ((33, 70), 64),
              ((17, 23, 29), 8), ((9, 40, 132), 4), ((20, 12, 260), 16)]
    pads = ["zero", "block_avg", "global_avg", "edge_avg", "block_min", "global_max"]
    n_cases = 0
    for dims, b in shapes:
        if len(dims) == 1:
            x = synth.random_walk1d(dims[0], 5)
        elif len(dims) == 2:
            x = synth.fourier2d(dims[0], dims[1], seed=6, value_range=40.0, offset=2.0)
        else:
            x = np.exp(synth.grf3d(dims, 7)).astype(np.float32)
        x = np.ascontiguousarray(x, np.float32)
        x.reshape(-1)[3] = np.nan
        for pad in pads:
            for eb, R in ((1e-3, 512), (1e-5, 8)):
                p = vsz.Params.make(dims, b, eb, "rel", R, pad)
                n = x.size
                f = vsz.Field(p, out_cap=n, fix_cap=n)
                f.compress(torch.from_numpy(x.reshape(-1)).cuda())
                got = f.to_host()
                po = oracle.Params(dims, b, eb, oracle.EB_REL, R, oracle.PAD_NAMES[pad])
                c = oracle.compress(po, x)
                for k in ("codes", "blk_off", "out_idx", "out_delta", "fix_idx", "fix_bits"):
                    assert np.array_equal(got[k], getattr(c, k)), (dims, b, pad, eb, k)
                xo = oracle.decompress(po, c).view(np.uint32)
                assert np.array_equal(f.reconstruct()[:n].cpu().numpy().view(np.uint32), xo), (dims, pad, eb)
                n_cases += 1
    # a batch of mixed fields (block slots, stashes, every class kernel)
    fields, xs = [], []
    for i, (dims, b) in enumerate(shapes):
        x = np.ascontiguousarray(np.exp(synth.grf3d(dims, 20 + i)), np.float32).reshape(-1)
        p = vsz.Params.make(dims, b, 1e-5, "rel", 16, pads[i % len(pads)])
        fields.append(vsz.Field(p, out_cap=x.size, fix_cap=x.size))
        xs.append(torch.from_numpy(x).cuda())
    bt = vsz.Batch(fields, xs, use_graph=False)
    outs = [torch.empty(x.numel(), dtype=torch.float32, device="cuda") for x in xs]
    bt.set_outputs(outs)
    bt.submit()
    bt.reconstruct()
    torch.cuda.synchronize()
    for f, x, o in zip(fields, xs, outs):
        h = f.header()
        assert h["status"] == 0 and h["recon_status"] == 0
        err = (o.double() - x.double()).abs().max().item()
        assert err <= h["eb_abs"] * (1 + 2.0 ** -20)
    word = vsz.debug_bounds_word()
    assert word == 0, word
    print("checked", n_cases, "cases and a batch of", len(fields), "fields")
''')


def test_bounds_checking_build_on_parity_shapes(tmp_path):
    from paper_2201_04614_gb300 import buildlib
    lib = buildlib.build(defines=("VSZ_DEBUG_BOUNDS",), out=str(tmp_path / "libvsz_debug.so"),
                         build_dir=str(tmp_path / "build"))
    env = dict(os.environ, VSZ_LIBRARY=lib)
    r = subprocess.run([sys.executable, "-c", f"ROOT = {ROOT!r}\n" + SCRIPT], env=env, capture_output=True,
                       text=True, timeout=1200)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "checked" in r.stdout
