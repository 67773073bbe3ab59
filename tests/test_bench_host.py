"""Host logic of bench.py, without a GPU: algorithmic bytes of each kernel
and of the mixed stream's compression, the batch kernels' names, the
profiled-traffic table and its source digests (and its per-value scaling),
the clock summary, the fallback peak, the stream's CPU samples and the
host-parallel oracle timing."""
import json
import os
import types

import numpy as np
import pytest

import bench


def test_algorithmic_bytes_per_kernel():
    n, nb, no, nf = 1000, 10, 7, 3
    assert bench.algorithmic_bytes("range", n, nb, no, nf, False) == 4 * n
    # x in; codes, staged outliers and fixups, block offsets out (+ the pad table)
    assert bench.algorithmic_bytes("lorenzo", n, nb, no, nf, False) == 4 * n + 2 * n + 8 * (no + nf) + 4 * nb
    assert bench.algorithmic_bytes("lorenzo", n, nb, no, nf, True) == 4 * n + 2 * n + 8 * (no + nf) + 8 * nb
    # codes, outliers, block offsets (+ pads) in, values out
    assert bench.algorithmic_bytes("recon", n, nb, no, nf, False) == 2 * n + 8 * no + 4 * (nb + 1) + 4 * n
    assert bench.algorithmic_bytes("compact_move", n, nb, no, nf, False) == 16 * (no + nf) + 8 * nb
    assert bench.algorithmic_bytes("fixups", n, nb, no, nf, False) == 12 * nf
    assert bench.algorithmic_bytes("begin", n, nb, no, nf, False) == 0


def test_step_bytes_are_sixteen_per_value():
    # range 4 + compression 6 + reconstruction 6 bytes per value when the
    # lists are empty: the step roofline that step_hbm_frac divides by
    n, nb = 512 ** 3, 64 ** 3
    total = sum(bench.algorithmic_bytes(k, n, nb, 0, 0, False) for k in ("range", "lorenzo", "recon"))
    assert total == 16 * n + 4 * nb + 4 * (nb + 1)


def test_job_gbps_and_rank_seeds():
    assert bench.job_gbps(1, 250_000_000, 1000.0) == pytest.approx(1.0)
    assert bench.job_gbps(4, 250_000_000, 1000.0) == pytest.approx(4.0)  # weak scaling: all ranks' values
    seeds = {bench.rank_field_seed(r) for r in range(8)}
    assert len(seeds) == 8 and bench.rank_field_seed(0) == 2  # rank 0 compresses the headline field


def test_profiled_traffic_follows_the_source_digest():
    with open(os.path.join(bench.ROOT, "profiles", "traffic.json")) as f:
        tab = json.load(f)
    for key, ent in tab.items():
        kernel, workload = key.split("|")
        if "dram_bytes_per_value" in ent:  # a smaller case, scaled by the values of a full launch
            want = round(ent["dram_bytes_per_value"] * 1000) if ent["src_digest"] == bench.kernel_sources_digest(kernel) \
                else None
            assert bench.profiled_traffic(kernel, workload, units=1000) == want, key
            continue
        want = ent["dram_bytes_per_launch"] if ent["src_digest"] == bench.kernel_sources_digest(kernel) else None
        assert bench.profiled_traffic(kernel, workload) == want, key
        assert ent["sources"] == list(bench.KERNEL_SOURCES[kernel.split("<")[0]])
    assert bench.profiled_traffic("k_lorenzo_nd<3,8,false,false>", "no such workload") is None


def test_digest_depends_only_on_the_listed_sources():
    d1 = bench.kernel_sources_digest("k_lorenzo_nd<3,8,false,false>")
    assert d1 == bench.kernel_sources_digest("k_recon_nd<3,8,false>")  # same source list
    assert d1 != bench.kernel_sources_digest("k_range")
    assert len(d1) == 16 and int(d1, 16) >= 0


def test_clock_summary_and_reasons():
    cs = bench.ClockSampler.__new__(bench.ClockSampler)
    cs.proc = None
    cs.samples = [(10.0, ["0", "2070", "2070", "900", "0x0", "Not Active", "Not Active", "Not Active", "Not Active"]),
                  (11.0, ["0", "2040", "2070", "1400", "0x4", "Not Active", "Not Active", "Not Active", "Active"]),
                  (12.0, ["0", "2070", "2070", "950", "0x0", "Not Active", "Not Active", "Not Active", "Not Active"]),
                  (50.0, ["0", "900", "2070", "100", "0x0", "Active", "Not Active", "Not Active", "Not Active"])]
    s = cs.summary(9.0, 13.0)  # the last sample lies outside the timed window
    assert s == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    cs.samples = []
    assert cs.summary(0.0, 1.0) is None


def test_fallback_peak_without_measurements(monkeypatch, tmp_path):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_peaks() == (6800.0, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6786.9}))
    assert bench.measured_peaks() == (6786.9, "measured")


def test_host_parallel_oracle_timing():
    import synth
    x3 = np.ascontiguousarray(synth.cfg2_field(32), np.float32)
    a = types.SimpleNamespace(pad="zero", block=8, field_eb=1e-4)
    v, threads, slabs, desc = bench.oracle_rate_parallel(x3, a, 0.2, threads=2)
    assert v > 0 and threads == 2 and slabs >= 2 and "2 threads" in desc
    assert bench.cpu_model()


class _P:
    def __init__(self, dims, block, pad):
        self.dims, self.block, self.pad = dims, block, pad

    @property
    def is_block_pad(self):
        return self.pad in (4, 5, 6)

    @property
    def is_edge_pad(self):
        return self.pad in (7, 8, 9)


class _F:
    def __init__(self, dims, block, pad):
        self.p = _P(dims, block, pad)
        self.n = int(np.prod(dims))
        self.nb = int(np.prod([-(-d // block) for d in dims]))


def test_stream_sequence_bytes_and_class_names():
    fields = [_F((1000,), 256, 0), _F((64, 64), 16, 6), _F((16, 16, 16), 8, 3), _F((32, 32), 16, 0)]
    heads = [{"n_out": 5, "n_fix": 1}, {"n_out": 0, "n_fix": 0}, {"n_out": 9, "n_fix": 0}, {"n_out": 2, "n_fix": 2}]
    sb = bench.sequence_bytes(fields, heads)
    keys = [bench.class_key(f.p) for f in fields]
    assert keys == [("batch_lorenzo", 1, 256), ("batch_lorenzo_bp", 2, 16), ("batch_lorenzo_gp", 3, 8),
                    ("batch_lorenzo", 2, 16)]
    # per class: 6 bytes per value + 8 per list entry + 4 per block (+ 4 per block for a block padding table)
    assert sb["per_kernel"][keys[0]] == 6 * 1000 + 8 * 6 + 4 * 4
    assert sb["per_kernel"][keys[1]] == 6 * 4096 + 8 * 16
    assert sb["per_kernel"][keys[2]] == 6 * 4096 + 8 * 9 + 4 * 8
    assert sb["per_kernel"][keys[3]] == 6 * 1024 + 8 * 4 + 4 * 4
    assert sb["per_kernel"][("batch_range", 0, 0)] == 4 * (1000 + 4096 + 4096 + 1024)
    assert sb["total"] == sum(v for k, v in sb["per_kernel"].items())
    assert bench.batch_kernel_name(keys[0]) == "k_lorenzo_1d_batch<256,false,false>"
    assert bench.batch_kernel_name(keys[1]) == "k_lorenzo_nd_batch<2,16,true,false>"
    assert bench.batch_kernel_name(keys[2]) == "k_lorenzo_nd_batch<3,8,false,true>"


def test_profiled_traffic_scales_per_value_entries(tmp_path):
    k = "k_lorenzo_nd_batch<3,8,false,false>"
    tab = {f"{k}|small": {"src_digest": bench.kernel_sources_digest(k), "dram_bytes_per_value": 6.25}}
    path = tmp_path / "traffic.json"
    path.write_text(json.dumps(tab))
    assert bench.profiled_traffic(k, "small", units=1000, path=str(path)) == 6250
    assert bench.profiled_traffic(k, "small", path=str(path)) is None  # no units, no figure
    tab[f"{k}|small"]["src_digest"] = "0" * 16
    path.write_text(json.dumps(tab))
    assert bench.profiled_traffic(k, "small", units=1000, path=str(path)) is None  # sources changed


def test_stream_slabs_are_block_aligned_and_bounded():
    x1 = np.arange(3_000_000, dtype=np.float32)
    for k in range(4):
        sl = bench.stream_slab((x1.size,), x1, k, 256)
        assert sl.size == 1 << 20 and int(sl[0]) % 256 == 0
    x2 = np.arange(200 * 96, dtype=np.float32)
    for k in range(5):
        sl = bench.stream_slab((200, 96), x2, k, 16)
        assert sl.shape == (64, 96) and (int(sl[0, 0]) // 96) % 16 == 0
    x3 = np.arange(100 * 6 * 5, dtype=np.float32)
    for k in range(5):
        sl = bench.stream_slab((100, 6, 5), x3, k, 8)
        assert sl.shape == (32, 6, 5) and (int(sl[0, 0, 0]) // 30) % 8 == 0


def test_oracle_stream_rate_on_a_small_stream():
    import synth
    specs = [("w", (300_000,), synth.random_walk1d(300_000, 1), 1e-3),
             ("c", (128, 96), synth.fourier2d(128, 96, seed=2), 1e-3),
             ("h", (40, 16, 24), synth.grf3d((40, 16, 24), 3), 1e-3)]
    v, elems, k, desc = bench.oracle_stream_rate(specs, 1e-3, 0.05)
    assert v > 0 and k >= 1 and elems > 0 and "oracle" in desc
    v, threads, slabs, desc = bench.oracle_stream_rate_parallel(specs, 1e-3, 0.05, threads=2)
    assert v > 0 and threads == 2 and slabs >= 2
