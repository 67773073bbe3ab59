"""Host logic of bench.py, without a GPU: algorithmic bytes of each kernel,
the profiled-traffic table and its source digests, the clock summary, the
fallback peak and the host-parallel oracle timing."""
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
        want = ent["dram_bytes_per_launch"] if ent["src_digest"] == bench.kernel_sources_digest(kernel) else None
        assert bench.profiled_traffic(kernel, workload) == want, key
        assert ent["sources"] == list(bench.KERNEL_SOURCES[kernel.split("<")[0]])
    assert bench.profiled_traffic("k_lorenzo_nd<3,8,false,false>", "no such workload") is None
    # the dominant kernel of the bench line has a current capture
    assert bench.profiled_traffic("k_lorenzo_nd<3,8,false,false>", "512^3 b8 eb0.0001 zero") is not None


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
    a = types.SimpleNamespace(pad="zero", block=8, eb=1e-4, radius=512)
    v, threads, slabs, desc = bench.oracle_rate_parallel(x3, a, 0.2, threads=2)
    assert v > 0 and threads == 2 and slabs >= 2 and "2 threads" in desc
    assert bench.cpu_model()
