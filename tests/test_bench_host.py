"""Host-side helpers of bench.py (no GPU): the gate on the stored DRAM
counters, the peak figures and their fallback, the CPU-oracle baseline's
bounded sample, replica throughput, and the parsing of the clock samples
that decides whether a run was throttled."""
import json
import os

import numpy as np
import pytest

import bench


def test_solve_traffic_applies_only_to_the_captured_source(monkeypatch):
    shapes = [(16384, 256), (8192, 8192), (2048, 131072)]
    n0s = [256, 512, 2048]
    monkeypatch.setattr(bench, "solve_source_sha256", lambda: bench.SOLVE_TRAFFIC_SHA256)
    mean, by_shape = bench.solve_traffic(shapes, n0s)
    stored = [bench.SOLVE_TRAFFIC[(n, k, n0)] for (n, k), n0 in zip(shapes, n0s)]
    assert mean == pytest.approx(sum(stored) / 3)
    assert by_shape["8192x8192"]["algorithmic_bytes"] == int(8 * (8192 * 8192 / 2 + 2 * 8192 * 8192))
    assert bench.solve_traffic([(16384, 256)], [128]) == (None, None)  # shape/n0 not captured
    monkeypatch.setattr(bench, "solve_source_sha256", lambda: "0" * 64)
    assert bench.solve_traffic(shapes, n0s) == (None, None)  # kernel changed since the capture


def test_measured_peaks_and_fallback(tmp_path, monkeypatch):
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"bf16_tflops": 1925.7, "bf16_tflops_sustained": 1712.9}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    burst, sustained, src = bench.measured_peaks()
    assert (burst, sustained) == (1925.7, 1712.9) and src.startswith("measured")
    os.remove(tmp_path / "MEASURED_PEAKS.json")
    burst, sustained, src = bench.measured_peaks()
    assert (burst, sustained) == (1900.0, 1700.0) and src.startswith("fallback")


def test_cpu_oracle_rate_takes_a_bounded_sample():
    shapes = [(64, 40), (96, 7)]
    data = bench.make_inputs(shapes, seed=3)
    rate, sample, cores = bench.cpu_oracle_rate(data, shapes, budget_s=0.05)
    assert rate > 0 and cores >= 1
    parts = sample.split("; ")
    assert parts[0].startswith("64:") and parts[1].startswith("96:")
    for part, (n, k) in zip(parts, shapes):
        used = int(part.split(":")[1].split("/")[0])
        assert 1 <= used <= k and part.endswith(f"/{k}")


def test_replica_throughput_counts_every_rank():
    assert bench.replica_throughput(1e12, 4, 1000.0) == pytest.approx(4e12)
    assert bench.replica_throughput(2e9, 1, 2.0) == pytest.approx(1e12)


class _Done:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def test_clock_sampler_reads_throttle_reasons(tmp_path):
    s = bench.ClockSampler(0)
    s.proc, s.fh = _Done(), open(os.devnull, "w")
    rows = ["0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
            "0, 1965, 2070, 1380.0, 0x4, Not Active, Not Active, Not Active, Active",
            "0, 2070, 2070, 950.0, 0x0, Not Active, Not Active, Not Active, Not Active",
            "garbage line"]
    with open(s.path, "w") as fh:
        fh.write("\n".join(rows) + "\n")
    out = s.stop()
    assert out["samples"] == 3 and out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]
    assert not os.path.exists(s.path)


def test_compact_precision_records():
    """The bench line's precision block: FP64 figures per c, one row per
    (c, inner format, diagonal multiply, residual), and a status that tells a met target, a missed one
    and a non-finite result apart."""
    recs = [{"c": 2, "n0": 1024, "fp64_solve_ms": 880.0, "fp64_fwd_err": 5.2e-16,
             "mixed": [{"inner": "fp16x3", "s_step": "fp32", "residual": "adaptive", "ms": 70.1, "iterations": 3,
                        "fwd_err": 7.0e-13, "bwd_err": 5.4e-15, "speedup_vs_fp64": 12.6, "converged": True},
                       {"inner": "tf32", "s_step": "tc", "residual": "adaptive", "n0": 256, "ms": 95.0, "iterations": 5,
                        "fwd_err": 3.4e-9, "bwd_err": 1e-15, "speedup_vs_fp64": 9.3, "converged": False}]},
            {"c": 6, "n0": 1024, "fp64_solve_ms": 881.0, "fp64_fwd_err": None,
             "mixed": [{"inner": "fp16x3", "s_step": "fp32", "residual": "sliced8", "ms": 5.0, "iterations": 1,
                        "fwd_err": None, "bwd_err": None, "speedup_vs_fp64": 176.2, "converged": False}]}]
    out = bench.compact_precision(recs)
    assert out["fp64"] == {"2": [880.0, 5.2e-16], "6": [881.0, None]}
    assert [r[-1] for r in out["rows"]] == ["ok", "miss", "nan"]
    assert out["rows"][2][-2] is None  # no speed-up is quoted for a non-finite result
    assert out["rows"][0][:7] == [2, "fp16x3", "fp32", "adaptive", 1024, 70.1, 3]
    assert out["rows"][1][4] == 256  # a combo on its own plan
    assert out["rows"][2][3] == "sliced8" and len(out["cols"]) == len(out["rows"][0])


def test_sliced_mma_flops_closed_form():
    """The sliced solve multiplies 36 digit-plane pairs over the update
    blocks (the strictly lower block triangle of L) and the strictly lower
    parts of the diagonal blocks: together n^2 k per pair when nb divides n
    (n^2 - N nb^2 of updates plus N nb^2 of diagonal multiplies)."""
    for n, k, nb in ((8192, 8192, 2048), (16384, 256, 1024), (2048, 3, 2048), (512, 5, 64)):
        assert bench.sliced_mma_flops(n, k, nb) == pytest.approx(36.0 * n * n * k)
    # a ragged last block of m rows: the update rows shrink accordingly
    n, k, nb = 1000, 7, 256
    m = n - 3 * nb
    upd = sum(2.0 * (n - (i + 1) * nb) * nb * k for i in range(3))
    assert bench.sliced_mma_flops(n, k, nb) == pytest.approx(36.0 * (upd + (3 * nb * nb + m * m) * k))
