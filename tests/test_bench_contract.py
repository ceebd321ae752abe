"""The bench's reference arm prints the JSON line the contract asks for (the
oracle's timing replaced by a fast stand-in here; the real leg times the
oracle on the host cores), with the same workload config as the GPU arm, and
only rank 0 prints under a multi-rank launch."""
import json
import types

import pytest

import bench


def _fake_sample(w, seconds):
    return {"value": 1.0e7, "unit": bench.UNIT, "cores": 4, "kind": "oracle", "sample": "stand-in",
            "seconds": 0.5, "cells": 5.0e6}


def _args(**kw):
    a = dict(gpus=1, steps=2, warmup=3, impl="reference", workload="rw4096", precision="fp32", band_form=0,
             no_fp64_path=True, no_motif_path=True, no_discord_path=True, no_cpu_baseline=True, cpu_seconds=1.0,
             p_sweep=None, ncu_case=None, mode=0, lrange=None, fp64_steps=3, e2e_steps=3, fp64_lrange=None, graphs=1, tc_tma=0)
    a.update(kw)
    return types.SimpleNamespace(**a)


def test_reference_line(monkeypatch, capsys):
    monkeypatch.setattr(bench, "cpu_oracle_sample", _fake_sample)
    monkeypatch.delenv("RANK", raising=False)
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    assert bench.run_reference(_args()) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["higher_is_better"] is True and line["steps"] == 2 and line["warmup"] == 3
    assert line["value"] == pytest.approx(1.0e7)
    assert line["ms_per_step"] == pytest.approx(500.0)
    assert set(line["cpu_baseline"]) == {"value", "unit", "cores", "kind", "sample"}
    assert line["e2e"] == {"value": line["value"], "unit": bench.UNIT, "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    import workloads
    assert line["config"] == bench.workload_config("rw4096", workloads.make("rw4096"))


def test_reference_line_batch_and_range(monkeypatch, capsys):
    # the batch workload's config describes its series; a stated sub-range
    # of lengths shows up in both arms' config
    monkeypatch.setattr(bench, "cpu_oracle_sample", _fake_sample)
    monkeypatch.delenv("RANK", raising=False)
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    assert bench.run_reference(_args(workload="batch256")) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["config"]["series"] == 256 and line["config"]["lengths_total"] > 256
    assert bench.run_reference(_args(workload="seismic2m")) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert (line["config"]["lmin"], line["config"]["lmax"]) == bench.DEFAULT_RANGE["seismic2m"]
    assert line["config"]["cells_per_step"] == 2097152 ** 2 * 9


def test_reference_other_ranks_print_nothing(monkeypatch, capsys):
    monkeypatch.setattr(bench, "cpu_oracle_sample", _fake_sample)
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    assert bench.run_reference(_args(gpus=2)) == 0
    assert capsys.readouterr().out.strip() == ""


def test_band_traffic_record_matches_the_band_kernel_source():
    # the DRAM bytes per cell that the bench line reports as the band
    # kernel's traffic were counted on this kernel source (else it reports
    # null); a change to the band kernel's files makes this fail until the
    # record is taken again
    import json
    import os
    import bench
    rec = json.load(open(os.path.join(bench.ROOT, "profiles", "band_kernel_traffic.json")))
    assert rec["kernel_source_sha"] == bench.kernel_source_hash()
    t = bench.measured_traffic(rec["cells_per_launch"])
    assert t is not None
    assert abs(t - (rec["dram_bytes_read"] + rec["dram_bytes_write"])) <= 1e-6 * t
