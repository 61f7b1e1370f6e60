"""Host logic of bench.py (CPU only): the reference arm's JSON line and its bounded sample,
the algorithmic work each roofline is computed from, and the DRAM-traffic lookup that
goes stale when a kernel's source changes."""
import contextlib
import hashlib
import io
import json
import math

import numpy as np
import pytest

import bench
import synth


def test_reference_arm_prints_the_contract_line():
    a = bench.parse(["--impl", "reference", "--workload", "square4", "--frames", "4",
                     "--steps", "2", "--warmup", "1"])
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.run_reference(a)
    lines = [l for l in buf.getvalue().splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["dtype"] == "f64" and d["steps"] == 2
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["value"] > 0 and math.isclose(d["cpu_baseline"]["value"], d["value"])
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["config"]["workload"].startswith("square4: M=4, J=2500, N=512")
    # per step: one frame, every cell, three methods (3 * 2500 cells per step)
    assert math.isclose(d["value"], 3 * 2500 / (d["ms_per_step"] / 1e3), rel_tol=1e-9)


@pytest.mark.parametrize("steps,warmup,stride", [(2, 1, 1), (9, 3, 1), (10, 3, 2), (20, 5, 3),
                                                 (100, 20, 10)])
def test_reference_arm_sample_is_bounded(steps, warmup, stride):
    """Beyond REF_FULL_STEPS steps the arm takes one cell in `stride` per step, so the whole
    run stays near REF_FULL_STEPS frames of full work whatever K and W are."""
    got = bench.reference_stride(warmup, steps)
    assert got == stride
    assert (warmup + steps) / got <= bench.REF_FULL_STEPS


class _Info:
    J, P, K, L, nnz = 60000, 28, 256, 300, 6720000


@pytest.mark.parametrize("method,prec,kind,amount", [
    ("conv", "bf16", "flop", 4.0 * 60000 * 28 * 255 * 2000),
    ("conv", "fp16x3", "flop", 3 * 4.0 * 60000 * 28 * 255 * 2000),
    ("slri", "bf16", "byte", 4.0 * 60000 * 2000),
    ("sspi", "bf16", "byte", 4.0 * 60000 * 2000),
    ("sspi", "fp32", "flop", 2.0 * 6720000 * 2000),
])
def test_contraction_work_per_launch(method, prec, kind, amount):
    """conv: 2JP(K-1) real MACs per frame (Eq. SRPomp) = 4JP(K-1) flop, three products for
    the hi+lo precisions; SLRI/SSPI on the tensor cores: the 4-byte map write per cell."""
    k, w = bench.contraction_work(method, prec, _Info, 2000, 16)
    assert k == kind and math.isclose(w, amount, rel_tol=1e-15)


def test_measured_traffic_goes_stale_with_the_kernel_source(tmp_path, monkeypatch):
    (tmp_path / "profiles").mkdir()
    src = tmp_path / "k.cu"
    src.write_text("__global__ void k() {}\n")
    rec = {"sources_sha256": {"k.cu": hashlib.sha256(src.read_bytes()).hexdigest()},
           "launches": {"uca8:F2000:conv:bf16": {"source": "k.cu", "dram_read": 100,
                                                 "dram_write": 23}}}
    (tmp_path / "profiles" / "traffic_x.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_traffic("uca8", 2000, "conv", "bf16") == 123
    assert bench.measured_traffic("uca8", 2000, "slri", "bf16") is None
    src.write_text("__global__ void k() { }\n")
    assert bench.measured_traffic("uca8", 2000, "conv", "bf16") is None


def test_serving_mix_is_seeded_and_within_the_workload_ranges():
    """64 sessions, M in {4, 8, 16, 32}, N in {512, 1024}, hop 256, SLRI (R 16 / 32) or
    SSPI (t 2 / 4), grids inside the session's room; the same seed gives the same mix."""
    a = bench.serving_sessions(64)
    b = bench.serving_sessions(64)
    assert len(a) == 64
    for x, y in zip(a, b):
        assert x["kw"] == y["kw"] and x["N"] == y["N"] and x["M"] == y["M"]
        assert np.array_equal(x["grid"], y["grid"]) and np.array_equal(x["mics"], y["mics"])
    assert {s["M"] for s in a} == {4, 8, 16, 32}
    for s in a:
        assert s["N"] in (512, 1024) and s["hop"] == 256 and s["mics"].shape == (s["M"], 3)
        assert (s["kw"]["method"], s["kw"].get("rank", s["kw"].get("taps"))) in {
            ("slri", 16), ("slri", 32), ("sspi", 2.0), ("sspi", 4.0)}
        lo, hi = np.zeros(3), np.asarray(s["room"], float)
        assert np.all(s["grid"] >= lo - 1e-9) and np.all(s["grid"] <= hi + 1e-9)
        assert 1000 <= s["grid"].shape[0] <= 150000


def test_shards_draw_distinct_seeded_frames():
    s = {bench.shard_seed(1002, r) for r in range(8)}
    assert len(s) == 8 and bench.shard_seed(1002, 0) == 1002
    w1 = synth.workload("square4", F=2, seed=bench.shard_seed(1002, 1))
    w1b = synth.workload("square4", F=2, seed=bench.shard_seed(1002, 1))
    w2 = synth.workload("square4", F=2, seed=bench.shard_seed(1002, 2))
    assert (w1["frames"] == w1b["frames"]).all()
    assert not (w1["frames"] == w2["frames"]).all()
    assert w1["frames"].shape == w2["frames"].shape


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    """Under torchrun (N > 1) the reference arm's other ranks exit without work or output."""
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("LOCAL_RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    a = bench.parse(["--impl", "reference", "--gpus", "2", "--workload", "square4",
                     "--frames", "4", "--steps", "2", "--warmup", "1"])
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.run_reference(a)
    assert buf.getvalue() == ""
