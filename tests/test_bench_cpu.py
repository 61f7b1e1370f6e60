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
    ("conv", "fp16x3", "flop", 4.0 * 60000 * 28 * 255 * 2000),
    ("slri", "bf16", "byte", 4.0 * 60000 * 2000),
    ("sspi", "bf16", "byte", 4.0 * 60000 * 2000),
    ("sspi", "fp32", "flop", 2.0 * 6720000 * 2000),
])
def test_contraction_work_per_launch(method, prec, kind, amount):
    """conv: 2JP(K-1) real MACs per frame (Eq. SRPomp) = 4JP(K-1) flop at every precision
    (the algorithm's work); SLRI/SSPI on the tensor cores: the 4-byte map write per cell."""
    k, w = bench.contraction_work(method, prec, _Info, 2000, 16)
    assert k == kind and math.isclose(w, amount, rel_tol=1e-15)


@pytest.mark.parametrize("prec,peak,bound", [
    ("bf16", 1895.8, "tensor"), ("fp16", 1895.8, "tensor"),
    ("fp16x3", 1895.8 / 3, "tensor"), ("bf16x3", 1895.8 / 3, "tensor"),
    ("tf32", 1895.8 * 1.1 / 2.25, "tensor"), ("tf32x3", 1895.8 * 1.1 / 2.25 / 3, "tensor"),
    ("fp32", 152 * 128 * 2 * 2070e6 / 1e12, "alu"),
])
def test_contraction_peak_matches_the_operand_type_and_split(prec, peak, bound):
    """The burst BF16 figure for kernels timed per step; TF32 at the nominal 1.1 / 2.25
    ratio; a hi+lo split runs three products per algorithmic MAC (peak / 3); FP32 FFMA
    from unit counts and the maximum SM clock."""
    pk = (6781.8, 1895.8, 1714.1, 2070.0, "measured")
    got, unit, b, _ = bench.contraction_peak(prec, "flop", pk)
    assert math.isclose(got, peak, rel_tol=1e-12) and unit == "TFLOP/s" and b == bound
    assert bench.contraction_peak(prec, "byte", pk)[:3] == (6781.8, "GB/s", "hbm")
    r = bench.roofline_of("conv", prec, _Info, 2000, 16, 6.26e-3, pk)
    assert math.isclose(r["achieved"], 4.0 * 60000 * 28 * 255 * 2000 / 6.26e-3 / 1e12, rel_tol=1e-12)
    assert math.isclose(r["frac"], r["achieved"] / peak, rel_tol=1e-12)


def test_argmax_report_counts_exact_neighbour_and_distant_picks():
    """A pick on the oracle's maximum, one on the next cell, one three cells away: exact
    1/3, within one cell 2/3; distances 0, h and 3h; the peak gap is 0 at the maximum.
    With a mirror-image twin of the maximum (an exact tie), a pick on the twin agrees up
    to ties and is at distance 0 from the nearest maximum."""
    g = synth.grid_box((0, 0, 0), (1.0, 1.0, 1.0), 0.1)
    J = g.shape[0]
    h = bench.grid_pitch(g)
    assert np.allclose(h, 0.1)
    ref = np.zeros((3, J))
    top = 555
    ref[:, top] = 1.0
    nb = int(np.argmin(np.linalg.norm(g - (g[top] + [0.1, 0, 0]), axis=1)))
    far = int(np.argmin(np.linalg.norm(g - (g[top] + [0, 0.3, 0]), axis=1)))
    rep = bench.argmax_report([top, nb, far], ref, g)
    assert rep["frames"] == 3 and math.isclose(rep["exact_index"], 1 / 3)
    assert math.isclose(rep["agree_up_to_ties"], 1 / 3)
    assert math.isclose(rep["within_one_cell"], 2 / 3)
    assert math.isclose(rep["dist_m_median"], 0.1, rel_tol=1e-9)
    assert math.isclose(rep["dist_m_max"], 0.3, rel_tol=1e-9)
    assert rep["peak_gap_median"] == 1.0 and rep["peak_gap_max"] == 1.0
    assert bench.argmax_report([top], ref[:1], g)["peak_gap_max"] == 0.0
    # an exact twin (rounding noise far below the tie tolerance) three cells away
    twin = ref[:1].copy()
    twin[0, far] = 1.0 - 1e-15
    rep = bench.argmax_report([far], twin, g)
    assert rep["exact_index"] == 0.0 and rep["agree_up_to_ties"] == 1.0
    assert rep["within_one_cell"] == 1.0 and rep["dist_m_max"] == 0.0
    # a plane grid: the axis with a single value does not count
    gp = synth.grid_plane((0.0, 0.0), (4.0, 4.0), (50, 50))
    assert np.isinf(bench.grid_pitch(gp)[2]) and np.allclose(bench.grid_pitch(gp)[:2], 0.08)


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


def test_committed_traffic_capture_matches_the_current_kernels():
    """The committed DRAM capture of the benchmark step applies to the kernels as they are
    (bench.py reports it as roofline.traffic only while their sources' sha256 match)."""
    t = bench.measured_traffic("uca8", 2000, "conv", "fp16x3")
    assert t is not None and 4.03e9 < t < 8.0e9


def test_clock_sampler_off_and_samples_from_the_mark(tmp_path):
    """--clock-ms 0 starts no sampler (stop() gives None); with samples, stop() keeps those
    written after mark(), the start of the timed region."""
    ck = bench.Clocks(0, interval_ms=0)
    ck.start()
    ck.mark()
    assert ck.stop() is None
    ck = bench.Clocks(0, interval_ms=20)
    ck.proc = None
    ck.n0 = 0
    line = "0, {sm}, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, {pc}\n"
    with open(ck.path, "w") as f:
        f.write(line.format(sm=300, pc="Not Active"))
    ck.n0 = ck._lines()  # the mark: one sample before the timed region
    with open(ck.path, "a") as f:
        f.write(line.format(sm=2070, pc="Active"))
        f.write(line.format(sm=2070, pc="Not Active"))

    class Done:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    ck.proc = Done()
    ck.f = open(ck.path, "a")
    r = ck.stop()
    assert r == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 2}


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
