"""Checkpoint / resume of a plan's offline fit (srp_plan_save, srp_plan_create_from_file):
a plan created from the file gives bit-identical maps without recomputing the fit, also at
another precision, and a file made for other inputs is refused."""
import numpy as np
import pytest

from tests import _ref as R
from tests.test_gpu_parity import S, _cuda, _run  # noqa: F401

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kw", [dict(method="slri", rank=8), dict(method="sspi", taps=2.0),
                                dict(method="lr", rank=6), dict(method="conv")],
                         ids=["slri", "sspi", "lr", "conv"])
@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_saved_plan_gives_identical_maps(S, tmp_path, kw, prec):
    w = R.workload("square4")
    args = (w["mic_xyz"], w["grid_xyz"], w["fs"], w["N"])
    fr = np.ascontiguousarray(w["frames"][:40])
    a = S.Plan(*args, precision=prec, max_frames=64, **kw)
    za, aa = _run(a, fr)
    path = tmp_path / f"{kw['method']}.plan"
    a.save(path)
    b = S.Plan(*args, precision=prec, max_frames=16, plan_file=path, **kw)  # another batch size
    zb, ab = _run(b, fr)
    assert np.array_equal(za, zb) and np.array_equal(aa, ab)
    if kw["method"] in ("slri", "lr"):
        assert np.array_equal(a.slri_sigma(kw["rank"] + 1), b.slri_sigma(kw["rank"] + 1))
    if kw["method"] == "sspi":
        for x, y in zip(a.sspi_taps(), b.sspi_taps()):
            assert np.array_equal(x, y)


def test_saved_fit_serves_another_precision(S, tmp_path):
    w = R.workload("square4")
    args = (w["mic_xyz"], w["grid_xyz"], w["fs"], w["N"])
    fr = np.ascontiguousarray(w["frames"][:40])
    S.Plan(*args, method="slri", rank=8, precision="fp32", max_frames=64).save(tmp_path / "s.plan")
    fresh = _run(S.Plan(*args, method="slri", rank=8, precision="fp16x3", max_frames=64), fr)
    loaded = _run(S.Plan(*args, method="slri", rank=8, precision="fp16x3", max_frames=64,
                         plan_file=tmp_path / "s.plan"), fr)
    assert np.array_equal(fresh[0], loaded[0]) and np.array_equal(fresh[1], loaded[1])


def test_plan_file_for_other_inputs_is_refused(S, tmp_path):
    w = R.workload("square4")
    args = (w["mic_xyz"], w["grid_xyz"], w["fs"], w["N"])
    S.Plan(*args, method="slri", rank=8, max_frames=8).save(tmp_path / "r8.plan")
    for kw in (dict(method="slri", rank=9), dict(method="sspi", taps=2.0)):
        with pytest.raises(S.SrpError) as e:
            S.Plan(*args, max_frames=8, plan_file=tmp_path / "r8.plan", **kw)
        assert e.value.status == S.SRP_EINVAL
    moved = w["mic_xyz"].copy()
    moved[0, 0] += 1e-3
    with pytest.raises(S.SrpError) as e:
        S.Plan(moved, *args[1:], method="slri", rank=8, max_frames=8, plan_file=tmp_path / "r8.plan")
    assert e.value.status == S.SRP_EINVAL
