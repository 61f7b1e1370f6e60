"""The allocation-free SLRI entry point against the plan-based entry point (GPU).

srp_slri_apply_static is for callers that cannot allocate device memory while they
process frames: a real-time audio thread with a per-frame deadline (cudaMalloc can block
and synchronise the whole device), or a host whose device memory belongs to its own
pool.  Its scratch is a static device array shared by all calls.

Each case builds an SLRI plan of rank R, takes the plan's own factors from its saved
plan file and passes them, with the plan's GCC samples, to the static entry point through
the C-ABI, twice in a row: first on all frames, then on a tail of the frames scaled by
1e-2, so that argmax keys left over from the first call (larger values) would win if the
call did not clear them.  Both results must match srp_map on the plan within the parity
tolerance of the other GPU tests (1e-5 relative per frame), with the same argmax, and no
device memory may be allocated during the calls (the device's free memory is unchanged and
libsrp's allocation hook, set to fail every allocation, is never hit).  Ranks 8..64 cover
the kernel's register layouts (4, 2 and 1 cells per thread); two cases sit at the scratch
limits (F * R = 1048576 with R = 64, and F = 65536 frames with R = 16).
"""
import ctypes as C

import numpy as np
import pytest

import synth
from tests import _ref as R

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _p(t):
    return C.c_void_p(t.data_ptr())


@pytest.mark.parametrize("rank,F", [(8, 100), (24, 100), (40, 100), (64, 100), (64, 16384),
                                    (16, 65536)])
def test_static_scratch_slri_matches_plan_entry_point(rank, F, tmp_path):
    import torch

    import paper_2306_08514_gb300 as S
    assert torch.cuda.is_available()
    w = R.workload("square4") if F == 100 else synth.workload("square4", F=F)
    plan = S.Plan(w["mic_xyz"], w["grid_xyz"], w["fs"], w["N"], method="slri", rank=rank,
                  max_frames=F)
    frames = torch.from_numpy(w["frames"]).cuda()
    ref_maps, ref_am = plan.map(frames)
    xi = plan.gcc_samples(frames)
    torch.cuda.synchronize()
    plan.save(tmp_path / "slri.plan")
    tall, fat, _, _ = R.read_slri_plan(tmp_path / "slri.plan")
    assert tall.shape[1] == rank and fat.shape[0] == rank
    tall_d = torch.from_numpy(np.ascontiguousarray(tall)).cuda()
    fat_d = torch.from_numpy(np.ascontiguousarray(fat)).cuda()
    J, L = w["grid_xyz"].shape[0], xi.shape[1]
    assert fat.shape[1] == L
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    tail = slice(F // 3, F)
    calls = [(xi, slice(0, F), 1.0), ((1e-2 * xi[tail]).contiguous(), tail, 1e-2)]
    outs = [(torch.empty((x.shape[0], J), device="cuda"),
             torch.empty((x.shape[0],), dtype=torch.int32, device="cuda")) for x, _, _ in calls]
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    S.srp_debug_fail_allocations(0, 1 << 30)
    try:
        for (x, _, _), (maps, am) in zip(calls, outs):
            S.srp_slri_apply_static(_p(x), _p(fat_d), _p(tall_d), x.shape[0], L, rank, J,
                                    _p(maps), _p(am), stream)
        torch.cuda.synchronize()
    finally:
        S.srp_debug_fail_allocations(0, 0)
    assert torch.cuda.mem_get_info()[0] == free0
    for (x, sl, scale), (maps, am) in zip(calls, outs):
        zr = scale * ref_maps[sl].cpu().numpy().astype(np.float64)  # the map is linear in xi
        z = maps.cpu().numpy().astype(np.float64)
        rel = np.sqrt(((z - zr) ** 2).sum(1) / (zr ** 2).sum(1))
        assert rel.max() <= TOL, rel.max()
        a = am.cpu().numpy()
        assert np.array_equal(a, np.argmax(z, axis=1))
        err = np.abs(z - zr).max(axis=1)
        n = len(a)
        assert np.all(zr[np.arange(n), a] >= zr.max(axis=1) - 2 * err - 1e-9 * scale)


def test_static_scratch_refuses_requests_beyond_its_size():
    import torch

    import paper_2306_08514_gb300 as S
    x = torch.zeros((4, 154), device="cuda")
    fat = torch.zeros((64, 154), device="cuda")
    tall = torch.zeros((100, 64), device="cuda")
    maps = torch.zeros((4, 100), device="cuda")
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for F, rank in ((65537, 8), (16385, 64), (200000, 16)):
        with pytest.raises(S.SrpError) as e:
            S.srp_slri_apply_static(_p(x), _p(fat), _p(tall), F, 154, rank, 100, _p(maps), None,
                                    stream)
        assert e.value.status == S.SRP_EINVAL and "static scratch" in S.srp_last_error()
    torch.cuda.synchronize()
