"""The allocation-free SLRI entry point against the plan-based entry point (GPU).

srp_slri_apply_static is for callers that cannot allocate device memory while they
process frames: a real-time audio thread with a per-frame deadline (cudaMalloc can block
and synchronise the whole device), or a host whose device memory belongs to its own
pool.  Its scratch is a static device array shared by all calls.  This test calls it
through the C-ABI twice in a row (the second call smaller, so stale scratch from the
first would show) and checks each result against srp_map on an SLRI plan of the same
rank, within the parity tolerance of the other GPU tests (1e-5 relative per frame).
"""
import ctypes as C

import numpy as np
import pytest

from tests import _ref as R

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _p(t):
    return C.c_void_p(t.data_ptr())


def test_static_scratch_slri_matches_plan_entry_point():
    import torch

    import paper_2306_08514_gb300 as S
    assert torch.cuda.is_available()
    w = R.workload("square4")
    rank = 8
    plan = S.Plan(w["mic_xyz"], w["grid_xyz"], w["fs"], w["N"], method="slri", rank=rank,
                  max_frames=64)
    frames = torch.from_numpy(w["frames"]).cuda()
    ref_maps, _ = plan.map(frames)
    xi = plan.gcc_samples(frames)
    torch.cuda.synchronize()
    # the rank-8 factors, columns in the sample order srp_gcc_samples writes
    _, _, _, perm = R.geometry("square4")
    tall, fat, _ = R.slri("square4", rank)
    tall_d = torch.from_numpy(np.ascontiguousarray(tall, dtype=np.float32)).cuda()
    fat_d = torch.from_numpy(np.ascontiguousarray(fat[:, perm], dtype=np.float32)).cuda()
    F, J, L = frames.shape[0], w["grid_xyz"].shape[0], xi.shape[1]
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for sl in (slice(0, F), slice(37, F)):
        x = xi[sl].contiguous()
        n = x.shape[0]
        maps = torch.empty((n, J), device="cuda")
        am = torch.empty((n,), dtype=torch.int32, device="cuda")
        S.srp_slri_apply_static(_p(x), _p(fat_d), _p(tall_d), n, L, rank, J, _p(maps), _p(am),
                                stream)
        torch.cuda.synchronize()
        z = maps.cpu().numpy()
        zr = ref_maps[sl].cpu().numpy().astype(np.float64)
        rel = np.sqrt(((z - zr) ** 2).sum(1) / (zr ** 2).sum(1))
        assert rel.max() <= TOL, rel.max()
        a = am.cpu().numpy()
        assert np.array_equal(a, np.argmax(z, axis=1))
        err = np.abs(z - zr).max(axis=1)
        assert np.all(zr[np.arange(n), a] >= zr.max(axis=1) - 2 * err - 1e-6)
    # requests beyond the static scratch are refused with a message, before any launch
    with pytest.raises(S.SrpError) as e:
        S.srp_slri_apply_static(_p(xi), _p(fat_d), _p(tall_d), 200000, L, rank, J, _p(ref_maps),
                                None, stream)
    assert e.value.status == S.SRP_EINVAL and "static scratch" in S.srp_last_error()
