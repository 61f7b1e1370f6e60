"""Failure detection on the GPU.  Every failure is made on the host side of a call, never
as a device fault, trap or endless wait: an injected allocation failure (a fake of the
failing cudaMalloc: SRP_ENOMEM, nothing leaks, the server refuses that session alone), a
tensor-core contraction whose producer issues no loads so that the consumers' bounded waits
(0.2 s) run out (SRP_ETIMEOUT, the plan stays usable), and a session closed while its
frames are in flight."""
import time

import numpy as np
import pytest

from tests import _ref as R
from tests.test_gpu_serving import S, _drain, _feed, _inputs, _open, _reference, stream_of  # noqa: F401

pytestmark = pytest.mark.gpu


def _square4(S):
    w = R.workload("square4")
    return w, (w["mic_xyz"], w["grid_xyz"], w["fs"], w["N"])


def _maps(plan, frames):
    import torch
    z, am = plan.map(frames)
    torch.cuda.synchronize()
    return z.cpu().numpy(), am.cpu().numpy()


def test_injected_allocation_failure_at_every_point_of_plan_creation(S):
    """Plan creation fails with SRP_ENOMEM at whichever of its allocations fails, releases
    what it held, and the next creation gives the same maps as before."""
    import torch
    w, args = _square4(S)
    kw = dict(method="sspi", taps=2.0, precision="bf16", max_frames=32)
    fr = torch.from_numpy(np.ascontiguousarray(w["frames"][:32])).cuda()
    ref = S.Plan(*args, **kw)
    z0, a0 = _maps(ref, fr)
    ref.close()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    failed_at = []
    try:
        for after in range(200):
            S.srp_debug_fail_allocations(after, 1 << 20)
            try:
                plan = S.Plan(*args, **kw)
            except S.SrpError as e:
                assert e.status == S.SRP_ENOMEM, e
                failed_at.append(after)
                continue
            S.srp_debug_fail_allocations(0, 0)
            z1, a1 = _maps(plan, fr)  # the allocations it needs all came through
            assert np.array_equal(z1, z0) and np.array_equal(a1, a0)
            plan.close()
            break
    finally:
        S.srp_debug_fail_allocations(0, 0)
    assert failed_at == list(range(len(failed_at))) and len(failed_at) >= 5
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] >= free0 - (8 << 20), "a failed creation leaked"
    z2, a2 = _maps(S.Plan(*args, **kw), fr)
    assert np.array_equal(z2, z0) and np.array_equal(a2, a0)


def test_server_refuses_a_session_whose_allocations_fail(S):
    srv = S.Server(hbm_budget=4 << 30, max_batch=8, streams=2, slots_per_session=2)
    good = _open(srv, "square4-conv")
    t0 = time.time()
    while srv.session_info(good)["state"] != "active":
        assert time.time() - t0 < 60
        time.sleep(0.01)
    S.srp_debug_fail_allocations(0, 1 << 20)
    try:
        bad = _open(srv, "uca8-sspi")
        t0 = time.time()
        while True:  # the builder fails the session; session_info then raises
            try:
                st = srv.session_info(bad)["state"]
            except S.SrpError:
                break
            assert st in ("queued", "active") and time.time() - t0 < 60
            time.sleep(0.01)
    finally:
        S.srp_debug_fail_allocations(0, 0)
    srv.close_session(bad)
    w, hop, kw, tol = _inputs("square4-conv")
    _feed(srv, {good: (stream_of(w["frames"], hop), hop)}, np.random.default_rng(7),
          np.random.default_rng(8))
    got = _drain(srv, [good], {good: w["F"]})[good]
    zr, ar = _reference(S, "square4-conv")
    z = np.stack([got[f][0] for f in range(w["F"])])
    assert R.per_frame_rel(z, zr.astype(np.float64)).max() <= tol
    srv.close()


@pytest.mark.parametrize("method,kw", [("slri", dict(rank=8)), ("sspi", dict(taps=2.0)),
                                       ("conv", {})])
@pytest.mark.parametrize("variant", [-1, 4])
def test_bounded_waits_run_out_and_the_plan_stays_usable(S, method, kw, variant):
    """The stall hook on the heuristic's kernel and on its cluster variant (two CTAs sharing
    the B tiles; SLRI and SSPI run it clustered, conv's split reduction unclustered): both
    CTAs of a cluster time out, meet at the cluster's closing barrier and return."""
    import torch
    w, args = _square4(S)
    fr = torch.from_numpy(np.ascontiguousarray(w["frames"][:32])).cuda()
    plan = S.Plan(*args, method=method, precision="bf16", max_frames=32, **kw)
    plan.set_variant(variant)
    z0, a0 = _maps(plan, fr)
    plan.status()
    plan.debug_stall_next_contraction()
    t0 = time.time()
    _maps(plan, fr)
    elapsed = time.time() - t0
    with pytest.raises(S.SrpError) as e:
        plan.status()
    assert e.value.status == S.SRP_ETIMEOUT
    assert elapsed < 10.0
    plan.status()  # the record is cleared
    z1, a1 = _maps(plan, fr)
    plan.status()
    assert np.array_equal(z1, z0) and np.array_equal(a1, a0)


@pytest.mark.parametrize("method,kw,variant", [("conv", {}, 4), ("conv", {}, 8), ("sspi", dict(taps=2.0), 8)])
def test_bounded_waits_run_out_in_clusters(S, method, kw, variant):
    """The stall hook on launches that do run in clusters (300 frames: three frame tiles;
    4616 cells: 19 cell tiles): 2 x 1 and 2 x 2 for conv's dense reduction, SSPI's
    block-sparse one as 2 x 1.  Every CTA of every cluster times out on its own barriers,
    the cluster's closing barrier completes, the call reports SRP_ETIMEOUT within the bound
    and the next call gives the maps of before."""
    import torch
    w = R.workload("uca8", 300, 13)
    args = (w["mic_xyz"], w["grid_xyz"], w["fs"], w["N"])
    fr = torch.from_numpy(np.ascontiguousarray(w["frames"])).cuda()
    plan = S.Plan(*args, method=method, precision="bf16", max_frames=300, **kw)
    plan.set_variant(variant)
    z0, a0 = _maps(plan, fr)
    plan.status()
    plan.debug_stall_next_contraction()
    t0 = time.time()
    _maps(plan, fr)
    elapsed = time.time() - t0
    with pytest.raises(S.SrpError) as e:
        plan.status()
    assert e.value.status == S.SRP_ETIMEOUT
    assert elapsed < 10.0
    plan.status()
    z1, a1 = _maps(plan, fr)
    plan.status()
    assert np.array_equal(z1, z0) and np.array_equal(a1, a0)


def test_stall_hook_needs_a_tensor_core_plan(S):
    w, args = _square4(S)
    plan = S.Plan(*args, method="slri", rank=8, precision="fp32", max_frames=8)
    with pytest.raises(S.SrpError) as e:
        plan.debug_stall_next_contraction()
    assert e.value.status == S.SRP_EUNSUPPORTED


def test_session_closed_with_frames_in_flight(S):
    """Closing a session while its launches run releases it once they finish; the other
    session keeps its exact results and the server's memory returns to one session's."""
    srv = S.Server(hbm_budget=4 << 30, max_batch=8, streams=2, slots_per_session=2)
    a = _open(srv, "uca8-sspi")
    b = _open(srv, "square4-conv")
    t0 = time.time()
    while not all(srv.session_info(s)["state"] == "active" for s in (a, b)):
        assert time.time() - t0 < 60
        time.sleep(0.01)
    both = srv.stats()["device_bytes"]
    wa, hopa, _, _ = _inputs("uca8-sspi")
    sig = stream_of(wa["frames"], hopa)
    for f in range(sig.shape[1] // hopa):  # no polling: launches are queued and in flight
        if not srv.push(a, sig[:, f * hopa:(f + 1) * hopa]):
            break
    srv.close_session(a)
    w, hop, kw, tol = _inputs("square4-conv")
    _feed(srv, {b: (stream_of(w["frames"], hop), hop)}, np.random.default_rng(9),
          np.random.default_rng(10))
    got = _drain(srv, [b], {b: w["F"]})[b]
    zr, ar = _reference(S, "square4-conv")
    z = np.stack([got[f][0] for f in range(w["F"])])
    assert R.per_frame_rel(z, zr.astype(np.float64)).max() <= tol
    t0 = time.time()
    while srv.stats()["device_bytes"] >= both:
        assert time.time() - t0 < 30, "the closed session was not released"
        time.sleep(0.01)
    srv.close()
