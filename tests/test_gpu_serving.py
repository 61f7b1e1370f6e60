"""The serving runtime (srp_server_*) on the GPU: continuous batching across sessions of
different arrays, grids, methods and precisions gives every session the maps it gets
alone, and the maps srp_map gives for the same frames; admission by HBM footprint;
back-pressure; a session whose plan cannot be built fails alone."""
import time

import numpy as np
import pytest

import oracle as O
import synth
from tests import _ref as R

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import paper_2306_08514_gb300 as S
    S.lib()
    return S


def stream_of(frames, hop):
    """The continuous multichannel signal [M][n] the frames were cut from."""
    F, M, N = frames.shape
    parts = [frames[0]] + [frames[f][:, N - hop:] for f in range(1, F)]
    return np.ascontiguousarray(np.concatenate(parts, axis=1))


SESSIONS = {
    # name: (workload, frames, grid subsample, hop, plan kwargs, tolerance vs srp_map)
    "uca8-slri": ("uca8", 40, 13, 256, dict(method="slri", rank=16, precision="fp16x3"), 1e-5),
    "uca8-sspi": ("uca8", 33, 17, 256, dict(method="sspi", taps=4.0, precision="bf16"), 1.5e-2),
    "square4-conv": ("square4", 29, 1, 256, dict(method="conv", precision="bf16"), 1.5e-2),
    "square4-sspi32": ("square4", 21, 1, 256, dict(method="sspi", taps=2.0, precision="fp32"), 1e-5),
}


def _inputs(name):
    wl, F, sub, hop, kw, tol = SESSIONS[name]
    w = R.workload(wl, F, sub)
    return w, hop, kw, tol


def _reference(S, name):
    import torch
    w, hop, kw, tol = _inputs(name)
    plan = S.Plan(w["mic_xyz"], w["grid_xyz"], w["fs"], w["N"], max_frames=64, **kw)
    maps, am = plan.map(torch.from_numpy(w["frames"]).cuda())
    torch.cuda.synchronize()
    return maps.cpu().numpy(), am.cpu().numpy()


def _drain(srv, sids, want, deadline=60.0):
    out = {s: {} for s in sids}
    t0 = time.time()
    while any(len(out[s]) < want[s] for s in sids):
        for s in sids:
            maps, am, idx, lat = srv.poll(s)
            for j in range(len(idx)):
                out[s][int(idx[j])] = (maps[j].copy(), int(am[j]), float(lat[j]))
        assert time.time() - t0 < deadline, "serving did not finish"
        time.sleep(0.001)
    return out


def _feed(srv, plan_of, order_rng, chunk_rng):
    """Push every session's stream in random interleaved chunks (1..3 hops)."""
    pos = {s: 0 for s in plan_of}
    streams = {s: v[0] for s, v in plan_of.items()}
    hops = {s: v[1] for s, v in plan_of.items()}
    live = [s for s in plan_of]
    while live:
        s = live[order_rng.integers(len(live))]
        n = int(chunk_rng.integers(1, 4)) * hops[s]
        seg = streams[s][:, pos[s]:pos[s] + n]
        while not srv.push(s, seg):
            time.sleep(0.0005)
            srv.poll(s)  # not expected: the queues are large enough here
        pos[s] += seg.shape[1]
        if pos[s] >= streams[s].shape[1]:
            live.remove(s)


def _open(srv, name):
    w, hop, kw, tol = _inputs(name)
    return srv.open(w["mic_xyz"], w["grid_xyz"], w["fs"], w["N"], hop, **kw)


def test_results_same_alone_and_in_the_mix(S):
    names = list(SESSIONS)
    refs = {n: _reference(S, n) for n in names}
    # alone: one session per server run
    alone = {}
    for n in names:
        srv = S.Server(hbm_budget=4 << 30, max_batch=8, streams=2, slots_per_session=2)
        sid = _open(srv, n)
        w, hop, kw, tol = _inputs(n)
        _feed(srv, {sid: (stream_of(w["frames"], hop), hop)}, np.random.default_rng(1),
              np.random.default_rng(2))
        alone[n] = _drain(srv, [sid], {sid: w["F"]})[sid]
        srv.close()
    # in the mix: all sessions at once, interleaved pushes, several streams
    srv = S.Server(hbm_budget=8 << 30, max_batch=8, streams=3, slots_per_session=3)
    sids = {n: _open(srv, n) for n in names}
    plan_of = {}
    for n, sid in sids.items():
        w, hop, kw, tol = _inputs(n)
        plan_of[sid] = (stream_of(w["frames"], hop), hop)
    _feed(srv, plan_of, np.random.default_rng(3), np.random.default_rng(4))
    mix = _drain(srv, list(sids.values()), {sids[n]: _inputs(n)[0]["F"] for n in names})
    st = srv.stats()
    assert st["frames_done"] == sum(_inputs(n)[0]["F"] for n in names)
    assert st["graph_launches"] > 0 and st["launches"] >= st["graph_launches"]
    assert 0 < st["latency_p50_s"] <= st["latency_p99_s"] <= st["latency_max_s"]
    srv.close()
    for n in names:
        w, hop, kw, tol = _inputs(n)
        zr, ar = refs[n]
        za = np.stack([alone[n][f][0] for f in range(w["F"])])
        zm = np.stack([mix[sids[n]][f][0] for f in range(w["F"])])
        am_m = np.array([mix[sids[n]][f][1] for f in range(w["F"])])
        # the same frames through srp_map, and alone vs in the mix
        assert R.per_frame_rel(za, zr.astype(np.float64)).max() <= tol, n
        assert R.per_frame_rel(zm, za.astype(np.float64)).max() <= tol, n
        assert np.array_equal(am_m, np.argmax(zm, axis=1)), n
    # one session against the FP64 oracle directly
    w, hop, kw, tol = _inputs("square4-sspi32")
    psi = R.psi_of(w["frames"])
    dt, Np, lags, perm = R.geometry("square4", w["F"], 1)
    xi_o, _ = O.gcc_samples_ifft(psi, lags, w["N"] // 2)
    Lam = O.interp_matrix(dt, w["fs"], lags)
    zo = O.srp_sspi(O.sspi_matrix(Lam, lags, int(round(2.0 * Lam.shape[0] * len(lags)))), xi_o)
    zm = np.stack([mix[sids["square4-sspi32"]][f][0] for f in range(w["F"])])
    assert R.per_frame_rel(zm, zo).max() <= 1e-5


def test_admission_by_footprint_and_release(S):
    w, hop, kw, tol = _inputs("uca8-slri")
    desc = S.make_desc(w["mic_xyz"], w["grid_xyz"], w["fs"], w["N"], max_frames=8, **kw)
    need = S.srp_plan_estimate_bytes(desc)
    one = need + 8 * 2 * (w["mic_xyz"].shape[0] * w["N"] + w["grid_xyz"].shape[0] + 1) * 4
    srv = S.Server(hbm_budget=int(one * 1.5), max_batch=8, streams=2, slots_per_session=2)
    a = _open(srv, "uca8-slri")
    b = _open(srv, "uca8-slri")
    t0 = time.time()
    while srv.session_info(a)["state"] != "active":
        assert time.time() - t0 < 30
        time.sleep(0.01)
    time.sleep(0.2)
    assert srv.session_info(b)["state"] == "queued"  # does not fit next to a
    assert srv.stats()["device_bytes"] <= int(one * 1.5)
    srv.close_session(a)
    t0 = time.time()
    while srv.session_info(b)["state"] != "active":
        assert time.time() - t0 < 30
        time.sleep(0.01)
    _feed(srv, {b: (stream_of(w["frames"], hop), hop)}, np.random.default_rng(5),
          np.random.default_rng(6))
    got = _drain(srv, [b], {b: w["F"]})[b]
    zr, ar = _reference(S, "uca8-slri")
    zb = np.stack([got[f][0] for f in range(w["F"])])
    assert R.per_frame_rel(zb, zr.astype(np.float64)).max() <= tol
    srv.close()


def test_back_pressure_and_failed_session(S):
    w, hop, kw, tol = _inputs("square4-conv")
    srv = S.Server(hbm_budget=2 << 30, max_batch=4, streams=1, slots_per_session=1,
                   pending_frames=4)
    sid = _open(srv, "square4-conv")
    sig = stream_of(w["frames"], hop)
    refused = False
    for f in range(64):  # without polling, the queue of 4 frames must fill up
        if not srv.push(sid, sig[:, f * hop:(f + 1) * hop]):
            refused = True
            break
    assert refused
    # a plan that cannot be built (an SLRI rank above the 25 cells of its grid: accepted
    # when the session opens, refused when its plan is built) fails its session only
    tiny = synth.grid_plane((1.0, 1.0), (3.0, 3.0), (5, 5))
    bad = srv.open(w["mic_xyz"], tiny, w["fs"], w["N"], hop, method="slri", rank=40,
                   precision="fp32")
    t0 = time.time()
    while True:
        try:
            st = srv.session_info(bad)["state"]
        except S.SrpError:
            break
        assert st in ("queued", "active") and time.time() - t0 < 30
        time.sleep(0.01)
    srv.close_session(bad)
    assert srv.session_info(sid)["state"] == "active"
    srv.close()


GROUPED = {
    # sessions whose FP32 plans qualify for grouped launches: two buckets (SLRI R = 16 on
    # the uca8 array, whole-vector SSPI), different grids in each
    "g-slri-13": ("uca8", 37, 13, 256, dict(method="slri", rank=16, precision="fp32")),
    "g-slri-17": ("uca8", 31, 17, 256, dict(method="slri", rank=16, precision="fp32")),
    "g-slri-23": ("uca8", 26, 23, 256, dict(method="slri", rank=14, precision="fp32")),
    "g-sspi-13": ("uca8", 29, 13, 256, dict(method="sspi", taps=4.0, precision="fp32")),
    "g-sspi-19": ("uca8", 35, 19, 256, dict(method="sspi", taps=2.0, precision="fp32")),
}


def test_grouped_launches_share_kernels_and_match_srp_map(S):
    """FP32 sessions on the fused front end share launches: one front-end kernel, one
    interpolation kernel and one argmax pass carry the frames of several sessions.  Every
    session's maps and estimates equal srp_map's on its own plan bit for bit (the grouped
    kernels run the same per-frame arithmetic), and launches carry more than one session
    on average."""
    import torch
    refs, inputs = {}, {}
    for n, (wl, F, sub, hop, kw) in GROUPED.items():
        w = R.workload(wl, F, sub)
        inputs[n] = (w, hop, kw)
        plan = S.Plan(w["mic_xyz"], w["grid_xyz"], w["fs"], w["N"], max_frames=64, **kw)
        maps, am = plan.map(torch.from_numpy(w["frames"]).cuda())
        torch.cuda.synchronize()
        refs[n] = (maps.cpu().numpy(), am.cpu().numpy())
        plan.close()
    srv = S.Server(hbm_budget=8 << 30, max_batch=8, streams=2, slots_per_session=3,
                   pending_frames=64, group_launches=True)
    sids = {n: srv.open(w["mic_xyz"], w["grid_xyz"], w["fs"], w["N"], hop, **kw)
            for n, (w, hop, kw) in inputs.items()}
    t0 = time.time()
    while any(srv.session_info(s)["state"] != "active" for s in sids.values()):
        assert time.time() - t0 < 120, "sessions not admitted"
        time.sleep(0.01)
    srv.reset_stats()
    plan_of = {sids[n]: (stream_of(w["frames"], hop), hop) for n, (w, hop, kw) in inputs.items()}
    _feed(srv, plan_of, np.random.default_rng(5), np.random.default_rng(6))
    got = _drain(srv, list(sids.values()), {sids[n]: inputs[n][0]["F"] for n in inputs})
    st = srv.stats()
    srv.close()
    for n, sid in sids.items():
        zr, ar = refs[n]
        F = inputs[n][0]["F"]
        assert sorted(got[sid]) == list(range(F))
        z = np.stack([got[sid][f][0] for f in range(F)])
        a = np.array([got[sid][f][1] for f in range(F)])
        assert np.array_equal(z, zr), n
        assert np.array_equal(a, ar), n
    assert st["group_launches"] > 0 and st["group_launches"] == st["launches"], st
    assert st["group_sessions"] > st["group_launches"], st  # launches shared by sessions
    assert st["group_frames"] == sum(inputs[n][0]["F"] for n in inputs), st
