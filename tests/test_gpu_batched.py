"""Batched mode: several sub-time-frames of uneven size in one pass.

Each frame must come out exactly as if it were tracked alone: decisions
bit-exact against the oracle run per frame (indices offset by the frame's
first cluster), fits within the parity tolerance, and bit-identical to the
per-frame GPU calls.  The CUDA-graph replay of the enqueue-only call must
reproduce the synchronous call."""
import numpy as np
import pytest

import tpcgen
from gpu_helpers import param_rel_err

pytestmark = pytest.mark.gpu

N_COLL = [1, 3, 2, 5, 1, 2, 4]


@pytest.fixture(scope="module")
def frames():
    return [tpcgen.time_frame(seed=500 + i, n_collisions=nc, mult_mean=300.0, frame_us=20.0 * nc, with_truth=False)
            for i, nc in enumerate(N_COLL)]


def _concat(evs):
    cat = {k: np.concatenate([getattr(e, k) for e in evs]) for k in ("sector", "row", "y", "zt")}
    off = np.concatenate([[0], np.cumsum([e.n for e in evs])]).astype(np.int32)
    return cat, off


def _dev(cat):
    import torch
    d = torch.device("cuda:0")
    return [torch.from_numpy(np.ascontiguousarray(cat[k])).to(d) for k in ("sector", "row", "y", "zt")]


def test_batched_equals_oracle_per_frame(orc, frames):
    import paper_1905_05515_b300 as tpc
    cat, off = _concat(frames)
    ev0 = frames[0]
    trk = tpc.Tracker(int(off[-1]), ev0.row_x, continuous=True, debug=True, n_frames=len(frames))
    res = trk.track_batched(*_dev(cat), off, bz=ev0.bz, v_drift=ev0.v_drift)
    g = {k: v.cpu().numpy() for k, v in vars(res).items() if hasattr(v, "cpu")}
    exp = {k: [] for k in ("up", "dn", "start", "clus", "assign", "frame", "p", "status", "chi2")}
    toff = 0
    for f, ev in enumerate(frames):
        r = orc.track_event(ev)
        o = off[f]
        exp["up"].append(np.where(r.up >= 0, r.up + o, -1))
        exp["dn"].append(np.where(r.dn >= 0, r.dn + o, -1))
        exp["start"].append(r.is_start)
        exp["clus"].append(r.tr_clus + o)
        exp["assign"].append(np.where(r.assign >= 0, r.assign + toff, -1))
        exp["frame"].append(np.full(r.n_tracks, f))
        exp["p"].append(r.tr_p)
        exp["status"].append(r.tr_status)
        exp["chi2"].append(r.tr_chi2)
        toff += r.n_tracks
    e = {k: np.concatenate(v) for k, v in exp.items()}
    np.testing.assert_array_equal(g["link_up"], e["up"])
    np.testing.assert_array_equal(g["link_dn"], e["dn"])
    np.testing.assert_array_equal(g["is_start"], e["start"])
    assert res.n_tracks == toff
    nc = int(g["clus_offset"][-1])
    np.testing.assert_array_equal(g["clus_index"][:nc], e["clus"])
    np.testing.assert_array_equal(g["assign"], e["assign"])
    np.testing.assert_array_equal(g["frame"], e["frame"])
    ok = (g["status"] == 0) & (e["status"] == 0)
    assert (g["status"] != e["status"]).sum() <= 1
    assert param_rel_err(g["param"][ok], e["p"][ok]).max() < 1e-4
    assert (np.abs(g["chi2"][ok] - e["chi2"][ok]) / np.maximum(e["chi2"][ok], 1)).max() < 1e-3


def test_batched_bit_identical_to_per_frame_calls(frames):
    import paper_1905_05515_b300 as tpc
    cat, off = _concat(frames)
    ev0 = frames[0]
    trk = tpc.Tracker(int(off[-1]), ev0.row_x, continuous=True, n_frames=len(frames))
    rb = trk.track_batched(*_dev(cat), off, bz=ev0.bz, v_drift=ev0.v_drift)
    pb, cb = rb.param.cpu().numpy(), rb.chi2.cpu().numpy()
    t = 0
    for f, ev in enumerate(frames):
        one = tpc.Tracker(ev.n, ev.row_x, continuous=True)
        r1 = one.track(*_dev({k: getattr(ev, k) for k in ("sector", "row", "y", "zt")}), bz=ev.bz, v_drift=ev.v_drift)
        T = r1.n_tracks
        np.testing.assert_array_equal(pb[t:t + T], r1.param.cpu().numpy())
        np.testing.assert_array_equal(cb[t:t + T], r1.chi2.cpu().numpy())
        t += T
    assert t == rb.n_tracks


def test_graph_replay_reproduces_the_synchronous_call(frames):
    import torch

    import paper_1905_05515_b300 as tpc
    cat, off = _concat(frames)
    ev0 = frames[0]
    ins = _dev(cat)
    trk = tpc.Tracker(int(off[-1]), ev0.row_x, continuous=True, n_frames=len(frames))
    ref = trk.track_batched(*ins, off, bz=ev0.bz, v_drift=ev0.v_drift)
    p_ref = ref.param.cpu().numpy().copy()
    c_ref = ref.clus_index[: int(ref.clus_offset[-1])].cpu().numpy().copy()
    run = trk.capture(*ins, off, bz=ev0.bz, v_drift=ev0.v_drift)
    for _ in range(2):
        trk.buf["param"].zero_()
        run.replay()
        torch.cuda.synchronize()
        res = run.result()
        assert res.n_tracks == ref.n_tracks
        np.testing.assert_array_equal(res.param.cpu().numpy(), p_ref)
        np.testing.assert_array_equal(res.clus_index[: int(res.clus_offset[-1])].cpu().numpy(), c_ref)


@pytest.mark.parametrize("group_clusters,n_streams", [(0, 1), (0, 3), (150_000, 2), (10**9, 2)])
def test_grouped_graph_equals_per_frame(frames, group_clusters, n_streams):
    """GroupedBatch (frame groups on several streams, one CUDA graph) gives
    every frame's tracks exactly as a per-frame tpc_track call does, on
    eager runs and on graph replays."""
    import torch

    import paper_1905_05515_b300 as tpc
    cat, off = _concat(frames)
    ev0 = frames[0]
    ins = _dev(cat)
    one = tpc.Tracker(int(np.diff(off).max()), ev0.row_x, continuous=True)
    ref = []
    for f in range(len(frames)):
        a, b = int(off[f]), int(off[f + 1])
        r = one.track(*(t[a:b] for t in ins), bz=ev0.bz, v_drift=ev0.v_drift)
        T = r.n_tracks
        ref.append(dict(param=r.param.cpu().numpy(), chi2=r.chi2.cpu().numpy(), assign=r.assign.cpu().numpy(),
                        clus=r.clus_index[:int(r.clus_offset[T].item()) if T else 0].cpu().numpy()))
    gb = tpc.GroupedBatch(*ins, off, ev0.row_x, group_clusters=group_clusters, n_streams=n_streams,
                          bz=ev0.bz, v_drift=ev0.v_drift)
    assert len(gb.groups) == len(tpc.batch.partition(off, group_clusters))
    for mode in ("eager", "graph", "graph"):
        if mode == "eager":
            gb.run()
        else:
            gb.replay()
        res = gb.results()
        for g, r in zip(gb.groups, res):
            fr = r.frame.cpu().numpy()
            co = r.clus_offset.cpu().numpy()
            asg = r.assign.cpu().numpy()
            t0 = 0
            for f in range(g.f0, g.f1):
                e = ref[f]
                T = e["param"].shape[0]
                sel = np.nonzero(fr == f)[0]
                assert sel.size == T and (T == 0 or sel[0] == t0)
                np.testing.assert_array_equal(r.param[t0:t0 + T].cpu().numpy(), e["param"])
                np.testing.assert_array_equal(r.chi2[t0:t0 + T].cpu().numpy(), e["chi2"])
                lo = int(off[f] - off[g.f0])
                clus = r.clus_index[int(co[t0]):int(co[t0 + T])].cpu().numpy() - lo
                np.testing.assert_array_equal(clus, e["clus"])
                a = asg[lo:lo + e["assign"].size]
                np.testing.assert_array_equal(np.where(a >= 0, a - t0, -1), e["assign"])
                t0 += T
    assert gb.n_launches > 0
    torch.cuda.synchronize()


def test_host_io_capture_equals_device_graph(frames):
    """A capture with per-group host input copies and result copies gives the
    device-resident graph's parameters, chi2 and assignments in host memory."""
    import paper_1905_05515_b300 as tpc
    cat, off = _concat(frames)
    ins = _dev(cat)
    ev0 = frames[0]
    gb = tpc.GroupedBatch(*ins, off, ev0.row_x, bz=ev0.bz, v_drift=ev0.v_drift, group_clusters=1, n_streams=2)
    gb.capture()
    gb.replay()
    want = gb.results()
    host = tuple(t.cpu().pin_memory() for t in ins)
    gb.capture(host_in=host)
    for t in ins:
        t.zero_()                      # the replay must take the clusters from host memory
    gb.replay()
    got = gb.host_results()
    assert len(got) == len(want)
    for (T, p, c2, a), w in zip(got, want):
        assert T == w.n_tracks
        assert np.array_equal(p.numpy(), w.param.cpu().numpy())
        assert np.array_equal(c2.numpy(), w.chi2.cpu().numpy())
        assert np.array_equal(a.numpy(), w.assign.cpu().numpy())


@pytest.mark.slow
def test_batched_call_above_2pow24_clusters():
    """A call of more than 2^24 clusters (the 50-collision frame and an
    8-collision frame, 19 M clusters) ranks the selector's tracklets with
    64-bit weights; per-frame calls (below 2^24) with 32-bit ones.  Both give
    the same tracks."""
    import paper_1905_05515_b300 as tpc
    evs = [tpcgen.time_frame(seed=3, with_truth=False), tpcgen.time_frame(seed=4, n_collisions=8, with_truth=False)]
    cat, off = _concat(evs)
    assert off[-1] > (1 << 24) and all(e.n <= (1 << 24) for e in evs)
    ev0 = evs[0]
    trk = tpc.Tracker(int(off[-1]), ev0.row_x, continuous=True, n_frames=2)
    rb = trk.track_batched(*_dev(cat), off, bz=ev0.bz, v_drift=ev0.v_drift)
    pb, ab = rb.param.cpu().numpy(), rb.assign.cpu().numpy()
    del trk
    t = 0
    for f, ev in enumerate(evs):
        one = tpc.Tracker(ev.n, ev.row_x, continuous=True)
        r1 = one.track(*_dev({k: getattr(ev, k) for k in ("sector", "row", "y", "zt")}), bz=ev.bz, v_drift=ev.v_drift)
        T = r1.n_tracks
        np.testing.assert_array_equal(pb[t:t + T], r1.param.cpu().numpy())
        a1 = r1.assign.cpu().numpy()
        np.testing.assert_array_equal(ab[off[f]:off[f + 1]], np.where(a1 >= 0, a1 + t, -1))
        t += T
        del one
    assert t == rb.n_tracks
