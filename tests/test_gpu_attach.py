"""Parity of the CUDA track-based cluster attachment (the attachment stage of
tpc_track, through the C ABI) with the oracle's (oracle/tpc_oracle_attach.c)
on the same seeded inputs: flags and adjacent tracks bit-exact, on single
events, continuous read-out frames, batched sub-time-frames, ragged and
degenerate inputs, and tube radius / pT cut settings that exercise every
flag.  At the full 50-collision frame, the flag definitions and the graph
replay are checked (the oracle's tracking of it takes minutes; its parity
test is marked slow)."""
import numpy as np
import pytest

import tpcgen

pytestmark = pytest.mark.gpu


def _dev(arrs):
    import torch
    d = torch.device("cuda:0")
    return [torch.from_numpy(np.ascontiguousarray(a)).to(d) for a in arrs]


def run_attach(ev, radius=1.5, pt_min=0.05, **kw):
    import torch

    import paper_1905_05515_b300 as tpc
    p = tpc.tpc_params_default(tube_radius=radius, pt_min_physics=pt_min, **kw)
    trk = tpc.Tracker(max(ev.n, 1), ev.row_x, n_sectors=ev.n_sectors, z_max=ev.z_max, continuous=ev.continuous,
                      params=p, attach=True)
    res = trk.track(*_dev((ev.sector, ev.row, ev.y, ev.zt)), bz=ev.bz, v_drift=ev.v_drift)
    torch.cuda.synchronize()
    return res.assign.cpu().numpy(), res.cl_flags.cpu().numpy(), res.adjacent.cpu().numpy(), res.n_tracks


def check(ev, orc, radius=1.5, pt_min=0.05, orc_params=None, **kw):
    assign, fl, adj, T = run_attach(ev, radius, pt_min, **kw)
    r = orc.track_event(ev, params=orc_params)
    adj_o, fl_o = orc.attach_event(ev, r, radius=radius, pt_min=pt_min)
    np.testing.assert_array_equal(assign, r.assign)
    np.testing.assert_array_equal(fl, fl_o)
    np.testing.assert_array_equal(adj, adj_o)
    counts = {k: int(((fl & b) > 0).sum()) for k, b in (("attached", 1), ("adjacent", 2), ("protected", 4),
                                                        ("remove", 8))}
    print(f"{ev.n} clusters, {T} tracks: {counts}")
    return fl, adj, counts


def test_one_sector(orc):
    check(tpcgen.one_sector(seed=1), orc)


@pytest.mark.parametrize("radius, pt_min", [(1.5, 0.05), (1.5, 0.3), (4.0, 0.3), (0.0, 0.05)])
def test_central_event_settings(orc, radius, pt_min):
    fl, adj, c = check(tpcgen.central_event(seed=2, n_tracks=1500, with_truth=False), orc, radius, pt_min)
    if radius > 0:
        assert c["adjacent"] > 0
    else:
        assert c["adjacent"] == 0
    if pt_min >= 0.3:
        assert c["remove"] > 0


def test_time_frame(orc):
    check(tpcgen.time_frame(seed=3, n_collisions=3, with_truth=False), orc, pt_min=0.25)


def test_packed_link_coordinates(orc):
    """The attachment reads full-precision coordinates whatever the link pass saw."""
    check(tpcgen.time_frame(seed=3, n_collisions=2, with_truth=False), orc, pt_min=0.25,
          orc_params=dict(orc.default_params(), packed_links=1), packed_links=1)


def test_ragged_and_degenerate(orc):
    for n_tracks, seed in ((1, 31), (7, 32), (33, 33), (257, 34)):
        check(tpcgen.central_event(seed=seed, n_tracks=n_tracks, with_truth=False), orc, pt_min=0.3)
    ev = tpcgen.generate(n_sectors=36, n_tracks=0, noise_frac=0.0, seed=41, with_truth=False)
    rng = np.random.default_rng(5)        # noise only: random clusters, no tracks
    n = 5000
    ev.sector = rng.integers(0, 36, n).astype(np.uint8)
    ev.row = rng.integers(0, 152, n).astype(np.uint8)
    ev.y = rng.uniform(-10, 10, n).astype(np.float32)
    ev.zt = rng.uniform(-250, 250, n).astype(np.float32)
    fl, adj, c = check(ev, orc)
    assert c["attached"] == 0 and c["adjacent"] == 0


def test_batched_frames(orc):
    import torch

    import paper_1905_05515_b300 as tpc
    evs = [tpcgen.time_frame(seed=600 + i, n_collisions=nc, mult_mean=300.0, frame_us=20.0 * nc, with_truth=False)
           for i, nc in enumerate([1, 3, 2])]
    cat = [np.concatenate([getattr(e, k) for e in evs]) for k in ("sector", "row", "y", "zt")]
    off = np.concatenate([[0], np.cumsum([e.n for e in evs])]).astype(np.int32)
    p = tpc.tpc_params_default(pt_min_physics=0.25)
    trk = tpc.Tracker(int(off[-1]), evs[0].row_x, continuous=True, params=p, n_frames=len(evs), attach=True)
    res = trk.track_batched(*_dev(cat), off, bz=evs[0].bz, v_drift=evs[0].v_drift)
    torch.cuda.synchronize()
    fl, adj = res.cl_flags.cpu().numpy(), res.adjacent.cpu().numpy()
    toff = 0
    for f, ev in enumerate(evs):
        r = orc.track_event(ev)
        adj_o, fl_o = orc.attach_event(ev, r, pt_min=0.25)
        a, b = off[f], off[f + 1]
        np.testing.assert_array_equal(fl[a:b], fl_o)
        np.testing.assert_array_equal(adj[a:b], np.where(adj_o >= 0, adj_o + toff, -1))
        toff += r.n_tracks


def test_full_frame_definitions_and_graph():
    """50-collision frame (16 M clusters): the flags follow their definitions,
    and the captured graph's replay gives the synchronous call's flags."""
    import torch

    import paper_1905_05515_b300 as tpc
    ev = tpcgen.time_frame(seed=3, with_truth=False)
    p = tpc.tpc_params_default(pt_min_physics=0.2)
    trk = tpc.Tracker(ev.n, ev.row_x, continuous=True, params=p, attach=True)
    ins = _dev((ev.sector, ev.row, ev.y, ev.zt))
    res = trk.track(*ins, bz=ev.bz, v_drift=ev.v_drift)
    torch.cuda.synchronize()
    T = res.n_tracks
    assign, fl, adj = res.assign.cpu().numpy(), res.cl_flags.cpu().numpy(), res.adjacent.cpu().numpy()
    att, adjf, prot, rem = ((fl & b) > 0 for b in (1, 2, 4, 8))
    assert (fl < 16).all()
    np.testing.assert_array_equal(att, assign >= 0)
    np.testing.assert_array_equal(adjf, adj >= 0)
    assert not (att & adjf).any()
    np.testing.assert_array_equal(rem, (att | adjf) & ~prot)
    assert adj.max() < T and adjf.sum() > 1000 and rem.sum() > 1000
    g = trk.capture(*ins, bz=ev.bz, v_drift=ev.v_drift)
    res.cl_flags.fill_(0xFF)
    g.replay()
    torch.cuda.synchronize()
    np.testing.assert_array_equal(res.cl_flags.cpu().numpy(), fl)
    np.testing.assert_array_equal(res.adjacent.cpu().numpy(), adj)


@pytest.mark.slow
def test_full_frame_parity(orc):
    """The whole 50-collision frame against the oracle (the oracle's tracking
    takes a few minutes)."""
    check(tpcgen.time_frame(seed=3, with_truth=False), orc, pt_min=0.2)
