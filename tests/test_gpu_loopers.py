"""Parity of the CUDA looper-leg identification (the looper stage of
tpc_track / tpc_track_batched, through the C ABI) with the oracle's
(oracle/tpc_oracle_loopers.c): the group of every track and its leg number
bit-exact, on continuous frames with loopers, another candidate threshold,
batched sub-time-frames, and inputs without candidates."""
import numpy as np
import pytest

import tpcgen

pytestmark = pytest.mark.gpu


def _dev(arrs):
    import torch
    d = torch.device("cuda:0")
    return [torch.from_numpy(np.ascontiguousarray(a)).to(d) for a in arrs]


def run_loopers(ev, **kw):
    import torch

    import paper_1905_05515_b300 as tpc
    p = tpc.tpc_params_default(**kw)
    trk = tpc.Tracker(max(ev.n, 1), ev.row_x, n_sectors=ev.n_sectors, z_max=ev.z_max, continuous=ev.continuous,
                      params=p, loopers=True)
    res = trk.track(*_dev((ev.sector, ev.row, ev.y, ev.zt)), bz=ev.bz, v_drift=ev.v_drift)
    torch.cuda.synchronize()
    return res.assign.cpu().numpy(), res.looper_group.cpu().numpy(), res.looper_leg.cpu().numpy()


@pytest.mark.parametrize("seed, ncoll, qmin", [(3, 3, 5.0), (4, 8, 5.0), (4, 8, 2.0)])
def test_frames(orc, seed, ncoll, qmin):
    ev = tpcgen.time_frame(seed=seed, n_collisions=ncoll, with_truth=False)
    assign, g, lg = run_loopers(ev, looper_qpt_min=qmin)
    r = orc.track_event(ev)
    np.testing.assert_array_equal(assign, r.assign)
    g_o, lg_o = orc.loopers(ev.sector, r, qpt_min=qmin)
    np.testing.assert_array_equal(g, g_o)
    np.testing.assert_array_equal(lg, lg_o)
    print(f"{ev.n} clusters: {int((g >= 0).sum())} legs in {len(set(g[g >= 0].tolist()))} groups")
    assert (g >= 0).sum() > 20


def test_without_candidates(orc):
    for ev in (tpcgen.central_event(seed=31, n_tracks=7, with_truth=False), tpcgen.one_sector(seed=1)):
        assign, g, lg = run_loopers(ev)
        r = orc.track_event(ev)
        g_o, lg_o = orc.loopers(ev.sector, r, n_sectors=ev.n_sectors)
        np.testing.assert_array_equal(g, g_o)
        np.testing.assert_array_equal(lg, lg_o)


def test_batched_frames(orc):
    import torch

    import paper_1905_05515_b300 as tpc
    evs = [tpcgen.time_frame(seed=610 + i, n_collisions=nc, frame_us=20.0 * nc, with_truth=False)
           for i, nc in enumerate([2, 4, 1])]
    cat = [np.concatenate([getattr(e, k) for e in evs]) for k in ("sector", "row", "y", "zt")]
    off = np.concatenate([[0], np.cumsum([e.n for e in evs])]).astype(np.int32)
    trk = tpc.Tracker(int(off[-1]), evs[0].row_x, continuous=True, n_frames=len(evs), loopers=True)
    res = trk.track_batched(*_dev(cat), off, bz=evs[0].bz, v_drift=evs[0].v_drift)
    torch.cuda.synchronize()
    g, lg = res.looper_group.cpu().numpy(), res.looper_leg.cpu().numpy()
    toff, n_groups = 0, 0
    for ev in evs:
        r = orc.track_event(ev)
        g_o, lg_o = orc.loopers(ev.sector, r)
        T = r.n_tracks
        np.testing.assert_array_equal(g[toff:toff + T], np.where(g_o >= 0, g_o + toff, -1))
        np.testing.assert_array_equal(lg[toff:toff + T], lg_o)
        n_groups += len(set(g_o[g_o >= 0].tolist()))
        toff += T
    assert toff == res.n_tracks and n_groups > 5
