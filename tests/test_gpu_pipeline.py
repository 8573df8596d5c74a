"""FramePipeline: frames from host memory, copies overlapping the tracking of
other frames.  Every frame's tracks, cluster lists and assignments equal a
synchronous tpc_track call on the same frame, whatever the pipeline depth and
however the frame sizes vary."""
import numpy as np
import pytest
import torch

import tpcgen

pytestmark = pytest.mark.gpu


def _frames():
    out = []
    for i, (seed, nc) in enumerate([(3, 2), (4, 1), (5, 3), (6, 1), (7, 2)]):
        out.append(tpcgen.time_frame(seed=seed, n_collisions=nc, with_truth=False))
    return out


@pytest.mark.parametrize("depth", [1, 2, 3])
def test_pipeline_equals_synchronous_calls(depth):
    import paper_1905_05515_b300 as tpc
    frames = _frames()
    n_max = max(ev.n for ev in frames)
    ev0 = frames[0]
    trk = tpc.Tracker(n_max, ev0.row_x, continuous=True)
    want = []
    for ev in frames:
        t = [torch.from_numpy(np.ascontiguousarray(getattr(ev, k))).cuda() for k in ("sector", "row", "y", "zt")]
        r = trk.track(*t, bz=ev.bz, v_drift=ev.v_drift)
        T = r.n_tracks
        want.append((T, r.param.cpu().numpy().copy(), r.chi2.cpu().numpy().copy(),
                     r.clus_offset.cpu().numpy().copy(), r.clus_index[:int(r.clus_offset[-1])].cpu().numpy().copy(),
                     r.assign.cpu().numpy().copy()))
    pipe = tpc.FramePipeline(n_max, ev0.row_x, depth=depth, bz=ev0.bz, v_drift=ev0.v_drift)
    got = []
    for ev in frames:
        host = [torch.from_numpy(np.ascontiguousarray(getattr(ev, k))) for k in ("sector", "row", "y", "zt")]
        r = pipe.push(*[h.pin_memory() for h in host])
        if r is not None:
            got.append(r)
            got[-1] = (r.n_tracks, r.param.numpy().copy(), r.chi2.numpy().copy(), r.clus_offset.numpy().copy(),
                       r.clus_index.numpy().copy(), r.assign.numpy().copy())
    for r in pipe.flush():
        got.append((r.n_tracks, r.param.numpy().copy(), r.chi2.numpy().copy(), r.clus_offset.numpy().copy(),
                    r.clus_index.numpy().copy(), r.assign.numpy().copy()))
    assert len(got) == len(want)
    for g, w in zip(got, want):
        assert g[0] == w[0]
        for a, b in zip(g[1:], w[1:]):
            assert np.array_equal(a, b)


def test_pipeline_rejects_bad_frames():
    import paper_1905_05515_b300 as tpc
    ev = tpcgen.time_frame(seed=3, n_collisions=1, with_truth=False)
    pipe = tpc.FramePipeline(ev.n, ev.row_x, depth=2)
    with pytest.raises(ValueError):
        pipe.push(torch.zeros(ev.n + 1, dtype=torch.uint8), torch.zeros(ev.n + 1, dtype=torch.uint8),
                  torch.zeros(ev.n + 1), torch.zeros(ev.n + 1))
    with pytest.raises(ValueError):
        pipe.push(torch.zeros(4, dtype=torch.int32), torch.zeros(4, dtype=torch.uint8), torch.zeros(4), torch.zeros(4))
    assert pipe.flush() == []
