"""The autotuner (paper_1905_05515_b300/autotune.py) picks, among settings
that change speed but never results, the fastest: on a forced two-point
space whose slow point is known (one y-bin per z-cell: every window search
scans the full width of its pad row) it must pick the other point, and the
tracks with the tuned settings must equal those with the defaults, bit for
bit; the grouping tuner's choice gives the per-frame tracks."""
import numpy as np
import pytest

import tpcgen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def batch():
    import torch
    frames = [tpcgen.time_frame(seed=70 + i, n_collisions=8, frame_us=160.0, with_truth=False) for i in range(3)]
    off = np.concatenate([[0], np.cumsum([f.n for f in frames])]).astype(np.int64)
    dev = torch.device("cuda:0")
    ins = tuple(torch.from_numpy(np.concatenate([getattr(f, k) for f in frames])).to(dev)
                for k in ("sector", "row", "y", "zt"))
    return ins, off


def _tracks(ins, off, params):
    import paper_1905_05515_b300 as tpc
    trk = tpc.Tracker(int(off[-1]), tpcgen.row_x_f32(), continuous=True, params=params, n_frames=off.size - 1)
    r = trk.track_batched(*ins, off.astype(np.int32), bz=0.5, v_drift=tpcgen.V_DRIFT)
    T = r.n_tracks
    return r.param[:T].cpu().numpy(), r.assign.cpu().numpy()


def test_picks_the_fastest_of_a_forced_two_point_space(batch):
    import paper_1905_05515_b300 as tpc
    ins, off = batch
    res = tpc.autotune.autotune(*ins, off.astype(np.int32), tpcgen.row_x_f32(), space={"y_bins": (1, 16)}, reps=3)
    table = {c["y_bins"]: ms for c, ms in res["table"]}
    print(f"autotune table (y_bins: ms): {table}")
    assert res["best"] == {"y_bins": min(table, key=table.get)} and res["ms"] == min(table.values())
    assert table[1] > 1.15 * table[16]          # the forced slow point is slow
    assert res["best"]["y_bins"] == 16
    p_t, a_t = _tracks(ins, off, tpc.autotune.apply(tpc.tpc_params_default(), res["best"]))
    p_d, a_d = _tracks(ins, off, tpc.tpc_params_default())
    p_1, a_1 = _tracks(ins, off, tpc.tpc_params_default(y_bins=1))
    for p, a in ((p_t, a_t), (p_1, a_1)):
        np.testing.assert_array_equal(p, p_d)
        np.testing.assert_array_equal(a, a_d)


def test_group_tuner_choice_gives_the_per_frame_tracks(batch):
    import torch

    import paper_1905_05515_b300 as tpc
    ins, off = batch
    params = tpc.tpc_params_default()
    res = tpc.autotune.autotune_groups(*ins, off, tpcgen.row_x_f32(), params,
                                       space={"group_clusters": (0, 1 << 30), "n_streams": (1, 2)}, reps=2)
    assert len(res["table"]) == 4 and res["ms"] == min(ms for _, ms in res["table"])
    gb = tpc.GroupedBatch(*ins, off, tpcgen.row_x_f32(), params=params, bz=0.5, v_drift=tpcgen.V_DRIFT,
                          **res["best"])
    gb.capture()
    gb.replay()
    p_g = torch.cat([r.param for r in gb.results()]).cpu().numpy()
    one = tpc.Tracker(int(np.max(np.diff(off))), tpcgen.row_x_f32(), continuous=True, params=params)
    p_f = np.concatenate([one.track(*(t[int(off[i]):int(off[i + 1])] for t in ins), bz=0.5,
                                    v_drift=tpcgen.V_DRIFT).param.cpu().numpy() for i in range(off.size - 1)])
    np.testing.assert_array_equal(p_g, p_f)
