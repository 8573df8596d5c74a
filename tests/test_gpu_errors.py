"""Error behaviour of the C ABI on a GPU: invalid clusters and capacity
overflow return error codes (no fault, no hang)."""
import numpy as np
import pytest

import tpcgen

pytestmark = pytest.mark.gpu


def _tensors(ev):
    import torch
    d = torch.device("cuda:0")
    return [torch.from_numpy(np.ascontiguousarray(a)).to(d) for a in (ev.sector, ev.row, ev.y, ev.zt)]


def test_invalid_sector_and_nonfinite_are_data_errors():
    import paper_1905_05515_b300 as tpc
    ev = tpcgen.one_sector(seed=1, with_truth=False)
    for mutate in ("sector", "row", "nan"):
        e = tpcgen.one_sector(seed=1, with_truth=False)
        if mutate == "sector":
            e.sector[10] = 3          # one-sector geometry: only sector 0 exists
        elif mutate == "row":
            e.row[5] = 200
        else:
            e.zt[7] = np.nan
        trk = tpc.Tracker(e.n, e.row_x, n_sectors=1)
        with pytest.raises(tpc.TpcError) as ex:
            trk.track(*_tensors(e))
        assert ex.value.code == tpc.TPC_ERR_DATA
    # the tracker stays usable after the error
    trk = tpc.Tracker(ev.n, ev.row_x, n_sectors=1)
    assert trk.track(*_tensors(ev)).n_tracks > 100


def test_output_capacity_overflow_reports_needed_sizes():
    import paper_1905_05515_b300 as tpc
    ev = tpcgen.one_sector(seed=1, with_truth=False)
    trk = tpc.Tracker(ev.n, ev.row_x, n_sectors=1, capacity_tracks=5)
    with pytest.raises(tpc.TpcError) as ex:
        trk.track(*_tensors(ev))
    assert ex.value.code == tpc.TPC_ERR_CAPACITY
    assert ex.value.needed["tracks"] > 5


def test_too_many_clusters_for_the_tracker():
    import paper_1905_05515_b300 as tpc
    ev = tpcgen.one_sector(seed=1, with_truth=False)
    trk = tpc.Tracker(100, ev.row_x, n_sectors=1)
    with pytest.raises(ValueError):
        trk.track(*_tensors(ev))


def test_repeated_calls_are_identical():
    import paper_1905_05515_b300 as tpc
    ev = tpcgen.central_event(seed=9, n_tracks=500, with_truth=False)
    trk = tpc.Tracker(ev.n, ev.row_x)
    ts = _tensors(ev)
    a = trk.track(*ts)
    ca, pa = a.clus_index[: int(a.clus_offset[-1])].cpu().numpy(), a.param.cpu().numpy()
    b = trk.track(*ts)
    np.testing.assert_array_equal(b.clus_index[: int(b.clus_offset[-1])].cpu().numpy(), ca)
    np.testing.assert_array_equal(b.param.cpu().numpy(), pa)
