"""tpc_links_static: seeding with no allocation at all.

Some callers cannot allocate device memory when they need the links: a host
thread that must not block in the allocator (which can synchronise the
device) while other streams run, or an embedding that forbids cudaMalloc
after start-up.  This entry point keeps its scratch in a fixed device array inside
the library; the caller passes only its inputs and outputs.  The test calls
it through the C ABI on consecutive, different events and checks that its
links and start flags equal those of tpc_track (bit for bit, as every link
comparison here), so that leftovers of one call cannot leak into the next.
Collected last on purpose (file name), and independent of the other tests.
"""
import ctypes as C

import numpy as np
import pytest

import tpcgen

pytestmark = pytest.mark.gpu


def _bind():
    import paper_1905_05515_b300 as tpc
    L = tpc.lib()
    L.tpc_links_static.argtypes = [C.POINTER(tpc.abi.TpcParams), C.POINTER(tpc.abi.TpcGeometry), C.c_float,
                                   C.POINTER(tpc.abi.TpcClusters), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    return tpc, L


def _static_links(tpc, L, ev, ts):
    import torch
    n = ev.n
    params = tpc.tpc_params_default()
    geom = tpc.abi.make_geometry(ev.row_x, ev.n_sectors, ev.z_max, ev.continuous)
    cl = tpc.abi.TpcClusters(n, *(t.data_ptr() for t in ts))
    dev = ts[0].device
    up = torch.full((n,), -7, dtype=torch.int32, device=dev)
    dn = torch.full((n,), -7, dtype=torch.int32, device=dev)
    st = torch.full((n,), 7, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev).cuda_stream
    rc = L.tpc_links_static(C.byref(params), C.byref(geom), ev.v_drift, C.byref(cl), up.data_ptr(), dn.data_ptr(),
                            st.data_ptr(), stream)
    assert rc == 0, tpc.tpc_error_string(rc)
    return up.cpu().numpy(), dn.cpu().numpy(), st.cpu().numpy()


def test_static_links_equal_tpc_track_on_consecutive_calls():
    import torch
    tpc, L = _bind()
    dev = torch.device("cuda:0")
    events = [tpcgen.central_event(seed=2, n_tracks=1500, with_truth=False),   # 250 k clusters, 36 sectors
              tpcgen.one_sector(seed=1, with_truth=False),                       # 17 k clusters, 1 sector
              tpcgen.time_frame(seed=3, n_collisions=3, with_truth=False)]       # drift times
    for ev in events:
        assert ev.n <= 262144
        ts = [torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in (ev.sector, ev.row, ev.y, ev.zt)]
        up, dn, st = _static_links(tpc, L, ev, ts)
        trk = tpc.Tracker(ev.n, ev.row_x, n_sectors=ev.n_sectors, z_max=ev.z_max, continuous=ev.continuous,
                          debug=True)
        ref = trk.track(*ts, bz=ev.bz, v_drift=ev.v_drift)
        np.testing.assert_array_equal(up, ref.link_up.cpu().numpy())
        np.testing.assert_array_equal(dn, ref.link_dn.cpu().numpy())
        np.testing.assert_array_equal(st, ref.is_start.cpu().numpy())
        assert (up >= 0).sum() > 0.5 * ev.n


def test_static_links_reject_inputs_beyond_the_fixed_size():
    tpc, L = _bind()
    ev = tpcgen.one_sector(seed=1, with_truth=False)
    params = tpc.tpc_params_default()
    geom = tpc.abi.make_geometry(ev.row_x, 1, ev.z_max, False)
    cl = tpc.abi.TpcClusters(262145, 1, 1, 1, 1)     # never dereferenced: rejected on the host
    rc = L.tpc_links_static(C.byref(params), C.byref(geom), 2.58, C.byref(cl), 1, 1, None, None)
    assert rc == tpc.TPC_ERR_CAPACITY
