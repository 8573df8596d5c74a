"""CPU-side checks of the C ABI library: it builds for sm_103a, loads, and
exports every function include/*.h declares; host-only entry points
validate their arguments (no GPU needed for these)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"#define[^\n]*", "", src)
        names |= set(re.findall(r"\b(tpc_\w+)\s*\(", src))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    import paper_1905_05515_b300 as tpc
    L = tpc.lib()
    names = _declared()
    assert "tpc_track" in names and "tpc_calib_backward" in names
    for nm in names:
        assert hasattr(L, nm), nm
    assert set(tpc.abi.EXPORTED) == set(names)


def test_params_and_workspace_size_host_only():
    import paper_1905_05515_b300 as tpc
    import tpcgen
    p = tpc.tpc_params_default()
    assert p.dy_link == 3.0 and p.refit_passes == 3
    g = tpc.abi.make_geometry(tpcgen.row_x_f32(), 36, 250.0, True)
    small = tpc.tpc_workspace_size(p, g, 1000)
    big = tpc.tpc_workspace_size(p, g, 16_000_000)
    assert 0 < small < big < 8 * 2**30
    with pytest.raises(tpc.TpcError):
        tpc.tpc_workspace_size(p, tpc.abi.make_geometry(np.array([1, 2], np.float32), 36, 250.0, False), 10)
    with pytest.raises(tpc.TpcError):
        tpc.tpc_workspace_size(p, tpc.abi.make_geometry(tpcgen.row_x_f32(), 5, 250.0, False), 10)
    bad = tpc.tpc_params_default(z_cell=0.2)       # cell below the 0.25 cm minimum
    with pytest.raises(tpc.TpcError):
        tpc.tpc_workspace_size(bad, g, 10)
    assert tpc.tpc_error_string(tpc.TPC_ERR_DATA).startswith("invalid cluster")


def test_track_rejects_null_arguments_without_touching_the_gpu():
    import paper_1905_05515_b300 as tpc
    import tpcgen
    L = tpc.lib()
    p = tpc.tpc_params_default()
    g = tpc.abi.make_geometry(tpcgen.row_x_f32(), 36, 250.0, False)
    rc = L.tpc_track(C.byref(p), C.byref(g), 0.5, 2.58, None, None, 0, None, None)
    assert rc == tpc.TPC_ERR_ARG


def test_calib_entry_points_validate_arguments_without_the_gpu():
    import paper_1905_05515_b300 as tpc
    import tpcgen
    L = tpc.lib()
    g = tpc.abi.make_geometry(tpcgen.row_x_f32(), 36, 250.0, True)
    b = C.c_size_t(0)
    assert L.tpc_calib_workspace_size(C.byref(g), 100, 15000, C.byref(b)) == tpc.TPC_OK
    # header, 48-byte reference checkpoints (one per 16 clusters plus one per track), 32 bytes per
    # track (final deviation), the track order (4 bytes per track, 16-byte padded)
    assert b.value == 256 + (15000 // 16 + 100 + 1) * 48 + 100 * 32 + (100 + 3) // 4 * 16
    assert L.tpc_calib_workspace_size(C.byref(g), -1, 10, C.byref(b)) == tpc.TPC_ERR_ARG
    p = tpc.tpc_params_default()
    tr = tpc.abi.TpcCalibTracks()
    tr.n_tracks = 0
    theta = (C.c_float * tpc.abi.calib_n_theta(36))()
    gz = tpc.abi.make_geometry(tpcgen.row_x_f32(), 36, 250.0, False)     # no drift times
    rc = L.tpc_calib_forward(C.byref(p), C.byref(gz), 0.5, 2.58, 0.01, C.byref(tr), C.cast(theta, C.c_void_p),
                             None, None, None, 0, None)
    assert rc == tpc.TPC_ERR_ARG
    rc = L.tpc_calib_forward(C.byref(p), C.byref(g), 0.5, 2.58, 0.0, C.byref(tr), C.cast(theta, C.c_void_p),
                             None, None, None, 0, None)
    assert rc == tpc.TPC_ERR_ARG                                           # vertex variance must be > 0
    tr.n_tracks = 5                                                        # null track arrays
    rc = L.tpc_calib_forward(C.byref(p), C.byref(g), 0.5, 2.58, 0.01, C.byref(tr), C.cast(theta, C.c_void_p),
                             None, None, None, 0, None)
    assert rc == tpc.TPC_ERR_ARG


def test_grid_parameter_limits_and_packed_workspace():
    import paper_1905_05515_b300 as tpc
    import tpcgen
    g = tpc.abi.make_geometry(tpcgen.row_x_f32(), 36, 250.0, True)
    d = tpc.tpc_params_default()
    assert d.tube_radius == np.float32(1.5) and d.pt_min_physics == np.float32(0.05)
    for bad in (dict(z_cell=0.1), dict(y_bins=0), dict(y_bins=65), dict(merge_pairs_per_1k=-1),
                dict(tube_radius=-0.5), dict(tube_radius=25.0), dict(tube_radius=float("nan")),
                dict(pt_min_physics=-1.0), dict(pt_min_physics=float("inf"))):
        with pytest.raises(tpc.TpcError):
            tpc.tpc_workspace_size(tpc.tpc_params_default(**bad), g, 1000)
    # any cell size at or above 0.25 cm works: searches visit the cells a window overlaps
    assert tpc.tpc_workspace_size(tpc.tpc_params_default(z_cell=1.0, y_bins=32), g, 1000) > 0
    plain = tpc.tpc_workspace_size(tpc.tpc_params_default(z_cell=3.5), g, 1000)
    packed = tpc.tpc_workspace_size(tpc.tpc_params_default(packed_links=1, z_cell=3.5), g, 1000)
    assert packed >= plain + 4 * 1000          # the 4-byte packed words


def test_rans_sizes_host_only():
    """The entropy coder's size queries (no device needed): the worst case is
    4 bytes per chunk plus 2 per symbol, the workspace grows with the stream,
    and out-of-range sizes are rejected."""
    import ctypes as C

    import paper_1905_05515_b300 as tpc
    L = tpc.lib()
    mb = C.c_int64(0)
    assert L.tpc_rans_max_bytes(10000, 4096, C.byref(mb)) == 0 and mb.value == 4 * 3 + 2 * 10000
    assert L.tpc_rans_max_bytes(0, 4096, C.byref(mb)) == 0 and mb.value == 0
    ws_small, ws_big = C.c_size_t(0), C.c_size_t(0)
    assert L.tpc_rans_workspace_size(1000, 4096, C.byref(ws_small)) == 0
    assert L.tpc_rans_workspace_size(10_000_000, 4096, C.byref(ws_big)) == 0
    assert 0 < ws_small.value < ws_big.value
    for n, chunk in ((-1, 4096), (1 << 31, 4096), (1000, 0), (1000, 65537)):
        assert L.tpc_rans_workspace_size(n, chunk, C.byref(ws_small)) == tpc.TPC_ERR_ARG
        assert L.tpc_rans_max_bytes(n, chunk, C.byref(mb)) == tpc.TPC_ERR_ARG
    # the binding refuses host tensors before any device work
    import torch
    with pytest.raises(ValueError):
        tpc.rans_encode(torch.zeros(10, dtype=torch.uint8))


def test_calib_select_rejects_bad_arguments_without_touching_the_gpu():
    import paper_1905_05515_b300 as tpc
    L = tpc.lib()
    assert L.tpc_calib_select(-1, None, None, None, 5.0, None, None) == tpc.TPC_ERR_ARG
    assert L.tpc_calib_select(3, None, None, None, 5.0, None, None) == tpc.TPC_ERR_ARG
    assert L.tpc_calib_select(3, 8, 8, 8, float("nan"), 8, None) == tpc.TPC_ERR_ARG
    assert L.tpc_calib_select(0, None, None, None, 5.0, None, None) == tpc.TPC_OK


def test_compress_entry_points_check_their_arguments():
    """Sizes and argument checks of the compressed-format calls, host only."""
    import paper_1905_05515_b300 as tpc
    L = tpc.lib()
    A = tpc.abi

    def cin(n=1000, T=10, na=500, ns=36, nr=152, ptr=1):
        p = C.c_void_p(ptr if ptr else None)
        return A.TpcCompressIn(n, ns, nr, p, p, p, p, T, na, p, p, p)

    ws, mv, mb = C.c_size_t(0), C.c_int64(0), C.c_int64(0)
    assert L.tpc_compress_workspace_size(C.byref(cin()), 4096, C.byref(ws)) == 0
    assert L.tpc_compress_max_size(C.byref(cin()), 4096, C.byref(mv), C.byref(mb)) == 0
    # worst-case stream values: NT, HS (tracks), 7 streams of attached clusters, UN (planes), UT, UY
    assert mv.value == 2 * 10 + 7 * 500 + 36 * 152 + 2 * 1000
    assert mb.value >= 12 * 524 and ws.value > 16 * 1000
    ws2 = C.c_size_t(0)
    L.tpc_compress_workspace_size(C.byref(cin(n=2000)), 4096, C.byref(ws2))
    assert ws2.value > ws.value
    for bad in (cin(n=-1), cin(T=-1), cin(ns=0), cin(nr=256), cin(ptr=0)):
        assert L.tpc_compress_workspace_size(C.byref(bad), 4096, C.byref(ws)) == A.TPC_ERR_ARG
    assert L.tpc_compress_workspace_size(C.byref(cin()), 0, C.byref(ws)) == A.TPC_ERR_ARG
    assert L.tpc_compress_workspace_size(C.byref(cin()), 65537, C.byref(ws)) == A.TPC_ERR_ARG
    counts = (C.c_int64 * 12)()
    # a null workspace, output or vals buffer is refused before any device work
    assert L.tpc_compress_fields(C.byref(cin()), 5, 6, None, 0, None, 0, counts, None) == A.TPC_ERR_ARG
    assert L.tpc_compress_frame(C.byref(cin()), 5, 6, 4096, None, 0, None, 0, counts, None) == A.TPC_ERR_ARG
    assert L.tpc_compress_frame(C.byref(cin()), 5, 99, 4096, C.c_void_p(1), 1 << 40, C.c_void_p(1), 1 << 40,
                                counts, None) == A.TPC_ERR_ARG


def test_calib_fit_checks_its_arguments():
    """Defaults, workspace size and argument checks of the closed-loop fit, host only."""
    import paper_1905_05515_b300 as tpc
    import tpcgen
    L = tpc.lib()
    A = tpc.abi
    o = A.TpcCalibFitOpts()
    assert L.tpc_calib_fit_defaults(C.byref(o)) == 0
    assert o.prior_sigma == pytest.approx(0.3) and o.rounds == 2 and o.max_iter == 300
    g = A.make_geometry(tpcgen.row_x_f32(), 36, 250.0, True)
    s1, s2, s0 = C.c_size_t(0), C.c_size_t(0), C.c_size_t(0)
    assert L.tpc_calib_fit_workspace_size(C.byref(g), 1000, 150_000, C.byref(s1)) == 0
    assert L.tpc_calib_fit_workspace_size(C.byref(g), 2000, 300_000, C.byref(s2)) == 0
    L.tpc_calib_workspace_size(C.byref(g), 1000, 150_000, C.byref(s0))
    assert s0.value < s1.value < s2.value
    p = tpc.tpc_params_default()
    tr = A.TpcCalibTracks()
    tr.n_tracks = 0
    th = C.c_void_p(1)
    rep = A.TpcCalibFitReport()
    bad = A.TpcCalibFitOpts()
    L.tpc_calib_fit_defaults(C.byref(bad))
    bad.prior_sigma = 0.0
    assert L.tpc_calib_fit(C.byref(p), C.byref(g), 0.5, 2.58, 0.01, C.byref(tr), C.byref(bad), th, None, 0, None,
                           None, C.byref(rep), None) == A.TPC_ERR_ARG
    # a dip-angle array needs a positive variance
    tr.tgl_ext = C.c_void_p(1)
    tr.tgl_var = 0.0
    assert L.tpc_calib_fit(C.byref(p), C.byref(g), 0.5, 2.58, 0.01, C.byref(tr), C.byref(o), th, None, 0, None,
                           None, C.byref(rep), None) == A.TPC_ERR_ARG
    tr.tgl_var = 9e-8
    # no workspace: capacity error, before any device work
    assert L.tpc_calib_fit(C.byref(p), C.byref(g), 0.5, 2.58, 0.01, C.byref(tr), C.byref(o), th, None, 0, None,
                           None, C.byref(rep), None) == A.TPC_ERR_CAPACITY
