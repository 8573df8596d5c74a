"""Pins of the oracle's cluster compression (tpc_oracle_compress.c) against
facts outside it: exact round trips (the coder alone and the whole format),
the coded size against the entropy of the coder's own tables (rANS codes a
symbol of frequency f out of 4096 in log2(4096 / f) bits up to a few bytes
per chunk), the quantisation error bound, zero residuals for tracks whose
integer positions lie on a line in row, and the invariants of the table
normalisation.

Paper, section "TPC Data Compression": an integer cluster format at the
intrinsic resolution, residuals to the tracks for attached clusters and
position differences otherwise, then a standard entropy coder (ANS).
"""
import types

import numpy as np
import pytest

import oracle
import tpcgen


def _entropy_bytes(sym, freq):
    return float(-np.log2(freq[sym].astype(np.float64) / 4096.0).sum() / 8.0)


@pytest.mark.parametrize("kind", ["uniform4", "geometric", "single", "bytes", "skewed"])
def test_rans_round_trip_and_size(kind):
    rng = np.random.default_rng(11)
    n = 20000
    sym = {"uniform4": lambda: rng.integers(0, 4, n),
           "geometric": lambda: np.minimum(rng.geometric(0.3, n) - 1, 255),
           "single": lambda: np.full(n, 7),
           "bytes": lambda: rng.integers(0, 256, n),
           "skewed": lambda: np.where(rng.random(n) < 0.999, 0, rng.integers(1, 256, n))}[kind]().astype(np.uint8)
    freq = oracle.rans_normalise(np.bincount(sym, minlength=256))
    data = oracle.rans_encode(sym, freq)
    assert np.array_equal(oracle.rans_decode(data, freq, n), sym)
    h = _entropy_bytes(sym, freq)
    assert h - 1.0 <= data.size <= h + 6.0, (kind, data.size, h)
    # a corrupted stream does not decode to the same symbols
    if data.size > 8:
        bad = data.copy()
        bad[data.size // 2] ^= 0x5A
        try:
            back = oracle.rans_decode(bad, freq, n)
            assert not np.array_equal(back, sym)
        except ValueError:
            pass


def test_table_normalisation():
    rng = np.random.default_rng(3)
    for _ in range(50):
        k = int(rng.integers(1, 257))
        h = np.zeros(256, np.int64)
        h[rng.choice(256, k, replace=False)] = rng.integers(1, 10000, k)
        f = oracle.rans_normalise(h).astype(np.int64)
        assert f.sum() == 4096
        assert ((f > 0) == (h > 0)).all()
        exact = 4096.0 * h / h.sum()
        if (exact[h > 0] >= 1.0).all():          # no symbol lifted to 1: largest remainders, within 1
            assert np.abs(f - exact)[h > 0].max() < 1.0
        else:                                    # the lifted units come from the largest frequencies
            lifted = int(((exact < 1.0) & (h > 0)).sum())
            assert np.abs(f - exact)[h > 0].max() <= 1.0 + lifted
    # one dominant symbol and 255 rare ones: every rare one keeps frequency 1
    h = np.ones(256, np.int64)
    h[0] = 10 ** 7
    f = oracle.rans_normalise(h)
    assert f[0] == 4096 - 255 and (f[1:] == 1).all()


def _quantised(ev):
    qy = np.rint(ev.y.astype(np.float64) * 32.0).astype(np.int64)
    qt = np.rint(ev.zt.astype(np.float64) * 64.0).astype(np.int64)
    return qy, qt


@pytest.mark.parametrize("make", [lambda: tpcgen.one_sector(seed=1, with_truth=False),
                                  lambda: tpcgen.central_event(seed=2, n_tracks=800, with_truth=False),
                                  lambda: tpcgen.time_frame(seed=3, n_collisions=2, with_truth=False)])
def test_format_round_trip(make):
    ev = make()
    r = oracle.track_event(ev)
    f = oracle.compress_fields(ev.sector, ev.row, ev.y, ev.zt, r, n_sectors=ev.n_sectors, n_rows=ev.row_x.size)
    s, rw, qy, qt = oracle.decompress_fields(f, r.n_tracks, ev.n, n_sectors=ev.n_sectors, n_rows=ev.row_x.size)
    ey, et = _quantised(ev)
    got = np.lexsort((qt, qy, rw, s))
    exp = np.lexsort((et, ey, ev.row, ev.sector))
    assert np.array_equal(s[got], ev.sector[exp]) and np.array_equal(rw[got], ev.row[exp])
    assert np.array_equal(qy[got], ey[exp]) and np.array_equal(qt[got], et[exp])
    # the integer format keeps positions to half a quantum
    assert np.abs(ev.y.astype(np.float64) - ey / 32.0).max() <= 1.0 / 64.0
    assert np.abs(ev.zt.astype(np.float64) - et / 64.0).max() <= 1.0 / 128.0
    # attached clusters come first, in track order
    att = r.tr_clus
    assert np.array_equal(s[:att.size], ev.sector[att]) and np.array_equal(qy[:att.size], ey[att])
    # every stream survives the coder
    for name, v in f.items():
        nb, ok = oracle.code_stream(v, chunk=4096)
        assert ok, name


def test_escapes_round_trip_at_their_edges():
    """Values at every escape boundary (1 to 4 raw bytes) come back exactly."""
    edges = [0, 1, 250, 251, 252, 253, 252 + 255, 252 + 256, 252 + 65535, 252 + 65536, 252 + (1 << 24) - 1,
             252 + (1 << 24), 0xFFFFFFFF]
    v = np.array(edges * 50, np.uint32)
    nb, ok = oracle.code_stream(v, chunk=64)
    assert ok
    raw = sum(0 if e < 252 else (1 if e - 252 < 256 else 2 if e - 252 < 65536 else 3 if e - 252 < 1 << 24 else 4)
              for e in edges) * 50
    assert nb >= raw


def test_line_tracks_have_zero_residuals():
    """Tracks whose quantised positions are linear in the row (integer slope
    per row, rows in steps of 1 and 2): every residual after a run's first
    two clusters is zero; the second cluster's is the slope times its step."""
    rows = np.array([3, 4, 5, 7, 9, 10, 11, 13], np.uint8)
    n_tr = 3
    sec, rw, y, zt = [], [], [], []
    for t in range(n_tr):
        a, b, c, d = 40 + 7 * t, 3 - 2 * t, 5000 + 100 * t, -11 + 3 * t
        sec += [t] * rows.size
        rw += rows.tolist()
        y += ((a + b * rows.astype(np.int64)) / 32.0).tolist()
        zt += ((c + d * rows.astype(np.int64)) / 64.0).tolist()
    n = len(sec)
    r = types.SimpleNamespace(n_tracks=n_tr, tr_off=np.arange(0, n + 1, rows.size, dtype=np.int32),
                              tr_clus=np.arange(n, dtype=np.int32), assign=np.repeat(np.arange(n_tr), rows.size))
    f = oracle.compress_fields(np.array(sec, np.uint8), np.array(rw, np.uint8), np.array(y, np.float32),
                               np.array(zt, np.float32), r, n_sectors=36, n_rows=152)
    ry = f["res_y"].reshape(n_tr, rows.size - 1)
    rt = f["res_t"].reshape(n_tr, rows.size - 1)
    assert (ry[:, 1:] == 0).all() and (rt[:, 1:] == 0).all()
    zz = lambda v: np.where(v >= 0, 2 * v, -2 * v - 1)  # noqa: E731
    assert np.array_equal(ry[:, 0], zz(np.array([3 - 2 * t for t in range(n_tr)])))
    assert np.array_equal(f["d_row"], np.tile(zz(np.diff(rows.astype(np.int64))), n_tr))
    assert (f["d_sector"] == 0).all() and f["head_y"].size == n_tr


def test_residual_streams_cost_less_than_positions():
    """On a generator frame the residuals to the tracks take fewer coded bits
    per cluster than the same clusters' absolute positions would, and the
    whole format compresses the 10-byte float clusters several-fold."""
    ev = tpcgen.time_frame(seed=3, n_collisions=2, with_truth=False)
    r = oracle.track_event(ev)
    f = oracle.compress_fields(ev.sector, ev.row, ev.y, ev.zt, r)
    nres = f["res_y"].size
    bits_res = 8.0 * oracle.code_stream(f["res_y"])[0] / nres
    ey, _ = _quantised(ev)
    zzy = np.where(ey >= 0, 2 * ey, -2 * ey - 1).astype(np.uint32)
    bits_abs = 8.0 * oracle.code_stream(zzy[r.tr_clus])[0] / r.tr_clus.size
    assert bits_res < 0.6 * bits_abs, (bits_res, bits_abs)
    total = sum(oracle.code_stream(v)[0] for v in f.values())
    factor = 10.0 * ev.n / total
    assert factor > 2.5, factor


def test_stream_containers_round_trip():
    """Every field stream of a frame, packed into its container and unpacked,
    comes back exactly; the container is the coded size plus its 12-byte
    header; a truncated container is refused."""
    ev = tpcgen.time_frame(seed=3, n_collisions=2, with_truth=False)
    r = oracle.track_event(ev)
    f = oracle.compress_fields(ev.sector, ev.row, ev.y, ev.zt, r)
    for name, v in f.items():
        data = oracle.pack_stream(v, chunk=1024)
        back = oracle.unpack_stream(data, vcap=max(v.size, 1))
        assert np.array_equal(back, v), name
        nb, _ = oracle.code_stream(v, chunk=1024, roundtrip=False)
        assert data.size == nb + 12, name
        with pytest.raises(ValueError):
            oracle.unpack_stream(data[:-1], vcap=max(v.size, 1))
    empty = oracle.pack_stream(np.zeros(0, np.uint32))
    assert empty.size == 12 + 512 and oracle.unpack_stream(empty).size == 0


def test_container_capacity_from_its_header():
    """Without a given capacity the unpacker sizes its output from the value
    count in the container's header: a stream of 100,000 equal values codes
    into far fewer bytes than values and still comes back."""
    v = np.zeros(100_000, np.uint32)
    data = oracle.pack_stream(v)
    assert data.size < v.size // 50
    assert np.array_equal(oracle.unpack_stream(data), v)
    w = np.concatenate([v, np.arange(300, dtype=np.uint32)])      # with escapes
    assert np.array_equal(oracle.unpack_stream(oracle.pack_stream(w, chunk=1024)), w)


def test_same_row_pair_predicts_the_previous_value():
    """Two consecutive clusters of a run on one row (a looper turning inside a
    sector) give no line to extrapolate: the next residual is taken against
    the previous value, and the format still round-trips."""
    rows = np.array([20, 21, 21, 22, 23], np.uint8)
    qy = np.array([100, 104, 109, 115, 118], np.int64)
    qt = np.array([7000, 6990, 6985, 6970, 6960], np.int64)
    y = (qy / 32.0).astype(np.float32)
    zt = (qt / 64.0).astype(np.float32)
    sec = np.full(rows.size, 4, np.uint8)
    r = types.SimpleNamespace(n_tracks=1, tr_off=np.array([0, rows.size], np.int32),
                              tr_clus=np.arange(rows.size, dtype=np.int32), assign=np.zeros(rows.size, np.int32))
    f = oracle.compress_fields(sec, rows, y, zt, r, n_sectors=36, n_rows=152)
    zz = lambda v: int(2 * v) if v >= 0 else int(-2 * v - 1)  # noqa: E731
    # residuals of clusters 1..4: previous value, line (rows 20, 21 -> 21), previous value (21, 21 share the
    # row), line through (21, 109) and (22, 115)
    line = lambda v0, r0, v1, r1, rr: v1 + ((v1 - v0) * (rr - r1)) // (r1 - r0)  # noqa: E731
    exp_y = [qy[1] - qy[0], qy[2] - line(qy[0], 20, qy[1], 21, 21), qy[3] - qy[2], qy[4] - line(qy[2], 21, qy[3], 22, 23)]
    assert f["res_y"].tolist() == [zz(v) for v in exp_y]
    s, rw, dy, dt = oracle.decompress_fields(f, 1, rows.size, n_sectors=36, n_rows=152)
    assert np.array_equal(rw, rows) and np.array_equal(dy, qy) and np.array_equal(dt, qt)
