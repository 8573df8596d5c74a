"""Parity of the CUDA rANS coder of the cluster compression
(tpc_rans_encode, through the C ABI) with the oracle's coder
(oracle/tpc_oracle_compress.c): the normalised table and every chunk's
bytes identical, on symbol streams of several distributions, ragged chunk
counts and the byte symbols of the oracle's compressed-format fields of a
generator frame; the empty stream codes nothing."""
import numpy as np
import pytest

import tpcgen

pytestmark = pytest.mark.gpu


def _gpu(sym, chunk):
    import torch

    import paper_1905_05515_b300 as tpc
    t = torch.from_numpy(np.ascontiguousarray(sym, np.uint8)).cuda()
    r = tpc.rans_encode(t, chunk)
    torch.cuda.synchronize()
    return (r.freq.cpu().numpy().view(np.uint32), r.chunk_bytes.cpu().numpy(), r.data.cpu().numpy())


def _check(orc, sym, chunk):
    freq, cb, data = _gpu(sym, chunk)
    if sym.size == 0:
        assert (freq == 0).all() and cb.size == 0 and data.size == 0
        return 0
    f_o = orc.rans_normalise(np.bincount(sym, minlength=256))
    np.testing.assert_array_equal(freq, f_o)
    nch = (sym.size + chunk - 1) // chunk
    assert cb.size == nch and int(cb.sum()) == data.size
    o = 0
    for c in range(nch):
        exp = orc.rans_encode(sym[c * chunk:(c + 1) * chunk], f_o)
        assert cb[c] == exp.size, c
        np.testing.assert_array_equal(data[o:o + cb[c]], exp)
        o += cb[c]
    return data.size


@pytest.mark.parametrize("kind, n, chunk", [("uniform4", 100_000, 4096), ("geometric", 77_777, 4096),
                                            ("single", 5000, 1000), ("bytes", 123_457, 8192),
                                            ("skewed", 300_001, 4096), ("bytes", 1, 4096), ("geometric", 4096, 4096),
                                            ("uniform4", 4097, 4096)])
def test_coder_matches_oracle(orc, kind, n, chunk):
    rng = np.random.default_rng(n)
    sym = {"uniform4": lambda: rng.integers(0, 4, n),
           "geometric": lambda: np.minimum(rng.geometric(0.3, n) - 1, 255),
           "single": lambda: np.full(n, 7),
           "bytes": lambda: rng.integers(0, 256, n),
           "skewed": lambda: np.where(rng.random(n) < 0.999, 0, rng.integers(1, 256, n))}[kind]().astype(np.uint8)
    _check(orc, sym, chunk)


def test_empty_stream(orc):
    _check(orc, np.zeros(0, np.uint8), 4096)


def _symbols(v):
    """Byte symbols of an integer stream (values >= 252 become escape
    symbols 251 + bytes of v - 252)."""
    v = np.asarray(v, np.int64)
    w = v - 252
    k = np.where(w < 1 << 8, 1, np.where(w < 1 << 16, 2, np.where(w < 1 << 24, 3, 4)))
    return np.where(v < 252, v, 251 + k).astype(np.uint8)


def test_format_fields_of_a_frame(orc):
    ev = tpcgen.time_frame(seed=3, n_collisions=3, with_truth=False)
    r = orc.track_event(ev)
    f = orc.compress_fields(ev.sector, ev.row, ev.y, ev.zt, r)
    coded = 0
    for name, v in f.items():
        coded += _check(orc, _symbols(v), 4096)
    assert coded > 0


# ---------------------------------------------------------------------------
# the whole format on the GPU (tpc_compress_fields / tpc_compress_frame)
# against the oracle's fields and containers, on the same tracks
# ---------------------------------------------------------------------------
def _dev(a, dt):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dt)).cuda()


def _format_check(orc, sector, row, y, zt, off, clus, assign, n_sectors, n_rows, chunk=4096, ey=5, et=6):
    import types

    import paper_1905_05515_b300 as tpc
    args = (_dev(sector, np.uint8), _dev(row, np.uint8), _dev(y, np.float32), _dev(zt, np.float32),
            _dev(off, np.int32), _dev(clus if len(clus) else np.zeros(0), np.int32), _dev(assign, np.int32))
    r = types.SimpleNamespace(n_tracks=len(off) - 1, tr_off=np.asarray(off, np.int32),
                              tr_clus=np.asarray(clus, np.int32), assign=np.asarray(assign, np.int32))
    exp = orc.compress_fields(sector, row, y, zt, r, n_sectors=n_sectors, n_rows=n_rows, ey=ey, et=et)
    got = tpc.compress_fields(*args, n_sectors=n_sectors, n_rows=n_rows, ey=ey, et=et)
    for name in exp:
        np.testing.assert_array_equal(got[name].cpu().numpy().view(np.uint32), exp[name], err_msg=name)
    data, sizes = tpc.compress_frame(*args, n_sectors=n_sectors, n_rows=n_rows, ey=ey, et=et, chunk=chunk)
    conts = [orc.pack_stream(exp[name], chunk) for name in exp]
    assert sizes == [c.size for c in conts]
    np.testing.assert_array_equal(data.cpu().numpy(), np.concatenate(conts))
    return data.numel()


@pytest.mark.parametrize("make", [lambda: tpcgen.time_frame(seed=3, n_collisions=3, with_truth=False),
                                  lambda: tpcgen.one_sector(seed=1, with_truth=False)])
def test_format_matches_oracle(orc, make):
    """Fields and containers of a frame byte-identical to the oracle's, with
    the oracle's own tracks as the tracks of both sides."""
    ev = make()
    r = orc.track_event(ev)
    nb = _format_check(orc, ev.sector, ev.row, ev.y, ev.zt, r.tr_off, r.tr_clus, r.assign, ev.n_sectors,
                       ev.row_x.size)
    assert nb < 10 * ev.n                  # smaller than the float clusters


def test_format_edge_cases(orc):
    """No tracks; one crowded plane of other clusters (more than the shared
    memory holds); tracks with sector changes, same-row neighbours and
    escapes; empty streams; several chunk sizes."""
    rng = np.random.default_rng(11)
    # a crowded plane and nothing attached
    n = 5000
    sec = np.full(n, 3, np.uint8)
    row = np.full(n, 17, np.uint8)
    y = rng.uniform(-20, 20, n).astype(np.float32)
    zt = rng.uniform(0, 1000, n).astype(np.float32)
    zt[:50] = zt[50]                       # ties in qt: qy and the index decide
    _format_check(orc, sec, row, y, zt, [0], [], np.full(n, -1), 36, 152, chunk=1000)
    # hand-made tracks over a random frame
    n = 3000
    sec = rng.integers(0, 36, n).astype(np.uint8)
    row = rng.integers(0, 152, n).astype(np.uint8)
    y = rng.uniform(-40, 40, n).astype(np.float32)
    zt = rng.uniform(0, 2000, n).astype(np.float32)
    perm = rng.permutation(n)[:2000]
    lens = [0, 1, 2, 5, 150, 300, 0, 40]
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int32)
    clus = perm[:off[-1]].astype(np.int32)
    # runs with same-row neighbours inside a sector
    a = off[4]
    sec[clus[a:a + 150]] = 7
    row[clus[a:a + 150]] = np.repeat(np.arange(75), 2)
    assign = np.full(n, -1, np.int32)
    for t in range(len(lens)):
        assign[clus[off[t]:off[t + 1]]] = t
    y[clus[off[5]:off[5] + 10]] = 3000.0   # large residuals: escapes
    for chunk in (1, 64, 4096):
        _format_check(orc, sec, row, y, zt, off, clus, assign, 36, 152, chunk=chunk)
    # other quantisation steps
    _format_check(orc, sec, row, y, zt, off, clus, assign, 36, 152, ey=3, et=8)
    # no clusters at all
    _format_check(orc, np.zeros(0), np.zeros(0), np.zeros(0), np.zeros(0), [0], [], np.zeros(0), 36, 152)


def test_format_full_frame(orc):
    """The 50-collision frame (16 M clusters) with track lists made from the
    generator's labels (each particle's clusters by row, noise unattached):
    fields and containers byte-identical to the oracle's at full size."""
    ev = tpcgen.time_frame(seed=3, n_collisions=50, with_truth=False)
    lab = ev.label.astype(np.int64)
    idx = np.nonzero(lab >= 0)[0]
    o = np.lexsort((idx, ev.row[idx], lab[idx]))
    clus = idx[o].astype(np.int32)
    labs = lab[clus]
    starts = np.concatenate([[0], np.nonzero(np.diff(labs))[0] + 1, [clus.size]]).astype(np.int32)
    assign = np.full(ev.n, -1, np.int32)
    assign[clus] = np.repeat(np.arange(starts.size - 1, dtype=np.int32), np.diff(starts))
    nb = _format_check(orc, ev.sector, ev.row, ev.y, ev.zt, starts, clus, assign, 36, 152)
    assert nb < 2.5 * ev.n
