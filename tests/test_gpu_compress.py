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
