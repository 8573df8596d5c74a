"""Pins of the oracle's seeding steps (time -> z, NeighboursFinder,
NeighboursCleaner, StartHitsFinder) against an O(N^2) brute force that
emulates every binary32 operation exactly (numpy float32 for + - * /,
rational arithmetic for the fused multiply-add), and against hand-built cases
whose answers follow from the stated reading of the method."""
import json
import os

import numpy as np
import pytest

from helpers import fma32

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "links_3row.json")
F = np.float32
DY, DZ, SMAX = F(3.0), F(3.0), F(0.5)


def brute_links(sector, row, y, z, row_x):
    """Exhaustive (up, down) search over every pair of clusters on the
    neighbouring rows of the same sector."""
    n = y.size
    nr = row_x.size
    up = np.full(n, -1, np.int32)
    dn = np.full(n, -1, np.int32)
    for h in range(n):
        r = int(row[h])
        if r < 1 or r > nr - 2:
            continue
        qu = F(row_x[r + 1]) / F(row_x[r])
        qd = F(row_x[r - 1]) / F(row_x[r])
        w = (F(row_x[r]) - F(row_x[r - 1])) / (F(row_x[r + 1]) - F(row_x[r - 1]))
        ypu, ypd = F(y[h]) * qu, F(y[h]) * qd
        U = [c for c in range(n) if sector[c] == sector[h] and row[c] == r + 1
             and abs(F(y[c]) - ypu) <= DY and abs(F(z[c]) - F(z[h])) <= DZ]
        D = [c for c in range(n) if sector[c] == sector[h] and row[c] == r - 1
             and abs(F(y[c]) - ypd) <= DY and abs(F(z[c]) - F(z[h])) <= DZ]
        best = None
        for u in U:
            for d in D:
                ey = fma32(F(y[u]) - F(y[d]), w, y[d]) - F(y[h])
                ez = fma32(F(z[u]) - F(z[d]), w, z[d]) - F(z[h])
                sc = fma32(ey, ey, F(ez) * F(ez))
                if not sc < SMAX:
                    continue
                key = (float(sc), u, d)
                if best is None or key < best:
                    best = key
        if best is not None:
            up[h], dn[h] = best[1], best[2]
    return up, dn


def _tiny_event(rng, n_rows=6, per_row=25, n_sectors=2, spread=2.5):
    row_x = (100.0 + np.arange(n_rows) * 1.0733).astype(np.float32)
    sector, row, y, z = [], [], [], []
    for s in range(n_sectors):
        for r in range(n_rows):
            k = rng.integers(per_row // 2, per_row + 1)
            sector += [s] * k
            row += [r] * k
            y += list(rng.uniform(-spread, spread, k))
            z += list(rng.uniform(-spread, spread, k))
    # a few exact duplicates to exercise the tie-breaks
    sector += sector[:5]
    row += row[:5]
    y += y[:5]
    z += z[:5]
    perm = rng.permutation(len(y))
    return (np.array(sector, np.uint8)[perm], np.array(row, np.uint8)[perm],
            np.array(y, np.float32)[perm], np.array(z, np.float32)[perm], row_x)


@pytest.mark.parametrize("seed", range(6))
def test_neighbours_finder_equals_brute_force(orc, seed):
    rng = np.random.default_rng(100 + seed)
    sector, row, y, z, row_x = _tiny_event(rng)
    r = orc.track(sector, row, y, z, row_x, n_sectors=36)
    up, dn = brute_links(sector, row, y, z, row_x)
    assert (up >= 0).sum() > 20
    np.testing.assert_array_equal(r.up_raw, up)
    np.testing.assert_array_equal(r.dn_raw, dn)


def test_time_to_z_and_links_in_continuous_mode(orc):
    """Continuous read-out: z = s (Zmax - v t) in binary32 (v t first), s = -1
    on the C side; links are then found on the converted z."""
    rng = np.random.default_rng(7)
    sector, row, y, z, row_x = _tiny_event(rng, n_sectors=2)
    sector = np.where(sector == 1, 20, 3).astype(np.uint8)      # one A-side, one C-side sector
    v = F(2.58)
    t = rng.uniform(0, 100, y.size).astype(np.float32)
    r = orc.track(sector, row, y, t, row_x, n_sectors=36, continuous=True, v_drift=float(v))
    zl = F(250.0) - v * t
    zexp = np.where(sector >= 18, -zl, zl).astype(np.float32)
    np.testing.assert_array_equal(r.z, zexp)
    up, dn = brute_links(sector, row, y, zexp, row_x)
    np.testing.assert_array_equal(r.up_raw, up)
    np.testing.assert_array_equal(r.dn_raw, dn)


def test_golden_hand_built_cases(orc):
    g = json.load(open(GOLDEN))
    row_x = np.array(g["row_x"], np.float32)
    for case in g["cases"]:
        cl = np.array(case["clusters"], np.float64)
        row = cl[:, 0].astype(np.uint8)
        r = orc.track(np.zeros(row.size, np.uint8), row, cl[:, 1].astype(np.float32),
                      cl[:, 2].astype(np.float32), row_x, n_sectors=1)
        for h, u in case["expect_up"].items():
            assert r.up_raw[int(h)] == u, case["name"]
        for h, d in case["expect_dn"].items():
            assert r.dn_raw[int(h)] == d, case["name"]


def test_cleaner_and_start_hits_rules(orc):
    rng = np.random.default_rng(9)
    sector, row, y, z, row_x = _tiny_event(rng, n_rows=8, per_row=12, spread=1.5)
    r = orc.track(sector, row, y, z, row_x, n_sectors=36)
    n = y.size
    for h in range(n):
        u, d = r.up_raw[h], r.dn_raw[h]
        assert r.up[h] == (u if u >= 0 and r.dn_raw[u] == h else -1)
        assert r.dn[h] == (d if d >= 0 and r.up_raw[d] == h else -1)
        s = r.up[h] >= 0 and r.dn[h] < 0 and r.up[r.up[h]] >= 0
        assert bool(r.is_start[h]) == s
    # cleaned links are mutual and adjacent-row
    for h in range(n):
        if r.up[h] >= 0:
            assert r.dn[r.up[h]] == h and row[r.up[h]] == row[h] + 1


def test_straight_track_gives_one_chain_and_one_start(orc):
    """Ten noise-free points of a line through the origin: rows 1..8 chain up
    (edge rows never act as middle hits, so their links are cleaned away) and
    the only start is the row-1 hit."""
    row_x = (100.0 + np.arange(10) * 1.0733).astype(np.float32)
    y = (row_x * np.float32(0.1)).astype(np.float32)
    z = (row_x * np.float32(-0.3)).astype(np.float32)
    row = np.arange(10, dtype=np.uint8)
    r = orc.track(np.zeros(10, np.uint8), row, y, z, row_x, n_sectors=1)
    assert list(r.up) == [-1, 2, 3, 4, 5, 6, 7, 8, -1, -1]
    assert list(r.dn) == [-1, -1, 1, 2, 3, 4, 5, 6, 7, -1]
    assert list(np.where(r.is_start)[0]) == [1]
    # the tracklet constructor then extends to both edge rows
    assert list(r.tracklet_hits(0)) == list(range(10))


def test_empty_and_degenerate_inputs(orc):
    row_x = (100.0 + np.arange(5)).astype(np.float32)
    e = np.zeros(0)
    r = orc.track(e.astype(np.uint8), e.astype(np.uint8), e.astype(np.float32), e.astype(np.float32), row_x)
    assert r.n_tracks == 0 and r.up.size == 0
    # a single cluster, and all clusters on one row
    r = orc.track(np.zeros(1, np.uint8), np.ones(1, np.uint8), np.zeros(1, np.float32),
                  np.zeros(1, np.float32), row_x)
    assert r.up_raw[0] == -1 and r.n_tracks == 0
    r = orc.track(np.zeros(50, np.uint8), np.full(50, 2, np.uint8), np.zeros(50, np.float32),
                  np.linspace(-1, 1, 50).astype(np.float32), row_x)
    assert (r.up_raw == -1).all() and r.n_tracks == 0
    with pytest.raises(ValueError):
        orc.track(np.full(1, 40, np.uint8), np.zeros(1, np.uint8), np.zeros(1, np.float32),
                  np.zeros(1, np.float32), row_x)


def _q256(v):
    """Nearest multiple of 2^-8 (ties to even), computed exactly with
    Python's rational arithmetic: the decoded 16-bit packed coordinate."""
    from fractions import Fraction
    out = np.empty(v.size, np.float32)
    for i, x in enumerate(np.asarray(v, np.float32)):
        out[i] = F(float(round(Fraction(float(x)) * 256) / 256))
    return out


@pytest.mark.parametrize("seed", range(3))
def test_packed_link_pass_equals_brute_force_on_rounded_coordinates(orc, seed):
    """Packed-coordinate variant: the link pass sees y, z rounded to 1/256 cm;
    the links equal an exhaustive search on the rounded values, and the
    tracker's other stages still see the full-precision clusters (z output
    unchanged)."""
    rng = np.random.default_rng(300 + seed)
    sector, row, y, z, row_x = _tiny_event(rng, spread=1.2)
    # coordinates on a 1/512 grid put many values exactly half-way between
    # two 1/256 steps: the ties-to-even rounding is exercised
    y = (np.round(y * 512) / 512).astype(np.float32)
    z = (np.round(z * 512) / 512).astype(np.float32)
    r = orc.track(sector, row, y, z, row_x, n_sectors=36, params={"packed_links": 1})
    up, dn = brute_links(sector, row, _q256(y), _q256(z), row_x)
    assert (up >= 0).sum() > 20
    np.testing.assert_array_equal(r.up_raw, up)
    np.testing.assert_array_equal(r.dn_raw, dn)
    np.testing.assert_array_equal(r.z, z)
    r0 = orc.track(sector, row, y, z, row_x, n_sectors=36)
    assert not np.array_equal(r.up_raw, r0.up_raw) or not np.array_equal(r.dn_raw, r0.dn_raw)


def test_packed_links_change_few_links_on_a_frame(orc):
    """On a continuous frame the rounding to 1/256 cm changes few links."""
    import tpcgen
    ev = tpcgen.time_frame(seed=31, n_collisions=1, mult_mean=800.0, with_truth=False)
    a = orc.track_event(ev)
    b = orc.track_event(ev, params={"packed_links": 1})
    diff = np.mean((a.up != b.up) | (a.dn != b.dn))
    assert diff < 2e-3
