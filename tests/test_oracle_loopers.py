"""Pins of the looper-leg identification (oracle/tpc_oracle_loopers.c;
sections "Introduction" and "TPC Data Compression": low-momentum particles
leave several legs, whose secondary legs below 200 MeV/c are removable).

* the file's own binary32 arctangent against the library's atan2 (binary64);
* hand-built exact helices: two points of one helix (one leg reversed into
  the tracker's convention of increasing x, as the tracker fits an inward
  leg) are grouped whatever whole turns separate them; the same helix with
  z shifted by 10 cm, a radius 5 cm larger, or the opposite turning sense
  is not;
* generator truth on a continuous frame: the groups are mostly legs of one
  particle, and the first leg in drift time is leg 0.
"""
import math

import numpy as np
import pytest

import tpcgen

BZ = 0.5
KB = -tpcgen.C_LIGHT * BZ


def test_own_atan2_against_the_library():
    import oracle
    rng = np.random.default_rng(3)
    pts = [(0.0, 1.0), (1.0, 0.0), (0.0, -1.0), (-1.0, 0.0), (1.0, 1.0), (-1.0, -1.0), (1e-30, -1.0), (-1e-30, -1.0)]
    pts += [tuple(v) for v in rng.normal(size=(2000, 2)) * rng.choice([1e-3, 1.0, 1e3], size=(2000, 1))]
    worst = 0.0
    for y, x in pts:
        y32, x32 = float(np.float32(y)), float(np.float32(x))
        worst = max(worst, abs(oracle.atan2_own(y32, x32) - math.atan2(y32, x32)))
    assert worst < 5e-7, worst          # a few binary32 ulps of pi
    assert oracle.atan2_own(0.0, 0.0) == 0.0


def _state(R, xc, yc, omega, psi, z, tgl_abs, sigma_q=1e-3):
    """Tracker state (sector, 21 floats) of the point at angle psi on the
    circle (centre xc, yc, radius R, turning sense omega = +1 counter-
    clockwise), moving along the helix; an inward-moving point is given in
    the tracker's convention (direction of increasing local x: sin(phi),
    q/pT and tan(lambda) change sign)."""
    X, Y = xc + R * math.cos(psi), yc + R * math.sin(psi)
    phi = psi + omega * math.pi / 2            # direction of motion
    a_glob = math.atan2(Y, X) % (2 * math.pi)
    s = int(a_glob // math.radians(20)) % 18
    al = math.radians(s * 20 + 10)
    x = X * math.cos(al) + Y * math.sin(al)
    y = -X * math.sin(al) + Y * math.cos(al)
    ph = phi - al
    k = omega / R                              # d sin(phi)/dx along the motion
    tl = tgl_abs
    if math.cos(ph) < 0:                       # inward: the tracker runs the other way
        ph += math.pi
        k, tl = -k, -tl
    st = np.zeros(21, np.float32)
    st[:6] = [x, y, z, math.sin(ph), tl, k / KB]
    st[6], st[8], st[11], st[15], st[20] = 0.01, 0.0225, 1e-4, 1e-4, sigma_q ** 2
    return s, st


def _group(pairs, qpt_min=5.0):
    import oracle
    sec = np.array([p[0] for p in pairs], np.int32)
    st = np.stack([p[1] for p in pairs]).astype(np.float32)
    g = np.zeros(len(pairs), np.int32)
    lg = np.zeros(len(pairs), np.int32)
    L = oracle.lib()
    P32 = oracle._P32
    rc = L.orc_loopers(36, 250.0, BZ, qpt_min, len(pairs), oracle._ptr(sec, P32), None,
                       oracle._ptr(st, oracle._PF), oracle._ptr(g, P32), oracle._ptr(lg, P32))
    assert rc == 0
    return g, lg


@pytest.mark.parametrize("R, tgl", [(60.0, 0.3), (100.0, 0.1), (120.0, 0.6)])
@pytest.mark.parametrize("omega", [1, -1])
def test_legs_of_one_exact_helix_are_grouped(R, tgl, omega):
    rng = np.random.default_rng(int(R * 10 + omega))
    xc, yc = R * math.cos(0.7), R * math.sin(0.7)     # a circle through the beam line
    n_ok = 0
    for turns in (0, 1, 2):
        psi1 = 0.7 + math.pi + omega * rng.uniform(0.5, 1.0)
        dpsi = math.pi * rng.uniform(0.5, 1.0) + 2 * math.pi * turns
        psi2 = psi1 + omega * dpsi
        z1 = 20.0
        z2 = z1 + tgl * R * dpsi
        if abs(z2) > 240:
            continue
        a = _state(R, xc, yc, omega, psi1, z1, tgl)
        b = _state(R, xc, yc, omega, psi2, z2, tgl)
        g, lg = _group([a, b])
        assert g.tolist() == [0, 0], (turns, g)
        assert sorted(lg.tolist()) == [0, 1]
        assert lg[0] == 0                                # smaller s z: the earlier leg (z grows)
        # not the same particle: z shifted, radius larger, or turning the other way
        for bad in (_state(R, xc, yc, omega, psi2, z2 + 10.0, tgl),
                    _state(R + 5.0, xc, yc, omega, psi2, z2, tgl),
                    _state(R, xc, yc, -omega, psi2, z2, tgl)):
            g2, _ = _group([a, bad])
            assert g2.tolist() == [-1, -1], (turns, g2)
        n_ok += 1
    assert n_ok >= 1 and (n_ok >= 2 or tgl * R > 40)    # steep, wide helices leave the drift volume within a turn


def test_candidates_only_below_the_momentum_limit():
    R = 400.0                                           # |q/pT| = 1/(|kb| R) = 1.67 < 5
    xc, yc = R, 0.0
    a = _state(R, xc, yc, 1, math.pi + 0.2, 10.0, 0.2)
    b = _state(R, xc, yc, 1, math.pi + 0.3, 10.0 + 0.2 * R * 0.1, 0.2)
    g, lg = _group([a, b])
    assert g.tolist() == [-1, -1] and lg.tolist() == [-1, -1]
    g, lg = _group([a, b], qpt_min=1.0)
    assert g.tolist() == [0, 0]


def test_groups_against_generator_truth(orc):
    """Continuous frame with 5 % loopers: >= 90 % of the groups hold the legs
    of one particle (measured 96 %); in those, leg 0 is the leg the particle
    crossed first (>= 90 %, measured 96 %); >= 55 % of the loopers with
    several candidate tracks have all of them in one group (measured 66 %:
    short legs, whose radius is known to worse than 5 cm, are not grouped)."""
    ev = tpcgen.time_frame(seed=4, n_collisions=8)
    r = orc.track_event(ev)
    g, lg = orc.loopers(ev.sector, r)
    T = r.n_tracks
    maj = np.full(T, -1)
    for t in range(T):
        v, k = np.unique(ev.label[r.track_clusters(t)], return_counts=True)
        maj[t] = v[np.argmax(k)]
    groups = {}
    for t in np.nonzero(g >= 0)[0]:
        groups.setdefault(int(g[t]), []).append(int(t))
    assert len(groups) > 200
    assert all(min(m) == k for k, m in groups.items())
    assert all(sorted(lg[m].tolist()) == list(range(len(m))) for m in groups.values())
    pure = [m for m in groups.values() if len(set(maj[m])) == 1]
    assert len(pure) >= 0.9 * len(groups)
    first_ok = 0
    for m in pure:
        first = m[int(np.argmin([ev.true_s[r.track_clusters(t)].min() for t in m]))]
        first_ok += lg[first] == 0
    assert first_ok >= 0.9 * len(pure)
    heads = orc.track_heads(r)
    cand = np.abs(r.trk_bot[heads][:, 5]) >= 5.0
    byp = {}
    for t in np.nonzero(cand)[0]:
        if maj[t] >= 0:
            byp.setdefault(int(maj[t]), []).append(int(t))
    multi = [ts for ts in byp.values() if len(ts) >= 2]
    full = sum(g[ts[0]] >= 0 and len(set(g[ts])) == 1 for ts in multi)
    assert full >= 0.55 * len(multi)
