"""Pins of the oracle's track-based cluster attachment (tpc_oracle_attach.c)
against facts outside it: the closed-form helix in binary64, a brute-force
tube search written from that closed form, the flag definitions, and the
special cases R = 0, pt_min = 0 and an unreachable pt_min.

Paper, section "TPC Data Compression": tubes of 1.5 cm around the tracks,
unattached clusters marked adjacent to the highest-pT track whose tube holds
them, protected clusters in the tubes of good tracks, removal of attached or
adjacent clusters that are not protected; tracks below 50 MeV/c not used.
"""
import math

import numpy as np
import pytest

import oracle
import tpcgen

KB_C = -2.99792458e-3
NST = 21


def helix_at(b, x, kb):
    """Closed-form position on the helix of state b = (x0, y, z, sin phi,
    tan lambda, q/pT) at the plane x (binary64): sin phi is linear in x, the
    circle gives y, z grows with the transverse arc."""
    x0, y0, z0, s0, t0, q = (float(v) for v in b[:6])
    k = kb * q
    s = s0 + k * (x - x0)
    if abs(s) >= 1.0:
        return None
    if abs(k) < 1e-12:
        dy = (x - x0) * s0 / math.sqrt(1 - s0 * s0)
        arc = math.hypot(x - x0, dy)
        arc = arc if x >= x0 else -arc
        return y0 + dy, z0 + t0 * arc, s
    dy = (math.sqrt(1 - s0 * s0) - math.sqrt(1 - s * s)) / k
    arc = (math.asin(s) - math.asin(s0)) / k
    return y0 + dy, z0 + t0 * arc, s


def test_step_pos32_follows_the_closed_form_helix():
    rng = np.random.default_rng(7)
    X = tpcgen.row_x_f32()
    kb = np.float32(KB_C * 0.5)
    n_checked = 0
    for _ in range(300):
        r0 = int(rng.integers(0, 120))
        q = rng.choice([-1, 1]) * math.exp(rng.uniform(math.log(0.2), math.log(15.0)))
        b = np.array([X[r0], rng.uniform(-15, 15), rng.uniform(-200, 200), rng.uniform(-0.7, 0.7),
                      rng.uniform(-1.5, 1.5), q], np.float32)
        p = b.copy()
        direction = 1 if rng.random() < 0.5 else -1
        rows = range(r0 + 1, min(r0 + 30, 152)) if direction > 0 else range(r0 - 1, max(r0 - 30, -1), -1)
        for r in rows:
            ok, p2 = oracle.step_pos32(p, X[r], kb)
            ref = helix_at(b, float(X[r]), float(kb))
            if ref is None or abs(ref[2]) > 0.998:
                break
            assert ok
            p = p2
            assert p[0] == X[r]
            assert abs(p[1] - ref[0]) < 2e-3 and abs(p[2] - ref[1]) < 2e-3 and abs(p[3] - ref[2]) < 1e-5, (b, r)
            n_checked += 1
    assert n_checked > 3000


def test_step_pos32_refuses_out_of_range_sin_phi():
    X = tpcgen.row_x_f32()
    kb = np.float32(KB_C * 0.5)
    b = np.array([X[10], 0, 0, 0.9985, 0.1, -5.0], np.float32)   # k = kb q/pT > 0: sin phi grows outward
    ok, p = oracle.step_pos32(b, X[12], kb)
    assert not ok and np.array_equal(p, b)
    ok, p = oracle.step_pos32(b, X[8], kb)          # inward it falls: allowed
    assert ok and p[3] < b[3]


def _segments(ev, r):
    """(sector, r_lo, r_hi, inner-end state, track index) of every segment,
    tracks numbered as the tracker numbers them"""
    seg_track = np.full(r.seg_trk.shape[0], -1)
    t = 0
    for a in range(r.seg_trk.shape[0]):
        if r.seg_prev[a] >= 0:
            continue
        b = a
        while b >= 0:
            seg_track[b] = t
            b = r.seg_next[b]
        t += 1
    head_q = np.zeros(t, np.float32)
    for a in range(r.seg_trk.shape[0]):
        if r.seg_prev[a] < 0:
            head_q[seg_track[a]] = abs(r.trk_bot[r.seg_trk[a], 5])
    out = []
    for a in range(r.seg_trk.shape[0]):
        h = r.tracklet_hits(r.seg_trk[a])
        out.append((int(ev.sector[h[0]]), int(ev.row[h[0]]), int(ev.row[h[-1]]), r.trk_bot[r.seg_trk[a]],
                    int(seg_track[a])))
    return out, head_q


def _brute_force(ev, r, radius, pt_min, margin=2e-3):
    """Per cluster: the tracks whose tube certainly holds it (distance below
    radius - margin, closed-form helix) and whether some track's tube
    boundary passes within margin of it (undecidable at this precision)."""
    X = ev.row_x.astype(np.float64)
    kb = float(np.float32(KB_C * ev.bz))
    segs, head_q = _segments(ev, r)
    pl = ev.sector.astype(np.int64) * len(X) + ev.row
    order = np.argsort(pl, kind="stable")
    bounds = np.searchsorted(pl[order], np.arange(ev.n_sectors * len(X) + 1))
    inside = [set() for _ in range(ev.n)]
    unsure = np.zeros(ev.n, bool)
    edge_seg = 0
    for (s, r_lo, r_hi, b, tr) in segs:
        rb = int(np.nonzero(X.astype(np.float32) == b[0])[0][0])
        traced = []
        for rows in (range(rb, r_hi + 1), range(rb - 1, r_lo - 1, -1)):
            for rr in rows:
                pos = helix_at(b, X[rr], kb)
                if pos is None or abs(pos[2]) >= 0.999 - 1e-4:
                    if pos is not None and abs(pos[2]) < 0.999 + 1e-4:
                        edge_seg += 1            # the binary32 trace may stop either side of this row
                    break
                if r_lo <= rr <= r_hi:
                    traced.append((rr, pos))
        for rr, (yp, zp, _) in traced:
            p = s * len(X) + rr
            idx = order[bounds[p]:bounds[p + 1]]
            d = np.hypot(ev.y[idx].astype(np.float64) - yp, r.z[idx].astype(np.float64) - zp)
            for c in idx[d < radius - margin]:
                inside[c].add(tr)
            unsure[idx[np.abs(d - radius) <= margin]] = True
    return inside, unsure, head_q, edge_seg


@pytest.mark.parametrize("radius", [1.5, 4.0])
def test_tube_and_adjacency_against_brute_force(radius):
    ev = tpcgen.central_event(seed=4, n_tracks=600)
    r = oracle.track_event(ev)
    pt_min = 0.3
    adj, fl = oracle.attach_event(ev, r, radius=radius, pt_min=pt_min)
    inside, unsure, head_q, edge_seg = _brute_force(ev, r, radius, pt_min)
    assert edge_seg <= 2
    qmax = np.float32(1.0) / np.float32(pt_min)
    n_multi = n_adj = n_prot_tube = 0
    for c in range(ev.n):
        if unsure[c]:
            continue
        trs = inside[c]
        att = r.assign[c] >= 0
        if att:
            assert not fl[c] & oracle.CL_ADJACENT and adj[c] == -1
        elif trs:
            best = min(trs, key=lambda t: (head_q[t], t))        # highest pT, then smaller index
            assert fl[c] & oracle.CL_ADJACENT and adj[c] == best, (c, trs, adj[c])
            n_adj += 1
            n_multi += len(trs) > 1
        else:
            assert not fl[c] & oracle.CL_ADJACENT and adj[c] == -1, c
        good_tube = any(head_q[t] <= qmax for t in trs)
        good_att = att and head_q[r.assign[c]] <= qmax
        assert bool(fl[c] & oracle.CL_PROTECTED) == (good_tube or good_att), c
        n_prot_tube += good_tube and not good_att
    assert n_adj > 20 and n_multi > 0 and n_prot_tube > 0
    assert unsure.sum() < 0.01 * ev.n


def test_flags_follow_their_definitions():
    ev = tpcgen.time_frame(seed=9, n_collisions=2, mult_mean=400)
    r = oracle.track_event(ev)
    adj, fl = oracle.attach_event(ev, r, radius=1.5, pt_min=0.25)
    att = (fl & oracle.CL_ATTACHED) > 0
    adjf = (fl & oracle.CL_ADJACENT) > 0
    prot = (fl & oracle.CL_PROTECTED) > 0
    rem = (fl & oracle.CL_REMOVE) > 0
    assert np.array_equal(att, r.assign >= 0)
    assert not (att & adjf).any()
    assert np.array_equal(adj >= 0, adjf)
    assert np.array_equal(rem, (att | adjf) & ~prot)
    assert (fl < 16).all()
    assert rem.sum() > 0 and adjf.sum() > 0 and (prot & ~att).sum() > 0
    # every cluster of a track below the cut that lies in no good tube is removed
    segs, head_q = _segments(ev, r)
    bad = head_q > np.float32(1.0) / np.float32(0.25)
    assert bad.sum() > 0
    on_bad = att & bad[np.maximum(r.assign, 0)]
    assert np.array_equal(rem[on_bad], ~prot[on_bad])


def test_special_cases():
    """Without the looper-leg category (loopers_first=False) the special
    cases of the tube radius and the momentum cut."""
    ev = tpcgen.time_frame(seed=9, n_collisions=2, mult_mean=400)
    r = oracle.track_event(ev)
    att = r.assign >= 0
    # a tube of radius 0 holds nothing: no adjacency, protection only by attachment
    adj, fl = oracle.attach_event(ev, r, radius=0.0, pt_min=0.05, loopers_first=False)
    assert (adj == -1).all() and not (fl & oracle.CL_ADJACENT).any()
    segs, head_q = _segments(ev, r)
    good_att = att & (head_q[np.maximum(r.assign, 0)] <= np.float32(1.0) / np.float32(0.05))
    assert np.array_equal((fl & oracle.CL_PROTECTED) > 0, good_att)
    # pt_min = 0: every track is good, nothing is removed, adjacent clusters are protected
    adj, fl = oracle.attach_event(ev, r, radius=1.5, pt_min=0.0, loopers_first=False)
    assert not (fl & oracle.CL_REMOVE).any()
    assert ((fl & oracle.CL_PROTECTED) > 0)[(fl & (oracle.CL_ATTACHED | oracle.CL_ADJACENT)) > 0].all()
    # an unreachable pt_min: no track is good, every attached or adjacent cluster is removed
    adj, fl = oracle.attach_event(ev, r, radius=1.5, pt_min=1e30, loopers_first=False)
    assert not (fl & oracle.CL_PROTECTED).any()
    assert np.array_equal((fl & oracle.CL_REMOVE) > 0, (fl & (oracle.CL_ATTACHED | oracle.CL_ADJACENT)) > 0)


def test_tubes_catch_the_clusters_tracking_missed():
    """Generator truth: a cluster of a tracked (non-looping) particle that the
    tracking left unattached, on a row inside the span of that particle's
    track in its sector, lies within 1.5 cm of the fitted trajectory and so is
    marked adjacent (to that track or to a higher-pT one crossing it)."""
    for ev in (tpcgen.central_event(seed=4, n_tracks=600), tpcgen.time_frame(seed=9, n_collisions=2, mult_mean=400)):
        r = oracle.track_event(ev)
        adj, fl = oracle.attach_event(ev, r)
        tracks_of = {}
        for t in range(r.n_tracks):
            v, cnt = np.unique(ev.label[r.track_clusters(t)], return_counts=True)
            tracks_of.setdefault(int(v[np.argmax(cnt)]), []).append(t)
        missed = []
        for c in np.nonzero((r.assign < 0) & (ev.label >= 0))[0]:
            if ev.trk_looper[ev.label[c]]:
                continue
            for t in tracks_of.get(int(ev.label[c]), []):
                cl = r.track_clusters(t)
                cl = cl[ev.sector[cl] == ev.sector[c]]
                if cl.size and ev.row[cl].min() <= ev.row[c] <= ev.row[cl].max():
                    missed.append(c)
                    break
        missed = np.array(missed, int)
        assert missed.size >= 5 and (adj[missed] >= 0).mean() >= 0.9, (missed.size, (adj[missed] >= 0).mean())


def test_secondary_looper_legs_are_removed():
    """The paper's category of secondary legs of loopers below 200 MeV/c: with
    pt_min = 0 (every track good otherwise) exactly the clusters attached to
    a secondary leg (leg >= 1) and in no good track's tube are removed, the
    primary legs' clusters stay; without the looper identification nothing
    is removed."""
    ev = tpcgen.time_frame(seed=4, n_collisions=4)
    r = oracle.track_event(ev)
    g, leg = oracle.loopers(ev.sector, r)
    assert (leg >= 1).sum() > 20
    adj0, fl0 = oracle.attach_event(ev, r, radius=1.5, pt_min=0.0, loopers_first=False)
    assert not (fl0 & oracle.CL_REMOVE).any()
    adj, fl = oracle.attach_event(ev, r, radius=1.5, pt_min=0.0)
    np.testing.assert_array_equal(adj, adj0)                  # adjacency does not depend on goodness
    att = r.assign >= 0
    sec = att & (leg[np.maximum(r.assign, 0)] >= 1)
    prim = att & (leg[np.maximum(r.assign, 0)] == 0)
    rem = (fl & oracle.CL_REMOVE) > 0
    prot = (fl & oracle.CL_PROTECTED) > 0
    assert rem[sec].sum() > 0.5 * sec.sum()
    np.testing.assert_array_equal(rem[sec], ~prot[sec])
    assert not rem[prim].any()
    assert not rem[att & ~sec].any()
