"""Pins of the merger's chi2 (orc_merge_chi2: outer end of piece A rotated
by +-20 degrees into the frame of the neighbouring sector, propagated to the
inner end of piece B there, chi2 over the five parameters with the summed
covariance; section "TPC Tracking", sector boundaries).  The facts used here
do not come from the oracle:

* a noise-free helix split at a sector boundary: both ends are exact generator
  states of one helix, so the chi2 is zero up to binary32 rounding;
* with the wrong sign of the rotation the same pairs are refused;
* with A's covariance zero the chi2 is the closed form d^T C_B^-1 d of the
  offset planted on B (numpy's solve);
* ends perturbed by draws from their own covariances: the chi2 of one track's
  two pieces follows the chi2 distribution with 5 degrees of freedom (mean 5,
  Kolmogorov-Smirnov test), which a dropped covariance term, a missed
  transport of A's covariance or a transposed index would break;
* a piece paired with another track's piece is refused (chi2 above the cut).

Across the central membrane (events with z given and a vertex spread along
z), the two pieces of a track share the wedge's local frame:

* a noise-free helix split at the membrane has zero chi2 with no rotation and
  is refused with the +-20 degree rotation of the neighbouring wedges;
* on an event, every merge across the membrane joins pieces of one generated
  track, nearly every crossing track found as two pieces of one wedge is
  merged, and the reversed pair (which also fits at small dip angles) is not
  what joins them;
* with drift times (z unknown up to the collision time) nothing is merged
  across the membrane.
"""
import math

import numpy as np
import pytest
from scipy import stats

import tpcgen
from helpers import track_truth_state

BZ = 0.5
KB64 = -tpcgen.C_LIGHT * BZ
COS20 = np.float32(math.cos(math.radians(20)))
SIN20 = np.float32(math.sin(math.radians(20)))
MERGE_CUT = 50.0


def _cov(c15):
    C = np.zeros((5, 5))
    k = 0
    for i in range(5):
        for j in range(i + 1):
            C[i, j] = C[j, i] = c15[k]
            k += 1
    return C


@pytest.fixture(scope="module")
def split_pairs(orc):
    """Tracks crossing exactly one boundary between neighbouring sectors of one
    side: (outermost cluster of piece A, innermost of piece B, direction,
    covariance at A's outer end, covariance at B's inner end).  The
    covariances are those of binary64 fits of each piece's exact crossings
    (realistic correlations; any positive-definite matrix would do)."""
    ev = tpcgen.central_event(seed=17, n_tracks=1500)
    out = []
    for t in range(ev.trk_pt.size):
        idx = np.where(ev.label == t)[0]
        if idx.size < 60:
            continue
        idx = idx[np.argsort(ev.true_s[idx])]
        s = ev.sector[idx].astype(int)
        k = np.where(s[1:] != s[:-1])[0]
        if k.size != 1:
            continue
        a_run, b_run = idx[:k[0] + 1], idx[k[0] + 1:]
        d = (s[-1] % 18 - s[0] % 18) % 18
        if a_run.size < 12 or b_run.size < 12 or s[0] // 18 != s[-1] // 18 or d not in (1, 17):
            continue

        def fitcov(run, n_passes):
            x = ev.row_x[ev.row[run]].astype(np.float64)
            st0 = np.zeros(21)
            st0[0] = x[-1]
            st0[1:6] = track_truth_state(ev, run[-1])
            st0[6], st0[8], st0[11], st0[15], st0[20] = 0.01, 0.0225, 0.25, 0.25, 100.0
            ok, st, _ = orc.fit64(ev.sector[run].astype(np.int32), x, ev.true_y[run], ev.true_z[run], st0, KB64,
                                  n_passes=n_passes)
            assert ok
            return st[6:]

        # two passes end at the outermost cluster, three at the innermost
        out.append((a_run[-1], b_run[0], 1 if d == 1 else -1, fitcov(a_run, 2), fitcov(b_run, 3)))
    assert len(out) >= 300
    return ev, out


def _ends(ev, a, b, ca, cb):
    top = np.zeros(21, np.float32)
    bot = np.zeros(21, np.float32)
    top[0] = ev.row_x[ev.row[a]]
    top[1:6] = track_truth_state(ev, a)
    top[6:] = ca
    bot[0] = ev.row_x[ev.row[b]]
    bot[1:6] = track_truth_state(ev, b)
    bot[6:] = cb
    return top, bot


def _kb32(orc):
    return np.float32(orc.KB_C) * np.float32(BZ)


def test_noise_free_split_helix_has_zero_chi2(orc, split_pairs):
    ev, pairs = split_pairs
    kb = _kb32(orc)
    worst = 0.0
    for a, b, d, ca, cb in pairs:
        top, bot = _ends(ev, a, b, ca, cb)
        worst = max(worst, orc.merge_chi2(top, bot, COS20, SIN20 if d > 0 else -SIN20, kb))
    assert worst < 1e-4, worst          # binary32 rounding of a state at |z| <= 250 cm


def test_wrong_rotation_sign_is_refused(orc, split_pairs):
    ev, pairs = split_pairs
    kb = _kb32(orc)
    c2 = [orc.merge_chi2(*_ends(ev, a, b, ca, cb), COS20, -SIN20 if d > 0 else SIN20, kb)
          for a, b, d, ca, cb in pairs]
    assert min(c2) > 100 * MERGE_CUT


def test_closed_form_with_exact_outer_state(orc, split_pairs):
    """A's covariance zero (it stays zero through rotation and propagation):
    the chi2 is d^T C_B^-1 d for the offset d planted on B's parameters."""
    ev, pairs = split_pairs
    kb = _kb32(orc)
    rng = np.random.default_rng(3)
    worst = 0.0
    for a, b, d, ca, cb in pairs[:200]:
        top, bot = _ends(ev, a, b, np.zeros(15), cb)
        Cb = _cov(cb)
        delta = 3.0 * rng.multivariate_normal(np.zeros(5), Cb)
        exact_b = bot[1:6].astype(np.float64)
        bot[1:6] = (exact_b - delta).astype(np.float32)
        # the planted offset as stored in binary32, against the exact crossing
        dd = exact_b - bot[1:6].astype(np.float64)
        expect = float(dd @ np.linalg.solve(Cb, dd))
        got = orc.merge_chi2(top, bot, COS20, SIN20 if d > 0 else -SIN20, kb)
        worst = max(worst, abs(got - expect) / max(expect, 1.0))
    assert worst < 2e-3, worst


def test_smeared_pieces_follow_chi2_with_five_dof(orc, split_pairs):
    ev, pairs = split_pairs
    kb = _kb32(orc)
    rng = np.random.default_rng(1)
    c2 = []
    for a, b, d, ca, cb in pairs:
        top, bot = _ends(ev, a, b, ca, cb)
        for _ in range(3):
            t2, b2 = top.copy(), bot.copy()
            t2[1:6] += rng.multivariate_normal(np.zeros(5), _cov(ca))
            b2[1:6] += rng.multivariate_normal(np.zeros(5), _cov(cb))
            c2.append(orc.merge_chi2(t2, b2, COS20, SIN20 if d > 0 else -SIN20, kb))
    c2 = np.array(c2)
    n = c2.size
    assert abs(c2.mean() - 5.0) < 4 * math.sqrt(10.0 / n), c2.mean()
    assert abs(c2.var() - 10.0) < 0.25 * 10.0, c2.var()
    assert stats.kstest(c2, stats.chi2(5).cdf).pvalue > 1e-3


def test_pieces_of_different_tracks_are_refused(orc, split_pairs):
    ev, pairs = split_pairs
    kb = _kb32(orc)
    c2 = []
    for i, (a, b, d, ca, cb) in enumerate(pairs):
        a2, b2, d2, ca2, cb2 = pairs[(i + 7) % len(pairs)]
        c2.append(orc.merge_chi2(*_ends(ev, a, b2, ca, cb2), COS20, SIN20 if d > 0 else -SIN20, kb))
    assert min(c2) > MERGE_CUT


# ---- central membrane --------------------------------------------------------------
def _fitcov(orc, ev, run, n_passes):
    x = ev.row_x[ev.row[run]].astype(np.float64)
    st0 = np.zeros(21)
    st0[0] = x[-1]
    st0[1:6] = track_truth_state(ev, run[-1])
    st0[6], st0[8], st0[11], st0[15], st0[20] = 0.01, 0.0225, 0.25, 0.25, 100.0
    ok, st, _ = orc.fit64(ev.sector[run].astype(np.int32), x, ev.true_y[run], ev.true_z[run], st0, KB64,
                          n_passes=n_passes)
    assert ok
    return st[6:]


@pytest.fixture(scope="module")
def membrane_ev():
    return tpcgen.central_event(seed=3, n_tracks=3000, vertex_z_sigma=20.0)


@pytest.fixture(scope="module")
def membrane_pairs(orc, membrane_ev):
    """Tracks crossing the membrane once inside one wedge: (outermost cluster
    on the vertex side, innermost on the other side, covariances as above)."""
    ev = membrane_ev
    out = []
    for t in range(ev.trk_pt.size):
        idx = np.where(ev.label == t)[0]
        if idx.size < 40:
            continue
        idx = idx[np.argsort(ev.true_s[idx])]
        s = ev.sector[idx].astype(int)
        k = np.where(s[1:] != s[:-1])[0]
        if k.size != 1 or s[0] % 18 != s[-1] % 18:
            continue
        a_run, b_run = idx[:k[0] + 1], idx[k[0] + 1:]
        if a_run.size < 12 or b_run.size < 12:
            continue
        out.append((a_run[-1], b_run[0], _fitcov(orc, ev, a_run, 2), _fitcov(orc, ev, b_run, 3)))
    assert len(out) >= 50
    return out


def test_membrane_split_helix_has_zero_chi2_without_rotation(orc, membrane_ev, membrane_pairs):
    ev = membrane_ev
    kb = _kb32(orc)
    for a, b, ca, cb in membrane_pairs:
        top, bot = _ends(ev, a, b, ca, cb)
        assert ev.sector[a] // 18 != ev.sector[b] // 18
        assert np.sign(top[2]) != np.sign(bot[2]) or min(abs(top[2]), abs(bot[2])) < 1.0
        assert orc.merge_chi2(top, bot, np.float32(1.0), np.float32(0.0), kb) < 1e-4
        # the rotation of a neighbouring wedge does not apply across the membrane
        assert orc.merge_chi2(top, bot, COS20, SIN20, kb) > MERGE_CUT
        assert orc.merge_chi2(top, bot, COS20, -SIN20, kb) > MERGE_CUT


def _majority(ev, r, a):
    tq = r.seg_trk[a]
    h = r.trk_hits[r.trk_off[tq]:r.trk_off[tq + 1]]
    v, c = np.unique(ev.label[h], return_counts=True)
    return int(v[c.argmax()]), c.max() / h.size


def test_membrane_merging_on_an_event(orc, membrane_ev):
    ev = membrane_ev
    r = orc.track_event(ev)
    ns = r.seg_trk.size
    sec = ev.sector[r.trk_start[r.seg_trk]].astype(int)
    side = sec // 18
    cross = [(a, int(r.seg_next[a])) for a in range(ns) if r.seg_next[a] >= 0 and side[a] != side[r.seg_next[a]]]
    assert len(cross) >= 40
    kb = _kb32(orc)
    for a, b in cross:
        la, fa = _majority(ev, r, a)
        lb, fb = _majority(ev, r, b)
        assert la == lb >= 0 and fa > 0.8 and fb > 0.8
        assert sec[a] % 18 == sec[b] % 18
        top, bot = r.trk_top[r.seg_trk[a]], r.trk_bot[r.seg_trk[b]]
        assert bot[0] >= top[0]                      # B continues A outward
        # the reversed pair (B's outer end to A's inner end) fits as well for
        # most of them: the outward order, not the chi2, tells them apart
    rev = [orc.merge_chi2(r.trk_top[r.seg_trk[b]], r.trk_bot[r.seg_trk[a]], np.float32(1.0), np.float32(0.0), kb)
           for a, b in cross]
    assert np.mean(np.array(rev) < MERGE_CUT) > 0.3
    # crossing tracks found as one piece on each side of one wedge: merged
    pieces = {}
    for a in range(ns):
        lab, frac = _majority(ev, r, a)
        if lab >= 0 and frac > 0.9:
            pieces.setdefault(lab, []).append(a)
    found = merged = 0
    for lab, segs in pieces.items():
        if len(segs) != 2 or side[segs[0]] == side[segs[1]] or sec[segs[0]] % 18 != sec[segs[1]] % 18:
            continue
        found += 1
        merged += r.seg_next[segs[0]] == segs[1] or r.seg_next[segs[1]] == segs[0]
    assert found >= 40 and merged >= 0.9 * found, (found, merged)
    # each merged track is still a valid track: ndf and sectors of one wedge
    for t in range(r.n_tracks):
        cl = r.track_clusters(t)
        assert r.tr_ndf[t] == 2 * cl.size - 5


def test_no_membrane_merging_with_drift_times(orc):
    ev = tpcgen.time_frame(seed=4, n_collisions=2, vertex_z_sigma=10.0, with_truth=False)
    r = orc.track_event(ev)
    side = ev.sector[r.trk_start[r.seg_trk]].astype(int) // 18
    nxt = r.seg_next
    assert (nxt >= 0).sum() > 0
    assert not any(side[a] != side[nxt[a]] for a in range(nxt.size) if nxt[a] >= 0)
