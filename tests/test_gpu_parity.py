"""Parity of the CUDA tracker (called through the C ABI) with the CPU oracle
on the same seeded inputs.  Decisions -- z after time->z, raw and cleaned
links, start hits, tracklet hit lists and end states, selector verdicts,
merged cluster lists, assignments -- are bit-exact.  Refitted parameters
agree within 1e-4 relative (measured against max(|p|, scale) with the scales
1 cm, 1 cm, 0.01, 0.01, 0.01 GeV^-1 of y, z, sin phi, tan lambda, q/pT) and
chi2 within 1e-3 relative of the binary64 oracle fit, on every track both
sides fit that is a fit of one helix (oracle chi2/ndf < 100).  Reported and
bounded as their own numbers: covered tracks with a parameter above 1e-4
(at most T/5000, each within 1e-3 of its standard deviation), tracks that
are not helix fits (their errors within 1e-3), refit status mismatches, and
tracks whose refit failed on both sides."""
import numpy as np
import pytest

import tpcgen
from gpu_helpers import CHI2_TOL, PARAM_TOL, compare_decisions, compare_fit, fit_summary, run_gpu

pytestmark = pytest.mark.gpu


def _check(ev, orc, params=None, fit=True, orc_params=None):
    g = run_gpu(ev, params=params)
    r = orc.track_event(ev, params=orc_params)
    bad = compare_decisions(ev, g, r)
    assert all(v == 0 for v in bad.values()), bad
    if fit:
        f = compare_fit(g, r)
        print(fit_summary(f))
        T = r.n_tracks
        # the spec bar on the covered tracks: parameters 1e-4, chi2 1e-3 relative;
        # parameters above 1e-4 are counted apart: at most T/5000 of the tracks, each
        # within 1e-3 of its standard deviation (a value far inside its own
        # uncertainty, e.g. q/pT ~ 0.01 +- 0.7 on a short track, has no meaningful
        # relative error); measured: 0 on every workload but the central event (1)
        assert f["n_param_over"] <= max(2, T // 5000), f
        assert f["param_over_sigma"] < 1e-3, f
        assert f["n_param_over"] > 0 or f["param_max"].max() < PARAM_TOL, f
        assert f["n_chi2_over"] == 0 and f["chi2_max"] < CHI2_TOL, f
        assert f["x_max"] < 1e-3, f
        # not helix fits (mis-merged looper legs): few, their errors bounded on their own
        assert f["n_not_helix"] <= max(5, T // 500), f
        assert f["not_helix_param_max"] < 1e-3 and f["not_helix_chi2_max"] < CHI2_TOL, f
        # refit status (one side's propagation left the helix domain): few
        assert f["status_mismatch"] <= max(2, T // 1000), f
    return g, r


def test_one_sector(orc):
    _check(tpcgen.one_sector(seed=1), orc)


@pytest.mark.parametrize("seed", [21, 22])
def test_one_sector_other_seeds(orc, seed):
    _check(tpcgen.one_sector(seed=seed, with_truth=False), orc)


def test_central_event_small(orc):
    _check(tpcgen.central_event(seed=2, n_tracks=1500, with_truth=False), orc)


def test_central_event_full(orc):
    """The full 10k-track central event (1.67 M clusters)."""
    _check(tpcgen.central_event(seed=2, with_truth=False), orc)


def test_time_frame_small(orc):
    _check(tpcgen.time_frame(seed=3, n_collisions=3, with_truth=False), orc)


def test_ragged_sizes(orc):
    """Sizes that are not multiples of any block or tile size."""
    for n_tracks, seed in ((1, 31), (7, 32), (33, 33), (257, 34)):
        _check(tpcgen.central_event(seed=seed, n_tracks=n_tracks, with_truth=False), orc)


def test_noise_only_and_tiny_inputs(orc):
    ev = tpcgen.central_event(seed=40, n_tracks=0, with_truth=False)
    assert ev.n == 0
    g = run_gpu(ev)
    assert g["n_tracks"] == 0
    ev = tpcgen.generate(n_sectors=36, n_tracks=0, noise_frac=0.0, seed=41, with_truth=False)
    # pure noise: many random clusters, no tracks expected
    rng = np.random.default_rng(5)
    n = 5000
    ev.sector = rng.integers(0, 36, n).astype(np.uint8)
    ev.row = rng.integers(0, 152, n).astype(np.uint8)
    ev.y = rng.uniform(-10, 10, n).astype(np.float32)
    ev.zt = rng.uniform(-250, 250, n).astype(np.float32)
    _check(ev, orc)


@pytest.mark.parametrize("mode, make", [(1, lambda: tpcgen.central_event(seed=2, n_tracks=1500, with_truth=False)),
                                        (1, lambda: tpcgen.time_frame(seed=3, n_collisions=3, with_truth=False)),
                                        (2, lambda: tpcgen.time_frame(seed=3, n_collisions=3, with_truth=False))])
def test_fp64_final_refit(orc, mode, make):
    """Binary64 covariance (Joseph form) and chi2 in the final pass: of every
    track (mode 1) or, with binary64 chi2 for every track, of the loopers only
    (mode 2)."""
    import paper_1905_05515_b300 as tpc
    ev = make()
    g = run_gpu(ev, params=tpc.tpc_params_default(fp64_final=mode))
    r = orc.track_event(ev)
    bad = compare_decisions(ev, g, r)
    assert all(v == 0 for v in bad.values()), bad
    ok = (g["status"] == 0) & (r.tr_status == 0)
    ce = np.abs(g["chi2_64"][ok] - r.tr_chi2[ok]) / r.tr_chi2[ok]
    diag = [0, 2, 5, 9, 14]
    cov_rel = (np.abs(g["cov64"][ok] - r.tr_c[ok]) / np.abs(r.tr_c[ok]))[:, diag]
    # the tracks the binary64 Joseph update is for: long looping low-pT tracks
    loop = ((np.abs(r.tr_p[ok, 4]) >= 5.0) | (r.tr_nclus[ok] > ev.row_x.shape[0]))
    helix = (r.tr_chi2[ok] / np.maximum(r.tr_ndf[ok], 1)) < 100.0
    print(f"binary64 mode {mode}: chi2 max rel {ce.max():.2e}; covariance diagonal max rel {cov_rel.max():.2e} "
          f"(loopers: {int(loop.sum())}, max {cov_rel[loop].max() if loop.any() else 0:.2e}; helix-fit loopers "
          f"max {cov_rel[loop & helix].max() if (loop & helix).any() else 0:.2e})")
    assert ce.max() < CHI2_TOL
    if ev.continuous:                         # the frames carry loopers, the central event none
        assert loop.sum() >= 5
        assert cov_rel[loop & helix].max() < 1e-4
    assert cov_rel[helix].max() < 1e-4


def test_fp64_loopers_only_mode():
    """Mode 2 takes the binary64 Joseph update exactly for the loopers: their
    covariance equals mode 1's bit for bit; the other tracks' final covariance
    is the binary32 update's (binary32-representable), their chi2 binary64."""
    import paper_1905_05515_b300 as tpc
    ev = tpcgen.time_frame(seed=3, n_collisions=3, with_truth=False)
    g1 = run_gpu(ev, params=tpc.tpc_params_default(fp64_final=1))
    g2 = run_gpu(ev, params=tpc.tpc_params_default(fp64_final=2))
    np.testing.assert_array_equal(g1["assign"], g2["assign"])
    qpt = np.abs(g2["param"][:, 4])
    nrow = ev.row_x.shape[0]
    loop = ((qpt >= 5.5) | (g2["nclus"] > nrow)) & (g2["status"] == 0)
    plain = (qpt <= 4.5) & (g2["nclus"] <= nrow) & (g2["status"] == 0)
    assert loop.sum() > 10 and plain.sum() > 100
    np.testing.assert_array_equal(g2["cov64"][loop], g1["cov64"][loop])
    c = g2["cov64"][plain]
    np.testing.assert_array_equal(c, c.astype(np.float32).astype(np.float64))
    assert np.all(np.isfinite(g2["chi2_64"][plain]))


@pytest.mark.parametrize("make", [lambda: tpcgen.time_frame(seed=3, n_collisions=3, with_truth=False),
                                  lambda: tpcgen.central_event(seed=2, n_tracks=1500, with_truth=False)])
def test_packed_link_coordinates(orc, make):
    """Packed-coordinate link pass: every decision bit-exact with the oracle
    running the same rounding, the fit within tolerance; the share of links
    the rounding changes is reported against the unpacked run."""
    import paper_1905_05515_b300 as tpc
    ev = make()
    g, r = _check(ev, orc, params=tpc.tpc_params_default(packed_links=1), orc_params={"packed_links": 1})
    g0 = run_gpu(ev)
    changed = np.mean((g["link_up"] != g0["link_up"]) | (g["link_dn"] != g0["link_dn"]))
    print(f"links changed by packing: {changed:.2e} of {ev.n} clusters")
    assert changed < 2e-3


@pytest.mark.parametrize("cap", [0, 1])
def test_merger_without_pair_list(orc, cap):
    """A pair list too small for the screened candidate pairs (none, or one
    per 1000 tracklet slots): the merger's direct path gives the same merges
    and tracks, bit-exact with the oracle."""
    import paper_1905_05515_b300 as tpc
    ev = tpcgen.time_frame(seed=3, n_collisions=3, with_truth=False)
    g, r = _check(ev, orc, params=tpc.tpc_params_default(merge_pairs_per_1k=cap))
    assert np.count_nonzero(np.asarray(r.seg_next) >= 0) > 10          # the event has merges to find


@pytest.mark.slow
def test_time_frame_full(orc):
    """The 50-collision continuous read-out frame (16 M clusters), whole-chain
    parity with the oracle (the oracle takes a few minutes here)."""
    _check(tpcgen.time_frame(seed=3, with_truth=False), orc)


def test_golden_line_cases(orc):
    """The hand-built straight-line cases (tests/golden/tracklets_b0.json):
    the GPU's tracklets, selector verdicts and tracks equal the hand-derived
    ones and the oracle's, bit for bit."""
    import os
    import types

    from helpers import golden_line_cases
    from test_oracle_golden_tracks import GOLDEN, check_golden_case
    X = tpcgen.row_x_f32()
    for case, sector, row, y, z in golden_line_cases(GOLDEN):
        ev = types.SimpleNamespace(n=y.size, row_x=X, n_sectors=1, z_max=250.0, continuous=False, sector=sector,
                                   row=row, y=y, zt=z, bz=0.0, v_drift=2.58)
        g, r = _check(ev, orc, fit=False)
        tk = g["tracklets"]
        off = g["clus_offset"]
        tracks = [g["clus_index"][off[t]:off[t + 1]] for t in range(int(g["n_tracks"]))]
        check_golden_case(case, y.size, tk["start"], tk["nhits"], tk["kept"], tracks)
    assert os.path.exists(GOLDEN)


@pytest.mark.parametrize("cap", [None, 0])
def test_membrane_crossing_merges(orc, cap):
    """An event with z given and the vertex spread along z (sigma 20 cm):
    tracks crossing the central membrane are merged across it, bit-exact with
    the oracle, through the pair list and through the direct path."""
    import paper_1905_05515_b300 as tpc
    ev = tpcgen.central_event(seed=3, n_tracks=3000, vertex_z_sigma=20.0, with_truth=False)
    params = None if cap is None else tpc.tpc_params_default(merge_pairs_per_1k=cap)
    g, r = _check(ev, orc, params=params)
    side = ev.sector[r.trk_start[r.seg_trk]].astype(int) // 18
    nxt = np.asarray(r.seg_next)
    cross = sum(1 for a in range(nxt.size) if nxt[a] >= 0 and side[a] != side[nxt[a]])
    assert cross >= 100, cross
