"""Hand-built TrackletConstructor / TrackletSelector cases (tests/golden/
tracklets_b0.json): straight lines at Bz = 0 whose tracklets, selector
verdicts and tracks were derived by hand from the reading of the method.
They pin the selector's tie-break (equal hit counts go to the smaller start
index, both orders of the same clusters) and the row-by-row following
(phase B crosses an empty row and takes every later row; phase C returns to
the start row and follows below it), and the following's state against the
least-squares line of numpy.linalg.lstsq."""
import os

import numpy as np

import tpcgen
from helpers import golden_line_cases

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "tracklets_b0.json")


def check_golden_case(case, n, trk_start, trk_nhits, trk_kept, tracks):
    exp = case["expect_tracklets"]
    np.testing.assert_array_equal(trk_start, exp["start"], err_msg=case["name"])
    np.testing.assert_array_equal(trk_nhits, exp["nhits"], err_msg=case["name"])
    np.testing.assert_array_equal(trk_kept, exp["kept"], err_msg=case["name"])
    want = case["expect_tracks"]
    if want == "all":
        want = [list(range(n))]
    elif isinstance(want, dict):
        want = [[i for i in range(n) if i not in want["all_but"]]]
    assert [list(map(int, t)) for t in tracks] == want, case["name"]


def lstsq_state(row, y, z, x_at):
    """(y, z, sin phi, tan lambda) of the least-squares line at plane x_at."""
    X = tpcgen.row_x_f32().astype(np.float64)
    x = X[row]
    A = np.stack([np.ones_like(x), x - x_at], 1)
    (ay, by), *_ = np.linalg.lstsq(A, y.astype(np.float64), rcond=None)
    (az, bz), *_ = np.linalg.lstsq(A, z.astype(np.float64), rcond=None)
    cphi = 1.0 / np.sqrt(1.0 + by * by)
    return np.array([ay, az, by * cphi, bz * cphi])


# binary32 rounding of a state accumulated over 150 updates (positions near 100 cm)
LSTSQ_TOL = np.array([2e-5, 2e-5, 3e-7, 5e-7])


def test_golden_line_cases(orc):
    X = tpcgen.row_x_f32()
    n_lstsq = 0
    for case, sector, row, y, z in golden_line_cases(GOLDEN):
        r = orc.track(sector, row, y, z, X, n_sectors=1, bz=0.0)
        tracks = [r.track_clusters(t) for t in range(r.n_tracks)]
        check_golden_case(case, y.size, r.trk_start, r.trk_nhits, r.trk_kept, tracks)
        if "expect_rejected" in case:
            assert np.nonzero(r.rejected)[0].tolist() == case["expect_rejected"], case["name"]
        if case.get("check_lstsq"):
            top = r.trk_top[0].astype(np.float64)
            assert top[0] == X[151]
            ls = lstsq_state(row, y, z, float(X[151]))
            assert np.all(np.abs(top[1:5] - ls) <= LSTSQ_TOL), (case["name"], top[1:5] - ls)
            if case["noise_cm"] > 0:
                # the least-squares line is not the generating line: the test discriminates
                part = case["parts"][0]
                dx = float(X[151]) - float(X[0])
                gen = np.array([part["y0"] + part["a"] * dx, part["z0"] + part["b"] * dx])
                assert np.all(np.abs(ls[:2] - gen) > 5 * LSTSQ_TOL[:2]), ls[:2] - gen
            n_lstsq += 1
    assert n_lstsq == 2
