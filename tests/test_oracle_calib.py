"""Pins of the calibration oracle (binary64 chi2 of the calibrated inward pass
with the primary-vertex pseudo-measurement, and its gradient).

What pins it to something other than itself:
* the B-spline basis against scipy's BSpline on the same knots;
* the measurement model against the generator's truth positions: with the
  true calibration the calibrated clusters scatter around the true points with
  the generator's sigma_y / sigma_z, with the nominal one they do not;
* the chi2 of the Kalman recursion against the minimum of the equivalent
  batch weighted least-squares problem solved with numpy's lstsq;
* chi2/ndf ~ 1 at the true calibration on clean primaries;
* invariance of the chi2 under a shift of the reference z (the reference is a
  linearisation point only);
* the gradient against central finite differences of the chi2;
* the derivative with respect to a measurement against twice the weighted
  smoothed residual of the least-squares solution (the identity the GPU
  backward pass uses).
"""
import numpy as np
import pytest

import tpcgen

QPT_MAX = 5.0


@pytest.fixture(scope="module")
def problem(orc):
    ev = tpcgen.calib_frame(seed=5, n_collisions=2, mult_mean=300)
    r = orc.track_event(ev)
    tc = tpcgen.track_collision_time(ev, r.tr_off, r.tr_clus)
    keep = (r.tr_status == 0) & (np.abs(r.tr_p[:, 4]) <= QPT_MAX)
    tc = np.where(keep, tc, np.nan).astype(np.float32)
    tr = orc.CalibTracks(r.tr_sector, r.tr_x, r.tr_p, r.tr_off, r.tr_clus, tc, ev.sector, ev.row, ev.y, ev.zt,
                         ev.row_x, v_nom=ev.v_drift)
    cal = tpcgen.calib_truth(5)
    th_true = np.concatenate([[cal["v_drift"], cal["t0"]], cal["spline"].ravel()])
    th_nom = np.zeros_like(th_true)
    th_nom[0] = ev.v_drift
    return ev, r, tr, th_true, th_nom


def test_bspline_matches_scipy(orc):
    from scipy.interpolate import BSpline
    k, n = 3, orc.CALIB_NSPL
    t = np.concatenate([np.zeros(k), np.linspace(0, 1, n - k + 1), np.ones(k)])
    us = np.concatenate([np.linspace(0, 1, 41), np.random.default_rng(0).random(200), [0.2, 0.4, 0.6, 0.8, 1.0]])
    for u in us:
        b, d = orc.bspline_all(u)
        for i in range(n):
            c = np.zeros(n)
            c[i] = 1.0
            s = BSpline(t, c, k, extrapolate=False)
            ref = s(u) if u < 1 else s(1 - 1e-15)
            dref = s.derivative()(u) if u < 1 else s.derivative()(1 - 1e-15)
            assert b[i] == pytest.approx(float(ref), abs=1e-12)
            assert d[i] == pytest.approx(float(dref), abs=1e-9)
        assert b.sum() == pytest.approx(1.0, abs=1e-14)


def test_measurement_model_against_truth(orc, problem):
    ev, r, tr, th_true, th_nom = problem
    sig = ev.label >= 0
    idx = np.nonzero(sig)[0][:20000]
    tc = ev.trk_tc[ev.label[idx]].astype(np.float32)
    my, mz = orc.calib_measure(tr, th_true, idx, tc)
    dy, dz = my - ev.true_y[idx], mz - ev.true_z[idx]
    assert abs(dy.mean()) < 0.005 and abs(dz.mean()) < 0.005
    assert 0.095 < dy.std() < 0.106
    assert 0.142 < dz.std() < 0.158
    my0, mz0 = orc.calib_measure(tr, th_nom, idx, tc)
    assert (my0 - ev.true_y[idx]).std() > 1.5 * dy.std()
    assert (mz0 - ev.true_z[idx]).std() > 1.5 * dz.std()


def _lsq_chi2(F, h, m, v, c0, anchor=None):
    """Minimum of the batch objective equivalent to the Kalman pass: prior
    N((m0 - h0, 0, 0, 0), C0) on the deviation d at step 0, measurements
    m_k = h_k + H Phi_k d + noise(v_k), Phi_k = F_k ... F_1."""
    n1 = F.shape[0]
    rows, rhs = [], []
    mu0 = np.array([m[0, 0] - h[0, 0], m[0, 1] - h[0, 1], 0, 0, 0])
    for i in range(5):                        # whitened prior rows
        e = np.zeros(5)
        e[i] = 1 / np.sqrt(c0[i])
        rows.append(e)
        rhs.append(mu0[i] / np.sqrt(c0[i]))
    Phi = np.eye(5)
    for k in range(1, n1):
        Phi = F[k] @ Phi
        for e in range(2):
            rows.append(Phi[e] / np.sqrt(v[k, e]))
            rhs.append((m[k, e] - h[k, e]) / np.sqrt(v[k, e]))
    if anchor is not None:                    # (tan(lambda) measured, reference tan(lambda), variance)
        tm, q3, var = anchor
        rows.append(Phi[3] / np.sqrt(var))
        rhs.append((tm - q3) / np.sqrt(var))
    A, b = np.array(rows), np.array(rhs)
    d, *_ = np.linalg.lstsq(A, b, rcond=None)
    res = A @ d - b
    return float(res @ res)


def test_chi2_equals_batch_least_squares(orc, problem):
    ev, r, tr, th_true, th_nom = problem
    p = orc.default_params()
    c0 = np.array([p["sigma_y"] ** 2, p["sigma_z"] ** 2, p["c0_snp"], p["c0_tgl"], p["c0_qpt"]], np.float64)
    c0[:2] = np.float32(p["sigma_y"]) ** 2, np.float32(p["sigma_z"]) ** 2
    chi2, used, _ = orc.calib(tr, th_nom, grad=False)
    cand = np.nonzero(used)[0]
    checked = 0
    for t in cand[:: max(1, cand.size // 25)]:
        ex = orc.calib_explain(tr, th_nom, int(t))
        assert ex is not None
        F, h, m, v, c2 = ex
        assert c2 == pytest.approx(chi2[t], rel=1e-12)
        ref = _lsq_chi2(F, h, m, v, c0)
        assert c2 == pytest.approx(ref, rel=1e-7, abs=1e-9)
        checked += 1
    assert checked >= 20


def test_dip_angle_anchor_equals_batch_least_squares(orc, problem):
    """The pass with the matched inner track's dip angle: its chi2 is the
    minimum of the batch problem with one more row, tan(lambda) at the vertex
    (the reference's dip angle is the tracker's, constant along the helix);
    the gradient through the extra update against central differences."""
    ev, r, tr, th_true, th_nom = problem
    p = orc.default_params()
    c0 = np.array([p["sigma_y"] ** 2, p["sigma_z"] ** 2, p["c0_snp"], p["c0_tgl"], p["c0_qpt"]], np.float64)
    c0[:2] = np.float32(p["sigma_y"]) ** 2, np.float32(p["sigma_z"]) ** 2
    tg = tpcgen.track_dip_angle(ev, r.tr_off, r.tr_clus)
    var = 9e-8
    chi2, used, _ = orc.calib(tr, th_nom, grad=False, tgl_ext=tg, tgl_var=var)
    free, _, _ = orc.calib(tr, th_nom, grad=False)
    cand = np.nonzero(used & np.isfinite(tg))[0]
    for t in cand[:: max(1, cand.size // 25)]:
        F, h, m, v, c2 = orc.calib_explain(tr, th_nom, int(t))
        assert c2 == pytest.approx(free[t], rel=1e-12)
        ref = _lsq_chi2(F, h, m, v, c0, anchor=(float(tg[t]), float(tr.param[t, 3]), var))
        assert chi2[t] == pytest.approx(ref, rel=1e-7, abs=1e-9)
        assert chi2[t] >= free[t]
    # tracks without a dip angle keep their chi2; a huge variance gives the free pass back
    nan = np.nonzero(used & ~np.isfinite(tg))[0]
    assert np.array_equal(chi2[nan], free[nan])
    loose, _, _ = orc.calib(tr, th_nom, grad=False, tgl_ext=tg, tgl_var=1e12)
    np.testing.assert_allclose(loose[used], free[used], rtol=1e-9, atol=1e-9)
    # gradient with the anchor against central differences (v, t0, one spline coefficient)
    sel = np.zeros(tr.n_tracks)
    sel[cand[:60]] = 1.0
    _, _, g = orc.calib(tr, th_true, weight=sel, tgl_ext=tg, tgl_var=var)

    def f(x):
        return float((orc.calib(tr, x, grad=False, tgl_ext=tg, tgl_var=var)[0] * sel).sum())

    for i, hs in ((0, 1e-6), (1, 1e-5), (2 + int(np.argmax(np.abs(g[2:]))), 1e-5)):
        e = np.zeros_like(th_true)
        e[i] = 1.0
        fd = (f(th_true + hs * e) - f(th_true - hs * e)) / (2 * hs)
        assert g[i] == pytest.approx(fd, rel=1e-5, abs=1e-6 * np.abs(g).max())


def test_chi2_per_dof_at_true_calibration(orc, problem):
    ev, r, tr, th_true, th_nom = problem
    n = np.diff(r.tr_off)
    pur = np.array([np.unique(ev.label[r.track_clusters(t)], return_counts=True)[1].max() / n[t]
                    for t in range(r.n_tracks)])
    c_true, used, _ = orc.calib(tr, th_true, grad=False)
    c_nom, used_n, _ = orc.calib(tr, th_nom, grad=False)
    sel = used & used_n & (pur == 1.0)
    assert sel.sum() > 500
    ndf = 2 * (n[sel] + 1) - 5
    q_true = c_true[sel] / ndf
    q_nom = c_nom[sel] / ndf
    assert 0.9 < np.median(q_true) < 1.05
    assert 0.9 < q_true.mean() < 1.15
    assert np.median(q_nom) > 1.3


def test_reference_z_shift_invariance(orc, problem):
    ev, r, tr, th_true, th_nom = problem
    c0, u0, g0 = orc.calib(tr, th_true)
    import dataclasses
    p2 = tr.param.copy()
    p2[:, 1] += np.float32(3.0)
    tr2 = dataclasses.replace(tr, param=p2)
    c1, u1, g1 = orc.calib(tr2, th_true)
    assert np.array_equal(u0, u1)
    np.testing.assert_allclose(c1[u0], c0[u0], rtol=1e-7, atol=1e-9)
    np.testing.assert_allclose(g1, g0, rtol=1e-6, atol=1e-6 * np.abs(g0).max())


def test_gradient_against_finite_differences(orc, problem):
    ev, r, tr, th_true, th_nom = problem
    rng = np.random.default_rng(3)
    th = th_true + np.concatenate([[0.002, 0.05], rng.normal(0, 0.05, th_true.size - 2)])
    w = rng.uniform(0.5, 1.5, tr.n_tracks)
    c, used, g = orc.calib(tr, th, weight=w)

    def f(x):
        cc, uu, _ = orc.calib(tr, x, weight=w, grad=False)
        assert np.array_equal(uu, used)
        return float((w * cc).sum())

    big = np.argsort(-np.abs(g[2:]))[:12] + 2
    idx = np.concatenate([[0, 1], big, rng.choice(np.arange(2, th.size), 8, replace=False)])
    for i in idx:
        h = 1e-6 * max(abs(th[i]), 1.0) if i < 2 else 1e-5
        e = np.zeros_like(th)
        e[i] = h
        fd = (f(th + e) - f(th - e)) / (2 * h)
        assert g[i] == pytest.approx(fd, rel=1e-5, abs=1e-6 * np.abs(g).max()), i


def test_gradient_is_linear_in_the_weights(orc, problem):
    ev, r, tr, th_true, th_nom = problem
    rng = np.random.default_rng(4)
    w1 = rng.uniform(0, 1, tr.n_tracks)
    w2 = rng.uniform(0, 1, tr.n_tracks)
    _, _, g1 = orc.calib(tr, th_true, weight=w1)
    _, _, g2 = orc.calib(tr, th_true, weight=w2)
    _, _, g12 = orc.calib(tr, th_true, weight=2 * w1 - w2)
    np.testing.assert_allclose(g12, 2 * g1 - g2, rtol=1e-9, atol=1e-9 * np.abs(g12).max())


def test_measurement_derivative_is_twice_the_weighted_smoothed_residual(orc, problem):
    """The identity the GPU backward pass is built on: d chi2 / d m_k =
    2 V_k^-1 (m_k - h_k - H Phi_k d*), with d* the least-squares deviation at
    step 0 (checked against central finite differences of the oracle's chi2
    in a cluster's y; the chi2 is quadratic in it, so the difference is exact
    up to rounding)."""
    import dataclasses
    ev, r, tr, th_true, th_nom = problem
    p = orc.default_params()
    c0 = np.array([np.float32(p["sigma_y"]) ** 2, np.float32(p["sigma_z"]) ** 2, p["c0_snp"], p["c0_tgl"],
                   p["c0_qpt"]], np.float64)
    chi2, used, _ = orc.calib(tr, th_true, grad=False)
    cand = np.nonzero(used)[0][::97][:6]
    for t in cand:
        F, h, m, v, c2 = orc.calib_explain(tr, th_true, int(t))
        n1 = F.shape[0]
        rows, rhs = [], []
        mu0 = np.array([m[0, 0] - h[0, 0], m[0, 1] - h[0, 1], 0, 0, 0])
        c0 = np.array([v[0, 0], v[0, 1], *c0[2:]])
        for i in range(5):
            e = np.zeros(5)
            e[i] = 1 / np.sqrt(c0[i])
            rows.append(e)
            rhs.append(mu0[i] / np.sqrt(c0[i]))
        Phis = [np.eye(5)]
        for k in range(1, n1):
            Phis.append(F[k] @ Phis[-1])
            for e in range(2):
                rows.append(Phis[-1][e] / np.sqrt(v[k, e]))
                rhs.append((m[k, e] - h[k, e]) / np.sqrt(v[k, e]))
        d0, *_ = np.linalg.lstsq(np.array(rows), np.array(rhs), rcond=None)
        n = n1 - 1
        for k in (0, n // 2, n - 1):
            dk = Phis[k] @ d0
            a_y = 2 * (m[k, 0] - h[k, 0] - dk[0]) / v[k, 0]
            # step k measures cluster n-1-k of the track's list (inner -> outer)
            c = int(tr.clus[tr.off[t] + n - 1 - k])

            def f(yc):
                y = tr.cl_y.copy()
                y[c] = yc
                cc, uu, _ = orc.calib(dataclasses.replace(tr, cl_y=y), th_true, grad=False)
                return cc[t]

            yp, ym = np.float32(tr.cl_y[c] + 1e-2), np.float32(tr.cl_y[c] - 1e-2)   # the binary32 inputs
            fd = (f(yp) - f(ym)) / (float(yp) - float(ym))
            assert a_y == pytest.approx(fd, rel=1e-5, abs=1e-6), (t, k)


def test_track_selection_cases():
    """The calibration's track selection on hand-made cases: refit status 0
    and |q/pT| <= 5 (binary32, the edge included) keep the collision time;
    a failed refit, |q/pT| just above 5 or a NaN parameter give NaN; a NaN
    collision time stays NaN."""
    import oracle
    q = np.array([0.0, 5.0, -5.0, np.nextafter(np.float32(5), np.float32(6)), np.nan, 1.0, 1.0], np.float32)
    param = np.zeros((q.size, 5), np.float32)
    param[:, 4] = q
    status = np.array([0, 0, 0, 0, 0, 1, 0], np.int32)
    tc = np.array([10, 20, 30, 40, 50, 60, np.nan], np.float32)
    out = oracle.calib_select(tc, status, param)
    exp = np.array([10, 20, 30, np.nan, np.nan, np.nan, np.nan], np.float32)
    np.testing.assert_array_equal(out, exp)


def test_z_error_follows_the_drift_time(orc, problem):
    """The z error of a cluster is its drift-time error carried through the
    calibration map: variance sigma_z^2 s^2 with s = (v / v_nom) (1 - d dz /
    d zl), the slope of the map taken at the nominal position; s = 1 at the
    nominal calibration.  The slope here comes from tpcgen's own basis by
    central differences."""
    ev, r, tr, th_true, th_nom = problem
    p = orc.default_params()
    sz2 = float(np.float32(p["sigma_z"])) ** 2
    used = orc.calib(tr, th_nom, grad=False)[1]
    t = int(np.nonzero(used)[0][3])
    F, h, m, v, c2 = orc.calib_explain(tr, th_nom, t)
    assert np.allclose(v[:-1, 1], sz2, rtol=1e-6)
    th = th_true.copy()
    F, h, m, v, c2 = orc.calib_explain(tr, th, t)
    n = tr.off[t + 1] - tr.off[t]
    coef = th[2:].reshape(36, 8, 8, 2)
    for k in range(n):
        c = int(tr.clus[tr.off[t] + n - 1 - k])
        s_ = int(tr.cl_sector[c])
        u = (tr.row_x[tr.cl_row[c]] - tr.row_x[0]) / (tr.row_x[-1] - tr.row_x[0])
        wn = (tr.z_max - tr.v_nom * (float(tr.cl_t[c]) - float(tr.tcoll[t]))) / tr.z_max
        bu = tpcgen.bspline_basis(np.array([u]), 8)[0]

        def dz(w):
            return float(bu @ coef[s_, :, :, 1] @ tpcgen.bspline_basis(np.array([w]), 8)[0])

        slope = (dz(wn + 1e-6) - dz(wn - 1e-6)) / 2e-6 / tr.z_max if 1e-6 < wn < 1 - 1e-6 else 0.0
        s = th[0] / tr.v_nom * (1.0 - slope)
        assert v[k, 1] == pytest.approx(sz2 * s * s, rel=1e-7), k
