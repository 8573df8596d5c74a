"""Pins of the oracle's Kalman mathematics (helix propagation, frame rotation,
update, multi-pass fit) against facts that do not come from the oracle:

* the generator's analytic helix/plane crossings (float64, exact geometry);
* central finite differences of the propagation (Jacobians);
* the information form of the Kalman update (a different formula);
* the closed-form weighted least-squares straight line at B = 0 (numpy lstsq);
* exact parameter recovery from noise-free helices;
* statistical invariants (chi2/ndf ~ 1, pulls ~ N(0, 1)).
"""
import math

import numpy as np
import pytest

import tpcgen
from helpers import is_spd, track_truth_state

BZ = 0.5
KB64 = -tpcgen.C_LIGHT * BZ            # exact d sin(phi)/dx per GeV^-1 at 0.5 T
COS20, SIN20 = math.cos(math.radians(20)), math.sin(math.radians(20))


@pytest.fixture(scope="module")
def ev():
    return tpcgen.central_event(seed=11, n_tracks=400)


def _sector_runs(ev, min_len=30, max_tracks=60):
    """Per track, the clusters of its longest single-sector run, ordered by path."""
    out = []
    for t in range(ev.trk_pt.size):
        idx = np.where(ev.label == t)[0]
        if idx.size < min_len:
            continue
        idx = idx[np.argsort(ev.true_s[idx])]
        sec = ev.sector[idx]
        cut = np.where(sec[1:] != sec[:-1])[0] + 1
        runs = np.split(idx, cut)
        run = max(runs, key=len)
        if len(run) >= min_len:
            out.append(run)
        if len(out) >= max_tracks:
            break
    return out


def _state_at(ev, cl, cov=1e-4):
    st = np.zeros(21)
    st[0] = ev.row_x[ev.row[cl]]
    st[1:6] = track_truth_state(ev, cl)
    for k in (0, 2, 5, 9, 14):
        st[6 + k] = cov
    return st


def test_prop64_matches_helix_crossings_forward_and_backward(orc, ev):
    worst = 0.0
    for run in _sector_runs(ev):
        for i, j in ((0, len(run) - 1), (len(run) - 1, 0), (5, 6), (12, 11), (3, 20), (25, 2)):
            a, b = run[i], run[j]
            ok, st = orc.prop64(_state_at(ev, a), float(ev.row_x[ev.row[b]]), KB64)
            assert ok
            err = np.abs(st[1:4] - track_truth_state(ev, b)[:3])
            worst = max(worst, err.max())
    assert worst < 1e-8, worst


def test_prop32_matches_helix_crossings(orc, ev):
    kb32 = np.float32(orc.KB_C) * np.float32(BZ)
    worst = 0.0
    for run in _sector_runs(ev):
        for i in range(0, len(run) - 1, 7):
            a, b = run[i], run[i + 1]
            for src, dst in ((a, b), (b, a)):
                ok, st = orc.prop32(_state_at(ev, src).astype(np.float32), ev.row_x[ev.row[dst]], kb32)
                assert ok
                err = np.abs(st[1:4].astype(np.float64) - track_truth_state(ev, dst)[:3])
                worst = max(worst, err.max())
    # one row step in binary32 at |y| <= 90 cm, |z| <= 250 cm
    assert worst < 1e-4, worst


def test_rotation_then_propagation_matches_crossing_in_next_sector(orc, ev):
    n = 0
    for t in range(ev.trk_pt.size):
        idx = np.where(ev.label == t)[0]
        if idx.size < 50:
            continue
        idx = idx[np.argsort(ev.true_s[idx])]
        s = ev.sector[idx]
        k = np.where(s[1:] != s[:-1])[0]
        if k.size == 0:
            continue
        a, b = idx[k[0]], idx[k[0] + 1]
        sa, sb = int(ev.sector[a]), int(ev.sector[b])
        d = (sb % 18 - sa % 18) % 18
        if sa // 18 != sb // 18 or d not in (1, 17):
            continue
        sn = SIN20 if d == 1 else -SIN20
        ok, st = orc.rot64(_state_at(ev, a), COS20, sn, KB64)
        assert ok
        ok, st = orc.prop64(st, float(ev.row_x[ev.row[b]]), KB64)
        assert ok
        np.testing.assert_allclose(st[1:4], track_truth_state(ev, b)[:3], atol=1e-8)
        n += 1
    assert n >= 20


def _jacobian_from_cov(step, st):
    """Column k of the transport matrix F from C' = F e_k e_k^T F^T (F_kk > 0)."""
    F = np.zeros((5, 5))
    for k in range(5):
        s = st.copy()
        s[6:] = 0
        kk = k * (k + 1) // 2 + k
        s[6 + kk] = 1.0
        ok, out = step(s)
        assert ok
        C = np.zeros((5, 5))
        q = 0
        for i in range(5):
            for j in range(i + 1):
                C[i, j] = C[j, i] = out[6 + q]
                q += 1
        F[:, k] = C[:, k] / math.sqrt(C[k, k])
    return F


def _fd_jacobian(step, st, h=(1e-6, 1e-6, 1e-7, 1e-7, 1e-6)):
    F = np.zeros((5, 5))
    for k in range(5):
        sp, sm = st.copy(), st.copy()
        sp[1 + k] += h[k]
        sm[1 + k] -= h[k]
        okp, op = step(sp)
        okm, om = step(sm)
        assert okp and okm
        F[:, k] = (op[1:6] - om[1:6]) / (2 * h[k])
    return F


@pytest.mark.parametrize("snp,qpt,dx", [(0.1, 0.5, 1.07), (-0.4, -3.0, 1.07), (0.3, 2.0, -1.07),
                                         (0.6, -1.5, 25.0), (-0.2, 0.2, -60.0), (0.0, 4.9, 0.3)])
def test_prop64_jacobian_matches_finite_differences(orc, snp, qpt, dx):
    st = np.zeros(21)
    st[0], st[1:6] = 120.0, [3.0, -40.0, snp, 0.7, qpt]
    step = lambda s: orc.prop64(s, 120.0 + dx, KB64)  # noqa: E731
    Fa = _jacobian_from_cov(step, st)
    Fd = _fd_jacobian(step, st)
    np.testing.assert_allclose(Fa, Fd, rtol=1e-6, atol=1e-7)


@pytest.mark.parametrize("snp,qpt,sn", [(0.1, 0.5, SIN20), (-0.3, -2.0, -SIN20), (0.5, 1.0, -SIN20)])
def test_rot64_jacobian_matches_finite_differences(orc, snp, qpt, sn):
    """Rotation followed by propagation to a fixed plane: the composite
    Jacobian (from the transported covariance) equals finite differences."""
    st = np.zeros(21)
    st[0], st[1:6] = 200.0, [30.0, 12.0, snp, -0.4, qpt]

    def step(s):
        ok, r = orc.rot64(s, COS20, sn, KB64)
        if not ok:
            return ok, r
        return orc.prop64(r, 210.0, KB64)

    Fa = _jacobian_from_cov(step, st)
    Fd = _fd_jacobian(step, st)
    np.testing.assert_allclose(Fa, Fd, rtol=1e-6, atol=1e-6)


def test_rotation_round_trip(orc):
    st = np.zeros(21)
    st[0], st[1:6] = 150.0, [10.0, 5.0, 0.2, 0.3, -1.0]
    rng = np.random.default_rng(0)
    A = rng.normal(size=(5, 5))
    C = A @ A.T + np.eye(5)
    st[6:] = [C[i, j] for i in range(5) for j in range(i + 1)]
    ok, a = orc.rot64(st, COS20, SIN20, KB64)
    ok2, b = orc.rot64(a, COS20, -SIN20, KB64)
    assert ok and ok2
    np.testing.assert_allclose(b[:6], st[:6], rtol=0, atol=1e-12)
    np.testing.assert_allclose(b[6:], st[6:], rtol=1e-9, atol=1e-9)


def test_update64_equals_information_form(orc):
    """Posterior precision = prior precision + H^T V^-1 H, and posterior mean
    solves C+^-1 p+ = C^-1 p + H^T V^-1 m (a different formula from the gain form)."""
    rng = np.random.default_rng(1)
    for _ in range(20):
        A = rng.normal(size=(5, 5))
        C = A @ A.T + 0.1 * np.eye(5)
        p = rng.normal(size=5)
        st = np.zeros(21)
        st[1:6] = p
        st[6:] = [C[i, j] for i in range(5) for j in range(i + 1)]
        m = rng.normal(size=2)
        vy, vz = 0.01, 0.0225
        ok, out, chi2 = orc.update64(st, m[0], m[1], vy, vz)
        assert ok
        Cp = np.zeros((5, 5))
        q = 0
        for i in range(5):
            for j in range(i + 1):
                Cp[i, j] = Cp[j, i] = out[6 + q]
                q += 1
        H = np.zeros((2, 5))
        H[0, 0] = H[1, 1] = 1
        Vi = np.diag([1 / vy, 1 / vz])
        np.testing.assert_allclose(np.linalg.inv(Cp), np.linalg.inv(C) + H.T @ Vi @ H, rtol=1e-8, atol=1e-8)
        rhs = np.linalg.solve(C, p) + H.T @ Vi @ m
        np.testing.assert_allclose(np.linalg.solve(Cp, out[1:6]), rhs, rtol=1e-8, atol=1e-8)
        # predicted chi2 = min over x of (x-p)C^-1(x-p) + (m-Hx)V^-1(m-Hx)
        x = out[1:6]
        direct = (x - p) @ np.linalg.solve(C, x - p) + (m - H @ x) @ Vi @ (m - H @ x)
        assert abs(chi2 - direct) < 1e-8 * max(1.0, chi2)


def test_update32_close_to_update64(orc):
    rng = np.random.default_rng(2)
    for _ in range(20):
        A = rng.normal(size=(5, 5))
        C = A @ A.T + 0.1 * np.eye(5)
        st = np.zeros(21)
        st[1:6] = rng.normal(size=5)
        st[6:] = [C[i, j] for i in range(5) for j in range(i + 1)]
        m = rng.normal(size=2)
        ok, o64, c64 = orc.update64(st, m[0], m[1], 0.01, 0.0225)
        ok2, o32, c32 = orc.update32(st.astype(np.float32), np.float32(m[0]), np.float32(m[1]),
                                     np.float32(0.01), np.float32(0.0225))
        assert ok and ok2
        np.testing.assert_allclose(o32[1:], o64[1:], rtol=2e-4, atol=2e-5)
        assert abs(c32 - c64) < 1e-4 * max(1, c64)


def test_update32_chi2_cut_leaves_state_untouched(orc):
    st = np.zeros(21, np.float32)
    st[6 + 0] = st[6 + 2] = 0.01
    st[6 + 5] = st[6 + 9] = st[6 + 14] = 1.0
    ok, out, chi2 = orc.update32(st, np.float32(5.0), np.float32(0.0), np.float32(0.01), np.float32(0.01),
                                 np.float32(10.0))
    assert not ok and chi2 > 10
    np.testing.assert_array_equal(out, st)


def test_prop32_jacobian_close_to_prop64(orc):
    """The binary32 transport (arcsine series) agrees with the exact FP64 one."""
    kb32 = np.float32(orc.KB_C) * np.float32(BZ)
    rng = np.random.default_rng(3)
    for _ in range(50):
        st = np.zeros(21)
        st[0] = rng.uniform(85, 247)
        st[1:6] = [rng.uniform(-20, 20), rng.uniform(-200, 200), rng.uniform(-0.7, 0.7),
                   rng.uniform(-1, 1), rng.uniform(-5, 5)]
        A = rng.normal(size=(5, 5)) * 0.1
        C = A @ A.T + 0.01 * np.eye(5)
        st[6:] = [C[i, j] for i in range(5) for j in range(i + 1)]
        dx = rng.choice([1.07, -1.07, 3.2, -2.1])
        ok64, o64 = orc.prop64(st, st[0] + dx, float(kb32))
        ok32, o32 = orc.prop32(st.astype(np.float32), np.float32(st[0] + dx), kb32)
        assert ok64 == ok32
        if ok64:
            np.testing.assert_allclose(o32[1:], o64[1:], rtol=1e-4, atol=2e-5)


def _straight_line_clusters(rng, n=60, snp=0.3, tgl=0.6, y0=2.0, z0=-30.0, smear=1.0):
    x = np.asarray(tpcgen.row_x_f32()[20:20 + n], np.float64)
    tanp = snp / math.sqrt(1 - snp * snp)
    cosp = math.sqrt(1 - snp * snp)
    y = y0 + (x - x[0]) * tanp + rng.normal(0, 0.1 * smear, n)
    z = z0 + (x - x[0]) / cosp * tgl + rng.normal(0, 0.15 * smear, n)
    return x, y, z


def _b0_fit_vs_lstsq(orc, rng, smear):
    """B = 0: Kalman fit (diffuse start, five passes) vs the weighted
    least-squares line y = a + b x, z = c + e x solved by numpy lstsq;
    tan(lambda) = e cos(phi)."""
    params = None
    snp, tgl = rng.uniform(-0.5, 0.5), rng.uniform(-1, 1)
    x, y, z = _straight_line_clusters(rng, snp=snp, tgl=tgl, smear=smear)
    st0 = np.zeros(21)
    st0[0] = x[-1]
    st0[1:6] = [y[-1], z[-1], snp + 0.05, tgl - 0.1, 0.0]
    st0[6 + 5] = st0[6 + 9] = 1e6          # diffuse start for the angles
    st0[6 + 14] = 1.0
    ok, st, chi2 = orc.fit64(np.zeros(x.size, np.int32), x, y, z, st0, 0.0, n_passes=5, params=params)
    assert ok and st[0] == x[0]
    A = np.stack([np.ones_like(x), x - x[0]], 1)
    (a, b), ry, *_ = np.linalg.lstsq(A / 0.1, y / 0.1, rcond=None)
    (c, e), rz, *_ = np.linalg.lstsq(A / 0.15, z / 0.15, rcond=None)
    cphi = 1 / math.sqrt(1 + b * b)
    lsq = np.array([a, c, b * cphi, e * cphi])
    truth_dist = np.abs(lsq - [y[0] * 0 + 2.0, -30.0, snp, tgl])
    return st[1:5] - lsq, chi2, float(ry[0] + rz[0]), truth_dist


def test_fit64_straight_line_at_zero_field_equals_least_squares(orc):
    """Small measurement noise (weights still sigma_y = 0.1, sigma_z = 0.15 cm):
    the fit reproduces the least-squares solution, which differs from the
    generating line by far more than the tolerance."""
    rng = np.random.default_rng(4)
    for _ in range(5):
        d, chi2, chi2_ls, tdist = _b0_fit_vs_lstsq(orc, rng, smear=1e-3)
        assert np.all(np.abs(d[:2]) < 2e-8), d
        assert np.all(np.abs(d[2:]) < 2e-10), d
        assert chi2 == pytest.approx(chi2_ls, rel=1e-5)
        assert tdist.max() > 100 * np.abs(d).max()


def test_fit64_straight_line_realistic_noise_close_to_least_squares(orc):
    """With sigma-sized noise the extended filter, linearised around its
    running estimate, differs from batch least squares only at second order
    (a few percent of sigma)."""
    rng = np.random.default_rng(5)
    for _ in range(10):
        d, chi2, chi2_ls, _ = _b0_fit_vs_lstsq(orc, rng, smear=1.0)
        assert np.all(np.abs(d[:2]) < 0.1 * np.array([0.1, 0.15])), d
        assert np.all(np.abs(d[2:]) < 5e-4), d
        assert chi2 == pytest.approx(chi2_ls, rel=1e-2)


def test_fit64_recovers_noise_free_helices(orc):
    """Exact generator crossings (no smearing): after three passes the fit
    returns the true parameters at the innermost cluster and chi2 ~ 0,
    including tracks spanning several sectors (frame rotations)."""
    ev = tpcgen.central_event(seed=12, n_tracks=120)
    n_multi = 0
    for t in range(ev.trk_pt.size):
        idx = np.where(ev.label == t)[0]
        if idx.size < 40:
            continue
        idx = idx[np.argsort(ev.true_s[idx])]
        secs = ev.sector[idx].astype(np.int32)
        n_multi += np.unique(secs).size > 1
        x = ev.row_x[ev.row[idx]].astype(np.float64)
        st0 = np.zeros(21)
        st0[0] = x[-1]
        tr = track_truth_state(ev, idx[-1])
        st0[1:6] = tr + [0.3, -0.2, 0.01, -0.01, 0.1 * (1 + abs(tr[4]))]
        st0[6 + 5] = st0[6 + 9] = 0.25
        st0[6 + 14] = 100.0
        ok, st, chi2 = orc.fit64(secs, x, ev.true_y[idx], ev.true_z[idx], st0, KB64)
        assert ok
        exp = track_truth_state(ev, idx[0])
        np.testing.assert_allclose(st[1:6], exp, rtol=1e-8, atol=1e-8)
        assert chi2 < 1e-6          # residuals below 1e-5 sigma
    assert n_multi >= 10


def test_oracle_tracks_statistics_and_covariance(orc):
    """On smeared events: chi2/ndf ~ 1, pulls of the refitted parameters
    against truth ~ N(0, 1), every output covariance symmetric positive definite."""
    ev = tpcgen.central_event(seed=13, n_tracks=800)
    r = orc.track_event(ev)
    pulls = []
    for t in range(r.n_tracks):
        if r.tr_status[t] != 0:
            continue
        assert is_spd(r.tr_c[t])
        cl = r.track_clusters(t)
        c0 = cl[0]
        v, k = np.unique(ev.label[cl], return_counts=True)
        # only tracks whose innermost cluster belongs to the majority particle
        if ev.label[c0] != v[np.argmax(k)] or ev.label[c0] < 0 or r.tr_nclus[t] < 60:
            continue
        c = r.tr_c[t]
        sig = np.sqrt([c[0], c[2], c[5], c[9], c[14]])
        # compare at the innermost cluster's plane with the exact crossing there
        pulls.append((r.tr_p[t] - track_truth_state(ev, c0)) / sig)
    pulls = np.array(pulls)
    assert len(pulls) > 300
    rms = np.sqrt(np.mean(pulls ** 2, axis=0))
    assert np.all(rms > 0.85) and np.all(rms < 1.2), rms
    ok = r.tr_status == 0
    ratio = r.tr_chi2[ok].sum() / r.tr_ndf[ok].sum()
    assert 0.9 < ratio < 1.1, ratio


def test_covariance_stays_spd_after_every_fp32_and_fp64_step(orc):
    """Step the binary32 and binary64 filters along long tracks (including low-pT
    ones) and check positive definiteness after every propagation and update."""
    ev = tpcgen.central_event(seed=14, n_tracks=150)
    kb32 = np.float32(orc.KB_C) * np.float32(BZ)
    n = 0
    for run in _sector_runs(ev, min_len=60, max_tracks=40):
        s32 = np.zeros(21, np.float32)
        s64 = np.zeros(21)
        c0 = run[0]
        for s in (s32, s64):
            s[0] = ev.row_x[ev.row[c0]]
            s[1:6] = [ev.y[c0], ev.true_z[c0], ev.true_snp[c0], 0.0, 0.0]
            s[6 + 0], s[6 + 2], s[6 + 5], s[6 + 9], s[6 + 14] = 0.01, 0.0225, 0.25, 0.25, 100.0
        for cl in run[1:]:
            x = ev.row_x[ev.row[cl]]
            ok32, s32 = orc.prop32(s32, x, kb32)
            ok64, s64 = orc.prop64(s64, float(x), float(kb32))
            if not (ok32 and ok64):
                break
            assert is_spd(s32[6:].astype(np.float64)) and is_spd(s64[6:])
            _, s32, _ = orc.update32(s32, ev.y[cl], np.float32(ev.true_z[cl]), np.float32(0.01),
                                     np.float32(0.0225))
            _, s64, _ = orc.update64(s64, float(ev.y[cl]), float(ev.true_z[cl]), 0.01, 0.0225)
            assert is_spd(s32[6:].astype(np.float64)) and is_spd(s64[6:])
            n += 1
    assert n > 1000
