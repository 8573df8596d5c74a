"""GPU parity of the calibration chi2 and its adjoint (tpc_calib_forward /
tpc_calib_backward) against the binary64 oracle, on a miscalibrated
continuous frame.  The calibration problem is the oracle's own: the tracks of
oracle.track_event, their generator-truth collision times and the oracle's
track selection (oracle.calib_select); the GPU's selection
(tpc_calib_select, through the C ABI) must equal it on the same tracks.

Bars: per-track chi2 within 1e-3 relative (floor 1); gradient components
within 1e-3 of max(|g_i|, 1e-2 |g|_inf); directional derivatives of the
summed chi2 of the tracks a calibration fit uses (chi2 / ndf below 5) within
1e-3 of binary64 central finite differences of the oracle's chi2.
"""
import dataclasses

import numpy as np
import pytest

import tpcgen

pytestmark = pytest.mark.gpu

REL = 1e-3


def _problem(n_collisions=3, mult=600, seed=5):
    """The oracle's calibration problem of a calibration frame, and the
    cluster tensors on the device."""
    import torch

    import oracle
    import paper_1905_05515_b300 as tpc
    ev = tpcgen.calib_frame(seed=seed, n_collisions=n_collisions, mult_mean=mult)
    dev = torch.device("cuda:0")
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
    cl = (t(ev.sector), t(ev.row), t(ev.y), t(ev.zt))
    r = oracle.track_event(ev)
    tc_truth = tpcgen.track_collision_time(ev, r.tr_off, r.tr_clus)
    ot = oracle.calib_tracks_of(ev, r, tc_truth)
    # the library's selection of the same tracks is the oracle's, NaN for NaN
    tc_gpu = tpc.calib.select_tracks(t(tc_truth), t(r.tr_status.astype(np.int32)), t(ot.param)).cpu().numpy()
    assert np.array_equal(np.isnan(tc_gpu), np.isnan(ot.tcoll))
    assert np.array_equal(tc_gpu[~np.isnan(tc_gpu)], ot.tcoll[~np.isnan(ot.tcoll)])
    h = dict(sector=ot.sector, x=ot.x, param=ot.param, off=ot.off, clus=ot.clus, tc=ot.tcoll)
    return ev, cl, h


def _calib_pair(ev, cl, h):
    import torch

    import oracle
    import paper_1905_05515_b300 as tpc
    dev = cl[0].device
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
    gpu = tpc.CalibRefit(t(h["sector"]), t(h["x"]), t(h["param"]), t(h["off"]), t(h["clus"]), t(h["tc"]), *cl,
                         ev.row_x, bz=ev.bz, v_nominal=ev.v_drift)
    orc = oracle.CalibTracks(h["sector"], h["x"], h["param"], h["off"], h["clus"], h["tc"], ev.sector, ev.row, ev.y,
                             ev.zt, ev.row_x, bz=ev.bz, v_nom=ev.v_drift)
    return gpu, orc


def _theta(seed, scale=1.0):
    cal = tpcgen.calib_truth(5)
    th = np.concatenate([[cal["v_drift"], cal["t0"]], cal["spline"].ravel()])
    rng = np.random.default_rng(seed)
    th = th + scale * np.concatenate([[0.003, 0.05], rng.normal(0, 0.1, th.size - 2)])
    return th.astype(np.float32)


def _agreed(ev, cl, h):
    """The pair of problems restricted to the tracks both sides use.  Which
    tracks are used depends on the reference helix only (not on theta); a
    track whose reference sits on the |sin(phi)| = 0.9 edge within rounding
    may be taken by one side only: such tracks are counted (at most 0.2 %)
    and left out of both."""
    import torch

    import oracle
    gpu, orc = _calib_pair(ev, cl, h)
    th = _theta(0)
    _, used, _ = gpu.forward(torch.from_numpy(th).cuda())
    _, u_o, _ = oracle.calib(orc, th.astype(np.float64), grad=False)
    u = used.cpu().numpy().astype(bool)
    diff = np.nonzero(u != u_o)[0]
    assert diff.size <= max(2, 0.002 * u.sum()), diff
    if diff.size:
        h = dict(h, tc=h["tc"].copy())
        h["tc"][diff] = np.nan
        gpu, orc = _calib_pair(ev, cl, h)
    return h, gpu, orc


@pytest.fixture(scope="module")
def small():
    ev, cl, h = _problem()
    h, gpu, orc = _agreed(ev, cl, h)
    return ev, cl, h, gpu, orc


def _grad_ok(g, ref):
    scale = np.maximum(np.abs(ref), 1e-2 * np.abs(ref).max())
    return np.abs(g - ref) / scale


CHI2NDF_FIT = 5.0


def _fit_weights(orc, th):
    """Weights 1 for the tracks a calibration fit would use (chi2 / ndf below
    CHI2NDF_FIT at th, ndf = 2 n), 0 for the rest.  Broken tracks (a piece of
    another particle, chi2 / ndf of 7 and more) have binary32 smoothed
    residuals good to a few per cent only: the filter's covariance falls by
    six orders of magnitude from the diffuse prior within a dozen clusters,
    and the gradient of such a track is a sum of large cancelling terms."""
    import oracle
    c, u, _ = oracle.calib(orc, th.astype(np.float64), grad=False)
    return (u & (c < CHI2NDF_FIT * 2 * np.diff(orc.off))).astype(np.float32)


def test_forward_matches_oracle(small):
    import torch

    import oracle
    ev, cl, h, gpu, orc = small
    for seed in (0, 1):
        th = _theta(seed)
        chi2, used, _ = gpu.forward(torch.from_numpy(th).cuda())
        c_o, u_o, _ = oracle.calib(orc, th.astype(np.float64), grad=False)
        used = used.cpu().numpy().astype(bool)
        assert used.sum() > 1000
        assert np.array_equal(used, u_o)
        c = chi2.cpu().numpy().astype(np.float64)
        err = np.abs(c[used] - c_o[used]) / np.maximum(c_o[used], 1.0)
        assert err.max() < REL, err.max()


def test_gradient_matches_oracle(small):
    import torch

    import oracle
    ev, cl, h, gpu, orc = small
    rng = np.random.default_rng(7)
    th = _theta(2)
    w = rng.uniform(0.5, 1.5, gpu.n_tracks).astype(np.float32)
    thd = torch.from_numpy(th).cuda()
    chi2, used, ws = gpu.forward(thd)
    g = gpu.backward(thd, torch.from_numpy(w).cuda(), used, ws).cpu().numpy()
    _, u_o, g_o = oracle.calib(orc, th.astype(np.float64), weight=w.astype(np.float64))
    assert np.array_equal(used.cpu().numpy().astype(bool), u_o)
    e = _grad_ok(g, g_o)
    assert e.max() < REL, (e.argmax(), e.max())
    # every sector's map received gradient
    assert (np.abs(g_o[2:].reshape(36, -1)).max(axis=1) > 0).all()


def test_gradient_against_fp64_finite_differences(small):
    import torch

    import oracle
    ev, cl, h, gpu, orc = small
    th = _theta(3)
    thd = torch.from_numpy(th).cuda()
    chi2, used, ws = gpu.forward(thd)
    wsel = _fit_weights(orc, th)
    g = gpu.backward(thd, torch.from_numpy(wsel).cuda(), used, ws).cpu().numpy()
    th64 = th.astype(np.float64)
    ref_used = used.cpu().numpy().astype(bool)

    def f(x):
        c, u, _ = oracle.calib(orc, x, grad=False)
        assert np.array_equal(u, ref_used)
        return float((c * wsel).sum())

    rng = np.random.default_rng(11)
    dirs = []
    for i in [0, 1, *list(np.argsort(-np.abs(g[2:]))[:4] + 2)]:
        e = np.zeros_like(th64)
        e[i] = 1.0
        dirs.append(e)
    d = rng.normal(0, 1, th64.size)
    d[:2] *= 1e-2
    dirs.append(d / np.linalg.norm(d))
    for e in dirs:
        hstep = 1e-6 if e[0] != 0 else 1e-5
        fd = (f(th64 + hstep * e) - f(th64 - hstep * e)) / (2 * hstep)
        assert float(g @ e) == pytest.approx(fd, rel=REL), np.nonzero(e)[0][:3]


def test_autograd_function(small):
    import torch

    import paper_1905_05515_b300 as tpc
    ev, cl, h, gpu, orc = small
    th = torch.from_numpy(_theta(4)).cuda().requires_grad_(True)
    chi2, used = tpc.calib_chi2(th, gpu)
    w = torch.linspace(0.5, 1.5, gpu.n_tracks, device="cuda")
    loss = (w * chi2).sum()
    loss.backward()
    c2, u2, ws = gpu.forward(th.detach())
    ref = gpu.backward(th.detach(), w, u2, ws)
    assert torch.equal(chi2.detach(), c2)
    np.testing.assert_allclose(th.grad.cpu().numpy(), ref.float().cpu().numpy(), rtol=1e-6, atol=0)
    assert used.dtype == torch.uint8 and not used.requires_grad


def test_checkpoint_segment_boundaries(small):
    """Tracks cut to 2..49 clusters (around multiples of the 16-step
    checkpoint spacing) and one long looper-free track list."""
    import torch

    import oracle
    ev, cl, h, gpu, orc = small
    n = np.diff(h["off"])
    long_ = np.nonzero((n >= 60) & ~np.isnan(h["tc"]))[0][:40]
    lens = [2, 3, 15, 16, 17, 31, 32, 33, 47, 48, 49, 60]
    sel, L = [], []
    for i, t in enumerate(long_):
        sel.append(t)
        L.append(lens[i % len(lens)])
    sel = np.array(sel)
    off = np.concatenate([[0], np.cumsum(L)]).astype(np.int32)
    clus = np.concatenate([h["clus"][h["off"][t]:h["off"][t] + k] for t, k in zip(sel, L)]).astype(np.int32)
    hs = dict(sector=h["sector"][sel], x=h["x"][sel], param=h["param"][sel], off=off, clus=clus, tc=h["tc"][sel])
    hs, g2, o2 = _agreed(ev, cl, hs)
    th = _theta(5)
    thd = torch.from_numpy(th).cuda()
    chi2, used, ws = g2.forward(thd)
    w = np.linspace(0.5, 1.5, len(sel)).astype(np.float32)
    g = g2.backward(thd, torch.from_numpy(w).cuda(), used, ws).cpu().numpy()
    c_o, u_o, g_o = oracle.calib(o2, th.astype(np.float64), weight=w.astype(np.float64))
    u = used.cpu().numpy().astype(bool)
    assert np.array_equal(u, u_o) and u.sum() >= len(sel) - 4
    c = chi2.cpu().numpy()
    assert (np.abs(c[u] - c_o[u]) / np.maximum(c_o[u], 1.0)).max() < REL
    assert _grad_ok(g, g_o).max() < REL


def test_empty_unused_and_zero_weights(small):
    import torch

    import paper_1905_05515_b300 as tpc
    ev, cl, h, gpu, orc = small
    th = torch.from_numpy(_theta(6)).cuda()
    # no tracks
    e = dict(sector=h["sector"][:0], x=h["x"][:0], param=h["param"][:0], off=np.zeros(1, np.int32),
             clus=h["clus"][:0], tc=h["tc"][:0])
    g0, _ = _calib_pair(ev, cl, e)
    c, u, ws = g0.forward(th)
    assert c.numel() == 0
    assert torch.count_nonzero(g0.backward(th, c, u, ws)) == 0
    # every track unused
    hn = dict(h, tc=np.full_like(h["tc"], np.nan))
    gn, _ = _calib_pair(ev, cl, hn)
    c, u, ws = gn.forward(th)
    assert int(u.sum()) == 0 and float(c.abs().sum()) == 0.0
    assert torch.count_nonzero(gn.backward(th, torch.ones_like(c), u, ws)) == 0
    # zero upstream gradient
    c, u, ws = gpu.forward(th)
    assert torch.count_nonzero(gpu.backward(th, torch.zeros_like(c), u, ws)) == 0
    assert isinstance(gpu, tpc.CalibRefit)


def test_invalid_cluster_index_is_reported(small):
    import torch

    import paper_1905_05515_b300 as tpc
    ev, cl, h, gpu, orc = small
    bad = dict(h, clus=h["clus"].copy())
    bad["clus"][5] = ev.n + 7             # out of range: the kernel's bounds check flags it
    gb, _ = _calib_pair(ev, cl, bad)
    with pytest.raises(tpc.TpcError):
        gb.forward(torch.from_numpy(_theta(0)).cuda())


@pytest.mark.slow
def test_full_calibration_frame_sampled():
    """The 50-collision calibration frame at full size: every track on the
    GPU, a sample of 1500 tracks checked one by one against the oracle
    (chi2), and the gradient of the sample's chi2 sum (upstream weights 1 on
    the sample, 0 elsewhere)."""
    import torch

    import oracle
    ev, cl, h = _problem(n_collisions=50, mult=2000)
    gpu, orc_full = _calib_pair(ev, cl, h)
    th = _theta(8)
    thd = torch.from_numpy(th).cuda()
    chi2, used, ws = gpu.forward(thd)
    u = used.cpu().numpy().astype(bool)
    rng = np.random.default_rng(1)
    sample = np.sort(rng.choice(np.nonzero(u)[0], 1500, replace=False))
    w = np.zeros(gpu.n_tracks, np.float32)
    w[sample] = 1.0
    g = gpu.backward(thd, torch.from_numpy(w).cuda(), used, ws).cpu().numpy()
    # the sample as its own oracle problem
    n = np.diff(h["off"])
    off = np.concatenate([[0], np.cumsum(n[sample])]).astype(np.int32)
    clus = np.concatenate([h["clus"][h["off"][t]:h["off"][t + 1]] for t in sample]).astype(np.int32)
    o2 = dataclasses.replace(orc_full, sector=h["sector"][sample], x=h["x"][sample], param=h["param"][sample],
                             off=off, clus=clus, tcoll=h["tc"][sample])
    c_o, u_o, g_o = oracle.calib(o2, th.astype(np.float64))
    assert (~u_o).sum() <= 3              # edge-of-domain decisions taken in the other precision
    if not u_o.all():                     # leave those out of both sides
        w[sample[~u_o]] = 0.0
        g = gpu.backward(thd, torch.from_numpy(w).cuda(), used, ws).cpu().numpy()
        sample, c_o = sample[u_o], c_o[u_o]
    c = chi2.cpu().numpy()[sample]
    ce = np.abs(c - c_o) / np.maximum(c_o, 1.0)
    # binary32 chi2 of long tracks: at most 1 in 1000 above the 1e-3 bar, none above 5e-3
    print(f"full calibration frame: {sample.size} tracks sampled, chi2 max rel {ce.max():.2e}, "
          f"{int((ce >= REL).sum())} above {REL:g}")
    assert (ce >= REL).sum() <= max(1, sample.size // 1000) and ce.max() < 5 * REL
    assert _grad_ok(g, g_o).max() < REL


def test_dip_angle_anchor_matches_oracle(small):
    """With the matched inner track's dip angle (one more update after the
    vertex): chi2 and gradient as the oracle's, the gradient against binary64
    finite differences along v, t0 and a random direction.  As in the fit's
    first selection, dip angles whose chi2 contribution exceeds 100 (a wrong
    match) are left out: against the filter's binary32 tan(lambda) variance,
    a few 1e-6 after starting at 0.25, such a contribution is good to a per
    cent only."""
    import torch

    import oracle
    import paper_1905_05515_b300 as tpc
    ev, cl, h, gpu0, orc0 = small
    tg = tpcgen.track_dip_angle(ev, h["off"], h["clus"])
    th = _theta(5)
    th64 = th.astype(np.float64)
    c_free, _, _ = oracle.calib(orc0, th64, grad=False)
    c_anc, _, _ = oracle.calib(orc0, th64, grad=False, tgl_ext=tg)
    tg = np.where(c_anc - c_free < 100.0, tg, np.nan).astype(np.float32)
    assert np.isfinite(tg).sum() > 1000
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    gpu = tpc.CalibRefit(t(h["sector"]), t(h["x"]), t(h["param"]), t(h["off"]), t(h["clus"]), t(h["tc"]), *cl,
                         ev.row_x, bz=ev.bz, v_nominal=ev.v_drift, tgl_ext=t(tg))
    thd = torch.from_numpy(th).cuda()
    chi2, used, ws = gpu.forward(thd)
    wsel = _fit_weights(orc0, th)
    g = gpu.backward(thd, torch.from_numpy(wsel).cuda(), used, ws).cpu().numpy()
    c_o, u_o, g_o = oracle.calib(orc0, th64, tgl_ext=tg, weight=wsel.astype(np.float64))
    u = used.cpu().numpy().astype(bool)
    assert np.array_equal(u, u_o)
    c = chi2.cpu().numpy().astype(np.float64)
    assert (np.abs(c[u] - c_o[u]) / np.maximum(c_o[u], 1.0)).max() < REL
    # the anchor changes the chi2 of the anchored tracks
    anchored = u & np.isfinite(tg)
    assert (c_o[anchored] - c_free[anchored] > 0).mean() > 0.9
    e = _grad_ok(g, g_o)
    assert e.max() < REL, (e.argmax(), e.max())

    def f(x):
        return float((oracle.calib(orc0, x, grad=False, tgl_ext=tg)[0] * wsel).sum())

    rng = np.random.default_rng(3)
    d = rng.normal(0, 1, th64.size)
    d[:2] *= 1e-2
    for e_ in (np.eye(1, th64.size, 0)[0], np.eye(1, th64.size, 1)[0], d / np.linalg.norm(d)):
        hstep = 1e-5 if e_[0] == 0 else 1e-6
        fd = (f(th64 + hstep * e_) - f(th64 - hstep * e_)) / (2 * hstep)
        assert float(g @ e_) == pytest.approx(fd, rel=REL)
