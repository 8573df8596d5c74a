"""Closed-loop calibration on the GPU (tpc_calib_fit): from the nominal
calibration, theta minimising the summed chi2 of the selected tracks plus the
spline prior, on a calibration frame generated with v_drift +0.3 %, t0 =
0.2 us and a 36 x 8 x 8 x 2 spline distortion map.  The calibration problem
is the oracle's own (oracle.track_event's tracks, their generator-truth
collision times, the oracle's selection, the matched inner tracks' dip angles
from generator truth smeared by 3e-4).

Checks: the recovered drift velocity and t0 against the generator's; the
calibrated cluster positions of the used tracks against those of the true
calibration (the part of the map the tracks see); the binary64 oracle finds
the result a minimum of the same objective: no lower than at the true
calibration and with a gradient far below the one at the start."""
import numpy as np
import pytest

import tpcgen

pytestmark = pytest.mark.gpu

PRIOR_SIGMA = 0.3


@pytest.fixture(scope="module")
def fitted():
    import torch

    import oracle
    import paper_1905_05515_b300 as tpc
    ev = tpcgen.calib_frame(seed=5, n_collisions=4)
    r = oracle.track_event(ev)
    tc = tpcgen.track_collision_time(ev, r.tr_off, r.tr_clus)
    ot = oracle.calib_tracks_of(ev, r, tc)
    tg = tpcgen.track_dip_angle(ev, r.tr_off, r.tr_clus)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    cl = (t(ev.sector), t(ev.row), t(ev.y), t(ev.zt))
    gpu = tpc.CalibRefit(t(ot.sector), t(ot.x), t(ot.param), t(ot.off), t(ot.clus), t(ot.tcoll), *cl, ev.row_x,
                         bz=ev.bz, v_nominal=ev.v_drift, tgl_ext=t(tg))
    th0 = tpc.calib.nominal_theta(ev.v_drift)
    th, rep = gpu.fit(th0, prior_sigma=PRIOR_SIGMA)
    cal = ev.calib
    th_true = np.concatenate([[cal["v_drift"], cal["t0"]], cal["spline"].ravel()])
    return ev, ot, tg, th0.cpu().numpy().astype(np.float64), th.cpu().numpy().astype(np.float64), th_true, rep


def _objective(orc_tracks, th, t_used, tgl_used, grad=True):
    import oracle
    import dataclasses
    tr = dataclasses.replace(orc_tracks, tcoll=t_used)
    c, u, g = oracle.calib(tr, th, grad=grad, tgl_ext=tgl_used)
    F = c[u].sum() + ((th[2:] / PRIOR_SIGMA) ** 2).sum()
    if g is not None:
        g = g.copy()
        g[2:] += 2 * th[2:] / PRIOR_SIGMA ** 2
    return F, g


def test_fit_recovers_drift_velocity_and_t0(fitted):
    ev, ot, tg, th0, th, th_true, rep = fitted
    assert rep["rounds"] == 3 and rep["tracks"] > 0.8 * np.isfinite(ot.tcoll).sum()
    assert rep["f_final"] < 0.7 * rep["f_start"]
    assert abs(th[0] / th_true[0] - 1) < 3e-4, th[0] / th_true[0] - 1      # a tenth of the +0.3 % offset
    assert abs(th[1] - th_true[1]) < 0.02, th[1]                            # a tenth of the 0.2 us shift


def test_fit_recovers_the_cluster_corrections(fitted):
    import oracle
    ev, ot, tg, th0, th, th_true, rep = fitted
    tu = rep["t_used"].cpu().numpy()
    use = np.isfinite(tu)
    idx = np.concatenate([ot.clus[ot.off[k]:ot.off[k + 1]] for k in np.nonzero(use)[0]])
    tcc = np.repeat(tu[use], np.diff(ot.off)[use])
    ref = oracle.calib_measure(ot, th_true, idx, tcc)
    err = [np.sqrt(((a - b) ** 2).mean()) for a, b in zip(oracle.calib_measure(ot, th, idx, tcc), ref)]
    err0 = [np.sqrt(((a - b) ** 2).mean()) for a, b in zip(oracle.calib_measure(ot, th0, idx, tcc), ref)]
    assert err[0] < 0.35 * err0[0] and err[1] < 0.2 * err0[1], (err, err0)


def test_fit_is_a_minimum_for_the_oracle(fitted):
    ev, ot, tg, th0, th, th_true, rep = fitted
    tu = rep["t_used"].cpu().numpy()
    gu = rep["tgl_used"].cpu().numpy()
    F_fit, g_fit = _objective(ot, th, tu, gu)
    F_true, _ = _objective(ot, th_true, tu, gu, grad=False)
    F_0, g_0 = _objective(ot, th0, tu, gu)
    assert F_fit <= F_true * (1 + 1e-5), (F_fit, F_true)
    assert F_fit == pytest.approx(rep["f_final"], rel=1e-3)
    D = np.full(th.size, PRIOR_SIGMA)
    D[0], D[1] = 0.01, 0.1
    assert np.linalg.norm(D * g_fit) < 1e-3 * np.linalg.norm(D * g_0)
