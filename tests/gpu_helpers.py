"""Run the CUDA tracker through its C ABI on a tpcgen.Event and bring the
results to the host, and compare them with the oracle."""
import numpy as np

PARAM_FLOOR = np.array([1.0, 1.0, 1e-2, 1e-2, 1e-2])   # cm, cm, -, -, 1/GeV


def run_gpu(ev, params=None, debug=True, capacity_tracks=None):
    import torch

    import paper_1905_05515_b300 as tpc
    dev = torch.device("cuda:0")
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
    trk = tpc.Tracker(max(ev.n, 1), ev.row_x, n_sectors=ev.n_sectors, z_max=ev.z_max, continuous=ev.continuous,
                      params=params, debug=debug, capacity_tracks=capacity_tracks)
    res = trk.track(t(ev.sector), t(ev.row), t(ev.y), t(ev.zt), bz=ev.bz, v_drift=ev.v_drift)
    torch.cuda.synchronize()
    out = {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in vars(res).items() if v is not None}
    T = res.n_tracks
    off = out["clus_offset"]
    out["clus_index"] = out["clus_index"][: int(off[-1]) if T else 0]
    out["tracklets"] = trk.export_tracklets()
    return out


def param_rel_err(g, o):
    """|gpu - oracle| / max(|oracle|, floor) per parameter."""
    return np.abs(g.astype(np.float64) - o) / np.maximum(np.abs(o), PARAM_FLOOR)


def compare_decisions(ev, g, r):
    """Bit-exact comparison of every integer / binary32 decision result.
    Returns a dict of mismatch counts (all must be zero)."""
    bad = {}
    bad["z"] = int((g["z"].view(np.uint32) != r.z.view(np.uint32)).sum())
    for k_g, k_o in (("link_up_raw", "up_raw"), ("link_dn_raw", "dn_raw"), ("link_up", "up"), ("link_dn", "dn")):
        bad[k_g] = int((g[k_g] != getattr(r, k_o)).sum())
    bad["is_start"] = int((g["is_start"] != r.is_start).sum())
    tk = g["tracklets"]
    bad["n_tracklets"] = abs(int(tk["start"].size) - int(r.trk_start.size))
    if tk["start"].size == r.trk_start.size:
        bad["trk_start"] = int((tk["start"] != r.trk_start).sum())
        bad["trk_nhits"] = int((tk["nhits"] != r.trk_nhits).sum())
        bad["trk_kept"] = int((tk["kept"] != r.trk_kept).sum())
        nh = 0
        for t in range(r.trk_start.size):
            h = r.tracklet_hits(t)
            if not np.array_equal(tk["hits"][t, : h.size], h):
                nh += 1
        bad["trk_hits"] = nh
        bad["trk_top"] = int((tk["top"].view(np.uint32) != r.trk_top.view(np.uint32)).any(axis=1).sum())
        bad["trk_bot"] = int((tk["bot"].view(np.uint32) != r.trk_bot.view(np.uint32)).any(axis=1).sum())
    bad["n_tracks"] = abs(int(g["n_tracks"]) - r.n_tracks)
    if g["n_tracks"] == r.n_tracks:
        bad["clus_offset"] = int((g["clus_offset"] != r.tr_off).sum())
        if g["clus_index"].size == r.tr_clus.size:
            bad["clus_index"] = int((g["clus_index"] != r.tr_clus).sum())
        else:
            bad["clus_index"] = -1
        bad["sector"] = int((g["sector"] != r.tr_sector).sum())
    bad["assign"] = int((g["assign"] != r.assign).sum())
    bad["n_rejected"] = abs(int(g["n_rejected"]) - int(r.rejected.sum()))
    return bad


CHI2NDF_FIT = 100.0   # above this the track is not a fit of one helix (mis-merged looper legs)
PARAM_TOL = 1e-4      # parameters, relative (the benchmark spec)
CHI2_TOL = 1e-3       # chi2, relative (the benchmark spec)


def compare_fit(g, r):
    """Refit parameters and chi2 against the binary64 oracle, as separately
    reported numbers.

    * covered: tracks both sides fitted whose oracle chi2/ndf is below
      CHI2NDF_FIT (fits of one helix).  On these the bar is relative:
      param_rel = |dp| / max(|p|, scale) with the scales 1 cm, 1 cm, 0.01,
      0.01, 0.01 GeV^-1 of y, z, sin phi, tan lambda, q/pT (a value that
      crosses zero is measured against its physical scale), chi2_rel =
      |dchi2| / chi2.
    * n_param_over / param_over_sigma: covered tracks with a parameter above
      PARAM_TOL and the largest of those errors in units of the parameter's
      standard deviation (reported and bounded apart by the tests).
    * n_not_helix and its errors: fitted tracks with chi2/ndf >= CHI2NDF_FIT
      (mis-merged looper legs, where least squares amplifies rounding).
    * status_mismatch: tracks one side fitted and the other did not;
      n_failed_both: tracks whose refit failed on both sides (a propagation
      left the helix domain; the state is the one at the failure point).
    """
    ndf = np.maximum(r.tr_ndf, 1)
    fitted = (g["status"] == 0) & (r.tr_status == 0)
    ok = fitted & (r.tr_chi2 / ndf < CHI2NDF_FIT)
    nh = fitted & ~ok
    gp = g["param"].astype(np.float64)
    pe = param_rel_err(gp[ok], r.tr_p[ok])
    sig = np.sqrt(np.maximum(r.tr_c[ok][:, [0, 2, 5, 9, 14]], 0.0))
    over = pe > PARAM_TOL
    over_sig = (np.abs(gp[ok] - r.tr_p[ok]) / np.maximum(sig, 1e-300))[over]
    chi2_o = r.tr_chi2[ok]
    ce = np.abs(g["chi2"][ok].astype(np.float64) - chi2_o) / chi2_o
    pe_nh = param_rel_err(gp[nh], r.tr_p[nh])
    ce_nh = np.abs(g["chi2"][nh].astype(np.float64) - r.tr_chi2[nh]) / r.tr_chi2[nh]
    xe = np.abs(g["x"][ok] - r.tr_x[ok])
    mx = lambda a: float(a.max()) if a.size else 0.0  # noqa: E731
    return dict(n_tracks=int(r.n_tracks), n_ok=int(ok.sum()), n_not_helix=int(nh.sum()),
                status_mismatch=int((g["status"] != r.tr_status).sum()),
                n_failed_both=int(((g["status"] != 0) & (r.tr_status != 0)).sum()),
                param_max=pe.max(axis=0) if pe.size else np.zeros(5),
                param_p99=np.percentile(pe, 99, axis=0) if pe.size else np.zeros(5),
                n_param_over=int(over.any(axis=1).sum()), param_over_sigma=mx(over_sig),
                chi2_max=mx(ce), n_chi2_over=int((ce > CHI2_TOL).sum()),
                not_helix_param_max=mx(pe_nh), not_helix_chi2_max=mx(ce_nh), x_max=mx(xe))


def fit_summary(f):
    return (f"fit parity: {f['n_ok']} of {f['n_tracks']} tracks covered, param max rel "
            f"{f['param_max'].max():.2e} (p99 {f['param_p99'].max():.2e}), {f['n_param_over']} over {PARAM_TOL:g} "
            f"(max {f['param_over_sigma']:.1e} sigma), chi2 max rel {f['chi2_max']:.2e} ({f['n_chi2_over']} over "
            f"{CHI2_TOL:g}); {f['n_not_helix']} not helix fits (param {f['not_helix_param_max']:.1e}, chi2 "
            f"{f['not_helix_chi2_max']:.1e}); {f['status_mismatch']} status mismatches, {f['n_failed_both']} refits "
            f"failed on both sides")
