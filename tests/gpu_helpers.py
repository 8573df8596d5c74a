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
    return bad


CHI2NDF_FIT = 100.0   # above this the track is not a fit of one helix (mis-merged looper legs)


def compare_fit(g, r):
    """Refit parameters and chi2 of tracks both sides fitted successfully and
    that are fits of a helix (oracle chi2/ndf below CHI2NDF_FIT; the others
    are counted in n_not_helix).  A parameter error counts relative to
    max(|p|, floor), or -- where the value lies far inside its own
    uncertainty, so that a relative error has no meaning -- as zero when it is
    below 1e-3 of the parameter's standard deviation."""
    ndf = np.maximum(r.tr_ndf, 1)
    fitted = (g["status"] == 0) & (r.tr_status == 0)
    ok = fitted & (r.tr_chi2 / ndf < CHI2NDF_FIT)
    pe = param_rel_err(g["param"][ok], r.tr_p[ok])
    sig = np.sqrt(np.maximum(r.tr_c[ok][:, [0, 2, 5, 9, 14]], 0.0))
    pe[np.abs(g["param"][ok].astype(np.float64) - r.tr_p[ok]) <= 1e-3 * sig] = 0.0
    ce = np.abs(g["chi2"][ok].astype(np.float64) - r.tr_chi2[ok]) / np.maximum(r.tr_chi2[ok], 1.0)
    xe = np.abs(g["x"][ok] - r.tr_x[ok])
    return dict(n_ok=int(ok.sum()), n_not_helix=int((fitted & ~ok).sum()),
                status_mismatch=int((g["status"] != r.tr_status).sum()),
                param_max=pe.max(axis=0) if pe.size else np.zeros(5), param_p99=np.percentile(pe, 99, axis=0) if pe.size else np.zeros(5),
                chi2_max=float(ce.max()) if ce.size else 0.0, x_max=float(xe.max()) if xe.size else 0.0)
