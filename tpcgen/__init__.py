"""Seeded synthetic ALICE-like TPC events (input data only).

This module produces the inputs that both the CPU oracle and the CUDA tracker
consume.  It holds none of the tracker's arithmetic: it intersects exact
helices with the pad-row planes analytically in float64 (global coordinates),
smears the crossings and, for continuous read-out, converts z to drift time.

Workload shapes (paper, sections "Tracking" and "TPC Tracking"; the numeric
laws are readings of the paper, listed with the input recipe in the design
notes):

* geometry: 36 sectors (18 per side, 20 degrees wide), 152 planar pad rows at
  local x = 85 .. 247 cm with uniform pitch, |z| <= 250 cm, Bz = 0.5 T;
* primaries from the origin: pT log-uniform in [0.2, 5] GeV/c, phi uniform,
  eta uniform in (-0.9, 0.9), charge +-1;
* continuous read-out frames: collisions at uniform times, multiplicity
  ceil(Exp(mean)), 5 % extra low-pT loopers (pT log-uniform 0.05 .. 0.2),
  clusters carry drift time t = t_c + (Zmax - |z|)/v_drift + t0 instead of z
  (section "Tracking": hits only have a time value);
* smearing sigma_y = 0.1 cm, sigma_z = 0.15 cm; uniform noise clusters.

Random numbers come from numpy's Philox-4x32-10 counter-based generator
(Salmon et al., SC'11), seeded per workload.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

C_LIGHT = 0.299792458e-2          # GeV / (T cm): R[cm] = pT / (C_LIGHT * B)
N_ROWS = 152
X_FIRST, X_LAST = 85.0, 247.0
Z_MAX = 250.0
SECTOR_DPHI_DEG = 20.0
RHO_OUT = 260.0                    # radial exit of the field cage (encloses every row plane)
MAX_TURNS = 10
SIGMA_Y, SIGMA_Z = 0.1, 0.15
V_DRIFT = 2.58                     # cm / us
FRAME_US = 1000.0                  # one time frame = 1 ms


def row_x_f32(n_rows: int = N_ROWS) -> np.ndarray:
    """Pad-row plane positions (local x, cm) as the float32 values every consumer uses."""
    r = np.arange(n_rows, dtype=np.float64)
    return (X_FIRST + r * (X_LAST - X_FIRST) / (n_rows - 1)).astype(np.float32)


def sector_alpha(n_sectors: int) -> np.ndarray:
    """Centre azimuth (rad) of each sector: (s mod 18) * 20 deg + 10 deg."""
    s = np.arange(n_sectors)
    return np.deg2rad((s % 18) * SECTOR_DPHI_DEG + SECTOR_DPHI_DEG / 2)


@dataclasses.dataclass
class Event:
    """One tracker input: cluster SoA (float32 / uint8) plus generator truth."""
    sector: np.ndarray          # u8 [N]
    row: np.ndarray             # u8 [N]
    y: np.ndarray               # f32 [N] sector-local y (cm)
    zt: np.ndarray              # f32 [N] z (cm) or drift time (us) when continuous
    charge: np.ndarray          # f32 [N] (carried, unused by the tracker)
    label: np.ndarray           # i32 [N] generating track, -1 for noise
    n_sectors: int
    row_x: np.ndarray           # f32 [n_rows]
    bz: float
    continuous: bool
    v_drift: float              # nominal drift velocity the tracker is given
    z_max: float
    # truth
    trk_pt: np.ndarray
    trk_phi0: np.ndarray
    trk_eta: np.ndarray
    trk_q: np.ndarray
    trk_tc: np.ndarray          # collision time (us), 0 for triggered events
    trk_coll: np.ndarray        # collision index
    trk_looper: np.ndarray      # bool
    n_collisions: int
    # per-cluster exact (unsmeared) crossing, float64; None when not requested
    true_y: np.ndarray | None = None
    true_z: np.ndarray | None = None
    true_snp: np.ndarray | None = None
    true_s: np.ndarray | None = None      # transverse path length from the vertex
    v_drift_true: float = V_DRIFT
    t0_true: float = 0.0
    calib: dict | None = None

    @property
    def n(self) -> int:
        return int(self.y.shape[0])

    def arrays(self):
        return self.sector, self.row, self.y, self.zt, self.charge


_helix = None


def _helix_lib():
    """The compiled crossing routine (tpcgen/helix.c), built on first use."""
    global _helix
    if _helix is None:
        import ctypes as C

        from . import build as _b
        L = C.CDLL(_b.build())
        PD = C.POINTER(C.c_double)
        P32 = C.POINTER(C.c_int32)
        L.helix_crossings.restype = C.c_int64
        L.helix_crossings.argtypes = [C.c_int64, PD, PD, PD, PD, PD, C.POINTER(C.c_uint8), C.c_int, PD, C.c_int, PD,
                                      C.c_double, C.c_int, C.POINTER(C.c_int64), P32, P32, P32, PD, PD, PD, PD]
        _helix = L
    return _helix


def _crossings(pt, phi0, eta, q, looper, bz, alphas, row_x64, z0=None):
    """All accepted plane crossings of helices from the origin (shifted in z
    by the vertex z0 of each track when given).

    Returns (track, wedge, row, y_local, z, snp_local, s).  The helix:
    direction phi(s) = phi0 + h s / R with h = -q sign(B), z = s tan(lambda);
    the plane of wedge a at x_local = X_r is crossed where
    sin(phi - alpha) = sin(phi0 - alpha) + h X_r / R.  A track ends at
    |z| > Z_MAX, at radius RHO_OUT, or after MAX_TURNS turns (loopers).
    """
    import ctypes as C
    L = _helix_lib()
    n = pt.shape[0]
    R = np.ascontiguousarray(pt / (C_LIGHT * abs(bz)))
    h = np.ascontiguousarray(-q * np.sign(bz))
    tgl = np.ascontiguousarray(np.sinh(eta))
    s_exit = np.where(2 * R > RHO_OUT, 2 * R * np.arcsin(np.minimum(RHO_OUT / (2 * R), 1.0)), np.inf)
    zv = np.zeros(n) if z0 is None else np.asarray(z0, np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        # the path to the end plate the track heads for
        s_z = np.where(tgl > 0, (Z_MAX - zv) / tgl, np.where(tgl < 0, (Z_MAX + zv) / -tgl, np.inf))
    s_max = np.ascontiguousarray(np.minimum(np.minimum(s_exit, MAX_TURNS * 2.0 * np.pi * R), s_z))
    phi0 = np.ascontiguousarray(phi0, np.float64)
    lp = np.ascontiguousarray(looper, np.uint8)
    al = np.ascontiguousarray(alphas, np.float64)
    X = np.ascontiguousarray(row_x64, np.float64)
    tan_half = math.tan(math.radians(SECTOR_DPHI_DEG / 2))
    PD = C.POINTER(C.c_double)
    P32 = C.POINTER(C.c_int32)
    counts = np.zeros(max(n, 1), np.int64)
    args = [n, R.ctypes.data_as(PD), h.ctypes.data_as(PD), phi0.ctypes.data_as(PD), tgl.ctypes.data_as(PD),
            s_max.ctypes.data_as(PD), lp.ctypes.data_as(C.POINTER(C.c_uint8)), al.size, al.ctypes.data_as(PD),
            X.size, X.ctypes.data_as(PD), tan_half, MAX_TURNS, counts.ctypes.data_as(C.POINTER(C.c_int64))]
    tot = L.helix_crossings(*args, None, None, None, None, None, None, None)
    trk = np.empty(tot, np.int32)
    wedge = np.empty(tot, np.int32)
    row = np.empty(tot, np.int32)
    y, z, snp, sp = (np.empty(tot) for _ in range(4))
    L.helix_crossings(*args, trk.ctypes.data_as(P32), wedge.ctypes.data_as(P32), row.ctypes.data_as(P32),
                      y.ctypes.data_as(PD), z.ctypes.data_as(PD), snp.ctypes.data_as(PD), sp.ctypes.data_as(PD))
    trk = trk.astype(np.int64)
    if z0 is not None:
        z = z + zv[trk]
    return trk, wedge, row, y, z, snp, sp


def _gen_tracks(rng, n, pt_lo, pt_hi, phi_lo, phi_hi):
    pt = np.exp(rng.uniform(math.log(pt_lo), math.log(pt_hi), n))
    phi0 = rng.uniform(phi_lo, phi_hi, n)
    eta = rng.uniform(-0.9, 0.9, n)
    q = np.where(rng.random(n) < 0.5, -1.0, 1.0)
    return pt, phi0, eta, q


def generate(n_sectors=36, n_tracks=None, n_collisions=0, mult_mean=2000.0,
             looper_frac=0.0, noise_frac=0.05, continuous=False, seed=1,
             bz=0.5, frame_us=FRAME_US, with_truth=True, v_drift_true=V_DRIFT,
             t0_true=0.0, calib=None, shuffle=True, vertex_z_sigma=0.0) -> Event:
    """Generate one event (triggered) or one continuous read-out frame.

    * triggered (``continuous=False``): ``n_tracks`` primaries at t = 0;
    * continuous: ``n_collisions`` collisions at uniform times in
      [0, frame_us), each with ceil(Exp(mult_mean)) primaries and
      ``looper_frac`` extra loopers; clusters carry drift time.
    ``calib`` (optional) distorts the cluster positions (see :func:`distortion`).
    ``vertex_z_sigma`` (cm, default 0: every vertex at the origin) spreads the
    primary vertex along z (Gaussian), so that tracks at small dip angles
    cross the central membrane between the A and C sides.
    """
    rng = np.random.Generator(np.random.Philox(seed))
    row_x = row_x_f32()
    row_x64 = row_x.astype(np.float64)
    alphas = sector_alpha(18 if n_sectors == 36 else 1)
    if n_sectors == 1:
        phi_lo, phi_hi = 0.0, math.radians(SECTOR_DPHI_DEG)
    else:
        phi_lo, phi_hi = 0.0, 2 * np.pi

    if continuous:
        mult = np.ceil(rng.exponential(mult_mean, n_collisions)).astype(np.int64)
        tcs = np.sort(rng.uniform(0.0, frame_us, n_collisions))
        n_prim = int(mult.sum())
        n_loop = [int(round(looper_frac * m)) for m in mult]
        coll_p = np.repeat(np.arange(n_collisions), mult)
        coll_l = np.repeat(np.arange(n_collisions), n_loop)
    else:
        n_collisions = 1
        n_prim = int(n_tracks)
        tcs = np.zeros(1)
        coll_p = np.zeros(n_prim, np.int64)
        coll_l = np.zeros(int(round(looper_frac * n_prim)), np.int64)
    n_loop_total = coll_l.size
    pt, phi0, eta, q = _gen_tracks(rng, n_prim, 0.2, 5.0, phi_lo, phi_hi)
    lpt, lphi0, leta, lq = _gen_tracks(rng, n_loop_total, 0.05, 0.2, phi_lo, phi_hi)

    zv = rng.normal(0.0, vertex_z_sigma, n_prim + n_loop_total) if vertex_z_sigma > 0 else None
    cp = _crossings(np.concatenate([pt, lpt]), np.concatenate([phi0, lphi0]), np.concatenate([eta, leta]),
                    np.concatenate([q, lq]), np.concatenate([np.zeros(n_prim, bool), np.ones(n_loop_total, bool)]),
                    bz, alphas, row_x64, z0=zv)
    t_idx, wedge, row, y_true, z_true, snp_true, s_true = cp

    trk_pt = np.concatenate([pt, lpt])
    trk_phi0 = np.concatenate([phi0, lphi0])
    trk_eta = np.concatenate([eta, leta])
    trk_q = np.concatenate([q, lq])
    trk_coll = np.concatenate([coll_p, coll_l]).astype(np.int64)
    trk_tc = tcs[trk_coll]
    trk_looper = np.concatenate([np.zeros(n_prim, bool), np.ones(n_loop_total, bool)])

    if n_sectors == 36:
        sector = wedge + 18 * (z_true < 0)
    else:
        sector = np.zeros_like(wedge)
    ns = y_true.size
    y_meas = y_true + rng.normal(0.0, SIGMA_Y, ns)
    z_meas = z_true + rng.normal(0.0, SIGMA_Z, ns)
    if calib is not None:
        dyc, dzc = distortion(calib, sector, row_x64[row], np.abs(z_meas))
        y_meas = y_meas + dyc
        # dz acts along the drift direction (towards larger |z|)
        z_meas = z_meas + np.where(z_true < 0, -dzc, dzc)

    # noise clusters
    n_noise = int(round(noise_frac * ns))
    nz_sector = rng.integers(0, n_sectors, n_noise)
    nz_row = rng.integers(0, N_ROWS, n_noise)
    tan_half = math.tan(math.radians(SECTOR_DPHI_DEG / 2))
    xr_n = row_x64[nz_row]
    nz_y = rng.uniform(-1.0, 1.0, n_noise) * xr_n * tan_half
    if continuous:
        nz_t = rng.uniform(0.0, frame_us + Z_MAX / v_drift_true, n_noise)
    else:
        zabs = rng.uniform(0.0, Z_MAX, n_noise)
        if n_sectors == 36:
            nz_z = np.where(nz_sector >= 18, -zabs, zabs)
        else:
            nz_z = rng.uniform(-Z_MAX, Z_MAX, n_noise)

    if continuous:
        t_meas = trk_tc[t_idx] + (Z_MAX - np.abs(z_meas)) / v_drift_true + t0_true
        zt = np.concatenate([t_meas, nz_t])
    else:
        zt = np.concatenate([z_meas, nz_z])
    sector_all = np.concatenate([sector, nz_sector]).astype(np.uint8)
    row_all = np.concatenate([row, nz_row]).astype(np.uint8)
    y_all = np.concatenate([y_meas, nz_y])
    label = np.concatenate([t_idx, np.full(n_noise, -1)]).astype(np.int32)
    charge = rng.uniform(10.0, 100.0, ns + n_noise)
    truth = None
    if with_truth:
        nan = np.full(n_noise, np.nan)
        truth = (np.concatenate([y_true, nan]), np.concatenate([z_true, nan]),
                 np.concatenate([snp_true, nan]), np.concatenate([s_true, nan]))
    perm = rng.permutation(ns + n_noise) if shuffle else np.arange(ns + n_noise)
    ev = Event(
        sector=sector_all[perm], row=row_all[perm], y=y_all[perm].astype(np.float32),
        zt=zt[perm].astype(np.float32), charge=charge[perm].astype(np.float32),
        label=label[perm], n_sectors=n_sectors, row_x=row_x, bz=bz,
        continuous=continuous, v_drift=V_DRIFT, z_max=Z_MAX,
        trk_pt=trk_pt, trk_phi0=trk_phi0, trk_eta=trk_eta, trk_q=trk_q,
        trk_tc=trk_tc, trk_coll=trk_coll, trk_looper=trk_looper,
        n_collisions=n_collisions, v_drift_true=v_drift_true, t0_true=t0_true,
        calib=calib)
    if truth is not None:
        ev.true_y, ev.true_z, ev.true_snp, ev.true_s = (a[perm] for a in truth)
    return ev


# ----------------------------------------------------------------------------
# calibration distortions (continuous frame with a miscalibration)
# ----------------------------------------------------------------------------
SPLINE_NX = SPLINE_NZ = 8


def bspline_basis(u: np.ndarray, n: int) -> np.ndarray:
    """Uniform clamped cubic B-spline basis, n coefficients, u in [0, 1] -> [len(u), n]."""
    k = 3
    n_int = n - k
    knots = np.concatenate([np.zeros(k), np.linspace(0.0, 1.0, n_int + 1), np.ones(k)])
    u = np.clip(np.atleast_1d(np.asarray(u, np.float64)), 0.0, 1.0)
    B = np.zeros((u.size, knots.size - 1))
    for i in range(knots.size - 1):
        lo, hi = knots[i], knots[i + 1]
        if hi > lo:
            B[:, i] = ((u >= lo) & (u < hi)) | ((hi == 1.0) & (u == 1.0))
    for d in range(1, k + 1):
        Bn = np.zeros((u.size, knots.size - 1 - d))
        for i in range(knots.size - 1 - d):
            den1 = knots[i + d] - knots[i]
            den2 = knots[i + d + 1] - knots[i + 1]
            t1 = (u - knots[i]) / den1 * B[:, i] if den1 > 0 else 0.0
            t2 = (knots[i + d + 1] - u) / den2 * B[:, i + 1] if den2 > 0 else 0.0
            Bn[:, i] = t1 + t2
        B = Bn
    return B


def distortion(calib: dict, sector, x, zabs):
    """Per-cluster (dy, dz) of the per-sector 8x8 cubic-spline distortion map."""
    coef = calib["spline"]               # [n_sectors, 8, 8, 2]
    bu = bspline_basis((np.asarray(x) - X_FIRST) / (X_LAST - X_FIRST), SPLINE_NX)
    bv = bspline_basis(np.asarray(zabs) / Z_MAX, SPLINE_NZ)
    c = coef[np.asarray(sector)]
    d = np.einsum("ni,nj,nijc->nc", bu, bv, c)
    return d[:, 0], d[:, 1]


# ----------------------------------------------------------------------------
# the workloads
# ----------------------------------------------------------------------------
def one_sector(seed=1, n_tracks=200, **kw) -> Event:
    """One TPC sector, 200 primaries from the origin, 5 % noise, z given."""
    return generate(n_sectors=1, n_tracks=n_tracks, noise_frac=0.05, continuous=False, seed=seed, **kw)


def central_event(seed=2, n_tracks=10000, **kw) -> Event:
    """Full TPC, one central Pb-Pb-like event: 10k primaries, 10 % noise, z given."""
    return generate(n_sectors=36, n_tracks=n_tracks, noise_frac=0.10, continuous=False, seed=seed, **kw)


def time_frame(seed=3, n_collisions=50, mult_mean=2000.0, frame_us=FRAME_US, **kw) -> Event:
    """Continuous read-out frame: overlapping collisions, 5 % loopers, drift times."""
    kw.setdefault("looper_frac", 0.05)
    kw.setdefault("noise_frac", 0.05)
    return generate(n_sectors=36, n_collisions=n_collisions, mult_mean=mult_mean,
                    continuous=True, seed=seed, frame_us=frame_us, **kw)


def calib_truth(seed=5, n_sectors=36):
    """Miscalibration of the calibration workload: v_drift +0.3 %, t0 = 0.2 us,
    per-sector 8x8 spline coefficients uniform in [-0.5, 0.5] cm."""
    rng = np.random.Generator(np.random.Philox(10_000 + seed))
    coef = rng.uniform(-0.5, 0.5, (n_sectors, SPLINE_NX, SPLINE_NZ, 2))
    return {"v_drift": 1.003 * V_DRIFT, "t0": 0.2, "spline": coef}


def calib_frame(seed=5, n_collisions=50, **kw) -> Event:
    """The continuous frame generated with a drift-velocity offset, a t0 shift and
    a distortion map; the tracker is given the nominal drift velocity."""
    cal = calib_truth(seed)
    return time_frame(seed=seed, n_collisions=n_collisions, v_drift_true=cal["v_drift"],
                      t0_true=cal["t0"], calib=cal, **kw)


def stf_batch(n_stf=64, seed0=1000, mult_mean=2000.0, max_coll=100, **kw):
    """Sub-time-frames of 1..100 collisions at 50 kHz (n collisions over n/50 ms)."""
    rng = np.random.Generator(np.random.Philox(seed0))
    ncoll = rng.integers(1, max_coll + 1, n_stf)
    return [time_frame(seed=seed0 + 1 + i, n_collisions=int(nc), mult_mean=mult_mean,
                       frame_us=float(nc) * 20.0, **kw) for i, nc in enumerate(ncoll)]


def track_collision_time(ev: Event, off, clus, min_frac: float = 0.5):
    """Generator-truth collision time of reconstructed tracks: the collision of
    the label that owns most of a track's clusters (at least ``min_frac`` of
    them, and not noise), NaN otherwise.  Stands in for the time that matching
    to the inner detectors would fix."""
    off = np.asarray(off, np.int64)
    clus = np.asarray(clus, np.int64)
    T = off.size - 1
    out = np.full(T, np.nan, np.float32)
    if T == 0 or ev.trk_tc is None:
        return out
    lab = ev.label[clus]
    for t in range(T):
        a, b = off[t], off[t + 1]
        if b <= a:
            continue
        vals, cnt = np.unique(lab[a:b], return_counts=True)
        k = int(np.argmax(cnt))
        if vals[k] >= 0 and cnt[k] >= min_frac * (b - a):
            out[t] = np.float32(ev.trk_tc[vals[k]])
    return out


def track_dip_angle(ev: Event, off, clus, sigma: float = 3e-4, seed: int = 7, min_frac: float = 0.5):
    """Generator-truth dip angle tan(lambda) = sinh(eta) of reconstructed
    tracks (the label owning most of a track's clusters, as
    :func:`track_collision_time`), smeared by a Gaussian of ``sigma``; NaN
    where no label owns ``min_frac`` of the clusters.  Stands in for the dip
    angle of the inner-detector track that matching pairs with it."""
    off = np.asarray(off, np.int64)
    clus = np.asarray(clus, np.int64)
    T = off.size - 1
    out = np.full(max(T, 0), np.nan, np.float32)
    if T <= 0:
        return out
    rng = np.random.Generator(np.random.Philox(20_000 + seed))
    noise = rng.standard_normal(T)
    lab = ev.label[clus]
    for t in range(T):
        a, b = off[t], off[t + 1]
        if b <= a:
            continue
        vals, cnt = np.unique(lab[a:b], return_counts=True)
        k = int(np.argmax(cnt))
        if vals[k] >= 0 and cnt[k] >= min_frac * (b - a):
            out[t] = np.float32(np.sinh(ev.trk_eta[vals[k]]) + sigma * noise[t])
    return out
