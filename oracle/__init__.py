"""CPU oracle of the TPC tracker (ctypes binding to oracle/liboracle.so).

TEST INFRASTRUCTURE ONLY: imported by tests/, by the smoke check and by the
benchmark's CPU-baseline / reference arm.  The product path never imports it.
"""
from __future__ import annotations

import ctypes as C
import dataclasses

import numpy as np

from . import build as _build

_lib = None
KB_C = np.float32(-2.99792458e-3)      # d sin(phi)/dx per (T * GeV^-1), binary32


class OrcParams(C.Structure):
    _fields_ = [("dy_link", C.c_float), ("dz_link", C.c_float), ("s_max_link", C.c_float),
                ("sigma_y", C.c_float), ("sigma_z", C.c_float),
                ("c0_snp", C.c_float), ("c0_tgl", C.c_float), ("c0_qpt", C.c_float),
                ("win_nsigma", C.c_float), ("win_min", C.c_float), ("win_max", C.c_float),
                ("chi2_cut", C.c_float), ("max_miss", C.c_int32), ("min_hits", C.c_int32),
                ("min_owned", C.c_int32), ("edge_margin", C.c_float),
                ("merge_dz", C.c_float), ("merge_chi2", C.c_float), ("refit_passes", C.c_int32),
                ("refit_inflate", C.c_float)]


class OrcGeom(C.Structure):
    _fields_ = [("n_sectors", C.c_int32), ("n_rows", C.c_int32), ("row_x", C.POINTER(C.c_float)),
                ("z_max", C.c_float), ("continuous", C.c_int32)]


_P32 = C.POINTER(C.c_int32)
_PF = C.POINTER(C.c_float)
_PD = C.POINTER(C.c_double)
_PU8 = C.POINTER(C.c_uint8)


class OrcResult(C.Structure):
    _fields_ = [("n", C.c_int32), ("z", _PF), ("up_raw", _P32), ("dn_raw", _P32), ("up", _P32),
                ("dn", _P32), ("is_start", _PU8),
                ("n_tracklets", C.c_int32), ("trk_start", _P32), ("trk_nhits", _P32), ("trk_off", _P32),
                ("trk_hits", _P32), ("trk_kept", _PU8), ("trk_top", _PF), ("trk_bot", _PF),
                ("n_seg", C.c_int32), ("seg_trk", _P32), ("seg_next", _P32), ("seg_prev", _P32),
                ("n_tracks", C.c_int32), ("tr_sector", _P32), ("tr_x", _PD), ("tr_p", _PD), ("tr_c", _PD),
                ("tr_chi2", _PD), ("tr_ndf", _P32), ("tr_status", _P32), ("tr_nclus", _P32),
                ("tr_off", _P32), ("tr_clus", _P32), ("assign", _P32),
                ("row_qup", C.c_float * 256), ("row_qdn", C.c_float * 256), ("row_w", C.c_float * 256)]


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(_build.build())
        L.orc_params_default.argtypes = [C.POINTER(OrcParams)]
        L.orc_track.argtypes = [C.POINTER(OrcParams), C.POINTER(OrcGeom), C.c_float, C.c_float, C.c_int32,
                                _PU8, _PU8, _PF, _PF, C.POINTER(OrcResult)]
        L.orc_free.argtypes = [C.POINTER(OrcResult)]
        L.orc_prop32.argtypes = [_PF, C.c_float, C.c_float]
        L.orc_rot32.argtypes = [_PF, C.c_float, C.c_float, C.c_float]
        L.orc_update32.argtypes = [_PF, C.c_float, C.c_float, C.c_float, C.c_float, C.c_float, _PF]
        L.orc_prop64.argtypes = [_PD, C.c_double, C.c_double]
        L.orc_rot64.argtypes = [_PD, C.c_double, C.c_double, C.c_double]
        L.orc_update64.argtypes = [_PD, C.c_double, C.c_double, C.c_double, C.c_double, _PD]
        L.orc_fit64.argtypes = [C.POINTER(OrcParams), C.POINTER(OrcGeom), C.c_double, C.c_int32, _P32,
                                _PD, _PD, _PD, C.c_int32, _PD, _PD]
        L.orc_merge_chi2.argtypes = [_PF, _PF, C.c_float, C.c_float, C.c_float]
        L.orc_merge_chi2.restype = C.c_float
        _lib = L
    return _lib


def default_params() -> dict:
    p = OrcParams()
    lib().orc_params_default(C.byref(p))
    return {name: getattr(p, name) for name, _ in OrcParams._fields_}


def _params(d: dict | None) -> OrcParams:
    p = OrcParams()
    lib().orc_params_default(C.byref(p))
    for k, v in (d or {}).items():
        setattr(p, k, v)
    return p


def _ptr(a, t):
    return a.ctypes.data_as(t)


@dataclasses.dataclass
class OracleResult:
    z: np.ndarray
    up_raw: np.ndarray
    dn_raw: np.ndarray
    up: np.ndarray
    dn: np.ndarray
    is_start: np.ndarray
    trk_start: np.ndarray
    trk_nhits: np.ndarray
    trk_off: np.ndarray
    trk_hits: np.ndarray
    trk_kept: np.ndarray
    trk_top: np.ndarray
    trk_bot: np.ndarray
    seg_trk: np.ndarray
    seg_next: np.ndarray
    seg_prev: np.ndarray
    tr_sector: np.ndarray
    tr_x: np.ndarray
    tr_p: np.ndarray
    tr_c: np.ndarray
    tr_chi2: np.ndarray
    tr_ndf: np.ndarray
    tr_status: np.ndarray
    tr_nclus: np.ndarray
    tr_off: np.ndarray
    tr_clus: np.ndarray
    assign: np.ndarray
    row_qup: np.ndarray
    row_qdn: np.ndarray
    row_w: np.ndarray

    @property
    def n_tracks(self) -> int:
        return int(self.tr_x.shape[0])

    def tracklet_hits(self, t: int) -> np.ndarray:
        return self.trk_hits[self.trk_off[t]:self.trk_off[t + 1]]

    def track_clusters(self, t: int) -> np.ndarray:
        return self.tr_clus[self.tr_off[t]:self.tr_off[t + 1]]


def _copy(ptr, n, dtype):
    if n == 0:
        return np.zeros(0, dtype)
    return np.ctypeslib.as_array(ptr, shape=(n,)).astype(dtype, copy=True)


def track(sector, row, y, zt, row_x, n_sectors=36, z_max=250.0, continuous=False, bz=0.5,
          v_drift=2.58, params: dict | None = None) -> OracleResult:
    """Run the whole oracle tracker on one event / frame (numpy inputs)."""
    L = lib()
    sector = np.ascontiguousarray(sector, np.uint8)
    row = np.ascontiguousarray(row, np.uint8)
    y = np.ascontiguousarray(y, np.float32)
    zt = np.ascontiguousarray(zt, np.float32)
    row_x = np.ascontiguousarray(row_x, np.float32)
    n = int(y.shape[0])
    P = _params(params)
    G = OrcGeom(n_sectors, row_x.shape[0], _ptr(row_x, _PF), z_max, int(continuous))
    R = OrcResult()
    rc = L.orc_track(C.byref(P), C.byref(G), bz, v_drift, n, _ptr(sector, _PU8), _ptr(row, _PU8),
                     _ptr(y, _PF), _ptr(zt, _PF), C.byref(R))
    if rc != 0:
        L.orc_free(C.byref(R))
        raise ValueError(f"oracle rejected the input (code {rc})")
    try:
        nt, ns, T = R.n_tracklets, R.n_seg, R.n_tracks
        trk_off = _copy(R.trk_off, nt + 1, np.int64)
        tr_off = _copy(R.tr_off, T + 1, np.int64)
        out = OracleResult(
            z=_copy(R.z, n, np.float32), up_raw=_copy(R.up_raw, n, np.int32), dn_raw=_copy(R.dn_raw, n, np.int32),
            up=_copy(R.up, n, np.int32), dn=_copy(R.dn, n, np.int32), is_start=_copy(R.is_start, n, np.uint8),
            trk_start=_copy(R.trk_start, nt, np.int32), trk_nhits=_copy(R.trk_nhits, nt, np.int32),
            trk_off=trk_off, trk_hits=_copy(R.trk_hits, int(trk_off[-1]), np.int32),
            trk_kept=_copy(R.trk_kept, nt, np.uint8),
            trk_top=_copy(R.trk_top, nt * 21, np.float32).reshape(nt, 21),
            trk_bot=_copy(R.trk_bot, nt * 21, np.float32).reshape(nt, 21),
            seg_trk=_copy(R.seg_trk, ns, np.int32), seg_next=_copy(R.seg_next, ns, np.int32),
            seg_prev=_copy(R.seg_prev, ns, np.int32),
            tr_sector=_copy(R.tr_sector, T, np.int32), tr_x=_copy(R.tr_x, T, np.float64),
            tr_p=_copy(R.tr_p, T * 5, np.float64).reshape(T, 5),
            tr_c=_copy(R.tr_c, T * 15, np.float64).reshape(T, 15),
            tr_chi2=_copy(R.tr_chi2, T, np.float64), tr_ndf=_copy(R.tr_ndf, T, np.int32),
            tr_status=_copy(R.tr_status, T, np.int32), tr_nclus=_copy(R.tr_nclus, T, np.int32),
            tr_off=tr_off, tr_clus=_copy(R.tr_clus, int(tr_off[-1]), np.int32),
            assign=_copy(R.assign, n, np.int32),
            row_qup=np.array(R.row_qup[:], np.float32), row_qdn=np.array(R.row_qdn[:], np.float32),
            row_w=np.array(R.row_w[:], np.float32))
    finally:
        L.orc_free(C.byref(R))
    return out


def track_event(ev, params: dict | None = None) -> OracleResult:
    """Oracle on a tpcgen.Event."""
    return track(ev.sector, ev.row, ev.y, ev.zt, ev.row_x, n_sectors=ev.n_sectors, z_max=ev.z_max,
                 continuous=ev.continuous, bz=ev.bz, v_drift=ev.v_drift, params=params)


# ---- single steps (for the pins) -------------------------------------------------
def prop32(st, x2, kb):
    s = np.ascontiguousarray(st, np.float32).copy()
    ok = lib().orc_prop32(_ptr(s, _PF), x2, kb)
    return bool(ok), s


def rot32(st, cs, sn, kb):
    s = np.ascontiguousarray(st, np.float32).copy()
    ok = lib().orc_rot32(_ptr(s, _PF), cs, sn, kb)
    return bool(ok), s


def update32(st, my, mz, vy, vz, chi2max=np.inf):
    s = np.ascontiguousarray(st, np.float32).copy()
    c2 = np.zeros(1, np.float32)
    ok = lib().orc_update32(_ptr(s, _PF), my, mz, vy, vz, chi2max, _ptr(c2, _PF))
    return bool(ok), s, float(c2[0])


def prop64(st, x2, kb):
    s = np.ascontiguousarray(st, np.float64).copy()
    ok = lib().orc_prop64(_ptr(s, _PD), x2, kb)
    return bool(ok), s


def rot64(st, cs, sn, kb):
    s = np.ascontiguousarray(st, np.float64).copy()
    ok = lib().orc_rot64(_ptr(s, _PD), cs, sn, kb)
    return bool(ok), s


def update64(st, my, mz, vy, vz):
    s = np.ascontiguousarray(st, np.float64).copy()
    c2 = np.zeros(1, np.float64)
    ok = lib().orc_update64(_ptr(s, _PD), my, mz, vy, vz, _ptr(c2, _PD))
    return bool(ok), s, float(c2[0])


def fit64(sector, x, y, z, st0, kb, n_passes=3, n_sectors=36, params: dict | None = None):
    """FP64 multi-pass Kalman fit of one cluster list (inner -> outer)."""
    sector = np.ascontiguousarray(sector, np.int32)
    x = np.ascontiguousarray(x, np.float64)
    y = np.ascontiguousarray(y, np.float64)
    z = np.ascontiguousarray(z, np.float64)
    st = np.ascontiguousarray(st0, np.float64).copy()
    rx = np.zeros(3, np.float32)
    P = _params(params)
    G = OrcGeom(n_sectors, rx.shape[0], _ptr(rx, _PF), 250.0, 0)
    chi2 = np.zeros(1)
    ok = lib().orc_fit64(C.byref(P), C.byref(G), kb, x.shape[0], _ptr(sector, _P32), _ptr(x, _PD),
                         _ptr(y, _PD), _ptr(z, _PD), n_passes, _ptr(st, _PD), _ptr(chi2, _PD))
    return bool(ok), st, float(chi2[0])


def merge_chi2(top, bot, cs, sn, kb):
    t = np.ascontiguousarray(top, np.float32)
    b = np.ascontiguousarray(bot, np.float32)
    return float(lib().orc_merge_chi2(_ptr(t, _PF), _ptr(b, _PF), cs, sn, kb))
