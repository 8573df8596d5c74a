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
                ("refit_inflate", C.c_float), ("packed_links", C.c_int32), ("back_jump", C.c_int32),
                ("outlier_chi2", C.c_float)]


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
                ("tr_off", _P32), ("tr_clus", _P32), ("assign", _P32), ("rejected", _PU8), ("n_rejected", C.c_int32),
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
        L.orc_helix64.argtypes = [_PD, _PD, C.c_double, C.c_double, _PD]
        L.orc_rotate64.argtypes = [_PD, _PD, C.c_double, C.c_double, C.c_double, _PD]
        L.orc_calib.argtypes = [C.POINTER(OrcParams), C.POINTER(OrcGeom), C.c_double, C.c_double, C.c_double,
                                C.c_int32, _P32, _PF, _PF, _P32, _P32, _PU8, _PU8, _PF, _PF, _PF, _PD, _PD, _PD,
                                _PU8, _PD, _PF, C.c_double]
        L.orc_calib_measure.argtypes = [C.POINTER(OrcGeom), _PD, C.c_int32, _PU8, _PU8, _PF, _PF, _PF, _PD, _PD]
        L.orc_calib_measure.restype = None
        L.orc_calib_explain.argtypes = [C.POINTER(OrcParams), C.POINTER(OrcGeom), C.c_double, C.c_double,
                                        C.c_double, _P32, _PF, _PF, _P32, _P32, _PU8, _PU8, _PF, _PF, _PF, _PD,
                                        C.c_int32, _PD, _PD, _PD, _PD, _PD]
        L.orc_calib_select.argtypes = [C.c_int32, _PF, _P32, _PF, C.c_float, _PF]
        L.orc_calib_select.restype = None
        L.orc_bspline_all.argtypes = [C.c_double, _PD, _PD]
        L.orc_bspline_all.restype = None
        L.orc_step_pos32.argtypes = [_PF, C.c_float, C.c_float]
        L.orc_loopers.argtypes = [C.c_int32, C.c_float, C.c_float, C.c_float, C.c_int32, _P32, _P32, _PF, _P32, _P32]
        L.orc_atan2_own.argtypes = [C.c_float, C.c_float]
        L.orc_atan2_own.restype = C.c_float
        _PU32 = C.POINTER(C.c_uint32)
        L.orc_rans_normalise.argtypes = [_PU32, _PU32]
        L.orc_rans_encode.argtypes = [_PU8, C.c_int32, _PU32, _PU8, _P32]
        L.orc_rans_decode.argtypes = [_PU8, C.c_int32, _PU32, C.c_int32, _PU8]
        L.orc_compress_fields.argtypes = [C.c_int32, C.c_int32, C.c_int32, _PU8, _PU8, _PF, _PF, C.c_int32,
                                          C.c_int32, C.c_int32, _P32, _P32, _P32, C.POINTER(_PU32),
                                          C.POINTER(C.c_int64)]
        L.orc_decompress_fields.argtypes = [C.c_int32, C.c_int32, C.POINTER(_PU32), C.POINTER(C.c_int64),
                                            C.c_int32, C.c_int32, _PU8, _PU8, _P32, _P32]
        L.orc_code_stream.argtypes = [_PU32, C.c_int64, C.c_int32, C.POINTER(C.c_int64), _P32]
        L.orc_pack_stream.argtypes = [_PU32, C.c_int64, C.c_int32, _PU8]
        L.orc_pack_stream.restype = C.c_int64
        L.orc_unpack_stream.argtypes = [_PU8, C.c_int64, _PU32, C.c_int64, C.POINTER(C.c_int64)]
        L.orc_unpack_stream.restype = C.c_int64
        L.orc_free_ptr.argtypes = [C.c_void_p]
        L.orc_free_ptr.restype = None
        L.orc_attach.argtypes = [C.POINTER(OrcGeom), C.c_float, C.c_int32, _PU8, _PU8, _PF, _PF, C.c_int32, _P32,
                                 _P32, _P32, _P32, _P32, _PF, _P32, C.c_float, C.c_float, _P32, _P32, _PU8]
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
    rejected: np.ndarray
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
            assign=_copy(R.assign, n, np.int32), rejected=_copy(R.rejected, n, np.uint8),
            row_qup=np.array(R.row_qup[:], np.float32), row_qdn=np.array(R.row_qdn[:], np.float32),
            row_w=np.array(R.row_w[:], np.float32))
    finally:
        L.orc_free(C.byref(R))
    return out


# ---- track-based cluster attachment ---------------------------------------------
CL_ATTACHED, CL_ADJACENT, CL_PROTECTED, CL_REMOVE = 1, 2, 4, 8


def attach(sector, row, y, r: OracleResult, row_x, n_sectors=36, bz=0.5, radius=1.5, pt_min=0.05,
           loopers_first=True, frame=None):
    """Cluster attachment of an oracle tracking result: (adjacent track per
    cluster or -1, flags CL_*) -- tubes of ``radius`` cm, tracks below
    ``pt_min`` GeV/c not good, nor (loopers_first) the secondary legs of
    loopers (tpc_oracle_attach.c, tpc_oracle_loopers.c)."""
    L = lib()
    sector = np.ascontiguousarray(sector, np.uint8)
    row = np.ascontiguousarray(row, np.uint8)
    y = np.ascontiguousarray(y, np.float32)
    z = np.ascontiguousarray(r.z, np.float32)
    row_x = np.ascontiguousarray(row_x, np.float32)
    n = int(y.shape[0])
    G = OrcGeom(n_sectors, row_x.shape[0], _ptr(row_x, _PF), 250.0, 0)
    i32 = lambda a: np.ascontiguousarray(a, np.int32)  # noqa: E731
    seg_trk, seg_next, seg_prev = i32(r.seg_trk), i32(r.seg_next), i32(r.seg_prev)
    trk_off, trk_hits, assign = i32(r.trk_off), i32(r.trk_hits), i32(r.assign)
    bot = np.ascontiguousarray(r.trk_bot, np.float32)
    adj = np.empty(max(n, 1), np.int32)
    fl = np.empty(max(n, 1), np.uint8)
    legs = None
    if loopers_first:
        legs = np.ascontiguousarray(loopers(sector, r, n_sectors=n_sectors, bz=bz, frame=frame)[1], np.int32)
    rc = L.orc_attach(C.byref(G), bz, n, _ptr(sector, _PU8), _ptr(row, _PU8), _ptr(y, _PF), _ptr(z, _PF),
                      int(seg_trk.shape[0]), _ptr(seg_trk, _P32), _ptr(seg_next, _P32), _ptr(seg_prev, _P32),
                      _ptr(trk_off, _P32), _ptr(trk_hits, _P32), _ptr(bot, _PF), _ptr(assign, _P32), radius, pt_min,
                      None if legs is None else _ptr(legs, _P32), _ptr(adj, _P32), _ptr(fl, _PU8))
    if rc != 0:
        raise ValueError(f"oracle attachment rejected the input (code {rc})")
    return adj[:n], fl[:n]


def attach_event(ev, r: OracleResult, radius=1.5, pt_min=0.05, loopers_first=True):
    """attach() on a tpcgen.Event and the oracle's result for it."""
    return attach(ev.sector, ev.row, ev.y, r, ev.row_x, n_sectors=ev.n_sectors, bz=ev.bz, radius=radius,
                  pt_min=pt_min, loopers_first=loopers_first)


LOOPER_QPT_MIN = 5.0     # |q/pT| (c/GeV) of a looper-leg candidate: pT below 200 MeV/c


def track_heads(r: OracleResult):
    """Per track: the tracklet index of its innermost piece (tracks are in the
    order of their innermost pieces' start indices)."""
    return r.seg_trk[r.seg_prev < 0]


def loopers(sector, r: OracleResult, n_sectors=36, bz=0.5, qpt_min=LOOPER_QPT_MIN, frame=None, z_max=250.0):
    """Looper-leg groups and leg numbers of an oracle tracking result
    (tpc_oracle_loopers.c): group[t] = smallest track of the legs of one
    particle (-1 alone), leg[t] = 0 for the earliest leg in drift."""
    heads = track_heads(r)
    T = r.n_tracks
    sec = np.ascontiguousarray(np.asarray(sector)[r.trk_start[heads]], np.int32)
    st = np.ascontiguousarray(r.trk_bot[heads], np.float32)
    fr = None if frame is None else np.ascontiguousarray(frame, np.int32)
    g = np.zeros(max(T, 1), np.int32)
    lg = np.zeros(max(T, 1), np.int32)
    rc = lib().orc_loopers(n_sectors, z_max, bz, qpt_min, T, _ptr(sec, _P32), None if fr is None else _ptr(fr, _P32),
                           _ptr(st, _PF), _ptr(g, _P32), _ptr(lg, _P32))
    if rc:
        raise ValueError(f"orc_loopers failed ({rc})")
    return g[:T], lg[:T]


def atan2_own(y, x):
    return float(lib().orc_atan2_own(np.float32(y), np.float32(x)))


def step_pos32(p, x2, kb):
    """One binary32 helix step of (x, y, z, sin phi, tan lambda, q/pT)."""
    s = np.ascontiguousarray(p, np.float32).copy()
    ok = lib().orc_step_pos32(_ptr(s, _PF), x2, kb)
    return bool(ok), s


# ---- cluster compression -----------------------------------------------------------
COMPRESS_STREAMS = ("n_track", "head_sector", "head_row", "head_y", "head_t", "d_sector", "d_row", "res_y",
                    "res_t", "u_count", "u_dt", "u_y")
_PU32 = C.POINTER(C.c_uint32)


def rans_normalise(hist):
    h = np.ascontiguousarray(hist, np.uint32)
    f = np.zeros(256, np.uint32)
    rc = lib().orc_rans_normalise(_ptr(h, _PU32), _ptr(f, _PU32))
    if rc:
        raise ValueError(f"empty histogram ({rc})")
    return f


def rans_encode(sym, freq):
    sym = np.ascontiguousarray(sym, np.uint8)
    freq = np.ascontiguousarray(freq, np.uint32)
    out = np.zeros(4 + 2 * sym.size, np.uint8)
    nb = C.c_int32(0)
    rc = lib().orc_rans_encode(_ptr(sym, _PU8), sym.size, _ptr(freq, _PU32), _ptr(out, _PU8), C.byref(nb))
    if rc:
        raise ValueError(f"rANS encode failed ({rc})")
    return out[:nb.value].copy()


def rans_decode(data, freq, n):
    data = np.ascontiguousarray(data, np.uint8)
    freq = np.ascontiguousarray(freq, np.uint32)
    sym = np.zeros(max(n, 1), np.uint8)
    rc = lib().orc_rans_decode(_ptr(data, _PU8), data.size, _ptr(freq, _PU32), n, _ptr(sym, _PU8))
    if rc:
        raise ValueError(f"rANS decode failed ({rc})")
    return sym[:n]


def compress_fields(sector, row, y, zt, r: OracleResult, n_sectors=36, n_rows=152, ey=5, et=6) -> dict:
    """The integer streams of the compressed format (before entropy coding)
    of a frame and the oracle's tracking result for it."""
    L = lib()
    sector = np.ascontiguousarray(sector, np.uint8)
    row = np.ascontiguousarray(row, np.uint8)
    y = np.ascontiguousarray(y, np.float32)
    zt = np.ascontiguousarray(zt, np.float32)
    off = np.ascontiguousarray(r.tr_off, np.int32)
    clus = np.ascontiguousarray(r.tr_clus, np.int32)
    assign = np.ascontiguousarray(r.assign, np.int32)
    vals = (_PU32 * 12)()
    counts = (C.c_int64 * 12)()
    rc = L.orc_compress_fields(n_sectors, n_rows, y.size, _ptr(sector, _PU8), _ptr(row, _PU8), _ptr(y, _PF),
                               _ptr(zt, _PF), ey, et, r.n_tracks, _ptr(off, _P32), _ptr(clus, _P32),
                               _ptr(assign, _P32), vals, counts)
    if rc:
        raise ValueError(f"compress_fields failed ({rc})")
    out = {}
    for k, name in enumerate(COMPRESS_STREAMS):
        m = int(counts[k])
        out[name] = np.ctypeslib.as_array(vals[k], shape=(max(m, 1),))[:m].copy()
        L.orc_free_ptr(C.cast(vals[k], C.c_void_p))
    return out


def decompress_fields(fields: dict, n_tracks, n, n_sectors=36, n_rows=152):
    """Quantised clusters (sector, row, qy, qt) back from the streams:
    attached clusters in track order, then the others plane by plane."""
    arrs = [np.ascontiguousarray(fields[k], np.uint32) for k in COMPRESS_STREAMS]
    vals = (_PU32 * 12)(*[_ptr(a, _PU32) for a in arrs])
    counts = (C.c_int64 * 12)(*[a.size for a in arrs])
    sector = np.zeros(max(n, 1), np.uint8)
    row = np.zeros(max(n, 1), np.uint8)
    qy = np.zeros(max(n, 1), np.int32)
    qt = np.zeros(max(n, 1), np.int32)
    rc = lib().orc_decompress_fields(n_sectors, n_rows, vals, counts, n_tracks, n, _ptr(sector, _PU8),
                                     _ptr(row, _PU8), _ptr(qy, _P32), _ptr(qt, _P32))
    if rc:
        raise ValueError(f"decompress_fields failed ({rc})")
    return sector[:n], row[:n], qy[:n], qt[:n]


def code_stream(v, chunk=4096, roundtrip=True):
    """Coded bytes of one integer stream (table, chunk sizes, rANS chunks,
    escapes) and whether every chunk decodes back exactly."""
    v = np.ascontiguousarray(v, np.uint32)
    nb = C.c_int64(0)
    ok = C.c_int32(0)
    rc = lib().orc_code_stream(_ptr(v, _PU32), v.size, chunk, C.byref(nb), C.byref(ok) if roundtrip else None)
    if rc:
        raise ValueError(f"code_stream failed ({rc})")
    return int(nb.value), bool(ok.value) if roundtrip else None


def pack_stream(v, chunk=4096) -> np.ndarray:
    """One integer stream as a self-contained coded container (format stated
    at orc_pack_stream in tpc_oracle_compress.c)."""
    v = np.ascontiguousarray(v, np.uint32)
    L = lib()
    size = L.orc_pack_stream(_ptr(v, _PU32), v.size, chunk, None)
    if size < 0:
        raise ValueError("pack_stream failed")
    out = np.zeros(size, np.uint8)
    if L.orc_pack_stream(_ptr(v, _PU32), v.size, chunk, _ptr(out, _PU8)) != size:
        raise ValueError("pack_stream failed")
    return out


def unpack_stream(data, vcap=None) -> np.ndarray:
    """The values of a container written by pack_stream.  Without vcap the
    capacity is the value count of the container's header (its first four
    bytes, little-endian); a very compressible stream holds more values than
    bytes."""
    data = np.ascontiguousarray(data, np.uint8)
    if vcap is None:
        if data.size < 12 + 512:
            raise ValueError("malformed container")
        vcap, chunk = (int(v) for v in data[:8].view("<u4"))
        # sanity bound: every chunk of `chunk` values carries at least its 4-byte size entry
        if vcap > chunk * max(1, (data.size - 12 - 512) // 4):
            raise ValueError("malformed container")
    vcap = int(vcap)
    v = np.zeros(max(vcap, 1), np.uint32)
    n = C.c_int64(0)
    used = lib().orc_unpack_stream(_ptr(data, _PU8), data.size, _ptr(v, _PU32), vcap, C.byref(n))
    if used < 0 or used != data.size:
        raise ValueError("malformed container")
    return v[:n.value]


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


def helix64(x, p, x2, kb):
    """FP64 helix step of a bare state with its Jacobian: (ok, x, p, F)."""
    xx = np.array([x], np.float64)
    pp = np.ascontiguousarray(p, np.float64).copy()
    F = np.zeros((5, 5))
    ok = lib().orc_helix64(_ptr(xx, _PD), _ptr(pp, _PD), x2, kb, _ptr(F, _PD))
    return bool(ok), float(xx[0]), pp, F


def rotate64(x, p, cs, sn, kb):
    """FP64 frame rotation of a bare state with its Jacobian: (ok, x, p, J)."""
    xx = np.array([x], np.float64)
    pp = np.ascontiguousarray(p, np.float64).copy()
    J = np.zeros((5, 5))
    ok = lib().orc_rotate64(_ptr(xx, _PD), _ptr(pp, _PD), cs, sn, kb, _ptr(J, _PD))
    return bool(ok), float(xx[0]), pp, J


# ---- calibration chi2 and gradient ------------------------------------------------
CALIB_NSPL = 8
VERTEX_VAR = 0.01      # primary-vertex pseudo-measurement variance (cm^2)
TGL_VAR = 9e-8       # dip angle of the matched inner track: variance (sigma 3e-4)


def calib_n_theta(n_sectors=36):
    return 2 + n_sectors * CALIB_NSPL * CALIB_NSPL * 2


@dataclasses.dataclass
class CalibTracks:
    """Tracks and clusters of a calibration problem (host arrays)."""
    sector: np.ndarray       # [T] int32
    x: np.ndarray            # [T] float32
    param: np.ndarray        # [T, 5] float32 (tracker z frame)
    off: np.ndarray          # [T+1] int32
    clus: np.ndarray         # cluster indices, inner -> outer
    tcoll: np.ndarray        # [T] float32, NaN = unused
    cl_sector: np.ndarray    # [n] uint8
    cl_row: np.ndarray       # [n] uint8
    cl_y: np.ndarray         # [n] float32
    cl_t: np.ndarray         # [n] float32 drift time (us)
    row_x: np.ndarray        # float32
    n_sectors: int = 36
    z_max: float = 250.0
    bz: float = 0.5
    v_nom: float = 2.58

    def __post_init__(self):
        self.sector = np.ascontiguousarray(self.sector, np.int32)
        self.x = np.ascontiguousarray(self.x, np.float32)
        self.param = np.ascontiguousarray(self.param, np.float32)
        self.off = np.ascontiguousarray(self.off, np.int32)
        self.clus = np.ascontiguousarray(self.clus, np.int32)
        self.tcoll = np.ascontiguousarray(self.tcoll, np.float32)
        self.cl_sector = np.ascontiguousarray(self.cl_sector, np.uint8)
        self.cl_row = np.ascontiguousarray(self.cl_row, np.uint8)
        self.cl_y = np.ascontiguousarray(self.cl_y, np.float32)
        self.cl_t = np.ascontiguousarray(self.cl_t, np.float32)
        self.row_x = np.ascontiguousarray(self.row_x, np.float32)

    @property
    def n_tracks(self):
        return int(self.x.shape[0])

    def geom(self):
        return OrcGeom(self.n_sectors, self.row_x.shape[0], _ptr(self.row_x, _PF), self.z_max, 1)


def calib(tr: CalibTracks, theta, weight=None, grad=True, params: dict | None = None, vtx_var=VERTEX_VAR,
          tgl_ext=None, tgl_var=TGL_VAR):
    """Per-track calibration chi2, used flags and (optionally) the gradient of
    sum_r weight[r] chi2_r with respect to theta (all binary64).  tgl_ext:
    per-track dip angle from outside the TPC (NaN: none), an update of
    variance tgl_var after the vertex step."""
    th = np.ascontiguousarray(theta, np.float64)
    assert th.shape == (calib_n_theta(tr.n_sectors),)
    T = tr.n_tracks
    chi2 = np.zeros(T)
    used = np.zeros(T, np.uint8)
    g = np.zeros_like(th) if grad else None
    w = None if weight is None else np.ascontiguousarray(weight, np.float64)
    te = None if tgl_ext is None else np.ascontiguousarray(tgl_ext, np.float32)
    P = _params(params)
    G = tr.geom()
    rc = lib().orc_calib(C.byref(P), C.byref(G), tr.bz, tr.v_nom, vtx_var, T, _ptr(tr.sector, _P32),
                         _ptr(tr.x, _PF), _ptr(tr.param, _PF), _ptr(tr.off, _P32), _ptr(tr.clus, _P32),
                         _ptr(tr.cl_sector, _PU8), _ptr(tr.cl_row, _PU8), _ptr(tr.cl_y, _PF), _ptr(tr.cl_t, _PF),
                         _ptr(tr.tcoll, _PF), _ptr(th, _PD), None if w is None else _ptr(w, _PD),
                         _ptr(chi2, _PD), _ptr(used, _PU8), None if g is None else _ptr(g, _PD),
                         None if te is None else _ptr(te, _PF), tgl_var)
    if rc:
        raise ValueError(f"orc_calib failed ({rc})")
    return chi2, used.astype(bool), g


CALIB_QPT_MAX = 5.0     # loopers below pT = 0.2 GeV/c are left out of the calibration


def calib_select(t_coll, status, param, qpt_max=CALIB_QPT_MAX):
    """Collision times with NaN for the tracks the calibration leaves out
    (failed refit, or |q/pT| > qpt_max on the binary32 parameters)."""
    t = np.ascontiguousarray(t_coll, np.float32)
    st = np.ascontiguousarray(status, np.int32)
    p = np.ascontiguousarray(param, np.float32).reshape(-1, 5)
    out = np.zeros(max(t.size, 1), np.float32)
    lib().orc_calib_select(t.size, _ptr(t, _PF), _ptr(st, _P32), _ptr(p, _PF), qpt_max, _ptr(out, _PF))
    return out[:t.size]


def calib_tracks_of(ev, r: OracleResult, t_coll=None, qpt_max=CALIB_QPT_MAX) -> CalibTracks:
    """The calibration problem of an oracle tracking result: the oracle's own
    tracks (binary32 parameters, as the calibration pass consumes them), the
    collision time of each (given, e.g. from generator truth) and the
    oracle's selection."""
    if t_coll is None:
        raise ValueError("t_coll (collision time per track) is needed")
    p32 = r.tr_p.astype(np.float32)
    tc = calib_select(t_coll, r.tr_status, p32, qpt_max)
    return CalibTracks(r.tr_sector, r.tr_x.astype(np.float32), p32, r.tr_off.astype(np.int32),
                       r.tr_clus.astype(np.int32), tc, ev.sector, ev.row, ev.y, ev.zt, ev.row_x,
                       n_sectors=ev.n_sectors, z_max=ev.z_max, bz=ev.bz, v_nom=ev.v_drift)


def calib_measure(tr: CalibTracks, theta, idx, tc):
    """Calibrated (m_y, m_z) of clusters idx, each with collision time tc."""
    th = np.ascontiguousarray(theta, np.float64)
    idx = np.asarray(idx)
    s = np.ascontiguousarray(tr.cl_sector[idx])
    r = np.ascontiguousarray(tr.cl_row[idx])
    y = np.ascontiguousarray(tr.cl_y[idx])
    t = np.ascontiguousarray(tr.cl_t[idx])
    tcc = np.ascontiguousarray(np.broadcast_to(np.asarray(tc, np.float32), idx.shape), np.float32)
    my = np.zeros(idx.size)
    mz = np.zeros(idx.size)
    G = tr.geom()
    lib().orc_calib_measure(C.byref(G), _ptr(th, _PD), idx.size, _ptr(s, _PU8), _ptr(r, _PU8), _ptr(y, _PF),
                            _ptr(t, _PF), _ptr(tcc, _PF), _ptr(my, _PD), _ptr(mz, _PD))
    return my, mz


def calib_explain(tr: CalibTracks, theta, r, params: dict | None = None, vtx_var=VERTEX_VAR):
    """One track's inward pass: per step F (5x5), reference (y, z), measurement
    and variances, and the chi2; None when a reference step fails."""
    th = np.ascontiguousarray(theta, np.float64)
    n = int(tr.off[r + 1] - tr.off[r])
    F = np.zeros((n + 1, 5, 5))
    h = np.zeros((n + 1, 2))
    m = np.zeros((n + 1, 2))
    v = np.zeros((n + 1, 2))
    chi2 = np.zeros(1)
    P = _params(params)
    G = tr.geom()
    rc = lib().orc_calib_explain(C.byref(P), C.byref(G), tr.bz, tr.v_nom, vtx_var, _ptr(tr.sector, _P32),
                                 _ptr(tr.x, _PF), _ptr(tr.param, _PF), _ptr(tr.off, _P32), _ptr(tr.clus, _P32),
                                 _ptr(tr.cl_sector, _PU8), _ptr(tr.cl_row, _PU8), _ptr(tr.cl_y, _PF),
                                 _ptr(tr.cl_t, _PF), _ptr(tr.tcoll, _PF), _ptr(th, _PD), r, _ptr(F, _PD),
                                 _ptr(h, _PD), _ptr(m, _PD), _ptr(v, _PD), _ptr(chi2, _PD))
    if rc:
        return None
    return F, h, m, v, float(chi2[0])


def bspline_all(u):
    b = np.zeros(CALIB_NSPL)
    d = np.zeros(CALIB_NSPL)
    lib().orc_bspline_all(float(u), _ptr(b, _PD), _ptr(d, _PD))
    return b, d
