"""ctypes mirror of include/tpc_track.h and include/tpc_calib.h (argument marshalling only)."""
from __future__ import annotations

import ctypes as C
import os

from . import build as _build

TPC_OK = 0
TPC_ERR_ARG = -1
TPC_ERR_CAPACITY = -2
TPC_ERR_TIMEOUT = -3
TPC_ERR_CUDA = -4
TPC_ERR_DATA = -5


class TpcError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        super().__init__(f"{what}: {tpc_error_string(code)} ({code})" if what else f"{tpc_error_string(code)} ({code})")


class TpcParams(C.Structure):
    _fields_ = [("dy_link", C.c_float), ("dz_link", C.c_float), ("s_max_link", C.c_float),
                ("sigma_y", C.c_float), ("sigma_z", C.c_float),
                ("c0_snp", C.c_float), ("c0_tgl", C.c_float), ("c0_qpt", C.c_float),
                ("win_nsigma", C.c_float), ("win_min", C.c_float), ("win_max", C.c_float),
                ("chi2_cut", C.c_float), ("max_miss", C.c_int32), ("min_hits", C.c_int32),
                ("min_owned", C.c_int32), ("edge_margin", C.c_float), ("merge_dz", C.c_float),
                ("merge_chi2", C.c_float), ("refit_passes", C.c_int32), ("refit_inflate", C.c_float),
                ("z_cell", C.c_float),
                ("max_z_cells", C.c_int32), ("y_bins", C.c_int32), ("tracklets_per_1k", C.c_int32),
                ("queue_blocks_per_sm", C.c_int32), ("fp64_final", C.c_int32),
                ("profile", C.c_int32), ("packed_links", C.c_int32), ("merge_pairs_per_1k", C.c_int32),
                ("tube_radius", C.c_float), ("pt_min_physics", C.c_float), ("outlier_chi2", C.c_float),
                ("looper_qpt_min", C.c_float)]


class TpcGeometry(C.Structure):
    _fields_ = [("n_sectors", C.c_int32), ("n_rows", C.c_int32), ("row_x", C.POINTER(C.c_float)),
                ("z_max", C.c_float), ("continuous", C.c_int32)]


class TpcClusters(C.Structure):
    _fields_ = [("n", C.c_int32), ("sector", C.c_void_p), ("row", C.c_void_p), ("y", C.c_void_p),
                ("zt", C.c_void_p)]


class TpcTracks(C.Structure):
    _fields_ = [("capacity_tracks", C.c_int32), ("capacity_clusters", C.c_int32),
                ("sector", C.c_void_p), ("x", C.c_void_p), ("param", C.c_void_p), ("cov", C.c_void_p),
                ("chi2", C.c_void_p), ("ndf", C.c_void_p), ("status", C.c_void_p), ("nclus", C.c_void_p),
                ("clus_offset", C.c_void_p), ("clus_index", C.c_void_p), ("assign", C.c_void_p),
                ("frame", C.c_void_p),
                ("cov64", C.c_void_p), ("chi2_64", C.c_void_p),
                ("z", C.c_void_p), ("link_up_raw", C.c_void_p), ("link_dn_raw", C.c_void_p),
                ("link_up", C.c_void_p), ("link_dn", C.c_void_p), ("is_start", C.c_void_p),
                ("cl_flags", C.c_void_p), ("adjacent", C.c_void_p),
                ("looper_group", C.c_void_p), ("looper_leg", C.c_void_p),
                ("n_tracks", C.c_int32), ("n_tracklets", C.c_int32), ("n_segments", C.c_int32),
                ("tracklets_needed", C.c_int64), ("tracks_needed", C.c_int64), ("clusters_needed", C.c_int64),
                ("n_launches", C.c_int32), ("stage_ms", C.c_float * 10), ("work", C.c_int64 * 5),
                ("n_rejected", C.c_int32), ("refit_event", C.c_void_p)]

class TpcCalibTracks(C.Structure):
    _fields_ = [("n_tracks", C.c_int32), ("sector", C.c_void_p), ("x", C.c_void_p), ("param", C.c_void_p),
                ("clus_offset", C.c_void_p), ("clus_index", C.c_void_p), ("t_coll", C.c_void_p),
                ("n_clusters", C.c_int64), ("cl_sector", C.c_void_p), ("cl_row", C.c_void_p),
                ("cl_y", C.c_void_p), ("cl_t", C.c_void_p), ("tgl_ext", C.c_void_p), ("tgl_var", C.c_float)]


class TpcCompressIn(C.Structure):
    _fields_ = [("n", C.c_int64), ("n_sectors", C.c_int32), ("n_rows", C.c_int32), ("sector", C.c_void_p),
                ("row", C.c_void_p), ("y", C.c_void_p), ("zt", C.c_void_p), ("n_tracks", C.c_int32),
                ("n_attached", C.c_int64), ("clus_offset", C.c_void_p), ("clus_index", C.c_void_p),
                ("assign", C.c_void_p)]


# stream order of tpc_compress_fields / tpc_compress_frame
CMP_STREAMS = ("n_track", "head_sector", "head_row", "head_y", "head_t", "d_sector", "d_row", "res_y", "res_t",
               "u_count", "u_dt", "u_y")


class TpcCalibFitOpts(C.Structure):
    _fields_ = [("prior_sigma", C.c_float), ("scale_v", C.c_float), ("scale_t0", C.c_float),
                ("max_iter", C.c_int32), ("rounds", C.c_int32), ("chi2ndf_first", C.c_float),
                ("anchor_cut_first", C.c_float), ("chi2ndf_cut", C.c_float), ("anchor_cut", C.c_float),
                ("ftol", C.c_double)]


class TpcCalibFitReport(C.Structure):
    _fields_ = [("f_start", C.c_double), ("f_final", C.c_double), ("evaluations", C.c_int32),
                ("rounds", C.c_int32), ("tracks", C.c_int32), ("anchors", C.c_int32)]


CALIB_NSPL = 8
CALIB_CKPT_STEPS = 16


def calib_n_theta(n_sectors: int) -> int:
    return 2 + n_sectors * CALIB_NSPL * CALIB_NSPL * 2


STAGES = ("prep", "bin", "neighbours", "clean_start", "tracklets", "select", "merge", "assemble", "refit")
ATTACH_STAGE = 9            # tpc_tracks.stage_ms index of the cluster attachment (when requested)
CL_ATTACHED, CL_ADJACENT, CL_PROTECTED, CL_REMOVE = 1, 2, 4, 8


EXPORTED = ("tpc_params_default", "tpc_workspace_size", "tpc_workspace_size_batched", "tpc_track",
            "tpc_track_batched", "tpc_prepare", "tpc_prepare_staging_size", "tpc_prepare_async", "tpc_track_async", "tpc_export_tracklets", "tpc_links_static",
            "tpc_error_string", "tpc_calib_workspace_size", "tpc_calib_forward", "tpc_calib_backward",
            "tpc_calib_status", "tpc_calib_select", "tpc_calib_fit_defaults", "tpc_calib_fit_workspace_size",
            "tpc_calib_fit", "tpc_rans_workspace_size", "tpc_rans_max_bytes", "tpc_rans_encode",
            "tpc_compress_workspace_size", "tpc_compress_max_size", "tpc_compress_fields", "tpc_compress_frame",
            "tpc_probe_fma")

_lib = None


def lib_path() -> str:
    return _build.LIB


def lib(build_if_missing: bool = True):
    """Load libtpcgpu.so (built in-tree for sm_103a); raises if it cannot."""
    global _lib
    if _lib is None:
        path = _build.build() if build_if_missing else _build.LIB
        if not os.path.exists(path):
            raise OSError(f"CUDA tracker library missing: {path}")
        L = C.CDLL(path)
        L.tpc_params_default.argtypes = [C.POINTER(TpcParams)]
        L.tpc_rans_workspace_size.argtypes = [C.c_int64, C.c_int32, C.POINTER(C.c_size_t)]
        L.tpc_rans_max_bytes.argtypes = [C.c_int64, C.c_int32, C.POINTER(C.c_int64)]
        L.tpc_rans_encode.argtypes = [C.c_void_p, C.c_int64, C.c_int32, C.c_void_p, C.c_size_t, C.c_void_p,
                                      C.c_void_p, C.c_void_p, C.c_int64, C.POINTER(C.c_int64), C.c_void_p]
        L.tpc_calib_fit_defaults.argtypes = [C.POINTER(TpcCalibFitOpts)]
        L.tpc_calib_fit_workspace_size.argtypes = [C.POINTER(TpcGeometry), C.c_int32, C.c_int64,
                                                   C.POINTER(C.c_size_t)]
        L.tpc_calib_fit.argtypes = [C.POINTER(TpcParams), C.POINTER(TpcGeometry), C.c_float, C.c_float, C.c_float,
                                    C.POINTER(TpcCalibTracks), C.POINTER(TpcCalibFitOpts), C.c_void_p, C.c_void_p,
                                    C.c_size_t, C.c_void_p, C.c_void_p, C.POINTER(TpcCalibFitReport), C.c_void_p]
        L.tpc_compress_workspace_size.argtypes = [C.POINTER(TpcCompressIn), C.c_int32, C.POINTER(C.c_size_t)]
        L.tpc_compress_max_size.argtypes = [C.POINTER(TpcCompressIn), C.c_int32, C.POINTER(C.c_int64),
                                            C.POINTER(C.c_int64)]
        L.tpc_compress_fields.argtypes = [C.POINTER(TpcCompressIn), C.c_int32, C.c_int32, C.c_void_p, C.c_size_t,
                                          C.c_void_p, C.c_int64, C.POINTER(C.c_int64), C.c_void_p]
        L.tpc_compress_frame.argtypes = [C.POINTER(TpcCompressIn), C.c_int32, C.c_int32, C.c_int32, C.c_void_p,
                                         C.c_size_t, C.c_void_p, C.c_int64, C.POINTER(C.c_int64), C.c_void_p]
        L.tpc_workspace_size.argtypes = [C.POINTER(TpcParams), C.POINTER(TpcGeometry), C.c_int64,
                                         C.POINTER(C.c_size_t)]
        L.tpc_track.argtypes = [C.POINTER(TpcParams), C.POINTER(TpcGeometry), C.c_float, C.c_float,
                                C.POINTER(TpcClusters), C.c_void_p, C.c_size_t, C.POINTER(TpcTracks), C.c_void_p]
        L.tpc_workspace_size_batched.argtypes = [C.POINTER(TpcParams), C.POINTER(TpcGeometry), C.c_int64, C.c_int32,
                                                 C.POINTER(C.c_size_t)]
        L.tpc_track_batched.argtypes = [C.POINTER(TpcParams), C.POINTER(TpcGeometry), C.c_float, C.c_float,
                                        C.POINTER(TpcClusters), C.c_int32, C.POINTER(C.c_int32), C.c_void_p,
                                        C.c_size_t, C.POINTER(TpcTracks), C.c_void_p]
        L.tpc_prepare.argtypes = [C.POINTER(TpcParams), C.POINTER(TpcGeometry), C.c_int32, C.c_int32,
                                  C.POINTER(C.c_int32), C.c_void_p, C.c_size_t, C.c_void_p]
        L.tpc_prepare_staging_size.argtypes = [C.c_int32, C.POINTER(C.c_size_t)]
        L.tpc_prepare_async.argtypes = [C.POINTER(TpcParams), C.POINTER(TpcGeometry), C.c_int32, C.c_int32,
                                        C.POINTER(C.c_int32), C.c_void_p, C.c_size_t, C.c_void_p, C.c_size_t,
                                        C.c_void_p]
        L.tpc_track_async.argtypes = [C.POINTER(TpcParams), C.POINTER(TpcGeometry), C.c_float, C.c_float,
                                      C.POINTER(TpcClusters), C.c_int32, C.c_void_p, C.c_size_t, C.POINTER(TpcTracks),
                                      C.c_void_p, C.c_void_p]
        L.tpc_export_tracklets.argtypes = [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p,
                                           C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_int32), C.c_void_p]
        L.tpc_calib_workspace_size.argtypes = [C.POINTER(TpcGeometry), C.c_int32, C.c_int64, C.POINTER(C.c_size_t)]
        L.tpc_calib_forward.argtypes = [C.POINTER(TpcParams), C.POINTER(TpcGeometry), C.c_float, C.c_float, C.c_float,
                                        C.POINTER(TpcCalibTracks), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                        C.c_size_t, C.c_void_p]
        L.tpc_calib_backward.argtypes = [C.POINTER(TpcParams), C.POINTER(TpcGeometry), C.c_float, C.c_float,
                                         C.c_float, C.POINTER(TpcCalibTracks), C.c_void_p, C.c_void_p, C.c_void_p,
                                         C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p]
        L.tpc_calib_status.argtypes = [C.c_void_p, C.POINTER(C.c_int32), C.c_void_p]
        L.tpc_calib_select.argtypes = [C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_float, C.c_void_p,
                                       C.c_void_p]
        L.tpc_probe_fma.argtypes = [C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_void_p, C.POINTER(C.c_int64),
                                    C.c_void_p]
        L.tpc_error_string.argtypes = [C.c_int]
        L.tpc_error_string.restype = C.c_char_p
        _lib = L
    return _lib


def tpc_error_string(code: int) -> str:
    return lib().tpc_error_string(int(code)).decode()


def tpc_params_default(**overrides) -> TpcParams:
    p = TpcParams()
    rc = lib().tpc_params_default(C.byref(p))
    if rc:
        raise TpcError(rc, "tpc_params_default")
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def make_geometry(row_x, n_sectors: int, z_max: float, continuous: bool):
    import numpy as np
    rx = np.ascontiguousarray(row_x, np.float32)
    g = TpcGeometry(n_sectors, rx.shape[0], rx.ctypes.data_as(C.POINTER(C.c_float)), z_max, int(continuous))
    g._keep = rx          # keep the host array alive with the struct
    return g


def tpc_workspace_size(params: TpcParams, geometry: TpcGeometry, n_clusters: int, n_frames: int = 1) -> int:
    out = C.c_size_t()
    rc = lib().tpc_workspace_size_batched(C.byref(params), C.byref(geometry), int(n_clusters), int(n_frames),
                                          C.byref(out))
    if rc:
        raise TpcError(rc, "tpc_workspace_size")
    return int(out.value)
