"""Differentiable calibration chi2 of the refit (binding of include/tpc_calib.h).

``CalibRefit`` holds the tracks (the tracker's output) and their clusters on
the device; ``calib_chi2(theta, calib)`` is a ``torch.autograd.Function``
returning the per-track calibration chi2, whose backward runs the CUDA
adjoint (tpc_calib_backward) from the checkpoints its forward stored.  Both
passes run in libtpcgpu.so; this module only marshals pointers.

theta (float32, device): [v_drift (cm/us), t0 (us), spline[n_sectors][8][8][2]]
with the spline the per-sector distortion map (dy, dz) over (pad-row radius,
|z|), see tpc_calib.h.
"""
from __future__ import annotations

import ctypes as C

import torch

from . import abi

VERTEX_VAR = 0.01          # primary-vertex pseudo-measurement variance (cm^2)
TGL_VAR = 9e-8             # dip angle of the matched inner track: variance (sigma 3e-4)
QPT_MAX = 5.0              # TPC_CALIB_QPT_MAX: tracks below pT = 0.2 GeV/c (loopers) are left out


def select_tracks(t_coll: torch.Tensor, status: torch.Tensor, param: torch.Tensor, qpt_max: float = QPT_MAX):
    """Collision times with NaN for the tracks the calibration leaves out
    (tpc_calib_select: failed refits and |q/pT| > qpt_max, the low-pT loopers
    whose later legs do not come from the vertex)."""
    T = int(t_coll.shape[0])
    dev = t_coll.device
    if dev.type != "cuda":
        raise RuntimeError("tpc_calib_select needs CUDA tensors")
    t_coll = t_coll.to(dtype=torch.float32).contiguous()
    status = status[:T].to(device=dev, dtype=torch.int32).contiguous()
    param = param[:T].to(device=dev, dtype=torch.float32).contiguous()
    out = torch.empty_like(t_coll)
    st = torch.cuda.current_stream(dev)
    rc = abi.lib().tpc_calib_select(T, C.c_void_p(t_coll.data_ptr()), C.c_void_p(status.data_ptr()),
                                    C.c_void_p(param.data_ptr()), float(qpt_max), C.c_void_p(out.data_ptr()),
                                    C.c_void_p(st.cuda_stream))
    if rc:
        raise abi.TpcError(rc, "tpc_calib_select")
    return out


def nominal_theta(v_drift: float, n_sectors: int = 36, device="cuda") -> torch.Tensor:
    th = torch.zeros(abi.calib_n_theta(n_sectors), dtype=torch.float32, device=device)
    th[0] = v_drift
    return th


class CalibRefit:
    """Tracks + clusters of one calibration problem, resident on the device.

    sector, x, param, clus_offset, clus_index: the tracker's output (first
    n_tracks rows), t_coll: collision time per track (NaN = not used, e.g.
    from :func:`select_tracks`), cl_*: the cluster SoA the indices refer to
    (cl_t = drift time in us).
    """

    def __init__(self, sector, x, param, clus_offset, clus_index, t_coll, cl_sector, cl_row, cl_y, cl_t, row_x,
                 n_sectors: int = 36, z_max: float = 250.0, bz: float = 0.5, v_nominal: float = 2.58,
                 params: abi.TpcParams | None = None, vertex_var: float = VERTEX_VAR, tgl_ext=None,
                 tgl_var: float = TGL_VAR):
        self.lib = abi.lib()
        dev = param.device
        if dev.type != "cuda":
            raise RuntimeError("the calibration pass needs CUDA tensors")
        T = int(x.shape[0])

        def prep(t, dt, n):
            t = t[:n] if t.dim() == 1 else t[:n]
            if t.dtype != dt or not t.is_cuda or not t.is_contiguous():
                t = t.to(device=dev, dtype=dt).contiguous()
            return t

        self.t = dict(sector=prep(sector, torch.int32, T), x=prep(x, torch.float32, T),
                      param=prep(param, torch.float32, T), clus_offset=prep(clus_offset, torch.int32, T + 1),
                      clus_index=clus_index.to(device=dev, dtype=torch.int32).contiguous(),
                      t_coll=prep(t_coll, torch.float32, T), cl_sector=cl_sector.contiguous(),
                      cl_row=cl_row.contiguous(), cl_y=cl_y.contiguous(), cl_t=cl_t.contiguous())
        if tgl_ext is not None:
            self.t["tgl_ext"] = prep(tgl_ext, torch.float32, T)
        for k, dt in (("cl_sector", torch.uint8), ("cl_row", torch.uint8), ("cl_y", torch.float32),
                      ("cl_t", torch.float32)):
            if self.t[k].dtype != dt or not self.t[k].is_cuda:
                raise ValueError(f"{k} must be a CUDA {dt} tensor")
        self.n_tracks = T
        self.n_clusters = int(self.t["cl_y"].shape[0])
        self.n_sectors = n_sectors
        self.n_theta = abi.calib_n_theta(n_sectors)
        self.geometry = abi.make_geometry(row_x, n_sectors, z_max, True)
        self.params = params if params is not None else abi.tpc_params_default()
        self.bz, self.v_nominal, self.vertex_var = float(bz), float(v_nominal), float(vertex_var)
        self.device = dev
        s = C.c_size_t(0)
        rc = self.lib.tpc_calib_workspace_size(C.byref(self.geometry), T, self.n_clusters, C.byref(s))
        if rc:
            raise abi.TpcError(rc, "tpc_calib_workspace_size")
        self.ws_bytes = int(s.value)
        st = self.t
        self._tracks = abi.TpcCalibTracks(T, st["sector"].data_ptr(), st["x"].data_ptr(), st["param"].data_ptr(),
                                          st["clus_offset"].data_ptr(), st["clus_index"].data_ptr(),
                                          st["t_coll"].data_ptr(), self.n_clusters, st["cl_sector"].data_ptr(),
                                          st["cl_row"].data_ptr(), st["cl_y"].data_ptr(), st["cl_t"].data_ptr(),
                                          st["tgl_ext"].data_ptr() if "tgl_ext" in st else None, float(tgl_var))

    @classmethod
    def from_result(cls, res, t_coll, sector, row, y, zt, row_x, **kw):
        """From a TrackResult of the tracker and the cluster tensors it tracked."""
        T = res.n_tracks
        return cls(res.sector[:T], res.x[:T], res.param[:T], res.clus_offset[:T + 1], res.clus_index, t_coll,
                   sector, row, y, zt, row_x, **kw)

    def _theta(self, theta):
        if theta.shape != (self.n_theta,) or theta.dtype != torch.float32 or not theta.is_cuda:
            raise ValueError(f"theta must be a CUDA float32 tensor of {self.n_theta} values")
        return theta.contiguous()

    def forward(self, theta: torch.Tensor, check: bool = True):
        """Per-track chi2 (float32 [T]), used flags (uint8 [T]) and the
        workspace holding the checkpoints of this pass."""
        theta = self._theta(theta)
        T = self.n_tracks
        chi2 = torch.empty(T, dtype=torch.float32, device=self.device)
        used = torch.empty(T, dtype=torch.uint8, device=self.device)
        ws = torch.empty(self.ws_bytes, dtype=torch.uint8, device=self.device)
        st = torch.cuda.current_stream(self.device)
        rc = self.lib.tpc_calib_forward(C.byref(self.params), C.byref(self.geometry), self.bz, self.v_nominal,
                                        self.vertex_var, C.byref(self._tracks), C.c_void_p(theta.data_ptr()),
                                        C.c_void_p(chi2.data_ptr()), C.c_void_p(used.data_ptr()),
                                        C.c_void_p(ws.data_ptr()), self.ws_bytes, C.c_void_p(st.cuda_stream))
        if rc:
            raise abi.TpcError(rc, "tpc_calib_forward")
        if check:
            self.check(ws)
        return chi2, used, ws

    def backward(self, theta: torch.Tensor, dchi2: torch.Tensor, used: torch.Tensor, ws: torch.Tensor,
                 check: bool = True) -> torch.Tensor:
        """Gradient (float64 [n_theta]) of sum_r dchi2[r] chi2_r."""
        theta = self._theta(theta)
        dchi2 = dchi2.to(device=self.device, dtype=torch.float32).contiguous()
        grad = torch.empty(self.n_theta, dtype=torch.float64, device=self.device)
        st = torch.cuda.current_stream(self.device)
        rc = self.lib.tpc_calib_backward(C.byref(self.params), C.byref(self.geometry), self.bz, self.v_nominal,
                                         self.vertex_var, C.byref(self._tracks), C.c_void_p(theta.data_ptr()),
                                         C.c_void_p(dchi2.data_ptr()), C.c_void_p(used.data_ptr()),
                                         C.c_void_p(ws.data_ptr()), self.ws_bytes, C.c_void_p(grad.data_ptr()),
                                         C.c_void_p(st.cuda_stream))
        if rc:
            raise abi.TpcError(rc, "tpc_calib_backward")
        if check:
            self.check(ws)
        return grad

    def fit(self, theta: torch.Tensor, **opts):
        """Closed-loop calibration (tpc_calib_fit): theta minimising the summed
        chi2 of the selected tracks plus the spline prior, from ``theta`` (a
        copy is returned with the report).  Keyword options: the fields of
        tpc_calib_fit_opts (prior_sigma, scale_v, scale_t0, max_iter, rounds,
        chi2ndf_first, anchor_cut_first, chi2ndf_cut, anchor_cut, ftol).  The
        report holds the last selection too: ``t_used`` / ``tgl_used`` (CUDA
        float32 [n_tracks], NaN where left out)."""
        th = self._theta(theta).clone()
        o = abi.TpcCalibFitOpts()
        self.lib.tpc_calib_fit_defaults(C.byref(o))
        for k, v in opts.items():
            if not hasattr(o, k):
                raise ValueError(f"unknown fit option {k}")
            setattr(o, k, v)
        s = C.c_size_t(0)
        rc = self.lib.tpc_calib_fit_workspace_size(C.byref(self.geometry), self.n_tracks, self.n_clusters,
                                                   C.byref(s))
        if rc:
            raise abi.TpcError(rc, "tpc_calib_fit_workspace_size")
        ws = torch.empty(int(s.value), dtype=torch.uint8, device=self.device)
        rep = abi.TpcCalibFitReport()
        st = torch.cuda.current_stream(self.device)
        tu = torch.empty(max(self.n_tracks, 1), dtype=torch.float32, device=self.device)
        gu = torch.empty_like(tu)
        rc = self.lib.tpc_calib_fit(C.byref(self.params), C.byref(self.geometry), self.bz, self.v_nominal,
                                    self.vertex_var, C.byref(self._tracks), C.byref(o), C.c_void_p(th.data_ptr()),
                                    C.c_void_p(ws.data_ptr()), int(s.value), C.c_void_p(tu.data_ptr()),
                                    C.c_void_p(gu.data_ptr()), C.byref(rep), C.c_void_p(st.cuda_stream))
        if rc:
            raise abi.TpcError(rc, "tpc_calib_fit")
        out = {k: getattr(rep, k) for k, _ in rep._fields_}
        out["t_used"] = tu[:self.n_tracks]
        out["tgl_used"] = gu[:self.n_tracks]
        return th, out

    def check(self, ws):
        err = C.c_int32(0)
        st = torch.cuda.current_stream(self.device)
        rc = self.lib.tpc_calib_status(C.c_void_p(ws.data_ptr()), C.byref(err), C.c_void_p(st.cuda_stream))
        if rc:
            raise abi.TpcError(rc, "tpc_calib_status")
        if err.value:
            raise abi.TpcError(abi.TPC_ERR_DATA, f"calibration pass (flags {err.value})")


class _CalibChi2(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, calib):
        chi2, used, ws = calib.forward(theta.detach())
        ctx.calib = calib
        ctx.save_for_backward(theta, used, ws)
        ctx.mark_non_differentiable(used)
        return chi2, used

    @staticmethod
    def backward(ctx, g_chi2, g_used):
        theta, used, ws = ctx.saved_tensors
        if g_chi2 is None:
            return None, None
        grad = ctx.calib.backward(theta.detach(), g_chi2, used, ws)
        return grad.to(theta.dtype), None


def calib_chi2(theta: torch.Tensor, calib: CalibRefit):
    """Per-track calibration chi2 (differentiable in theta) and the used flags."""
    return _CalibChi2.apply(theta, calib)
