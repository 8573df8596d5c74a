"""Tracker: owns the device workspace and output buffers for one maximum input
size and calls tpc_track on torch's current CUDA stream."""
from __future__ import annotations

import ctypes as C
import dataclasses

import numpy as np
import torch

from . import abi


def _p(t: torch.Tensor | None):
    return None if t is None else C.c_void_p(t.data_ptr())


@dataclasses.dataclass
class TrackResult:
    """Device tensors (views of the tracker's buffers, valid until its next call)."""
    n_tracks: int
    sector: torch.Tensor
    x: torch.Tensor
    param: torch.Tensor
    cov: torch.Tensor
    chi2: torch.Tensor
    ndf: torch.Tensor
    status: torch.Tensor
    nclus: torch.Tensor
    clus_offset: torch.Tensor
    clus_index: torch.Tensor
    assign: torch.Tensor
    cov64: torch.Tensor | None = None
    chi2_64: torch.Tensor | None = None
    z: torch.Tensor | None = None
    link_up_raw: torch.Tensor | None = None
    link_dn_raw: torch.Tensor | None = None
    link_up: torch.Tensor | None = None
    link_dn: torch.Tensor | None = None
    is_start: torch.Tensor | None = None
    cl_flags: torch.Tensor | None = None      # [n] uint8 CL_* flags (attach=True)
    adjacent: torch.Tensor | None = None      # [n] int32 adjacent track or -1 (attach=True)
    looper_group: torch.Tensor | None = None  # [T] int32 smallest track of the legs of one particle, -1 alone
    looper_leg: torch.Tensor | None = None    # [T] int32 leg number (0 = earliest in drift), -1 alone
    n_tracklets: int = 0
    n_segments: int = 0
    n_launches: int = 0
    n_rejected: int = 0                        # clusters the rejection before the refit took out
    stage_ms: dict | None = None
    work: dict | None = None


class Tracker:
    """Pre-allocates everything tpc_track needs for up to ``n_max`` clusters."""

    def __init__(self, n_max: int, row_x, n_sectors: int = 36, z_max: float = 250.0, continuous: bool = False,
                 params: abi.TpcParams | None = None, device="cuda", capacity_tracks: int | None = None,
                 debug: bool = False, n_frames: int = 1, attach: bool = False, loopers: bool = False):
        if not torch.cuda.is_available():
            raise RuntimeError("the TPC tracker needs a CUDA device")
        self.lib = abi.lib()
        self.params = params if params is not None else abi.tpc_params_default()
        self.geometry = abi.make_geometry(row_x, n_sectors, z_max, continuous)
        self.n_max = int(n_max)
        self.device = torch.device(device)
        self.n_frames = int(n_frames)
        self.ws_bytes = abi.tpc_workspace_size(self.params, self.geometry, self.n_max, self.n_frames)
        self.workspace = torch.empty(self.ws_bytes, dtype=torch.uint8, device=self.device)
        cap_t = capacity_tracks if capacity_tracks is not None else max(1024, self.n_max // 16)
        cap_c = max(1, self.n_max)
        d = self.device
        n1 = max(1, self.n_max)
        self.buf = dict(
            sector=torch.empty(cap_t, dtype=torch.int32, device=d),
            x=torch.empty(cap_t, dtype=torch.float32, device=d),
            param=torch.empty(cap_t, 5, dtype=torch.float32, device=d),
            cov=torch.empty(cap_t, 15, dtype=torch.float32, device=d),
            chi2=torch.empty(cap_t, dtype=torch.float32, device=d),
            ndf=torch.empty(cap_t, dtype=torch.int32, device=d),
            status=torch.empty(cap_t, dtype=torch.int32, device=d),
            nclus=torch.empty(cap_t, dtype=torch.int32, device=d),
            clus_offset=torch.empty(cap_t + 1, dtype=torch.int32, device=d),
            clus_index=torch.empty(cap_c, dtype=torch.int32, device=d),
            assign=torch.empty(n1, dtype=torch.int32, device=d),
            frame=torch.empty(cap_t, dtype=torch.int32, device=d),
        )
        if self.params.fp64_final:
            self.buf["cov64"] = torch.empty(cap_t, 15, dtype=torch.float64, device=d)
            self.buf["chi2_64"] = torch.empty(cap_t, dtype=torch.float64, device=d)
        if debug:
            self.buf["z"] = torch.empty(n1, dtype=torch.float32, device=d)
            for k in ("link_up_raw", "link_dn_raw", "link_up", "link_dn"):
                self.buf[k] = torch.empty(n1, dtype=torch.int32, device=d)
            self.buf["is_start"] = torch.empty(n1, dtype=torch.uint8, device=d)
        if attach:      # track-based cluster attachment (params.tube_radius, params.pt_min_physics)
            self.buf["cl_flags"] = torch.empty(n1, dtype=torch.uint8, device=d)
            self.buf["adjacent"] = torch.empty(n1, dtype=torch.int32, device=d)
        if loopers:     # looper-leg groups and leg numbers per track (params.looper_qpt_min)
            self.buf["looper_group"] = torch.empty(cap_t, dtype=torch.int32, device=d)
            self.buf["looper_leg"] = torch.empty(cap_t, dtype=torch.int32, device=d)
        self.capacity_tracks = cap_t
        self.capacity_clusters = cap_c
        self.debug = debug
        self.attach = attach
        self.loopers = loopers

    def _tracks_struct(self) -> abi.TpcTracks:
        b = self.buf
        t = abi.TpcTracks()
        t.capacity_tracks = self.capacity_tracks
        t.capacity_clusters = self.capacity_clusters
        for k in ("sector", "x", "param", "cov", "chi2", "ndf", "status", "nclus", "clus_offset", "clus_index",
                  "assign", "frame", "cov64", "chi2_64", "z", "link_up_raw", "link_dn_raw", "link_up", "link_dn",
                  "is_start", "cl_flags", "adjacent", "looper_group", "looper_leg"):
            setattr(t, k, b[k].data_ptr() if k in b else None)
        return t

    def _check_inputs(self, sector, row, y, zt):
        n = int(y.shape[0])
        if n > self.n_max:
            raise ValueError(f"{n} clusters > tracker capacity {self.n_max}")
        for a, dt in ((sector, torch.uint8), (row, torch.uint8), (y, torch.float32), (zt, torch.float32)):
            if a.dtype != dt or not a.is_cuda or not a.is_contiguous() or a.shape[0] != n:
                raise ValueError("clusters must be contiguous CUDA tensors: sector/row uint8, y/zt float32")
        return n

    def _result(self, out, n, T) -> TrackResult:
        b = self.buf
        res = TrackResult(n_tracks=T, sector=b["sector"][:T], x=b["x"][:T], param=b["param"][:T],
                          cov=b["cov"][:T], chi2=b["chi2"][:T], ndf=b["ndf"][:T], status=b["status"][:T],
                          nclus=b["nclus"][:T], clus_offset=b["clus_offset"][:T + 1],
                          clus_index=b["clus_index"], assign=b["assign"][:n])
        res.frame = b["frame"][:T]
        if out is not None:
            res.n_tracklets, res.n_segments, res.n_launches = out.n_tracklets, out.n_segments, out.n_launches
            res.n_rejected = out.n_rejected
            res.stage_ms = {k: float(out.stage_ms[i]) for i, k in enumerate(abi.STAGES)}
            if self.attach:
                res.stage_ms["attach"] = float(out.stage_ms[abi.ATTACH_STAGE])
            res.work = dict(zip(("trk_prop", "trk_upd", "trk_cand", "refit_prop", "merge_chi2"),
                                (int(v) for v in out.work)))
        if "cov64" in b:
            res.cov64, res.chi2_64 = b["cov64"][:T], b["chi2_64"][:T]
        if self.attach:
            res.cl_flags, res.adjacent = b["cl_flags"][:n], b["adjacent"][:n]
        if self.loopers:
            res.looper_group, res.looper_leg = b["looper_group"][:T], b["looper_leg"][:T]
        if self.debug:
            res.z = b["z"][:n]
            res.link_up_raw, res.link_dn_raw = b["link_up_raw"][:n], b["link_dn_raw"][:n]
            res.link_up, res.link_dn = b["link_up"][:n], b["link_dn"][:n]
            res.is_start = b["is_start"][:n]
        return res

    @staticmethod
    def _raise(rc, out, what):
        err = abi.TpcError(rc, what)
        err.needed = dict(tracklets=out.tracklets_needed, tracks=out.tracks_needed, clusters=out.clusters_needed)
        raise err

    def track(self, sector: torch.Tensor, row: torch.Tensor, y: torch.Tensor, zt: torch.Tensor, bz: float = 0.5,
              v_drift: float = 2.58, stream: torch.cuda.Stream | None = None) -> TrackResult:
        """One event or time frame (tpc_track)."""
        n = self._check_inputs(sector, row, y, zt)
        cl = abi.TpcClusters(n, sector.data_ptr(), row.data_ptr(), y.data_ptr(), zt.data_ptr())
        out = self._tracks_struct()
        st = stream if stream is not None else torch.cuda.current_stream(self.device)
        rc = self.lib.tpc_track(C.byref(self.params), C.byref(self.geometry), float(bz), float(v_drift),
                                C.byref(cl), C.c_void_p(self.workspace.data_ptr()), self.ws_bytes, C.byref(out),
                                C.c_void_p(st.cuda_stream))
        if rc:
            self._raise(rc, out, "tpc_track")
        return self._result(out, n, out.n_tracks)

    def track_batched(self, sector, row, y, zt, frame_offsets, bz: float = 0.5, v_drift: float = 2.58,
                      stream: torch.cuda.Stream | None = None) -> TrackResult:
        """Several independent time frames in one pass (tpc_track_batched);
        frame_offsets: n_frames + 1 cluster offsets (host)."""
        n = self._check_inputs(sector, row, y, zt)
        off = np.ascontiguousarray(frame_offsets, np.int32)
        nf = off.shape[0] - 1
        if nf > self.n_frames:
            raise ValueError(f"{nf} frames > tracker capacity {self.n_frames}")
        cl = abi.TpcClusters(n, sector.data_ptr(), row.data_ptr(), y.data_ptr(), zt.data_ptr())
        out = self._tracks_struct()
        st = stream if stream is not None else torch.cuda.current_stream(self.device)
        ws_bytes = abi.tpc_workspace_size(self.params, self.geometry, n, nf)
        rc = self.lib.tpc_track_batched(C.byref(self.params), C.byref(self.geometry), float(bz), float(v_drift),
                                        C.byref(cl), nf, off.ctypes.data_as(C.POINTER(C.c_int32)),
                                        C.c_void_p(self.workspace.data_ptr()), ws_bytes, C.byref(out),
                                        C.c_void_p(st.cuda_stream))
        if rc:
            self._raise(rc, out, "tpc_track_batched")
        return self._result(out, n, out.n_tracks)

    def capture(self, sector, row, y, zt, frame_offsets=None, bz: float = 0.5, v_drift: float = 2.58):
        """Record the whole chain for these (fixed) input buffers as a CUDA
        graph (tpc_prepare + tpc_track_async).  Returns a GraphRun whose
        replay() re-runs it; results appear in this tracker's buffers."""
        n = self._check_inputs(sector, row, y, zt)
        off = np.ascontiguousarray(frame_offsets if frame_offsets is not None else [0, n], np.int32)
        nf = off.shape[0] - 1
        ws_bytes = abi.tpc_workspace_size(self.params, self.geometry, n, nf)
        st = torch.cuda.Stream(self.device)
        rc = self.lib.tpc_prepare(C.byref(self.params), C.byref(self.geometry), n, nf,
                                  off.ctypes.data_as(C.POINTER(C.c_int32)), C.c_void_p(self.workspace.data_ptr()),
                                  ws_bytes, C.c_void_p(st.cuda_stream))
        if rc:
            raise abi.TpcError(rc, "tpc_prepare")
        counts = torch.zeros(8, dtype=torch.int32, device=self.device)
        cl = abi.TpcClusters(n, sector.data_ptr(), row.data_ptr(), y.data_ptr(), zt.data_ptr())
        out = self._tracks_struct()
        args = (C.byref(self.params), C.byref(self.geometry), float(bz), float(v_drift), C.byref(cl), nf,
                C.c_void_p(self.workspace.data_ptr()), ws_bytes, C.byref(out), C.c_void_p(counts.data_ptr()))
        # one eager run on the capture stream, then the capture
        with torch.cuda.stream(st):
            rc = self.lib.tpc_track_async(*args, C.c_void_p(st.cuda_stream))
            if rc:
                raise abi.TpcError(rc, "tpc_track_async")
        st.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=st):
            rc = self.lib.tpc_track_async(*args, C.c_void_p(torch.cuda.current_stream(self.device).cuda_stream))
        if rc:
            raise abi.TpcError(rc, "tpc_track_async (capture)")
        return GraphRun(self, graph, counts, n, (cl, out))

    def export_tracklets(self, stream: torch.cuda.Stream | None = None):
        """Tracklets of the last call (host numpy arrays, ascending start index)."""
        nr = self.geometry.n_rows
        nt = C.c_int32()
        st = stream if stream is not None else torch.cuda.current_stream(self.device)
        rc = self.lib.tpc_export_tracklets(C.c_void_p(self.workspace.data_ptr()), 0, nr, None, None, None, None,
                                           None, None, C.byref(nt), C.c_void_p(st.cuda_stream))
        if rc not in (abi.TPC_OK, abi.TPC_ERR_CAPACITY):
            raise abi.TpcError(rc, "tpc_export_tracklets")
        cap = max(1, int(nt.value))
        start = np.zeros(cap, np.int32)
        nhits = np.zeros(cap, np.int32)
        kept = np.zeros(cap, np.uint8)
        hits = np.zeros((cap, nr), np.int32)
        top = np.zeros((cap, 21), np.float32)
        bot = np.zeros((cap, 21), np.float32)
        rc = self.lib.tpc_export_tracklets(C.c_void_p(self.workspace.data_ptr()), cap, nr, start.ctypes.data,
                                           nhits.ctypes.data, kept.ctypes.data, hits.ctypes.data, top.ctypes.data,
                                           bot.ctypes.data, C.byref(nt), C.c_void_p(st.cuda_stream))
        if rc:
            raise abi.TpcError(rc, "tpc_export_tracklets")
        k = int(nt.value)
        return dict(start=start[:k], nhits=nhits[:k], kept=kept[:k], hits=hits[:k], top=top[:k], bot=bot[:k])


class GraphRun:
    """A captured tracking chain; replay() enqueues it on the current stream."""

    def __init__(self, tracker: Tracker, graph, counts: torch.Tensor, n: int, keep):
        self.tracker, self.graph, self.counts, self.n, self._keep = tracker, graph, counts, n, keep

    def replay(self):
        self.graph.replay()

    def result(self) -> TrackResult:
        """Synchronise and wrap the buffers (n_tracks read from the device counts)."""
        c = self.counts.cpu().tolist()
        if c[3]:
            raise abi.TpcError(c[3], "captured tpc_track_async")
        res = self.tracker._result(None, self.n, int(c[0]))
        res.n_tracklets, res.n_segments = int(c[1]), int(c[2])
        return res


def tpc_track(sector, row, y, zt, row_x, n_sectors=36, z_max=250.0, continuous=False, bz=0.5, v_drift=2.58,
              params: abi.TpcParams | None = None, debug=False) -> TrackResult:
    """One-shot call: allocate a Tracker for this input and run tpc_track."""
    trk = Tracker(int(y.shape[0]), row_x, n_sectors=n_sectors, z_max=z_max, continuous=continuous, params=params,
                  device=y.device, debug=debug)
    return trk.track(sector, row, y, zt, bz=bz, v_drift=v_drift)
