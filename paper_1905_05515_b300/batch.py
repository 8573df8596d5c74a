"""Grouped, graph-captured tracking of many sub-time-frames.

The frames of a batch are cut into groups of consecutive frames holding at
most ``group_clusters`` clusters (a larger frame is a group of its own).
Each group is one tpc_prepare_async + tpc_track_async chain (every stage one
launch over the group's frames), enqueued on one of ``n_streams`` streams;
groups on one stream reuse that stream's workspace in turn, chains on
different streams run concurrently (one group's latency-bound tracklet tail
overlaps the next group's bandwidth-bound binning).  The whole batch is
captured once as a CUDA graph and replayed.  A group's working set stays
near the L2 size instead of the whole batch's, which is what makes grouping
faster than one launch per stage over all frames.  Every group has its own
output buffers; results are identical to tracking each frame alone.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import abi
from .tracker import TrackResult


def partition(frame_offsets, group_clusters: int):
    """Consecutive frame ranges [(f0, f1), ...] of at most group_clusters
    clusters each (a single larger frame forms its own group);
    group_clusters <= 0 gives one frame per group."""
    off = np.asarray(frame_offsets, np.int64)
    nf = off.size - 1
    groups, f0 = [], 0
    while f0 < nf:
        f1 = f0 + 1
        if group_clusters > 0:
            while f1 < nf and off[f1 + 1] - off[f0] <= group_clusters:
                f1 += 1
        groups.append((f0, f1))
        f0 = f1
    return groups


class _Group:
    """Output buffers, staging and call structures of one frame group."""

    def __init__(self, gb: "GroupedBatch", f0: int, f1: int, ins):
        self.f0, self.f1 = f0, f1
        off = gb.offsets
        self.a, self.b = int(off[f0]), int(off[f1])
        self.n = self.b - self.a
        self.nf = f1 - f0
        self.local_off = np.ascontiguousarray(off[f0:f1 + 1] - off[f0], np.int32)
        d = gb.device
        cap_t = max(1024, self.n // 16)
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
            clus_index=torch.empty(max(1, self.n), dtype=torch.int32, device=d),
            assign=torch.empty(max(1, self.n), dtype=torch.int32, device=d),
            frame=torch.empty(cap_t, dtype=torch.int32, device=d),
        )
        if gb.params.fp64_final:
            self.buf["cov64"] = torch.empty(cap_t, 15, dtype=torch.float64, device=d)
            self.buf["chi2_64"] = torch.empty(cap_t, dtype=torch.float64, device=d)
        self.counts = torch.zeros(8, dtype=torch.int32, device=d)
        out = abi.TpcTracks()
        out.capacity_tracks = cap_t
        out.capacity_clusters = max(1, self.n)
        for k in ("sector", "x", "param", "cov", "chi2", "ndf", "status", "nclus", "clus_offset", "clus_index",
                  "assign", "frame", "cov64", "chi2_64"):
            setattr(out, k, self.buf[k].data_ptr() if k in self.buf else None)
        self.out = out
        sector, row, y, zt = ins
        self.cl = abi.TpcClusters(self.n, sector.data_ptr() + self.a, row.data_ptr() + self.a,
                                  y.data_ptr() + 4 * self.a, zt.data_ptr() + 4 * self.a)
        sz = C.c_size_t(0)
        rc = gb.lib.tpc_prepare_staging_size(self.nf, C.byref(sz))
        if rc:
            raise abi.TpcError(rc, "tpc_prepare_staging_size")
        self.staging = torch.empty(int(sz.value), dtype=torch.uint8).pin_memory()
        self.ws_bytes = abi.tpc_workspace_size(gb.params, gb.geometry, self.n, self.nf)
        self.cap_t = cap_t
        self.host = None                 # page-locked results of a host-I/O capture

    def host_buffers(self):
        if self.host is None:
            self.host = dict(param=torch.empty(self.cap_t, 5, dtype=torch.float32).pin_memory(),
                             chi2=torch.empty(self.cap_t, dtype=torch.float32).pin_memory(),
                             assign=torch.empty(max(1, self.n), dtype=torch.int32).pin_memory(),
                             counts=torch.zeros(8, dtype=torch.int32).pin_memory())
        return self.host


class GroupedBatch:
    """Sub-time-frames of one batch, tracked in frame groups on several
    streams and captured as one CUDA graph (see the module docstring).

    sector, row, y, zt: the concatenated clusters of all frames (contiguous
    CUDA tensors, uint8 / uint8 / float32 / float32); frame_offsets: n_frames + 1
    host offsets.  The input tensors must stay alive and in place: the graph
    reads them at replay.
    """

    def __init__(self, sector, row, y, zt, frame_offsets, row_x, params: abi.TpcParams | None = None,
                 group_clusters: int = 32_000_000, n_streams: int = 2, n_sectors: int = 36, z_max: float = 250.0,
                 continuous: bool = True, bz: float = 0.5, v_drift: float = 2.58):
        if not torch.cuda.is_available() or not y.is_cuda:
            raise RuntimeError("the TPC tracker needs CUDA tensors")
        for a, dt in ((sector, torch.uint8), (row, torch.uint8), (y, torch.float32), (zt, torch.float32)):
            if a.dtype != dt or not a.is_contiguous() or a.shape[0] != y.shape[0]:
                raise ValueError("clusters must be contiguous CUDA tensors: sector/row uint8, y/zt float32")
        self.lib = abi.lib()
        self.device = y.device
        self.params = params if params is not None else abi.tpc_params_default()
        self.geometry = abi.make_geometry(row_x, n_sectors, z_max, continuous)
        self.offsets = np.asarray(frame_offsets, np.int64)
        if self.offsets[0] != 0 or self.offsets[-1] != y.shape[0] or np.any(np.diff(self.offsets) < 0):
            raise ValueError("frame_offsets must run from 0 to the cluster count, non-decreasing")
        self.bz, self.v_drift = float(bz), float(v_drift)
        self.n_streams = max(1, int(n_streams))
        self.group_clusters = int(group_clusters)
        self._ins = (sector, row, y, zt)
        self.groups = [_Group(self, f0, f1, self._ins) for f0, f1 in partition(self.offsets, group_clusters)]
        self.streams = [torch.cuda.Stream(self.device) for _ in range(self.n_streams)]
        # one workspace per stream, sized for the largest group it runs
        self.ws = []
        for s in range(self.n_streams):
            need = max((g.ws_bytes for g in self.groups[s::self.n_streams]), default=1)
            self.ws.append((torch.empty(need, dtype=torch.uint8, device=self.device), need))
        self.graph = None

    def _enqueue(self, host_in=None):
        """All groups, each on its stream; the caller's stream waits for all.
        With host_in (page-locked CPU tensors of the whole batch), every group
        first copies its clusters from there and afterwards copies its
        parameters, chi2 (whole capacity), counts and assignments to its
        page-locked host buffers, on its own stream."""
        main = torch.cuda.current_stream(self.device)
        for st in self.streams:
            st.wait_stream(main)
        for i, g in enumerate(self.groups):
            s = i % self.n_streams
            ws, wsb = self.ws[s]
            h = C.c_void_p(self.streams[s].cuda_stream)
            if host_in is not None:
                with torch.cuda.stream(self.streams[s]):
                    for dst, src in zip(self._ins, host_in):
                        dst[g.a:g.b].copy_(src[g.a:g.b], non_blocking=True)
            rc = self.lib.tpc_prepare_async(C.byref(self.params), C.byref(self.geometry), g.n, g.nf,
                                            g.local_off.ctypes.data_as(C.POINTER(C.c_int32)),
                                            C.c_void_p(g.staging.data_ptr()), g.staging.numel(),
                                            C.c_void_p(ws.data_ptr()), wsb, h)
            if rc:
                raise abi.TpcError(rc, "tpc_prepare_async")
            rc = self.lib.tpc_track_async(C.byref(self.params), C.byref(self.geometry), self.bz, self.v_drift,
                                          C.byref(g.cl), g.nf, C.c_void_p(ws.data_ptr()), wsb, C.byref(g.out),
                                          C.c_void_p(g.counts.data_ptr()), h)
            if rc:
                raise abi.TpcError(rc, "tpc_track_async")
            if host_in is not None:
                hb = g.host_buffers()
                with torch.cuda.stream(self.streams[s]):
                    hb["param"].copy_(g.buf["param"], non_blocking=True)
                    hb["chi2"].copy_(g.buf["chi2"], non_blocking=True)
                    hb["counts"].copy_(g.counts, non_blocking=True)
                    hb["assign"][:g.n].copy_(g.buf["assign"][:g.n], non_blocking=True)
        for st in self.streams:
            main.wait_stream(st)

    def run(self):
        """Enqueue the batch eagerly (no graph)."""
        self._enqueue()

    def capture(self, host_in=None):
        """Capture the batch as a CUDA graph (after one eager run, which
        loads the kernels).  host_in: page-locked CPU tensors (sector, row,
        y, zt) of the whole batch to copy from at every replay, with the
        results copied back (host_results); they must stay alive."""
        for a, b in zip(host_in or (), self._ins):
            if a.device.type != "cpu" or not a.is_pinned() or a.dtype != b.dtype or a.shape != b.shape:
                raise ValueError("host_in: page-locked CPU tensors shaped like the device inputs")
        self._host_in = host_in
        self._enqueue(host_in)
        torch.cuda.synchronize(self.device)
        cap = torch.cuda.Stream(self.device)
        cap.wait_stream(torch.cuda.current_stream(self.device))
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph, stream=cap):
            self._enqueue(host_in)
        return self

    def host_results(self):
        """Per group (after a replay of a host-I/O capture; synchronises):
        (n_tracks, parameters [T, 5], chi2 [T], assignments [n]) as views of
        the group's page-locked buffers."""
        torch.cuda.synchronize(self.device)
        out = []
        for g in self.groups:
            hb = g.host
            c = hb["counts"].tolist()
            if c[3]:
                raise abi.TpcError(c[3], f"frames {g.f0}..{g.f1 - 1}")
            T = int(c[0])
            out.append((T, hb["param"][:T], hb["chi2"][:T], hb["assign"][:g.n]))
        return out

    def host_io_bytes(self):
        """(host-to-device, device-to-host) bytes one host-I/O replay copies."""
        h2d = sum(g.n * 10 for g in self.groups)
        d2h = sum(g.cap_t * 24 + 32 + 4 * g.n for g in self.groups)
        return h2d, d2h

    def replay(self):
        if self.graph is None:
            self.capture()
        self.graph.replay()

    @property
    def n_launches(self) -> int:
        """Kernels of this library per run or replay (copies not counted)."""
        return sum(int(g.out.n_launches) for g in self.groups)

    def results(self) -> list[TrackResult]:
        """Per-group results (synchronises; views of the group buffers)."""
        torch.cuda.synchronize(self.device)
        out = []
        for g in self.groups:
            c = g.counts.cpu().tolist()
            if c[3]:
                raise abi.TpcError(c[3], f"frames {g.f0}..{g.f1 - 1}")
            T = int(c[0])
            b = g.buf
            r = TrackResult(n_tracks=T, sector=b["sector"][:T], x=b["x"][:T], param=b["param"][:T],
                            cov=b["cov"][:T], chi2=b["chi2"][:T], ndf=b["ndf"][:T], status=b["status"][:T],
                            nclus=b["nclus"][:T], clus_offset=b["clus_offset"][:T + 1],
                            clus_index=b["clus_index"], assign=b["assign"][:g.n])
            r.frame = b["frame"][:T] + g.f0
            r.n_tracklets, r.n_segments = int(c[1]), int(c[2])
            if "cov64" in b:
                r.cov64, r.chi2_64 = b["cov64"][:T], b["chi2_64"][:T]
            out.append(r)
        return out

    def param(self) -> torch.Tensor:
        """Track parameters of the whole batch in frame order."""
        return torch.cat([r.param for r in self.results()])
