"""Tracking a stream of frames held in host memory.

Every frame's clusters are copied to the GPU, tracked, and its tracks copied
back into page-locked host buffers.  FramePipeline keeps ``depth`` slots,
each with its own CUDA stream, device input buffers, workspace and output
buffers: while one slot's frame is being tracked, the next frame's clusters
are copied in on another slot's stream and the previous frame's tracks are
copied out, so the copies run beside the tracking instead of between frames.
The tracking runs one frame at a time up to the refit: each slot's chain waits
for the event the library records when the previous frame's refit starts
(tpc_tracks.refit_event), so a frame's first stages run beside the previous
frame's refit, whose last long tracks keep few SMs busy, while frames do not
otherwise compete for the SMs and the L2.

A push enqueues, on its slot's stream and without host synchronisation, the
host-to-device copies, tpc_prepare_async and tpc_track_async, and a copy of
the device counts (tracks, clusters in tracks).  Collecting a frame waits for
its counts, then enqueues device-to-host copies of exactly the filled parts
of the outputs and waits for them; the other slots' work goes on meanwhile.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
from collections import deque

import numpy as np
import torch

from . import abi


@dataclasses.dataclass
class HostTracks:
    """One frame's tracks in page-locked host memory (views of its slot's
    buffers, valid until the slot is reused ``depth`` pushes later)."""
    n_tracks: int
    n_clusters: int
    param: torch.Tensor          # [T, 5]
    cov: torch.Tensor            # [T, 15]
    chi2: torch.Tensor           # [T]
    ndf: torch.Tensor            # [T]
    nclus: torch.Tensor          # [T]
    clus_offset: torch.Tensor    # [T + 1]
    clus_index: torch.Tensor     # [clus_offset[T]]
    assign: torch.Tensor         # [n]
    d2h_bytes: int
    h2d_bytes: int


class _Slot:
    def __init__(self, pipe: "FramePipeline"):
        d = pipe.device
        n1 = max(1, pipe.n_max)
        self.stream = torch.cuda.Stream(d)
        self.ins = dict(sector=torch.empty(n1, dtype=torch.uint8, device=d),
                        row=torch.empty(n1, dtype=torch.uint8, device=d),
                        y=torch.empty(n1, dtype=torch.float32, device=d),
                        zt=torch.empty(n1, dtype=torch.float32, device=d))
        self.ws_bytes = abi.tpc_workspace_size(pipe.params, pipe.geometry, pipe.n_max, 1)
        self.ws = torch.empty(self.ws_bytes, dtype=torch.uint8, device=d)
        cap_t = pipe.capacity_tracks
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
            clus_index=torch.empty(n1, dtype=torch.int32, device=d),
            assign=torch.empty(n1, dtype=torch.int32, device=d),
            frame=torch.empty(cap_t, dtype=torch.int32, device=d),
        )
        if pipe.params.fp64_final:
            self.buf["cov64"] = torch.empty(cap_t, 15, dtype=torch.float64, device=d)
            self.buf["chi2_64"] = torch.empty(cap_t, dtype=torch.float64, device=d)
        self.out = abi.TpcTracks()
        self.out.capacity_tracks = cap_t
        self.out.capacity_clusters = n1
        for k in ("sector", "x", "param", "cov", "chi2", "ndf", "status", "nclus", "clus_offset", "clus_index",
                  "assign", "frame", "cov64", "chi2_64"):
            setattr(self.out, k, self.buf[k].data_ptr() if k in self.buf else None)
        self.counts = torch.zeros(8, dtype=torch.int32, device=d)
        self.h_counts = torch.zeros(8, dtype=torch.int32).pin_memory()
        self.counts_ready = torch.cuda.Event()
        self.done = torch.cuda.Event()
        # recorded by the library when this slot's frame starts its refit; the
        # first record on the slot's stream creates the CUDA event
        self.refit_started = torch.cuda.Event()
        self.refit_started.record(self.stream)
        self.out.refit_event = self.refit_started.cuda_event
        sz = C.c_size_t(0)
        rc = pipe.lib.tpc_prepare_staging_size(1, C.byref(sz))
        if rc:
            raise abi.TpcError(rc, "tpc_prepare_staging_size")
        self.staging = torch.empty(int(sz.value), dtype=torch.uint8).pin_memory()
        self.host = dict(param=(cap_t, 5), cov=(cap_t, 15), chi2=(cap_t,), ndf=(cap_t,), nclus=(cap_t,),
                         clus_offset=(cap_t + 1,))
        self.host = {k: torch.empty(sh, dtype=self.buf[k].dtype).pin_memory() for k, sh in self.host.items()}
        self.host["clus_index"] = torch.empty(n1, dtype=torch.int32).pin_memory()
        self.host["assign"] = torch.empty(n1, dtype=torch.int32).pin_memory()
        self.n = 0
        self.h2d = 0
        self.busy = False
        self.srcs = None


class FramePipeline:
    """Frames from host memory through the tracker with copies overlapping
    the tracking of other frames (see the module docstring).

    push(sector, row, y, zt) takes one frame as CPU tensors (uint8, uint8,
    float32, float32; page-locked for asynchronous copies, else they are
    copied into page-locked memory first) and returns the tracks of the
    oldest pending frame once all slots are in use, else None; flush()
    returns the tracks of every pending frame, oldest first.
    """

    def __init__(self, n_max: int, row_x, depth: int = 2, params: abi.TpcParams | None = None,
                 n_sectors: int = 36, z_max: float = 250.0, continuous: bool = True, bz: float = 0.5,
                 v_drift: float = 2.58, device="cuda", capacity_tracks: int | None = None):
        if not torch.cuda.is_available():
            raise RuntimeError("the TPC tracker needs a CUDA device")
        self.lib = abi.lib()
        self.device = torch.device(device)
        self.params = params if params is not None else abi.tpc_params_default()
        self.geometry = abi.make_geometry(row_x, n_sectors, z_max, continuous)
        self.n_max = int(n_max)
        self.bz, self.v_drift = float(bz), float(v_drift)
        self.capacity_tracks = capacity_tracks if capacity_tracks is not None else max(1024, self.n_max // 16)
        self.slots = [_Slot(self) for _ in range(max(1, int(depth)))]
        self.next = 0
        self.pending: deque[_Slot] = deque()
        self.n_launches = 0
        self.last_tracked: torch.cuda.Event | None = None

    def push(self, sector, row, y, zt) -> HostTracks | None:
        n = int(y.shape[0])
        if n > self.n_max or n < 1:
            raise ValueError(f"{n} clusters: the pipeline takes 1..{self.n_max} per frame")
        srcs = {}
        for k, a, dt in (("sector", sector, torch.uint8), ("row", row, torch.uint8), ("y", y, torch.float32),
                         ("zt", zt, torch.float32)):
            a = torch.as_tensor(a)
            if a.dtype != dt or a.shape[0] != n or a.device.type != "cpu":
                raise ValueError("frame clusters: CPU tensors sector/row uint8, y/zt float32 of one length")
            a = a.contiguous()
            srcs[k] = a if a.is_pinned() else a.pin_memory()
        s = self.slots[self.next]
        res = None
        if s.busy:                       # all slots in use: this one holds the oldest frame
            assert self.pending[0] is s
            res = self._collect(self.pending.popleft())
        self.next = (self.next + 1) % len(self.slots)
        st = s.stream
        h = C.c_void_p(st.cuda_stream)
        off = np.array([0, n], np.int32)
        with torch.cuda.stream(st):
            for k, a in srcs.items():
                s.ins[k][:n].copy_(a, non_blocking=True)
            # one frame tracked at a time up to its refit (frames tracked side by
            # side share the SMs and the L2 and are slower together); the copies
            # overlap, and so do this frame's first stages and the previous
            # frame's refit
            if self.last_tracked is not None:
                st.wait_event(self.last_tracked)
            rc = self.lib.tpc_prepare_async(C.byref(self.params), C.byref(self.geometry), n, 1,
                                            off.ctypes.data_as(C.POINTER(C.c_int32)),
                                            C.c_void_p(s.staging.data_ptr()), s.staging.numel(),
                                            C.c_void_p(s.ws.data_ptr()), s.ws_bytes, h)
            if rc:
                raise abi.TpcError(rc, "tpc_prepare_async")
            cl = abi.TpcClusters(n, s.ins["sector"].data_ptr(), s.ins["row"].data_ptr(), s.ins["y"].data_ptr(),
                                 s.ins["zt"].data_ptr())
            rc = self.lib.tpc_track_async(C.byref(self.params), C.byref(self.geometry), self.bz, self.v_drift,
                                          C.byref(cl), 1, C.c_void_p(s.ws.data_ptr()), s.ws_bytes, C.byref(s.out),
                                          C.c_void_p(s.counts.data_ptr()), h)
            if rc:
                raise abi.TpcError(rc, "tpc_track_async")
            self.last_tracked = s.refit_started
            s.h_counts.copy_(s.counts, non_blocking=True)
            s.counts_ready.record(st)
        self.n_launches += int(s.out.n_launches)
        s.n, s.h2d, s.busy = n, sum(int(a.numel() * a.element_size()) for a in srcs.values()), True
        s.srcs = srcs                    # the asynchronous copies read these until the frame is collected
        self.pending.append(s)
        return res

    def flush(self) -> list[HostTracks]:
        out = []
        while self.pending:
            out.append(self._collect(self.pending.popleft()))
        return out

    def _collect(self, s: _Slot) -> HostTracks:
        s.counts_ready.synchronize()
        c = s.h_counts.tolist()
        if c[3]:
            raise abi.TpcError(c[3], "tpc_track_async")
        T, nc, n = int(c[0]), int(c[4]), s.n
        d2h = 0
        with torch.cuda.stream(s.stream):
            for k in ("param", "cov", "chi2", "ndf", "nclus", "clus_offset"):
                m = T + 1 if k == "clus_offset" else T
                s.host[k][:m].copy_(s.buf[k][:m], non_blocking=True)
                d2h += m * s.buf[k][0].numel() * s.buf[k].element_size()
            s.host["clus_index"][:nc].copy_(s.buf["clus_index"][:nc], non_blocking=True)
            s.host["assign"][:n].copy_(s.buf["assign"][:n], non_blocking=True)
            s.done.record(s.stream)
        d2h += 4 * nc + 4 * n
        s.done.synchronize()
        s.busy, s.srcs = False, None
        hs = s.host
        return HostTracks(n_tracks=T, n_clusters=n, param=hs["param"][:T], cov=hs["cov"][:T], chi2=hs["chi2"][:T],
                          ndf=hs["ndf"][:T], nclus=hs["nclus"][:T], clus_offset=hs["clus_offset"][:T + 1],
                          clus_index=hs["clus_index"][:nc], assign=hs["assign"][:n], d2h_bytes=d2h,
                          h2d_bytes=s.h2d)
