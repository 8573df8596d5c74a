"""Entropy coder of the cluster compression (tpc_rans_encode): rANS of byte
symbols, one static 12-bit table per stream, independent chunks; the byte
format is stated in include/tpc_compress.h."""
from __future__ import annotations

import ctypes as C
import dataclasses

import torch

from . import abi


@dataclasses.dataclass
class RansStream:
    freq: torch.Tensor          # [256] uint32 (int32 storage): the table
    chunk_bytes: torch.Tensor   # [n_chunks] int32: coded bytes per chunk
    data: torch.Tensor          # [total] uint8: the chunks back to back
    chunk: int


def rans_encode(sym: torch.Tensor, chunk: int = 4096) -> RansStream:
    """Code a CUDA uint8 tensor of symbols; synchronises the current stream
    to read the coded size."""
    if sym.dtype != torch.uint8 or not sym.is_cuda or not sym.is_contiguous() or sym.dim() != 1:
        raise ValueError("symbols: a contiguous 1-D CUDA uint8 tensor")
    L = abi.lib()
    n = int(sym.numel())
    ws = C.c_size_t(0)
    rc = L.tpc_rans_workspace_size(n, chunk, C.byref(ws))
    if rc:
        raise abi.TpcError(rc, "tpc_rans_workspace_size")
    mb = C.c_int64(0)
    L.tpc_rans_max_bytes(n, chunk, C.byref(mb))
    d = sym.device
    work = torch.empty(int(ws.value), dtype=torch.uint8, device=d)
    freq = torch.empty(256, dtype=torch.int32, device=d)
    nch = (n + chunk - 1) // chunk
    cb = torch.empty(max(nch, 1), dtype=torch.int32, device=d)
    out = torch.empty(max(int(mb.value), 1), dtype=torch.uint8, device=d)
    total = C.c_int64(0)
    rc = L.tpc_rans_encode(C.c_void_p(sym.data_ptr() if n else 0), n, chunk, C.c_void_p(work.data_ptr()), ws.value,
                           C.c_void_p(freq.data_ptr()), C.c_void_p(cb.data_ptr()), C.c_void_p(out.data_ptr()),
                           out.numel(), C.byref(total), C.c_void_p(torch.cuda.current_stream(d).cuda_stream))
    if rc:
        raise abi.TpcError(rc, "tpc_rans_encode")
    return RansStream(freq=freq, chunk_bytes=cb[:nch], data=out[:int(total.value)], chunk=chunk)


def _compress_in(sector, row, y, zt, clus_offset, clus_index, assign, n_sectors, n_rows):
    for name, t, dt in (("sector", sector, torch.uint8), ("row", row, torch.uint8), ("y", y, torch.float32),
                        ("zt", zt, torch.float32), ("clus_offset", clus_offset, torch.int32),
                        ("clus_index", clus_index, torch.int32), ("assign", assign, torch.int32)):
        if t.dtype != dt or not t.is_cuda or not t.is_contiguous():
            raise ValueError(f"{name}: a contiguous CUDA {dt} tensor")
    T = int(clus_offset.numel()) - 1
    if T < 0:
        raise ValueError("clus_offset needs n_tracks + 1 entries")
    na = int(clus_offset[-1].item()) if T > 0 else 0
    ptr = lambda t: C.c_void_p(t.data_ptr() if t.numel() else 0)  # noqa: E731
    return abi.TpcCompressIn(int(y.numel()), n_sectors, n_rows, ptr(sector), ptr(row), ptr(y), ptr(zt), T, na,
                             ptr(clus_offset), ptr(clus_index), ptr(assign))


def compress_fields(sector, row, y, zt, clus_offset, clus_index, assign, n_sectors=36, n_rows=152, ey=5, et=6):
    """The integer streams of the compressed cluster format (tpc_compress_fields),
    as a dict of CUDA arrays (uint32 values in int32 storage) by stream name."""
    L = abi.lib()
    cin = _compress_in(sector, row, y, zt, clus_offset, clus_index, assign, n_sectors, n_rows)
    ws = C.c_size_t(0)
    if L.tpc_compress_workspace_size(C.byref(cin), 4096, C.byref(ws)):
        raise abi.TpcError(abi.TPC_ERR_ARG, "tpc_compress_workspace_size")
    mv = C.c_int64(0)
    L.tpc_compress_max_size(C.byref(cin), 4096, C.byref(mv), None)
    d = y.device
    work = torch.empty(int(ws.value), dtype=torch.uint8, device=d)
    vals = torch.empty(max(int(mv.value), 1), dtype=torch.int32, device=d)
    counts = (C.c_int64 * 12)()
    rc = L.tpc_compress_fields(C.byref(cin), ey, et, C.c_void_p(work.data_ptr()), ws.value,
                               C.c_void_p(vals.data_ptr()), vals.numel(), counts,
                               C.c_void_p(torch.cuda.current_stream(d).cuda_stream))
    if rc:
        raise abi.TpcError(rc, "tpc_compress_fields")
    out, o = {}, 0
    for k, name in enumerate(abi.CMP_STREAMS):
        out[name] = vals[o:o + counts[k]]
        o += counts[k]
    return out


def compress_buffers(sector, row, y, zt, clus_offset, clus_index, assign, n_sectors=36, n_rows=152, chunk=4096):
    """Workspace and output buffers (uint8 CUDA tensors) large enough for
    compress_frame of these inputs."""
    L = abi.lib()
    cin = _compress_in(sector, row, y, zt, clus_offset, clus_index, assign, n_sectors, n_rows)
    ws = C.c_size_t(0)
    if L.tpc_compress_workspace_size(C.byref(cin), chunk, C.byref(ws)):
        raise abi.TpcError(abi.TPC_ERR_ARG, "tpc_compress_workspace_size")
    mb = C.c_int64(0)
    L.tpc_compress_max_size(C.byref(cin), chunk, None, C.byref(mb))
    d = y.device
    return (torch.empty(int(ws.value), dtype=torch.uint8, device=d),
            torch.empty(max(int(mb.value), 1), dtype=torch.uint8, device=d))


def compress_frame(sector, row, y, zt, clus_offset, clus_index, assign, n_sectors=36, n_rows=152, ey=5, et=6,
                   chunk=4096, workspace=None, out=None):
    """The compressed frame (tpc_compress_frame): a CUDA uint8 tensor of the 12
    stream containers back to back, and the byte size of each.  workspace /
    out may be passed in (uint8 CUDA tensors, large enough) to reuse them."""
    L = abi.lib()
    cin = _compress_in(sector, row, y, zt, clus_offset, clus_index, assign, n_sectors, n_rows)
    ws = C.c_size_t(0)
    if L.tpc_compress_workspace_size(C.byref(cin), chunk, C.byref(ws)):
        raise abi.TpcError(abi.TPC_ERR_ARG, "tpc_compress_workspace_size")
    mb = C.c_int64(0)
    L.tpc_compress_max_size(C.byref(cin), chunk, None, C.byref(mb))
    d = y.device
    if workspace is None or workspace.numel() < int(ws.value):
        workspace = torch.empty(int(ws.value), dtype=torch.uint8, device=d)
    if out is None or out.numel() < int(mb.value):
        out = torch.empty(max(int(mb.value), 1), dtype=torch.uint8, device=d)
    sizes = (C.c_int64 * 12)()
    rc = L.tpc_compress_frame(C.byref(cin), ey, et, chunk, C.c_void_p(workspace.data_ptr()), workspace.numel(),
                              C.c_void_p(out.data_ptr()), out.numel(), sizes,
                              C.c_void_p(torch.cuda.current_stream(d).cuda_stream))
    if rc:
        raise abi.TpcError(rc, "tpc_compress_frame")
    sz = [int(v) for v in sizes]
    return out[:sum(sz)], sz
