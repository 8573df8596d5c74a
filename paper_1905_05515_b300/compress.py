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
