"""B300-native TPC cellular-automaton + Kalman tracker (thin Python binding).

Every step of the tracking chain runs in the CUDA kernels of libtpcgpu.so,
called through its C ABI (include/tpc_track.h, include/tpc_calib.h).  PyTorch only provides device
memory and the current CUDA stream.  There is no CPU fallback: without the
compiled library or a CUDA device the calls raise.
"""
from .abi import (TPC_ERR_ARG, TPC_ERR_CAPACITY, TPC_ERR_CUDA, TPC_ERR_DATA, TPC_ERR_TIMEOUT, TPC_OK,
                  TpcError, lib, tpc_error_string, tpc_params_default, tpc_workspace_size)
from . import autotune, batch, calib, compress
from .batch import GroupedBatch
from .calib import CalibRefit, calib_chi2
from .compress import RansStream, compress_fields, compress_frame, rans_encode
from .pipeline import FramePipeline, HostTracks
from .tracker import GraphRun, Tracker, TrackResult, tpc_track

__all__ = ["compress", "rans_encode", "compress_fields", "compress_frame", "RansStream", "Tracker", "TrackResult", "GraphRun", "GroupedBatch", "FramePipeline", "HostTracks", "autotune", "batch", "calib", "CalibRefit", "calib_chi2", "tpc_track", "tpc_params_default", "tpc_workspace_size", "tpc_error_string",
           "lib", "TpcError", "TPC_OK", "TPC_ERR_ARG", "TPC_ERR_CAPACITY", "TPC_ERR_TIMEOUT", "TPC_ERR_CUDA",
           "TPC_ERR_DATA"]
