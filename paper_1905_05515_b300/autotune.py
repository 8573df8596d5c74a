"""Autotuner: picks the settings that change speed but never results.

* y_bins, z_cell -- granularity of the per-row grid (tile shape of the
  cluster binning and of every window search);
* queue_blocks_per_sm -- width of the TrackletConstructor work queue;
* group_clusters, n_streams -- granularity of a graph-captured batch of
  sub-time-frames (frames per launch group) and how many groups run
  concurrently (GroupedBatch).

Every candidate runs the given (batched) input with CUDA events; the fastest
median wins.  Results are identical for every candidate (the searches are
order- and grid-independent), so tuning never trades accuracy.
"""
from __future__ import annotations

import itertools
import json
import statistics

import numpy as np
import torch

from . import abi
from .batch import GroupedBatch
from .tracker import Tracker

DEFAULT_SPACE = {"y_bins": (8, 16, 24), "z_cell": (2.0, 3.5, 5.0), "queue_blocks_per_sm": (0, 8)}
GROUP_SPACE = {"group_clusters": (0, 8_000_000, 16_000_000, 32_000_000, 64_000_000), "n_streams": (1, 2, 3)}


def autotune(sector, row, y, zt, frame_offsets, row_x, n_sectors=36, z_max=250.0, continuous=True, bz=0.5,
             v_drift=2.58, space: dict | None = None, reps: int = 3, base: abi.TpcParams | None = None,
             log=None) -> dict:
    """Time every combination of `space` on this input; returns
    {"best": {...}, "ms": best_ms, "table": [(config, ms), ...]}."""
    space = space or DEFAULT_SPACE
    off = np.ascontiguousarray(frame_offsets, np.int32)
    nf = off.shape[0] - 1
    n = int(y.shape[0])
    keys = list(space)
    table = []
    trackers = {}
    for combo in itertools.product(*(space[k] for k in keys)):
        cfg = dict(zip(keys, combo))
        p = abi.tpc_params_default()
        if base is not None:
            for name, _ in abi.TpcParams._fields_:
                setattr(p, name, getattr(base, name))
        for k, v in cfg.items():
            setattr(p, k, v)
        key = (cfg.get("y_bins"),)
        if key not in trackers:
            trackers.clear()
            torch.cuda.empty_cache()
            trackers[key] = Tracker(n, row_x, n_sectors=n_sectors, z_max=z_max, continuous=continuous, params=p,
                                    n_frames=nf)
        trk = trackers[key]
        trk.params = p
        trk.track_batched(sector, row, y, zt, off, bz=bz, v_drift=v_drift)     # warm-up
        times = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            trk.track_batched(sector, row, y, zt, off, bz=bz, v_drift=v_drift)
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        ms = statistics.median(times)
        table.append((cfg, ms))
        if log:
            log(f"autotune {cfg} {ms:.3f} ms")
    trackers.clear()
    best_cfg, best_ms = min(table, key=lambda t: t[1])
    return {"best": best_cfg, "ms": best_ms, "table": table}


def autotune_groups(sector, row, y, zt, frame_offsets, row_x, params: abi.TpcParams, n_sectors=36, z_max=250.0,
                    continuous=True, bz=0.5, v_drift=2.58, space: dict | None = None, reps: int = 3,
                    log=None) -> dict:
    """Time graph replays of GroupedBatch for every (group_clusters,
    n_streams) of `space` on this input; same return shape as autotune."""
    space = space or GROUP_SPACE
    keys = list(space)
    table = []
    for combo in itertools.product(*(space[k] for k in keys)):
        cfg = dict(zip(keys, combo))
        gb = GroupedBatch(sector, row, y, zt, frame_offsets, row_x, params=params, n_sectors=n_sectors,
                          z_max=z_max, continuous=continuous, bz=bz, v_drift=v_drift, **cfg)
        gb.capture()
        gb.replay()
        times = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            gb.replay()
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        del gb
        torch.cuda.empty_cache()
        ms = statistics.median(times)
        table.append((cfg, ms))
        if log:
            log(f"autotune {cfg} {ms:.3f} ms")
    best_cfg, best_ms = min(table, key=lambda t: t[1])
    return {"best": best_cfg, "ms": best_ms, "table": table}


def apply(params: abi.TpcParams, tuned: dict) -> abi.TpcParams:
    for k, v in tuned.items():
        setattr(params, k, v)
    return params


def save(result: dict, path: str):
    with open(path, "w") as f:
        json.dump({"best": result["best"], "ms": result["ms"],
                   "table": [[c, m] for c, m in result["table"]]}, f, indent=1)
