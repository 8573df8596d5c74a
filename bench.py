#!/usr/bin/env python
"""Throughput of the B300 TPC tracker on the 50-collision continuous read-out
frame: TPC clusters/s tracked (CA seeding + Kalman following, selection,
merging, refit), and ms per 50-collision frame.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One step = the whole chain over the frame, as one replay of its captured CUDA
graph (tpc_prepare + tpc_track_async; inputs resident in HBM; 16 M clusters,
160 MB of cluster SoA, larger than the 126 MB L2); the stage times come from
synchronous tpc_track calls with stage events, e2e from tpc_track with host
copies.  Under
torchrun each rank tracks its own frame (different seed): independent
replicas, no collective on the data path ("weak" scaling).  Rank 0 prints one
JSON line.  --impl reference times the CPU oracle on a bounded sample of the
same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "TPC clusters/s tracked (CA + Kalman fit) on 1 B300; ms per 50-collision frame"
WORKLOAD = "50-collision continuous read-out frame (36 sectors x 152 rows, Bz 0.5 T, drift times)"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
# FP32 CUDA-core peak: 148 SMs x 128 FP32 lanes x 2 flop (FMA) x 2.032 GHz
FP32_PEAK_TFLOPS = 148 * 128 * 2 * 2.032e9 / 1e12
# binary32 flops of one step of each decision-path primitive, counted from the
# operation lists in tpc_dev.cuh (FMA = 2, add/mul/div/sqrt = 1)
FLOPS_PROP = 181      # prop32: 71 for the state and Jacobian terms + 110 for F C F^T
FLOPS_UPDATE = 130    # update32: innovation, 2x2 inverse, chi2, gain, state, covariance
FLOPS_CAND = 5        # one grid candidate in the following window: 2 sub + fused distance
FLOPS_MERGE = 520     # merge_chi2: rot32 (~90) + prop32 (181) + 5x5 Cholesky solve (~250)
# binary64 flops of one step of the binary64 final refit pass, counted from its
# operation lists in tpc_fit.cuh / tpc_refit.cu: covariance transport F C F^T
# (64 FMA) + Joseph update (gain 30, (I - KH)C 64, V K 10, C+ 120, residual,
# S, 1/det, chi2 24)
FLOPS_REFIT64 = 376
# nominal B300 binary64 rate (no measured FP64 peak is available)
# DRAM bytes (read + write) per cluster of the frame of one stage (both
# tracklet passes), from the committed ncu capture of the same kernel build
# (profiles/k_tracklets_frame20.md, 20-collision frame, scaled by clusters);
# None once the kernel changes
# Cluster attachment, algorithmic bytes per input cluster: clearing its
# adjacency key and tube mark (8 + 1), one read of its sorted record by the
# tube scan (16), the flag pass reading assignment, key and mark (4 + 8 + 1)
# and writing flags and adjacent track (1 + 4).
ATTACH_B_PER_CLUSTER = 43
# DRAM bytes per input cluster of the three main attachment kernels (trace,
# visit, flags) in an ncu capture of the 35-collision frame (26.5 + 78.8 + 15.9),
# scaled to a launch by the cluster count
NCU_ATTACH_TRAFFIC_B_PER_CLUSTER = 121.2
NCU_TRAFFIC_B_PER_CLUSTER = {"tracklets": 193.7}
# Cluster compression, algorithmic bytes per input cluster (the coded output
# is added per frame): one read of its sector, row, y, zt (10) and of its
# assignment (4), one read of its entry in the track cluster lists (4).
COMPRESS_B_PER_CLUSTER = 18


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--collisions", type=int, default=50)
    ap.add_argument("--cpu-sample-collisions", type=int, default=8)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-attach", action="store_true",
                    help="frame: skip the timing of the optional cluster attachment stage")
    ap.add_argument("--no-compress", action="store_true", help="frame: skip the cluster compression object")
    ap.add_argument("--no-fit", action="store_true", help="calib: skip the closed-loop fit object")
    ap.add_argument("--no-batch", action="store_true",
                    help="frame workload: skip the bounded sub-time-frame batch object (graph vs per-frame loop)")
    ap.add_argument("--batch-stf", type=int, default=16, help="frame workload: sub-time-frames of the batch object")
    ap.add_argument("--batch-max-coll", type=int, default=40,
                    help="frame workload: batch object frames of U{1..N} collisions")
    ap.add_argument("--workload", choices=("frame", "stf_batch", "calib"), default="frame",
                    help="frame: the 50-collision frame; stf_batch: sub-time-frames of 1..max-coll collisions")
    ap.add_argument("--n-stf", type=int, default=64)
    ap.add_argument("--max-coll", type=int, default=100)
    ap.add_argument("--mult", type=float, default=2000.0)
    ap.add_argument("--tune", action="store_true", help="autotune grid and queue settings on the first 8 STFs")
    ap.add_argument("--group-clusters", type=int, default=32_000_000,
                    help="stf_batch: clusters per frame group of the graph (without --tune)")
    ap.add_argument("--n-streams", type=int, default=2, help="stf_batch: concurrent frame groups (without --tune)")
    ap.add_argument("--no-single-call", action="store_true",
                    help="stf_batch: skip the one-call-over-all-frames comparison (its workspace holds the batch)")
    ap.add_argument("--no-packed", action="store_true",
                    help="stf_batch: full-precision link pass (default: 16-bit packed link coordinates)")
    ap.add_argument("--no-fp64-final", action="store_true",
                    help="stf_batch: binary32 final refit (default: binary64 Joseph update of the loopers, binary64 chi2)")
    ap.add_argument("--fp64-all", action="store_true",
                    help="stf_batch: binary64 Joseph covariance update of every track in the final refit pass")
    return ap.parse_args()


def dist_setup(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if ws > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "ours" else "gloo"
        dist.init_process_group(backend)
        pg = dist
    return ws, rank, local, pg


def over_ranks(pg, dev, times, counts):
    """Replicas: the slowest rank's times (max over ranks) and the work of all
    ranks (sum); without a process group the local values."""
    if pg is None:
        return tuple(times), tuple(counts)
    import torch
    t = torch.tensor(list(times), dtype=torch.float64, device=dev)
    c = torch.tensor(list(counts), dtype=torch.float64, device=dev)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    pg.all_reduce(c, op=pg.ReduceOp.SUM)
    return tuple(float(x) for x in t.tolist()), tuple(float(x) for x in c.tolist())


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                       "-i", str(self.index), "-lms", "100"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.p is not None:
            self.p.terminate()
            self.p.wait()
        self.f.flush()

    def summary(self):
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        sm, smax, reasons = [], None, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for r in rows:
            try:
                sm.append(float(r[1]))
                smax = float(r[2])
                for nm, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def peaks():
    try:
        return json.load(open(PEAKS_FILE))
    except OSError:
        return {}


_FMA_PEAK = {}


def fma_peak(dev, precision=32):
    """Fused multiply-add throughput of this GPU (TFLOP/s) from the library's
    probe kernel (tpc_probe_fma: 8 independent chains per thread, 148 x 8
    blocks of 256 threads), timed with CUDA events on the launching stream
    after warm-up launches; the best of the timed launches."""
    import ctypes as C

    import torch

    import paper_1905_05515_b300 as tpc
    key = (str(dev), precision)
    if key in _FMA_PEAK:
        return _FMA_PEAK[key]
    L = tpc.lib()
    blocks, threads = 148 * 8, 256
    iters = (1 << 14) if precision == 32 else (1 << 7)
    out = torch.empty(blocks, dtype=torch.float32 if precision == 32 else torch.float64, device=dev)
    st = torch.cuda.current_stream(dev)
    flops = C.c_int64(0)

    def launch():
        rc = L.tpc_probe_fma(precision, blocks, threads, iters, C.c_void_p(out.data_ptr()), C.byref(flops),
                             C.c_void_p(st.cuda_stream))
        if rc:
            raise tpc.TpcError(rc, "tpc_probe_fma")

    for _ in range(3):
        launch()
    best = None
    for _ in range(10 if precision == 32 else 3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        launch()
        e1.record(st)
        torch.cuda.synchronize(dev)
        t = e0.elapsed_time(e1) / 1e3
        best = t if best is None else min(best, t)
    _FMA_PEAK[key] = flops.value / best / 1e12
    return _FMA_PEAK[key]


def cpu_baseline(n_coll: int, seed: int):
    """The oracle as it stands, single-threaded, on a bounded frame of the same generator."""
    import oracle
    import tpcgen
    ev = tpcgen.time_frame(seed=seed, n_collisions=n_coll, with_truth=False)
    t0 = time.perf_counter()
    cpu0 = time.process_time()
    r = oracle.track_event(ev)
    dt = time.perf_counter() - t0
    cpu = time.process_time() - cpu0
    out = {"value": ev.n / dt, "unit": "clusters/s", "cores": 1, "kind": "oracle",
           "sample": f"{n_coll}-collision frame of the same generator (seed {seed}), {ev.n} clusters, "
                     f"{r.n_tracks} tracks, {dt:.1f} s wall / {cpu:.1f} s CPU, single thread"}
    out["all_cores"] = cpu_all_cores(n_coll, seed)
    return out


def _oracle_frame(job):
    import oracle
    import tpcgen
    seed, n_coll = job
    ev = tpcgen.time_frame(seed=seed, n_collisions=n_coll, with_truth=False)
    t0 = time.perf_counter()
    oracle.track_event(ev)
    return ev.n, time.perf_counter() - t0


def cpu_all_cores(n_coll: int, seed: int):
    """The oracle on every host core: one independent frame per process (frames
    shard with no exchange), spawned processes; bounded to 32 processes."""
    import concurrent.futures as cf
    import multiprocessing as mp
    cores = max(1, min(os.cpu_count() or 1, 32))
    jobs = [(seed + 100 + k, n_coll) for k in range(cores)]
    t0 = time.perf_counter()
    with cf.ProcessPoolExecutor(cores, mp_context=mp.get_context("spawn")) as ex:
        res = list(ex.map(_oracle_frame, jobs))
    wall = time.perf_counter() - t0
    n = sum(r[0] for r in res)
    slow = max(r[1] for r in res)
    return {"value": n / slow, "unit": "clusters/s", "cores": cores, "kind": "oracle",
            "sample": f"{cores} {n_coll}-collision frames tracked side by side, one per spawned process ({n} "
                      f"clusters); value = all clusters over the slowest process's tracking time ({slow:.1f} s; "
                      f"{wall:.1f} s wall with process start-up and frame generation)"}


def run_reference(args, ws, rank, pg):
    if rank != 0:
        return
    import oracle
    import tpcgen
    oracle.lib()
    n_coll = args.cpu_sample_collisions
    evs = [tpcgen.time_frame(seed=900 + i, n_collisions=n_coll, with_truth=False)
           for i in range(args.warmup + args.steps)]
    for ev in evs[:args.warmup]:
        oracle.track_event(ev)
    t0 = time.perf_counter()
    n = 0
    for ev in evs[args.warmup:]:
        oracle.track_event(ev)
        n += ev.n
    dt = time.perf_counter() - t0
    v = n / dt
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "clusters/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32/f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD + f", bounded to {n_coll} collisions per step for the CPU",
                       "n_collisions": n_coll, "clusters_per_step": n // args.steps},
            "cpu_baseline": {"value": v, "unit": "clusters/s", "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} frames of {n_coll} collisions, single thread"},
            "e2e": {"value": v, "unit": "clusters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def batch_object(cat, off, ncoll, dev, steps, warmup, max_coll):
    """Batched mode at bounded size: the same sub-time-frames tracked by a
    loop of synchronous tpc_track calls (one per frame) and by one replay of
    a captured GroupedBatch graph (frame groups on two streams), in the
    configuration of the batched workload (binary64 final refit of the
    loopers, 16-bit packed link coordinates); both timed with CUDA events,
    outputs compared bit for bit."""
    import numpy as np
    import torch

    import paper_1905_05515_b300 as tpc
    import tpcgen
    host = {k: torch.from_numpy(np.ascontiguousarray(v)) for k, v in cat.items()}
    dv = {k: v.to(dev) for k, v in host.items()}
    ins = (dv["sector"], dv["row"], dv["y"], dv["zt"])
    row_x = tpcgen.row_x_f32()
    params = tpc.tpc_params_default(tracklets_per_1k=60, fp64_final=2, packed_links=1)
    nstf = len(ncoll)
    vd, bz = tpcgen.V_DRIFT, 0.5
    big = int(np.max(np.diff(off)))
    one = tpc.Tracker(big, row_x, continuous=True, params=params, device=dev)

    def per_frame():
        ps = []
        for i in range(nstf):
            a, b = int(off[i]), int(off[i + 1])
            ps.append(one.track(*(t[a:b] for t in ins), bz=bz, v_drift=vd).param.clone())
        return ps

    def timed(fn, k):
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(k):
            fn()
        e1.record()
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / k

    for _ in range(max(1, warmup)):
        per_frame()
    ms_frame = timed(per_frame, steps)
    p_frame = torch.cat(per_frame()).cpu().numpy()
    launches_frame = sum(one.track(*(t[int(off[i]):int(off[i + 1])] for t in ins), bz=bz, v_drift=vd).n_launches
                         for i in range(nstf))
    del one
    torch.cuda.empty_cache()
    gb = tpc.GroupedBatch(*ins, off, row_x, params=params, bz=bz, v_drift=vd, group_clusters=32_000_000,
                          n_streams=2)
    gb.capture()
    for _ in range(max(1, warmup)):
        gb.replay()
    ms_graph = timed(gb.replay, steps)
    res = gb.results()
    p_graph = torch.cat([r.param for r in res]).cpu().numpy()
    n_tracks = sum(r.n_tracks for r in res)
    same = bool(np.array_equal(p_graph, p_frame))
    out = {"workload": f"{nstf} sub-time-frames of U{{1..{max_coll}}} collisions "
                       f"(multiplicity Exp(2000), 50 kHz), binary64 final refit of the loopers, packed link "
                       f"coordinates", "clusters": int(off[-1]), "collisions": int(ncoll.sum()),
           "tracks": int(n_tracks), "groups": len(gb.groups), "graph_ms": ms_graph, "per_frame_ms": ms_frame,
           "speedup_vs_per_frame": ms_frame / ms_graph, "identical_to_per_frame": same,
           "graph_clusters_per_s": int(off[-1]) / (ms_graph / 1e3),
           "per_frame_clusters_per_s": int(off[-1]) / (ms_frame / 1e3),
           "graph_launches": gb.n_launches, "per_frame_launches": launches_frame,
           "timing": "CUDA events around one replay (graph) or one loop of synchronous calls (per frame), "
                     f"mean of {steps}"}
    del gb, res, dv
    torch.cuda.empty_cache()
    return out


def run_ours(args, ws, rank, local, pg):
    import numpy as np
    import torch

    import paper_1905_05515_b300 as tpc
    import tpcgen
    batch_in = None
    if not args.no_batch:
        # generated in a spawned process pool before this process uses CUDA
        batch_in = make_stf_batch(args.batch_stf, args.batch_max_coll, 2000.0, seed0=2000 + 100 * rank)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    ev = tpcgen.time_frame(seed=3 + rank, n_collisions=args.collisions, with_truth=False)
    n = ev.n
    host = {k: torch.from_numpy(np.ascontiguousarray(getattr(ev, k))).pin_memory()
            for k in ("sector", "row", "y", "zt")}
    dv = {k: v.to(dev) for k, v in host.items()}
    params = tpc.tpc_params_default(profile=1)
    trk = tpc.Tracker(n, ev.row_x, n_sectors=36, z_max=ev.z_max, continuous=True, params=params, device=dev)
    args_t = (dv["sector"], dv["row"], dv["y"], dv["zt"])
    stream = torch.cuda.current_stream(dev)

    def barrier():
        if pg is not None:
            pg.barrier()

    for _ in range(args.warmup):
        res = trk.track(*args_t, bz=ev.bz, v_drift=ev.v_drift)
    torch.cuda.synchronize()

    # ---- stage breakdown: synchronous calls with the library's stage events
    stage_sum = {k: 0.0 for k in tpc.abi.STAGES}
    work_sum = {}
    for _ in range(args.steps):
        res = trk.track(*args_t, bz=ev.bz, v_drift=ev.v_drift)
        for k, v in res.stage_ms.items():
            stage_sum[k] += v
        for k, v in res.work.items():
            work_sum[k] = work_sum.get(k, 0) + v
    n_tracks = res.n_tracks
    p_sync = res.param[:n_tracks].cpu().numpy().copy()

    # ---- device-resident timed region: the whole chain of one frame captured
    # as a CUDA graph (tpc_prepare + tpc_track_async), one replay per step
    trk.params.profile = 0
    run = trk.capture(*args_t, bz=ev.bz, v_drift=ev.v_drift)
    launches_per_step = trk.track(*args_t, bz=ev.bz, v_drift=ev.v_drift).n_launches
    for _ in range(args.warmup):
        run.replay()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            run.replay()
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
    ms = e0.elapsed_time(e1)
    launches = launches_per_step * args.steps
    rg = run.result()
    same_as_sync = bool(rg.n_tracks == n_tracks and np.array_equal(rg.param[:n_tracks].cpu().numpy(), p_sync))

    # ---- end to end from host memory: the public streaming API, FramePipeline
    # (per frame: host->device copies of the clusters, tracking, device->host
    # copies of the filled outputs; a frame's copies run beside the tracking of
    # the next one), and the synchronous tpc_track call with the same copies
    pipe = tpc.FramePipeline(n, ev.row_x, depth=2, n_sectors=36, z_max=ev.z_max, continuous=True, bz=ev.bz,
                             v_drift=ev.v_drift, device=dev)
    hin = (host["sector"], host["row"], host["y"], host["zt"])
    for _ in range(2):
        pipe.push(*hin)
    pipe.flush()
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    d2h_list, h2d = [], 0
    for _ in range(args.steps):
        r = pipe.push(*hin)
        if r is not None:
            d2h_list.append(r.d2h_bytes)
            h2d = r.h2d_bytes
    for r in pipe.flush():
        d2h_list.append(r.d2h_bytes)
        h2d = r.h2d_bytes
    e2e_s = time.perf_counter() - t0
    pipe_same = bool(r.n_tracks == n_tracks and np.array_equal(r.param.numpy(), p_sync))
    del pipe
    torch.cuda.empty_cache()
    barrier()

    T_cap = trk.capacity_tracks
    outs = {"param": (T_cap, 5), "cov": (T_cap, 15), "chi2": (T_cap,), "ndf": (T_cap,), "nclus": (T_cap,),
            "clus_offset": (T_cap + 1,)}
    h_out = {k: torch.empty(sh, dtype=trk.buf[k].dtype).pin_memory() for k, sh in outs.items()}
    h_clus = torch.empty(trk.capacity_clusters, dtype=torch.int32).pin_memory()
    h_assign = torch.empty(n, dtype=torch.int32).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for k in dv:
            dv[k].copy_(host[k], non_blocking=True)
        rs = trk.track(*args_t, bz=ev.bz, v_drift=ev.v_drift)
        T = rs.n_tracks
        for k in outs:
            m = T + 1 if k == "clus_offset" else T
            h_out[k][:m].copy_(trk.buf[k][:m], non_blocking=True)
        nc = int(rs.clus_offset[-1].item()) if T else 0
        h_clus[:nc].copy_(trk.buf["clus_index"][:nc], non_blocking=True)
        h_assign.copy_(rs.assign, non_blocking=True)
        torch.cuda.synchronize()
    sync_s = time.perf_counter() - t0
    barrier()

    # ---- the optional track-based cluster attachment (not part of the step
    # above): its stage time from profiled synchronous calls of a tracker with
    # the attachment outputs, its flag counts and its roofline
    attach = None
    if not args.no_attach:
        trk_a = tpc.Tracker(n, ev.row_x, n_sectors=36, z_max=ev.z_max, continuous=True,
                            params=tpc.tpc_params_default(profile=1), device=dev, attach=True)
        for _ in range(args.warmup):
            trk_a.track(*args_t, bz=ev.bz, v_drift=ev.v_drift)
        a_ms = []
        for _ in range(args.steps):
            ra = trk_a.track(*args_t, bz=ev.bz, v_drift=ev.v_drift)
            a_ms.append(ra.stage_ms["attach"])
        fl = ra.cl_flags
        counts = {k: int(((fl & b) != 0).sum().item()) for k, b in (("attached", tpc.abi.CL_ATTACHED),
                                                                    ("adjacent", tpc.abi.CL_ADJACENT),
                                                                    ("protected", tpc.abi.CL_PROTECTED),
                                                                    ("remove", tpc.abi.CL_REMOVE))}
        same_assign = bool(torch.equal(ra.assign, rs.assign))
        t_att = sum(a_ms) / len(a_ms)
        hbm = peaks().get("hbm_gbs")
        ach = ATTACH_B_PER_CLUSTER * n / (t_att / 1e3) / 1e9
        attach = {"ms": round(t_att, 4), "tube_radius_cm": float(trk_a.params.tube_radius),
                  "pt_min_gev": float(trk_a.params.pt_min_physics), "counts": counts,
                  "tracks_identical_to_step": same_assign,
                  "roofline": {"bound": "hbm", "achieved": round(ach, 1), "unit": "GB/s",
                               "peak": hbm if hbm else 6400.0,
                               "frac": round(ach / (hbm if hbm else 6400.0), 4),
                               "bytes_per_cluster": ATTACH_B_PER_CLUSTER,
                               "traffic": NCU_ATTACH_TRAFFIC_B_PER_CLUSTER * n,
                               "peak_note": "measured" if hbm else "fallback"}}
        del trk_a, ra, fl
        torch.cuda.empty_cache()
    barrier()

    # ---- the cluster compression of the frame (not part of the step): the
    # compressed format of the frame's clusters with the step's tracks
    compress = None
    if not args.no_compress:
        T = rs.n_tracks
        off = rs.clus_offset[:T + 1].contiguous()
        na = int(off[-1].item()) if T else 0
        cargs = (dv["sector"], dv["row"], dv["y"], dv["zt"], off, rs.clus_index[:na].contiguous(),
                 rs.assign.contiguous())
        cw, co = tpc.compress.compress_buffers(*cargs)
        for _ in range(args.warmup):
            data, sizes = tpc.compress_frame(*cargs, workspace=cw, out=co)
        first = data.clone()
        ce = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        c_ms = []
        for _ in range(args.steps):
            ce[0].record(stream)
            data, sizes = tpc.compress_frame(*cargs, workspace=cw, out=co)
            ce[1].record(stream)
            torch.cuda.synchronize()
            c_ms.append(ce[0].elapsed_time(ce[1]))
        t_c = sum(c_ms) / len(c_ms)
        total = sum(sizes)
        hbm = peaks().get("hbm_gbs") or 6400.0
        alg = COMPRESS_B_PER_CLUSTER * n + total
        compress = {"ms": round(t_c, 4), "bytes": total, "bytes_per_cluster": round(total / n, 4),
                    "factor_vs_float_clusters": round(10.0 * n / total, 3),
                    "input_gb_per_s": round(10.0 * n / (t_c / 1e3) / 1e9, 1),
                    "stream_bytes": dict(zip(tpc.abi.CMP_STREAMS, sizes)),
                    "repeat_identical": bool(torch.equal(first, data)),
                    "roofline": {"bound": "hbm", "achieved": round(alg / (t_c / 1e3) / 1e9, 1), "unit": "GB/s",
                                 "peak": hbm, "frac": round(alg / (t_c / 1e3) / 1e9 / hbm, 4),
                                 "bytes_per_cluster": COMPRESS_B_PER_CLUSTER, "traffic": None,
                                 "peak_note": "measured" if peaks().get("hbm_gbs") else "fallback"},
                    "timing": "CUDA events around tpc_compress_frame (it synchronises twice to read stream sizes)"}
        del cw, co, data, first
        torch.cuda.empty_cache()
    barrier()

    # ---- the bounded batch object: graph-captured frame groups against the per-frame loop
    batch = None
    if batch_in is not None:
        batch = batch_object(*batch_in, dev, max(3, args.steps // 2), args.warmup, args.batch_max_coll)
    barrier()
    # ---- measured FMA rates (roofline denominators of the Kalman stages)
    fp32_peak, fp64_peak = fma_peak(dev, 32), fma_peak(dev, 64)

    # ---- max over ranks, totals
    (ms_max, e2e_max, sync_max), (n_total,) = over_ranks(pg, dev, (ms, e2e_s, sync_s), (float(n),))
    if rank != 0:
        return
    value = n_total * args.steps / (ms_max / 1e3)
    per_step = {k: v / args.steps for k, v in stage_sum.items()}
    w = {k: v / args.steps for k, v in work_sum.items()}
    dom = max(per_step, key=per_step.get)
    pk_all = dict(peaks(), fp32_tflops_measured=fp32_peak)
    n_assigned = int(rs.clus_offset[-1].item()) if rs.n_tracks else 0
    roof = roofline(dom, per_step, w, n, pk_all, n_assigned)
    stage_roofs = {}
    for st_ in per_step:
        rf = roofline(st_, per_step, w, n, pk_all, n_assigned)
        stage_roofs[st_] = {"bound": rf["bound"], "achieved": round(rf["achieved"], 3), "unit": rf["unit"],
                            "frac": round(rf["frac"], 4)}
    line = {
        "metric": METRIC, "value": value, "unit": "clusters/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD if args.collisions == 50 else WORKLOAD.replace("50-collision", f"{args.collisions}-collision"),
                   "n_collisions": args.collisions, "clusters": n, "tracks_found": n_tracks,
                   "collisions_per_s": args.collisions * ws * args.steps / (ms_max / 1e3),
                   "ms_per_frame": ms_max / args.steps,
                   "l2": "inputs (10 B/cluster, 160 MB) and workspace exceed the 126 MB L2; no flush",
                   "replicas": ws, "step": "one replay of the frame's captured CUDA graph (all stages)",
                   "graph_identical_to_sync_call": same_as_sync,
                   "e2e_api": "FramePipeline, depth 2 (copies of a frame beside the tracking of the next)",
                   "e2e_pipeline_identical_to_sync_call": pipe_same,
                   "e2e_sync_call_clusters_per_s": n_total * args.steps / sync_max},
        "roofline": roof,
        "stage_ms": {k: round(v, 4) for k, v in per_step.items()},
        "stage_rooflines": stage_roofs,
        "work_per_step": w,
        "e2e": {"value": n_total * args.steps / e2e_max, "unit": "clusters/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": int(sum(d2h_list) / len(d2h_list))},
        "gpu_launches": launches,
        "clocks": clk.summary(),
    }
    line["measured_peaks"] = {"fp32_tflops": round(fp32_peak, 2), "fp64_tflops": round(fp64_peak, 3),
                              "how": "tpc_probe_fma: 148 x 8 blocks x 256 threads x 8 independent FMA chains, "
                                     "best of the CUDA-event-timed launches after warm-up"}
    if attach is not None:
        line["attach"] = attach
    if compress is not None:
        line["compress"] = compress
    if batch is not None:
        line["batch"] = batch
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.cpu_sample_collisions, seed=3)
    print(json.dumps(line), flush=True)


def _gen_stf(args):
    import tpcgen
    seed, nc, mult = args
    ev = tpcgen.time_frame(seed=seed, n_collisions=int(nc), mult_mean=mult, frame_us=float(nc) * 20.0,
                           with_truth=False)
    return ev.sector, ev.row, ev.y, ev.zt, ev.n


def make_stf_batch(n_stf, max_coll, mult, seed0=1000):
    """Sub-time-frames of U{1..max_coll} collisions at 50 kHz (n collisions over
    n/50 ms), generated in a spawned process pool before any CUDA use."""
    import concurrent.futures as cf
    import multiprocessing as mp

    import numpy as np
    rng = np.random.Generator(np.random.Philox(seed0))
    ncoll = rng.integers(1, max_coll + 1, n_stf)
    jobs = [(seed0 + 1 + i, int(nc), mult) for i, nc in enumerate(ncoll)]
    workers = max(1, min(len(jobs), (os.cpu_count() or 2) // 2))
    with cf.ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn")) as ex:
        parts = list(ex.map(_gen_stf, jobs))
    sizes = np.array([p[4] for p in parts], np.int64)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    cat = {}
    for k, name in enumerate(("sector", "row", "y", "zt")):
        cat[name] = np.concatenate([p[k] for p in parts])
    return cat, off, ncoll


def _oracle_stf(job):
    """One sub-time-frame through the oracle (process-pool worker)."""
    import oracle
    import tpcgen
    sector, row, y, zt, packed = job
    t0 = time.perf_counter()
    r = oracle.track(sector, row, y, zt, tpcgen.row_x_f32(), n_sectors=36, z_max=250.0, continuous=True, bz=0.5,
                     v_drift=tpcgen.V_DRIFT, params={"packed_links": int(packed)})
    dt = time.perf_counter() - t0
    return dict(dt=dt, n_tracks=r.n_tracks, tr_clus=r.tr_clus, assign=r.assign, tr_status=r.tr_status, tr_p=r.tr_p,
                tr_chi2=r.tr_chi2, tr_ndf=r.tr_ndf, tr_c=r.tr_c)


def _stf_errors(k, a, b, r, res, base, fp64):
    """Errors of frame k of the batch's results against the oracle's run of it
    (decisions exact; fit relative to the binary64 oracle refit on the tracks
    that are fits of one helix, chi2/ndf < 100 in the oracle, the others
    counted)."""
    import numpy as np
    fr = res.frame.cpu().numpy()
    idx = np.nonzero(fr == k)[0]
    err = {"frame": int(k), "clusters": b - a, "tracks_gpu": int(idx.size), "tracks_oracle": int(r["n_tracks"])}
    if idx.size == r["n_tracks"] and idx.size > 0:
        t_lo, t_hi = int(idx[0]), int(idx[-1]) + 1
        co = res.clus_offset.cpu().numpy()
        ci = res.clus_index[int(co[t_lo]):int(co[t_hi])].cpu().numpy() - (a - base)
        asg = res.assign[a - base:b - base].cpu().numpy()
        asg = np.where(asg >= 0, asg - t_lo, -1)
        err["clusters_mismatch"] = int(ci.size != r["tr_clus"].size or (ci != r["tr_clus"]).sum())
        err["assign_mismatch"] = int((asg != r["assign"]).sum())
        st = res.status[t_lo:t_hi].cpu().numpy()
        both = (st == 0) & (r["tr_status"] == 0)
        helix = r["tr_chi2"] < 100.0 * np.maximum(r["tr_ndf"], 1)
        ok = both & helix
        err["status_mismatch"] = int((st != r["tr_status"]).sum())
        err["not_helix"] = int((both & ~helix).sum())
        p = res.param[t_lo:t_hi].cpu().numpy().astype(np.float64)[ok]
        floor = np.array([1.0, 1.0, 1e-2, 1e-2, 1e-2])
        pe = np.abs(p - r["tr_p"][ok]) / np.maximum(np.abs(r["tr_p"][ok]), floor)
        # the parity bar: 1e-4 relative; tracks above it are counted, and those
        # of them also beyond 1e-3 of the parameter's sigma counted apart
        sig = np.sqrt(np.abs(r["tr_c"][ok][:, [0, 2, 5, 9, 14]]))
        over = pe > 1e-4
        err["param_over_tol"] = int(over.any(axis=1).sum())
        err["param_over_tol_beyond_1e-3_sigma"] = int((over & (np.abs(p - r["tr_p"][ok]) > 1e-3 * sig)).any(axis=1).sum())
        chi = (res.chi2_64 if fp64 else res.chi2)[t_lo:t_hi].cpu().numpy().astype(np.float64)[ok]
        ce = np.abs(chi - r["tr_chi2"][ok]) / np.maximum(r["tr_chi2"][ok], 1.0)
        cov = (res.cov64 if fp64 else res.cov)[t_lo:t_hi].cpu().numpy().astype(np.float64)[ok]
        dg = [0, 2, 5, 9, 14]
        ve = np.abs(cov[:, dg] - r["tr_c"][ok][:, dg]) / np.abs(r["tr_c"][ok][:, dg])
        err.update(param_rel_max=pe.max(axis=0).tolist() if pe.size else None,
                   param_rel_p99=np.percentile(pe, 99, axis=0).tolist() if pe.size else None,
                   chi2_rel_max=float(ce.max()) if ce.size else None,
                   cov_diag_rel_max=float(ve.max()) if ve.size else None)
    return err


def batch_cpu_baseline(pool, jobs, picks, wall, off, results, fp64):
    """cpu_baseline of the batch: the oracle as it stands on a seeded sample
    of sub-time-frames (the smallest and seven random ones of at most 8 M
    clusters), one process per frame on the host cores, and the batch's
    errors against it on every sampled frame.  jobs: the pool's pending results; results(k) ->
    (result holding frame k, its first cluster index)."""
    out = [j.get() for j in jobs]
    wall = time.perf_counter() - wall
    errs, n_tot, t_tot = [], 0, 0.0
    for k, r in zip(picks, out):
        a, b = int(off[k]), int(off[k + 1])
        res, base = results(k)
        errs.append(_stf_errors(k, a, b, r, res, base, fp64))
        n_tot += b - a
        t_tot += r["dt"]
    pool.close()
    worst = {key: sum((e.get(key) or 0) for e in errs) for key in ("clusters_mismatch", "assign_mismatch",
                                                                  "status_mismatch", "not_helix",
                                                                  "param_over_tol",
                                                                  "param_over_tol_beyond_1e-3_sigma")}
    pmax = [max((e["param_rel_max"] or [0] * 5)[i] for e in errs) for i in range(5)]
    return {"value": n_tot / wall, "unit": "clusters/s", "cores": len(picks), "kind": "oracle",
            "single_thread_clusters_per_s": n_tot / t_tot,
            "sample": f"{len(picks)} sub-time-frames of the batch (the smallest and 7 seeded random ones of at most "
                      f"8 M clusters: the largest, 42 M, takes the oracle minutes; {n_tot} clusters), one oracle "
                      f"process each on the host cores, {wall:.1f} s wall",
            "error_vs_oracle": {"frames": [int(k) for k in picks], **worst, "param_rel_max": pmax,
                                "chi2_rel_max": max((e.get("chi2_rel_max") or 0) for e in errs),
                                "cov_diag_rel_max": max((e.get("cov_diag_rel_max") or 0) for e in errs),
                                "tracks_match": all(e["tracks_gpu"] == e["tracks_oracle"] for e in errs)}}


def run_batch(args, ws, rank, local, pg):
    """Batched mode: the whole sub-time-frame batch per step, tracked as a
    graph-captured GroupedBatch (frame groups on several streams), against
    the per-frame loop (one tpc_track call per frame) and one
    tpc_track_batched call over all frames; all three give the same tracks."""
    import numpy as np
    cat, off, ncoll = make_stf_batch(args.n_stf, args.max_coll, args.mult, seed0=1000 + 100 * rank)
    import torch

    import paper_1905_05515_b300 as tpc
    import tpcgen
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    n = int(off[-1])
    host = {k: torch.from_numpy(np.ascontiguousarray(v)).pin_memory() for k, v in cat.items()}
    dv = {k: v.to(dev) for k, v in host.items()}
    ins = (dv["sector"], dv["row"], dv["y"], dv["zt"])
    row_x = tpcgen.row_x_f32()
    off32 = off.astype(np.int32)
    fp64_mode = 0 if args.no_fp64_final else (1 if args.fp64_all else 2)
    fp64 = fp64_mode > 0
    packed = not args.no_packed
    params = tpc.tpc_params_default(tracklets_per_1k=60, fp64_final=fp64_mode, packed_links=int(packed))
    nstf = len(ncoll)
    vd, bz = tpcgen.V_DRIFT, 0.5
    log = lambda m: print(m, file=sys.stderr)  # noqa: E731
    tuned = {}
    if args.tune:
        k = min(8, nstf)
        sub = tuple(t[:int(off[k])] for t in ins)
        t1 = tpc.autotune.autotune(*sub, off32[:k + 1], row_x, base=params, log=log)
        tpc.autotune.apply(params, t1["best"])
        k = min(16, nstf)
        sub = tuple(t[:int(off[k])] for t in ins)
        t2 = tpc.autotune.autotune_groups(*sub, off[:k + 1], row_x, params, bz=bz, v_drift=vd, log=log)
        tuned = {**t1["best"], **t2["best"]}
    group = {"group_clusters": tuned.get("group_clusters", args.group_clusters),
             "n_streams": tuned.get("n_streams", args.n_streams)}

    def timed(fn, steps):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    # ---- per-frame loop
    big = int(np.max(np.diff(off)))
    one = tpc.Tracker(big, row_x, continuous=True, params=params)

    def per_frame():
        ps = []
        for i in range(nstf):
            a, b = int(off[i]), int(off[i + 1])
            ps.append(one.track(*(t[a:b] for t in ins), bz=bz, v_drift=vd).param.clone())
        return ps

    for _ in range(min(args.warmup, 1)):
        per_frame()
    ms_frame = timed(per_frame, max(1, args.steps // 2))
    p_frame = torch.cat(per_frame()).cpu().numpy()
    one.params.profile = 1
    pf_stage_ms = {k: 0.0 for k in tpc.abi.STAGES}
    pf_work = {}
    pf_sizes = []                    # (clusters, ms) of every frame: time against size
    for i in range(nstf):
        a, b = int(off[i]), int(off[i + 1])
        r1 = one.track(*(t[a:b] for t in ins), bz=bz, v_drift=vd)
        pf_sizes.append((b - a, sum(r1.stage_ms.values())))
        for k, v in r1.stage_ms.items():
            pf_stage_ms[k] += v
        for k, v in r1.work.items():
            pf_work[k] = pf_work.get(k, 0) + v
    one.params.profile = 0
    del one
    torch.cuda.empty_cache()

    # ---- one tpc_track_batched call over every frame
    ms_batch, same_batch, stage_ms = None, None, None
    if not args.no_single_call:
        trk = tpc.Tracker(n, row_x, continuous=True, params=params, n_frames=nstf)
        trk.track_batched(*ins, off32, bz=bz, v_drift=vd)
        ms_batch = timed(lambda: trk.track_batched(*ins, off32, bz=bz, v_drift=vd), max(1, args.steps // 2))
        same_batch = bool(np.array_equal(trk.track_batched(*ins, off32, bz=bz, v_drift=vd).param.cpu().numpy(),
                                         p_frame))
        trk.params.profile = 1
        stage_ms = trk.track_batched(*ins, off32, bz=bz, v_drift=vd).stage_ms
        trk.params.profile = 0
        del trk
        torch.cuda.empty_cache()

    # ---- grouped graph (the timed headline)
    gb = tpc.GroupedBatch(*ins, off, row_x, params=params, bz=bz, v_drift=vd, **group)
    gb.capture()
    for _ in range(args.warmup):
        gb.replay()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        ms_graph = timed(gb.replay, args.steps)
    res = gb.results()
    p_graph = torch.cat([r.param for r in res]).cpu().numpy()
    n_tracks = sum(r.n_tracks for r in res)
    same = bool(np.array_equal(p_graph, p_frame))
    # end to end from host memory: the same graph captured with every group's
    # host->device copy of its clusters and device->host copy of its results
    # (parameters and chi2 at the group's track capacity, counts, assignments)
    # on its own stream, so copies of one group overlap the tracking of others
    gb.capture(host_in=(host["sector"], host["row"], host["y"], host["zt"]))
    gb.replay()
    gb.host_results()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        gb.replay()
        hres = gb.host_results()
    e2e_s = (time.perf_counter() - t0) / args.steps
    e2e_same = bool(np.array_equal(torch.cat([h[1] for h in hres]).numpy(), p_graph))
    h2d, d2h = gb.host_io_bytes()
    # time against frame size: a linear fit over the frames, and ns per cluster
    # of the smallest and the largest third
    nz = np.array(pf_sizes, dtype=np.float64)
    order = np.argsort(nz[:, 0])
    third = max(1, len(order) // 3)
    fit = np.polyfit(nz[:, 0] / 1e6, nz[:, 1], 1)
    scaling = {"frames": len(order), "clusters_min": int(nz[:, 0].min()), "clusters_max": int(nz[:, 0].max()),
               "fit_ms_per_M_clusters": float(fit[0]), "fit_intercept_ms": float(fit[1]),
               "ns_per_cluster_smallest_third": float(1e6 * nz[order[:third], 1].sum() / nz[order[:third], 0].sum()),
               "ns_per_cluster_largest_third": float(1e6 * nz[order[-third:], 1].sum() / nz[order[-third:], 0].sum())}
    # roofline of the dominant stage of the per-frame calls (stage events)
    dom = max(pf_stage_ms, key=pf_stage_ms.get)
    fp32_peak, fp64_peak = fma_peak(dev, 32), fma_peak(dev, 64)
    if dom == "refit" and fp64_mode == 1:
        fl = pf_work["refit_prop"] / params.refit_passes * FLOPS_REFIT64
        ach = fl / (pf_stage_ms["refit"] / 1e3) / 1e12
        roof = {"bound": "fp64", "stage": "refit", "achieved": ach, "peak": fp64_peak, "unit": "TFLOP/s",
                "frac": ach / fp64_peak, "traffic": None,
                "peak_note": "measured binary64 FMA rate (tpc_probe_fma, CUDA events); the stage time includes "
                             "the two binary32 passes"}
    else:
        roof = roofline(dom, pf_stage_ms, pf_work, n, dict(peaks(), fp32_tflops_measured=fp32_peak))
    (ms_graph, e2e_s), (n_all,) = over_ranks(pg, dev, (ms_graph, e2e_s), (float(n),))
    if rank != 0:
        return
    line = {
        "metric": METRIC + " (batched sub-time-frames)", "value": n_all / (ms_graph / 1e3), "unit": "clusters/s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_graph,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"{nstf} sub-time-frames of U{{1..{args.max_coll}}} collisions, "
                               f"multiplicity Exp({args.mult:g}), one batch per step",
                   "clusters": n, "collisions": int(ncoll.sum()), "tracks_found": n_tracks,
                   "groups": len(gb.groups), **group,
                   "graph_ms": ms_graph, "per_frame_ms": ms_frame, "single_call_ms": ms_batch,
                   "e2e_api": "GroupedBatch graph captured with per-group host I/O (host_in)",
                   "e2e_identical": e2e_same,
                   "speedup_vs_per_frame": ms_frame / ms_graph, "identical_to_per_frame": same,
                   "single_call_identical": same_batch, "tuned": tuned or None,
                   "single_call_stage_ms": {k: round(v, 3) for k, v in stage_ms.items()} if stage_ms else None,
                   "per_frame_stage_ms": {k: round(v, 3) for k, v in pf_stage_ms.items()},
                   "per_frame_scaling": scaling,
                   "final_refit": {0: "fp32", 1: "fp64 Joseph covariance of every track + fp64 chi2",
                                   2: "fp64 Joseph covariance of the loopers (|q/pT| >= 5 or more clusters than "
                                      "rows), fp32 update of the others, fp64 chi2"}[fp64_mode],
                   "link_coordinates": "16-bit packed (1/256 cm)" if packed else "fp32",
                   "l2": "inputs (10 B/cluster) exceed the 126 MB L2; no flush"},
        "roofline": roof,
        "e2e": {"value": n_all / e2e_s, "unit": "clusters/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": gb.n_launches * args.steps,
        "clocks": clk.summary(),
    }
    if not args.no_cpu_baseline:
        import multiprocessing as mp
        sizes = np.diff(off)
        rng = np.random.default_rng(7)
        rest = [k for k in range(nstf) if k != int(np.argmin(sizes)) and sizes[k] <= 8_000_000]
        picks = [int(np.argmin(sizes))] + sorted(rng.choice(rest, min(7, len(rest)), replace=False).tolist())
        pool = mp.get_context("spawn").Pool(len(picks))
        wall = time.perf_counter()
        jobs = [pool.apply_async(_oracle_stf, ((cat["sector"][int(off[k]):int(off[k + 1])],
                                                cat["row"][int(off[k]):int(off[k + 1])],
                                                cat["y"][int(off[k]):int(off[k + 1])],
                                                cat["zt"][int(off[k]):int(off[k + 1])], packed),))
                for k in picks]

        def holding(k):
            gi = next(i for i, g in enumerate(gb.groups) if g.f0 <= k < g.f1)
            return res[gi], gb.groups[gi].a

        line["cpu_baseline"] = batch_cpu_baseline(pool, jobs, picks, wall, off, holding, fp64)
    print(json.dumps(line), flush=True)


# binary32 flops per step of the calibration pass, counted from the operation
# lists in tpc_calib.cu / tpc_fit.cuh: reference helix step 60, deviation
# propagation 12, covariance transport 100, update 80, calibrated measurement
# (w B-spline basis 40, 4 x 4 spline sums 64, chain rule 10) 114; the backward
# recomputes the reference step (60) and the measurement (114), forms the
# smoothed residual (6), applies the inverse step Jacobians (16) and adds the
# 4 x 4 x 2 gradient products (70); both evaluate the map's slope at the
# nominal position for the error scale of m_z (basis 40, 4 x 4 sums 32,
# scale and variance 6) and the backward adds its 4 x 4 variance-term
# products (40)
FLOPS_CALIB_FWD = 444
FLOPS_CALIB_BWD = 384


def run_calib(args, ws, rank, local, pg):
    """Calibration workload: the 50-collision frame generated with v_drift
    +0.3 %, t0 = 200 ns and a 36 x 8 x 8 spline distortion map; the tracker
    (untimed) finds the tracks, then one step = the calibration chi2 of every
    selected track and its gradient with respect to theta through
    torch.autograd (tpc_calib_forward + tpc_calib_backward)."""
    import numpy as np
    import torch

    import paper_1905_05515_b300 as tpc
    import tpcgen
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    ev = tpcgen.calib_frame(seed=5 + rank, n_collisions=args.collisions)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
    cl = (t(ev.sector), t(ev.row), t(ev.y), t(ev.zt))
    trk = tpc.Tracker(ev.n, ev.row_x, continuous=True, device=dev)
    res = trk.track(*cl, bz=ev.bz, v_drift=ev.v_drift)
    T = res.n_tracks
    off = res.clus_offset[:T + 1].cpu().numpy()
    clus = res.clus_index[:int(off[-1])].cpu().numpy()
    tc = tpc.calib.select_tracks(t(tpcgen.track_collision_time(ev, off, clus)), res.status[:T], res.param[:T])
    tg = t(tpcgen.track_dip_angle(ev, off, clus))
    calib = tpc.CalibRefit.from_result(res, tc, *cl, ev.row_x, bz=ev.bz, v_nominal=ev.v_drift, tgl_ext=tg)
    theta = tpc.calib.nominal_theta(ev.v_drift, device=dev).requires_grad_(True)

    def step():
        theta.grad = None
        chi2, used = tpc.calib_chi2(theta, calib)
        chi2.sum().backward()
        return used

    for _ in range(args.warmup):
        used = step()
    torch.cuda.synchronize()
    u = used.cpu().numpy().astype(bool)
    n_steps = int((np.diff(off)[u] + 1).sum())        # clusters + the vertex of every used track
    stream = torch.cuda.current_stream(dev)
    ev_f = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    f_ms = b_ms = 0.0
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            theta.grad = None
            ev_f[0].record(stream)
            chi2, used = tpc.calib_chi2(theta, calib)
            ev_f[1].record(stream)
            chi2.sum().backward()
            ev_f[2].record(stream)
            torch.cuda.synchronize()
            f_ms += ev_f[0].elapsed_time(ev_f[1])
            b_ms += ev_f[1].elapsed_time(ev_f[2])
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    f_ms /= args.steps
    b_ms /= args.steps
    grad = theta.grad.detach().cpu().numpy()
    # the two kernels alone (no autograd, no status read), CUDA events on the stream
    th_d = theta.detach()
    ones = torch.ones(calib.n_tracks, device=dev)
    c_, used_k, ws_k = calib.forward(th_d, check=False)
    kf = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    fk_ms = bk_ms = 0.0
    for _ in range(args.steps):
        kf[0].record(stream)
        c_, used_k, ws_k = calib.forward(th_d, check=False)
        kf[1].record(stream)
        calib.backward(th_d, ones, used_k, ws_k, check=False)
        kf[2].record(stream)
        torch.cuda.synchronize()
        fk_ms += kf[0].elapsed_time(kf[1])
        bk_ms += kf[1].elapsed_time(kf[2])
    fk_ms /= args.steps
    bk_ms /= args.steps
    calib.check(ws_k)
    # end to end: theta from pinned host memory, chi2 sum and gradient back
    h_theta = theta.detach().cpu().pin_memory()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        with torch.no_grad():
            theta.copy_(h_theta, non_blocking=True)
        theta.grad = None
        chi2, used = tpc.calib_chi2(theta, calib)
        loss = chi2.sum()
        loss.backward()
        float(loss.item())
        theta.grad.cpu()
    e2e_s = (time.perf_counter() - t0) / args.steps
    # the closed-loop fit from the nominal calibration (tpc_calib_fit)
    cal = ev.calib
    fit = None
    torch.cuda.synchronize()
    if not args.no_fit:
        tf0 = time.perf_counter()
        th_fit, rep = calib.fit(tpc.calib.nominal_theta(ev.v_drift, device=dev))
        fit_s = time.perf_counter() - tf0
        th_fit = th_fit.cpu().numpy().astype(np.float64)
        spl_true = np.asarray(cal["spline"]).ravel()
        fit = {"s": round(fit_s, 3), "evaluations": rep["evaluations"], "rounds": rep["rounds"],
               "tracks": rep["tracks"], "dip_angles": rep["anchors"], "f_start": rep["f_start"],
               "f_final": rep["f_final"], "v_fit": th_fit[0], "v_true": cal["v_drift"],
               "v_rel_err": th_fit[0] / cal["v_drift"] - 1.0, "t0_fit_us": th_fit[1], "t0_true_us": cal["t0"],
               "map_rms_err_cm": float(np.sqrt(((th_fit[2:] - spl_true) ** 2).mean())),
               "map_rms_true_cm": float(np.sqrt((spl_true ** 2).mean())),
               "how": "L-BFGS over theta on the GPU chi2 and gradient, prior sigma 0.3 cm on the map, "
                      "dip angles of the matched inner tracks (generator truth smeared by 3e-4)"}
    pk = fma_peak(dev, 32)
    (ms, e2e_s), (steps_all,) = over_ranks(pg, dev, (ms, e2e_s), (float(n_steps),))
    if rank != 0:
        return
    dom, t_dom, fl = (("calib_backward", bk_ms, FLOPS_CALIB_BWD) if bk_ms >= fk_ms
                      else ("calib_forward", fk_ms, FLOPS_CALIB_FWD))
    bw_tf = n_steps * fl / (t_dom * 1e-3) / 1e12
    line = {
        "metric": "calibration chi2 + adjoint gradient, track clusters/s on 1 B300",
        "value": steps_all / (ms / 1e3), "unit": "track clusters/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"{args.collisions}-collision calibration frame (v_drift +0.3 %, t0 200 ns, "
                               "36 x 8 x 8 spline map), theta at the nominal calibration",
                   "tracks": T, "tracks_used": int(u.sum()), "pass_steps": n_steps, "forward_ms": f_ms,
                   "backward_ms": b_ms, "forward_kernel_ms": fk_ms, "backward_kernel_ms": bk_ms,
                   "grad_v_t0": grad[:2].tolist(),
                   "l2": "clusters (160 MB) and checkpoints exceed the 126 MB L2; no flush"},
        "roofline": {"bound": "alu", "stage": dom, "achieved": bw_tf, "peak": pk, "unit": "TFLOP/s",
                     "frac": bw_tf / pk, "traffic": None,
                     "peak_note": "measured binary32 FMA rate (tpc_probe_fma, CUDA events)"},
        "e2e": {"value": steps_all / e2e_s, "unit": "track clusters/s",
                "h2d_bytes_per_step": 4 * theta.numel(), "d2h_bytes_per_step": 4 + 4 * theta.numel()},
        "gpu_launches": 2 * args.steps,
        "clocks": clk.summary(),
    }
    if fit is not None:
        line["fit"] = fit
    if not args.no_cpu_baseline:
        import oracle
        rng = np.random.default_rng(0)
        pick = np.sort(rng.choice(np.nonzero(u)[0], min(3000, int(u.sum())), replace=False))
        n = np.diff(off)
        o_off = np.concatenate([[0], np.cumsum(n[pick])]).astype(np.int32)
        o_cl = np.concatenate([clus[off[k]:off[k + 1]] for k in pick]).astype(np.int32)
        h = lambda x: x[:T].cpu().numpy()  # noqa: E731
        tr = oracle.CalibTracks(h(res.sector)[pick], h(res.x)[pick], h(res.param)[pick], o_off, o_cl,
                                tc.cpu().numpy()[pick], ev.sector, ev.row, ev.y, ev.zt, ev.row_x, bz=ev.bz,
                                v_nom=ev.v_drift)
        th0 = np.zeros(tr_n := oracle.calib_n_theta(36))
        th0[0] = np.float32(ev.v_drift)
        c0 = time.perf_counter()
        _, uo, _ = oracle.calib(tr, th0)
        dt = time.perf_counter() - c0
        steps_o = int((n[pick][uo] + 1).sum())
        line["cpu_baseline"] = {"value": steps_o / dt, "unit": "track clusters/s", "cores": 1, "kind": "oracle",
                                "sample": f"{pick.size} of the used tracks ({steps_o} pass steps), chi2 + gradient "
                                          f"in binary64, {dt:.1f} s, single thread, theta of {tr_n} values"}
    print(json.dumps(line), flush=True)


def roofline(stage, per_step, w, n, pk, n_assigned=None):
    """Roofline of a stage: algorithmic work of one call / its event-timed
    duration (binary32 flops for the Kalman stages, bytes for the others).
    n_assigned: clusters in tracks (the assembly's unit)."""
    t = per_step[stage] / 1e3
    if stage in ("tracklets", "merge", "refit"):
        if stage == "tracklets":
            # algorithmic: one propagation and one update per input cluster
            # (one tracklet pass); executed: the counted steps, back-jumps,
            # empty rows and window candidates included
            algo = n * (FLOPS_PROP + FLOPS_UPDATE)
            flops = w["trk_prop"] * FLOPS_PROP + w["trk_upd"] * FLOPS_UPDATE + w["trk_cand"] * FLOPS_CAND
        elif stage == "merge":
            flops = algo = w["merge_chi2"] * FLOPS_MERGE          # one chi2 per screened pair
        else:
            # three passes of one propagation and one update per track cluster
            flops = w["refit_prop"] * (FLOPS_PROP + FLOPS_UPDATE)
            algo = 3 * (n_assigned if n_assigned is not None else n) * (FLOPS_PROP + FLOPS_UPDATE)
        ach = algo / t / 1e12
        tb = NCU_TRAFFIC_B_PER_CLUSTER.get(stage)
        pk32 = pk.get("fp32_tflops_measured")
        peak = pk32 if pk32 else FP32_PEAK_TFLOPS
        return {"bound": "alu", "stage": stage, "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                "frac": ach / peak, "executed_tflops": flops / t / 1e12, "executed_frac": flops / t / 1e12 / peak,
                "algorithmic_flops_per_launch": algo, "traffic": tb * n if tb is not None else None,
                "peak_note": ("measured binary32 FMA rate (tpc_probe_fma, CUDA events)" if pk32 else
                              "FP32 CUDA-core peak 148 SM x 128 lanes x 2 x 2.032 GHz (derived)")}
    bytes_per = {"prep": 18, "bin": 40, "neighbours": 22, "clean_start": 28}.get(stage, 0)
    hbm = pk.get("hbm_gbs", 6400.0)
    ach = bytes_per * n / t / 1e9
    if stage == "select":        # 24 B per tracklet hit: slot, weight atomic, ownership read
        ach = 24.0 * w.get("trk_upd", 0) / t / 1e9
    elif stage == "assemble" and n_assigned is not None:   # 44 B per assigned cluster
        ach = 44.0 * n_assigned / t / 1e9
    return {"bound": "hbm", "stage": stage, "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
            "traffic": None, "peak_note": "measured" if "hbm_gbs" in pk else "fallback"}


def main():
    args = parse()
    ws, rank, local, pg = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, ws, rank, pg)
    elif args.workload == "stf_batch":
        run_batch(args, ws, rank, local, pg)
    elif args.workload == "calib":
        run_calib(args, ws, rank, local, pg)
    else:
        run_ours(args, ws, rank, local, pg)
    if pg is not None:
        pg.barrier()
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
