/*
 * tpc_track.h -- C ABI of the B300 TPC tracker (libtpcgpu.so).
 *
 * The library reconstructs tracks from TPC clusters on one GPU with the
 * method of Rohr, Gorbunov, Schmidt, Shahoyan, "GPU-based Online Track
 * Reconstruction for the ALICE TPC in Run 3 with Continuous Read-Out":
 *   - section "Tracking", first two bullets: in the seeding phase the drift
 *     time is scaled linearly to z with the average drift velocity and tracks
 *     are assumed to come from the origin; a preliminary fit then finds the
 *     full track and a later fit refines it;
 *   - section "TPC Tracking": the combinatorial part is confined to a
 *     cellular-automaton seeding (NeighboursFinder, NeighboursCleaner,
 *     StartHitsFinder); one hypothesis per track is followed with a Kalman
 *     filter (TrackletConstructor), overlapping candidates are resolved
 *     (TrackletSelector), sector pieces are merged across sector boundaries
 *     and refitted with several fit iterations.
 *
 * Conventions (all entry points):
 *   - Pointers named "device" are CUDA device memory owned by the caller;
 *     the library never frees them and never allocates device memory.
 *   - All work is enqueued on the caller's stream (a cudaStream_t passed as
 *     void*; NULL = legacy default stream).  The tracking calls fork some
 *     independent work (buffer initialisation beside the tracklet stage, the
 *     cluster rejection beside the merger, the refit order beside the
 *     cluster-list fill) onto a side stream of the library and join it back
 *     before its results are used, with events, so the work still completes
 *     in `stream`'s order and a stream capture of the call holds both
 *     branches.  The side stream and its two events are
 *     created at the first call for each (device, caller stream) and kept
 *     until the process exits.
 *   - Return value: TPC_OK (0) or a negative TPC_ERR_* code; no exception
 *     crosses the ABI.  tpc_error_string() names the code.
 *   - Units: cm, microseconds, Tesla, GeV/c.
 *   - Numerics: links, start hits, tracklet hit lists, ownership and merge
 *     decisions are IEEE binary32 with a fixed operation order (bit-exact
 *     against the CPU oracle); the refit is binary32 (optionally binary64 for
 *     the final covariance update and chi2).
 */
#ifndef TPC_TRACK_H
#define TPC_TRACK_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TPC_OK 0
#define TPC_ERR_ARG (-1)       /* invalid argument (null pointer, bad size, bad geometry) */
#define TPC_ERR_CAPACITY (-2)  /* workspace / output capacity too small; see the *_needed fields */
#define TPC_ERR_TIMEOUT (-3)   /* a bounded device-side wait gave up */
#define TPC_ERR_CUDA (-4)      /* a CUDA runtime call failed */
#define TPC_ERR_DATA (-5)      /* a cluster has sector/row out of range or a non-finite coordinate */

/* Stages timed with params.profile (indices into tpc_tracks.stage_ms). */
#define TPC_STAGE_PREP 0        /* time -> z, validation, grid extent */
#define TPC_STAGE_BIN 1         /* per-row grid binning (histogram, scan, scatter) */
#define TPC_STAGE_NEIGHBOURS 2  /* NeighboursFinder */
#define TPC_STAGE_CLEAN_START 3 /* NeighboursCleaner + StartHitsFinder */
#define TPC_STAGE_TRACKLETS 4   /* TrackletConstructor */
#define TPC_STAGE_SELECT 5      /* TrackletSelector */
#define TPC_STAGE_MERGE 6       /* cross-sector merger */
#define TPC_STAGE_ASSEMBLE 7    /* merged cluster lists and assignments */
#define TPC_STAGE_REFIT 8       /* Kalman refit */
#define TPC_STAGE_ATTACH 9      /* track-based cluster attachment (when tpc_tracks.cl_flags is set) */
#define TPC_N_STAGES 10

/* Cluster attachment flags (tpc_tracks.cl_flags), paper section "TPC Data
 * Compression", cluster rejection: */
#define TPC_CL_ATTACHED 1   /* attached to a track (assign >= 0) */
#define TPC_CL_ADJACENT 2   /* not attached, inside the tube of a track (tpc_tracks.adjacent) */
#define TPC_CL_PROTECTED 4  /* attached to a good track or inside the tube of one */
#define TPC_CL_REMOVE 8     /* attached or adjacent and not protected: to be removed */

/* Method parameters.  tpc_params_default() fills the values of the reading
 * used throughout (seeding windows, straightness cut, cluster errors,
 * priors, following window and cuts, selector and merger cuts). */
typedef struct {
    float dy_link, dz_link;      /* NeighboursFinder windows (cm) around y*x_other/x_mid and z */
    float s_max_link;            /* straightness cut: (chord deviation)^2 < s_max_link (cm^2) */
    float sigma_y, sigma_z;      /* cluster position errors (cm) */
    float c0_snp, c0_tgl, c0_qpt;/* prior variances of sin(phi), tan(lambda), q/pT */
    float win_nsigma, win_min, win_max; /* following window clamp(n*sigma, min, max) (cm) */
    float chi2_cut;              /* per-update chi2 cut while following (2 dof) */
    int32_t max_miss;            /* stop following after this many consecutive empty rows */
    int32_t min_hits;            /* tracklets shorter than this are dropped */
    int32_t min_owned;           /* selector: owned hits a tracklet needs */
    float edge_margin;           /* stop following when |y| > x tan(10 deg) + margin (cm) */
    float merge_dz;              /* merger: |z_B - z_A| window before the chi2 test (cm) */
    float merge_chi2;            /* merger: chi2 (5 dof) cut */
    int32_t refit_passes;        /* refit passes, alternating inward / outward (odd: ends inward) */
    float refit_inflate;         /* each pass restarts with the previous sin(phi), tan(lambda), q/pT
                                    covariance times this factor (y, z from the first measurement) */
    /* acceleration structure and capacities (do not change results) */
    float z_cell;                /* minimum grid cell length in z (cm, >= 0.25; default 5): the length
                                    grows so that at most max_z_cells cells cover a frame's z extent.
                                    Every search visits all cells its window overlaps, so any cell
                                    size gives the same results. */
    int32_t max_z_cells;         /* maximum grid z-cells per pad row */
    int32_t y_bins;              /* grid y-bins per z-cell, 1..64 (default 16): each pad row's width
                                    split evenly */
    int32_t tracklets_per_1k;    /* tracklet capacity per 1000 clusters (minimum 4096 total) */
    int32_t queue_blocks_per_sm; /* TrackletConstructor work-queue width: blocks per SM taking start
                                    hits from the queue (0: as many as the capacity needs, up to 16) */
    int32_t fp64_final;          /* final refit pass in binary64: 0 off; 1 covariance (Joseph form) and chi2 of
                                    every track in binary64; 2 the binary64 Joseph update for long looping
                                    low-pT tracks only (|q/pT| >= 5 c/GeV after the earlier passes, or more
                                    clusters than pad rows), the binary32 update for the others, chi2 of
                                    every track in binary64.  cov64 holds the final covariance either way. */
    int32_t profile;             /* 1: record CUDA events on the stream at stage boundaries (tpc_tracks.stage_ms) */
    int32_t packed_links;        /* 1: the link pass reads y, z as 16-bit packed fields of a fixed-point
                                    coordinate with step 2^-8 cm (decoded relative to the middle hit), i.e.
                                    it sees both rounded to the nearest 1/256 cm; other stages see full
                                    precision.  Needs z-cells under 60 cm (TPC_ERR_CAPACITY otherwise). */
    int32_t merge_pairs_per_1k;  /* merger: capacity of the list of screened candidate pairs, per 1000
                                    tracklet slots (default 4000; >= 0).  Beyond it the merger evaluates
                                    the pairs of each segment end directly (same result, slower); 0
                                    always does. */
    float tube_radius;           /* cluster attachment: tube radius around each track (cm, 0..20; default
                                    1.5).  The tube follows each sector piece of a track: its
                                    TrackletConstructor state at its innermost hit (binary32, after all
                                    of its hits) is propagated row by row through the rows of the
                                    piece's hits, stopping at the first refused step; a cluster of the
                                    piece's sector on a traced row lies in the tube when
                                    dy^2 + dz^2 < R^2 from the traced point. */
    float pt_min_physics;        /* cluster attachment: tracks with pT below this (GeV/c; default 0.05)
                                    are not good (not used for physics).  A track's pT, here and for
                                    the adjacency order, is 1 / |q/pT| of the inner-end state of its
                                    innermost piece: good when |q/pT| <= 1 / pt_min_physics (binary32;
                                    0: every track is good). */
    float outlier_chi2;          /* cluster rejection before the refit (section "TPC Tracking": the fit
                                    rejects clusters; default 25, 0: off).  Each kept tracklet's state at
                                    its innermost hit (binary32, after all of its hits) is carried with the
                                    decision-path helix step up through the rows of its hits; an owned hit
                                    with dy^2/sigma_y^2 + dz^2/sigma_z^2 > outlier_chi2 to it leaves the
                                    track's cluster list, the refit and the assignment (assign = -1),
                                    unless fewer than 5 owned hits of the tracklet would remain.  A refused
                                    step ends the check of that tracklet.  Bit-exact on any hardware that
                                    rounds each operation. */
    float looper_qpt_min;        /* looper legs: tracks with |q/pT| >= this (c/GeV, default 5: pT below
                                    200 MeV/c) are looper-leg candidates (see tpc_tracks.looper_group) */
} tpc_params;

/* Detector geometry (host memory). */
typedef struct {
    int32_t n_sectors;           /* 36 (sectors 0..17 at z > 0, 18..35 at z < 0) or 1 (one wedge, both z signs) */
    int32_t n_rows;              /* pad rows, 3..255 */
    const float *row_x;          /* host [n_rows]: local x of each pad-row plane (cm), increasing */
    float z_max;                 /* drift length (cm) */
    int32_t continuous;          /* 0: clusters carry z (cm); 1: drift time (us), z = s (z_max - v_drift t) */
} tpc_geometry;

/* Input clusters: device SoA, n entries each. */
typedef struct {
    int32_t n;
    const uint8_t *sector;       /* device [n] */
    const uint8_t *row;          /* device [n] */
    const float *y;              /* device [n] sector-local y (cm) */
    const float *zt;             /* device [n] z (cm) or drift time (us) */
} tpc_clusters;

/* Outputs: device arrays allocated by the caller with the stated capacities.
 * Tracks are ordered by the input index of the start hit of their innermost
 * sector piece; each track's state is at its innermost cluster, in the frame
 * of that cluster's sector (alpha = (sector mod 18) * 20 + 10 degrees). */
typedef struct {
    int32_t capacity_tracks;     /* rows available in the per-track arrays */
    int32_t capacity_clusters;   /* entries available in clus_index */
    int32_t *sector;             /* [T] sector of the output frame */
    float *x;                    /* [T] local x of the output state (cm) */
    float *param;                /* [T][5] y, z, sin(phi), tan(lambda), q/pT */
    float *cov;                  /* [T][15] lower-triangular covariance, row-major packed */
    float *chi2;                 /* [T] chi2 of the last refit pass */
    int32_t *ndf;                /* [T] 2 * nclus - 5 */
    int32_t *status;             /* [T] 0 ok; 1 refit propagation failed (state at the failure point) */
    int32_t *nclus;              /* [T] clusters of the track */
    int32_t *clus_offset;        /* [T+1] offsets into clus_index */
    int32_t *clus_index;         /* [capacity_clusters] input cluster indices, inner -> outer */
    int32_t *assign;             /* [n] track index of each input cluster, -1 if unassigned */
    int32_t *frame;              /* nullable [T]: time frame of each track (tpc_track_batched) */
    double *cov64;               /* nullable [T][15]: binary64 covariance when fp64_final */
    double *chi2_64;             /* nullable [T]: binary64 chi2 when fp64_final */
    /* nullable intermediate results, indexed by input cluster (parity checks) */
    float *z;                    /* [n] z after the time -> z conversion */
    int32_t *link_up_raw, *link_dn_raw;   /* [n] NeighboursFinder best pair (input index or -1) */
    int32_t *link_up, *link_dn;           /* [n] after NeighboursCleaner */
    uint8_t *is_start;                    /* [n] StartHitsFinder flag */
    /* nullable cluster attachment (paper, section "TPC Data Compression"); the stage runs when
     * cl_flags is set.  A cluster attached to no track is adjacent to the track of highest pT
     * (smallest |q/pT|, then the smaller track index) whose tube holds it. */
    uint8_t *cl_flags;                    /* [n] TPC_CL_* flags */
    int32_t *adjacent;                    /* [n] adjacent track index, -1 if not adjacent (nullable) */
    /* nullable looper legs (paper, sections "Introduction" and "TPC Data Compression": a low-pT particle
     * leaves several legs; the stage runs when either array, or cl_flags, is set).  Tracks whose
     * innermost piece has |q/pT| >= looper_qpt_min are candidates; two candidates of one time frame are
     * legs of one particle when their circles in the transverse plane agree (centre within
     * 2 s + 2 cm, radius within 2 s + 1 cm, s the combined radius uncertainty from the q/pT variance;
     * legs known to worse than 5 cm are not grouped), |tan(lambda)| within 0.05, and their z
     * difference is the helix's z advance over the turning angle between them plus whole turns
     * (at most 10) within 3 cm + the radius uncertainty's share; all binary32 on the decision path.
     * With cl_flags, a secondary leg (looper_leg >= 1) is not a good track (the paper's removal
     * category of secondary legs of loopers below 200 MeV/c). */
    int32_t *looper_group;                /* [T] smallest track of the legs of one particle, -1 alone */
    int32_t *looper_leg;                  /* [T] leg number in ascending s z (0 = the earliest leg of the
                                             drift, s = +1 on the A side, -1 on the C side), -1 alone */
    /* filled on return (host-visible fields of this struct) */
    int32_t n_tracks;
    int32_t n_tracklets;
    int32_t n_segments;
    int64_t tracklets_needed;    /* on TPC_ERR_CAPACITY */
    int64_t tracks_needed;
    int64_t clusters_needed;
    int32_t n_launches;          /* kernels this call launched */
    float stage_ms[TPC_N_STAGES];/* with params.profile: device time of each stage (see TPC_STAGE_*) */
    int64_t work[5];             /* with params.profile: tracklet propagations, tracklet updates, grid
                                    candidates examined while following, refit propagations, merger
                                    chi2 evaluations */
    int32_t n_rejected;          /* clusters the rejection before the refit took out of their tracks
                                    (tpc_track, tpc_track_batched) */
    /* nullable input: a cudaEvent_t (passed as void*) that the tracking calls record on `stream`
     * once every input of the track refit is complete, just before the refit (after it only the
     * refit and the optional looper-leg and attachment stages run).  A caller streaming frames
     * through separate workspaces and outputs may let the next frame's chain wait on this event
     * instead of on the end of the call: the next frame's first stages then run beside this
     * frame's refit, whose last long tracks keep few SMs busy.  Not recorded when the call fails
     * before the refit. */
    void *refit_event;
} tpc_tracks;

#define TPC_MAX_CLUSTERS 2145386495LL   /* INT32_MAX - 2^21 */

/* Fill *p with the default parameters.  Returns TPC_OK, or TPC_ERR_ARG for p == NULL. */
int tpc_params_default(tpc_params *p);

/* Bytes of device workspace tpc_track needs for n_clusters clusters with
 * these parameters and geometry; written to *bytes.  n_clusters is at most
 * TPC_MAX_CLUSTERS (cluster indices are int32).  Errors: TPC_ERR_ARG. */
int tpc_workspace_size(const tpc_params *p, const tpc_geometry *g, int64_t n_clusters, size_t *bytes);

/* Track one event or continuous read-out frame (sections "Tracking" and
 * "TPC Tracking").  Inputs: cluster SoA (device), magnetic field bz (T)
 * along z, average drift velocity v_drift (cm/us, used when
 * g->continuous).  workspace: device buffer of ws_bytes >= tpc_workspace_size.
 * The call enqueues the whole chain on `stream`, then waits for it
 * (one device->host read of the counts) and fills out->n_tracks etc.
 * Errors: TPC_ERR_ARG (bad arguments), TPC_ERR_DATA (bad cluster),
 * TPC_ERR_CAPACITY (workspace or outputs too small: *_needed fields set),
 * TPC_ERR_CUDA.  Output arrays beyond n_tracks are unspecified. */
int tpc_track(const tpc_params *p, const tpc_geometry *g, float bz, float v_drift,
              const tpc_clusters *cl, void *workspace, size_t ws_bytes, tpc_tracks *out,
              void *stream);

/* Workspace for tpc_track_batched / tpc_prepare: n_clusters in total over
 * n_frames frames (1 .. 4096).  Errors: TPC_ERR_ARG. */
int tpc_workspace_size_batched(const tpc_params *p, const tpc_geometry *g, int64_t n_clusters, int32_t n_frames,
                               size_t *bytes);

/* Track a batch of independent time frames (sub-time-frames of uneven sizes)
 * in one pass: every stage is one launch over all frames.  The clusters of
 * frame k are entries frame_offsets[k] .. frame_offsets[k+1]-1 of `cl`
 * (host array, n_frames + 1 entries, frame_offsets[0] = 0,
 * frame_offsets[n_frames] = cl->n).  Each frame is tracked exactly as
 * tpc_track would track it alone (same links, tracklets, tracks and fits,
 * with input indices offset by frame_offsets[k]); the tracks of all frames
 * come in one list ordered by input index, out->frame (if not null) gives the
 * frame of each track.  Workspace: tpc_workspace_size_batched.  Errors as
 * tpc_track. */
int tpc_track_batched(const tpc_params *p, const tpc_geometry *g, float bz, float v_drift, const tpc_clusters *cl,
                      int32_t n_frames, const int32_t *frame_offsets, void *workspace, size_t ws_bytes,
                      tpc_tracks *out, void *stream);

/* Write the per-row tables, the frame offsets and the workspace header that
 * tpc_track_async reads (pageable host copies; not capturable).  Call once
 * per (workspace, geometry, parameters, frame offsets); synchronises the
 * stream.  Errors: TPC_ERR_ARG, TPC_ERR_CAPACITY, TPC_ERR_CUDA. */
int tpc_prepare(const tpc_params *p, const tpc_geometry *g, int32_t n_clusters, int32_t n_frames,
                const int32_t *frame_offsets, void *workspace, size_t ws_bytes, void *stream);

/* Bytes of pinned host staging that tpc_prepare_async needs for n_frames
 * frames.  Errors: TPC_ERR_ARG. */
int tpc_prepare_staging_size(int32_t n_frames, size_t *bytes);

/* tpc_prepare without host synchronisation, capturable in a CUDA graph: the
 * tables, offsets and header are written into host_staging (caller-owned
 * page-locked host memory of tpc_prepare_staging_size bytes, which must stay
 * valid and unchanged while the copies may run, i.e. for the lifetime of a
 * graph that captured them) and copied from there on `stream`.  Lets one
 * workspace serve several frame groups in turn: prepare group A, track A,
 * prepare group B, track B on the same stream.  Errors: TPC_ERR_ARG,
 * TPC_ERR_CAPACITY, TPC_ERR_CUDA. */
int tpc_prepare_async(const tpc_params *p, const tpc_geometry *g, int32_t n_clusters, int32_t n_frames,
                      const int32_t *frame_offsets, void *host_staging, size_t staging_bytes, void *workspace,
                      size_t ws_bytes, void *stream);

/* Enqueue the whole chain (as tpc_track_batched) without any host
 * synchronisation or host copy, so that the call can be captured in a CUDA
 * graph and replayed.  Requires a prior tpc_prepare or tpc_prepare_async on
 * the same workspace with the same n_clusters and n_frames.  Of the
 * host-visible fields of *out only n_launches (kernels enqueued) is filled;
 * instead dev_counts (device int32[6]) receives n_tracks, n_tracklets,
 * n_segments, an error code (0, TPC_ERR_DATA or TPC_ERR_CAPACITY), clusters
 * in tracks and start hits found.  params.profile
 * is ignored.  Errors detected on the host: TPC_ERR_ARG, TPC_ERR_CAPACITY,
 * TPC_ERR_CUDA. */
int tpc_track_async(const tpc_params *p, const tpc_geometry *g, float bz, float v_drift, const tpc_clusters *cl,
                    int32_t n_frames, void *workspace, size_t ws_bytes, tpc_tracks *out, int32_t *dev_counts,
                    void *stream);

/* Export the tracklets of the last tpc_track call that used `workspace`
 * (TrackletConstructor and TrackletSelector results, for parity checks).
 * Host outputs, rows in ascending start-hit input index:
 *   start[nt]  input index of the start hit;  nhits[nt];  kept[nt] (0/1);
 *   hits[nt * hits_stride]  input indices in ascending row, unused entries -1
 *                           (hits_stride >= n_rows);
 *   top[nt * 21], bot[nt * 21]  x, p[5], c[15] right after the outermost
 *                           fitted hit / at the innermost hit.
 * capacity = rows available in the host arrays (0 with null arrays: only
 * query the count); *nt_out receives the tracklet count.  Synchronises `stream`, then reads the workspace with blocking copies.
 * Errors: TPC_ERR_ARG (null pointer, workspace not written by tpc_track,
 * hits_stride too small), TPC_ERR_CAPACITY (capacity < tracklet count; *nt_out
 * is set), TPC_ERR_CUDA. */
int tpc_export_tracklets(const void *workspace, int32_t capacity, int32_t hits_stride, int32_t *start,
                         int32_t *nhits, uint8_t *kept, int32_t *hits, float *top, float *bot,
                         int32_t *nt_out, void *stream);

/* Seeding without any allocation: time -> z, per-row grid binning,
 * NeighboursFinder and NeighboursCleaner for at most
 * TPC_LINKS_STATIC_MAX_CLUSTERS clusters, with all scratch memory in a fixed
 * device array inside the library.  The paper has no counterpart; this entry
 * point exists for callers that cannot allocate device memory: a host thread
 * that must not block on the allocator (cudaMalloc can synchronise the
 * device) while other streams run, or an embedding that forbids cudaMalloc
 * after start-up (a plug-in inside a host framework that owns all device
 * memory).  They still pass their own device inputs and outputs; nothing else
 * is allocated, by them or by the library.
 *   - The call copies the row table and plane offsets from host memory,
 *     reads the data-error flag back and ends by synchronising `stream`: it
 *     must not be made while `stream` (or the legacy stream) is being
 *     captured into a CUDA graph.
 *   - Outputs (device, indexed by input cluster): link_up, link_dn (cleaned
 *     links, input index or -1), is_start (nullable, 0/1).  They equal the
 *     link_up / link_dn / is_start outputs of tpc_track on the same input.
 *   - Limit: n <= TPC_LINKS_STATIC_MAX_CLUSTERS; larger inputs return
 *     TPC_ERR_CAPACITY without touching the GPU.  n_sectors * n_rows <= 9180.
 *   - The fixed array holds TPC_LINKS_STATIC_SCRATCH_BYTES on every GPU that
 *     loads the library, until the process exits.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress); make that first call before any stream capture.
 *   - Every call uses the same array and leaves its contents behind (the
 *     call clears what must start at zero).  Calls that overlap on the GPU --
 *     on two streams, or from two host threads -- race on it: serialise them.
 * Errors: TPC_ERR_ARG, TPC_ERR_CAPACITY, TPC_ERR_DATA, TPC_ERR_CUDA. */
#define TPC_LINKS_STATIC_MAX_CLUSTERS 262144
#define TPC_LINKS_STATIC_SCRATCH_BYTES 14417664
int tpc_links_static(const tpc_params *p, const tpc_geometry *g, float v_drift, const tpc_clusters *cl,
                     int32_t *link_up, int32_t *link_dn, uint8_t *is_start, void *stream);

/* Human-readable name of a return code (static string). */
const char *tpc_error_string(int code);

#ifdef __cplusplus
}
#endif
#endif
