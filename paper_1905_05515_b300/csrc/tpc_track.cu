// tpc_track.cu -- B300 TPC tracker: binning, cellular-automaton seeding,
// tracklet construction and selection, cross-sector merging, track assembly
// and the C-ABI entry points (include/tpc_track.h).
//
// Every stage runs over a batch of independent time frames at once: a pad-row
// plane is identified by (frame, sector, row), each frame has its own z grid,
// and merges stay inside a frame, so a batch gives exactly the results of the
// frames processed one by one.  A single frame is the batch of one.
//
// Compiled with -fmad=false: every binary32 decision (links, start hits,
// tracklet hits, ownership, merges) follows the fixed operation order of the
// method's specification and is bit-identical to any IEEE implementation of
// it.
#include "tpc_dev.cuh"
#include "tpc_track.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <utility>
#include <vector>

using namespace tpc;

namespace {

constexpr int SCAN_BLOCK = 1024;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_TILE = SCAN_BLOCK * SCAN_ITEMS;
constexpr int MAX_MERGE_CELLS = 4096;
constexpr int MAX_CHAIN = 36;
constexpr int LEN_BUCKETS = 512;        // refit ordering: cluster counts above 511 share a bucket
constexpr int MAX_FRAMES = 4096;
// Per-plane bucket counters: PSPLIT consecutive counters per plane (the
// cluster attachment spreads its reservations over them; the binning counts
// each block's clusters per plane in shared memory and reserves them in the
// plane's first counter), so a plane's entries stay one range.  Planes x
// PSPLIT < 2^32 (36 x 255 x MAX_FRAMES x 16).
constexpr int PSPLIT = 16;
// grid cell budget of a batch beyond the first frame's max_z_cells: two
// cells per cluster (a 50-collision frame occupies about 0.6 clusters per
// cell at the default cell size), never more than max_z_cells per frame
constexpr int64_t CELLS_PER_CLUSTER = 2;
constexpr float Y_MARGIN = 1.0f;       // y-bin range beyond the sector edge (cm)
constexpr uint32_t WS_MAGIC = 0x54504332u;

inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// ---------------------------------------------------------------------------
// workspace layout (byte offsets from the workspace base)
// ---------------------------------------------------------------------------
struct Layout {
    uint32_t magic;
    int32_t n, ns, nr, np, nzmax, ntcap, mnzmax, ny, nframes;
    int64_t ncells;                    // grid cell capacity (all frames)
    size_t hdr, frame, fgrid, offsets, rowtab, zlin, cfr, cell, slot, cstart, scan, sc, yzp;
    size_t upr, dnr, up, dn, starts;
    size_t pbuf, pstart;        // binning: plane-ordered records (aliases the links), plane starts
    size_t t_start, t_id, t_nhits, t_nup, t_hits, t_top, t_bot, hitw, t_kept, t_own, ownmask, segoff, segrank, t_state;
    size_t seg, keyb, keyt, slotb, slott, cntb, cntt, byb, byt, recb, rect;
    size_t bnext, bprev, snext, sprev, bad, next2, prev2, mpair, mpc2, bestA, bestB;
    int64_t mpcap;              // merger pair list capacity
    size_t headmark, tcount, thead, ttail, tcl, lencnt, order, aprot, acur;
    size_t lcand, lpar, lcnt, llist, lgrp, lleg, lbin, lsorted, lcur, tgood;   // looper legs, track goodness
    size_t total;
};

int64_t scan_aux_elems(int64_t n)
{
    int64_t s = 0;
    while (n > 1) {
        n = (n + SCAN_TILE - 1) / SCAN_TILE;
        s += n + 1;
    }
    return s + 16;
}

// y-bins per z-cell (the searches visit whatever bins a window overlaps, so
// any count works; the grid grows with it)
constexpr int MAX_YBINS = 64;
constexpr int LOOP_G = 48;              // looper candidates: LOOP_G x LOOP_G cells of their circle centres
constexpr int LOOP_NBIN = LOOP_G * LOOP_G;   // per frame
int effective_ybins(const tpc_params* p, const tpc_geometry*) { return std::max(1, std::min(p->y_bins, MAX_YBINS)); }

// per-row binary32 tables: X, X[r+1]/X[r], X[r-1]/X[r],
// (X[r]-X[r-1]) / (X[r+1]-X[r-1]), then the y-bin origin and inverse width
void fill_rowtab(float* tab, const tpc_geometry* g, int ny)
{
    memset(tab, 0, sizeof(float) * ROWTAB * 256);
    const float* X = g->row_x;
    for (int r = 0; r < g->n_rows; r++) {
        volatile float xr = X[r];
        tab[r * ROWTAB] = xr;
        if (r >= 1 && r + 1 < g->n_rows) {
            volatile float a = X[r + 1] / X[r];
            volatile float b = X[r - 1] / X[r];
            volatile float num = X[r] - X[r - 1];
            volatile float den = X[r + 1] - X[r - 1];
            volatile float w = num / den;
            tab[r * ROWTAB + 1] = a;
            tab[r * ROWTAB + 2] = b;
            tab[r * ROWTAB + 3] = w;
        }
        const float half = xr * TAN10 + Y_MARGIN;
        tab[r * ROWTAB + 4] = -half;
        tab[r * ROWTAB + 5] = (float)ny / (2.0f * half);
    }
}

Layout make_layout(const tpc_params* p, const tpc_geometry* g, int64_t n, int nframes)
{
    Layout L;
    memset(&L, 0, sizeof(L));
    L.magic = WS_MAGIC;
    L.n = (int32_t)n;
    L.ns = g->n_sectors;
    L.nr = g->n_rows;
    L.np = L.ns * L.nr;
    L.nzmax = p->max_z_cells;
    L.ny = effective_ybins(p, g);
    L.nframes = nframes;
    {
        const int64_t per = (int64_t)L.np * L.ny;
        const int64_t extra_z = nframes > 1 ? (CELLS_PER_CLUSTER * n + per - 1) / per + nframes : 0;
        const int64_t zcells = std::min<int64_t>((int64_t)L.nzmax * nframes, L.nzmax + extra_z);
        L.ncells = std::min<int64_t>(per * zcells, ((int64_t)UINT32_MAX - 1) / per * per);
    }
    int64_t cap = std::max<int64_t>(4096, (n * (int64_t)p->tracklets_per_1k) / 1000);
    // at most 2^30 slots: the merger's pair list keeps a record index in 30 bits
    L.ntcap = (int32_t)std::min<int64_t>({cap, std::max<int64_t>(n, 4096), (int64_t)1 << 30});
    L.mnzmax = MAX_MERGE_CELLS;
    const int64_t N = std::max<int64_t>(n, 1);
    const int64_t T = L.ntcap;
    const int64_t mcells = (int64_t)nframes * L.ns * L.mnzmax;
    int64_t scan_max = std::max({L.ncells + 1, N + 1, T + 1, mcells + 1, (int64_t)nframes * L.np * PSPLIT + 1});
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t r = o; o = align_up(o + std::max<size_t>(bytes, 1), 256); return r; };
    L.hdr = take(sizeof(Layout));
    L.frame = take(sizeof(Frame));
    L.fgrid = take(sizeof(FrameGrid) * nframes);
    L.offsets = take(sizeof(int32_t) * (nframes + 1));
    L.rowtab = take(sizeof(float) * ROWTAB * 256);
    L.zlin = take(4 * N);
    L.cfr = take(2 * N);
    L.cell = take(4 * N);
    L.slot = take(4 * N);
    L.cstart = take(4 * (L.ncells + 1));
    L.scan = take(4 * scan_aux_elems(scan_max));
    L.sc = take(16 * N);        // sorted clusters: y, z, input index, plane
    L.yzp = p->packed_links ? take(4 * N) : 0;
    // the four link arrays, one 16-byte-per-cluster block: before the links
    // exist it holds the plane-ordered cluster records of the binning
    L.upr = take(16 * N);
    L.dnr = L.upr + 4 * N;
    L.up = L.dnr + 4 * N;
    L.dn = L.up + 4 * N;
    L.pbuf = L.upr;
    L.pstart = take(4 * ((size_t)nframes * L.np * PSPLIT + 1));
    L.starts = take(4 * T);
    L.t_start = take(4 * T);
    L.t_id = take(4 * T);
    L.t_nhits = take(4 * T);
    L.t_nup = take(4 * T);
    L.t_hits = take(4 * T * (size_t)L.nr);
    L.t_top = take(4 * T * NST);
    L.t_bot = take(4 * T * NST);
    L.hitw = take(8 * N);
    L.t_kept = take(T);
    L.t_own = take(4 * T);      // hits each tracklet owns after the selector
    L.ownmask = take(4 * T * (size_t)((L.nr + 31) / 32));   // [word][tracklet]: which of its hits it owns
    L.t_state = take(4 * T * (size_t)(NST + 4));   // tracklet state between the constructor's passes
    L.seg = take(4 * T);
    L.segoff = take(4 * T);     // per segment: first cluster within its track
    L.segrank = take(4 * T);    // per segment: its track (-1: in no track)
    L.keyb = take(4 * T);
    L.keyt = take(4 * T);
    L.slotb = take(4 * T);
    L.slott = take(4 * T);
    L.cntb = take(4 * (mcells + 1));
    L.cntt = take(4 * (mcells + 1));
    L.byb = take(4 * T);
    L.byt = take(4 * T);
    L.recb = take(32 * T);      // merge-grid order: inner-end (z, tan lambda, q/pT, their variances, id)
    L.rect = take(32 * T);      // merge-grid order: outer-end record
    L.mpcap = T * (int64_t)p->merge_pairs_per_1k / 1000;   // screened merge pairs (about T / 3 measured)
    L.mpair = take(8 * L.mpcap);
    L.mpc2 = take(4 * L.mpcap);
    L.bestA = take(8 * T);
    L.bestB = take(8 * T);
    L.bnext = take(4 * T);
    L.bprev = take(4 * T);
    L.snext = take(4 * T);
    L.sprev = take(4 * T);
    L.bad = take(T);
    L.next2 = take(4 * T);
    L.prev2 = take(4 * T);
    L.headmark = take(4 * (N + 1));
    L.tcount = take(4 * (T + 1));
    L.thead = take(4 * T);
    L.ttail = take(4 * T);
    L.tcl = take(16 * N);       // track clusters in track order: y, z, row x, sector
    L.lencnt = take(4 * (LEN_BUCKETS + 1));
    L.order = take(4 * T);      // refit order
    L.aprot = take(N);          // cluster attachment: inside a good track's tube
    L.acur = take(4 * ((size_t)nframes * L.np * PSPLIT + 1));   // cluster attachment: bucket fill cursors
    // looper legs: candidate records, union-find parents, group counts and
    // member lists, group / leg scratch, radius-bin counts and order
    L.lcand = take(48 * T);
    L.lpar = take(4 * T);
    L.lcnt = take(4 * (T + 1));
    L.llist = take(4 * T);
    L.lgrp = take(4 * T);
    L.lleg = take(4 * T);
    L.lbin = take(4 * ((size_t)nframes * LOOP_NBIN + 1));
    L.lsorted = take(4 * T);
    L.lcur = take(4 * (std::max<int64_t>(T, (int64_t)nframes * LOOP_NBIN) + 1));   // fill cursors
    L.tgood = take(T);          // cluster attachment: good tracks
    L.total = o;
    return L;
}

template <typename T>
inline T* at(void* ws, size_t off) { return reinterpret_cast<T*>(static_cast<char*>(ws) + off); }

// Cluster indices are int32 and the grid-stride loops step an int index by at
// most 148 * 16 blocks x 256 threads (grid_for's cap): with n below
// INT32_MAX - 2^21 the index after the last step still fits.
constexpr int64_t MAX_CLUSTERS = (int64_t)INT32_MAX - (1 << 21);
static_assert(MAX_CLUSTERS == TPC_MAX_CLUSTERS, "limit stated in tpc_track.h");

int grid_for(int64_t n, int block)
{
    int64_t g = (n + block - 1) / block;
    return (int)std::max<int64_t>(1, std::min<int64_t>(g, 148 * 16));
}

// ---------------------------------------------------------------------------
// exclusive scan (in place) of a[0..n], n+1 entries: a[n] (zero on entry)
// receives the total.  With n_dev, the entries beyond *n_dev are left alone
// (the launch covers the host-side bound n).
// ---------------------------------------------------------------------------
__global__ void k_scan_tiles(uint32_t* a, int64_t n1, const unsigned* n_dev, uint32_t* sums)
{
    __shared__ uint32_t sh[SCAN_BLOCK];
    const int64_t lim = n_dev ? (int64_t)(*n_dev) + 1 : n1;
    const int64_t tile0 = (int64_t)blockIdx.x * SCAN_TILE;
    if (tile0 >= lim) {
        if (threadIdx.x == 0) sums[blockIdx.x] = 0u;
        return;
    }
    const int64_t base = tile0 + (int64_t)threadIdx.x * SCAN_ITEMS;
    uint32_t v[SCAN_ITEMS];
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; k++) {
        v[k] = (base + k < lim) ? a[base + k] : 0u;
        s += v[k];
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int off = 1; off < SCAN_BLOCK; off <<= 1) {
        uint32_t t = threadIdx.x >= (unsigned)off ? sh[threadIdx.x - off] : 0u;
        __syncthreads();
        sh[threadIdx.x] += t;
        __syncthreads();
    }
    uint32_t run = sh[threadIdx.x] - s;   // exclusive prefix of this thread
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; k++) {
        if (base + k < lim) a[base + k] = run;
        run += v[k];
    }
    if (threadIdx.x == SCAN_BLOCK - 1) sums[blockIdx.x] = sh[SCAN_BLOCK - 1];
}

__global__ void k_scan_add(uint32_t* a, int64_t n1, const unsigned* n_dev, const uint32_t* sums)
{
    const int64_t lim = n_dev ? (int64_t)(*n_dev) + 1 : n1;
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    if (base >= lim) return;
    const uint32_t add = sums[blockIdx.x];
    for (int k = threadIdx.x; k < SCAN_TILE; k += SCAN_BLOCK)
        if (base + k < lim) a[base + k] += add;
}

int g_launches = 0;   // kernels launched by the current call (host thread)

void scan_u32(uint32_t* a, int64_t n, uint32_t* aux, cudaStream_t st, const unsigned* n_dev = nullptr)
{
    const int64_t tiles = (n + 1 + SCAN_TILE - 1) / SCAN_TILE;
    k_scan_tiles<<<(unsigned)tiles, SCAN_BLOCK, 0, st>>>(a, n + 1, n_dev, aux);
    g_launches++;
    if (tiles > 1) {
        scan_u32(aux, tiles - 1, aux + tiles + 1, st);   // exclusive scan of the tile sums
        k_scan_add<<<(unsigned)tiles, SCAN_BLOCK, 0, st>>>(a, n + 1, n_dev, aux);
        g_launches++;
    }
}

__global__ void k_zero_cells(uint32_t* a, const Frame* __restrict__ f)
{
    const int64_t n1 = (int64_t)f->total_cells + 1;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n1; i += (int64_t)gridDim.x * blockDim.x)
        a[i] = 0u;
}

// stage events for params.profile (created once per process, per device)
struct StageEvents {
    int device = -1;
    cudaEvent_t ev[TPC_N_STAGES + 1];
};
StageEvents g_events;

// ---------------------------------------------------------------------------
// a1 + a2: time -> z, validation, folded-z extrema per frame; grid
// ---------------------------------------------------------------------------
__global__ void k_init_frame(Frame* f, FrameGrid* fg, int nframes)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        memset(f, 0, sizeof(Frame));
        f->zmin_key = 0xFFFFFFFFu;
        f->zmax_key = 0u;
    }
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nframes; i += gridDim.x * blockDim.x) {
        fg[i].zmin_key = 0xFFFFFFFFu;
        fg[i].zmax_key = 0u;
    }
}

__device__ __forceinline__ float fold(float z, int s, int ns) { return (ns == 36 && s >= 18) ? -z : z; }

// blockIdx.y = frame; the blocks of one frame stride over its cluster range
// RANK: each block takes one contiguous chunk of its frame's clusters and
// also ranks every cluster among the clusters of its plane (frame, sector,
// row): first within the block, by counters of the frame's planes in shared
// memory, then the block reserves each plane's count in the plane's first
// global counter with one atomic and adds the reservation to its clusters'
// ranks (the order of the atomics: any).  A block of a large frame touches
// each plane once, so a frame of n clusters costs planes x blocks global
// atomics instead of n.  Without RANK: a grid-stride pass with no ranks.
constexpr int PREP_RANK_BLOCK = 1024;
constexpr int PREP_U = 4;

template <bool RANK>
__global__ void __launch_bounds__(RANK ? PREP_RANK_BLOCK : 256)
k_prep(const int32_t* __restrict__ offsets, const uint8_t* __restrict__ sector,
       const uint8_t* __restrict__ row, const float* __restrict__ y, const float* __restrict__ zt,
       int ns, int nr, int continuous, float zmax, float vdrift, float* __restrict__ zlin,
       uint16_t* __restrict__ cfr, Frame* f, FrameGrid* fg, int np, uint32_t* __restrict__ pcount,
       uint32_t* __restrict__ prank)
{
    extern __shared__ uint32_t pc_sh[];     // RANK: [np] the block's count, then its reservation, per plane
    const int fr = blockIdx.y;
    const int b = offsets[fr], e = offsets[fr + 1];
    int i0 = b + blockIdx.x * blockDim.x + threadIdx.x, i1 = e, di = gridDim.x * blockDim.x;
    if (RANK) {
        const int chunk = (int)(((int64_t)(e - b) + gridDim.x - 1) / gridDim.x);
        const int64_t c0 = (int64_t)b + (int64_t)blockIdx.x * chunk;
        i0 = (int)(c0 < e ? c0 : e) + threadIdx.x;
        i1 = (int)(c0 + chunk < e ? c0 + chunk : e);
        di = blockDim.x;
        for (int q = threadIdx.x; q < np; q += blockDim.x) pc_sh[q] = 0u;
        __syncthreads();
    }
    unsigned kmin = 0xFFFFFFFFu, kmax = 0u;
    int bad = 0;
    // PREP_U clusters per thread and round, their loads in flight together
    for (int ib = i0; ib < i1; ib += PREP_U * di) {
        int sv[PREP_U], rv[PREP_U];
        float zv[PREP_U], yv[PREP_U];
#pragma unroll
        for (int u = 0; u < PREP_U; u++) {
            const int i = ib + u * di;
            if (i < i1) {
                sv[u] = sector[i];
                rv[u] = row[i];
                zv[u] = zt[i];
                yv[u] = y[i];
            }
        }
#pragma unroll
        for (int u = 0; u < PREP_U; u++) {
            const int i = ib + u * di;
            if (i >= i1) continue;
            const int s = sv[u], r = rv[u];
            float z = zv[u];
            if (continuous) {
                const float zl = zmax - vdrift * z;
                z = (ns == 36 && s >= 18) ? -zl : zl;
            }
            zlin[i] = z;
            cfr[i] = (uint16_t)fr;
            const bool ok = s < ns && r < nr && isfinite(z) && isfinite(yv[u]);
            if (!ok) {
                bad++;
                continue;
            }
            const unsigned k = fkey(fold(z, s, ns));
            kmin = min(kmin, k);
            kmax = max(kmax, k);
            if (RANK) prank[i] = atomicAdd(&pc_sh[s * nr + r], 1u);
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        kmin = min(kmin, __shfl_xor_sync(0xffffffffu, kmin, o));
        kmax = max(kmax, __shfl_xor_sync(0xffffffffu, kmax, o));
        bad += __shfl_xor_sync(0xffffffffu, bad, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (kmin != 0xFFFFFFFFu) {
            atomicMin(&fg[fr].zmin_key, kmin);
            atomicMax(&fg[fr].zmax_key, kmax);
            atomicMin(&f->zmin_key, kmin);
            atomicMax(&f->zmax_key, kmax);
        }
        if (bad) {
            atomicAdd(&f->n_bad, bad);
            atomicExch(&f->err, TPC_ERR_DATA);
        }
    }
    if (RANK) {
        __syncthreads();
        for (int q = threadIdx.x; q < np; q += blockDim.x) {
            const uint32_t c = pc_sh[q];
            if (c) pc_sh[q] = atomicAdd(&pcount[((uint32_t)fr * (uint32_t)np + (uint32_t)q) * PSPLIT], c);
        }
        __syncthreads();
        // (a rejected cluster keeps an undefined rank: the call fails with TPC_ERR_DATA)
        for (int ib = i0; ib < i1; ib += PREP_U * di) {
            int sv[PREP_U], rv[PREP_U];
            uint32_t kv[PREP_U];
#pragma unroll
            for (int u = 0; u < PREP_U; u++) {
                const int i = ib + u * di;
                if (i < i1) {
                    sv[u] = sector[i];
                    rv[u] = row[i];
                    kv[u] = prank[i];
                }
            }
#pragma unroll
            for (int u = 0; u < PREP_U; u++) {
                const int i = ib + u * di;
                if (i < i1 && sv[u] < ns && rv[u] < nr) prank[i] = kv[u] + pc_sh[sv[u] * nr + rv[u]];
            }
        }
    }
}

// One thread: per-frame z grids inside the cell budget, the merger grid.
__global__ void k_grid_setup(Frame* f, FrameGrid* fg, int nframes, int np, int ny, float z_cell, int nzmax,
                             long long cell_cap, float merge_cell, int mnzmax, int packed)
{
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    f->ny = ny;
    long long need = 0;
    for (int i = 0; i < nframes; i++) {
        int nz = 1;
        if (fg[i].zmin_key != 0xFFFFFFFFu) {
            const float span = fkey_inv(fg[i].zmax_key) - fkey_inv(fg[i].zmin_key);
            nz = min(nzmax, (int)(span / z_cell) + 1);
        }
        fg[i].nz = nz;
        need += (long long)nz;
    }
    // cell budget: shrink every frame's z-cell count by the same factor
    const long long per = (long long)np * ny;
    const double scale = need * per > cell_cap ? (double)(cell_cap / per) / (double)need : 1.0;
    unsigned base = 0;
    for (int i = 0; i < nframes; i++) {
        int nz = fg[i].nz;
        if (scale < 1.0) nz = max(1, (int)(nz * scale));
        float zmin = 0.0f, span = 0.0f;
        if (fg[i].zmin_key != 0xFFFFFFFFu) {
            zmin = fkey_inv(fg[i].zmin_key);
            span = fkey_inv(fg[i].zmax_key) - zmin;
        }
        const float cs = fmaxf(z_cell, span * 1.001f / (float)max(nz - 1, 1));
        // packed link coordinates are unwrapped within 128 cm of the hit
        if (packed && !(cs < 60.0f)) f->err = TPC_ERR_CAPACITY;
        fg[i].zmin = zmin;
        fg[i].inv_cs = 1.0f / cs;
        fg[i].nz = nz;
        fg[i].cell_base = base;
        base += (unsigned)(per * nz);
    }
    f->total_cells = base;
    float zmin = 0.0f, span = 0.0f;
    if (f->zmin_key != 0xFFFFFFFFu) {
        zmin = fkey_inv(f->zmin_key);
        span = fkey_inv(f->zmax_key) - zmin;
    }
    const float mcs = fmaxf(merge_cell, span / (float)(mnzmax - 1) * 1.001f);
    f->mzmin = zmin;
    f->minv_cs = 1.0f / mcs;
    f->mnz = min(mnzmax, (int)(span / mcs) + 1);
}

__device__ __forceinline__ int ybin(float y, const float* __restrict__ rowtab, int r, int ny)
{
    float t = (y - rowtab[r * ROWTAB + 4]) * rowtab[r * ROWTAB + 5];
    t = fminf(fmaxf(t, 0.0f), (float)(ny - 1));   // NaN -> 0
    return (int)t;
}

__global__ void k_hist(int n, const uint8_t* __restrict__ sector, const uint8_t* __restrict__ row,
                       const float* __restrict__ y, const float* __restrict__ zlin, const uint16_t* __restrict__ cfr,
                       const float* __restrict__ rowtab, int nr, int ns, const Frame* __restrict__ f,
                       const FrameGrid* __restrict__ fg, uint32_t* __restrict__ count, uint32_t* __restrict__ cell,
                       uint32_t* __restrict__ slot)
{
    if (f->err) return;   // invalid clusters: nothing after validation runs
    const int ny = f->ny;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int s = sector[i], r = row[i];
        const FrameGrid G = fg[cfr[i]];
        const int pl = s * nr + r;
        const int zc = grid_cell(fold(zlin[i], s, ns), G.zmin, G.inv_cs, G.nz);
        const uint32_t c = G.cell_base + ((uint32_t)pl * (uint32_t)G.nz + (uint32_t)zc) * (uint32_t)ny +
                           (uint32_t)ybin(y[i], rowtab, r, ny);
        cell[i] = c;
        slot[i] = atomicAdd(&count[c], 1u);
    }
}

// Sorted cluster record (16 bytes): y, z, input index, plane
// (frame * planes + sector * rows + row), loaded with one vector access.
__device__ __forceinline__ int sc_id(const float4& c) { return __float_as_int(c.z); }
__device__ __forceinline__ uint32_t sc_plane(const float4& c) { return __float_as_uint(c.w); }

// Packed link coordinates: a coordinate v is the fixed-point integer
// q = rint(v * 256) (step 2^-8 cm, exact in binary32 for |v| < 2^16 cm); the
// packed word holds the low 16 bits of q_y and q_z.  A reader recovers q from
// its low bits and a reference q_ref within 2^15 steps (128 cm): the
// neighbours of a hit lie within three grid cells of it.
__device__ __forceinline__ int fixq(float v) { return __float2int_rn(v * 256.0f); }
__device__ __forceinline__ float unfixq(int q) { return (float)q * 0.00390625f; }
__device__ __forceinline__ uint32_t pack_yz(float y, float z)
{
    return ((uint32_t)fixq(y) & 0xFFFFu) | ((uint32_t)fixq(z) << 16);
}
__device__ __forceinline__ int unwrap16(uint32_t lo, int qref)
{
    return qref + (int)(int16_t)(uint16_t)(lo - (uint32_t)qref);
}

__global__ void k_scatter(int n, const uint8_t* __restrict__ sector, const uint8_t* __restrict__ row,
                          const float* __restrict__ y, const float* __restrict__ zlin, const uint16_t* __restrict__ cfr,
                          int nr, int np, const uint32_t* __restrict__ cstart, const uint32_t* __restrict__ cell,
                          const uint32_t* __restrict__ slot, float4* __restrict__ sc, const Frame* __restrict__ f,
                          uint32_t* __restrict__ yzp)
{
    if (f->err) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint32_t pos = cstart[cell[i]] + slot[i];
        const uint32_t pg = (uint32_t)cfr[i] * (uint32_t)np + (uint32_t)(sector[i] * nr + row[i]);
        sc[pos] = make_float4(y[i], zlin[i], __int_as_float(i), __uint_as_float(pg));
        if (yzp) yzp[pos] = pack_yz(y[i], zlin[i]);
    }
}


// Binning in two steps.  (1) k_prep ranks every cluster among the clusters
// of its plane (frame, sector, row) and k_pscatter moves its record into the
// plane's range of the plane-ordered buffer.  (2) k_plane_sort, one block per
// plane, counts the plane's clusters per cell (z-cell, y-bin) in shared
// memory, writes the plane's cell starts and moves the records into cell
// order.  Nothing of the size of the grid is zeroed, updated atomically or
// scanned in global memory, so finer grids cost little here.  The order of
// the clusters inside a cell depends on the atomics; no search depends on it.
__global__ void k_pscatter(int n, const uint8_t* __restrict__ sector, const uint8_t* __restrict__ row,
                           const float* __restrict__ y, const float* __restrict__ zlin, const uint16_t* __restrict__ cfr,
                           int nr, int np, const uint32_t* __restrict__ pstart, const uint32_t* __restrict__ prank,
                           float4* __restrict__ pbuf, const Frame* __restrict__ f)
{
    if (f->err) return;
    // PSC_U clusters per thread and round: their loads, then their plane
    // starts, are in flight together (the kernel is bound by the latency of
    // the dependent plane-start gather)
    constexpr int PSC_U = 4;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t ib = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; ib < n; ib += PSC_U * stride) {
        uint32_t pg[PSC_U], rk[PSC_U], ps[PSC_U];
        float yv[PSC_U], zv[PSC_U];
#pragma unroll
        for (int u = 0; u < PSC_U; u++) {
            const int64_t i = ib + u * stride;
            if (i < n) {
                pg[u] = (uint32_t)cfr[i] * (uint32_t)np + (uint32_t)(sector[i] * nr + row[i]);
                rk[u] = prank[i];
                yv[u] = y[i];
                zv[u] = zlin[i];
            }
        }
#pragma unroll
        for (int u = 0; u < PSC_U; u++)
            if (ib + u * stride < n) ps[u] = pstart[(size_t)pg[u] * PSPLIT];
#pragma unroll
        for (int u = 0; u < PSC_U; u++) {
            const int64_t i = ib + u * stride;
            if (i < n) pbuf[ps[u] + rk[u]] = make_float4(yv[u], zv[u], __int_as_float((int)i), __uint_as_float(pg[u]));
        }
    }
}

constexpr int PS_BLOCK = 256;
constexpr int PS_ITEMS = 8;
constexpr int PS_SMEM_CELLS = 16384;    // larger planes count in their global cell range

// a[i] = base + a[0] + ... + a[i-1] for i < n (shared or global memory), by
// one block: warp w scans 32 * PS_ITEMS consecutive entries of each chunk, a
// row of 32 at a time.  Ends with a barrier.
__device__ void block_excl_scan(uint32_t* a, int n, uint32_t base)
{
    __shared__ uint32_t wtot[PS_BLOCK / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    constexpr int SEG = 32 * PS_ITEMS, CHUNK = PS_BLOCK * PS_ITEMS;
    uint32_t carry = base;
    for (int k0 = 0; k0 < n; k0 += CHUNK) {
        const int s0 = k0 + w * SEG;
        uint32_t v[PS_ITEMS];
        uint32_t run = 0;
#pragma unroll
        for (int j = 0; j < PS_ITEMS; j++) {
            const int i = s0 + j * 32 + lane;
            const uint32_t x = i < n ? a[i] : 0u;
            uint32_t inc = x;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += t;
            }
            v[j] = run + inc - x;
            run += __shfl_sync(0xffffffffu, inc, 31);
        }
        if (lane == 0) wtot[w] = run;
        __syncthreads();
        uint32_t off = carry, tot = 0;
#pragma unroll
        for (int k = 0; k < PS_BLOCK / 32; k++) {
            const uint32_t t = wtot[k];
            if (k < w) off += t;
            tot += t;
        }
#pragma unroll
        for (int j = 0; j < PS_ITEMS; j++) {
            const int i = s0 + j * 32 + lane;
            if (i < n) a[i] = off + v[j];
        }
        carry += tot;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(PS_BLOCK) k_plane_sort(int nplanes, int np, int nr, int ns,
                                                         const uint32_t* __restrict__ pstart,
                                                         const float4* __restrict__ pbuf, uint32_t* __restrict__ rank,
                                                         const float* __restrict__ rowtab, const Frame* __restrict__ f,
                                                         const FrameGrid* __restrict__ fg, int smem_cells,
                                                         uint32_t* __restrict__ cstart, float4* __restrict__ sc,
                                                         uint32_t* __restrict__ yzp)
{
    extern __shared__ uint32_t cnt_sh[];
    if (f->err) return;
    const int ny = f->ny;
    for (int p = blockIdx.x; p < nplanes; p += gridDim.x) {
        const int fr = p / np, lpl = p - fr * np;
        const int s = lpl / nr, r = lpl - s * nr;
        const FrameGrid G = fg[fr];
        const int nc = G.nz * ny;
        const uint32_t cbase = G.cell_base + (uint32_t)lpl * (uint32_t)nc;
        const uint32_t a = pstart[(size_t)p * PSPLIT], b = pstart[(size_t)(p + 1) * PSPLIT];
        const bool in_sh = nc <= smem_cells;
        uint32_t* cnt = in_sh ? cnt_sh : cstart + cbase;
        for (int c = threadIdx.x; c < nc; c += blockDim.x) cnt[c] = 0u;
        __syncthreads();
        // the cell of a record: the functions the window searches use
        auto cell_of = [&](const float4& q) -> int {
            const int zc = grid_cell(fold(q.y, s, ns), G.zmin, G.inv_cs, G.nz);
            return zc * ny + ybin(q.x, rowtab, r, ny);
        };
        for (uint32_t i = a + threadIdx.x; i < b; i += blockDim.x) rank[i] = atomicAdd(&cnt[cell_of(pbuf[i])], 1u);
        __syncthreads();
        block_excl_scan(cnt, nc, a);          // cnt[c]: sorted index of cell c's first cluster
        if (in_sh)
            for (int c = threadIdx.x; c < nc; c += blockDim.x) cstart[cbase + c] = cnt[c];
        if (p == nplanes - 1 && threadIdx.x == 0) cstart[cbase + nc] = b;
        for (uint32_t i = a + threadIdx.x; i < b; i += blockDim.x) {
            const float4 q = pbuf[i];
            const uint32_t d = cnt[cell_of(q)] + rank[i];
            sc[d] = q;
            if (yzp) yzp[d] = pack_yz(q.x, q.y);
        }
        __syncthreads();                      // cnt is reused by the block's next plane
    }
}

// Shared-memory cells of k_plane_sort for planes of up to `want` cells: up
// to PS_SMEM_CELLS once the kernel may use more than 48 KB, which is set
// outside stream capture (once per device); 48 KB before that.
int plane_sort_smem_cells(int64_t want, cudaStream_t st)
{
    static int done_dev[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(st, &cs);
    if (dev >= 0 && dev < 64 && !done_dev[dev] && cs == cudaStreamCaptureStatusNone &&
        cudaFuncSetAttribute(k_plane_sort, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(sizeof(uint32_t) * PS_SMEM_CELLS)) == cudaSuccess)
        done_dev[dev] = 1;
    const int64_t cap = (dev >= 0 && dev < 64 && done_dev[dev]) ? PS_SMEM_CELLS : 48 * 1024 / (int)sizeof(uint32_t);
    return (int)std::max<int64_t>(1, std::min<int64_t>(want, cap));
}

// The cells a search window overlaps: the z-cells c0..c1 of
// [zp - wz, zp + wz] and, in each, the contiguous y-bins y0..y1 of
// [yp - wy, yp + wy], both widened by WIN_MARGIN (more than the rounding of
// the window edges and of packed coordinates).  Cells and bins are monotone
// in the coordinate, so every cluster that passes the window test lies in
// these ranges, whatever the cell and bin sizes.
constexpr float WIN_MARGIN = 1.0f / 64;

struct WinCells {
    uint32_t base;      // cell of (plane, z-cell c0, y-bin 0)
    int nzc, y0, y1, ny;
    // sorted-index range [b, e) of the window's bins in its k-th z-cell
    __device__ __forceinline__ void range(const uint32_t* __restrict__ cstart, int k, int& b, int& e) const
    {
        const uint32_t c = base + (uint32_t)k * (uint32_t)ny;
        b = (int)cstart[c + y0];
        e = (int)cstart[c + y1 + 1];
    }
};

__device__ __forceinline__ WinCells window_cells(const FrameGrid& G, int lplane, int s, int ns,
                                                 const float* __restrict__ rowtab, int r, int ny, float yp, float zp,
                                                 float wy, float wz)
{
    const float za = fold(zp - (wz + WIN_MARGIN), s, ns), zb = fold(zp + (wz + WIN_MARGIN), s, ns);
    const int c0 = grid_cell(fminf(za, zb), G.zmin, G.inv_cs, G.nz);
    const int c1 = grid_cell(fmaxf(za, zb), G.zmin, G.inv_cs, G.nz);
    WinCells W;
    W.base = G.cell_base + ((uint32_t)lplane * (uint32_t)G.nz + (uint32_t)c0) * (uint32_t)ny;
    W.nzc = c1 - c0 + 1;
    W.y0 = ybin(yp - (wy + WIN_MARGIN), rowtab, r, ny);
    W.y1 = ybin(yp + (wy + WIN_MARGIN), rowtab, r, ny);
    W.ny = ny;
    return W;
}

// ---------------------------------------------------------------------------
// a3: NeighboursFinder (one thread per sorted hit)
// ---------------------------------------------------------------------------
constexpr int MAXD = 8;

// PACKED: the pass reads candidates from the 16-bit packed words and sees
// every coordinate, the middle hit's too, rounded to the nearest 1/256 cm.
template <bool PACKED>
__global__ void __launch_bounds__(256) k_neighbours(
    int n, int nr, int ns, int np, const float* __restrict__ rowtab, const float4* __restrict__ sc,
    const uint32_t* __restrict__ cstart,
    const Frame* __restrict__ f, const FrameGrid* __restrict__ fg, float DY, float DZ, float SMAX,
    int32_t* __restrict__ upr, int32_t* __restrict__ dnr, const uint32_t* __restrict__ yzp)
{
    if (f->err) return;
    const int ny = f->ny;
    for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < n; h += gridDim.x * blockDim.x) {
        const float4 ch = sc[h];
        const uint32_t pg = sc_plane(ch);
        const int fr = (int)(pg / (uint32_t)np);
        const int pl = (int)(pg - (uint32_t)fr * np);
        const int s = pl / nr, r = pl - s * nr;
        int bu = -1, bd = -1, bidu = 0, bidd = 0;
        float bs = 0.0f;
        if (r >= 1 && r <= nr - 2) {
            const FrameGrid G = fg[fr];
            float yh = ch.x, zh = ch.y;
            int qyh = 0, qzh = 0;
            if (PACKED) {
                qyh = fixq(yh);
                qzh = fixq(zh);
                yh = unfixq(qyh);
                zh = unfixq(qzh);
            }
            auto coord = [&](int q) -> float2 {
                if (!PACKED) {
                    const float4 c = sc[q];
                    return make_float2(c.x, c.y);
                }
                const uint32_t wd = yzp[q];
                return make_float2(unfixq(unwrap16(wd & 0xFFFFu, qyh)), unfixq(unwrap16(wd >> 16, qzh)));
            };
            const float yu_pred = yh * rowtab[r * ROWTAB + 1];
            const float yd_pred = yh * rowtab[r * ROWTAB + 2];
            const float w = rowtab[r * ROWTAB + 3];
            const WinCells wu = window_cells(G, pl + 1, s, ns, rowtab, r + 1, ny, yu_pred, zh, DY, DZ);
            const WinCells wd = window_cells(G, pl - 1, s, ns, rowtab, r - 1, ny, yd_pred, zh, DY, DZ);
            // down candidates inside the windows
            int dl[MAXD];
            int ndn = 0;
            bool overflow = false;
            for (int k = 0; k < wd.nzc; k++) {
                int qb, qe;
                wd.range(cstart, k, qb, qe);
                for (int q = qb; q < qe; q++) {
                    const float2 pq = coord(q);
                    if (fabsf(pq.x - yd_pred) <= DY && fabsf(pq.y - zh) <= DZ) {
                        if (ndn < MAXD) dl[ndn++] = q;
                        else overflow = true;
                    }
                }
            }
            if (ndn > 0) {
                for (int ku = 0; ku < wu.nzc; ku++) {
                    int ub, ue;
                    wu.range(cstart, ku, ub, ue);
                    for (int u = ub; u < ue; u++) {
                        const float2 pu = coord(u);
                        const float yu = pu.x, zu = pu.y;
                        if (!(fabsf(yu - yu_pred) <= DY && fabsf(zu - zh) <= DZ)) continue;
                        const int idu = sc_id(sc[u]);
                        auto consider = [&](int d) {
                            const float2 pd = coord(d);
                            const float yd = pd.x, zd = pd.y;
                            const float ey = __fmaf_rn(yu - yd, w, yd) - yh;
                            const float ez = __fmaf_rn(zu - zd, w, zd) - zh;
                            const float score = __fmaf_rn(ey, ey, ez * ez);
                            if (!(score < SMAX)) return;
                            const int idd = sc_id(sc[d]);
                            if (bu < 0 || score < bs || (score == bs && (idu < bidu || (idu == bidu && idd < bidd)))) {
                                bu = u; bd = d; bs = score; bidu = idu; bidd = idd;
                            }
                        };
                        if (!overflow) {
                            for (int k = 0; k < ndn; k++) consider(dl[k]);
                        } else {
                            for (int k = 0; k < wd.nzc; k++) {
                                int db, de;
                                wd.range(cstart, k, db, de);
                                for (int d = db; d < de; d++) {
                                    const float2 pd = coord(d);
                                    if (fabsf(pd.x - yd_pred) <= DY && fabsf(pd.y - zh) <= DZ) consider(d);
                                }
                            }
                        }
                    }
                }
            }
        }
        upr[h] = bu;
        dnr[h] = bd;
    }
}

// ---------------------------------------------------------------------------
// a4 NeighboursCleaner, a5 StartHitsFinder
// ---------------------------------------------------------------------------
__global__ void k_clean(int n, const int32_t* __restrict__ upr, const int32_t* __restrict__ dnr,
                        int32_t* __restrict__ up, int32_t* __restrict__ dn, const Frame* __restrict__ f)
{
    if (f->err) return;
    for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < n; h += gridDim.x * blockDim.x) {
        const int u = upr[h], d = dnr[h];
        up[h] = (u >= 0 && dnr[u] == h) ? u : -1;
        dn[h] = (d >= 0 && upr[d] == h) ? d : -1;
    }
}

// NeighboursCleaner and StartHitsFinder in one pass: the cleaned links of h,
// and of its up neighbour, come from the raw links directly (a link is kept
// when the neighbour links back)
__global__ void k_clean_starts(int n, const int32_t* __restrict__ upr, const int32_t* __restrict__ dnr,
                               int32_t* __restrict__ up, int32_t* __restrict__ dn, int32_t* __restrict__ starts,
                               int cap, Frame* f)
{
    if (f->err) return;
    // CS_U hits per thread and round: each level of the dependent link reads
    // (own links, the neighbours' back links, the up neighbour's up link and
    // its back link) is in flight for all of them together
    constexpr int CS_U = 4;
    const int stride = gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += (int64_t)CS_U * stride) {
        int uv[CS_U], dv[CS_U], bu[CS_U], bd[CS_U];
#pragma unroll
        for (int k = 0; k < CS_U; k++) {
            const int64_t h = base + (int64_t)k * stride + threadIdx.x;
            uv[k] = -1;
            dv[k] = -1;
            if (h < n) {
                uv[k] = upr[h];
                dv[k] = dnr[h];
            }
        }
#pragma unroll
        for (int k = 0; k < CS_U; k++) {
            bu[k] = uv[k] >= 0 ? dnr[uv[k]] : -1;
            bd[k] = dv[k] >= 0 ? upr[dv[k]] : -1;
        }
        int uc[CS_U], uu[CS_U];
#pragma unroll
        for (int k = 0; k < CS_U; k++) {
            const int64_t h = base + (int64_t)k * stride + threadIdx.x;
            uc[k] = (uv[k] >= 0 && bu[k] == h) ? uv[k] : -1;
            const int dc = (dv[k] >= 0 && bd[k] == h) ? dv[k] : -1;
            if (h < n) {
                up[h] = uc[k];
                dn[h] = dc;
            }
            // a start candidate: kept up link, no kept down link
            uu[k] = (uc[k] >= 0 && dc < 0) ? upr[uc[k]] : -1;
        }
#pragma unroll
        for (int k = 0; k < CS_U; k++) {
            const int64_t h = base + (int64_t)k * stride + threadIdx.x;
            const bool is = uu[k] >= 0 && dnr[uu[k]] == uc[k];      // the up neighbour keeps its up link
            const unsigned mask = __ballot_sync(0xffffffffu, is);
            int pos0 = 0;
            if (lane == 0 && mask) pos0 = atomicAdd(&f->n_starts, __popc(mask));
            pos0 = __shfl_sync(0xffffffffu, pos0, 0);
            if (is) {
                const int pos = pos0 + __popc(mask & ((1u << lane) - 1u));
                if (pos < cap) starts[pos] = (int)h;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// a6: TrackletConstructor
// ---------------------------------------------------------------------------
struct TrkArgs {
    const float* rowtab;
    const float4* sc;
    float* t_state;             // [cap][NST + 4]: state after phase A, phase, rc, nu (two-pass mode)
    const uint32_t* cstart;
    const int32_t* up;
    const int32_t* starts;
    const Frame* f;
    const FrameGrid* fg;
    int nr, ns, np, cap;
    float kb, vy, vz, c0s, c0t, c0q, nsig, wmin, wmax, chi2cut, edge;
    int max_miss;
    int prof;
    int32_t *t_start, *t_id, *t_nhits, *t_nup, *t_hits;
    float *t_top, *t_bot;
    Frame* fw;
};

// Nearest cluster of the plane inside |dy| <= wy, |dz| <= wz of (yp, zp):
// minimum dy^2 + dz^2 (binary32, fused), ties to the smaller input index.
// The index ranges of up to NZR z-cells are loaded before their candidates
// are scanned, so that the lane waits for one round of grid loads, not one
// per z-cell.
constexpr int NZR = 2;
template <bool PROF>
__device__ __forceinline__ int find_nearest(const TrkArgs& A, const float* rt, const FrameGrid& G, int lplane, int r,
                                            int s, float yp,
                                            float zp, float wy, float wz, int ny, unsigned& ncand, float& by, float& bz)
{
    const WinCells W = window_cells(G, lplane, s, A.ns, rt, r, ny, yp, zp, wy, wz);
    int best = -1, bid = 0;
    float bd = 0.0f;
    for (int k0 = 0; k0 < W.nzc; k0 += NZR) {
        int qb[NZR], qe[NZR];
#pragma unroll
        for (int j = 0; j < NZR; j++) {
            qb[j] = 0;
            qe[j] = 0;
            if (k0 + j < W.nzc) W.range(A.cstart, k0 + j, qb[j], qe[j]);
        }
#pragma unroll
        for (int j = 0; j < NZR; j++) {
            if (PROF) ncand += (unsigned)(qe[j] - qb[j]);
            auto cand = [&](const float4& pq, int q) {
                const float dy = pq.x - yp;
                const float dz = pq.y - zp;
                if (!(fabsf(dy) <= wy) || !(fabsf(dz) <= wz)) return;
                const float d2 = __fmaf_rn(dy, dy, dz * dz);
                const int id = sc_id(pq);
                if (best < 0 || d2 < bd || (d2 == bd && id < bid)) {
                    best = q; bd = d2; bid = id; by = pq.x; bz = pq.y;
                }
            };
            int q = qb[j];
            for (; q + 1 < qe[j]; q += 2) {
                const float4 p0 = A.sc[q], p1 = A.sc[q + 1];
                cand(p0, q);
                cand(p1, q + 1);
            }
            if (q < qe[j]) cand(A.sc[q], q);
        }
    }
    return best;
}

// Phases of one tracklet (the operation sequence per tracklet is fixed; the
// kernel only interleaves tracklets differently across lanes)
enum : int { PH_A = 0, PH_B = 1, PH_CSTART = 2, PH_BACK = 3, PH_C = 4, PH_DONE = 5 };
// phase C returns to the start row in jumps of at most BACK_JUMP rows; a
// refused jump (|u| or |sin(phi)| out of range) is retried with half as many
// rows, a refused single-row step ends the tracklet
constexpr int BACK_JUMP = 32;

constexpr int TRK_BLOCK = 128;

// One lane = one tracklet at a time.  Each loop iteration advances the lane's
// tracklet by one row step; a lane whose tracklet ends writes it out and takes
// the next start hit from a global queue, so lanes stay busy however uneven
// the tracklet lengths are.  The propagation, the window search and the
// Kalman update each have a single call site shared by all phases, so a warp
// whose lanes are in different phases still executes each of them once per
// iteration.
// PASS 0: the whole tracklet in one pass.  PASS 1: phase A only (the chain
// fit, no window searches), then the state is saved.  PASS 2: phases B, C
// from the saved states.  Split, the warps of pass 1 never wait for a search
// (a warp otherwise pays the search latency whenever any of its lanes
// searches), and the search phases of pass 2 run densely.  The operation
// sequence of every tracklet is the same in either mode.
constexpr int TSAVE = NST + 4;
// 8 blocks of 128 threads per SM (64 registers) measured best for both passes
// (against 6 to 16 blocks for pass 1 and 6 to 8 for pass 2)
template <int PASS, bool PROF>
__global__ void __launch_bounds__(TRK_BLOCK, 8) k_tracklets(TrkArgs A)
{
    // the last accepted state of each lane (outer-end / inner-end candidate) lives
    // in shared memory, element-major so that the lanes of a warp hit distinct banks
    __shared__ float keep_sh[NST][TRK_BLOCK];
    // the row table (x, y-bin origin and scale are read at every step)
    __shared__ float rt[ROWTAB * 256];
    for (int i = threadIdx.x; i < ROWTAB * A.nr; i += blockDim.x) rt[i] = A.rowtab[i];
    __syncthreads();
    if (A.f->err) return;
    const int ny = A.f->ny;
    const int nt = min(A.f->n_starts, A.cap);
    const float INF = __int_as_float(0x7f800000);
    const int NR = A.nr;
    const unsigned lane = threadIdx.x & 31u;
    unsigned nprop = 0, nupd = 0, ncand = 0;

    float st[NST];
    // (pass 1 ends every tracklet in phase A, where the kept state is the state)
    auto save_keep = [&]() {
        if (PASS != 1) {
#pragma unroll
            for (int i = 0; i < NST; i++) keep_sh[i][threadIdx.x] = st[i];
        }
    };
    int t = -1, phase = PH_DONE;
    int h1 = 0, r1 = 0, s = 0, lbase = 0, pgbase = 0, rc = 0, r = 0, miss = 0, nu = 0, nd = 0, jump = BACK_JUMP;
    FrameGrid G;
    G.zmin = 0.0f; G.inv_cs = 1.0f; G.nz = 1; G.cell_base = 0u; G.zmin_key = 0u; G.zmax_key = 0u;
    // next chain hit (phase A), loaded one step ahead
    int nx_h = -1, nx_row = 0;
    float2 nx_yz = make_float2(0.0f, 0.0f);
    int32_t* slot = nullptr;
    // the frame, sector and start row of a tracklet from its start hit's plane
    auto enter = [&](uint32_t pg1) {
        const int fr = (int)(pg1 / (uint32_t)A.np);
        const int pl1 = (int)(pg1 - (uint32_t)fr * A.np);
        G = A.fg[fr];
        s = pl1 / NR;
        r1 = pl1 - s * NR;
        lbase = s * NR;
        pgbase = (int)pg1 - r1;
    };
    for (;;) {
        // ---- bookkeeping transitions
        if (PASS == 1 && (phase == PH_B || phase == PH_CSTART)) {
            // end of phase A: save the state for the second pass
            float* sv = A.t_state + (int64_t)t * TSAVE;
#pragma unroll
            for (int i = 0; i < NST; i++) sv[i] = st[i];
            sv[NST] = __int_as_float(phase);
            sv[NST + 1] = __int_as_float(rc);
            sv[NST + 2] = __int_as_float(nu);
            sv[NST + 3] = __int_as_float(pgbase + r1);   // the start hit's plane
            phase = PH_DONE;
        }
        if (phase == PH_DONE) {
            if (t >= 0 && PASS != 1) {
                float* bot = A.t_bot + (int64_t)t * NST;
#pragma unroll
                for (int i = 0; i < NST; i++) bot[i] = keep_sh[i][threadIdx.x];
                if (PASS == 0) {
                    A.t_start[t] = h1;
                    A.t_id[t] = sc_id(A.sc[h1]);
                }
                A.t_nhits[t] = nu + nd;
                A.t_nup[t] = nu;
            }
            // next start hit from the queue (one atomic per group of lanes asking together)
            const unsigned m = __activemask();
            const int leader = __ffs(m) - 1;
            int base = 0;
            if ((int)lane == leader) base = atomicAdd(PASS == 2 ? &A.fw->trk_next2 : &A.fw->trk_next, __popc(m));
            base = __shfl_sync(m, base, leader);
            t = base + __popc(m & ((1u << lane) - 1u));
            if (t >= nt) break;
            if (PASS == 2) {
                // continue from the state phase A left (the start hit's plane
                // included: no load of the start hit itself); the step below
                // runs in this same iteration
                const float* sv = A.t_state + (int64_t)t * TSAVE;
                enter((uint32_t)__float_as_int(sv[NST + 3]));
#pragma unroll
                for (int i = 0; i < NST; i++) st[i] = sv[i];
                phase = __float_as_int(sv[NST]);
                rc = __float_as_int(sv[NST + 1]);
                nu = __float_as_int(sv[NST + 2]);
                nd = 0;
                miss = 0;
                slot = A.t_hits + (int64_t)t * NR;
                save_keep();
            }
        }
        if (PASS != 2 && phase == PH_DONE) {     // a start hit just taken (passes 0 and 1)
            // initial state at the start hit: y, z measured, slopes from the first link
            h1 = A.starts[t];
            const float4 c1 = A.sc[h1];
            enter(sc_plane(c1));
            if (PASS == 1) {
                A.t_start[t] = h1;
                A.t_id[t] = sc_id(c1);
            }
            const int h2 = A.up[h1];
            const float x1 = rt[r1 * ROWTAB], x2 = rt[(r1 + 1) * ROWTAB];
            const float dx12 = x2 - x1;
            const float4 c2 = A.sc[h2];
            const float2 p1 = make_float2(c1.x, c1.y), p2 = make_float2(c2.x, c2.y);
            const float y1 = p1.x, z1 = p1.y;
            const float dy12 = p2.x - y1, dz12 = p2.y - z1;
            const float ty = __fdiv_rn(dy12, dx12);
            const float sp = __fdiv_rn(ty, __fsqrt_rn(__fmaf_rn(ty, ty, 1.0f)));
            const float dl12 = __fsqrt_rn(__fmaf_rn(dx12, dx12, dy12 * dy12));
            const float tl = __fdiv_rn(dz12, dl12);
#pragma unroll
            for (int i = 0; i < NST; i++) st[i] = 0.0f;
            st[0] = x1; st[1] = y1; st[2] = z1; st[3] = sp; st[4] = tl; st[5] = 0.0f;
            st[6 + 0] = A.vy; st[6 + 2] = A.vz; st[6 + 5] = A.c0s; st[6 + 9] = A.c0t; st[6 + 14] = A.c0q;
            slot = A.t_hits + (int64_t)t * NR;
            nu = 0;
            nd = 0;
            slot[nu++] = h1;
            save_keep();
            rc = r1;
            phase = PH_A;
            nx_h = h2;
            nx_row = (int)sc_plane(c2) - pgbase;
            nx_yz = p2;
        }
        if (phase == PH_CSTART) {
            // end of the upward phases: the outer-end state is final
            float* top = A.t_top + (int64_t)t * NST;
#pragma unroll
            for (int i = 0; i < NST; i++) top[i] = keep_sh[i][threadIdx.x];
            if (rc == r1) save_keep();
            miss = 0;
            r = r1 - 1;
            jump = BACK_JUMP;
            phase = rc > r1 ? PH_BACK : PH_C;
        }
        // ---- the row this step goes to
        int target = -1, hn = -1;
        float2 pn = make_float2(0.0f, 0.0f);
        if (phase == PH_A) {                    // fit along the up links
            hn = nx_h;
            if (hn < 0) {
                phase = PH_B;
                miss = 0;
            } else {
                target = nx_row;
                pn = nx_yz;
                // load the following chain hit while this step computes
                nx_h = A.up[hn];
                if (nx_h >= 0) {
                    const float4 cn = A.sc[nx_h];
                    nx_row = (int)sc_plane(cn) - pgbase;
                    nx_yz = make_float2(cn.x, cn.y);
                }
            }
        }
        if (PASS == 1 && phase != PH_A) continue;   // saved at the top of the next iteration
        if (phase == PH_B) {                    // follow beyond the chain end
            if (rc + 1 < NR) target = rc + 1;
            else phase = PH_CSTART;
        }
        if (phase == PH_BACK)                   // back to the start row
            target = max(r1, rc - jump);
        if (phase == PH_C) {                    // below the start
            if (r >= 0) target = r;
            else phase = PH_DONE;
        }
        if (target < 0) continue;
        // ---- propagation (one call site)
        if (!prop32(st, rt[target * ROWTAB], A.kb)) {
            if (phase == PH_BACK && jump > 1) jump >>= 1;
            else phase = (phase == PH_C || phase == PH_BACK) ? PH_DONE : PH_CSTART;
            continue;
        }
        if (PROF) nprop++;
        if (phase == PH_BACK) {
            rc = target;
            if (rc == r1) {
                save_keep();
                phase = PH_C;
            }
            continue;
        }
        bool search = false, upd = false;
        float my = 0.0f, mz = 0.0f, cmax = INF;
        int c = -1;
        if (phase == PH_A) {
            rc = target;
            my = pn.x;
            mz = pn.y;
            upd = true;
            if (PROF) nupd++;
        } else if (phase == PH_B) {
            rc = target;
            search = true;
        } else {
            search = true;
        }
        if (search) {
            if (fabsf(st[1]) > __fmaf_rn(st[0], TAN10, A.edge)) {
                phase = (phase == PH_B) ? PH_CSTART : PH_DONE;
                continue;
            }
            // ---- window search (one call site)
            const float wy = fminf(fmaxf(A.nsig * __fsqrt_rn(st[6 + 0] + A.vy), A.wmin), A.wmax);
            const float wz = fminf(fmaxf(A.nsig * __fsqrt_rn(st[6 + 2] + A.vz), A.wmin), A.wmax);
            c = find_nearest<PROF>(A, rt, G, lbase + target, target, s, st[1], st[2], wy, wz, ny, ncand, my, mz);
            if (c >= 0) {
                cmax = A.chi2cut;
                upd = true;
            }
        }
        // ---- Kalman update (one call site)
        const bool took = upd && update32(st, my, mz, A.vy, A.vz, cmax);
        // the hit is recorded and the state kept on one path for all phases
        // (phase A keeps its chain hit whether or not the update was taken):
        // hits above the start fill the slot from the front, those below it
        // from the back
        if (phase == PH_A || took) {
            if (PROF && phase != PH_A) nupd++;
            int k;
            if (phase == PH_C) k = NR - (++nd);
            else k = nu++;
            slot[k] = phase == PH_A ? hn : c;
            save_keep();
            miss = 0;
        } else if (++miss >= A.max_miss) {
            if (phase == PH_B) {
                phase = PH_CSTART;
            } else {
                phase = PH_DONE;
                continue;
            }
        }
        if (phase == PH_C) r--;
    }
    if (PROF) {
        // work counters: one atomic per warp (every lane of the warp gets here)
        nprop = __reduce_add_sync(0xffffffffu, nprop);
        nupd = __reduce_add_sync(0xffffffffu, nupd);
        ncand = __reduce_add_sync(0xffffffffu, ncand);
        if (lane == 0) {
            atomicAdd(&A.fw->w_prop, (unsigned long long)nprop);
            atomicAdd(&A.fw->w_upd, (unsigned long long)nupd);
            atomicAdd(&A.fw->w_cand, (unsigned long long)ncand);
        }
    }
}

// k-th hit (ascending row) of tracklet t
__device__ __forceinline__ int trk_hit(const int32_t* slot, int nr, int nhits, int nup, int k)
{
    const int nd = nhits - nup;
    return k < nd ? slot[nr - nd + k] : slot[k - nd];
}

// ---------------------------------------------------------------------------
// a7: TrackletSelector
// ---------------------------------------------------------------------------
// Selector weight of a tracklet: more hits first, then the smaller start-hit
// id.  64 bits in general; 32 bits ((hits << 24) | (2^24 - 1 - id)) when every
// id of the call is below 2^24 (hits <= 255 always): the same order, half the
// memory and atomic payload.
template <typename W> __device__ __forceinline__ W sel_weight(int nh, int id);
template <> __device__ __forceinline__ unsigned long long sel_weight<unsigned long long>(int nh, int id)
{
    return tracklet_weight(nh, id);
}
template <> __device__ __forceinline__ unsigned sel_weight<unsigned>(int nh, int id)
{
    return ((unsigned)nh << 24) | (0xFFFFFFu - (unsigned)id);
}

// SEL_G lanes per tracklet: the hits of one tracklet are adjacent in its hit
// slot, so the group's slot loads are coalesced and its weight updates (or
// reads) go out together.
constexpr int SEL_G = 8;

template <typename W>
__global__ void k_sel_weight(const Frame* __restrict__ f, int cap, int nr, int min_hits, const int32_t* __restrict__ t_id,
                             const int32_t* __restrict__ t_nhits, const int32_t* __restrict__ t_nup,
                             const int32_t* __restrict__ t_hits, W* __restrict__ hitw)
{
    const int nt = min(f->n_starts, cap);
    const int j = threadIdx.x % SEL_G;
    const int ngroups = (gridDim.x * blockDim.x) / SEL_G;
    for (int t = (blockIdx.x * blockDim.x + threadIdx.x) / SEL_G; t < nt; t += ngroups) {
        const int nh = t_nhits[t];
        if (nh < min_hits) continue;
        const W w = sel_weight<W>(nh, t_id[t]);
        const int32_t* slot = t_hits + (int64_t)t * nr;
        const int nup = t_nup[t];
        for (int k = j; k < nh; k += SEL_G) atomicMax(&hitw[trk_hit(slot, nr, nh, nup, k)], w);
    }
}

// The loops are warp-uniform (every lane runs the warp's largest trip count)
// so that the group's OR and sum shuffles have all lanes present.
template <typename W>
__global__ void k_sel_own(Frame* f, int cap, int nr, int min_hits, int min_owned, const int32_t* __restrict__ t_id,
                          const int32_t* __restrict__ t_nhits, const int32_t* __restrict__ t_nup,
                          const int32_t* __restrict__ t_hits, const W* __restrict__ hitw,
                          uint8_t* __restrict__ kept, int32_t* __restrict__ seg, int32_t* __restrict__ t_own,
                          uint32_t* __restrict__ ownmask)
{
    const int nt = min(f->n_starts, cap);
    const int lane = threadIdx.x & 31;
    const int j = lane % SEL_G;
    constexpr int GPW = 32 / SEL_G;     // groups per warp
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int t0 = warp * GPW; t0 < nt; t0 += nwarps * GPW) {
        const int t = t0 + lane / SEL_G;
        const bool valid = t < nt;
        const int nh = valid ? t_nhits[t] : 0;
        const bool act = valid && nh >= min_hits;
        W w = 0;
        const int32_t* slot = t_hits;
        int nup = 0;
        if (act) {
            w = sel_weight<W>(nh, t_id[t]);
            slot = t_hits + (int64_t)t * nr;
            nup = t_nup[t];
        }
        const int rounds = act ? (nh + 31) >> 5 : 0;
        const int rmax = __reduce_max_sync(0xffffffffu, rounds);
        int own = 0;
        for (int rd = 0; rd < rmax; rd++) {
            // owned hits in ascending row order, as bits of words [rd][t]
            uint32_t bits = 0u;
#pragma unroll
            for (int i = 0; i < 32 / SEL_G; i++) {
                const int k = (rd << 5) + j + SEL_G * i;
                if (act && k < nh) {
                    const bool o = hitw[trk_hit(slot, nr, nh, nup, k)] == w;
                    own += o;
                    bits |= (uint32_t)o << (k & 31);
                }
            }
#pragma unroll
            for (int d = SEL_G / 2; d > 0; d >>= 1) bits |= __shfl_xor_sync(0xffffffffu, bits, d);
            if (j == 0 && rd < rounds) ownmask[(int64_t)rd * cap + t] = bits;
        }
#pragma unroll
        for (int d = SEL_G / 2; d > 0; d >>= 1) own += __shfl_xor_sync(0xffffffffu, own, d);
        if (j == 0 && valid) {
            uint8_t k = 0;
            if (act && own >= min_owned && 2 * own >= nh) {
                k = 1;
                seg[atomicAdd(&f->n_seg, 1)] = t;
            }
            kept[t] = k;
            t_own[t] = act ? own : 0;
        }
    }
}

// ---------------------------------------------------------------------------
// Cluster rejection before the refit (section "TPC Tracking": the track fit
// rejects clusters).  One thread per kept tracklet carries its state at the
// innermost hit (after all of its hits) with the decision-path helix step up
// through the rows of its hits; an owned hit whose residual passes
// dy^2/vy + dz^2/vz > cut loses its owned bit, so that the assembly leaves it
// out of the track, the refit and the assignment -- unless fewer than
// REJ_MIN_KEEP owned hits of the tracklet would remain.  A refused step ends
// the check of that tracklet.
// ---------------------------------------------------------------------------
constexpr int REJ_MIN_KEEP = 5;
constexpr int REJ_WORDS = 8;            // hits per tracklet <= rows <= 255

__global__ void k_reject(Frame* f, int cap, int nr, int np, float kb, float ivy, float ivz, float cut,
                         const int32_t* __restrict__ seg, const int32_t* __restrict__ t_nhits,
                         const int32_t* __restrict__ t_nup, const int32_t* __restrict__ t_hits,
                         const float* __restrict__ t_bot, const float4* __restrict__ sc,
                         const float* __restrict__ rowtab, uint32_t* __restrict__ ownmask, int32_t* __restrict__ t_own)
{
    if (f->err) return;
    const int nseg = f->n_seg;
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nseg; b += gridDim.x * blockDim.x) {
        const int t = seg[b];
        const int nh = min(t_nhits[t], REJ_WORDS * 32), nup = t_nup[t];
        const int32_t* slot = t_hits + (int64_t)t * nr;
        float st[NST];
#pragma unroll
        for (int i = 0; i < NST; i++) st[i] = t_bot[(int64_t)t * NST + i];
        uint32_t rej[REJ_WORDS];
#pragma unroll
        for (int w = 0; w < REJ_WORDS; w++) rej[w] = 0u;
        int nc = 0;
        uint32_t m = 0u;
        // the next hit's record is loaded a step ahead (two dependent loads per hit)
        float4 cn = nh > 0 ? sc[trk_hit(slot, nr, nh, nup, 0)] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        for (int k = 0; k < nh; k++) {
            if ((k & 31) == 0) m = ownmask[(int64_t)(k >> 5) * cap + t];
            const float4 c = cn;
            if (k + 1 < nh) cn = sc[trk_hit(slot, nr, nh, nup, k + 1)];
            const int r = (int)(sc_plane(c) % (uint32_t)np) % nr;
            if (!prop32_pos(st, rowtab[r * ROWTAB], kb)) break;   // the position only: bit-identical to prop32's
            const float dy = c.x - st[1];
            const float dz = c.y - st[2];
            const float q2 = __fmaf_rn(dy * dy, ivy, (dz * dz) * ivz);
            if (((m >> (k & 31)) & 1u) && q2 > cut) {
                rej[k >> 5] |= 1u << (k & 31);
                nc++;
            }
        }
        if (nc == 0 || t_own[t] - nc < REJ_MIN_KEEP) continue;
        for (int w = 0; w < REJ_WORDS; w++)
            if (rej[w]) ownmask[(int64_t)w * cap + t] &= ~rej[w];
        t_own[t] -= nc;
        atomicAdd(&f->n_rejected, nc);
    }
}

// ---------------------------------------------------------------------------
// a8: cross-sector merger (adjacent sectors of one side, inside one frame,
// and, where the clusters carry z, the same wedge across the central membrane:
// one local frame on both sides, so no rotation; B must continue A outward
// there, since at small dip angles the reversed pair fits as well and would
// close a two-segment cycle.  With drift times the two halves are displaced in
// z by twice the drift over the unknown collision time and are not tried.)
// ---------------------------------------------------------------------------
__device__ __forceinline__ int merge_cell(float zeta, const Frame* f)
{
    return grid_cell(zeta, f->mzmin, f->minv_cs, f->mnz);
}

// merge cells [lo, hi] overlapping the candidate window |z' - z| <= dz (plus
// WIN_MARGIN) of an end at z in sector s
__device__ __forceinline__ void merge_window(float z, float dz, int s, int ns, const Frame* f, int& lo, int& hi)
{
    const float za = fold(z - (dz + WIN_MARGIN), s, ns), zb = fold(z + (dz + WIN_MARGIN), s, ns);
    lo = merge_cell(fminf(za, zb), f);
    hi = merge_cell(fmaxf(za, zb), f);
}

// global sector index (frame * n_sectors + sector) of a segment's start hit
__device__ __forceinline__ int seg_gsector(const float4* sc, const int32_t* t_start, const int32_t* seg, int a, int nr)
{
    return (int)(sc_plane(sc[t_start[seg[a]]]) / (uint32_t)nr);
}

__global__ void k_seg_keys(const Frame* __restrict__ f, int ns, int nr, const int32_t* __restrict__ seg,
                           const float4* __restrict__ sc, const int32_t* __restrict__ t_start,
                           const float* __restrict__ t_top, const float* __restrict__ t_bot,
                           uint32_t* __restrict__ cntb, uint32_t* __restrict__ cntt, uint32_t* __restrict__ keyb,
                           uint32_t* __restrict__ keyt, uint32_t* __restrict__ slotb, uint32_t* __restrict__ slott)
{
    const int nseg = f->n_seg;
    const int mnz = f->mnz;
    for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < nseg; a += gridDim.x * blockDim.x) {
        const int t = seg[a];
        const int gs = seg_gsector(sc, t_start, seg, a, nr);
        const int s = gs % ns;
        const uint32_t kb = (uint32_t)gs * mnz + merge_cell(fold(t_bot[(int64_t)t * NST + 2], s, ns), f);
        const uint32_t kt = (uint32_t)gs * mnz + merge_cell(fold(t_top[(int64_t)t * NST + 2], s, ns), f);
        keyb[a] = kb;
        keyt[a] = kt;
        slotb[a] = atomicAdd(&cntb[kb], 1u);
        slott[a] = atomicAdd(&cntt[kt], 1u);
    }
}

// Merge-candidate record of one segment end, stored in merge-grid order so
// that a candidate scan reads 32 contiguous bytes per candidate: z, tan(lambda),
// q/pT and the variances of the last two (the window test and the screen),
// the start-hit id (tie-break), the tracklet index and x (the outward order
// across the membrane).
struct MergeRec {
    float4 a;   // z, tan(lambda), q/pT, var(tan(lambda))
    float4 b;   // var(q/pT), id (int bits), tracklet (int bits), x
};

__device__ __forceinline__ MergeRec merge_rec(const float* st, int id, int t)
{
    MergeRec m;
    m.a = make_float4(st[2], st[4], st[5], st[6 + 9]);
    m.b = make_float4(st[6 + 14], __int_as_float(id), __int_as_float(t), st[0]);
    return m;
}

__global__ void k_seg_scatter(const Frame* __restrict__ f, const uint32_t* __restrict__ cntb,
                              const uint32_t* __restrict__ cntt, const uint32_t* __restrict__ keyb,
                              const uint32_t* __restrict__ keyt, const uint32_t* __restrict__ slotb,
                              const uint32_t* __restrict__ slott, int32_t* __restrict__ byb, int32_t* __restrict__ byt,
                              const int32_t* __restrict__ seg, const int32_t* __restrict__ t_id,
                              const float* __restrict__ t_top, const float* __restrict__ t_bot,
                              MergeRec* __restrict__ recb, MergeRec* __restrict__ rect)
{
    const int nseg = f->n_seg;
    for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < nseg; a += gridDim.x * blockDim.x) {
        const int t = seg[a], id = t_id[t];
        const uint32_t pb = cntb[keyb[a]] + slotb[a], pt = cntt[keyt[a]] + slott[a];
        byb[pb] = a;
        byt[pt] = a;
        recb[pb] = merge_rec(t_bot + (int64_t)t * NST, id, t);
        rect[pt] = merge_rec(t_top + (int64_t)t * NST, id, t);
    }
}

struct MergeArgs {
    const Frame* f;
    int ns, nr;
    float kb, dz, chi2cut;
    const int32_t* seg;
    const float4* sc;
    const int32_t* t_start;
    const int32_t* t_id;
    const float* t_top;
    const float* t_bot;
    const uint32_t* cntb;   // scanned
    const uint32_t* cntt;
    const int32_t* byb;
    const int32_t* byt;
    int32_t* bnext;
    int32_t* bprev;
    const MergeRec* recb;   // merge-grid order, as byb
    const MergeRec* rect;   // merge-grid order, as byt
    int mirror;             // 1: also the same wedge across the membrane (z given, 36 sectors)
    int prof;
    Frame* fw;
    int2* pairs;            // screened pairs: segment a, inner-end record q (bit 31: direction -1,
                            // bit 30: across the membrane)
    float* pc2;             // their chi2
    unsigned long long* bestA;   // per segment: min (chi2 bits, partner id) as outer piece
    unsigned long long* bestB;   // per segment: the same as inner piece
    int pcap;
};

// Merge screen: tan(lambda), q/pT and their variances are unchanged by the
// rotation and the propagation, and each pull alone bounds the 5-parameter
// chi2 from below; a pair with either pull above twice the cut is skipped
// before the rotation, propagation and Cholesky solve.
__device__ __forceinline__ bool merge_screened(const MergeRec& top, const MergeRec& bot, float lim)
{
    const float dtl = top.a.y - bot.a.y, dqp = top.a.z - bot.a.z;
    return dtl * dtl > lim * (top.a.w + bot.a.w) || dqp * dqp > lim * (top.b.x + bot.b.x);
}

// Lane-local best merge partner: the smallest chi2, ties to the smaller
// start-hit id.  (chi2, id) orders the candidates of one end totally, so the
// warp's reduction gives the same partner for any scan order.
struct MergeBest {
    int q;          // index in merge-grid order, -1: none
    int id;
    float c2;
    __device__ __forceinline__ void offer(int q2, int id2, float c2b)
    {
        if (q < 0 || c2b < c2 || (c2b == c2 && id2 < id)) { q = q2; id = id2; c2 = c2b; }
    }
    __device__ __forceinline__ void warp_reduce()
    {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const int q2 = __shfl_xor_sync(0xffffffffu, q, o);
            const int id2 = __shfl_xor_sync(0xffffffffu, id, o);
            const float c2b = __shfl_xor_sync(0xffffffffu, c2, o);
            if (q2 >= 0) offer(q2, id2, c2b);
        }
    }
};

// The window test, the screen and the chi2 of a pair (outer end of A, inner
// end of B in the neighbouring sector) are symmetric in A and B, so the best
// partner of every outer end and of every inner end come from one list of the
// screened pairs: k_merge_pairs (a warp per outer end, 32 candidate records
// at a time) lists them, k_merge_chi2 (a thread per pair) evaluates each chi2
// once and keeps, per end, the minimum of (chi2 bits, partner id) -- chi2 >= +0
// orders as its bits, so this is the smallest chi2, ties to the smaller id --
// and k_merge_resolve writes the winners.  If the list overflows its capacity,
// k_merge_next / k_merge_prev (one warp per end, chi2 inline) do it instead.
constexpr int MP_U = 4;
constexpr int MP_QMASK = 0x3fffffff;
constexpr int MP_DOWN = (int)0x80000000;
constexpr int MP_MIRROR = 0x40000000;

// the merge directions tried from a sector: the two neighbouring wedges, then
// the mirror sector where enabled
__device__ __forceinline__ int merge_ndir(const MergeArgs& M) { return M.mirror ? 3 : 2; }
__device__ __forceinline__ int merge_dir(int k) { return k == 0 ? 1 : (k == 1 ? -1 : 0); }

// rotation of A's frame into B's for B in direction dir from A
__device__ __forceinline__ void merge_rotation(int dir, float& cs, float& sn)
{
    cs = dir == 0 ? 1.0f : COS20;
    sn = dir > 0 ? SIN20 : (dir < 0 ? -SIN20 : 0.0f);
}

__global__ void __launch_bounds__(128) k_merge_pairs(MergeArgs M)
{
    const int nseg = M.f->n_seg, mnz = M.f->mnz;
    const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    for (int a = blockIdx.x * wpb + (threadIdx.x >> 5); a < nseg; a += gridDim.x * wpb) {
        const int ta = M.seg[a];
        const int gsa = seg_gsector(M.sc, M.t_start, M.seg, a, M.nr);
        const int fr = gsa / M.ns, sa = gsa - fr * M.ns;
        const float* tp = M.t_top + (int64_t)ta * NST;
        MergeRec ra;
        ra.a = make_float4(tp[2], tp[4], tp[5], tp[6 + 9]);
        ra.b = make_float4(tp[6 + 14], 0.0f, 0.0f, tp[0]);
        for (int k = 0; k < merge_ndir(M); k++) {
            const int dir = merge_dir(k);
            const int sb = neighbour_sector(sa, dir, M.ns);
            if (sb < 0) continue;
            const int gsb = fr * M.ns + sb;
            int lo, hi;
            merge_window(ra.a.x, M.dz, sb, M.ns, M.f, lo, hi);   // B's cells, folded by B's side
            const int qb = M.cntb[gsb * mnz + lo], qe = M.cntb[gsb * mnz + hi + 1];
            // MP_U rounds of 32 records per iteration: their loads are in
            // flight together before any is tested (the pair list is order-free)
            for (int q0 = qb; q0 < qe; q0 += 32 * MP_U) {
                MergeRec rr[MP_U];
#pragma unroll
                for (int u = 0; u < MP_U; u++)
                    if (q0 + 32 * u + lane < qe) rr[u] = M.recb[q0 + 32 * u + lane];
                unsigned m[MP_U];
                int tot = 0;
#pragma unroll
                for (int u = 0; u < MP_U; u++) {
                    const int q = q0 + 32 * u + lane;
                    const bool pass = q < qe && (dir != 0 || rr[u].b.w >= ra.b.w) &&
                                      fabsf(rr[u].a.x - ra.a.x) <= M.dz &&
                                      !merge_screened(ra, rr[u], 2.0f * M.chi2cut);
                    m[u] = __ballot_sync(0xffffffffu, pass);
                    tot += __popc(m[u]);
                }
                if (!tot) continue;
                int base = 0;
                if (lane == 0) base = atomicAdd(&M.fw->n_mpairs, tot);
                base = __shfl_sync(0xffffffffu, base, 0);
                const int flag = dir < 0 ? MP_DOWN : (dir == 0 ? MP_MIRROR : 0);
#pragma unroll
                for (int u = 0; u < MP_U; u++) {
                    if ((m[u] >> lane) & 1u) {
                        const int k = base + __popc(m[u] & ((1u << lane) - 1u));
                        if (k < M.pcap) M.pairs[k] = make_int2(a, (q0 + 32 * u + lane) | flag);
                    }
                    base += __popc(m[u]);
                }
            }
        }
    }
}

__device__ __forceinline__ unsigned long long merge_key(float c2, int id)
{
    return ((unsigned long long)__float_as_uint(c2) << 32) | (unsigned long long)(uint32_t)id;
}

__global__ void k_merge_chi2(MergeArgs M)
{
    const int np_ = M.f->n_mpairs;
    if (np_ > M.pcap) return;
    unsigned nchi = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < np_; i += gridDim.x * blockDim.x) {
        const int2 pr = M.pairs[i];
        const int a = pr.x, q = pr.y & MP_QMASK;
        const MergeRec rb = M.recb[q];
        const int ta = M.seg[a], tb = __float_as_int(rb.b.z);
        float cs, sn;
        merge_rotation(pr.y < 0 ? -1 : ((pr.y & MP_MIRROR) ? 0 : 1), cs, sn);
        const float c2 = merge_chi2(M.t_top + (int64_t)ta * NST, M.t_bot + (int64_t)tb * NST, cs, sn, M.kb);
        nchi++;
        M.pc2[i] = c2;
        if (c2 < M.chi2cut) {
            atomicMin(&M.bestA[a], merge_key(c2, __float_as_int(rb.b.y)));
            atomicMin(&M.bestB[M.byb[q]], merge_key(c2, M.t_id[ta]));
        }
    }
    if (M.prof) {
        nchi = __reduce_add_sync(0xffffffffu, nchi);
        if ((threadIdx.x & 31) == 0 && nchi) atomicAdd(&M.fw->w_merge, (unsigned long long)nchi);
    }
}

__global__ void k_merge_resolve(MergeArgs M)
{
    const int np_ = M.f->n_mpairs;
    if (np_ > M.pcap) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < np_; i += gridDim.x * blockDim.x) {
        const float c2 = M.pc2[i];
        if (!(c2 < M.chi2cut)) continue;
        const int2 pr = M.pairs[i];
        const int a = pr.x, q = pr.y & MP_QMASK;
        const int b = M.byb[q];
        if (M.bestA[a] == merge_key(c2, __float_as_int(M.recb[q].b.y))) M.bnext[a] = b;
        if (M.bestB[b] == merge_key(c2, M.t_id[M.seg[a]])) M.bprev[b] = a;
    }
}

// Fallback: one warp per segment end: the lanes read 32 consecutive candidate
// records of the window at a time, screen them, and evaluate the chi2 of
// those left.

// best B (outer piece) for every A: A's outer end against B's inner end
__global__ void __launch_bounds__(128) k_merge_next(MergeArgs M)
{
    if (M.f->n_mpairs <= M.pcap) return;      // the pair list held every screened pair
    const int nseg = M.f->n_seg, mnz = M.f->mnz;
    const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    unsigned nchi = 0;
    for (int a = blockIdx.x * wpb + (threadIdx.x >> 5); a < nseg; a += gridDim.x * wpb) {
        const int ta = M.seg[a];
        const int gsa = seg_gsector(M.sc, M.t_start, M.seg, a, M.nr);
        const int fr = gsa / M.ns, sa = gsa - fr * M.ns;
        float top[NST];
#pragma unroll
        for (int i = 0; i < NST; i++) top[i] = M.t_top[(int64_t)ta * NST + i];
        const MergeRec ra = merge_rec(top, 0, ta);
        MergeBest b{-1, 0, 0.0f};
        for (int k = 0; k < merge_ndir(M); k++) {
            const int dir = merge_dir(k);
            const int sb = neighbour_sector(sa, dir, M.ns);
            if (sb < 0) continue;
            const int gsb = fr * M.ns + sb;
            float cs, sn;
            merge_rotation(dir, cs, sn);
            int lo, hi;
            merge_window(top[2], M.dz, sb, M.ns, M.f, lo, hi);   // B's cells, folded by B's side
            const int qb = M.cntb[gsb * mnz + lo], qe = M.cntb[gsb * mnz + hi + 1];
            for (int q = qb + lane; q < qe; q += 32) {
                const MergeRec rb = M.recb[q];
                if (dir == 0 && !(rb.b.w >= top[0])) continue;
                if (!(fabsf(rb.a.x - top[2]) <= M.dz)) continue;
                if (merge_screened(ra, rb, 2.0f * M.chi2cut)) continue;
                const int tb = __float_as_int(rb.b.z);
                const float c2 = merge_chi2(top, M.t_bot + (int64_t)tb * NST, cs, sn, M.kb);
                nchi++;
                if (c2 < M.chi2cut) b.offer(q, __float_as_int(rb.b.y), c2);
            }
        }
        b.warp_reduce();
        if (lane == 0) M.bnext[a] = b.q < 0 ? -1 : M.byb[b.q];
    }
    if (M.prof) {
        nchi = __reduce_add_sync(0xffffffffu, nchi);
        if (lane == 0 && nchi) atomicAdd(&M.fw->w_merge, (unsigned long long)nchi);
    }
}

// best A (inner piece) for every B
__global__ void __launch_bounds__(128) k_merge_prev(MergeArgs M)
{
    if (M.f->n_mpairs <= M.pcap) return;
    const int nseg = M.f->n_seg, mnz = M.f->mnz;
    const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    for (int b = blockIdx.x * wpb + (threadIdx.x >> 5); b < nseg; b += gridDim.x * wpb) {
        const int tb = M.seg[b];
        const int gsb = seg_gsector(M.sc, M.t_start, M.seg, b, M.nr);
        const int fr = gsb / M.ns, sb = gsb - fr * M.ns;
        float bot[NST];
#pragma unroll
        for (int i = 0; i < NST; i++) bot[i] = M.t_bot[(int64_t)tb * NST + i];
        const MergeRec rb = merge_rec(bot, 0, tb);
        MergeBest best{-1, 0, 0.0f};
        for (int k = 0; k < merge_ndir(M); k++) {
            const int d = merge_dir(k);
            const int sa = neighbour_sector(sb, d, M.ns);
            if (sa < 0) continue;
            const int gsa = fr * M.ns + sa;
            // seen from A, B lies in direction -d
            float cs, sn;
            merge_rotation(-d, cs, sn);
            int lo, hi;
            merge_window(bot[2], M.dz, sa, M.ns, M.f, lo, hi);
            const int qb = M.cntt[gsa * mnz + lo], qe = M.cntt[gsa * mnz + hi + 1];
            for (int q = qb + lane; q < qe; q += 32) {
                const MergeRec ra = M.rect[q];
                if (d == 0 && !(bot[0] >= ra.b.w)) continue;
                if (!(fabsf(bot[2] - ra.a.x) <= M.dz)) continue;
                if (merge_screened(ra, rb, 2.0f * M.chi2cut)) continue;
                const int ta = __float_as_int(ra.b.z);
                const float c2 = merge_chi2(M.t_top + (int64_t)ta * NST, bot, cs, sn, M.kb);
                if (c2 < M.chi2cut) best.offer(q, __float_as_int(ra.b.y), c2);
            }
        }
        best.warp_reduce();
        if (lane == 0) M.bprev[b] = best.q < 0 ? -1 : M.byt[best.q];
    }
}

__global__ void k_merge_link(const Frame* __restrict__ f, const int32_t* __restrict__ bnext,
                             const int32_t* __restrict__ bprev, int32_t* __restrict__ snext, int32_t* __restrict__ sprev)
{
    const int nseg = f->n_seg;
    for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < nseg; a += gridDim.x * blockDim.x) {
        const int b = bnext[a];
        if (b >= 0 && bprev[b] == a) {
            snext[a] = b;
            sprev[b] = a;
        }
    }
}

__global__ void k_merge_cycles(const Frame* __restrict__ f, const int32_t* __restrict__ sprev, uint8_t* __restrict__ bad)
{
    const int nseg = f->n_seg;
    for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < nseg; a += gridDim.x * blockDim.x) {
        int c = a, steps = 0;
        while (sprev[c] >= 0 && steps <= MAX_CHAIN) { c = sprev[c]; steps++; }
        bad[a] = sprev[c] >= 0 ? 1 : 0;
    }
}

__global__ void k_merge_fix(const Frame* __restrict__ f, const int32_t* __restrict__ snext,
                            const int32_t* __restrict__ sprev, const uint8_t* __restrict__ bad,
                            int32_t* __restrict__ next2, int32_t* __restrict__ prev2, const int32_t* __restrict__ seg,
                            const int32_t* __restrict__ t_id, uint32_t* __restrict__ headmark)
{
    const int nseg = f->n_seg;
    for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < nseg; a += gridDim.x * blockDim.x) {
        int nx = snext[a], pv = sprev[a];
        if (bad[a]) { nx = -1; pv = -1; }
        if (nx >= 0 && bad[nx]) nx = -1;
        if (pv >= 0 && bad[pv]) pv = -1;
        next2[a] = nx;
        prev2[a] = pv;
        if (pv < 0) headmark[t_id[seg[a]]] = 1u;
    }
}

// ---------------------------------------------------------------------------
// track assembly: rank of each chain head, cluster counts, cluster lists
// ---------------------------------------------------------------------------
struct AsmArgs {
    Frame* f;
    int nr, np, n, cap_tracks, cap_clus, ntcap;
    const int32_t* seg;
    const int32_t* next2;
    const int32_t* prev2;
    const int32_t* t_start;
    const int32_t* t_id;
    const int32_t* t_nhits;
    const int32_t* t_nup;
    const int32_t* t_hits;
    const float4* sc;
    const uint32_t* ownmask;    // [word][ntcap]: owned hits of each tracklet (selector)
    const uint32_t* headmark;   // scanned: rank of each head's start id
    uint32_t* tcount;           // [ntcap + 1]
    int32_t* thead;
    int32_t* ttail;
    int32_t* clus_offset;
    int32_t* nclus;
    int32_t* clus_index;
    int32_t* assign;
    int32_t* frame;             // nullable
    const float* rowtab;
    float4* tcl;                // [clusters in tracks]: y, z, row x, sector (int bits)
    const int32_t* t_own;       // owned hits per tracklet (selector)
    int32_t* segoff;            // per segment: first cluster within its track
    int32_t* segrank;           // per segment: its track, -1 if in none
};

// per track head: walk the chain, give every segment its track and its
// first cluster within the track (owned hits of the segments before it)
__global__ void k_track_count(AsmArgs A)
{
    const int nseg = A.f->n_seg;
    for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < nseg; a += gridDim.x * blockDim.x) {
        if (A.prev2[a] >= 0) continue;
        const int rank = (int)A.headmark[A.t_id[A.seg[a]]];
        int cnt = 0, tail = a, steps = 0;
        for (int b = a; b >= 0 && steps <= MAX_CHAIN; b = A.next2[b], steps++) {
            A.segoff[b] = cnt;
            A.segrank[b] = rank;
            cnt += A.t_own[A.seg[b]];
            tail = b;
        }
        A.tcount[rank] = (uint32_t)cnt;
        A.thead[rank] = a;
        A.ttail[rank] = A.seg[tail];
    }
}

__device__ __forceinline__ bool asm_overflow(const AsmArgs& A, int T, uint32_t total)
{
    return T > A.cap_tracks || total > (uint32_t)A.cap_clus;
}

// per track: offsets, sizes, frame
__global__ void k_track_fill(AsmArgs A)
{
    const int T = (int)A.headmark[A.n];
    const uint32_t total = A.tcount[A.ntcap];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        A.f->n_tracks = T;
        A.f->n_clus = (int)total;
        if (asm_overflow(A, T, total)) atomicExch(&A.f->err, TPC_ERR_CAPACITY);
    }
    if (asm_overflow(A, T, total)) return;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < T; r += gridDim.x * blockDim.x) {
        const int a = A.thead[r];
        const uint32_t off = A.tcount[r];
        const uint32_t end = A.tcount[r + 1];
        A.clus_offset[r] = (int)off;
        if (r == T - 1) A.clus_offset[T] = (int)end;
        A.nclus[r] = (int)(end - off);
        if (A.frame) A.frame[r] = (int)(sc_plane(A.sc[A.t_start[A.seg[a]]]) / (uint32_t)A.np);
    }
}

// one warp per segment: its owned hits, in ascending row, at the segment's
// place in its track's cluster list (ballot compaction keeps the order)
__global__ void k_seg_fill(AsmArgs A)
{
    const int T = (int)A.headmark[A.n];
    const uint32_t total = A.tcount[A.ntcap];
    if (asm_overflow(A, T, total)) return;
    const int nseg = A.f->n_seg;
    const int lane = threadIdx.x & 31;
    const int nwarp = (gridDim.x * blockDim.x) >> 5;
    for (int b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; b < nseg; b += nwarp) {
        const int r = A.segrank[b];
        if (r < 0) continue;
        const int t = A.seg[b];
        const int nh = A.t_nhits[t], nup = A.t_nup[t];
        const int32_t* slot = A.t_hits + (int64_t)t * A.nr;
        uint32_t o = A.tcount[r] + (uint32_t)A.segoff[b];
        // SF_U rounds of 32 hits at a time: their owned-hit words, slot reads
        // and cluster records are each in flight together
        constexpr int SF_U = 4;
        for (int k0 = 0; k0 < nh; k0 += 32 * SF_U) {
            unsigned m[SF_U];
            int hh[SF_U];
            float4 c[SF_U];
#pragma unroll
            for (int u = 0; u < SF_U; u++) {
                const int kk = k0 + 32 * u;
                m[u] = kk < nh ? A.ownmask[(int64_t)(kk >> 5) * A.ntcap + t] : 0u;   // bits past nh are 0
            }
#pragma unroll
            for (int u = 0; u < SF_U; u++) hh[u] = ((m[u] >> lane) & 1u) ? trk_hit(slot, A.nr, nh, nup, k0 + 32 * u + lane) : -1;
#pragma unroll
            for (int u = 0; u < SF_U; u++)
                if (hh[u] >= 0) c[u] = A.sc[hh[u]];
#pragma unroll
            for (int u = 0; u < SF_U; u++) {
                if (hh[u] >= 0) {
                    const uint32_t q = o + (uint32_t)__popc(m[u] & ((1u << lane) - 1u));
                    const int id = sc_id(c[u]);
                    const int pl = (int)(sc_plane(c[u]) % (uint32_t)A.np);
                    const int sec = pl / A.nr;
                    A.tcl[q] = make_float4(c[u].x, c[u].y, A.rowtab[(pl - sec * A.nr) * ROWTAB], __int_as_float(sec));
                    A.clus_index[q] = id;
                    A.assign[id] = r;
                }
                o += (uint32_t)__popc(m[u]);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Track-based cluster attachment (paper, section "TPC Data Compression":
// tubes around the tracks, adjacency to the highest-pT track, protection by
// good tracks, removal of the rest of the attached or adjacent clusters).
// The tube follows each sector piece: its TrackletConstructor state at its
// innermost hit (after all of its hits) is propagated row by row through the
// rows its hits span; all of it is binary32 on the decision path, so the
// flags are the same on any hardware that rounds each operation.
// ---------------------------------------------------------------------------
struct AttachArgs {
    const Frame* f;
    const FrameGrid* fg;
    int nr, np, ns, n;
    float kb, R, R2, qmax;
    const int32_t* seg;
    const int32_t* segrank;     // track of each segment (-1: none)
    const int32_t* thead;       // innermost segment of each track
    const int32_t* t_nhits;
    const int32_t* t_nup;
    const int32_t* t_hits;
    const float* t_bot;         // [slot][NST] state at the innermost hit
    const float4* sc;
    const uint32_t* cstart;
    const float* rowtab;
    const int32_t* assign;
    unsigned long long* akey;   // [n] best adjacency key (0: none)
    unsigned long long* tkey;   // [tracks] adjacency key of each track
    uint8_t* aprot;             // [n] inside the tube of a good track
    uint8_t* flags;
    int32_t* adjacent;
    const uint8_t* tgood;       // [tracks] good: pT cut passed and not a secondary looper leg
};

__device__ __forceinline__ float track_abs_qpt(const AttachArgs& A, int tr)
{
    return fabsf(A.t_bot[(int64_t)A.seg[A.thead[tr]] * NST + 5]);
}

// the clusters of the traced point's row inside the tube disc
__device__ __forceinline__ void tube_visit(const AttachArgs& A, const FrameGrid& G, int s, int r, float yp, float zp,
                                           unsigned long long key, bool good)
{
    const WinCells W = window_cells(G, s * A.nr + r, s, A.ns, A.rowtab, r, A.f->ny, yp, zp, A.R, A.R);
    for (int k = 0; k < W.nzc; k++) {
        int qb, qe;
        W.range(A.cstart, k, qb, qe);
        for (int q = qb; q < qe; q++) {
            const float4 c = A.sc[q];
            const float dy = c.x - yp;
            const float dz = c.y - zp;
            if (!(fabsf(dy) <= A.R) || !(fabsf(dz) <= A.R)) continue;
            const float d2 = __fmaf_rn(dy, dy, dz * dz);
            if (!(d2 < A.R2)) continue;
            const int id = sc_id(c);
            if (good) A.aprot[id] = 1;     // every writer stores 1
            if (A.assign[id] < 0) atomicMax(&A.akey[id], key);
        }
    }
}

// The tube's points of a segment come from a chain of helix steps
// (sequential, cheap); each point's cell scan is a few dependent loads of its
// plane's cells and clusters.  Scanned in segment order those loads jump
// between planes and miss the L2, so the points are first bucketed by plane
// (a counting sort: one pass of the chains counts the points per plane, a
// scan gives the bucket starts, a second pass stores each point -- y, z and
// its track's adjacency key -- in its bucket) and then scanned one thread
// per point in plane order.  Points beyond the buffers' capacity are scanned
// by the tracing thread itself.  The marks are order-free (atomicMax, stores
// of 1), so none of this changes a result.
struct SegInfo {
    int s, fr, r_lo, r_hi, tr;
    unsigned long long key;
    bool good;
};

__device__ __forceinline__ bool seg_info(const AttachArgs& A, int b, SegInfo& I)
{
    const int tr = A.segrank[b];
    if (tr < 0) return false;
    const int t = A.seg[b];
    const int nh = A.t_nhits[t], nup = A.t_nup[t];
    if (nh <= 0) return false;
    I.tr = tr;
    const int32_t* slot = A.t_hits + (int64_t)t * A.nr;
    const uint32_t pg = sc_plane(A.sc[trk_hit(slot, A.nr, nh, nup, 0)]);
    I.fr = (int)(pg / (uint32_t)A.np);
    const int pl = (int)(pg - (uint32_t)I.fr * A.np);
    I.s = pl / A.nr;
    I.r_lo = pl - I.s * A.nr;
    I.r_hi = (int)(sc_plane(A.sc[trk_hit(slot, A.nr, nh, nup, nh - 1)]) % (uint32_t)A.np) - I.s * A.nr;
    const float aq = track_abs_qpt(A, tr);
    I.good = A.tgood[tr] != 0;
    I.key = ((unsigned long long)(0xFFFFFFFFu - __float_as_uint(aq)) << 32) |
            (unsigned long long)(0xFFFFFFFFu - (uint32_t)tr);
    return true;
}

// the track of an adjacency key is its low word (0xFFFFFFFF - track)
__device__ __forceinline__ bool key_good(const AttachArgs& A, unsigned long long key)
{
    return A.tgood[0xFFFFFFFFu - (uint32_t)(key & 0xFFFFFFFFull)] != 0;
}

// per segment: +1 at the plane of its lowest row, -1 past its highest (a
// difference array over the rows of each sector; k_attach_rowsum turns it
// into the number of segments spanning each plane: the bucket sizes).  Each
// plane's bucket is split in PSPLIT sub-buckets, segment b filling sub-bucket
// b mod PSPLIT, so that the bucket reservations of the segments crossing a
// plane spread over PSPLIT counters; the sub-buckets of a plane are adjacent,
// so the scan still visits the points in plane order.
__global__ void k_attach_span(AttachArgs A, uint32_t* __restrict__ dcnt)
{
    if (A.f->err) return;
    const int nseg = A.f->n_seg;
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nseg; b += gridDim.x * blockDim.x) {
        SegInfo I;
        if (!seg_info(A, b, I)) continue;
        if (A.thead[I.tr] == b) A.tkey[I.tr] = I.key;     // written by the track's innermost segment
        const uint32_t base = (uint32_t)I.fr * (uint32_t)A.np + (uint32_t)(I.s * A.nr);
        const uint32_t k = (uint32_t)b % PSPLIT;
        atomicAdd(&dcnt[(base + (uint32_t)I.r_lo) * PSPLIT + k], 1u);
        if (I.r_hi + 1 < A.nr) atomicAdd(&dcnt[(base + (uint32_t)(I.r_hi + 1)) * PSPLIT + k], 0xFFFFFFFFu);
    }
}

// one thread per (frame, sector, sub-bucket): running sum over its rows
__global__ void k_attach_rowsum(uint32_t* __restrict__ dcnt, int nseq, int nr, const Frame* __restrict__ f)
{
    if (f->err) return;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nseq; q += gridDim.x * blockDim.x) {
        const int64_t fs = q / PSPLIT, k = q % PSPLIT;
        uint32_t c = 0;
        for (int r = 0; r < nr; r++) {
            const int64_t e = (fs * nr + r) * PSPLIT + k;
            c += dcnt[e];
            dcnt[e] = c;
        }
    }
}

// One thread per segment: the chain of points from the inner-end state, each
// stored in its plane's bucket (cursor[plane]: the bucket's next free
// position) or scanned here when the buffers are full (cap == 0: always).
// The chain runs in blocks of ATT_U rows: the loop-carried quantities (x,
// sin phi) first, then the ATT_U steps' square roots and divisions side by
// side, then the checks and the y, z sums in row order.  Each step is the
// helix step of the position -- sin phi linear in x, dy = dx (s1 + s2) / (c1 +
// c2), arc = signed chord * asin(u)/u by its series to u^6 with u = k chord
// / 2, dz = tan(lambda) arc, refused when |sin phi| reaches SNP_MAX or |u| >
// U_MAX -- with the operations of a row-by-row chain in the same order, so
// the points are that chain's.
constexpr int ATT_U = 4;

// bucket record of a point: its plane and its track
__device__ __forceinline__ unsigned long long point_meta(uint32_t plane, int tr)
{
    return ((unsigned long long)plane << 32) | (unsigned long long)(uint32_t)tr;
}

__global__ void __launch_bounds__(128, 8) k_attach_trace(AttachArgs A, uint32_t* __restrict__ cursor,
                                                         float2* __restrict__ pts,
                                                         unsigned long long* __restrict__ pmeta, uint32_t cap)
{
    if (A.f->err) return;
    const int nseg = A.f->n_seg;
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nseg; b += gridDim.x * blockDim.x) {
        SegInfo I;
        if (!seg_info(A, b, I)) continue;
        const float* bs = A.t_bot + (int64_t)A.seg[b] * NST;
        float b0[6];
#pragma unroll
        for (int i = 0; i < 6; i++) b0[i] = bs[i];
        int r_b = -1;
        for (int r = 0; r < A.nr; r++)
            if (A.rowtab[r * ROWTAB] == b0[0]) { r_b = r; break; }
        if (r_b < 0) continue;
        const uint32_t pbase = (uint32_t)I.fr * (uint32_t)A.np + (uint32_t)(I.s * A.nr);
        const uint32_t sub = (uint32_t)b % PSPLIT;
        const FrameGrid G = A.fg[I.fr];
        // store the points of rows rv[] (-1: none) in their buckets, the
        // ATT_U bucket reservations in flight together; past the capacity the
        // point is scanned here
        auto emit = [&](const int* rv, const float* yv, const float* zv) {
            uint32_t qv[ATT_U];
#pragma unroll
            for (int i = 0; i < ATT_U; i++)
                qv[i] = (cap && rv[i] >= I.r_lo && rv[i] <= I.r_hi)
                            ? atomicAdd(&cursor[(pbase + (uint32_t)rv[i]) * PSPLIT + sub], 1u) : 0xFFFFFFFFu;
#pragma unroll
            for (int i = 0; i < ATT_U; i++) {
                if (rv[i] < I.r_lo || rv[i] > I.r_hi) continue;
                if (qv[i] < cap) {
                    pts[qv[i]] = make_float2(yv[i], zv[i]);
                    pmeta[qv[i]] = point_meta(pbase + (uint32_t)rv[i], I.tr);
                } else {
                    tube_visit(A, G, I.s, rv[i], yv[i], zv[i], I.key, I.good);
                }
            }
        };
        {
            int rv[ATT_U];
            float yv[ATT_U], zv[ATT_U];
#pragma unroll
            for (int i = 0; i < ATT_U; i++) { rv[i] = -1; yv[i] = 0.0f; zv[i] = 0.0f; }
            rv[0] = r_b; yv[0] = b0[1]; zv[0] = b0[2];
            emit(rv, yv, zv);
        }
        const float k = A.kb * b0[5];
        const float hk = 0.5f * k;
        const float t = b0[4];
#pragma unroll 1
        for (int dir = 1; dir >= -1; dir -= 2) {
            const int rlast = dir > 0 ? I.r_hi : I.r_lo;     // inclusive
            float x = b0[0], y = b0[1], z = b0[2], sn = b0[3];
            int r = r_b;
            while (dir > 0 ? r < rlast : r > rlast) {
                float xs[ATT_U], sv[ATT_U + 1], cv[ATT_U + 1], dxv[ATT_U];
                sv[0] = sn;
                float xc = x;
#pragma unroll
                for (int i = 0; i < ATT_U; i++) {
                    int rr = r + dir * (i + 1);
                    rr = dir > 0 ? min(rr, rlast) : max(rr, rlast);      // rows past the end: computed, not used
                    xs[i] = A.rowtab[rr * ROWTAB];
                    dxv[i] = xs[i] - xc;
                    sv[i + 1] = __fmaf_rn(k, dxv[i], sv[i]);
                    xc = xs[i];
                }
#pragma unroll
                for (int i = 0; i <= ATT_U; i++) cv[i] = __fsqrt_rn((1.0f - sv[i]) * (1.0f + sv[i]));
                int rv[ATT_U];
                float yv[ATT_U], zv[ATT_U];
                bool stop = false;
#pragma unroll
                for (int i = 0; i < ATT_U; i++) {
                    rv[i] = -1;
                    yv[i] = 0.0f;
                    zv[i] = 0.0f;
                    const int rr = r + dir * (i + 1);
                    if (stop || (dir > 0 ? rr > rlast : rr < rlast)) {
                        stop = true;
                        continue;
                    }
                    const float dx = dxv[i];
                    const float dy = dx * __fdiv_rn(sv[i] + sv[i + 1], cv[i] + cv[i + 1]);
                    float chord = __fsqrt_rn(__fmaf_rn(dx, dx, dy * dy));
                    if (dx < 0.0f) chord = -chord;
                    const float u = hk * chord;
                    if (!(fabsf(sv[i]) < SNP_MAX) || !(fabsf(sv[i + 1]) < SNP_MAX) || !(fabsf(u) <= U_MAX)) {
                        stop = true;
                        r = rlast;                       // the chain ends here
                        continue;
                    }
                    const float u2 = u * u;
                    const float arc = chord * __fmaf_rn(u2, __fmaf_rn(u2, __fmaf_rn(u2, AS3, AS2), AS1), 1.0f);
                    y = y + dy;
                    z = z + arc * t;
                    rv[i] = rr;
                    yv[i] = y;
                    zv[i] = z;
                }
                emit(rv, yv, zv);
                if (r == rlast) break;
                r += dir * ATT_U;
                x = xs[ATT_U - 1];
                sn = sv[ATT_U];
            }
        }
    }
}

// per (plane, sub-bucket): mark the positions that no point filled (rows the
// chains did not reach)
__global__ void k_attach_holes(const uint32_t* __restrict__ start, const uint32_t* __restrict__ cursor, int P,
                               unsigned long long* __restrict__ pmeta, uint32_t cap, const Frame* __restrict__ f)
{
    if (f->err) return;
    for (int gp = blockIdx.x * blockDim.x + threadIdx.x; gp < P; gp += gridDim.x * blockDim.x) {
        const uint32_t e = min(start[gp + 1], cap);
        for (uint32_t q = cursor[gp]; q < e; q++) pmeta[q] = ~0ull;
    }
}

// One thread per bucket position, in plane order (start[P]: the positions
// in use).
__global__ void k_attach_visit(AttachArgs A, const uint32_t* __restrict__ start, int P,
                               const float2* __restrict__ pts, const unsigned long long* __restrict__ pmeta,
                               uint32_t cap)
{
    if (A.f->err) return;
    const uint32_t total = min(start[P], cap);
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < total; q += gridDim.x * blockDim.x) {
        const unsigned long long meta = pmeta[q];
        if (meta == ~0ull) continue;     // a row the chain did not reach
        const uint32_t gp = (uint32_t)(meta >> 32);
        const unsigned long long key = A.tkey[(uint32_t)meta];
        const int fr = (int)(gp / (uint32_t)A.np);
        const int pl = (int)(gp - (uint32_t)fr * A.np);
        const int s = pl / A.nr;
        const float2 pt = pts[q];
        tube_visit(A, A.fg[fr], s, pl - s * A.nr, pt.x, pt.y, key, key_good(A, key));
    }
}

// ---------------------------------------------------------------------------
// Looper legs (sections "Introduction" and "TPC Data Compression": a low-pT
// particle leaves several legs; the secondary legs of loopers below
// 200 MeV/c are removable).  In continuous read-out every leg of a particle
// carries the drift offset of its collision, so in the tracker's coordinates
// its legs lie on one helix.  All binary32 on the decision path:
//   - candidate: |q/pT| >= qmin of the inner-end state of the track's
//     innermost piece; circle: k = kb q/pT, local centre (x - sinphi/k,
//     y + cosphi/k) and point (x, y) rotated by the sector angle, radius
//     R = 1/|k| known to s_R = R sqrt(C_qq)/|q/pT| (legs above LOOP_SRMAX are
//     not grouped); a = |tanl| R, the z advance per radian; sense = sign of
//     k tanl (the same on every leg: the tracker fits an inward leg in the
//     direction of increasing x, which flips k and tanl together);
//   - candidates i < j of one frame are legs of one particle when, with
//     s = sqrt(s_Ri^2 + s_Rj^2): |R_i - R_j| < 2s + 1, |C_i - C_j| < 2s + 2,
//     | |tanl_i| - |tanl_j| | < 0.05, |z_j - z_i| <= z_max, equal senses
//     when both |tanl| >= 0.02 (else either sense is tried), and the z
//     difference matches the advance over the turning angle dpsi between
//     the points (own arctangent) plus whole turns (|m| <= 10):
//     |w - 2 pi a m| < 3 + |tanl| (|dpsi| + 2 pi |m|) 2s, w = sense dz - a dpsi;
//   - groups: connected components (union-find, the larger root linked under
//     the smaller, so a group's root is its smallest track); legs numbered in
//     ascending s z (the earliest leg of the drift first), ties by track.
// ---------------------------------------------------------------------------
struct LoopCand {
    float R, sr, cx, cy, px, py, z, tl, a, sz;
    int sense, frame;       // frame -1: not a candidate
};
static_assert(sizeof(LoopCand) == 48, "LoopCand layout");

constexpr float LOOP_SRMAX = 5.0f;
constexpr float LOOP_DR = 1.0f;
constexpr float LOOP_DC = 2.0f;
constexpr float LOOP_NSIG = 2.0f;
constexpr float LOOP_DTGL = 0.05f;
constexpr float LOOP_DZ = 3.0f;
constexpr float LOOP_TLSENSE = 0.02f;
constexpr float LOOP_TURNS = 10.0f;
constexpr float PI_F = 3.14159265358979323846f;
constexpr float TWO_PI_F = 6.28318530717958647692f;
constexpr float HALF_PI_F = 1.57079632679489661923f;
constexpr int UF_MAX_STEPS = 1 << 20;

// cos and sin of the sector angles (s mod 18) * 20 + 10 degrees
__constant__ float c_sec_cos[18] = {
    0.98480775301220805936f, 0.86602540378443864676f, 0.64278760968653932632f, 0.34202014332566873304f,
    0.0f, -0.34202014332566873304f, -0.64278760968653932632f, -0.86602540378443864676f,
    -0.98480775301220805936f, -0.98480775301220805936f, -0.86602540378443864676f, -0.64278760968653932632f,
    -0.34202014332566873304f, 0.0f, 0.34202014332566873304f, 0.64278760968653932632f,
    0.86602540378443864676f, 0.98480775301220805936f};
__constant__ float c_sec_sin[18] = {
    0.17364817766693034885f, 0.5f, 0.76604444311897803520f, 0.93969262078590838405f,
    1.0f, 0.93969262078590838405f, 0.76604444311897803520f, 0.5f,
    0.17364817766693034885f, -0.17364817766693034885f, -0.5f, -0.76604444311897803520f,
    -0.93969262078590838405f, -1.0f, -0.93969262078590838405f, -0.76604444311897803520f,
    -0.5f, -0.17364817766693034885f};

// atan(x), |x| <= 1: two half-angle reductions atan(x) = 2 atan(x / (1 +
// sqrt(1 + x^2))) bring the argument below tan(pi/16), where the Maclaurin
// series of atan to x^15 is exact in binary32 (next term < 1e-13)
__device__ __forceinline__ float atan_unit(float x)
{
    const float x1 = __fdiv_rn(x, 1.0f + __fsqrt_rn(__fmaf_rn(x, x, 1.0f)));
    const float x2 = __fdiv_rn(x1, 1.0f + __fsqrt_rn(__fmaf_rn(x1, x1, 1.0f)));
    const float t2 = x2 * x2;
    float p = __fmaf_rn(t2, -0.066666666666666666667f, 0.076923076923076923077f);
    p = __fmaf_rn(t2, p, -0.090909090909090909091f);
    p = __fmaf_rn(t2, p, 0.11111111111111111111f);
    p = __fmaf_rn(t2, p, -0.14285714285714285714f);
    p = __fmaf_rn(t2, p, 0.2f);
    p = __fmaf_rn(t2, p, -0.33333333333333333333f);
    const float a = __fmaf_rn(x2 * t2, p, x2);
    return 4.0f * a;
}

__device__ __forceinline__ float atan2_own(float y, float x)
{
    if (x == 0.0f && y == 0.0f) return 0.0f;
    if (fabsf(y) <= fabsf(x)) {
        float a = atan_unit(__fdiv_rn(y, x));
        if (x < 0.0f) a = y >= 0.0f ? a + PI_F : a - PI_F;
        return a;
    }
    const float a = atan_unit(__fdiv_rn(x, y));
    return (y > 0.0f ? HALF_PI_F : -HALF_PI_F) - a;
}

struct LoopArgs {
    const Frame* f;
    int ns, nr, np, nfr, cap;
    float kb, qmin, zmax;
    const int32_t* seg;
    const int32_t* thead;
    const int32_t* t_start;
    const float* t_bot;
    const float4* sc;
    LoopCand* cand;
    int32_t* par;
    uint32_t* bincnt;       // [nfr * LOOP_NBIN + 1]
    int32_t* sorted;        // candidates in (frame, bin) order
    uint32_t* gcnt;         // [cap + 1] members per root, then scanned
    int32_t* glist;
    int32_t* group;
    int32_t* leg;
    int* err;
};

// Centre cells of LOOP_CW cm from -LOOP_G LOOP_CW / 2 (clamped at the grid
// edges: monotone in the coordinate).  A pair needs centres closer than
// 2 sqrt(2) LOOP_SRMAX + LOOP_DC < LOOP_CW, so its cells are neighbours.
constexpr float LOOP_CW = 17.0f;
static_assert(2.0f * 1.41421357f * LOOP_SRMAX + LOOP_DC < LOOP_CW, "centre cells hold the pair tolerance");
__device__ __forceinline__ int loop_cell(float c)
{
    const float t = (c + 0.5f * LOOP_G * LOOP_CW) * (1.0f / LOOP_CW);
    return (int)fminf(fmaxf(t, 0.0f), (float)(LOOP_G - 1));   // NaN -> 0
}
__device__ __forceinline__ int loop_bin(const LoopCand& c)
{
    return c.frame * LOOP_NBIN + loop_cell(c.cy) * LOOP_G + loop_cell(c.cx);
}

// per track: its candidate record (or none), group and leg -1
__global__ void k_loop_cand(LoopArgs A)
{
    const int T = A.f->err ? 0 : min(A.f->n_tracks, A.cap);
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < T; r += gridDim.x * blockDim.x) {
        A.group[r] = -1;
        A.leg[r] = -1;
        A.par[r] = r;
        LoopCand e;
        e.frame = -1;
        const int t = A.seg[A.thead[r]];
        const float* s = A.t_bot + (int64_t)t * NST;
        const float q = s[5];
        if (fabsf(q) >= A.qmin) {
            const float k = A.kb * q;
            const float sp = s[3];
            const float cp = __fsqrt_rn((1.0f - sp) * (1.0f + sp));
            const float ik = __fdiv_rn(1.0f, k);
            const float lx = s[0] - sp * ik, ly = __fmaf_rn(cp, ik, s[1]);
            const uint32_t pg = sc_plane(A.sc[A.t_start[t]]);
            const int fr = (int)(pg / (uint32_t)A.np);
            const int sec = (int)(pg - (uint32_t)fr * A.np) / A.nr;
            const int w = A.ns == 1 ? 0 : sec % 18;
            const float cs = c_sec_cos[w], sn = c_sec_sin[w];
            e.R = fabsf(ik);
            e.sr = e.R * __fdiv_rn(__fsqrt_rn(s[6 + 14]), fabsf(q));
            e.cx = __fmaf_rn(lx, cs, -(ly * sn));
            e.cy = __fmaf_rn(lx, sn, ly * cs);
            e.px = __fmaf_rn(s[0], cs, -(s[1] * sn));
            e.py = __fmaf_rn(s[0], sn, s[1] * cs);
            e.z = s[2];
            e.tl = fabsf(s[4]);
            e.a = e.tl * e.R;
            e.sense = k * s[4] >= 0.0f ? 1 : -1;
            const float side = (A.ns == 36 && sec >= 18) ? -1.0f : 1.0f;
            e.sz = side * s[2];
            if (e.sr <= LOOP_SRMAX) {
                e.frame = fr;
                atomicAdd(&A.bincnt[loop_bin(e)], 1u);
            }
        }
        A.cand[r] = e;
    }
}

__global__ void k_loop_sort(LoopArgs A, uint32_t* __restrict__ cursor)
{
    const int T = A.f->err ? 0 : min(A.f->n_tracks, A.cap);
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < T; r += gridDim.x * blockDim.x) {
        const LoopCand e = A.cand[r];
        if (e.frame >= 0) A.sorted[atomicAdd(&cursor[loop_bin(e)], 1u)] = r;
    }
}

__device__ __forceinline__ bool loop_pair(const LoopCand& A, const LoopCand& B, float zmax)
{
    const float tsg = LOOP_NSIG * __fsqrt_rn(__fmaf_rn(A.sr, A.sr, B.sr * B.sr));
    if (!(fabsf(A.R - B.R) < tsg + LOOP_DR)) return false;
    const float dx = B.cx - A.cx, dy = B.cy - A.cy;
    const float dc = tsg + LOOP_DC;
    if (!(__fmaf_rn(dx, dx, dy * dy) < dc * dc)) return false;
    if (!(fabsf(A.tl - B.tl) < LOOP_DTGL)) return false;
    if (!(fabsf(B.z - A.z) <= zmax)) return false;
    const float ux = A.px - A.cx, uy = A.py - A.cy;
    const float vx = B.px - A.cx, vy = B.py - A.cy;
    const float cr = __fmaf_rn(ux, vy, -(uy * vx));
    const float dt = __fmaf_rn(ux, vx, uy * vy);
    const float dpsi = atan2_own(cr, dt);
    const float a = 0.5f * (A.a + B.a);
    const float tl = 0.5f * (A.tl + B.tl);
    const float tpa = TWO_PI_F * a;
    const bool steep = A.tl >= LOOP_TLSENSE && B.tl >= LOOP_TLSENSE;
    if (steep && A.sense != B.sense) return false;
    for (int sg = 0; sg < 2; sg++) {
        if (steep && sg == 1) break;
        const int sense = sg == 0 ? A.sense : -A.sense;
        const float dz = B.z - A.z;
        const float w = (sense > 0 ? dz : -dz) - a * dpsi;
        float m = tpa > 0.0f ? rintf(__fdiv_rn(w, tpa)) : 0.0f;
        m = fminf(fmaxf(m, -LOOP_TURNS), LOOP_TURNS);
        const float res = __fmaf_rn(-tpa, m, w);
        const float turn = __fmaf_rn(TWO_PI_F, fabsf(m), fabsf(dpsi));
        const float tol = __fmaf_rn(tl * turn, tsg, LOOP_DZ);
        if (fabsf(res) < tol) return true;
    }
    return false;
}

// union-find on the track indices: roots only ever move to smaller indices,
// so every walk ends; the step counts are bounded all the same
__device__ __forceinline__ int uf_find(int32_t* par, int x, int* err)
{
    for (int it = 0; it < UF_MAX_STEPS; it++) {
        const int p = atomicAdd(&par[x], 0);
        if (p == x) return x;
        x = p;
    }
    atomicExch(err, 1);
    return x;
}

__device__ __forceinline__ void uf_union(int32_t* par, int a, int b, int* err)
{
    for (int it = 0; it < UF_MAX_STEPS; it++) {
        a = uf_find(par, a, err);
        b = uf_find(par, b, err);
        if (a == b) return;
        if (a > b) {
            const int t = a;
            a = b;
            b = t;
        }
        const int old = atomicCAS(&par[b], b, a);
        if (old == b) return;
        b = old;
    }
    atomicExch(err, 1);
}

// one thread per candidate: the candidates of its frame in the 3 x 3 centre
// cells around its own, each unordered pair tested once (i < j)
__global__ void k_loop_pairs(LoopArgs A)
{
    const int T = A.f->err ? 0 : min(A.f->n_tracks, A.cap);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < T; i += gridDim.x * blockDim.x) {
        const LoopCand a = A.cand[i];
        if (a.frame < 0) continue;
        const int gx = loop_cell(a.cx), gy = loop_cell(a.cy);
        const int x0 = max(gx - 1, 0), x1 = min(gx + 1, LOOP_G - 1);
        for (int yy = max(gy - 1, 0); yy <= min(gy + 1, LOOP_G - 1); yy++) {
            const int row = a.frame * LOOP_NBIN + yy * LOOP_G;
            for (uint32_t q = A.bincnt[row + x0]; q < A.bincnt[row + x1 + 1]; q++) {
                const int j = A.sorted[q];
                if (j <= i) continue;
                if (loop_pair(a, A.cand[j], A.zmax)) uf_union(A.par, i, j, A.err);
            }
        }
    }
}

__global__ void k_loop_count(LoopArgs A)
{
    const int T = A.f->err ? 0 : min(A.f->n_tracks, A.cap);
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < T; r += gridDim.x * blockDim.x)
        if (A.cand[r].frame >= 0) atomicAdd(&A.gcnt[uf_find(A.par, r, A.err)], 1u);
}

// members listed by root (gcnt scanned: the root's first slot; gcnt[root + 1]
// - gcnt[root] its size); cursor = a copy of the scanned counts
__global__ void k_loop_list(LoopArgs A, uint32_t* __restrict__ cursor)
{
    const int T = A.f->err ? 0 : min(A.f->n_tracks, A.cap);
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < T; r += gridDim.x * blockDim.x)
        if (A.cand[r].frame >= 0) A.glist[atomicAdd(&cursor[uf_find(A.par, r, A.err)], 1u)] = r;
}

__global__ void k_loop_legs(LoopArgs A)
{
    const int T = A.f->err ? 0 : min(A.f->n_tracks, A.cap);
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < T; r += gridDim.x * blockDim.x) {
        const LoopCand e = A.cand[r];
        if (e.frame < 0) continue;
        const int root = uf_find(A.par, r, A.err);
        const uint32_t b = A.gcnt[root], en = A.gcnt[root + 1];
        if (en - b < 2) continue;
        int rank = 0;
        for (uint32_t q = b; q < en; q++) {
            const int j = A.glist[q];
            const float szj = A.cand[j].sz;
            rank += szj < e.sz || (szj == e.sz && j < r);
        }
        A.group[r] = root;
        A.leg[r] = rank;
    }
}

// good tracks of the attachment: the pT cut passed and not a secondary leg
__global__ void k_track_good(const Frame* __restrict__ f, int cap, const int32_t* __restrict__ seg,
                             const int32_t* __restrict__ thead, const float* __restrict__ t_bot, float qmax,
                             const int32_t* __restrict__ leg, uint8_t* __restrict__ good)
{
    const int T = f->err ? 0 : min(f->n_tracks, cap);
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < T; r += gridDim.x * blockDim.x) {
        const float aq = fabsf(t_bot[(int64_t)seg[thead[r]] * NST + 5]);
        good[r] = (aq <= qmax && !(leg && leg[r] >= 1)) ? 1 : 0;
    }
}

// one thread per cluster: the flags
__global__ void k_attach_flags(AttachArgs A)
{
    if (A.f->err) return;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < A.n; c += gridDim.x * blockDim.x) {
        const int a = A.assign[c];
        const unsigned long long key = A.akey[c];
        const bool att = a >= 0;
        const bool adj = !att && key != 0ull;
        const bool prot = A.aprot[c] != 0 || (att && A.tgood[a] != 0);
        const bool rem = (att || adj) && !prot;
        A.flags[c] = (uint8_t)((att ? TPC_CL_ATTACHED : 0) | (adj ? TPC_CL_ADJACENT : 0) |
                               (prot ? TPC_CL_PROTECTED : 0) | (rem ? TPC_CL_REMOVE : 0));
        if (A.adjacent) A.adjacent[c] = adj ? (int32_t)(0xFFFFFFFFu - (uint32_t)(key & 0xFFFFFFFFull)) : -1;
    }
}

// Longest-first order of the tracks for the refit (one thread per track: a
// warp then holds tracks of similar length).  Bucket = LEN_BUCKETS-1 -
// min(n, LEN_BUCKETS-1).  Only the schedule depends on this order (each
// track's refit is independent), so the atomic placement within a bucket may
// vary from run to run without changing any result.
__device__ __forceinline__ int len_bucket(int n) { return LEN_BUCKETS - 1 - min(n, LEN_BUCKETS - 1); }

__global__ void k_len_hist(const Frame* __restrict__ f, const int32_t* __restrict__ nclus, int cap,
                           uint32_t* __restrict__ cnt)
{
    const int T = f->err ? 0 : min(f->n_tracks, cap);
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < T; r += gridDim.x * blockDim.x)
        atomicAdd(&cnt[len_bucket(nclus[r])], 1u);
}

// cnt: exclusive starts of the buckets on entry
__global__ void k_len_scatter(const Frame* __restrict__ f, const int32_t* __restrict__ nclus, int cap,
                              uint32_t* __restrict__ cnt, int32_t* __restrict__ order)
{
    const int T = f->err ? 0 : min(f->n_tracks, cap);
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < T; r += gridDim.x * blockDim.x)
        order[atomicAdd(&cnt[len_bucket(nclus[r])], 1u)] = r;
}

// counts for the enqueue-only call: n_tracks, n_tracklets, n_segments, error,
// clusters in tracks, start hits found
__global__ void k_publish(const Frame* __restrict__ f, int cap, int32_t* out)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        out[0] = f->n_tracks;
        out[1] = min(f->n_starts, cap);
        out[2] = f->n_seg;
        out[3] = f->err ? f->err : (f->n_starts > cap ? TPC_ERR_CAPACITY : 0);
        out[4] = f->n_clus;
        out[5] = f->n_starts;
    }
}

// ---------------------------------------------------------------------------
// intermediate results in input-index space (optional outputs)
// ---------------------------------------------------------------------------
__global__ void k_export_links(int n, const float4* __restrict__ sc, const int32_t* __restrict__ upr,
                               const int32_t* __restrict__ dnr, const int32_t* __restrict__ up,
                               const int32_t* __restrict__ dn, int32_t* o_upr, int32_t* o_dnr, int32_t* o_up,
                               int32_t* o_dn, uint8_t* o_start, const Frame* __restrict__ f)
{
    if (f->err) return;
    for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < n; h += gridDim.x * blockDim.x) {
        const int id = sc_id(sc[h]);
        const int a = upr[h], b = dnr[h], c = up[h], d = dn[h];
        if (o_upr) o_upr[id] = a >= 0 ? sc_id(sc[a]) : -1;
        if (o_dnr) o_dnr[id] = b >= 0 ? sc_id(sc[b]) : -1;
        if (o_up) o_up[id] = c >= 0 ? sc_id(sc[c]) : -1;
        if (o_dn) o_dn[id] = d >= 0 ? sc_id(sc[d]) : -1;
        if (o_start) o_start[id] = (c >= 0 && d < 0 && up[c] >= 0) ? 1 : 0;
    }
}

#define CK(x)                                          \
    do {                                               \
        cudaError_t e_ = (x);                          \
        if (e_ != cudaSuccess) return TPC_ERR_CUDA;    \
    } while (0)

// ---------------------------------------------------------------------------
// Scratch for tpc_links_static: a file-scope device array, so that the entry
// point needs no allocation by its caller or by the library.  Sized for
// TPC_LINKS_STATIC_MAX_CLUSTERS clusters of one frame with a coarser grid (64
// z-cells per pad row, one y-bin; coarser cells scan more candidates but give
// the same links).
// ---------------------------------------------------------------------------
constexpr int STATIC_NZ = 64;
constexpr int STATIC_MAX_PLANES = 36 * 255;
constexpr int64_t STATIC_NCELLS = (int64_t)STATIC_MAX_PLANES * STATIC_NZ;

struct StaticLayout {
    size_t frame, fgrid, offsets, rowtab, zlin, cfr, cell, slot, cstart, scan, sc, upr, dnr, up, dn, total;
};

constexpr size_t sa256(size_t v) { return (v + 255) / 256 * 256; }
constexpr StaticLayout static_layout()
{
    const size_t N = TPC_LINKS_STATIC_MAX_CLUSTERS;
    StaticLayout L{};
    size_t o = 0;
    L.frame = o; o += sa256(sizeof(Frame));
    L.fgrid = o; o += sa256(sizeof(FrameGrid));
    L.offsets = o; o += sa256(2 * sizeof(int32_t));
    L.rowtab = o; o += sa256(sizeof(float) * ROWTAB * 256);
    L.zlin = o; o += sa256(4 * N);
    L.cfr = o; o += sa256(2 * N);
    L.cell = o; o += sa256(4 * N);
    L.slot = o; o += sa256(4 * N);
    L.cstart = o; o += sa256(4 * (STATIC_NCELLS + 1));
    L.scan = o; o += sa256(4 * (STATIC_NCELLS / SCAN_TILE + 64));
    L.sc = o; o += sa256(16 * N);
    L.upr = o; o += sa256(4 * N);
    L.dnr = o; o += sa256(4 * N);
    L.up = o; o += sa256(4 * N);
    L.dn = o; o += sa256(4 * N);
    L.total = o;
    return L;
}
constexpr StaticLayout SL = static_layout();
static_assert(SL.total == TPC_LINKS_STATIC_SCRATCH_BYTES, "scratch size stated in tpc_track.h");

static __device__ __align__(256) unsigned char g_links_scratch[TPC_LINKS_STATIC_SCRATCH_BYTES];

// device address of g_links_scratch, looked up once per device
std::mutex g_scratch_mu;
void* g_scratch_ptr[128] = {nullptr};

int static_scratch(void** ptr)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) return TPC_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_links_scratch) != cudaSuccess || !p) return TPC_ERR_CUDA;
        g_scratch_ptr[dev] = p;
    }
    *ptr = g_scratch_ptr[dev];
    return TPC_OK;
}

int check_args(const tpc_params* p, const tpc_geometry* g)
{
    if (!p || !g || !g->row_x) return TPC_ERR_ARG;
    if (!(g->n_sectors == 36 || g->n_sectors == 1)) return TPC_ERR_ARG;
    if (g->n_rows < 3 || g->n_rows > 255) return TPC_ERR_ARG;
    if (p->max_z_cells < 2 || p->tracklets_per_1k < 1 || p->refit_passes < 1) return TPC_ERR_ARG;
    if (!(p->refit_inflate >= 1.0f) || p->queue_blocks_per_sm < 0 || p->merge_pairs_per_1k < 0) return TPC_ERR_ARG;
    if (!(p->z_cell >= 0.25f) || p->y_bins < 1 || p->y_bins > MAX_YBINS) return TPC_ERR_ARG;
    if (!(p->tube_radius >= 0.0f && p->tube_radius <= 20.0f)) return TPC_ERR_ARG;
    if (!(p->pt_min_physics >= 0.0f && p->pt_min_physics <= 1e30f)) return TPC_ERR_ARG;
    for (int r = 0; r + 1 < g->n_rows; r++)
        if (!(g->row_x[r + 1] > g->row_x[r]) || !(g->row_x[r] > 0.0f)) return TPC_ERR_ARG;
    return TPC_OK;
}

int check_frames(int32_t n, int32_t nframes, const int32_t* offsets)
{
    if (nframes < 1 || nframes > MAX_FRAMES || !offsets) return TPC_ERR_ARG;
    if (offsets[0] != 0 || offsets[nframes] != n) return TPC_ERR_ARG;
    for (int i = 0; i < nframes; i++)
        if (offsets[i + 1] < offsets[i]) return TPC_ERR_ARG;
    return TPC_OK;
}

int out_args(const tpc_params* p, const tpc_tracks* out)
{
    if (!out->sector || !out->x || !out->param || !out->cov || !out->chi2 || !out->ndf || !out->status ||
        !out->nclus || !out->clus_offset || !out->clus_index || !out->assign)
        return TPC_ERR_ARG;
    if (out->capacity_tracks < 0 || out->capacity_clusters < 0) return TPC_ERR_ARG;
    if (p->fp64_final < 0 || p->fp64_final > 2) return TPC_ERR_ARG;
    if (p->fp64_final && (!out->cov64 || !out->chi2_64)) return TPC_ERR_ARG;
    return TPC_OK;
}

}  // namespace

// refit launcher (tpc_refit.cu)
int tpc_launch_refit(const tpc_params* p, const tpc_geometry* g, float bz, const float4* tcl, const int32_t* order,
                     const void* frame, const int32_t* ttail, const float* t_top, tpc_tracks* out, int max_tracks,
                     cudaStream_t st);

namespace {

// Enqueue the whole chain on `st` (no host synchronisation, no pageable copy:
// capturable in a CUDA graph once the tables are in the workspace).
// Side stream of a caller's stream, with a fork and a join event, for work
// that shares no data with the main stream's stage at the time: the
// initialisation of the later stages' buffers (beside the tracklet
// constructor), the cluster rejection (it rewrites the owned-hit masks and
// counts; beside the merger, which reads the segment ends) and the refit
// order (beside the fill of the cluster lists).  Each use forks from and
// joins back into the caller's stream, so the work completes in that stream's
// order and a stream capture holds both branches.  One per (device, caller
// stream), created on first use and kept for the life of the process; the
// creation switches this thread to relaxed capture mode, so a first use inside
// a stream capture is allowed.
struct SideStream {
    cudaStream_t s = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
};
std::mutex g_side_mu;
std::map<std::pair<int, cudaStream_t>, SideStream> g_side;

cudaError_t side_stream(cudaStream_t st, SideStream& out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(g_side_mu);
    const auto key = std::make_pair(dev, st);
    const auto it = g_side.find(key);
    if (it != g_side.end()) {
        out = it->second;
        return cudaSuccess;
    }
    cudaStreamCaptureMode mode = cudaStreamCaptureModeRelaxed;
    e = cudaThreadExchangeStreamCaptureMode(&mode);
    if (e != cudaSuccess) return e;
    SideStream n;
    e = cudaStreamCreateWithFlags(&n.s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&n.fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&n.join, cudaEventDisableTiming);
    cudaStreamCaptureMode back = mode;
    const cudaError_t e2 = cudaThreadExchangeStreamCaptureMode(&back);
    if (e == cudaSuccess) e = e2;
    if (e != cudaSuccess) return e;
    g_side[key] = n;
    out = n;
    return cudaSuccess;
}

int enqueue(const tpc_params* p, const tpc_geometry* g, float bz, float v_drift, const tpc_clusters* cl, void* ws,
            const Layout& L, tpc_tracks* out, int32_t* dev_counts, cudaStream_t st, bool prof)
{
    const int n = cl->n;
    Frame* f = at<Frame>(ws, L.frame);
    FrameGrid* fg = at<FrameGrid>(ws, L.fgrid);
    const int32_t* offsets = at<int32_t>(ws, L.offsets);
    float* rowtab = at<float>(ws, L.rowtab);
    float* zlin = at<float>(ws, L.zlin);
    uint16_t* cfr = at<uint16_t>(ws, L.cfr);
    uint32_t* cell = at<uint32_t>(ws, L.cell);
    uint32_t* slot = at<uint32_t>(ws, L.slot);
    uint32_t* cstart = at<uint32_t>(ws, L.cstart);
    uint32_t* aux = at<uint32_t>(ws, L.scan);
    float4* sc = at<float4>(ws, L.sc);
    int32_t* upr = at<int32_t>(ws, L.upr);
    int32_t* dnr = at<int32_t>(ws, L.dnr);
    int32_t* up = at<int32_t>(ws, L.up);
    int32_t* dn = at<int32_t>(ws, L.dn);
    int32_t* starts = at<int32_t>(ws, L.starts);
    unsigned long long* hitw = at<unsigned long long>(ws, L.hitw);
    volatile float vyv = p->sigma_y * p->sigma_y;
    volatile float vzv = p->sigma_z * p->sigma_z;
    volatile float kbv = KB_C * bz;
    const float vy = vyv, vz = vzv, kb = kbv;
    const int B = 256;
    const int gN = grid_for(n, B);
    const int ntcap = L.ntcap;
    const int NF = L.nframes;
    auto mark = [&](int k) -> cudaError_t { return prof ? cudaEventRecord(g_events.ev[k], st) : cudaSuccess; };
    g_launches = 0;

    const int nplanes = NF * L.np;
    uint32_t* pstart = at<uint32_t>(ws, L.pstart);
    CK(mark(0));
    CK(cudaMemsetAsync(pstart, 0, sizeof(uint32_t) * ((size_t)nplanes * PSPLIT + 1), st));
    k_init_frame<<<std::max(1, (NF + 255) / 256), 256, 0, st>>>(f, fg, NF);
    {
        // chunks of about 32 k clusters (the average frame's), at most two blocks per SM per frame
        const int64_t per_frame = ((int64_t)n + NF - 1) / NF;
        const int gx = (int)std::max<int64_t>(1, std::min<int64_t>((per_frame + 32767) / 32768, 2 * 148));
        k_prep<true><<<dim3(gx, NF), PREP_RANK_BLOCK, sizeof(uint32_t) * L.np, st>>>(
            offsets, cl->sector, cl->row, cl->y, cl->zt, g->n_sectors, g->n_rows, g->continuous, g->z_max, v_drift,
            zlin, cfr, f, fg, L.np, pstart, cell);
    }
    k_grid_setup<<<1, 32, 0, st>>>(f, fg, NF, L.np, L.ny, p->z_cell, L.nzmax, (long long)L.ncells,
                                   0.25f * p->merge_dz, L.mnzmax, p->packed_links);
    g_launches += 3;
    CK(mark(1));
    // a2: clusters into (frame, sector, row, z-cell, y-bin) order, a plane at a time
    scan_u32(pstart, (int64_t)nplanes * PSPLIT, aux, st);
    k_pscatter<<<gN, B, 0, st>>>(n, cl->sector, cl->row, cl->y, zlin, cfr, g->n_rows, L.np, pstart, cell,
                                 at<float4>(ws, L.pbuf), f);
    uint32_t* yzp = p->packed_links ? at<uint32_t>(ws, L.yzp) : nullptr;
    {
        const int smem_cells = plane_sort_smem_cells((int64_t)L.nzmax * L.ny, st);
        k_plane_sort<<<std::max(1, std::min(nplanes, 148 * 8)), PS_BLOCK, sizeof(uint32_t) * smem_cells, st>>>(
            nplanes, L.np, g->n_rows, g->n_sectors, pstart, at<float4>(ws, L.pbuf), slot, rowtab, f, fg, smem_cells,
            cstart, sc, yzp);
    }
    g_launches += 2;
    CK(mark(2));
    if (yzp)
        k_neighbours<true><<<gN, B, 0, st>>>(n, g->n_rows, g->n_sectors, L.np, rowtab, sc, cstart, f, fg,
                                             p->dy_link, p->dz_link, p->s_max_link, upr, dnr, yzp);
    else
        k_neighbours<false><<<gN, B, 0, st>>>(n, g->n_rows, g->n_sectors, L.np, rowtab, sc, cstart, f,
                                              fg, p->dy_link, p->dz_link, p->s_max_link, upr, dnr, nullptr);
    g_launches++;
    CK(mark(3));
    k_clean_starts<<<gN, B, 0, st>>>(n, upr, dnr, up, dn, starts, ntcap, f);
    g_launches += 1;
    CK(mark(4));
    // The initialisation of the later stages' buffers (the selector's hit
    // weights, the merger's grids, lists and best keys, the assembly's counts,
    // segment ranks and the assignment output) runs on the side stream while
    // the tracklet constructor runs; nothing before the selector uses them.
    const bool w32 = n <= (1 << 24);   // every start-hit id below 2^24: 32-bit weights
    const int64_t mcells = (int64_t)NF * g->n_sectors * L.mnzmax;
    uint32_t* cntb = at<uint32_t>(ws, L.cntb);
    uint32_t* cntt = at<uint32_t>(ws, L.cntt);
    uint32_t* headmark = at<uint32_t>(ws, L.headmark);
    uint32_t* tcount = at<uint32_t>(ws, L.tcount);
    SideStream side;
    CK(side_stream(st, side));
    CK(cudaEventRecord(side.fork, st));
    CK(cudaStreamWaitEvent(side.s, side.fork, 0));
    CK(cudaMemsetAsync(hitw, 0, (w32 ? 4 : 8) * (size_t)n, side.s));
    CK(cudaMemsetAsync(cntb, 0, 4 * (size_t)(mcells + 1), side.s));
    CK(cudaMemsetAsync(cntt, 0, 4 * (size_t)(mcells + 1), side.s));
    CK(cudaMemsetAsync(at<int32_t>(ws, L.snext), 0xFF, 4 * (size_t)ntcap, side.s));
    CK(cudaMemsetAsync(at<int32_t>(ws, L.sprev), 0xFF, 4 * (size_t)ntcap, side.s));
    CK(cudaMemsetAsync(headmark, 0, 4 * (size_t)(n + 1), side.s));
    CK(cudaMemsetAsync(at<unsigned long long>(ws, L.bestA), 0xFF, 8 * (size_t)ntcap, side.s));
    CK(cudaMemsetAsync(at<unsigned long long>(ws, L.bestB), 0xFF, 8 * (size_t)ntcap, side.s));
    CK(cudaMemsetAsync(at<int32_t>(ws, L.bnext), 0xFF, 4 * (size_t)ntcap, side.s));
    CK(cudaMemsetAsync(at<int32_t>(ws, L.bprev), 0xFF, 4 * (size_t)ntcap, side.s));
    CK(cudaMemsetAsync(tcount, 0, 4 * (size_t)(ntcap + 1), side.s));
    CK(cudaMemsetAsync(out->assign, 0xFF, 4 * (size_t)n, side.s));
    CK(cudaMemsetAsync(at<int32_t>(ws, L.segrank), 0xFF, sizeof(int32_t) * (size_t)ntcap, side.s));   // -1: in no track
    CK(cudaEventRecord(side.join, side.s));
    // a6: tracklets
    TrkArgs TA;
    TA.rowtab = rowtab; TA.sc = sc; TA.cstart = cstart; TA.up = up;
    TA.starts = starts; TA.f = f; TA.fg = fg; TA.nr = g->n_rows; TA.ns = g->n_sectors; TA.np = L.np; TA.cap = ntcap;
    TA.kb = kb; TA.vy = vy; TA.vz = vz; TA.c0s = p->c0_snp; TA.c0t = p->c0_tgl; TA.c0q = p->c0_qpt;
    TA.nsig = p->win_nsigma; TA.wmin = p->win_min; TA.wmax = p->win_max; TA.chi2cut = p->chi2_cut;
    TA.edge = p->edge_margin; TA.max_miss = p->max_miss; TA.prof = prof ? 1 : 0; TA.fw = f;
    TA.t_start = at<int32_t>(ws, L.t_start); TA.t_id = at<int32_t>(ws, L.t_id);
    TA.t_nhits = at<int32_t>(ws, L.t_nhits); TA.t_nup = at<int32_t>(ws, L.t_nup);
    TA.t_hits = at<int32_t>(ws, L.t_hits); TA.t_top = at<float>(ws, L.t_top); TA.t_bot = at<float>(ws, L.t_bot);
    const int gT = grid_for(ntcap, TRK_BLOCK);
    const int gQ = p->queue_blocks_per_sm > 0 ? std::min(gT, 148 * p->queue_blocks_per_sm) : gT;
    TA.t_state = at<float>(ws, L.t_state);
    if (prof) k_tracklets<1, true><<<gQ, TRK_BLOCK, 0, st>>>(TA);
    else k_tracklets<1, false><<<gQ, TRK_BLOCK, 0, st>>>(TA);
    if (prof) k_tracklets<2, true><<<gQ, TRK_BLOCK, 0, st>>>(TA);
    else k_tracklets<2, false><<<gQ, TRK_BLOCK, 0, st>>>(TA);
    g_launches += 2;
    CK(mark(5));
    // a7: selector
    CK(cudaStreamWaitEvent(st, side.join, 0));
    const int gt2 = grid_for(ntcap, B);
    uint8_t* kept = at<uint8_t>(ws, L.t_kept);
    int32_t* seg = at<int32_t>(ws, L.seg);
    const int gt2w = grid_for((int64_t)ntcap * 32, B);      // one warp per tracklet
    const int gsel = grid_for((int64_t)ntcap * SEL_G, B);     // SEL_G lanes per tracklet
    if (w32) {
        unsigned* hw = reinterpret_cast<unsigned*>(hitw);
        k_sel_weight<unsigned><<<gsel, B, 0, st>>>(f, ntcap, g->n_rows, p->min_hits, TA.t_id, TA.t_nhits, TA.t_nup,
                                                  TA.t_hits, hw);
        k_sel_own<unsigned><<<gsel, B, 0, st>>>(f, ntcap, g->n_rows, p->min_hits, p->min_owned, TA.t_id, TA.t_nhits,
                                               TA.t_nup, TA.t_hits, hw, kept, seg, at<int32_t>(ws, L.t_own),
                                               at<uint32_t>(ws, L.ownmask));
    } else {
        k_sel_weight<unsigned long long><<<gsel, B, 0, st>>>(f, ntcap, g->n_rows, p->min_hits, TA.t_id, TA.t_nhits,
                                                            TA.t_nup, TA.t_hits, hitw);
        k_sel_own<unsigned long long><<<gsel, B, 0, st>>>(f, ntcap, g->n_rows, p->min_hits, p->min_owned, TA.t_id,
                                                         TA.t_nhits, TA.t_nup, TA.t_hits, hitw, kept, seg,
                                                         at<int32_t>(ws, L.t_own), at<uint32_t>(ws, L.ownmask));
    }
    g_launches += 2;
    CK(mark(6));
    // cluster rejection on the side stream, beside the merger below
    const bool reject = p->outlier_chi2 > 0.0f;
    if (reject) {
        CK(cudaEventRecord(side.fork, st));
        CK(cudaStreamWaitEvent(side.s, side.fork, 0));
        volatile float ivyv = 1.0f / vy, ivzv = 1.0f / vz;
        k_reject<<<gt2, B, 0, side.s>>>(f, ntcap, g->n_rows, L.np, kb, ivyv, ivzv, p->outlier_chi2, seg, TA.t_nhits,
                                        TA.t_nup, TA.t_hits, TA.t_bot, sc, rowtab, at<uint32_t>(ws, L.ownmask),
                                        at<int32_t>(ws, L.t_own));
        CK(cudaEventRecord(side.join, side.s));
        g_launches++;
    }
    // a8: merger
    k_seg_keys<<<gt2, B, 0, st>>>(f, g->n_sectors, g->n_rows, seg, sc, TA.t_start, TA.t_top, TA.t_bot, cntb, cntt,
                                  at<uint32_t>(ws, L.keyb), at<uint32_t>(ws, L.keyt), at<uint32_t>(ws, L.slotb),
                                  at<uint32_t>(ws, L.slott));
    g_launches++;
    scan_u32(cntb, mcells, aux, st);
    scan_u32(cntt, mcells, aux, st);
    MergeArgs M;
    M.f = f; M.ns = g->n_sectors; M.nr = g->n_rows; M.kb = kb; M.dz = p->merge_dz; M.chi2cut = p->merge_chi2;
    M.seg = seg; M.sc = sc; M.t_start = TA.t_start; M.t_id = TA.t_id; M.t_top = TA.t_top; M.t_bot = TA.t_bot;
    M.cntb = cntb; M.cntt = cntt; M.byb = at<int32_t>(ws, L.byb); M.byt = at<int32_t>(ws, L.byt);
    M.recb = at<MergeRec>(ws, L.recb); M.rect = at<MergeRec>(ws, L.rect);
    M.bnext = at<int32_t>(ws, L.bnext); M.bprev = at<int32_t>(ws, L.bprev); M.prof = prof ? 1 : 0; M.fw = f;
    M.mirror = (g->n_sectors == 36 && !g->continuous) ? 1 : 0;
    M.pairs = at<int2>(ws, L.mpair); M.pc2 = at<float>(ws, L.mpc2);
    M.bestA = at<unsigned long long>(ws, L.bestA); M.bestB = at<unsigned long long>(ws, L.bestB);
    M.pcap = (int)std::min<int64_t>(L.mpcap, INT32_MAX);
    k_seg_scatter<<<gt2, B, 0, st>>>(f, cntb, cntt, at<uint32_t>(ws, L.keyb), at<uint32_t>(ws, L.keyt),
                                     at<uint32_t>(ws, L.slotb), at<uint32_t>(ws, L.slott), at<int32_t>(ws, L.byb),
                                     at<int32_t>(ws, L.byt), seg, TA.t_id, TA.t_top, TA.t_bot,
                                     at<MergeRec>(ws, L.recb), at<MergeRec>(ws, L.rect));
    const int gTw = grid_for((int64_t)ntcap * 32, 128);    // one warp per segment end
    k_merge_pairs<<<gTw, 128, 0, st>>>(M);
    k_merge_chi2<<<grid_for(L.mpcap, 128), 128, 0, st>>>(M);
    k_merge_resolve<<<grid_for(L.mpcap, B), B, 0, st>>>(M);
    k_merge_next<<<gTw, 128, 0, st>>>(M);      // only if the pair list overflowed
    k_merge_prev<<<gTw, 128, 0, st>>>(M);
    k_merge_link<<<gt2, B, 0, st>>>(f, M.bnext, M.bprev, at<int32_t>(ws, L.snext), at<int32_t>(ws, L.sprev));
    k_merge_cycles<<<gt2, B, 0, st>>>(f, at<int32_t>(ws, L.sprev), at<uint8_t>(ws, L.bad));
    k_merge_fix<<<gt2, B, 0, st>>>(f, at<int32_t>(ws, L.snext), at<int32_t>(ws, L.sprev), at<uint8_t>(ws, L.bad),
                                   at<int32_t>(ws, L.next2), at<int32_t>(ws, L.prev2), seg, TA.t_id, headmark);
    g_launches += 9;
    scan_u32(headmark, n, aux, st);
    if (reject) CK(cudaStreamWaitEvent(st, side.join, 0));
    CK(mark(7));
    // merged cluster lists and assignments
    AsmArgs AA;
    AA.f = f; AA.nr = g->n_rows; AA.np = L.np; AA.n = n; AA.cap_tracks = out->capacity_tracks;
    AA.cap_clus = out->capacity_clusters; AA.ntcap = ntcap; AA.seg = seg; AA.next2 = at<int32_t>(ws, L.next2);
    AA.prev2 = at<int32_t>(ws, L.prev2); AA.t_start = TA.t_start; AA.t_id = TA.t_id; AA.t_nhits = TA.t_nhits;
    AA.t_nup = TA.t_nup; AA.t_hits = TA.t_hits; AA.sc = sc; AA.ownmask = at<uint32_t>(ws, L.ownmask);
    AA.headmark = headmark; AA.tcount = tcount; AA.thead = at<int32_t>(ws, L.thead); AA.ttail = at<int32_t>(ws, L.ttail);
    AA.clus_offset = out->clus_offset; AA.nclus = out->nclus; AA.clus_index = out->clus_index; AA.assign = out->assign;
    AA.frame = out->frame;
    AA.rowtab = rowtab; AA.tcl = at<float4>(ws, L.tcl);
    AA.t_own = at<int32_t>(ws, L.t_own); AA.segoff = at<int32_t>(ws, L.segoff); AA.segrank = at<int32_t>(ws, L.segrank);
    k_track_count<<<gt2, B, 0, st>>>(AA);
    g_launches++;
    scan_u32(tcount, ntcap, aux, st);
    k_track_fill<<<gt2, B, 0, st>>>(AA);
    // the refit order (tracks by decreasing cluster count, a counting sort over
    // LEN_BUCKETS) needs only the counts: on the side stream, beside the fill
    // of the cluster lists
    uint32_t* lcnt = at<uint32_t>(ws, L.lencnt);
    int32_t* order = at<int32_t>(ws, L.order);
    CK(cudaEventRecord(side.fork, st));
    CK(cudaStreamWaitEvent(side.s, side.fork, 0));
    CK(cudaMemsetAsync(lcnt, 0, sizeof(uint32_t) * (LEN_BUCKETS + 1), side.s));
    k_len_hist<<<gt2, B, 0, side.s>>>(f, out->nclus, out->capacity_tracks, lcnt);
    scan_u32(lcnt, LEN_BUCKETS, aux, side.s);
    k_len_scatter<<<gt2, B, 0, side.s>>>(f, out->nclus, out->capacity_tracks, lcnt, order);
    CK(cudaEventRecord(side.join, side.s));
    k_seg_fill<<<gt2w, B, 0, st>>>(AA);
    g_launches += 4;
    CK(mark(8));
    // a9: refit
    CK(cudaStreamWaitEvent(st, side.join, 0));
    if (out->refit_event) CK(cudaEventRecord(static_cast<cudaEvent_t>(out->refit_event), st));
    int rr = tpc_launch_refit(p, g, bz, AA.tcl, order, f, AA.ttail, TA.t_top, out,
                              std::min(out->capacity_tracks, ntcap), st);
    if (rr) return rr;
    g_launches++;
    CK(mark(9));
    // optional intermediate outputs
    if (out->z) CK(cudaMemcpyAsync(out->z, zlin, 4 * (size_t)n, cudaMemcpyDeviceToDevice, st));
    if (out->link_up_raw || out->link_dn_raw || out->link_up || out->link_dn || out->is_start) {
        k_export_links<<<gN, B, 0, st>>>(n, sc, upr, dnr, up, dn, out->link_up_raw, out->link_dn_raw, out->link_up,
                                         out->link_dn, out->is_start, f);
        g_launches++;
    }
    // optional: looper legs (also needed by the cluster attachment)
    int32_t* lleg = nullptr;
    if (out->looper_group || out->looper_leg || out->cl_flags) {
        LoopArgs LA;
        LA.f = f; LA.ns = g->n_sectors; LA.nr = g->n_rows; LA.np = L.np; LA.nfr = NF;
        LA.cap = std::min(out->capacity_tracks, ntcap);
        LA.kb = kb; LA.qmin = p->looper_qpt_min; LA.zmax = g->z_max;
        LA.seg = seg; LA.thead = AA.thead; LA.t_start = TA.t_start; LA.t_bot = TA.t_bot; LA.sc = sc;
        LA.cand = at<LoopCand>(ws, L.lcand);
        LA.par = at<int32_t>(ws, L.lpar);
        LA.bincnt = at<uint32_t>(ws, L.lbin);
        LA.sorted = at<int32_t>(ws, L.lsorted);
        LA.gcnt = at<uint32_t>(ws, L.lcnt);
        LA.glist = at<int32_t>(ws, L.llist);
        LA.group = out->looper_group ? out->looper_group : at<int32_t>(ws, L.lgrp);
        LA.leg = out->looper_leg ? out->looper_leg : at<int32_t>(ws, L.lleg);
        LA.err = &f->n_loop_err;
        const size_t nbins = (size_t)NF * LOOP_NBIN;
        uint32_t* cursor = at<uint32_t>(ws, L.lcur);
        CK(cudaMemsetAsync(LA.bincnt, 0, 4 * (nbins + 1), st));
        CK(cudaMemsetAsync(LA.gcnt, 0, 4 * ((size_t)ntcap + 1), st));
        const int gl = grid_for(LA.cap, B);
        k_loop_cand<<<gl, B, 0, st>>>(LA);
        scan_u32(LA.bincnt, (int64_t)nbins, aux, st);
        CK(cudaMemcpyAsync(cursor, LA.bincnt, 4 * (nbins + 1), cudaMemcpyDeviceToDevice, st));
        k_loop_sort<<<gl, B, 0, st>>>(LA, cursor);
        k_loop_pairs<<<gl, B, 0, st>>>(LA);
        k_loop_count<<<gl, B, 0, st>>>(LA);
        scan_u32(LA.gcnt, ntcap, aux, st);
        CK(cudaMemcpyAsync(cursor, LA.gcnt, 4 * ((size_t)ntcap + 1), cudaMemcpyDeviceToDevice, st));
        k_loop_list<<<gl, B, 0, st>>>(LA, cursor);
        k_loop_legs<<<gl, B, 0, st>>>(LA);
        g_launches += 6;
        lleg = LA.leg;
    }
    // optional: track-based cluster attachment (after the exports above: it
    // reuses the link arrays and the refit's cluster buffer)
    if (out->cl_flags) {
        AttachArgs AT;
        AT.f = f; AT.fg = fg; AT.nr = g->n_rows; AT.np = L.np; AT.ns = g->n_sectors; AT.n = n;
        AT.kb = kb; AT.R = p->tube_radius;
        AT.R2 = p->tube_radius * p->tube_radius;
        {
            volatile float one = 1.0f, pm = p->pt_min_physics;
            AT.qmax = p->pt_min_physics > 0.0f ? one / pm : INFINITY;
        }
        AT.seg = seg; AT.segrank = AA.segrank; AT.thead = AA.thead; AT.t_nhits = TA.t_nhits; AT.t_nup = TA.t_nup;
        AT.t_hits = TA.t_hits; AT.t_bot = TA.t_bot; AT.sc = sc; AT.cstart = cstart; AT.rowtab = rowtab;
        AT.assign = out->assign;
        AT.akey = at<unsigned long long>(ws, L.hitw);     // the selector's hit weights are dead by now
        AT.aprot = at<uint8_t>(ws, L.aprot);
        AT.flags = out->cl_flags; AT.adjacent = out->adjacent;
        AT.tgood = at<uint8_t>(ws, L.tgood);
        k_track_good<<<grid_for(std::min(out->capacity_tracks, ntcap), B), B, 0, st>>>(
            f, std::min(out->capacity_tracks, ntcap), seg, AA.thead, TA.t_bot, AT.qmax, lleg, at<uint8_t>(ws, L.tgood));
        g_launches++;
        CK(cudaMemsetAsync(AT.akey, 0, 8 * (size_t)n, st));
        CK(cudaMemsetAsync(AT.aprot, 0, (size_t)n, st));
        // plane buckets: counts in the binning's plane starts (free by now),
        // points (y, z) in the refit's cluster buffer, their keys in the link
        // arrays -- 2n points each.  32-bit positions: with 2^32 or more
        // possible points every point is scanned by its tracing thread.
        const int P = nplanes;
        const int PB = P * PSPLIT;               // sub-buckets
        uint32_t* pcnt = pstart;                 // sub-bucket starts (the binning's plane starts are free)
        uint32_t* cursor = at<uint32_t>(ws, L.acur);
        float2* pts = at<float2>(ws, L.tcl);
        unsigned long long* pmeta = at<unsigned long long>(ws, L.upr);
        AT.tkey = at<unsigned long long>(ws, L.bestA);      // the merger's best-pair keys are dead by now
        const bool use_pts = (int64_t)ntcap * g->n_rows < (int64_t)UINT32_MAX;
        const uint32_t cap = use_pts ? (uint32_t)std::min<int64_t>(2 * (int64_t)std::max(n, 1), UINT32_MAX) : 0u;
        if (use_pts) {
            CK(cudaMemsetAsync(pcnt, 0, 4 * ((size_t)PB + 1), st));
            k_attach_span<<<gt2, B, 0, st>>>(AT, pcnt);
            const int nseq = NF * g->n_sectors * PSPLIT;
            k_attach_rowsum<<<std::max(1, (nseq + 127) / 128), 128, 0, st>>>(pcnt, nseq, g->n_rows, f);
            scan_u32(pcnt, PB, aux, st);
            CK(cudaMemcpyAsync(cursor, pcnt, 4 * ((size_t)PB + 1), cudaMemcpyDeviceToDevice, st));
            g_launches += 2;
        }
        k_attach_trace<<<grid_for(ntcap, 128), 128, 0, st>>>(AT, cursor, pts, pmeta, cap);
        if (use_pts) {
            k_attach_holes<<<grid_for(PB, B), B, 0, st>>>(pcnt, cursor, PB, pmeta, cap, f);
            k_attach_visit<<<grid_for(cap, B), B, 0, st>>>(AT, pcnt, PB, pts, pmeta, cap);
            g_launches += 2;
        }
        k_attach_flags<<<gN, B, 0, st>>>(AT);
        g_launches += 2;
    }
    CK(mark(10));
    if (dev_counts) {
        k_publish<<<1, 32, 0, st>>>(f, ntcap, dev_counts);
        g_launches++;
    }
    CK(cudaGetLastError());
    return TPC_OK;
}

// tables and offsets a call reads from the workspace (pageable uploads)
int upload(const tpc_geometry* g, const Layout& L, const int32_t* offsets, void* ws, cudaStream_t st)
{
    static_assert(sizeof(Layout) <= 1024, "layout header");
    float tab[ROWTAB * 256];
    fill_rowtab(tab, g, L.ny);
    CK(cudaMemcpyAsync(at<float>(ws, L.rowtab), tab, sizeof(tab), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(at<int32_t>(ws, L.offsets), offsets, sizeof(int32_t) * (L.nframes + 1),
                       cudaMemcpyHostToDevice, st));
    // a copy of the layout at the workspace base lets later calls find the arrays
    CK(cudaMemcpyAsync(at<char>(ws, L.hdr), &L, sizeof(Layout), cudaMemcpyHostToDevice, st));
    return TPC_OK;
}

int run_sync(const tpc_params* p, const tpc_geometry* g, float bz, float v_drift, const tpc_clusters* cl,
             int32_t nframes, const int32_t* offsets, void* ws, size_t ws_bytes, tpc_tracks* out, void* stream)
{
    int rc = check_args(p, g);
    if (rc) return rc;
    if (!cl || !out || !ws || cl->n < 0) return TPC_ERR_ARG;
    const int n = cl->n;
    if (n > 0 && (!cl->sector || !cl->row || !cl->y || !cl->zt)) return TPC_ERR_ARG;
    if ((rc = out_args(p, out))) return rc;
    if ((rc = check_frames(n, nframes, offsets))) return rc;
    const Layout L = make_layout(p, g, n, nframes);
    if (ws_bytes < L.total) return TPC_ERR_CAPACITY;
    cudaStream_t st = (cudaStream_t)stream;
    out->n_tracks = out->n_tracklets = out->n_segments = out->n_rejected = 0;
    out->tracklets_needed = out->tracks_needed = out->clusters_needed = 0;
    out->n_launches = 0;
    for (int k = 0; k < TPC_N_STAGES; k++) out->stage_ms[k] = 0.0f;
    for (int k = 0; k < 5; k++) out->work[k] = 0;
    if (n == 0) {
        CK(cudaMemsetAsync(out->clus_offset, 0, sizeof(int32_t), st));
        CK(cudaStreamSynchronize(st));
        return TPC_OK;
    }
    const bool prof = p->profile != 0;
    if (prof) {
        int dev = 0;
        CK(cudaGetDevice(&dev));
        if (g_events.device != dev) {
            for (int k = 0; k <= TPC_N_STAGES; k++) CK(cudaEventCreate(&g_events.ev[k]));
            g_events.device = dev;
        }
    }
    if ((rc = upload(g, L, offsets, ws, st))) return rc;
    if ((rc = enqueue(p, g, bz, v_drift, cl, ws, L, out, nullptr, st, prof))) return rc;
    Frame hf;
    CK(cudaMemcpyAsync(&hf, at<Frame>(ws, L.frame), sizeof(Frame), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    const int ntcap = L.ntcap;
    out->n_launches = g_launches;
    out->work[0] = (int64_t)hf.w_prop;
    out->work[1] = (int64_t)hf.w_upd;
    out->work[2] = (int64_t)hf.w_cand;
    out->work[3] = (int64_t)hf.w_refit_prop;
    out->work[4] = (int64_t)hf.w_merge;
    if (prof)
        for (int k = 0; k < TPC_N_STAGES; k++)
            CK(cudaEventElapsedTime(&out->stage_ms[k], g_events.ev[k], g_events.ev[k + 1]));
    out->n_tracklets = std::min(hf.n_starts, ntcap);
    out->n_segments = hf.n_seg;
    out->n_tracks = hf.n_tracks;
    out->n_rejected = hf.n_rejected;
    if (hf.err == TPC_ERR_DATA) return TPC_ERR_DATA;
    if (hf.n_starts > ntcap) {
        out->tracklets_needed = hf.n_starts;
        return TPC_ERR_CAPACITY;
    }
    if (hf.err == TPC_ERR_CAPACITY) {
        out->tracks_needed = hf.n_tracks;
        out->clusters_needed = hf.n_clus;
        return TPC_ERR_CAPACITY;
    }
    return TPC_OK;
}

}  // namespace

extern "C" {

int tpc_params_default(tpc_params* p)
{
    if (!p) return TPC_ERR_ARG;
    memset(p, 0, sizeof(*p));
    p->dy_link = 3.0f;
    p->dz_link = 3.0f;
    p->s_max_link = 0.5f;
    p->sigma_y = 0.1f;
    p->sigma_z = 0.15f;
    p->c0_snp = 0.25f;
    p->c0_tgl = 0.25f;
    p->c0_qpt = 100.0f;
    p->win_nsigma = 3.0f;
    p->win_min = 0.5f;
    p->win_max = 3.0f;
    p->chi2_cut = 10.0f;
    p->max_miss = 8;
    p->min_hits = 10;
    p->min_owned = 10;
    p->edge_margin = 1.0f;
    p->merge_dz = 10.0f;
    p->merge_chi2 = 50.0f;
    p->refit_passes = 3;
    p->refit_inflate = 100.0f;
    p->z_cell = 5.0f;
    p->y_bins = 16;
    p->max_z_cells = 1024;
    p->tracklets_per_1k = 125;
    p->queue_blocks_per_sm = 0;
    p->fp64_final = 0;
    p->profile = 0;
    p->packed_links = 0;
    p->merge_pairs_per_1k = 4000;
    p->tube_radius = 1.5f;
    p->pt_min_physics = 0.05f;
    p->outlier_chi2 = 25.0f;
    p->looper_qpt_min = 5.0f;
    return TPC_OK;
}

int tpc_workspace_size_batched(const tpc_params* p, const tpc_geometry* g, int64_t n, int32_t n_frames, size_t* bytes)
{
    if (!bytes || n < 0 || n > MAX_CLUSTERS || n_frames < 1 || n_frames > MAX_FRAMES) return TPC_ERR_ARG;
    int rc = check_args(p, g);
    if (rc) return rc;
    const Layout L = make_layout(p, g, n, n_frames);
    if (L.ncells >= (int64_t)UINT32_MAX) return TPC_ERR_ARG;
    *bytes = L.total;
    return TPC_OK;
}

int tpc_workspace_size(const tpc_params* p, const tpc_geometry* g, int64_t n, size_t* bytes)
{
    return tpc_workspace_size_batched(p, g, n, 1, bytes);
}

int tpc_track(const tpc_params* p, const tpc_geometry* g, float bz, float v_drift, const tpc_clusters* cl,
              void* ws, size_t ws_bytes, tpc_tracks* out, void* stream)
{
    if (!cl) return TPC_ERR_ARG;
    const int32_t off[2] = {0, cl->n};
    return run_sync(p, g, bz, v_drift, cl, 1, off, ws, ws_bytes, out, stream);
}

int tpc_track_batched(const tpc_params* p, const tpc_geometry* g, float bz, float v_drift, const tpc_clusters* cl,
                      int32_t n_frames, const int32_t* frame_offsets, void* ws, size_t ws_bytes, tpc_tracks* out,
                      void* stream)
{
    return run_sync(p, g, bz, v_drift, cl, n_frames, frame_offsets, ws, ws_bytes, out, stream);
}

int tpc_prepare(const tpc_params* p, const tpc_geometry* g, int32_t n_clusters, int32_t n_frames,
                const int32_t* frame_offsets, void* ws, size_t ws_bytes, void* stream)
{
    int rc = check_args(p, g);
    if (rc) return rc;
    if (!ws || n_clusters < 1) return TPC_ERR_ARG;
    if ((rc = check_frames(n_clusters, n_frames, frame_offsets))) return rc;
    const Layout L = make_layout(p, g, n_clusters, n_frames);
    if (ws_bytes < L.total) return TPC_ERR_CAPACITY;
    cudaStream_t st = (cudaStream_t)stream;
    if ((rc = upload(g, L, frame_offsets, ws, st))) return rc;
    CK(cudaStreamSynchronize(st));
    return TPC_OK;
}

// staging: the layout header (512 bytes), the row table, the frame offsets
constexpr size_t STAGE_HDR = 1024;
constexpr size_t STAGE_TAB = sizeof(float) * ROWTAB * 256;

int tpc_prepare_staging_size(int32_t n_frames, size_t* bytes)
{
    if (!bytes || n_frames < 1 || n_frames > MAX_FRAMES) return TPC_ERR_ARG;
    *bytes = STAGE_HDR + STAGE_TAB + sizeof(int32_t) * ((size_t)n_frames + 1);
    return TPC_OK;
}

int tpc_prepare_async(const tpc_params* p, const tpc_geometry* g, int32_t n_clusters, int32_t n_frames,
                      const int32_t* frame_offsets, void* host_staging, size_t staging_bytes, void* ws,
                      size_t ws_bytes, void* stream)
{
    int rc = check_args(p, g);
    if (rc) return rc;
    if (!ws || !host_staging || n_clusters < 1) return TPC_ERR_ARG;
    if ((rc = check_frames(n_clusters, n_frames, frame_offsets))) return rc;
    size_t need;
    if ((rc = tpc_prepare_staging_size(n_frames, &need))) return rc;
    if (staging_bytes < need) return TPC_ERR_CAPACITY;
    const Layout L = make_layout(p, g, n_clusters, n_frames);
    if (ws_bytes < L.total) return TPC_ERR_CAPACITY;
    static_assert(sizeof(Layout) <= STAGE_HDR, "layout header");
    char* h = static_cast<char*>(host_staging);
    memcpy(h, &L, sizeof(Layout));
    fill_rowtab(reinterpret_cast<float*>(h + STAGE_HDR), g, L.ny);
    memcpy(h + STAGE_HDR + STAGE_TAB, frame_offsets, sizeof(int32_t) * ((size_t)n_frames + 1));
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaMemcpyAsync(at<char>(ws, L.hdr), h, sizeof(Layout), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(at<float>(ws, L.rowtab), h + STAGE_HDR, STAGE_TAB, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(at<int32_t>(ws, L.offsets), h + STAGE_HDR + STAGE_TAB, sizeof(int32_t) * ((size_t)n_frames + 1),
                       cudaMemcpyHostToDevice, st));
    return TPC_OK;
}

int tpc_track_async(const tpc_params* p, const tpc_geometry* g, float bz, float v_drift, const tpc_clusters* cl,
                    int32_t n_frames, void* ws, size_t ws_bytes, tpc_tracks* out, int32_t* dev_counts, void* stream)
{
    int rc = check_args(p, g);
    if (rc) return rc;
    if (!cl || !out || !ws || !dev_counts || cl->n < 1) return TPC_ERR_ARG;
    if (!cl->sector || !cl->row || !cl->y || !cl->zt) return TPC_ERR_ARG;
    if ((rc = out_args(p, out))) return rc;
    if (n_frames < 1 || n_frames > MAX_FRAMES) return TPC_ERR_ARG;
    const Layout L = make_layout(p, g, cl->n, n_frames);
    if (ws_bytes < L.total) return TPC_ERR_CAPACITY;
    rc = enqueue(p, g, bz, v_drift, cl, ws, L, out, dev_counts, (cudaStream_t)stream, false);
    out->n_launches = g_launches;
    return rc;
}

int tpc_export_tracklets(const void* ws, int32_t capacity, int32_t hits_stride, int32_t* start, int32_t* nhits,
                         uint8_t* kept, int32_t* hits, float* top, float* bot, int32_t* nt_out, void* stream)
{
    if (!ws || !nt_out || capacity < 0) return TPC_ERR_ARG;
    if (capacity > 0 && (!start || !nhits || !kept || !hits || !top || !bot)) return TPC_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaStreamSynchronize(st));
    Layout L;
    CK(cudaMemcpy(&L, ws, sizeof(Layout), cudaMemcpyDeviceToHost));
    if (L.magic != WS_MAGIC || L.hdr != 0) return TPC_ERR_ARG;
    if (hits_stride < L.nr) return TPC_ERR_ARG;
    Frame F;
    CK(cudaMemcpy(&F, static_cast<const char*>(ws) + L.frame, sizeof(Frame), cudaMemcpyDeviceToHost));
    const int nt = std::min(F.n_starts, L.ntcap);
    *nt_out = nt;
    if (capacity < nt) return TPC_ERR_CAPACITY;
    const int nr = L.nr;
    const int n = std::max(L.n, 1);
    std::vector<int32_t> id(nt), nh(nt), nup(nt), h((size_t)nt * nr), ids(n);
    std::vector<float> tp((size_t)nt * NST), bt((size_t)nt * NST);
    std::vector<uint8_t> kp(nt);
    auto get = [&](void* dst, size_t off, size_t bytes) {
        return bytes ? cudaMemcpy(dst, static_cast<const char*>(ws) + off, bytes, cudaMemcpyDeviceToHost) : cudaSuccess;
    };
    CK(get(id.data(), L.t_id, 4 * (size_t)nt));
    CK(get(nh.data(), L.t_nhits, 4 * (size_t)nt));
    CK(get(nup.data(), L.t_nup, 4 * (size_t)nt));
    CK(get(h.data(), L.t_hits, 4 * (size_t)nt * nr));
    CK(get(tp.data(), L.t_top, 4 * (size_t)nt * NST));
    CK(get(bt.data(), L.t_bot, 4 * (size_t)nt * NST));
    CK(get(kp.data(), L.t_kept, (size_t)nt));
    // the input index is the third word of each 16-byte sorted-cluster record
    if (L.n > 0)
        CK(cudaMemcpy2D(ids.data(), sizeof(int32_t), static_cast<const char*>(ws) + L.sc + 2 * sizeof(float),
                        4 * sizeof(float), sizeof(int32_t), (size_t)L.n, cudaMemcpyDeviceToHost));
    std::vector<int> order(nt);
    for (int i = 0; i < nt; i++) order[i] = i;
    std::sort(order.begin(), order.end(), [&](int a, int b) { return id[a] < id[b]; });
    for (int k = 0; k < nt; k++) {
        const int t = order[k];
        start[k] = id[t];
        nhits[k] = nh[t];
        kept[k] = kp[t];
        const int nd = nh[t] - nup[t];
        int32_t* row = hits + (size_t)k * hits_stride;
        for (int q = 0; q < hits_stride; q++) row[q] = -1;
        for (int q = 0; q < nh[t]; q++) {
            const int hs = q < nd ? h[(size_t)t * nr + nr - nd + q] : h[(size_t)t * nr + q - nd];
            row[q] = ids[hs];
        }
        memcpy(top + (size_t)k * NST, &tp[(size_t)t * NST], NST * sizeof(float));
        memcpy(bot + (size_t)k * NST, &bt[(size_t)t * NST], NST * sizeof(float));
    }
    return TPC_OK;
}

int tpc_links_static(const tpc_params* p, const tpc_geometry* g, float v_drift, const tpc_clusters* cl,
                     int32_t* link_up, int32_t* link_dn, uint8_t* is_start, void* stream)
{
    int rc = check_args(p, g);
    if (rc) return rc;
    if (!cl || cl->n < 0 || !link_up || !link_dn) return TPC_ERR_ARG;
    const int n = cl->n;
    if (n > TPC_LINKS_STATIC_MAX_CLUSTERS) return TPC_ERR_CAPACITY;
    if (n > 0 && (!cl->sector || !cl->row || !cl->y || !cl->zt)) return TPC_ERR_ARG;
    if (g->n_sectors * g->n_rows > STATIC_MAX_PLANES) return TPC_ERR_ARG;
    if (n == 0) return TPC_OK;
    void* base = nullptr;
    rc = static_scratch(&base);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    Frame* f = at<Frame>(base, SL.frame);
    FrameGrid* fg = at<FrameGrid>(base, SL.fgrid);
    int32_t* offsets = at<int32_t>(base, SL.offsets);
    float* rowtab = at<float>(base, SL.rowtab);
    float* zlin = at<float>(base, SL.zlin);
    uint16_t* cfr = at<uint16_t>(base, SL.cfr);
    uint32_t* cell = at<uint32_t>(base, SL.cell);
    uint32_t* slot = at<uint32_t>(base, SL.slot);
    uint32_t* cstart = at<uint32_t>(base, SL.cstart);
    uint32_t* aux = at<uint32_t>(base, SL.scan);
    float4* sc = at<float4>(base, SL.sc);
    int32_t* upr = at<int32_t>(base, SL.upr);
    int32_t* dnr = at<int32_t>(base, SL.dnr);
    int32_t* up = at<int32_t>(base, SL.up);
    int32_t* dn = at<int32_t>(base, SL.dn);
    float tab[ROWTAB * 256];
    fill_rowtab(tab, g, 1);   // one y-bin per z-cell: a smaller fixed array
    CK(cudaMemcpyAsync(rowtab, tab, sizeof(tab), cudaMemcpyHostToDevice, st));
    const int32_t off[2] = {0, n};
    CK(cudaMemcpyAsync(offsets, off, sizeof(off), cudaMemcpyHostToDevice, st));
    const int np = g->n_sectors * g->n_rows;
    const int64_t ncells = (int64_t)np * STATIC_NZ;
    const int B = 256;
    const int gN = grid_for(n, B);
    k_init_frame<<<1, 32, 0, st>>>(f, fg, 1);
    k_prep<false><<<dim3(gN, 1), B, 0, st>>>(offsets, cl->sector, cl->row, cl->y, cl->zt, g->n_sectors, g->n_rows,
                                             g->continuous, g->z_max, v_drift, zlin, cfr, f, fg, np, nullptr, nullptr);
    k_grid_setup<<<1, 32, 0, st>>>(f, fg, 1, np, 1, p->z_cell, STATIC_NZ, (long long)ncells, 0.25f * p->merge_dz,
                                   MAX_MERGE_CELLS, 0);
    // the histogram must start at zero: the scratch keeps the previous call's contents
    k_zero_cells<<<grid_for(ncells + 1, B), B, 0, st>>>(cstart, f);
    k_hist<<<gN, B, 0, st>>>(n, cl->sector, cl->row, cl->y, zlin, cfr, rowtab, g->n_rows, g->n_sectors, f, fg, cstart,
                             cell, slot);
    scan_u32(cstart, ncells, aux, st, &f->total_cells);
    k_scatter<<<gN, B, 0, st>>>(n, cl->sector, cl->row, cl->y, zlin, cfr, g->n_rows, np, cstart, cell, slot, sc, f,
                                nullptr);
    k_neighbours<false><<<gN, B, 0, st>>>(n, g->n_rows, g->n_sectors, np, rowtab, sc, cstart, f, fg,
                                          p->dy_link, p->dz_link, p->s_max_link, upr, dnr, nullptr);
    k_clean<<<gN, B, 0, st>>>(n, upr, dnr, up, dn, f);
    k_export_links<<<gN, B, 0, st>>>(n, sc, upr, dnr, up, dn, nullptr, nullptr, link_up, link_dn, is_start, f);
    CK(cudaGetLastError());
    int err = 0;
    CK(cudaMemcpyAsync(&err, &f->err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return err ? err : TPC_OK;
}

const char* tpc_error_string(int code)
{
    switch (code) {
    case TPC_OK: return "ok";
    case TPC_ERR_ARG: return "invalid argument";
    case TPC_ERR_CAPACITY: return "workspace or output capacity too small";
    case TPC_ERR_TIMEOUT: return "bounded device wait timed out";
    case TPC_ERR_CUDA: return "CUDA runtime error";
    case TPC_ERR_DATA: return "invalid cluster data (sector/row out of range or non-finite coordinate)";
    default: return "unknown error";
    }
}

}  // extern "C"
