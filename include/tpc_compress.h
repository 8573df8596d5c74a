/*
 * tpc_compress.h -- C ABI of the entropy coder of the cluster compression.
 *
 * Paper: section "TPC Data Compression", step 4: the cluster fields, once
 * reduced to small residuals, go through a standard entropy coder (the
 * paper names Huffman, arithmetic and ANS coding).  This library codes byte
 * symbols with rANS (range asymmetric numeral systems):
 *   - one static frequency table for the whole stream, 12-bit (sum 4096),
 *     from the stream's histogram by largest remainders: f = floor(4096 h /
 *     N); the missing units go one each to the present symbols with the
 *     largest remainders (4096 h) mod N, ties to the smaller symbol; then a
 *     present symbol left at 0 gets 1, the surplus taken back one unit at a
 *     time from the largest frequency above 1, ties to the smaller symbol;
 *   - the stream is cut into chunks of `chunk` symbols (the last one
 *     shorter), each coded independently: 32-bit state starting at 2^23,
 *     symbols coded last to first, byte renormalisation keeping the state in
 *     [2^23, 2^31); a chunk's bytes are its final state (4 bytes, most
 *     significant first) followed by its renormalisation bytes in decode
 *     order -- a decoder reads the state, then for each symbol takes the
 *     slot x mod 4096, the symbol s owning it, sets x = f_s (x >> 12) + slot
 *     - c_s, and shifts in bytes while x < 2^23;
 *   - the coded chunks are stored back to back in chunk order.
 * Everything is integer arithmetic: the bytes are the same on any hardware.
 *
 * All pointers are device memory owned by the caller unless stated.  Work
 * goes on `stream` (a cudaStream_t, NULL for the legacy stream).  Returns
 * TPC_OK or a negative TPC_ERR_* code (tpc_track.h).
 */
#ifndef TPC_COMPRESS_H
#define TPC_COMPRESS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Largest stream and chunk sizes. */
#define TPC_RANS_MAX_SYMBOLS ((int64_t)1 << 31)
#define TPC_RANS_MAX_CHUNK 65536

/* Workspace bytes of tpc_rans_encode for n symbols in chunks of `chunk`
 * (host only; TPC_ERR_ARG for n outside [0, TPC_RANS_MAX_SYMBOLS) or chunk
 * outside [1, TPC_RANS_MAX_CHUNK]). */
int tpc_rans_workspace_size(int64_t n, int32_t chunk, size_t *bytes);

/* Worst-case coded bytes (4 + 2 per symbol per chunk); size `out` for it. */
int tpc_rans_max_bytes(int64_t n, int32_t chunk, int64_t *bytes);

/* Code the n byte symbols `sym` (device) in chunks of `chunk`.
 *   freq        [256] device: the normalised table (0 for absent symbols).
 *   chunk_bytes [ceil(n / chunk)] device: coded bytes of each chunk.
 *   out         device, out_cap bytes (>= tpc_rans_max_bytes): the chunks.
 *   total       host: total coded bytes (the call synchronises `stream` to
 *               read it and the device-side error flag), may be NULL: then
 *               nothing waits and a device-side failure (a table that does
 *               not normalise, a chunk that overflows its slot) is not
 *               reported -- freq, chunk_bytes and out are then unspecified.
 *               Callers that cannot wait should call once with total set
 *               to validate a stream shape, or check the outputs themselves.
 * workspace: device, tpc_rans_workspace_size bytes, caller-owned; its
 * contents need not be initialised.  n = 0 codes nothing (all tables 0).
 * Errors: TPC_ERR_ARG (sizes, null pointers, out_cap too small),
 * TPC_ERR_CUDA. */
int tpc_rans_encode(const uint8_t *sym, int64_t n, int32_t chunk, void *workspace, size_t ws_bytes,
                    uint32_t *freq, int32_t *chunk_bytes, uint8_t *out, int64_t out_cap, int64_t *total,
                    void *stream);

/* ------------------------------------------------------------------------
 * The compressed cluster format (section "TPC Data Compression", steps 1-4)
 * on the GPU: integer cluster fields, residuals of track clusters to their
 * tracks, differences of the other clusters, each field stream entropy coded
 * with the coder above.
 *
 *   integer format: qy = nearest integer to y 2^ey, qt = nearest integer to
 *     zt 2^et (binary32 product, ties to even);
 *   clusters of tracks, track by track in output order: per track its cluster
 *     count (NT); its clusters form runs of one sector; the first cluster of a
 *     run is stored whole -- sector (HS, first run of a track only; later runs
 *     as the sector step DS, which every cluster after the first carries),
 *     row (HR), zigzag qy (HY), zigzag qt (HT) -- each later one as its row
 *     step (DR) and the zigzag residuals of qy and qt (RY, RT) to a
 *     prediction from the run's previous clusters: the previous value after
 *     one cluster, the line through the previous two (in row, integer
 *     arithmetic, quotient truncated toward zero) after two or more -- the
 *     previous value when those two share a row;
 *   other clusters (assign < 0), plane by plane (sector-major), sorted by
 *     (qt, qy, input index): their count (UN), zigzag qt of the first and qt
 *     steps after it (UT), zigzag qy (UY);
 *   zigzag(v) = 2v for v >= 0, -2v - 1 otherwise (as uint32).
 * Stream order: NT, HS, HR, HY, HT, DS, DR, RY, RT, UN, UT, UY.
 *
 * Each stream is coded as a container (integers little-endian):
 *   u32 n (values), u32 chunk, u32 nraw, u16 freq[256], u32
 *   chunk_bytes[ceil(n / chunk)], the rANS chunks back to back, the escape
 *   bytes; a value v < 252 is the byte symbol v, a larger one the symbol
 *   251 + k followed by the k little-endian bytes (k = 1..4, the fewest that
 *   hold it) of v - 252 in the escape bytes.
 * ---------------------------------------------------------------------- */
#define TPC_CMP_N_STREAMS 12

typedef struct {
    int64_t n;                    /* clusters */
    int32_t n_sectors, n_rows;    /* planes: n_sectors x n_rows (<= 255 rows) */
    const uint8_t *sector;        /* [n] device */
    const uint8_t *row;           /* [n] device */
    const float *y;               /* [n] device, local y (cm) */
    const float *zt;              /* [n] device, drift time (us) or z (cm) */
    int32_t n_tracks;
    int64_t n_attached;           /* clus_offset[n_tracks] (host value) */
    const int32_t *clus_offset;   /* [n_tracks + 1] device, from 0, non-decreasing */
    const int32_t *clus_index;    /* [n_attached] device, cluster indices, innermost first */
    const int32_t *assign;        /* [n] device, track of each cluster or < 0 */
} tpc_compress_in;

/* Workspace bytes of tpc_compress_fields / tpc_compress_frame (host only). */
int tpc_compress_workspace_size(const tpc_compress_in *in, int32_t chunk, size_t *bytes);

/* Upper bound of the values of all streams together (for tpc_compress_fields)
 * and of the coded bytes of all containers (for tpc_compress_frame). */
int tpc_compress_max_size(const tpc_compress_in *in, int32_t chunk, int64_t *max_values, int64_t *max_bytes);

/* The integer streams only: vals (device, vals_cap uint32) receives the
 * streams back to back in stream order; counts (host, 12) their lengths.
 * Synchronises `stream` to read the lengths.  Errors: TPC_ERR_ARG (null or
 * inconsistent arguments, vals_cap too small), TPC_ERR_DATA (a sector or
 * row out of range, an offset table that is not non-decreasing from 0 to
 * n_attached, a cluster index out of range), TPC_ERR_CUDA. */
int tpc_compress_fields(const tpc_compress_in *in, int32_t ey, int32_t et, void *workspace, size_t ws_bytes,
                        uint32_t *vals, int64_t vals_cap, int64_t *counts, void *stream);

/* The whole compressed frame: the 12 containers back to back in stream order
 * in out (device, out_cap bytes >= max_bytes); bytes (host, 12) the size of
 * each container.  chunk: symbols per rANS chunk (1..TPC_RANS_MAX_CHUNK).
 * Synchronises `stream` (the sizes are read back).  Errors as
 * tpc_compress_fields. */
int tpc_compress_frame(const tpc_compress_in *in, int32_t ey, int32_t et, int32_t chunk, void *workspace,
                       size_t ws_bytes, uint8_t *out, int64_t out_cap, int64_t *bytes, void *stream);

#ifdef __cplusplus
}
#endif
#endif
