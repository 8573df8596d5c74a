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

#ifdef __cplusplus
}
#endif
#endif
