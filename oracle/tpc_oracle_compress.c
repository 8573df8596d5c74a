/*
 * tpc_oracle_compress.c -- plain CPU oracle of the cluster compression
 * (paper, section "TPC Data Compression": an integer cluster format with as
 * many bits as the intrinsic resolution needs, residuals of the clusters to
 * their tracks for attached clusters and position differences otherwise, a
 * standard entropy coder -- ANS among those the paper names).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by tests/, never by the product path.
 * Shares no code with the CUDA tracker.
 *
 * Readings of what the paper leaves open:
 *   - integer format: qy = nearest integer to y * 2^ey, qt = nearest integer
 *     to zt * 2^et (ties to even; ey = 5: 1/32 cm, a third of the 0.1 cm
 *     cluster error; et = 6: 1/64 us of drift time, 0.04 cm at 2.58 cm/us);
 *   - residuals to the track: the clusters of a track in its output order
 *     (innermost first) form runs of one sector; the first cluster of a run is
 *     stored whole (sector, row, qy, qt), each later one as its row step and
 *     its residuals to a prediction the decoder can repeat from what it has
 *     already decoded: the previous cluster of the run, or the straight line
 *     through the previous two, in row (integer arithmetic, the division
 *     truncated toward zero; the previous value when those two share a
 *     row);
 *   - clusters attached to no track: per (sector, row) plane, in ascending
 *     (qt, qy, input index), their number, the first qt and then qt steps,
 *     and qy;
 *   - entropy coder: every field is a stream of unsigned integers (zigzag for
 *     signed ones); values below 252 are byte symbols, larger ones an escape
 *     symbol 251 + k followed by the k bytes of v - 252 in a side stream; each
 *     stream is coded by rANS with 32-bit state, 12-bit frequencies and byte
 *     renormalisation (state kept in [2^23, 2^31)), in independent chunks of
 *     a fixed number of symbols, with one static frequency table per stream
 *     normalised from its histogram by largest remainders (every present
 *     symbol at least 1; the rule is stated at orc_rans_normalise).
 *
 * Pins (tests/test_oracle_compress.py): exact round trip of the whole
 * format and of the coder alone; coded size against the entropy of the
 * normalised tables; the quantisation error bound; zero residuals for tracks
 * whose integer positions lie on a line in row; the table normalisation's
 * invariants.
 *
 * Build: as tpc_oracle.c.
 */
#include "tpc_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define RANS_L     (1u << 23)
#define RANS_BITS  12
#define RANS_M     (1u << RANS_BITS)

/* ------------------------------------------------------------ rANS coder */

/* Normalised frequencies (sum RANS_M) of a histogram of byte symbols, 0 for
 * absent symbols (largest remainder): f = floor(M h / N); the M - sum f
 * missing units go, one each, to the present symbols with the largest
 * remainders (M h) mod N, ties to the smaller symbol; then every present
 * symbol left at 0 gets 1, the surplus taken back one unit at a time from the
 * largest frequency above 1 (ties to the smaller symbol).  Returns 0, or -1
 * for an empty histogram. */
int orc_rans_normalise(const uint32_t *hist, uint32_t *freq)
{
    uint64_t total = 0;
    for (int s = 0; s < 256; s++) total += hist[s];
    if (total == 0) {
        for (int s = 0; s < 256; s++) freq[s] = 0;
        return -1;
    }
    uint64_t rem[256];
    uint8_t got[256];
    int64_t sum = 0;
    for (int s = 0; s < 256; s++) {
        const uint64_t m = (uint64_t)hist[s] * RANS_M;
        freq[s] = (uint32_t)(m / total);
        rem[s] = m % total;
        got[s] = 0;
        sum += freq[s];
    }
    while (sum < (int64_t)RANS_M) {
        int best = -1;
        for (int s = 0; s < 256; s++) {
            if (hist[s] == 0 || got[s]) continue;
            if (best < 0 || rem[s] > rem[best]) best = s;
        }
        if (best < 0) return -2;          /* cannot happen: fewer missing units than present symbols */
        freq[best]++;
        got[best] = 1;
        sum++;
    }
    for (int s = 0; s < 256; s++)
        if (hist[s] > 0 && freq[s] == 0) { freq[s] = 1; sum++; }
    while (sum > (int64_t)RANS_M) {
        int best = -1;
        for (int s = 0; s < 256; s++) {
            if (freq[s] <= 1) continue;
            if (best < 0 || freq[s] > freq[best]) best = s;
        }
        if (best < 0) return -2;          /* cannot happen: 256 frequencies of 1 sum to 256 */
        freq[best]--;
        sum--;
    }
    return 0;
}

/* Code n symbols with the table freq: the bytes come out in decode order in
 * out[0..*nbytes).  The symbols are coded last to first; the final state is
 * written first (4 bytes, most significant first), then the renormalisation
 * bytes of the symbols in decode order.  out must hold 4 + 2 n bytes. */
int orc_rans_encode(const uint8_t *sym, int32_t n, const uint32_t *freq, uint8_t *out, int32_t *nbytes)
{
    uint32_t cum[257];
    cum[0] = 0;
    for (int s = 0; s < 256; s++) cum[s + 1] = cum[s] + freq[s];
    if (cum[256] != RANS_M) return -1;
    /* bytes are produced in reverse; collect them at the end of a scratch
     * buffer and move them to the front */
    size_t cap = 4 + 2 * (size_t)(n > 0 ? n : 0);
    uint8_t *tmp = (uint8_t *)malloc(cap > 0 ? cap : 1);
    size_t p = cap;
    uint32_t x = RANS_L;
    for (int32_t i = n - 1; i >= 0; i--) {
        uint32_t f = freq[sym[i]];
        if (f == 0) { free(tmp); return -2; }
        uint32_t xmax = ((RANS_L >> RANS_BITS) << 8) * f;
        while (x >= xmax) { tmp[--p] = (uint8_t)(x & 0xFF); x >>= 8; }
        x = ((x / f) << RANS_BITS) + (x % f) + cum[sym[i]];
    }
    tmp[--p] = (uint8_t)(x & 0xFF);
    tmp[--p] = (uint8_t)((x >> 8) & 0xFF);
    tmp[--p] = (uint8_t)((x >> 16) & 0xFF);
    tmp[--p] = (uint8_t)(x >> 24);
    *nbytes = (int32_t)(cap - p);
    memcpy(out, tmp + p, cap - p);
    free(tmp);
    return 0;
}

/* Inverse of orc_rans_encode: n symbols from in[0..nbytes). */
int orc_rans_decode(const uint8_t *in, int32_t nbytes, const uint32_t *freq, int32_t n, uint8_t *sym)
{
    uint32_t cum[257];
    uint8_t slot2sym[RANS_M];
    cum[0] = 0;
    for (int s = 0; s < 256; s++) {
        cum[s + 1] = cum[s] + freq[s];
        for (uint32_t k = cum[s]; k < cum[s + 1] && k < RANS_M; k++) slot2sym[k] = (uint8_t)s;
    }
    if (cum[256] != RANS_M || nbytes < 4) return -1;
    int32_t p = 0;
    uint32_t x = ((uint32_t)in[0] << 24) | ((uint32_t)in[1] << 16) | ((uint32_t)in[2] << 8) | in[3];
    p = 4;
    for (int32_t i = 0; i < n; i++) {
        uint32_t slot = x & (RANS_M - 1);
        uint8_t s = slot2sym[slot];
        sym[i] = s;
        x = freq[s] * (x >> RANS_BITS) + slot - cum[s];
        while (x < RANS_L) {
            if (p >= nbytes) return -2;
            x = (x << 8) | in[p++];
        }
    }
    return p == nbytes && x == RANS_L ? 0 : -3;
}

/* --------------------------------------------------- integer streams */
typedef struct {
    uint32_t *v;
    int64_t n, cap;
} ustream;

static void us_push(ustream *s, uint32_t v)
{
    if (s->n == s->cap) {
        s->cap = s->cap ? 2 * s->cap : 1024;
        s->v = (uint32_t *)realloc(s->v, sizeof(uint32_t) * (size_t)s->cap);
    }
    s->v[s->n++] = v;
}

static uint32_t zz(int64_t v) { return v >= 0 ? (uint32_t)(2 * v) : (uint32_t)(-2 * v - 1); }
static int64_t unzz(uint32_t u) { return (u & 1u) ? -(int64_t)(u >> 1) - 1 : (int64_t)(u >> 1); }

/* prediction of a run's next value from its previous one or two clusters
 * (the previous value when those two share a row: no line through them) */
static int64_t predict(int nprev, int64_t v0, int r0, int64_t v1, int r1, int r)
{
    if (nprev < 2 || r1 == r0) return v1;
    return v1 + ((v1 - v0) * (int64_t)(r - r1)) / (int64_t)(r1 - r0);
}

/* streams of the format, in this order */
enum { S_NT, S_HS, S_HR, S_HY, S_HT, S_DS, S_DR, S_RY, S_RT, S_UN, S_UT, S_UY, N_STREAMS };

static int32_t qround(float v, int e)
{
    return (int32_t)rintf(v * ldexpf(1.0f, e));
}

static const int32_t *cmp_key_qt, *cmp_key_qy;
static int cmp_unatt(const void *a, const void *b)
{
    int32_t i = *(const int32_t *)a, j = *(const int32_t *)b;
    if (cmp_key_qt[i] != cmp_key_qt[j]) return cmp_key_qt[i] < cmp_key_qt[j] ? -1 : 1;
    if (cmp_key_qy[i] != cmp_key_qy[j]) return cmp_key_qy[i] < cmp_key_qy[j] ? -1 : 1;
    return (i > j) - (i < j);
}

/* The integer fields of every stream (before the entropy coder).  vals gets
 * N_STREAMS malloc'ed arrays, counts their lengths. */
int orc_compress_fields(int32_t n_sectors, int32_t n_rows, int32_t n, const uint8_t *sector, const uint8_t *row,
                        const float *y, const float *zt, int32_t ey, int32_t et, int32_t n_tracks,
                        const int32_t *clus_offset, const int32_t *clus_index, const int32_t *assign,
                        uint32_t **vals, int64_t *counts)
{
    ustream S[N_STREAMS];
    memset(S, 0, sizeof(S));
    int32_t *qy = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t *qt = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    for (int32_t i = 0; i < n; i++) {
        qy[i] = qround(y[i], ey);
        qt[i] = qround(zt[i], et);
    }
    /* attached clusters, track by track */
    for (int32_t t = 0; t < n_tracks; t++) {
        int32_t a = clus_offset[t], b = clus_offset[t + 1];
        us_push(&S[S_NT], (uint32_t)(b - a));
        int run = 0, rp0 = 0, rp1 = 0, sec = -1;
        int64_t y0 = 0, y1 = 0, t0 = 0, t1 = 0;
        for (int32_t k = a; k < b; k++) {
            int c = clus_index[k];
            int s = sector[c], r = row[c];
            if (k > a) us_push(&S[S_DS], zz((int64_t)s - sec));
            if (k == a || s != sec) {
                if (k == a) us_push(&S[S_HS], (uint32_t)s);
                us_push(&S[S_HR], (uint32_t)r);
                us_push(&S[S_HY], zz(qy[c]));
                us_push(&S[S_HT], zz(qt[c]));
                run = 1;
            } else {
                us_push(&S[S_DR], zz((int64_t)r - rp1));
                us_push(&S[S_RY], zz((int64_t)qy[c] - predict(run, y0, rp0, y1, rp1, r)));
                us_push(&S[S_RT], zz((int64_t)qt[c] - predict(run, t0, rp0, t1, rp1, r)));
                run++;
            }
            sec = s;
            rp0 = rp1; y0 = y1; t0 = t1;
            rp1 = r; y1 = qy[c]; t1 = qt[c];
        }
    }
    /* the others, plane by plane */
    int NP = n_sectors * n_rows;
    int32_t *cnt = (int32_t *)calloc((size_t)NP + 1, sizeof(int32_t));
    for (int32_t i = 0; i < n; i++)
        if (assign[i] < 0) cnt[sector[i] * n_rows + row[i] + 1]++;
    for (int p = 0; p < NP; p++) cnt[p + 1] += cnt[p];
    int32_t *ord = (int32_t *)malloc(sizeof(int32_t) * (size_t)(cnt[NP] > 0 ? cnt[NP] : 1));
    int32_t *fill = (int32_t *)malloc(sizeof(int32_t) * (size_t)NP);
    memcpy(fill, cnt, sizeof(int32_t) * (size_t)NP);
    for (int32_t i = 0; i < n; i++)
        if (assign[i] < 0) ord[fill[sector[i] * n_rows + row[i]]++] = i;
    cmp_key_qt = qt; cmp_key_qy = qy;
    for (int p = 0; p < NP; p++) {
        int32_t a = cnt[p], b = cnt[p + 1];
        qsort(ord + a, (size_t)(b - a), sizeof(int32_t), cmp_unatt);
        us_push(&S[S_UN], (uint32_t)(b - a));
        for (int32_t k = a; k < b; k++) {
            int c = ord[k];
            us_push(&S[S_UT], k == a ? zz(qt[c]) : (uint32_t)(qt[c] - qt[ord[k - 1]]));
            us_push(&S[S_UY], zz(qy[c]));
        }
    }
    for (int s = 0; s < N_STREAMS; s++) {
        vals[s] = S[s].v ? S[s].v : (uint32_t *)malloc(sizeof(uint32_t));
        counts[s] = S[s].n;
    }
    free(qy); free(qt); free(cnt); free(ord); free(fill);
    return 0;
}

/* Clusters back from the integer fields: sector, row, qy, qt of the attached
 * clusters in track order, then of the others in plane order. */
int orc_decompress_fields(int32_t n_sectors, int32_t n_rows, const uint32_t *const *vals, const int64_t *counts,
                          int32_t n_tracks, int32_t n, uint8_t *sector, uint8_t *row, int32_t *qy, int32_t *qt)
{
    int64_t ix[N_STREAMS];
    memset(ix, 0, sizeof(ix));
#define TAKE(s) (ix[s] < counts[s] ? vals[s][ix[s]++] : (err = 1, 0u))
    int err = 0;
    int32_t o = 0;
    for (int32_t t = 0; t < n_tracks && !err; t++) {
        int32_t m = (int32_t)TAKE(S_NT);
        int run = 0, rp0 = 0, rp1 = 0, sec = -1;
        int64_t y0 = 0, y1 = 0, t0 = 0, t1 = 0;
        for (int32_t k = 0; k < m && !err; k++) {
            int s, r;
            int64_t vy, vt;
            if (k == 0) s = (int)TAKE(S_HS);
            else s = (int)(sec + unzz(TAKE(S_DS)));
            if (k == 0 || s != sec) {
                r = (int)TAKE(S_HR);
                vy = unzz(TAKE(S_HY));
                vt = unzz(TAKE(S_HT));
                run = 1;
            } else {
                r = (int)(rp1 + unzz(TAKE(S_DR)));
                vy = predict(run, y0, rp0, y1, rp1, r) + unzz(TAKE(S_RY));
                vt = predict(run, t0, rp0, t1, rp1, r) + unzz(TAKE(S_RT));
                run++;
            }
            if (o >= n) return -1;
            sector[o] = (uint8_t)s; row[o] = (uint8_t)r; qy[o] = (int32_t)vy; qt[o] = (int32_t)vt;
            o++;
            sec = s;
            rp0 = rp1; y0 = y1; t0 = t1;
            rp1 = r; y1 = vy; t1 = vt;
        }
    }
    for (int p = 0; p < n_sectors * n_rows && !err; p++) {
        int32_t m = (int32_t)TAKE(S_UN);
        int64_t prev = 0;
        for (int32_t k = 0; k < m && !err; k++) {
            uint32_t u = TAKE(S_UT);
            int64_t vt = k == 0 ? unzz(u) : prev + (int64_t)u;
            if (o >= n) return -1;
            sector[o] = (uint8_t)(p / n_rows); row[o] = (uint8_t)(p % n_rows);
            qt[o] = (int32_t)vt; qy[o] = (int32_t)unzz(TAKE(S_UY));
            prev = vt;
            o++;
        }
    }
#undef TAKE
    if (err) return -2;
    for (int s = 0; s < N_STREAMS; s++)
        if (ix[s] != counts[s]) return -3;
    return o == n ? 0 : -4;
}

/* ------------------------------------------------ byte symbols + coder */

/* Byte symbols of an integer stream: v < 252 as itself, else the symbol
 * 251 + k followed by the k bytes (least significant first, k = 1..4 the
 * fewest that hold it) of v - 252 in the raw side stream.  Returns the symbol
 * count; *nraw gets the raw byte count. */
int64_t orc_symbolise(const uint32_t *v, int64_t n, uint8_t *sym, uint8_t *raw, int64_t *nraw)
{
    int64_t r = 0;
    for (int64_t i = 0; i < n; i++) {
        if (v[i] < 252u) { sym[i] = (uint8_t)v[i]; continue; }
        const uint32_t w = v[i] - 252u;
        const int k = w < (1u << 8) ? 1 : w < (1u << 16) ? 2 : w < (1u << 24) ? 3 : 4;
        sym[i] = (uint8_t)(251 + k);
        for (int b = 0; b < k; b++) raw[r++] = (uint8_t)(w >> (8 * b));
    }
    *nraw = r;
    return n;
}

/* Inverse of orc_symbolise.  Returns 0, or -1 when the raw stream does not
 * match the symbols. */
int orc_desymbolise(const uint8_t *sym, int64_t n, const uint8_t *raw, int64_t nraw, uint32_t *v)
{
    int64_t r = 0;
    for (int64_t i = 0; i < n; i++) {
        if (sym[i] < 252) { v[i] = sym[i]; continue; }
        const int k = sym[i] - 251;
        if (r + k > nraw) return -1;
        uint32_t w = 0;
        for (int b = 0; b < k; b++) w |= (uint32_t)raw[r++] << (8 * b);
        v[i] = w + 252u;
    }
    return r == nraw ? 0 : -1;
}

/* Coded size of one stream (bytes: frequency table of 256 x 2 bytes, the
 * chunks' byte counts of 4 bytes each, their coded bytes, the raw side
 * stream), and optionally the round trip of its symbols through the coder.
 * chunk: symbols per rANS chunk. */
int orc_code_stream(const uint32_t *v, int64_t n, int32_t chunk, int64_t *bytes, int32_t *roundtrip_ok)
{
    uint8_t *sym = (uint8_t *)malloc((size_t)(n > 0 ? n : 1));
    uint8_t *raw = (uint8_t *)malloc(4 * (size_t)(n > 0 ? n : 1));   /* at most 4 raw bytes per value */
    int64_t nraw = 0;
    orc_symbolise(v, n, sym, raw, &nraw);
    uint32_t hist[256] = {0}, freq[256];
    for (int64_t i = 0; i < n; i++) hist[sym[i]]++;
    int64_t total = 0;
    int ok = 1;
    if (n > 0) {
        if (orc_rans_normalise(hist, freq)) { free(sym); free(raw); return -1; }
        uint8_t *out = (uint8_t *)malloc(4 + 2 * (size_t)chunk);
        uint8_t *back = (uint8_t *)malloc((size_t)chunk);
        for (int64_t a = 0; a < n; a += chunk) {
            int32_t m = (int32_t)(n - a < chunk ? n - a : chunk), nb = 0;
            if (orc_rans_encode(sym + a, m, freq, out, &nb)) { ok = 0; break; }
            total += nb + 4;
            if (roundtrip_ok) {
                if (orc_rans_decode(out, nb, freq, m, back) || memcmp(back, sym + a, (size_t)m)) ok = 0;
            }
        }
        free(out); free(back);
        total += 2 * 256;
        if (roundtrip_ok) {
            uint32_t *w = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n);
            if (orc_desymbolise(sym, n, raw, nraw, w) || memcmp(w, v, sizeof(uint32_t) * (size_t)n)) ok = 0;
            free(w);
        }
    }
    total += nraw;
    *bytes = total;
    if (roundtrip_ok) *roundtrip_ok = ok;
    free(sym); free(raw);
    return 0;
}

void orc_free_ptr(void *p) { free(p); }

/* --------------------------------------------------- stream container */
/* One coded stream as bytes (all integers little-endian):
 *   u32 n (values), u32 chunk, u32 nraw (escape bytes),
 *   u16 freq[256] (the table; all 0 when n = 0),
 *   u32 chunk_bytes[ceil(n / chunk)], the chunks back to back, the escape
 *   bytes.
 * orc_pack_stream writes it to out (NULL: size only) and returns its size,
 * or -1 on error. */
static void put32(uint8_t *o, int64_t *p, uint32_t v)
{
    if (o) for (int b = 0; b < 4; b++) o[*p + b] = (uint8_t)(v >> (8 * b));
    *p += 4;
}

static uint32_t get32(const uint8_t *in, int64_t p)
{
    return (uint32_t)in[p] | ((uint32_t)in[p + 1] << 8) | ((uint32_t)in[p + 2] << 16) | ((uint32_t)in[p + 3] << 24);
}

int64_t orc_pack_stream(const uint32_t *v, int64_t n, int32_t chunk, uint8_t *out)
{
    if (n < 0 || n > 0xFFFFFFFFLL || chunk < 1) return -1;
    uint8_t *sym = (uint8_t *)malloc((size_t)(n > 0 ? n : 1));
    uint8_t *raw = (uint8_t *)malloc(4 * (size_t)(n > 0 ? n : 1));
    int64_t nraw = 0;
    orc_symbolise(v, n, sym, raw, &nraw);
    uint32_t hist[256] = {0}, freq[256] = {0};
    for (int64_t i = 0; i < n; i++) hist[sym[i]]++;
    if (n > 0 && orc_rans_normalise(hist, freq)) { free(sym); free(raw); return -1; }
    const int64_t nch = n > 0 ? (n + chunk - 1) / chunk : 0;
    int64_t p = 0;
    put32(out, &p, (uint32_t)n);
    put32(out, &p, (uint32_t)chunk);
    put32(out, &p, (uint32_t)nraw);
    for (int s = 0; s < 256; s++) {
        if (out) { out[p] = (uint8_t)(freq[s] & 0xFF); out[p + 1] = (uint8_t)(freq[s] >> 8); }
        p += 2;
    }
    int64_t sizes_at = p;
    p += 4 * nch;
    uint8_t *buf = (uint8_t *)malloc(4 + 2 * (size_t)chunk);
    for (int64_t c = 0; c < nch; c++) {
        const int32_t m = (int32_t)(n - c * chunk < chunk ? n - c * chunk : chunk);
        int32_t nb = 0;
        if (orc_rans_encode(sym + c * chunk, m, freq, buf, &nb)) { free(buf); free(sym); free(raw); return -1; }
        int64_t q = sizes_at + 4 * c;
        put32(out, &q, (uint32_t)nb);
        if (out) memcpy(out + p, buf, (size_t)nb);
        p += nb;
    }
    if (out) memcpy(out + p, raw, (size_t)nraw);
    p += nraw;
    free(buf); free(sym); free(raw);
    return p;
}

/* Inverse of orc_pack_stream: the n values (n read from the container,
 * returned through *n_out; v holds at least that many).  Returns the bytes
 * consumed, or -1 when the container is malformed. */
int64_t orc_unpack_stream(const uint8_t *in, int64_t nbytes, uint32_t *v, int64_t vcap, int64_t *n_out)
{
    if (nbytes < 12 + 512) return -1;
    const int64_t n = get32(in, 0);
    const int32_t chunk = (int32_t)get32(in, 4);
    const int64_t nraw = get32(in, 8);
    if (chunk < 1 || n > vcap) return -1;
    uint32_t freq[256];
    int64_t p = 12;
    for (int s = 0; s < 256; s++, p += 2) freq[s] = (uint32_t)in[p] | ((uint32_t)in[p + 1] << 8);
    const int64_t nch = n > 0 ? (n + chunk - 1) / chunk : 0;
    if (p + 4 * nch > nbytes) return -1;
    const int64_t sizes_at = p;
    p += 4 * nch;
    uint8_t *sym = (uint8_t *)malloc((size_t)(n > 0 ? n : 1));
    for (int64_t c = 0; c < nch; c++) {
        const int32_t m = (int32_t)(n - c * chunk < chunk ? n - c * chunk : chunk);
        const int64_t nb = get32(in, sizes_at + 4 * c);
        if (p + nb > nbytes || orc_rans_decode(in + p, (int32_t)nb, freq, m, sym + c * chunk)) { free(sym); return -1; }
        p += nb;
    }
    if (p + nraw > nbytes || orc_desymbolise(sym, n, in + p, nraw, v)) { free(sym); return -1; }
    p += nraw;
    free(sym);
    *n_out = n;
    return p;
}
