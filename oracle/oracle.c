/*
 * oracle.c -- plain, slow, single-threaded CPU oracle for parametric voxel
 * generation of 3D straight-line segments (the "Parametric Method", Section 3).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing on the product path may call this code:
 * only the tests, the smoke check and the CPU-baseline leg of the benchmark use
 * it. It shares no code, header, table or helper with the CUDA library.
 *
 * What it computes (Section 3, Eq. (2)-(3) and the algorithm of Fig. 3):
 *   a segment has start S and end E (integer lattice points);
 *   N is the step count, W = (E - S) / N the step vector, and
 *   G_k = S + W * k for k = 0, 1, ..., N are the sample points;
 *   the voxel of G_k is the lattice point nearest to G_k on each axis.
 *
 * Readings where the paper is silent or garbled:
 *   - N = max(|dx|, |dy|, |dz|) (Chebyshev length), not int(|E - S|) of Eq. (1):
 *     this makes the major axis advance by exactly one voxel per step.
 *   - k runs from 0 to N (Eq. (3)), so the start voxel is included: N + 1 voxels.
 *   - N = 0 (S == E) yields the single voxel S.
 *   - "nearest" on a tie (G_k exactly half-way between two lattice points) picks
 *     the point farther from S.
 *   - the arithmetic is exact: W * k is kept as the rational (E - S) * k / N.
 *   - packed list formats: 32-bit = x | y << 10 | z << 20 (every dim <= 1024),
 *     64-bit = x | y << 21 | z << 42; occupancy volume: bit (x + w*(y + h*z)),
 *     little-endian bit order inside 32-bit words, OR-ed in.
 */
#include <stdint.h>
#include <stddef.h>

/* Status values; the numbering mirrors the public error enum on purpose so a
 * test can compare them, but is written out here independently. */
enum {
    ORACLE_OK = 0,
    ORACLE_ERR_INVALID_ARG = 1,
    ORACLE_ERR_OUT_OF_BOUNDS = 2,
    ORACLE_ERR_PACK_WIDTH = 3
};

static int64_t abs64(int64_t v) { return v < 0 ? -v : v; }

/* N for one segment: the largest coordinate difference (Chebyshev length). */
int64_t oracle_steps(const int32_t *seg)
{
    int64_t n = 0;
    for (int a = 0; a < 3; ++a) {
        int64_t d = abs64((int64_t)seg[3 + a] - (int64_t)seg[a]);
        if (d > n) n = d;
    }
    return n;
}

/*
 * Lattice coordinate nearest to  s + num / den  (den > 0), ties resolved away
 * from s. With m = |num|, the distance from s in whole voxels is the integer q
 * nearest to m / den with halves rounded up:  q = floor((2m + den) / (2 den)).
 * Exact for every int32 input (128-bit intermediate).
 */
static int64_t nearest_away_from_start(int64_t s, __int128 num, int64_t den)
{
    __int128 m = num < 0 ? -num : num;
    __int128 q = (2 * m + den) / (2 * (__int128)den);
    return num < 0 ? s - (int64_t)q : s + (int64_t)q;
}

/* Sample k with N steps: the lattice point nearest to G_k = S + W*k, W = (E-S)/N. */
static void voxel_of_sample(const int32_t *seg, int64_t k, int64_t N, int64_t *out3)
{
    for (int a = 0; a < 3; ++a) {
        int64_t S = seg[a];
        int64_t E = seg[3 + a];
        if (N == 0) {
            out3[a] = S;
        } else {
            /* W_a * k = (E_a - S_a) * k / N, kept as a rational */
            __int128 num = (__int128)(E - S) * k;
            out3[a] = nearest_away_from_start(S, num, N);
        }
    }
}

/* Voxel k of a segment: the lattice point nearest to G_k = S + W*k (Eq. (3)). */
void oracle_voxel(const int32_t *seg, int64_t k, int64_t *out3)
{
    voxel_of_sample(seg, k, oracle_steps(seg), out3);
}

/* Validation of a call: dims in [1, 2^21]; every endpoint inside [0, dim);
 * a 32-bit packed list needs every dim <= 1024. Returns the first error. */
int oracle_validate(const int32_t *segs, int64_t n, const int32_t *dims, int want_list32)
{
    if (n < 0) return ORACLE_ERR_INVALID_ARG;
    for (int a = 0; a < 3; ++a)
        if (dims[a] < 1 || dims[a] > (1 << 21)) return ORACLE_ERR_INVALID_ARG;
    if (want_list32)
        for (int a = 0; a < 3; ++a)
            if (dims[a] > 1024) return ORACLE_ERR_PACK_WIDTH;
    for (int64_t s = 0; s < n; ++s)
        for (int c = 0; c < 6; ++c) {
            int32_t v = segs[6 * s + c];
            if (v < 0 || v >= dims[c % 3]) return ORACLE_ERR_OUT_OF_BOUNDS;
        }
    return ORACLE_OK;
}

/* Per-segment voxel counts N + 1. */
void oracle_count(const int32_t *segs, int64_t n, int32_t *counts)
{
    for (int64_t s = 0; s < n; ++s) counts[s] = (int32_t)(oracle_steps(segs + 6 * s) + 1);
}

/* Exclusive prefix sum of the counts; offsets[n] is the total voxel count V. */
void oracle_offsets(const int32_t *counts, int64_t n, int64_t *offsets)
{
    int64_t run = 0;
    for (int64_t s = 0; s < n; ++s) {
        offsets[s] = run;
        run += counts[s];
    }
    offsets[n] = run;
}

/* The packed list encodings of one voxel. */
static uint32_t pack32(const int64_t *v)
{
    return (uint32_t)v[0] | ((uint32_t)v[1] << 10) | ((uint32_t)v[2] << 20);
}

static uint64_t pack64(const int64_t *v)
{
    return (uint64_t)v[0] | ((uint64_t)v[1] << 21) | ((uint64_t)v[2] << 42);
}

/* Fig. 3 for every segment in order: append voxel k for k = 0..N.
 * At most `cap` words are written; the return value is V, the number the
 * segments produce, so V > cap tells the caller the buffer was too small. */
int64_t oracle_list32(const int32_t *segs, int64_t n, uint32_t *out, int64_t cap)
{
    int64_t g = 0;
    for (int64_t s = 0; s < n; ++s) {
        const int32_t *seg = segs + 6 * s;
        int64_t N = oracle_steps(seg);
        for (int64_t k = 0; k <= N; ++k) {
            int64_t v[3];
            oracle_voxel(seg, k, v);
            if (g < cap) out[g] = pack32(v);
            ++g;
        }
    }
    return g;
}

int64_t oracle_list64(const int32_t *segs, int64_t n, uint64_t *out, int64_t cap)
{
    int64_t g = 0;
    for (int64_t s = 0; s < n; ++s) {
        const int32_t *seg = segs + 6 * s;
        int64_t N = oracle_steps(seg);
        for (int64_t k = 0; k <= N; ++k) {
            int64_t v[3];
            oracle_voxel(seg, k, v);
            if (g < cap) out[g] = pack64(v);
            ++g;
        }
    }
    return g;
}

/* Sets bit lin of the volume: bit lin % 32 of word lin / 32 (little-endian). */
static void set_bit(uint32_t *mask, uint64_t lin)
{
    mask[lin / 32] |= (uint32_t)1 << (lin % 32);
}

/* OR every voxel of every segment into the occupancy volume of n_words words.
 * Returns V, or -1 if some voxel fell outside the volume (that bit is skipped). */
int64_t oracle_bitmask(const int32_t *segs, int64_t n, const int32_t *dims, uint32_t *mask,
                       int64_t n_words)
{
    int64_t w = dims[0], h = dims[1];
    int64_t g = 0;
    int outside = 0;
    for (int64_t s = 0; s < n; ++s) {
        const int32_t *seg = segs + 6 * s;
        int64_t N = oracle_steps(seg);
        for (int64_t k = 0; k <= N; ++k) {
            int64_t v[3];
            oracle_voxel(seg, k, v);
            uint64_t lin = (uint64_t)(v[0] + w * (v[1] + h * v[2]));
            if (lin / 32 < (uint64_t)n_words)
                set_bit(mask, lin);
            else
                outside = 1;
            ++g;
        }
    }
    return outside ? -1 : g;
}

/* z of voxel k of a segment with N steps (Eq. (3), as oracle_voxel). */
static int64_t voxel_z(const int32_t *seg, int64_t k, int64_t N)
{
    int64_t v[3];
    voxel_of_sample(seg, k, N, v);
    return v[2];
}

/* The smallest k in [0, N + 1] at which "z(k) >= zt" (rising: dz >= 0) or
 * "z(k) < zt" (falling: dz < 0) holds, N + 1 if none: along a segment z moves
 * monotonically from S_z to E_z (the rounding of Eq. (3) is monotone in k), so
 * the predicate is false up to some k and true from there on, and bisection
 * finds that k. */
static int64_t first_step_past(const int32_t *seg, int64_t N, int64_t zt, int rising)
{
    int64_t lo = 0, hi = N + 1;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        int64_t z = voxel_z(seg, mid, N);
        int holds = rising ? (z >= zt) : (z < zt);
        if (holds)
            hi = mid;
        else
            lo = mid + 1;
    }
    return lo;
}

/* The part of the occupancy volume with z in [z0, z1): the voxels of every
 * segment with z0 <= z < z1 (Eq. (3), as oracle_bitmask) OR-ed into `slab`, a
 * volume of w x h x (z1 - z0) voxels whose bit index is x + w * (y + h * (z - z0)).
 * When z0 * w * h is a multiple of 32, slab word j is word j + z0 * w * h / 32 of
 * the whole volume, so a large volume can be checked slab by slab. The voxels of
 * a segment inside the slab are those of one range of k (z is monotone in k),
 * found by bisection; each is still tested against the slab. Returns the number
 * of voxels OR-ed in, or -1 if the slab has fewer than n_words words for them. */
int64_t oracle_bitmask_zslab(const int32_t *segs, int64_t n, const int32_t *dims, int64_t z0, int64_t z1,
                             uint32_t *slab, int64_t n_words)
{
    const int64_t w = dims[0];
    const int64_t h = dims[1];
    int64_t in_slab = 0;
    int outside = 0;
    for (int64_t s = 0; s < n; ++s) {
        const int32_t *seg = segs + 6 * s;
        int64_t N = oracle_steps(seg);
        int rising = seg[5] >= seg[2];
        int64_t kb = first_step_past(seg, N, rising ? z0 : z1, rising);
        int64_t ke = first_step_past(seg, N, rising ? z1 : z0, rising);
        for (int64_t k = kb; k < ke; ++k) {
            int64_t v[3];
            oracle_voxel(seg, k, v);
            if (v[2] < z0 || v[2] >= z1) continue;
            uint64_t bit = (uint64_t)(v[0] + w * v[1] + w * h * (v[2] - z0));
            if (bit / 32 < (uint64_t)n_words)
                slab[bit / 32] |= (uint32_t)1 << (bit % 32);
            else
                outside = 1;
            ++in_slab;
        }
    }
    return outside ? -1 : in_slab;
}

/* Voxels of segments [s_begin, s_end) only, written as x, y, z triples; at most
 * `cap` voxels are written, the return value is the number produced. */
int64_t oracle_voxels_xyz(const int32_t *segs, int64_t s_begin, int64_t s_end, int64_t *xyz,
                          int64_t cap)
{
    int64_t g = 0;
    for (int64_t s = s_begin; s < s_end; ++s) {
        const int32_t *seg = segs + 6 * s;
        int64_t N = oracle_steps(seg);
        for (int64_t k = 0; k <= N; ++k) {
            if (g < cap)
                oracle_voxel(seg, k, xyz + 3 * g);
            ++g;
        }
    }
    return g;
}

/* Number of 32-byte sectors (8 words) of the volume holding at least one set
 * bit: with a zeroed volume before the call, the sectors a generation touched. */
int64_t oracle_sectors_touched(const uint32_t *mask, int64_t n_words)
{
    int64_t touched = 0;
    for (int64_t base = 0; base < n_words; base += 8) {
        int any = 0;
        for (int64_t j = base; j < base + 8 && j < n_words; ++j)
            if (mask[j]) any = 1;
        touched += any;
    }
    return touched;
}

/* Set-bit count of the volume (number of distinct occupied voxels). */
int64_t oracle_popcount(const uint32_t *mask, int64_t n_words)
{
    int64_t c = 0;
    for (int64_t j = 0; j < n_words; ++j) {
        uint32_t x = mask[j];
        while (x) { x &= x - 1; ++c; }
    }
    return c;
}

/*
 * The Euclidean-N variant: Eq. (1)-(2) read literally. N = int(|E - S|), the
 * integer part of the Euclidean length, i.e. the largest integer whose square
 * does not exceed dx^2 + dy^2 + dz^2. The samples are again G_k = S + W k,
 * W = (E - S) / N, k = 0..N, each mapped to its nearest lattice point (ties
 * away from S); since N can exceed the largest |d_a|, two samples can fall in
 * one voxel, and the voxel set V of Fig. 3 holds it once. The samples move
 * monotonically along each axis, by at most one voxel per step, so a repeated
 * voxel is always the previous sample's: a voxel is added when it differs from
 * the previous sample's voxel. N = 0 (S == E) gives the single voxel S.
 */

/* Integer square root, digit by digit in base 4: the largest r with r*r <= x. */
int64_t oracle_isqrt(int64_t x)
{
    uint64_t v = (uint64_t)x, r = 0, bit = (uint64_t)1 << 62;
    while (bit > v) bit >>= 2;
    while (bit) {
        if (v >= r + bit) {
            v -= r + bit;
            r = (r >> 1) + bit;
        } else {
            r >>= 1;
        }
        bit >>= 2;
    }
    return (int64_t)r;
}

/* N of Eq. (1): int(|E - S|). */
int64_t oracle_euclid_steps(const int32_t *seg)
{
    int64_t sq = 0;
    for (int a = 0; a < 3; ++a) {
        int64_t d = (int64_t)seg[3 + a] - (int64_t)seg[a];
        sq += d * d;
    }
    return oracle_isqrt(sq);
}

/* The voxel of sample k with the Euclidean N. */
void oracle_euclid_voxel(const int32_t *seg, int64_t k, int64_t *out3)
{
    voxel_of_sample(seg, k, oracle_euclid_steps(seg), out3);
}

/* Walks the samples of one segment and calls back for every voxel added. */
typedef void (*oracle_emit_fn)(void *ctx, const int64_t *v);

static int64_t euclid_segment(const int32_t *seg, oracle_emit_fn emit, void *ctx)
{
    int64_t N = oracle_euclid_steps(seg);
    int64_t prev[3] = {0, 0, 0};
    int64_t added = 0;
    for (int64_t k = 0; k <= N; ++k) {
        int64_t v[3];
        voxel_of_sample(seg, k, N, v);
        if (k > 0 && v[0] == prev[0] && v[1] == prev[1] && v[2] == prev[2]) continue;
        if (emit) emit(ctx, v);
        prev[0] = v[0];
        prev[1] = v[1];
        prev[2] = v[2];
        ++added;
    }
    return added;
}

/* Voxels per segment (int64) and their total. */
int64_t oracle_euclid_count(const int32_t *segs, int64_t n, int64_t *counts)
{
    int64_t total = 0;
    for (int64_t s = 0; s < n; ++s) {
        int64_t c = euclid_segment(segs + 6 * s, 0, 0);
        if (counts) counts[s] = c;
        total += c;
    }
    return total;
}

struct list_ctx {
    void *out;
    int64_t cap, g;
    int wide;
};

static void emit_list(void *p, const int64_t *v)
{
    struct list_ctx *c = (struct list_ctx *)p;
    if (c->g < c->cap) {
        if (c->wide)
            ((uint64_t *)c->out)[c->g] = pack64(v);
        else
            ((uint32_t *)c->out)[c->g] = pack32(v);
    }
    ++c->g;
}

int64_t oracle_euclid_list32(const int32_t *segs, int64_t n, uint32_t *out, int64_t cap)
{
    struct list_ctx c = {out, cap, 0, 0};
    for (int64_t s = 0; s < n; ++s) euclid_segment(segs + 6 * s, emit_list, &c);
    return c.g;
}

int64_t oracle_euclid_list64(const int32_t *segs, int64_t n, uint64_t *out, int64_t cap)
{
    struct list_ctx c = {out, cap, 0, 1};
    for (int64_t s = 0; s < n; ++s) euclid_segment(segs + 6 * s, emit_list, &c);
    return c.g;
}

struct mask_ctx {
    uint32_t *mask;
    int64_t w, h, n_words;
    int outside;
};

static void emit_mask(void *p, const int64_t *v)
{
    struct mask_ctx *c = (struct mask_ctx *)p;
    uint64_t lin = (uint64_t)(v[0] + c->w * (v[1] + c->h * v[2]));
    if (lin / 32 < (uint64_t)c->n_words)
        set_bit(c->mask, lin);
    else
        c->outside = 1;
}

/* OR the variant's voxels into the volume; -1 if a voxel fell outside it. */
int64_t oracle_euclid_bitmask(const int32_t *segs, int64_t n, const int32_t *dims, uint32_t *mask,
                              int64_t n_words)
{
    struct mask_ctx c = {mask, dims[0], dims[1], n_words, 0};
    int64_t g = 0;
    for (int64_t s = 0; s < n; ++s) g += euclid_segment(segs + 6 * s, emit_mask, &c);
    return c.outside ? -1 : g;
}
