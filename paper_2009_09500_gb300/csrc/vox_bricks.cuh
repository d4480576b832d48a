// vox_bricks.cuh -- the occupancy volume by brick ownership (sm_103a).
//
// OR-ing each voxel into the volume with a global atomic costs one L2/DRAM
// read-modify-write of a 32-byte sector per voxel (the volume is far larger than
// L2 for big scenes), which makes the volume store DRAM-bound at a small fraction
// of the bandwidth. Instead the volume is cut into bricks of whole 32-bit words
// (B0 x B1 x B2 voxels, B0 a multiple of 32, at most 32768 words), every segment
// is cut into pieces that stay inside one brick, the pieces are counting-sorted
// by brick, and one CTA owns each brick: it ORs the brick's voxels into a
// shared-memory bitmap and merges the bitmap into the volume in one pass (a TMA
// tensor reduce-OR, or a store of the whole brick for a fresh volume). Each
// volume sector then crosses DRAM at most twice (read + write), whatever the
// number of voxels in it.
//
//   k_bin_count    pieces per brick (lanes walk segments' pieces, global atomics)
//   k_scan<false>  exclusive scan of the per-brick counts (decoupled look-back)
//   k_bin_scatter  pieces written into their brick's bucket
//   k_brick_volume one CTA per brick: voxels -> shared bitmap -> volume
//
// A piece is (segment, first step k, length). The steps at which a segment's
// coordinate on an axis enters the next brick follow from the same exact rounding
// as the voxels themselves (Eq. (3) with nearest-lattice rounding): the offset
// q(k) = floor((2 k A + N) / (2 N)) first reaches Q at k = ceil(N (2Q - 1) / (2A)).
#pragma once

#include <cuda.h>

#include <cstdint>
#include <type_traits>

#include "vox_device.cuh"

namespace vox {

constexpr int kBrickThreads = 1024;  // one CTA per SM (the bitmap takes 128 KB)
constexpr int kBrickWordsMax = 32768;  // 128 KB shared bitmap per brick
constexpr int32_t kNoStep = 0x7fffffff;
constexpr int32_t kStPieces = 7;  // VOX_ERR_WORKSPACE: a brick-major volume needs every piece binned

struct BrickGeom {
    int32_t B[3];       // brick extent in voxels per axis (powers of two, B[0] >= 32)
    int32_t logB[3];    // log2(B[a])
    int32_t nb[3];      // bricks per axis
    int32_t bxw;        // words per brick row, B[0] / 32
    int32_t log_bxw;    // log2(bxw)
    int32_t log_b1;     // log2(B[1])
    int32_t row_words;  // words per volume row, w / 32
    int32_t dim[3];     // volume extent
    int32_t words;      // words per brick, bxw * B[1] * B[2]
    int64_t n_bricks;
    // Pieces are bucketed by slot = (brick, length class, replica), brick-major,
    // classes longest first: after the scan a brick's pieces are contiguous and
    // already ordered by length, so that a warp taking 32 consecutive pieces gets
    // pieces of similar length. Each (brick, class) has `reps` counters (segment
    // s uses replica s % reps) so that atomics on one brick spread over several
    // addresses when there are few bricks with many pieces each.
    int32_t reps;       // 1 or 8 (segment s uses replica s & (reps - 1))
    int64_t n_slots;    // n_bricks * kPieceClasses * reps
};

constexpr int kPieceClasses = 22;  // half octaves of the piece length (<= 1024)
constexpr int64_t kMaxBricks = int64_t(1) << 26;

// Brick shape for a volume whose rows are whole 32-bit words (w % 32 == 0):
// B0 = the largest 32 * 2^k not above min(w, 256) voxels along x (whole words),
// then B1 x B2 rows (powers of two) so that a brick has at most kBrickWordsMax
// words: 256 x 64 x 64 (128 KB) for wide volumes. Two things set the shape:
// segments in random directions cross the fewer brick faces the more cube-like
// and large the brick is (fewer pieces), and the brick's store writes one
// request per brick row, so rows of 32 bytes (B0 = 256) store about three times
// faster than rows of 16 bytes (measured: 18 against 56 us per 128 MiB volume).
// replicas: 8 counter replicas per (brick, class) when there are few bricks
// (a single scene), else 1 (and always 1 inside a batch of scenes).
__host__ __device__ inline bool brick_geom(int32_t w, int32_t h, int32_t d, BrickGeom *G, bool replicas)
{
    if (w < 1 || h < 1 || d < 1 || w % 32 != 0) return false;
    int32_t b0 = 32;
    while (2 * b0 <= w && 2 * b0 <= 256) b0 *= 2;
    G->B[0] = b0;
    G->bxw = b0 / 32;
    G->log_bxw = 0;
    while ((1 << G->log_bxw) < G->bxw) ++G->log_bxw;
    const int32_t rows = kBrickWordsMax / G->bxw;
    int32_t p2 = 1;
    while ((2 * p2) * (2 * p2) <= rows) p2 *= 2;
    G->B[1] = (2 * p2 * p2 <= rows) ? 2 * p2 : p2;
    G->B[2] = p2;
    G->log_b1 = 0;
    while ((1 << G->log_b1) < G->B[1]) ++G->log_b1;
    G->dim[0] = w;
    G->dim[1] = h;
    G->dim[2] = d;
    G->row_words = w / 32;
    G->words = G->bxw * G->B[1] * G->B[2];
    for (int a = 0; a < 3; ++a) {
        G->logB[a] = 0;
        while ((1 << G->logB[a]) < G->B[a]) ++G->logB[a];
    }
    int64_t nb = 1;
    for (int a = 0; a < 3; ++a) {
        G->nb[a] = (G->dim[a] + G->B[a] - 1) / G->B[a];
        nb *= G->nb[a];
    }
    G->n_bricks = nb;
    G->reps = (replicas && nb <= 32768) ? 8 : 1;
    G->n_slots = nb * kPieceClasses * G->reps;
    return nb <= kMaxBricks && G->words <= kBrickWordsMax;
}

// A scene of a batch as the brick path sees it: its geometry (one replica), its
// first brick and first slot in the batch's numbering, and its volume.
struct SceneBricks {
    BrickGeom G;
    int64_t brick_base;
    int64_t slot_base;
    uint32_t *mask;
};

// Length class of a piece, longest first: 0 for the longest half octave.
__device__ __forceinline__ int32_t piece_class_desc(int32_t len)
{
    const uint32_t l = static_cast<uint32_t>(len);
    const int32_t oct = 31 - __clz(l);
    const int32_t cls = 2 * oct + (oct > 0 ? static_cast<int32_t>((l >> (oct - 1)) & 1u) : 0);
    return kPieceClasses - 1 - cls;
}

// Slots fit 31 bits: with 8 replicas there are at most 32768 bricks, else at
// most 2^26 bricks and one replica.
__device__ __forceinline__ uint32_t piece_slot(const BrickGeom &G, int32_t brick, int32_t len, int32_t rep)
{
    return (static_cast<uint32_t>(brick) * kPieceClasses + static_cast<uint32_t>(piece_class_desc(len))) *
               static_cast<uint32_t>(G.reps) +
           static_cast<uint32_t>(rep);
}

// Crossing steps of one axis. The segment's offset on the axis,
// q(k) = floor((2 k A + N) / (2 N)), first reaches Q at
// k = ceil(N (2Q - 1) / (2A)) (for 1 <= Q <= A <= N). Along the segment the
// axis enters a new brick at Q_1, Q_1 + B, Q_1 + 2B, ...: with
// T_j = N (2 Q_j - 1) + 2A - 1 = 2A k_j + rem_j, one division gives k_1 and
// rem_1, and each later crossing follows from T_{j+1} = T_j + 2NB without a
// division, 2NB = 2A qs + rs having been divided once.
struct AxisCrossings {
    int32_t left;  // crossings still ahead
    int32_t nk;    // step of the next crossing (kNoStep when none)
    int32_t rem;   // T_j mod 2A for the crossing at nk
    int32_t qs, rs;
    int32_t twoA;

    __device__ __forceinline__ void init(int32_t S, int32_t E, int32_t A, int32_t N, int32_t logB)
    {
        const int32_t b0 = S >> logB, be = E >> logB;  // coordinates are inside the volume (>= 0)
        left = abs(be - b0);
        nk = kNoStep;
        if (left == 0) return;
        const int32_t B = 1 << logB;
        const int32_t Q = be > b0 ? (b0 + 1) * B - S : S - b0 * B + 1;
        twoA = 2 * A;
        if (N <= 46340) {  // T < 2 N^2 + 2N < 2^32
            const uint32_t T = static_cast<uint32_t>(N) * static_cast<uint32_t>(2 * Q - 1) + static_cast<uint32_t>(twoA - 1);
            const uint32_t k = T / static_cast<uint32_t>(twoA);
            nk = static_cast<int32_t>(k);
            rem = static_cast<int32_t>(T - k * static_cast<uint32_t>(twoA));
        } else {
            const uint64_t T = static_cast<uint64_t>(N) * static_cast<uint64_t>(2 * Q - 1) + static_cast<uint64_t>(twoA - 1);
            const uint64_t k = T / static_cast<uint64_t>(twoA);
            nk = static_cast<int32_t>(k);
            rem = static_cast<int32_t>(T - k * static_cast<uint64_t>(twoA));
        }
        if (left > 1) {  // 2NB < 2^31 (N < 2^21, B <= 256)
            const uint32_t step = 2u * static_cast<uint32_t>(N) * static_cast<uint32_t>(B);
            const uint32_t q = step / static_cast<uint32_t>(twoA);
            qs = static_cast<int32_t>(q);
            rs = static_cast<int32_t>(step - q * static_cast<uint32_t>(twoA));
        }
    }

    __device__ __forceinline__ void advance()
    {
        if (--left == 0) {
            nk = kNoStep;
            return;
        }
        nk += qs;
        rem += rs;
        if (rem >= twoA) {
            rem -= twoA;
            ++nk;
        }
    }
};

// The maximal runs of consecutive steps of one segment that stay in one brick,
// in increasing k: init() at the segment's start, then next() gives one run per
// call. Endpoints must be inside the volume. Brick indices fit 32 bits (at most
// 2^26 bricks). kEuclid: the steps are the samples of the Euclidean-N variant,
// N = int(|E - S|) (the crossing formula holds for any N >= max |d_a|).
template <bool kEuclid = false>
struct PieceWalker {
    AxisCrossings ax[3];
    int32_t bstep[3];
    int32_t brick, k, N;

    __device__ __forceinline__ void init(const int32_t *rec, const BrickGeom &G)
    {
        int32_t A[3];
        N = 0;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            A[a] = abs(rec[3 + a] - rec[a]);
            N = max(N, A[a]);
        }
        if constexpr (kEuclid) N = euclid_steps(rec);
        brick = (rec[0] >> G.logB[0]) + G.nb[0] * ((rec[1] >> G.logB[1]) + G.nb[1] * (rec[2] >> G.logB[2]));
        const int32_t stride[3] = {1, G.nb[0], G.nb[0] * G.nb[1]};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            ax[a].init(rec[a], rec[3 + a], A[a], N, G.logB[a]);
            bstep[a] = rec[3 + a] >= rec[a] ? stride[a] : -stride[a];
        }
        k = 0;
    }

    // The current run (brick b, first step k_lo, len steps); advances to the
    // next one and returns false if this run was the segment's last.
    __device__ __forceinline__ bool next(int32_t &b, int32_t &k_lo, int32_t &len)
    {
        const int32_t kn = min(min(ax[0].nk, ax[1].nk), min(ax[2].nk, N + 1));
        b = brick;
        k_lo = k;
        len = kn - k;
        if (kn > N) return false;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (ax[a].nk == kn) {
                brick += bstep[a];
                ax[a].advance();
            }
        }
        k = kn;
        return true;
    }
};

// Calls f(brick, k_lo, len) for every maximal run of consecutive steps of the
// segment that stays in one brick, in increasing k (PieceWalker in a loop).
template <bool kEuclid = false, typename F>
__device__ __forceinline__ void for_each_piece(const int32_t *rec, const BrickGeom &G, F &&f)
{
    PieceWalker<kEuclid> pw;
    pw.init(rec, G);
    bool more = true;
    while (more) {
        int32_t b, k_lo, len;
        more = pw.next(b, k_lo, len);
        f(b, k_lo, len);
    }
}

// Pieces are at most kPieceMaxLen steps long: a longer run in one brick is cut
// into parts of kPieceMaxLen (the last one shorter), so that no lane of the
// brick kernel walks a long piece while the rest of its CTA waits.
constexpr int32_t kPieceMaxLen = 64;

// piece = segment (32 bits) | first step (22 bits) | length - 1 (10 bits)
__device__ __forceinline__ uint64_t pack_piece(int64_t seg, int32_t k_lo, int32_t len)
{
    return static_cast<uint64_t>(static_cast<uint32_t>(seg)) | (static_cast<uint64_t>(k_lo) << 32) |
           (static_cast<uint64_t>(len - 1) << 54);
}

__device__ __forceinline__ bool endpoints_inside(const int32_t *r, const BrickGeom &G)
{
    return (unsigned)r[0] < (unsigned)G.dim[0] && (unsigned)r[3] < (unsigned)G.dim[0] &&
           (unsigned)r[1] < (unsigned)G.dim[1] && (unsigned)r[4] < (unsigned)G.dim[1] &&
           (unsigned)r[2] < (unsigned)G.dim[2] && (unsigned)r[5] < (unsigned)G.dim[2];
}

struct BinParams {
    const int32_t *segs;
    int64_t n;
    BrickGeom G;
    int32_t *brick_count;     // [n_slots], zeroed before k_bin_count
    int64_t *cursor;          // [n_slots], exclusive offsets (k_bin_scatter bumps them)
    const int64_t *brick_off; // [n_slots + 1]; brick_off[n_slots] = number of pieces
    uint64_t *pieces;         // [capacity]
    int64_t capacity;
    const int32_t *status;
    const SceneBricks *sb;    // batched: each scene's geometry and numbering (else null)
    const int32_t *scene_of;  // batched: scene of every segment
    int32_t n_scenes;
};

// The geometry a segment's pieces follow and the first slot of its volume, or
// null for a segment outside every scene (only after a table error, which the
// status word holds; the batched kernels check it first).
template <bool kBatched>
__device__ __forceinline__ const BrickGeom *segment_geom(const BinParams &p, int64_t s, int64_t &slot_base)
{
    if constexpr (kBatched) {
        const int32_t k = __ldg(p.scene_of + s);
        if (static_cast<uint32_t>(k) >= static_cast<uint32_t>(p.n_scenes)) return nullptr;
        slot_base = p.sb[k].slot_base;
        return &p.sb[k].G;
    } else {
        slot_base = 0;
        return &p.G;
    }
}

__device__ __forceinline__ void load_record(const int32_t *segs, int64_t s, int32_t *r)
{
    const int2 *p = reinterpret_cast<const int2 *>(segs + 6 * s);
    const int2 a = __ldg(p), b = __ldg(p + 1), c = __ldg(p + 2);
    r[0] = a.x; r[1] = a.y; r[2] = b.x; r[3] = b.y; r[4] = c.x; r[5] = c.y;
}

// Binning work loop, shared by the counting and the scattering pass (CTAs of
// kBinThreads threads, persistent grid). Each warp takes batches of kBinBatch
// consecutive segments, orders each batch by length octave, longest first (a
// counting sort in the warp's shared memory), and walks the segments in that
// order, lane l taking the l-th of every 32: the lanes of a warp then walk
// segments of similar length, so that a warp does not wait for one long
// segment while its other lanes idle (lengths may span three orders of
// magnitude). emit(slot, seg, k_lo, len) is called for every piece (runs in one
// brick cut to at most kPieceMaxLen steps) with its slot in the batch's slot
// numbering. A segment with an endpoint outside its volume has no pieces (the
// count kernel reports it).
constexpr int kBinThreads = 256;
constexpr int kBinWarps = kBinThreads / 32;
constexpr int kBinPer = 4;                 // segments per lane and batch
constexpr int kBinBatch = 32 * kBinPer;    // segments per warp batch
constexpr int kBinOctaves = 22;            // octaves of N + 1 <= 2^21

template <bool kEuclid, bool kBatched, typename Emit>
__device__ __forceinline__ void bin_loop(const BinParams &p, Emit &&emit)
{
    __shared__ int32_t s_recs[kBinWarps][kBinBatch * 6];
    __shared__ uint8_t s_order[kBinWarps][kBinBatch];
    __shared__ int32_t s_hist[kBinWarps][32];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t gw = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
    int32_t *const recs = s_recs[wib];
    for (int64_t b0 = gw * kBinBatch; b0 < p.n; b0 += nw * kBinBatch) {
        s_hist[wib][lane] = 0;
        __syncwarp();
        // the batch's records, and each segment's rank within its octave (longest first)
        int32_t oct[kBinPer], rank[kBinPer];
#pragma unroll
        for (int i = 0; i < kBinPer; ++i) {
            const int j = i * 32 + lane;
            const int64_t s = b0 + j;
            oct[i] = -1;
            if (s < p.n) {
                int32_t r[6];
                load_record(p.segs, s, r);
#pragma unroll
                for (int c = 0; c < 6; ++c) recs[6 * j + c] = r[c];
                // the octave of N + 1 from unsigned differences: a segment with an
                // endpoint outside the volume (skipped below) still gets a valid one
                const uint32_t dx = static_cast<uint32_t>(abs(r[3] - r[0]));
                const uint32_t dy = static_cast<uint32_t>(abs(r[4] - r[1]));
                const uint32_t dz = static_cast<uint32_t>(abs(r[5] - r[2]));
                const uint32_t octave = 31 - __clz(max(dx, max(dy, dz)) | 1u);
                oct[i] = kBinOctaves - 1 - static_cast<int32_t>(min(octave, static_cast<uint32_t>(kBinOctaves - 1)));
                rank[i] = atomicAdd(&s_hist[wib][oct[i]], 1);
            }
        }
        __syncwarp();
        // octave starts: exclusive scan of the octave counts (one per lane)
        const int32_t h = s_hist[wib][lane];
        int32_t inc = h;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        const int32_t total = __shfl_sync(0xffffffffu, inc, 31);
#pragma unroll
        for (int i = 0; i < kBinPer; ++i) {
            const int32_t start = __shfl_sync(0xffffffffu, inc - h, max(oct[i], 0));
            if (oct[i] >= 0) s_order[wib][start + rank[i]] = static_cast<uint8_t>(i * 32 + lane);
        }
        __syncwarp();
#pragma unroll 1
        for (int i = 0; i < kBinPer; ++i) {
            const int q = i * 32 + lane;
            if (q >= total) continue;
            const int j = s_order[wib][q];
            const int64_t s = b0 + j;
            int64_t slot_base;
            const BrickGeom *Gp = segment_geom<kBatched>(p, s, slot_base);
            if (Gp == nullptr) continue;
            const int32_t *r = recs + 6 * j;
            if (!endpoints_inside(r, *Gp)) continue;
            const int32_t rep = static_cast<int32_t>(s) & (Gp->reps - 1);
            PieceWalker<kEuclid> pw;
            pw.init(r, *Gp);
            bool more = true;
            while (more) {
                int32_t b, k_lo, len;
                more = pw.next(b, k_lo, len);
                while (len > 0) {
                    const int32_t part = min(len, kPieceMaxLen);
                    emit(slot_base + piece_slot(*Gp, b, part, rep), s, k_lo, part);
                    k_lo += part;
                    len -= part;
                }
            }
        }
        __syncwarp();  // the warp's shared arrays are free for the next batch
    }
}

// Pieces per slot (persistent grid).
template <bool kEuclid, bool kBatched = false>
__global__ void __launch_bounds__(kBinThreads) k_bin_count(BinParams p)
{
    // single volume: no status check (this pass may run beside the count + scan
    // that resets the status word); it reads only the segments and the host's
    // geometry, writes only the slot counts, and skips segments with endpoints
    // outside the volume (reported by the count kernel)
    // a batch reads the scene map and numbering, valid only without an error
    // (decided by the whole warp: the walk's shuffles and votes need every lane)
    if (kBatched && __any_sync(0xffffffffu, ld_volatile_i32(p.status) != 0)) return;
    bin_loop<kEuclid, kBatched>(p, [&](int64_t slot, int64_t, int32_t, int32_t) {
        atomicAdd(p.brick_count + slot, 1);
    });
}

// Pieces written into their slots (persistent grid). p.G.n_slots: the number of
// slots (all scenes' when batched). Slot reservations of up to four pieces are
// in flight together before their stores, so the returning atomics' latency
// overlaps.
template <bool kEuclid, bool kBatched = false>
__global__ void __launch_bounds__(kBinThreads) k_bin_scatter(BinParams p)
{
    // an earlier error: write nothing (decided by the whole warp, whose walk takes
    // shuffles and votes; the status word may be set by a kernel on another stream)
    if (__any_sync(0xffffffffu, ld_volatile_i32(p.status) != 0)) return;
    if (__ldg(p.brick_off + p.G.n_slots) > p.capacity) return;  // the volume falls back to atomics
    constexpr int kBatch = 4;
    int64_t bb[kBatch];
    uint64_t val[kBatch];
    int nb = 0;
    auto flush = [&]() {
        unsigned long long pos[kBatch];
#pragma unroll
        for (int e = 0; e < kBatch; ++e)
            if (e < nb) pos[e] = atomicAdd(reinterpret_cast<unsigned long long *>(p.cursor + bb[e]), 1ull);
#pragma unroll
        for (int e = 0; e < kBatch; ++e)
            if (e < nb) p.pieces[pos[e]] = val[e];
        nb = 0;
    };
    bin_loop<kEuclid, kBatched>(p, [&](int64_t slot, int64_t seg, int32_t k, int32_t len) {
#pragma unroll
        for (int e = 0; e < kBatch; ++e)
            if (e == nb) {
                bb[e] = slot;
                val[e] = pack_piece(seg, k, len);
            }
        if (++nb == kBatch) flush();
    });
    if (nb) flush();
}

struct BrickParams {
    const int32_t *segs;
    BrickGeom G;
    const int64_t *brick_off;  // [n_slots + 1]
    const uint64_t *pieces;
    int64_t capacity;
    uint32_t *mask;
    int32_t *status;
    uint32_t *ticket;  // zeroed before launch
    int32_t use_tma;   // merge by one TMA tensor reduce-OR (or store) per brick (tensor map valid)
    int32_t fresh;     // write every brick (zeros included) instead of OR-ing into the volume
    int32_t bricked;   // brick-major volume: brick b is words `words` at mask + b * words (one bulk copy)
    const SceneBricks *sb;       // batched: each scene's geometry, numbering and volume (G.n_slots,
    int32_t n_scenes;            // G.n_bricks: the batch's totals; merged by plain stores)
    const int32_t *brick_scene;  // batched: the scene of every brick
};

// TMA tensor reduction of a whole brick tile from shared memory into the volume:
// every word of the box (bxw x B1 x B2 words at word coordinates x, y, z) is
// OR-ed into global memory by the L2, asynchronously; parts of the box outside
// the volume are skipped by the hardware.
__device__ __forceinline__ void tma_reduce_or_3d(const CUtensorMap *tmap, const void *smem, int32_t x, int32_t y,
                                                 int32_t z)
{
    asm volatile(
        "cp.reduce.async.bulk.tensor.3d.global.shared::cta.or.tile.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(
            reinterpret_cast<uint64_t>(tmap)),
        "r"(x), "r"(y), "r"(z), "r"(smem_addr(smem))
        : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}

// 1-D bulk copy of a whole brick bitmap to global memory (brick-major volume);
// both addresses 16-byte aligned, size a multiple of 16.
__device__ __forceinline__ void bulk_store_1d(void *gmem, const void *smem, uint32_t bytes)
{
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(reinterpret_cast<uint64_t>(gmem)),
                 "r"(smem_addr(smem)), "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}

// TMA tensor store of a whole brick tile (the volume's previous content there is
// replaced); parts of the box outside the volume are skipped by the hardware.
__device__ __forceinline__ void tma_store_3d(const CUtensorMap *tmap, const void *smem, int32_t x, int32_t y, int32_t z)
{
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(
                     reinterpret_cast<uint64_t>(tmap)),
                 "r"(x), "r"(y), "r"(z), "r"(smem_addr(smem))
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}

__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// Merge a brick's shared bitmap into the volume. Brick row (ly, lz) holds bxw
// words that are contiguous in the volume; a warp covers 32 consecutive words
// (or 32 consecutive 16-byte units, when rows and the volume allow them).
// OR mode reads and writes only touched words; fresh mode writes every word of
// the brick inside the volume (zeros included) and reads none. Eight
// independent loads per thread are issued before the stores, so DRAM latency is
// paid once per group, not once per word. The brick owns its words: plain
// loads and stores suffice.
__device__ __forceinline__ void merge_brick(const uint32_t *bits, const BrickGeom &G, int32_t X0, int32_t Y0,
                                            int32_t Z0, uint32_t *mask, bool fresh)
{
    const int t = threadIdx.x;
    if ((G.bxw & 3) == 0 && (G.row_words & 3) == 0 && (reinterpret_cast<uintptr_t>(mask) & 15u) == 0) {
        // 16-byte units (a brick row holds bxw / 4 of them): the brick's first word
        // in a row, X0 / 32, is a multiple of bxw and the volume's rows are whole
        // 16-byte units, so every unit is aligned and lies in or beyond the row
        // as a whole; four units per thread in flight
        constexpr int kGroup4 = 4;
        const uint4 *b4 = reinterpret_cast<const uint4 *>(bits);
        uint4 *m4 = reinterpret_cast<uint4 *>(mask);
        const int32_t units = G.words >> 2;
        const int32_t log_bxu = G.log_bxw - 2;
        const int32_t row_units = G.row_words >> 2;
        const int32_t x_unit = X0 / 128;
        for (int q0 = 0; q0 < units; q0 += kGroup4 * kBrickThreads) {
            uint4 v[kGroup4], old[kGroup4];
            int64_t gu[kGroup4];
            bool wr[kGroup4];
#pragma unroll
            for (int e = 0; e < kGroup4; ++e) {
                const int q = q0 + e * kBrickThreads + t;
                v[e] = make_uint4(0u, 0u, 0u, 0u);
                gu[e] = 0;
                wr[e] = false;
                if (q < units) {
                    const uint4 b = b4[q];
                    const int32_t row = q >> log_bxu, col = q & ((1 << log_bxu) - 1);
                    const int32_t y = Y0 + (row & (G.B[1] - 1)), z = Z0 + (row >> G.log_b1);
                    if ((fresh || (b.x | b.y | b.z | b.w) != 0u) && y < G.dim[1] && z < G.dim[2] &&
                        x_unit + col < row_units) {
                        v[e] = b;
                        wr[e] = true;
                        gu[e] = x_unit + col + static_cast<int64_t>(row_units) * (y + static_cast<int64_t>(G.dim[1]) * z);
                    }
                }
            }
#pragma unroll
            for (int e = 0; e < kGroup4; ++e) old[e] = (wr[e] && !fresh) ? m4[gu[e]] : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
            for (int e = 0; e < kGroup4; ++e)
                if (wr[e])
                    m4[gu[e]] = make_uint4(old[e].x | v[e].x, old[e].y | v[e].y, old[e].z | v[e].z, old[e].w | v[e].w);
        }
        return;
    }
    constexpr int kGroup = 8;
    for (int q0 = 0; q0 < G.words; q0 += kGroup * kBrickThreads) {
        uint32_t v[kGroup], old[kGroup];
        int64_t gw[kGroup];
        bool wr[kGroup];
#pragma unroll
        for (int e = 0; e < kGroup; ++e) {
            const int q = q0 + e * kBrickThreads + t;
            v[e] = 0;
            gw[e] = 0;
            wr[e] = false;
            if (q < G.words) {
                const uint32_t b = bits[q];
                const int32_t row = q >> G.log_bxw, col = q & (G.bxw - 1);
                const int32_t y = Y0 + (row & (G.B[1] - 1)), z = Z0 + (row >> G.log_b1);
                if ((fresh || b != 0) && y < G.dim[1] && z < G.dim[2] && X0 / 32 + col < G.row_words) {
                    v[e] = b;
                    wr[e] = true;
                    gw[e] = X0 / 32 + col + static_cast<int64_t>(G.row_words) * (y + static_cast<int64_t>(G.dim[1]) * z);
                }
            }
        }
#pragma unroll
        for (int e = 0; e < kGroup; ++e) old[e] = (wr[e] && !fresh) ? mask[gw[e]] : 0u;
#pragma unroll
        for (int e = 0; e < kGroup; ++e)
            if (wr[e]) mask[gw[e]] = old[e] | v[e];
    }
}

// A brick taken from the ticket counter: its index, its pieces [lo, hi) and its
// origin (and, in a batch, its scene's geometry and volume).
struct BrickInfo {
    int64_t brick;
    int64_t lo, hi;
    int32_t origin[3];
    BrickGeom geom;      // batched: the brick's scene geometry
    uint32_t *bmask;     // batched: the scene's volume
};

struct BrickSmem {
    alignas(128) uint32_t bits[kBrickWordsMax];  // also the TMA source tile (128-byte aligned)
    BrickInfo info[3];   // a ring: the brick in hand, the next one, and the one after (taken ahead)
    int32_t next_group;  // next group of 32 pieces of the brick to hand to a warp
};

// Take the next brick ticket and describe the brick (one thread).
template <bool kBatched>
__device__ __forceinline__ void take_brick(const BrickParams &p, bool overflow, BrickInfo &I)
{
    const int64_t b = atomicAdd(p.ticket, 1u);
    I.brick = b;
    if (b >= p.G.n_bricks) return;
    int64_t lb = b;  // the brick's index in its volume
    const BrickGeom *Gt = &p.G;
    int64_t first_slot;
    if constexpr (kBatched) {  // the brick's scene and its geometry
        const int32_t k = __ldg(p.brick_scene + b);
        I.geom = p.sb[k].G;
        I.bmask = p.sb[k].mask;
        lb = b - p.sb[k].brick_base;
        first_slot = p.sb[k].slot_base + lb * kPieceClasses;
        Gt = &I.geom;
    } else {
        first_slot = b * kPieceClasses * p.G.reps;
    }
    const int64_t rest = lb / Gt->nb[0];
    I.origin[0] = static_cast<int32_t>(lb - rest * Gt->nb[0]) * Gt->B[0];
    I.origin[1] = static_cast<int32_t>(rest % Gt->nb[1]) * Gt->B[1];
    I.origin[2] = static_cast<int32_t>(rest / Gt->nb[1]) * Gt->B[2];
    const int64_t slots_per_brick = static_cast<int64_t>(kPieceClasses) * Gt->reps;
    I.lo = overflow ? 0 : __ldg(p.brick_off + first_slot);
    I.hi = overflow ? 0 : __ldg(p.brick_off + first_slot + slots_per_brick);
}

// One CTA per brick (dynamic tickets, taken two bricks ahead by the last warp
// while the others walk, so that no barrier waits for a ticket). The brick's
// pieces arrive ordered by length class, longest first (the bucket order of the
// binning). Group w of 32 consecutive pieces goes to warp w, further groups to
// the warps that ask a shared counter first: the lanes of a warp walk pieces of
// similar length (at most kPieceMaxLen steps), longest groups first. A warp's
// first group of the next brick is loaded while it walks the current brick
// (its pieces during the walk, their segment records after it), so that, with
// about as many groups per brick as warps, most groups start without waiting
// for global memory. Each lane enters its piece's segment at the piece's first
// step (one division per minor axis) and steps through the piece with the
// carry recurrence, OR-ing bits into the brick's shared bitmap; the bitmap is
// then merged into the volume.
template <bool kEuclid, bool kBatched = false>
__global__ void __launch_bounds__(kBrickThreads) k_brick_volume(BrickParams p, const __grid_constant__ CUtensorMap tmap)
{
    extern __shared__ __align__(128) unsigned char brick_smem_raw[];
    BrickSmem &sm = *reinterpret_cast<BrickSmem *>(brick_smem_raw);
    const int t = threadIdx.x;
    const int lane = t & 31;
    const int warp = t >> 5;
    // an earlier error: write nothing, decided by the whole CTA (the status word may
    // be set meanwhile by a kernel on another stream, and the CTA meets at barriers)
    if (__syncthreads_or(ld_volatile_i32(p.status) != 0)) return;
    // pieces that did not fit: the gated atomics pass ORs the voxels in (after a
    // fresh volume has been cleared here, brick by brick)
    const bool overflow = __ldg(p.brick_off + p.G.n_slots) > p.capacity;
    if (overflow && p.bricked) {  // no atomics fallback for this layout
        if (blockIdx.x == 0 && t == 0) set_status(p.status, kStPieces);
        return;
    }
    if (overflow && !p.fresh) return;
    const bool async_store = p.use_tma || p.bricked;  // the bitmap leaves by the bulk-copy unit
    const int64_t total_bricks = p.G.n_bricks;
    using St = typename std::conditional<kEuclid, EuclidStepper<uint32_t, uint32_t>, Stepper<uint32_t, uint32_t>>::type;
    // this warp's first group of the brick in hand, when loaded ahead
    bool have_pref = false;
    uint64_t pc_pref = 0;
    int32_t rec_pref[6] = {0, 0, 0, 0, 0, 0};
    // ring positions of the brick in hand, the next one and the one after
    int cur = 0, nxt = 1, aft = 2;
    const bool taker = t == kBrickThreads - 32;  // lane 0 of the last warp takes the tickets
    if (taker) {
        take_brick<kBatched>(p, overflow, sm.info[0]);
        take_brick<kBatched>(p, overflow, sm.info[1]);
    }
    while (true) {
        __syncthreads();
        const BrickInfo &I = sm.info[cur];
        const BrickInfo &NI = sm.info[nxt];
        const int64_t b = I.brick;
        if (b >= total_bricks) break;
        const BrickGeom &G = kBatched ? I.geom : p.G;
        const int32_t X0 = I.origin[0], Y0 = I.origin[1], Z0 = I.origin[2];
        const uint32_t bw = static_cast<uint32_t>(G.B[0]);
        const uint32_t bwh = static_cast<uint32_t>(G.B[0]) * static_cast<uint32_t>(G.B[1]);
        const int64_t lo = I.lo, cnt = I.hi - I.lo;
        const bool next_ok = NI.brick < total_bricks;
        const int64_t lo_n = NI.lo, cnt_n = next_ok ? NI.hi - NI.lo : 0;
        if (cnt == 0 && !p.fresh) {
            have_pref = false;
            if (taker) take_brick<kBatched>(p, overflow, sm.info[aft]);  // read by no one now
            const int c = cur;
            cur = nxt;
            nxt = aft;
            aft = c;
            continue;
        }
        // the warp's first group (group `warp`): loaded ahead, or its pieces now
        // (their records after the clear, so that the latency overlaps it)
        int32_t grp = warp;
        int64_t j = static_cast<int64_t>(grp) * 32 + lane;
        uint64_t pc = have_pref ? pc_pref : (j < cnt ? __ldg(p.pieces + lo + j) : 0ull);
        int32_t rec[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) rec[c] = rec_pref[c];
        // the next brick's first group for this warp: its pieces now, consumed after the walk
        const int64_t jn = static_cast<int64_t>(warp) * 32 + lane;
        const uint64_t pc_n = jn < cnt_n ? __ldg(p.pieces + lo_n + jn) : 0ull;
        if (t == 0) {
            sm.next_group = kBrickThreads / 32;  // groups beyond the first round, on demand
            if (async_store) bulk_wait_read_all();  // the previous brick's copy must have read the tile
        }
        __syncthreads();
        {  // words is a multiple of 4 (bxw * B1 * B2 with B1 * B2 >= 8)
            uint4 *z = reinterpret_cast<uint4 *>(sm.bits);
            for (int q = t; q < G.words / 4; q += kBrickThreads) z[q] = make_uint4(0u, 0u, 0u, 0u);
        }
        if (!have_pref && j < cnt) load_record(p.segs, static_cast<int64_t>(pc & 0xffffffffull), rec);
        __syncthreads();
        // the brick after the next one: its ticket is taken while the CTA walks this
        // one (its ring slot held the brick before this one, read by no one now)
        if (taker) take_brick<kBatched>(p, overflow, sm.info[aft]);
        // brick-local bit index of (x, y, z): (x - X0) + B0 (y - Y0) + B0 B1 (z - Z0),
        // kept modulo 2^32 while stepping (only the local value is ever used)
        const uint32_t origin = static_cast<uint32_t>(X0) + static_cast<uint32_t>(Y0) * bw +
                                static_cast<uint32_t>(Z0) * bwh;
#pragma unroll 1
        while (static_cast<int64_t>(grp) * 32 < cnt) {
            if (j < cnt) {
                const int32_t len = static_cast<int32_t>(pc >> 54) + 1;
                St st;
                st.enter(rec, static_cast<int32_t>((pc >> 32) & 0x3fffffull), bw, bwh);
                st.L -= origin;
                // one shared-memory atomic per voxel: cheaper than branching to
                // merge runs of the same word (measured on both workload shapes);
                // repeated samples of the Euclidean variant set the same bit again
                int32_t e = 0;
                for (; e + 8 <= len; e += 8) {
#pragma unroll
                    for (int v = 0; v < 8; ++v) {
                        atomicOr(sm.bits + (st.L >> 5), 1u << (st.L & 31u));
                        st.template step<false, true>();
                    }
                }
                for (; e < len; ++e) {
                    atomicOr(sm.bits + (st.L >> 5), 1u << (st.L & 31u));
                    st.template step<false, true>();
                }
            }
            __syncwarp();
            if (lane == 0) grp = atomicAdd(&sm.next_group, 1);
            grp = __shfl_sync(0xffffffffu, grp, 0);
            j = static_cast<int64_t>(grp) * 32 + lane;
            if (j < cnt) {
                pc = __ldg(p.pieces + lo + j);
                load_record(p.segs, static_cast<int64_t>(pc & 0xffffffffull), rec);
            }
        }
        // the next brick's first group: its pieces have arrived, now their records
        have_pref = next_ok;
        pc_pref = pc_n;
        if (jn < cnt_n) load_record(p.segs, static_cast<int64_t>(pc_n & 0xffffffffull), rec_pref);
        __syncthreads();
        if (p.bricked) {
            if (t == 0) {
                fence_proxy_async_smem();
                bulk_store_1d(p.mask + b * G.words, sm.bits, static_cast<uint32_t>(G.words) * 4u);
            }
        } else if (p.use_tma) {
            if (t == 0) {
                fence_proxy_async_smem();  // the bitmap's generic writes, visible to the TMA unit
                if (p.fresh) tma_store_3d(&tmap, sm.bits, X0 / 32, Y0, Z0);
                else tma_reduce_or_3d(&tmap, sm.bits, X0 / 32, Y0, Z0);
            }
        } else {
            uint32_t *const mask = kBatched ? I.bmask : p.mask;
            if (mask != nullptr) merge_brick(sm.bits, G, X0, Y0, Z0, mask, p.fresh != 0);
            __syncthreads();
        }
        const int c = cur;
        cur = nxt;
        nxt = aft;
        aft = c;
    }
    if (async_store && t == 0) bulk_wait_all();  // copies complete before the CTA's memory goes
}

// Brick-major volume -> row-major volume: one warp per volume row (y, z), lanes
// over the row's words; each word comes from its brick's row (bxw contiguous
// words), so reads stay sector-sized and writes are coalesced.
__global__ void __launch_bounds__(256) k_unbrick(const uint32_t *bricked, BrickGeom G, uint32_t *mask)
{
    const int lane = threadIdx.x & 31;
    const int64_t rows = static_cast<int64_t>(G.dim[1]) * G.dim[2];
    const int64_t warps = static_cast<int64_t>(gridDim.x) * (blockDim.x / 32);
    for (int64_t r = static_cast<int64_t>(blockIdx.x) * (blockDim.x / 32) + (threadIdx.x >> 5); r < rows; r += warps) {
        const int32_t y = static_cast<int32_t>(r % G.dim[1]);
        const int32_t z = static_cast<int32_t>(r / G.dim[1]);
        const int64_t bbase = static_cast<int64_t>(G.nb[0]) * ((y >> G.logB[1]) + static_cast<int64_t>(G.nb[1]) * (z >> G.logB[2]));
        const int64_t inrow = static_cast<int64_t>(G.bxw) * ((y & (G.B[1] - 1)) + static_cast<int64_t>(G.B[1]) * (z & (G.B[2] - 1)));
        uint32_t *out = mask + r * G.row_words;
        for (int32_t xw = lane; xw < G.row_words; xw += 32) {
            const int64_t brick = bbase + (xw >> G.log_bxw);
            out[xw] = __ldg(bricked + brick * G.words + inrow + (xw & (G.bxw - 1)));
        }
    }
}

// Brick-major -> row-major through the bulk-copy unit: each CTA (one warp, of
// which thread 0 works) takes half bricks in a grid-stride order; a half brick
// is contiguous in the brick-major layout (z is the slowest axis inside a
// brick), so it arrives in shared memory with one 1-D bulk copy and leaves with
// one TMA tensor store of a half-brick box. Several CTAs per SM keep loads and
// stores in flight together. Every wait is bounded; on expiry the status (if
// any) records a timeout and the CTA stops after one more bounded wait for its
// copy in flight.
constexpr int kUnbrickSplit = 2;

__global__ void __launch_bounds__(32) k_unbrick_tma(const uint32_t *bricked, BrickGeom G,
                                                    const __grid_constant__ CUtensorMap tmap, int32_t *status,
                                                    uint64_t wait_ns)
{
    extern __shared__ __align__(128) unsigned char unbrick_smem_raw[];
    uint32_t *buf = reinterpret_cast<uint32_t *>(unbrick_smem_raw);
    __shared__ uint64_t bar;
    if (threadIdx.x != 0) return;
    const int32_t part_words = G.words / kUnbrickSplit;
    const int32_t part_rows = G.B[2] / kUnbrickSplit;
    mbar_init(&bar, 1);
    fence_barrier_init();
    uint32_t phase = 0;
    const int64_t n_parts = G.n_bricks * kUnbrickSplit;
    for (int64_t q = blockIdx.x; q < n_parts; q += gridDim.x) {
        const int64_t b = q / kUnbrickSplit;
        const int32_t h = static_cast<int32_t>(q - b * kUnbrickSplit);
        const int64_t rest = b / G.nb[0];
        const int32_t X0 = static_cast<int32_t>(b - rest * G.nb[0]) * G.B[0];
        const int32_t Y0 = static_cast<int32_t>(rest % G.nb[1]) * G.B[1];
        const int32_t Z0 = static_cast<int32_t>(rest / G.nb[1]) * G.B[2];
        bulk_wait_read_all();  // the previous store has read the buffer
        mbar_arrive_expect_tx(&bar, static_cast<uint32_t>(part_words) * 4u);
        bulk_copy_g2s(buf, bricked + b * G.words + static_cast<int64_t>(h) * part_words,
                      static_cast<uint32_t>(part_words) * 4u, &bar);
        if (!mbar_wait_bounded(&bar, phase, wait_ns)) {
            if (status != nullptr) set_status(status, 5);  // VOX_ERR_TIMEOUT
            mbar_wait_bounded(&bar, phase, wait_ns);
            break;
        }
        phase ^= 1u;
        tma_store_3d(&tmap, buf, X0 / 32, Y0, Z0 + h * part_rows);
    }
    bulk_wait_all();
}

}  // namespace vox
