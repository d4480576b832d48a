// vox_kernels.cuh -- the three kernels of the voxelization hot path (sm_103a):
//
//   k_scan        per-segment voxel count N + 1 (+ endpoint validation) fused
//                 with a single-pass decoupled look-back exclusive scan
//                 (Merrill & Garland, 2016) into int64 offsets;
//   k_generate    voxel-parallel generation: each CTA owns a contiguous range of
//                 global voxel ids, stages windows of segment records and offsets
//                 into shared memory with 1-D TMA bulk copies, maps each thread's
//                 run of R voxels back to (segment, k) by a search in the staged
//                 offsets, and steps through the run with the exact integer
//                 recurrence, writing packed coordinates and/or OR-ing bits.
//
// The paper's multi-segment kernel pads every segment to N_max threads (Section 5,
// Fig. 4b) and names the resulting divergence as its main loss for segments of
// arbitrary length; the scan plus the voxel-range split here give every CTA the
// same number of voxels whatever the length mix.
#pragma once

#include <cstddef>
#include <cstdint>
#include <type_traits>

#include "vox_device.cuh"

namespace vox {

__device__ __forceinline__ int64_t min64(int64_t a, int64_t b) { return a < b ? a : b; }
__device__ __forceinline__ int64_t max64(int64_t a, int64_t b) { return a > b ? a : b; }

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;  // segments per scan tile

constexpr uint64_t kDescAgg = 1ull << 62;  // tile aggregate published
constexpr uint64_t kDescInc = 2ull << 62;  // tile inclusive prefix published
constexpr uint64_t kDescValue = (1ull << 62) - 1;

constexpr int kGenThreads = 256;
constexpr int kWindowSegs = 256;   // segment records staged per window (even)

// Status codes written by the kernels (same values as the public vox_status).
constexpr int32_t kStOutOfBounds = 2;
constexpr int32_t kStCapacity = 4;
constexpr int32_t kStTimeout = 5;

// Device view of vox_scene (same layout): one scene of a batch.
struct SceneDesc {
    int64_t seg_begin;  // first segment of the scene in the batch's segment array
    int64_t n;          // segments of the scene
    int32_t w, h, d;    // volume extent
    int32_t reserved;
    uint32_t *mask;     // the scene's volume, or null
};
static_assert(sizeof(SceneDesc) == 40, "scene layout");

struct ScanParams {
    const int32_t *segs;       // [n][6] (segment counts) or null
    const int32_t *counts_in;  // [n] (plain counts) or null
    int64_t *offsets_copy;     // [n] second copy of the exclusive offsets, or null
    int64_t n;
    int32_t w, h, d;
    int32_t *counts;       // [n] or null
    int64_t *offsets;      // [n + 4] workspace copy (entry n = total, then padding)
    int64_t *offsets_out;  // [n + 1] caller copy or null
    uint64_t *desc;        // [n_tiles] tile descriptors, zeroed before launch
    uint32_t *ticket;      // dynamic tile counter, zeroed before launch
    int32_t *status;
    int64_t n_tiles;
    int64_t stall_tile;  // test hook: this tile publishes nothing (-1: off)
    uint64_t wait_ns;    // bound of every wait
    const SceneDesc *scenes;  // batched: per-segment dims come from the segment's scene
    const int32_t *scene_of;  // batched: scene index of every segment (else null)
    int32_t n_scenes;
};

// ---------------------------------------------------------------- count + scan
// kFromSegments: the counts are N + 1 of each segment (with endpoint checks);
// otherwise they are read from p.counts_in (e.g. pieces per brick).
// kEuclid: the count of a segment is its sample count with the Euclidean N of
// Eq. (1), int(|E - S|) + 1.
template <bool kFromSegments, bool kEuclid = false>
__global__ void __launch_bounds__(kScanThreads) k_scan(ScanParams p)
{
    __shared__ __align__(16) int32_t s_cnt[kScanTile];
    __shared__ int64_t s_loc[kScanTile];
    __shared__ int64_t s_warp[kScanThreads / 32];
    __shared__ int64_t s_excl;
    __shared__ int64_t s_total;
    __shared__ uint32_t s_tile;

    const int t = threadIdx.x;
    const int lane = t & 31;
    const int warp = t >> 5;
    if (t == 0) s_tile = atomicAdd(p.ticket, 1u);
    __syncthreads();
    const int64_t tile = s_tile;
    if (tile >= p.n_tiles) return;  // only if the ticket was not reset: publish nothing
    const int64_t base = tile * kScanTile;

    // counts, read in a strided (coalesced) order
    bool bad = false;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        const int idx = j * kScanThreads + t;
        const int64_t s = base + idx;
        int32_t c = 0;
        if (!kFromSegments) {
            if (s < p.n) c = __ldg(p.counts_in + s);
        } else if (s < p.n) {
            const int2 *r = reinterpret_cast<const int2 *>(p.segs + 6 * s);
            const int2 a = __ldg(r), b = __ldg(r + 1), e = __ldg(r + 2);
            const int32_t x0 = a.x, y0 = a.y, z0 = b.x, x1 = b.y, y1 = e.x, z1 = e.y;
            int32_t W = p.w, H = p.h, D = p.d;
            if (p.scene_of != nullptr) {  // batched: the segment's own scene
                const int32_t k = __ldg(p.scene_of + s);
                W = H = D = 0;  // an unmapped segment fails the bounds check
                if ((unsigned)k < (unsigned)p.n_scenes) {
                    W = p.scenes[k].w;
                    H = p.scenes[k].h;
                    D = p.scenes[k].d;
                }
            }
            const bool ok = (unsigned)x0 < (unsigned)W && (unsigned)x1 < (unsigned)W &&
                            (unsigned)y0 < (unsigned)H && (unsigned)y1 < (unsigned)H &&
                            (unsigned)z0 < (unsigned)D && (unsigned)z1 < (unsigned)D;
            if (ok) {
                if constexpr (kEuclid) {
                    const int32_t rec[6] = {x0, y0, z0, x1, y1, z1};
                    c = euclid_steps(rec) + 1;
                } else {
                    c = max(abs(x1 - x0), max(abs(y1 - y0), abs(z1 - z0))) + 1;
                }
            } else {
                bad = true;
                c = 1;
            }
            if (p.counts) p.counts[s] = c;
        }
        s_cnt[idx] = c;
    }
    if (bad) set_status(p.status, kStOutOfBounds);
    __syncthreads();

    // blocked exclusive scan: thread t owns segments 8t .. 8t+7 of the tile
    int32_t v[kScanItems];
    {
        const int4 *src = reinterpret_cast<const int4 *>(s_cnt + kScanItems * t);
        const int4 u0 = src[0], u1 = src[1];
        v[0] = u0.x; v[1] = u0.y; v[2] = u0.z; v[3] = u0.w;
        v[4] = u1.x; v[5] = u1.y; v[6] = u1.z; v[7] = u1.w;
    }
    int32_t ex[kScanItems];
    int32_t run = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        ex[k] = run;
        run += v[k];
    }
    int64_t inc = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    int64_t warp_base = 0, total = 0;
#pragma unroll
    for (int wi = 0; wi < kScanThreads / 32; ++wi) {
        const int64_t sw = s_warp[wi];
        if (wi < warp) warp_base += sw;
        total += sw;
    }
    const int64_t thread_excl = warp_base + inc - run;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) s_loc[kScanItems * t + k] = thread_excl + ex[k];

    // decoupled look-back by warp 0
    if (warp == 0) {
        const bool stall = (tile == p.stall_tile);
        int64_t excl = 0;
        if (tile == 0) {
            if (lane == 0 && !stall) st_relaxed_u64(p.desc, kDescInc | static_cast<uint64_t>(total));
        } else {
            if (lane == 0 && !stall) st_relaxed_u64(p.desc + tile, kDescAgg | static_cast<uint64_t>(total));
            int64_t look = tile - 1;
            uint64_t t0 = 0;
            bool timed_out = false;
            while (true) {
                const int64_t idx = look - lane;
                const uint64_t dv = idx >= 0 ? ld_relaxed_u64(p.desc + idx) : kDescInc;
                const uint32_t flag = static_cast<uint32_t>(dv >> 62);
                const uint32_t inc_mask = __ballot_sync(0xffffffffu, flag == 2u);
                const uint32_t zero_mask = __ballot_sync(0xffffffffu, flag == 0u);
                const int first_inc = inc_mask ? __ffs(inc_mask) - 1 : 32;
                const uint32_t need = first_inc >= 31 ? 0xffffffffu : ((2u << first_inc) - 1u);
                if (zero_mask & need) {
                    // a predecessor has not published yet: spin, within a bound (the
                    // clock is read by lane 0 so that the whole warp decides alike)
                    const uint64_t now = __shfl_sync(0xffffffffu, globaltimer_ns(), 0);
                    if (t0 == 0) t0 = now;
                    if (now - t0 <= p.wait_ns) {
                        __nanosleep(64);
                        continue;
                    }
                    timed_out = true;
                    if (lane == 0) set_status(p.status, kStTimeout);
                }
                int64_t part = (lane <= first_inc && flag != 0u) ? static_cast<int64_t>(dv & kDescValue) : 0;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
                excl += part;
                if (first_inc < 32 || timed_out) break;
                look -= 32;
                t0 = 0;
            }
            if (lane == 0 && !stall) st_relaxed_u64(p.desc + tile, kDescInc | static_cast<uint64_t>(excl + total));
        }
        if (lane == 0) {
            s_excl = excl;
            s_total = total;
        }
    }
    __syncthreads();

    const int64_t excl = s_excl;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        const int idx = j * kScanThreads + t;
        const int64_t s = base + idx;
        if (s < p.n) {
            const int64_t o = excl + s_loc[idx];
            p.offsets[s] = o;
            if (p.offsets_out) p.offsets_out[s] = o;
            if (p.offsets_copy) p.offsets_copy[s] = o;
        }
    }
    if (tile == p.n_tiles - 1 && t == 0) {
        const int64_t V = excl + s_total;
        p.offsets[p.n] = V;
        // padding entries: even-sized bulk copies of the offsets may read them
        p.offsets[p.n + 1] = V;
        p.offsets[p.n + 2] = V;
        p.offsets[p.n + 3] = V;
        if (p.offsets_out) p.offsets_out[p.n] = V;
    }
}

// ------------------------------------------------------------------ generation
// kOutSegRuns: with kOutList32 alone, runs cut at segment ends (launch tuning list_runs)
// kOutWarpDedup: with kOutMask alone, words merged across the warp before their atomics
enum : int { kOutList32 = 1, kOutList64 = 2, kOutMask = 4, kOutSegRuns = 8, kOutWarpDedup = 16 };

struct GenParams {
    const int32_t *segs;     // [n][6], 16-byte aligned
    int64_t n;
    const int64_t *offsets;  // [n + 4], 16-byte aligned (workspace)
    int32_t w, h, d;
    void *list;              // uint32 / uint64 list or null
    int64_t capacity;
    uint32_t *mask;          // volume or null
    int32_t *status;
    uint64_t wait_ns;
    int64_t min_per_cta;     // smallest voxel range worth a CTA (multiple of 4)
    const int64_t *gate_total;  // if set, run only when *gate_total > gate_cap
    int64_t gate_cap;
    const SceneDesc *scenes;    // batched volume: per-segment volume from its scene
    const int32_t *scene_of;    // (else null: one volume, p.w / p.h / p.mask)
    int32_t n_scenes;
    int32_t interleave;         // voxel tiles dealt round-robin to CTAs (else one range per CTA)
};

// Stage word of the pass's voxel at position x in the linear layout: two pad
// words after every 2R positions, so that threads writing runs of R (or 2R)
// voxels that start at multiples of R hit different banks (at most two-way), and
// pairs (x even) never straddle a pad.
template <int R>
__host__ __device__ constexpr int32_t lin_index(int32_t x)
{
    return x + 2 * (x / (2 * R));
}

// Shared memory of k_generate: the staged window of segments and, for list
// outputs, the pass's voxels. Runs of R consecutive voxels that may cross into
// the next segments use a transposed layout (run slot u of thread t at u * S + t,
// S = 256 + 32 / R, or 257 for R >= 32) that is free of bank conflicts when the
// threads write their runs and when the pass is read back four voxels per thread
// (two-way for R = 64, where a warp reads 16 slots of each of two threads). A
// 32-bit list alone with kOutSegRuns cuts its runs at segment ends instead,
// staged linearly (lin_index).
template <int R, int OUT>
struct GenLayout {
    static constexpr bool kList = (OUT & (kOutList32 | kOutList64)) != 0;
    static constexpr bool kWide = (OUT & kOutList64) != 0;
    static constexpr bool kSegRuns = OUT == (kOutList32 | kOutSegRuns);
    static constexpr int S = kGenThreads + (R >= 32 ? 1 : 32 / R);
    static constexpr int kPlanes = kWide ? 2 : 1;
    // positions 0 .. kGenThreads R + 3 (a pass starts up to 3 after a multiple of 4), read in pairs
    static constexpr int kLinWords = (lin_index<R>(kGenThreads * R + 3) + 2 + 3) & ~3;
    static constexpr int kTransWords = kList ? kPlanes * R * S : 4;
    static constexpr int kStageWords = kSegRuns ? kLinWords : kTransWords;
};

// The two TMA destinations (offs, recs) must start on 16-byte boundaries; they
// lead the struct and their sizes are multiples of 16 (checked below).
template <int R, int OUT>
struct GenSmem {
    alignas(16) int64_t offs[kWindowSegs + 2];
    alignas(16) int32_t recs[kWindowSegs * 6];
    alignas(16) uint32_t stage[GenLayout<R, OUT>::kStageWords];
    int32_t runstart[kWindowSegs + 1];      // segment-cut runs: first run of each window segment
    int32_t warp_tot[kGenThreads / 32];     // block scan
    int64_t pass_lo, pass_hi;               // voxel range of the current pass
    uint64_t bar;
    int64_t V;
    int32_t go;
    int32_t pad;
};
static_assert((kWindowSegs + 2) * sizeof(int64_t) % 16 == 0, "offs size");
static_assert(kWindowSegs * 6 * sizeof(int32_t) % 16 == 0, "recs size");
using GenSmemL32 = GenSmem<32, 1>;
using GenSmemL64M = GenSmem<16, 6>;
using GenSmemM = GenSmem<32, 4>;
static_assert(offsetof(GenSmemL32, offs) % 16 == 0 && offsetof(GenSmemL32, recs) % 16 == 0 &&
                  offsetof(GenSmemL64M, recs) % 16 == 0 && offsetof(GenSmemM, recs) % 16 == 0 &&
                  offsetof(GenSmemL32, bar) % 8 == 0,
              "TMA destinations must be 16-byte aligned");

// Largest s in [lo, hi) with offsets[s] <= g, given offsets[lo] <= g < offsets[hi]:
// a 256-ary search where each round every thread probes one position. Must be
// called by all threads of the CTA with the same arguments.
__device__ __forceinline__ int64_t find_segment_block(const int64_t *offsets, int64_t lo, int64_t hi, int64_t g)
{
    while (hi - lo > 1) {
        const int64_t span = hi - lo;
        const int64_t stride = (span + kGenThreads - 1) / kGenThreads;
        const int64_t pos = lo + static_cast<int64_t>(threadIdx.x) * stride;
        const bool le = pos < hi && __ldg(offsets + pos) <= g;
        const int cnt = __syncthreads_count(le);  // probes 0 .. cnt-1 satisfy (monotone)
        const int64_t nlo = lo + static_cast<int64_t>(cnt - 1) * stride;
        const int64_t nhi = min(hi, lo + static_cast<int64_t>(cnt) * stride);
        lo = nlo;
        hi = nhi;
    }
    return lo;
}

// Largest j in [0, cnt) with offs[j] <= g (offs[0] <= g < offs[cnt]); cnt <= kWindowSegs.
__device__ __forceinline__ int32_t find_in_window(const int64_t *offs, int32_t cnt, int64_t g)
{
    int32_t lo = 0;
#pragma unroll
    for (int32_t step = kWindowSegs / 2; step > 0; step >>= 1) {
        const int32_t m = lo + step;
        if (m < cnt && offs[m] <= g) lo = m;
    }
    return lo;
}

// Largest j in [0, cnt) with rs[j] <= r (rs[0] = 0 <= r < rs[cnt]); the segment
// found has at least one run, since a segment without runs shares its rs entry
// with the next one.
__device__ __forceinline__ int32_t find_run(const int32_t *rs, int32_t cnt, int32_t r)
{
    int32_t lo = 0;
#pragma unroll
    for (int32_t step = kWindowSegs / 2; step > 0; step >>= 1) {
        const int32_t m = lo + step;
        if (m < cnt && rs[m] <= r) lo = m;
    }
    return lo;
}

// Exclusive prefix sum of v over the CTA (kGenThreads threads, all calling);
// total receives the sum. warp_tot: kGenThreads / 32 words of shared memory,
// free until the caller's next barrier.
__device__ __forceinline__ int32_t block_exclusive_scan(int32_t v, int32_t *warp_tot, int32_t &total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int32_t inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) warp_tot[wid] = inc;
    __syncthreads();
    int32_t base = 0, tot = 0;
#pragma unroll
    for (int i = 0; i < kGenThreads / 32; ++i) {
        const int32_t x = warp_tot[i];
        base += i < wid ? x : 0;
        tot += x;
    }
    total = tot;
    return base + inc - v;
}

// OR `bits` into a volume word as a reduction (no return value), asking L2 to
// keep the line (the volume is re-touched; list lines are not).
__device__ __forceinline__ void red_or_keep(uint32_t *addr, uint32_t bits, uint64_t policy)
{
    asm volatile("red.relaxed.gpu.global.or.L2::cache_hint.b32 [%0], %1, %2;" ::"l"(addr), "r"(bits), "l"(policy)
                 : "memory");
}

// Warp-aggregated OR: the lanes with `pred` each hold (addr, bits); lanes with the
// same word address form a group (__match_any_sync), the group's bits are OR-ed
// together (__reduce_or_sync), and the group's first lane issues one reduction
// for the group. Called by the whole warp (converged).
__device__ __forceinline__ void warp_red_or(bool pred, uint32_t *addr, uint32_t bits, uint64_t policy)
{
    const uint32_t fm = __ballot_sync(0xffffffffu, pred);
    if (pred) {
        const uint32_t grp = __match_any_sync(fm, reinterpret_cast<unsigned long long>(addr));
        const uint32_t all = __reduce_or_sync(grp, bits);
        if ((threadIdx.x & 31) == static_cast<unsigned>(__ffs(grp) - 1)) red_or_keep(addr, all, policy);
    }
}

template <int R, int OUT, bool LIN64>
__global__ void __launch_bounds__(kGenThreads, 3) k_generate(GenParams p)
{
    using L = GenLayout<R, OUT>;
    using PackT = typename std::conditional<L::kWide, uint64_t, uint32_t>::type;
    using LinT = typename std::conditional<LIN64, uint64_t, uint32_t>::type;
    constexpr bool kList = L::kList;
    constexpr bool kMask = (OUT & kOutMask) != 0;
    constexpr bool kWarpDedup = (OUT & kOutWarpDedup) != 0;
    static_assert(!kWarpDedup || OUT == (kOutMask | kOutWarpDedup), "warp-merged atomics: volume alone");
    constexpr int kPass = kGenThreads * R;
    constexpr int S = L::S;
    static_assert(R % 4 == 0 && 32 % R == 0 || R == 32 || R == 64, "run length");

    extern __shared__ __align__(16) unsigned char smem_raw[];
    GenSmem<R, OUT> &sm = *reinterpret_cast<GenSmem<R, OUT> *>(smem_raw);
    const int t = threadIdx.x;

    // prologue decided by one thread so that the whole CTA agrees
    if (t == 0) {
        int32_t go = ld_volatile_i32(p.status) == 0;  // an earlier error: write nothing
        if (p.gate_total != nullptr && __ldg(p.gate_total) <= p.gate_cap) go = 0;  // brick path took it
        const int64_t V = __ldg(p.offsets + p.n);
        if (go && kList && V > p.capacity) {
            set_status(p.status, kStCapacity);
            go = 0;
        }
        sm.V = V;
        sm.go = go;
        mbar_init(&sm.bar, 1);
        fence_barrier_init();
    }
    __syncthreads();
    if (!sm.go) return;
    const int64_t V = sm.V;
    // voxel ranges: one contiguous range per CTA (a multiple of 4 long), or
    // tiles of one pass dealt round-robin, so that the CTAs sweep the voxel
    // order together (the volumes they touch at any moment stay few and hot)
    int64_t per = (V + gridDim.x - 1) / gridDim.x;
    per = max(per, p.min_per_cta);
    per = (per + 3) & ~int64_t(3);
    if (p.interleave) per = kPass;

    uint64_t keep_policy = 0;
    if (kMask) asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(keep_policy));
    uint32_t phase = 0;

    LinT w = static_cast<LinT>(p.w);
    LinT wh = static_cast<LinT>(p.w) * static_cast<LinT>(p.h);
    uint32_t *mask_s = p.mask;
    const bool batched = p.scene_of != nullptr;
    // the volume of segment `seg` (batched): dims and base pointer of its scene
#define VOX_USE_SCENE_OF(seg)                                              \
    do {                                                                   \
        const SceneDesc &sd_ = p.scenes[__ldg(p.scene_of + (seg))];        \
        w = static_cast<LinT>(sd_.w);                                      \
        wh = static_cast<LinT>(sd_.w) * static_cast<LinT>(sd_.h);          \
        mask_s = sd_.mask;                                                 \
    } while (0)
    PackT *const list = static_cast<PackT *>(p.list);
    for (int64_t range = blockIdx.x;; range += gridDim.x) {
    const int64_t gA = range * per;
    if (gA >= V) break;
    const int64_t gB = min64(gA + per, V);
    int64_t s_cur = find_segment_block(p.offsets, 0, p.n, gA);
    int64_t g0 = gA;
    while (g0 < gB) {
        // ---- stage a window of segment records and offsets (TMA bulk copies)
        const int64_t s_base = s_cur & ~int64_t(1);
        const int32_t cnt = static_cast<int32_t>(min64(kWindowSegs, p.n - s_base));
        const int32_t cnt_bulk = cnt & ~1;           // 24 * even bytes is a multiple of 16
        const int32_t off_entries = (cnt + 3) & ~1;  // entries s_base .. s_base+cnt (+1 pad), even
        __syncthreads();                             // previous window fully consumed
        if (t == 0) {
            fence_proxy_async_smem();
            const uint32_t rec_bytes = static_cast<uint32_t>(cnt_bulk) * 24u;
            const uint32_t off_bytes = static_cast<uint32_t>(off_entries) * 8u;
            mbar_arrive_expect_tx(&sm.bar, rec_bytes + off_bytes);
            if (rec_bytes) bulk_copy_g2s(sm.recs, p.segs + 6 * s_base, rec_bytes, &sm.bar);
            bulk_copy_g2s(sm.offs, p.offsets + s_base, off_bytes, &sm.bar);
        }
        if (cnt != cnt_bulk && t < 6) sm.recs[6 * cnt_bulk + t] = __ldg(p.segs + 6 * (s_base + cnt_bulk) + t);
        const bool landed = mbar_wait_bounded(&sm.bar, phase, p.wait_ns);
        phase ^= 1u;
        if (__syncthreads_or(!landed)) {
            // a copy did not land in time: report, give it one more bounded wait, stop
            if (t == 0) set_status(p.status, kStTimeout);
            if (!landed) mbar_wait_bounded(&sm.bar, phase ^ 1u, p.wait_ns);
            return;
        }

        const int64_t win_end = sm.offs[cnt];  // first voxel after the window's segments
        int64_t g_end = gB;
        if (win_end < gB) g_end = win_end & ~int64_t(3);

        // runs cut at segment ends (kOutSegRuns): lanes of a warp do not wait on
        // each other's segment changes when segment lengths differ; runs across
        // segment ends (below) cost less when every lane changes segment at the
        // same step (segments of one length that R divides, or that divides R)
        if constexpr (L::kSegRuns) {
            {
                // the voxels of window segment j in [g0, g_end) form ceil(len / R)
                // runs of R consecutive voxels (the last one shorter); thread t of a
                // pass takes run r0 + t and enters its segment once
                int32_t c = 0;
                if (t < cnt) {
                    const int64_t a = max64(sm.offs[t], g0), b = min64(sm.offs[t + 1], g_end);
                    if (b > a) c = static_cast<int32_t>((b - a + R - 1) / R);
                }
                int32_t total_runs;
                const int32_t first = block_exclusive_scan(c, sm.warp_tot, total_runs);
                sm.runstart[t] = first;
                if (t == kGenThreads - 1) sm.runstart[kGenThreads] = first + c;
                __syncthreads();
                for (int32_t r0 = 0; r0 < total_runs; r0 += kGenThreads) {
                    const int32_t r = r0 + t;
                    const int32_t n_runs = min(kGenThreads, total_runs - r0);
                    int32_t j = 0, len = 0;
                    int64_t g = 0;
                    if (r < total_runs) {
                        j = find_run(sm.runstart, cnt, r);
                        g = max64(sm.offs[j], g0) + static_cast<int64_t>(r - sm.runstart[j]) * R;
                        len = static_cast<int32_t>(min64(R, min64(sm.offs[j + 1], g_end) - g));
                    }
                    if (t == 0) sm.pass_lo = g;
                    if (t == n_runs - 1) sm.pass_hi = g + len;
                    __syncthreads();
                    // stage position x holds voxel gb + x; gb is a multiple of 4, so
                    // that 4-voxel groups and 16-byte aligned list addresses coincide
                    const int64_t gb = sm.pass_lo & ~int64_t(3);
                    const int32_t xs = static_cast<int32_t>(sm.pass_lo - gb);
                    const int32_t xe = static_cast<int32_t>(sm.pass_hi - gb);
                    if (r < total_runs) {
                        Stepper<PackT, LinT> st;
                        st.enter(sm.recs + 6 * j, static_cast<int32_t>(g - sm.offs[j]), w, wh);
                        int32_t x = static_cast<int32_t>(g - gb);
                        int32_t u = 0;
                        for (; u < len && (x & 3) != 0; ++u, ++x) {  // up to a multiple of 4
                            sm.stage[lin_index<R>(x)] = static_cast<uint32_t>(st.P);
                            st.template step<true, false>();
                        }
                        // groups of four: one pointer, fixed offsets; a group never
                        // straddles the pad after 2R positions
                        uint32_t *sp = sm.stage + lin_index<R>(x);
                        for (; u + 4 <= len; u += 4) {
#pragma unroll
                            for (int v = 0; v < 4; ++v) {
                                sp[v] = static_cast<uint32_t>(st.P);
                                st.template step<true, false>();
                            }
                            x += 4;
                            sp += (x & (2 * R - 1)) == 0 ? 6 : 4;
                        }
                        for (; u < len; ++u, ++x) {
                            sm.stage[lin_index<R>(x)] = static_cast<uint32_t>(st.P);
                            st.template step<true, false>();
                        }
                    }
                    __syncthreads();
                    // write the pass out: voxels gb + [xs, xe), two per thread and
                    // round (8-byte stores), the pass's first and last pair word by word
                    for (int32_t x0 = 2 * t; x0 < xe; x0 += 2 * kGenThreads) {
                        const uint2 v = *reinterpret_cast<const uint2 *>(sm.stage + lin_index<R>(x0));
                        if (x0 >= xs && x0 + 2 <= xe) {
                            *reinterpret_cast<uint2 *>(list + gb + x0) = v;
                        } else {
                            if (x0 >= xs) list[gb + x0] = v.x;
                            if (x0 + 1 >= xs && x0 + 1 < xe) list[gb + x0 + 1] = v.y;
                        }
                    }
                    __syncthreads();
                }
            }
        } else if constexpr (kWarpDedup) {
            // the volume alone, words merged across the warp: thread t takes the R
            // consecutive voxels from gp + t R as below, but the warp walks its 32
            // runs in step (R iterations, finished lanes idle), so that at every
            // step the lanes whose word just ended can merge it with the other
            // lanes' equal words before one reduction per distinct word
            for (int64_t gp = g0; gp < g_end; gp += kPass) {
                const int64_t g = gp + static_cast<int64_t>(t) * R;
                const int32_t len = g < g_end ? static_cast<int32_t>(min64(R, g_end - g)) : 0;
                Stepper<PackT, LinT> st;
                int32_t j = 0, left = 0;
                if (len > 0) {
                    j = find_in_window(sm.offs, cnt, g);
                    if (batched) VOX_USE_SCENE_OF(s_base + j);
                    const int32_t k = static_cast<int32_t>(g - sm.offs[j]);
                    st.enter(sm.recs + 6 * j, k, w, wh);
                    left = st.left;
                }
                uint32_t *cur = nullptr;  // the word being filled (address) and its bits
                uint32_t acc = 0;
                for (int32_t u = 0; u < R; ++u) {
                    uint32_t *fw = nullptr;
                    uint32_t fb = 0;
                    if (u < len) {
                        uint32_t *const word = mask_s + (st.L >> 5);
                        if (word != cur) {
                            fw = cur;
                            fb = acc;
                            cur = word;
                            acc = 0;
                        }
                        acc |= 1u << (static_cast<uint32_t>(st.L) & 31u);
                        if (left > 0) {
                            st.template step<false, true>();
                            --left;
                        } else if (u + 1 < len) {  // the run continues in the next segment
                            ++j;
                            if (batched) VOX_USE_SCENE_OF(s_base + j);
                            st.enter(sm.recs + 6 * j, 0, w, wh);
                            left = st.left;
                        }
                    }
                    warp_red_or(fb != 0 && mask_s != nullptr && fw != nullptr, fw, fb, keep_policy);
                }
                warp_red_or(acc != 0 && mask_s != nullptr && cur != nullptr, cur, acc, keep_policy);
            }
        } else
        // ---- passes over [g0, g_end): thread t takes the R consecutive voxels
        // starting at gp + t R, walking segment by segment
        for (int64_t gp = g0; gp < g_end; gp += kPass) {
            const int64_t g = gp + static_cast<int64_t>(t) * R;
            if (g < g_end) {
                const int32_t len = static_cast<int32_t>(min64(R, g_end - g));
                int32_t j = find_in_window(sm.offs, cnt, g);
                if (kMask && batched) VOX_USE_SCENE_OF(s_base + j);
                Stepper<PackT, LinT> st;
                st.enter(sm.recs + 6 * j, static_cast<int32_t>(g - sm.offs[j]), w, wh);
                uint32_t *sp = sm.stage + t;
                LinT cur_word = static_cast<LinT>(~LinT(0));
                uint32_t acc = 0;
                int32_t u = 0;
                while (true) {
                    const int32_t m = min(st.left + 1, len - u);  // voxels taken from this segment
                    int32_t e = 0;
                    if constexpr (kList && !kMask) {
                        // four voxels per iteration: stores at fixed offsets from one pointer
                        for (; e + 4 <= m; e += 4) {
#pragma unroll
                            for (int v = 0; v < 4; ++v) {
                                sp[v * S] = static_cast<uint32_t>(st.P);
                                if (L::kWide)
                                    sp[R * S + v * S] = static_cast<uint32_t>(static_cast<uint64_t>(st.P) >> 32);
                                st.template step<true, false>();
                            }
                            sp += 4 * S;
                        }
                    }
                    for (; e < m; ++e) {
                        if (kList) {
                            sp[0] = static_cast<uint32_t>(st.P);
                            if (L::kWide) sp[R * S] = static_cast<uint32_t>(static_cast<uint64_t>(st.P) >> 32);
                            sp += S;
                        }
                        if (kMask) {
                            const LinT word = st.L >> 5;
                            if (word != cur_word) {
                                if (acc && mask_s) red_or_keep(mask_s + cur_word, acc, keep_policy);
                                cur_word = word;
                                acc = 0;
                            }
                            acc |= 1u << (static_cast<uint32_t>(st.L) & 31u);
                        }
                        st.template step<kList, kMask>();
                    }
                    u += m;
                    if (u >= len) break;
                    ++j;  // the run continues in the next segment of the window
                    if (kMask && batched) {  // the next segment may live in another volume
                        if (acc && mask_s) red_or_keep(mask_s + cur_word, acc, keep_policy);
                        acc = 0;
                        cur_word = static_cast<LinT>(~LinT(0));
                        VOX_USE_SCENE_OF(s_base + j);
                    }
                    st.enter(sm.recs + 6 * j, 0, w, wh);
                }
                if (kMask && acc && mask_s) red_or_keep(mask_s + cur_word, acc, keep_policy);  // scenes may have no volume
            }
            if (kList) {
                // ---- write the pass out: four consecutive voxels per thread, 16-byte stores
                __syncthreads();
                const int32_t pass_len = static_cast<int32_t>(min64(kPass, g_end - gp));
                const int32_t n4 = pass_len >> 2;
                for (int32_t q = t; q < n4; q += kGenThreads) {
                    const int32_t p0 = 4 * q;
                    // voxels p0 .. p0+3 sit in slots p0 % R .. +3 of thread p0 / R
                    // (R is a multiple of 4): one base index, three fixed strides
                    const uint32_t *src = sm.stage + (p0 % R) * S + p0 / R;
                    uint32_t lo[4], hi[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        lo[e] = src[e * S];
                        if (L::kWide) hi[e] = src[R * S + e * S];
                    }
                    if constexpr (L::kWide) {
                        ulonglong2 *dst = reinterpret_cast<ulonglong2 *>(list + gp + p0);
                        dst[0] = make_ulonglong2(lo[0] | (static_cast<unsigned long long>(hi[0]) << 32),
                                                 lo[1] | (static_cast<unsigned long long>(hi[1]) << 32));
                        dst[1] = make_ulonglong2(lo[2] | (static_cast<unsigned long long>(hi[2]) << 32),
                                                 lo[3] | (static_cast<unsigned long long>(hi[3]) << 32));
                    } else {
                        *reinterpret_cast<uint4 *>(list + gp + p0) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
                    }
                }
                if (t == 0) {
                    for (int32_t pe = 4 * n4; pe < pass_len; ++pe) {
                        const int32_t idx = (pe % R) * S + pe / R;
                        uint64_t v = sm.stage[idx];
                        if (L::kWide) v |= static_cast<uint64_t>(sm.stage[R * S + idx]) << 32;
                        list[gp + pe] = static_cast<PackT>(v);
                    }
                }
                __syncthreads();
            }
        }
        g0 = g_end;
        if (g0 < gB) s_cur = (g0 >= win_end) ? s_base + cnt : s_base + find_in_window(sm.offs, cnt, g0);
    }
    if (!p.interleave) break;
    }
#undef VOX_USE_SCENE_OF
}

// Batched scenes: check the scene table (contiguous, in order, covering all n
// segments; dims in range; 32-bit lists need edges <= 1024) and record each
// segment's scene. One CTA per scene. Any error goes to *status and the
// generation kernels then write nothing.
__global__ void __launch_bounds__(256) k_scene_map(const SceneDesc *scenes, int32_t n_scenes, int64_t n_total,
                                                   int32_t *scene_of, int32_t *status, int32_t list32)
{
    const int32_t k = blockIdx.x;
    const SceneDesc sd = scenes[k];
    const int64_t expect = k == 0 ? 0 : scenes[k - 1].seg_begin + scenes[k - 1].n;
    const int32_t lim = 1 << 21;
    bool ok = sd.n >= 0 && sd.seg_begin == expect && sd.seg_begin + sd.n <= n_total && sd.reserved == 0 &&
              sd.w >= 1 && sd.h >= 1 && sd.d >= 1 && sd.w <= lim && sd.h <= lim && sd.d <= lim;
    if (k == n_scenes - 1) ok = ok && sd.seg_begin + sd.n == n_total;
    if (threadIdx.x == 0) {
        if (!ok) set_status(status, 1);  // VOX_ERR_INVALID_ARG
        else if (list32 && (sd.w > 1024 || sd.h > 1024 || sd.d > 1024)) set_status(status, 3);  // PACK_WIDTH
    }
    if (!ok) return;
    for (int64_t i = threadIdx.x; i < sd.n; i += blockDim.x) scene_of[sd.seg_begin + i] = k;
}

// Fresh batched volumes: scene blockIdx.y's volume zeroed by kSceneClearCtas
// CTAs (16-byte stores from the first 16-byte boundary on), after k_scene_map
// has checked the table (nothing written otherwise).
constexpr unsigned kSceneClearCtas = 512;
__global__ void __launch_bounds__(256) k_scene_clear(const SceneDesc *scenes, const int32_t *status)
{
    if (ld_volatile_i32(status) != 0) return;
    const SceneDesc sd = scenes[blockIdx.y];
    if (sd.mask == nullptr) return;
    const int64_t words = (static_cast<int64_t>(sd.w) * sd.h * sd.d + 31) / 32;
    const int64_t tid = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t nthreads = static_cast<int64_t>(gridDim.x) * blockDim.x;
    // words before the first 16-byte boundary, then whole 16-byte groups, then the tail
    const int64_t head = min64(words, static_cast<int64_t>((16 - (reinterpret_cast<uintptr_t>(sd.mask) & 15)) & 15) / 4);
    if (tid < head) sd.mask[tid] = 0u;
    uint4 *body = reinterpret_cast<uint4 *>(sd.mask + head);
    const int64_t groups = (words - head) / 4;
    for (int64_t i = tid; i < groups; i += nthreads) body[i] = make_uint4(0u, 0u, 0u, 0u);
    const int64_t tail0 = head + 4 * groups;
    if (tail0 + tid < words) sd.mask[tail0 + tid] = 0u;
}

// The brick numbering of a batch: every scene's geometry (one counter replica),
// first brick and first slot, in scene order. One CTA: each thread takes a
// chunk of consecutive scenes, a block scan of the chunks' brick counts gives
// the chunks' first bricks. A scene that cannot take bricks, or a total that
// differs from the caller's, is VOX_ERR_INVALID_ARG (nothing is written after).
constexpr int kSceneBrickThreads = 256;
__global__ void __launch_bounds__(kSceneBrickThreads) k_scene_bricks(const SceneDesc *scenes, int32_t n_scenes,
                                                                    SceneBricks *sb, int32_t *brick_scene,
                                                                    int64_t total_bricks, int32_t *status)
{
    __shared__ int64_t s_sum[kSceneBrickThreads];
    __shared__ int32_t s_bad;
    const int t = threadIdx.x;
    if (__syncthreads_or(ld_volatile_i32(status) != 0)) return;  // the table was refused (the CTA agrees)
    if (t == 0) s_bad = 0;
    __syncthreads();
    const int32_t per = (n_scenes + kSceneBrickThreads - 1) / kSceneBrickThreads;
    const int32_t k0 = min(n_scenes, t * per), k1 = min(n_scenes, k0 + per);
    int64_t own = 0;
    for (int32_t k = k0; k < k1; ++k) {  // geometry of the chunk; bases below
        SceneBricks e;
        if (!brick_geom(scenes[k].w, scenes[k].h, scenes[k].d, &e.G, false)) {
            s_bad = 1;
            e.G.n_bricks = 0;
        }
        e.mask = scenes[k].mask;
        sb[k] = e;
        own += e.G.n_bricks;
    }
    s_sum[t] = own;
    __syncthreads();
    for (int o = 1; o < kSceneBrickThreads; o <<= 1) {  // inclusive scan of the chunks' counts
        const int64_t v = t >= o ? s_sum[t - o] : 0;
        __syncthreads();
        s_sum[t] += v;
        __syncthreads();
    }
    const bool ok = !s_bad && s_sum[kSceneBrickThreads - 1] == total_bricks;
    int64_t next = s_sum[t] - own;
    for (int32_t k = k0; k < k1; ++k) {
        sb[k].brick_base = next;
        sb[k].slot_base = next * kPieceClasses;
        if (ok)  // the scene of every brick (sized by total_bricks)
            for (int64_t b = 0; b < sb[k].G.n_bricks; ++b) brick_scene[next + b] = k;
        next += sb[k].G.n_bricks;
    }
    if (t == kSceneBrickThreads - 1 && !ok) set_status(status, 1);  // VOX_ERR_INVALID_ARG
}

// First global voxel id of every scene (and V at index n_scenes).
__global__ void k_scene_base(const SceneDesc *scenes, int32_t n_scenes, const int64_t *offsets, int64_t n_total,
                             int64_t *base, int64_t *base_out, const int32_t *status)
{
    const int64_t k = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (k > n_scenes || ld_volatile_i32(status) != 0) return;
    const int64_t v = k < n_scenes ? __ldg(offsets + scenes[k].seg_begin) : __ldg(offsets + n_total);
    base[k] = v;
    if (base_out) base_out[k] = v;
}

}  // namespace vox
