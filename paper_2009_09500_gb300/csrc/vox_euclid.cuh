// vox_euclid.cuh -- the Euclidean-N variant of Eq. (1)-(2) (sm_103a).
//
// N = int(|E - S|), the integer part of the Euclidean length; the samples are
// G_k = S + W k, W = (E - S) / N, k = 0..N, each mapped to its nearest lattice
// point exactly as in the main path (the rounding of Eq. (3) with this N). Since
// N can exceed max |d_a|, consecutive samples can share a voxel, and the voxel
// set of Fig. 3 holds it once: a sample adds its voxel only when some axis moved
// at that step (the first sample of a segment always adds).
//
// Work is split into runs of consecutive samples in global sample order (the
// scan of per-segment sample counts N + 1 gives each segment's first sample):
//   k_euclid_warp<false>  voxels added per run (a warp walks 32 runs)
//   k_scan<false>         exclusive scan of the run counts (output positions)
//   k_euclid_warp<true>   the list: the voxels, written compacted at their run's
//                         position (segment offsets and volume atomics on the way)
//   k_euclid_runs<true>   one thread per run: the volume's atomics or the segment
//                         offsets when no list is written, and the gated
//                         atomics after the brick path
#pragma once

#include <cstdint>

#include "vox_device.cuh"
#include "vox_kernels.cuh"
#include "vox_list.cuh"

namespace vox {

constexpr int64_t kEuclidMinRun = 32;       // samples per run at least
constexpr int64_t kEuclidRunSlots = 1 << 20;  // run slots at least (more for many segments)


struct EuclidParams {
    const int32_t *segs;
    int64_t n;
    const int64_t *offsets;  // [n + 1] first sample of every segment; [n] = samples in all
    int32_t w, h;
    int64_t n_runs;          // run slots
    int32_t *run_count;      // [n_runs] voxels added per run (count pass)
    const int64_t *run_off;  // [n_runs + 1] first output position per run (write pass)
    void *list;
    int64_t capacity;
    uint32_t *mask;
    int64_t *seg_off;        // [n] first output position per segment, or null
    int32_t *status;
    const int64_t *gate_total;  // if set (write pass), run only when *gate_total > gate_cap
    int64_t gate_cap;
};

// One thread per run of consecutive samples (grid-stride over the run slots).
template <bool kWrite, int OUT, bool LIN64>
__global__ void __launch_bounds__(256) k_euclid_runs(EuclidParams p)
{
    using PackT = typename std::conditional<(OUT & kOutList64) != 0, uint64_t, uint32_t>::type;
    using LinT = typename std::conditional<LIN64, uint64_t, uint32_t>::type;
    constexpr bool kList = (OUT & (kOutList32 | kOutList64)) != 0;
    constexpr bool kMask = (OUT & kOutMask) != 0;
    if (ld_volatile_i32(p.status) != 0) return;  // an earlier error: write nothing
    if (kWrite && p.gate_total != nullptr && __ldg(p.gate_total) <= p.gate_cap) return;  // the bricks took it
    const int64_t Vs = __ldg(p.offsets + p.n);
    const int64_t L = max(kEuclidMinRun, (Vs + p.n_runs - 1) / p.n_runs);
    if (kWrite && kList && __ldg(p.run_off + p.n_runs) > p.capacity) {
        if (blockIdx.x == 0 && threadIdx.x == 0) set_status(p.status, kStCapacity);
        return;
    }
    uint64_t keep_policy = 0;
    if (kWrite && kMask) asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(keep_policy));
    const LinT w = static_cast<LinT>(p.w);
    const LinT wh = static_cast<LinT>(p.w) * static_cast<LinT>(p.h);
    PackT *const list = static_cast<PackT *>(p.list);
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t j = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; j < p.n_runs; j += stride) {
        const int64_t g0 = j * L;
        if (g0 >= Vs) {
            if (!kWrite) p.run_count[j] = 0;
            continue;
        }
        const int64_t g1 = min(g0 + L, Vs);
        // the segment holding sample g0: largest s with offsets[s] <= g0
        int64_t lo = 0, hi = p.n;
        while (hi - lo > 1) {
            const int64_t mid = (lo + hi) >> 1;
            if (__ldg(p.offsets + mid) <= g0) lo = mid;
            else hi = mid;
        }
        int64_t s = lo;
        const int64_t seg_begin = __ldg(p.offsets + s);
        int64_t seg_end = __ldg(p.offsets + s + 1);
        int32_t rec[6];
        {
            const int2 *q = reinterpret_cast<const int2 *>(p.segs + 6 * s);
            const int2 a = __ldg(q), b = __ldg(q + 1), c = __ldg(q + 2);
            rec[0] = a.x; rec[1] = a.y; rec[2] = b.x; rec[3] = b.y; rec[4] = c.x; rec[5] = c.y;
        }
        // the next segment's record and end, loaded ahead so that crossing into it
        // does not wait on memory (segment n - 1 has no successor: nothing loaded)
        int2 na = make_int2(0, 0), nb = na, nc = na;
        int64_t next_end = seg_end;
        auto prefetch = [&](int64_t t) {
            if (t + 1 < p.n && seg_end < g1) {
                const int2 *q = reinterpret_cast<const int2 *>(p.segs + 6 * (t + 1));
                na = __ldg(q);
                nb = __ldg(q + 1);
                nc = __ldg(q + 2);
                next_end = __ldg(p.offsets + t + 2);
            }
        };
        prefetch(s);
        // a segment's N is its sample count minus one (the scan counted N + 1)
        const int32_t k0 = static_cast<int32_t>(g0 - seg_begin);
        EuclidStepper<PackT, LinT> st;
        bool add, first;
        if (k0 == 0) {
            st.enter_n(rec, static_cast<int32_t>(seg_end - seg_begin - 1), 0, w, wh);
            add = first = true;
        } else {  // sample k0 adds a voxel when some axis moved from sample k0 - 1
            st.enter_n(rec, static_cast<int32_t>(seg_end - seg_begin - 1), k0 - 1, w, wh);
            add = st.template step<kWrite && kList, kWrite && kMask>();
            first = false;
        }
        const int64_t base = (kWrite && (kList || p.seg_off != nullptr)) ? __ldg(p.run_off + j) : 0;
        int32_t cnt = 0;
        LinT cur_word = static_cast<LinT>(~LinT(0));
        uint32_t acc = 0;
        // samples g0 + i, i < n_i; the current segment ends before sample g0 + i_end
        // (both below 2^31: a run is short and a segment has at most 2^22 samples)
        const int32_t n_i = static_cast<int32_t>(g1 - g0);
        int32_t i_end = static_cast<int32_t>(seg_end - g0);
        for (int32_t i = 0; i < n_i; ++i) {
            if (i == i_end) {  // the next segment starts here
                ++s;
                const int32_t N = static_cast<int32_t>(next_end - seg_end) - 1;
                seg_end = next_end;
                i_end = static_cast<int32_t>(seg_end - g0);
                rec[0] = na.x; rec[1] = na.y; rec[2] = nb.x; rec[3] = nb.y; rec[4] = nc.x; rec[5] = nc.y;
                prefetch(s);
                st.enter_n(rec, N, 0, w, wh);
                add = first = true;
            }
            if (add) {
                if constexpr (kWrite) {
                    if (kList) list[base + cnt] = st.P;
                    if (first && p.seg_off != nullptr) p.seg_off[s] = base + cnt;
                    if constexpr (kMask) {
                        const LinT word = st.L >> 5;
                        if (word != cur_word) {
                            if (acc) red_or_keep(p.mask + cur_word, acc, keep_policy);
                            cur_word = word;
                            acc = 0;
                        }
                        acc |= 1u << (static_cast<uint32_t>(st.L) & 31u);
                    }
                }
                ++cnt;
            }
            first = false;
            if (i + 1 < i_end) add = st.template step<kWrite && kList, kWrite && kMask>();
        }
        if (kWrite && kMask && acc) red_or_keep(p.mask + cur_word, acc, keep_policy);
        if (!kWrite) p.run_count[j] = cnt;
    }
}

// The warp walk (the count pass and the list writer): a warp takes 32
// consecutive runs, one per lane, and finds the segment of its first sample with
// one 32-ary search in the sample offsets. Segment records and offsets then come
// from per-warp windows of 64 segments in shared memory (coalesced loads), so a
// lane enters a segment, or crosses into the next one, without waiting on global
// memory. A lane's walk is a loop over the parts of its run that lie in one
// segment: at the top of each pass every lane that needs one enters its next
// segment (one division per axis, taken by the lanes together rather than each
// at its own step), then walks the part in a tight loop. A lane stops when it is
// done, its next segment lies beyond the window, or (list) its row is full; when
// every lane has stopped, full rows are flushed and the walk goes on in the same
// window, else the window moves on. Count pass: the voxels each run adds (run_count).
// List pass: each lane appends its voxels to its own row of the warp's stage
// (32 entries for 32-bit lists, 16 for 64-bit ones, rows padded by one entry so
// that lanes at equal fill hit different banks), and a flush writes every row,
// row by row, with coalesced stores at the rows' list positions. Segment offsets
// and (optionally) the volume's atomics are written on the way.
template <typename PackT>
__host__ __device__ constexpr int euclid_row() { return sizeof(PackT) == 4 ? 32 : 16; }

// Largest j in [0, cnt) with offs[j] <= r, given offs[0] <= r < offs[cnt], cnt <= 64.
__device__ __forceinline__ int32_t find_in_window64(const int64_t *offs, int32_t cnt, int64_t r)
{
    int32_t lo = 0;
#pragma unroll
    for (int32_t step = 32; step > 0; step >>= 1) {
        const int32_t m = lo + step;
        if (m < cnt && offs[m] <= r) lo = m;
    }
    return lo;
}

constexpr int kEuclidWarps = 4;  // warps per CTA of the warp walk
constexpr int kEuclidWin = 64;   // segments per staged window

template <typename PackT, bool kRows>
struct EuclidWarpSmem {
    int64_t offs[kEuclidWin + 1];  // sample offsets of the window's segments (+ the next)
    int32_t recs[kEuclidWin * 6];  // the window's segment records
    PackT rows[kRows ? 32 * (euclid_row<PackT>() + 1) : 1];
};

template <bool kWrite, int OUT, bool LIN64>
__global__ void __launch_bounds__(32 * kEuclidWarps, kWrite ? 1 : 12) k_euclid_warp(EuclidParams p)
{
    using PackT = typename std::conditional<(OUT & kOutList64) != 0, uint64_t, uint32_t>::type;
    using LinT = typename std::conditional<LIN64, uint64_t, uint32_t>::type;
    constexpr bool kList = kWrite && (OUT & (kOutList32 | kOutList64)) != 0;
    constexpr bool kMask = kWrite && (OUT & kOutMask) != 0;
    constexpr int kRow = euclid_row<PackT>();
    constexpr int kStride = kRow + 1;
    using Smem = EuclidWarpSmem<PackT, kList>;
    __shared__ Smem smem_all[kEuclidWarps];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    Smem &sm = smem_all[wib];
    // an earlier error: write nothing (decided by the whole warp, which votes later)
    if (__any_sync(0xffffffffu, ld_volatile_i32(p.status) != 0)) return;
    if (kList && __ldg(p.run_off + p.n_runs) > p.capacity) {
        if (blockIdx.x == 0 && threadIdx.x == 0) set_status(p.status, kStCapacity);
        return;
    }
    const int64_t Vs = __ldg(p.offsets + p.n);
    const int64_t L = max(kEuclidMinRun, (Vs + p.n_runs - 1) / p.n_runs);
    uint64_t keep_policy = 0;
    if (kMask) asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(keep_policy));
    const LinT w = static_cast<LinT>(p.w);
    const LinT wh = static_cast<LinT>(p.w) * static_cast<LinT>(p.h);
    PackT *const list = static_cast<PackT *>(p.list);
    PackT *const row = sm.rows + (kList ? lane * kStride : 0);
    const int64_t n_groups = (p.n_runs + 31) / 32;
    const int64_t warps = static_cast<int64_t>(gridDim.x) * kEuclidWarps;
    for (int64_t grp = static_cast<int64_t>(blockIdx.x) * kEuclidWarps + wib; grp < n_groups; grp += warps) {
        const int64_t j = grp * 32 + lane;
        const int64_t g0 = j * L;  // the run's first sample
        const bool has = j < p.n_runs && g0 < Vs;
        // samples g0 + i, i < n_i (below 2^31: a run is short)
        const int32_t n_i = has ? static_cast<int32_t>(min64(g0 + L, Vs) - g0) : 0;
        int32_t cnt = 0;
        if (__any_sync(0xffffffffu, has)) {  // lane 0 has a run whenever any lane has
            int64_t ws = warp_find_segment(p.offsets, p.n, grp * 32 * L, lane);  // first segment of the window
            int32_t i = 0;
            int32_t i_end = 0;     // end of the current segment, as a sample index of the run
            bool in_seg = false;   // stepping state valid for the current segment
            bool add = false;      // the current sample adds its voxel
            int64_t cur = 0;       // the current segment
            EuclidStepper<PackT, LinT> st;
            int64_t outp = (kWrite && has && (kList || p.seg_off != nullptr)) ? __ldg(p.run_off + j) : 0;
            int32_t f = 0;         // entries in this lane's row
            LinT cur_word = static_cast<LinT>(~LinT(0));
            uint32_t acc = 0;
            auto flush = [&]() {
                __syncwarp();
#pragma unroll 1
                for (int l = 0; l < 32; ++l) {
                    const int fl = __shfl_sync(0xffffffffu, f, l);
                    const int64_t ol = __shfl_sync(0xffffffffu, outp, l);
                    if (lane < fl) list[ol + lane] = sm.rows[l * kStride + lane];
                }
                __syncwarp();
                outp += f;
                f = 0;
            };
            while (true) {  // windows of segments
                const int32_t wcnt = static_cast<int32_t>(min64(kEuclidWin, p.n - ws));
                if (wcnt <= 0) break;  // unreachable for a consistent scan; keeps the loop finite
                __syncwarp();  // every lane is done with the previous window
                for (int32_t q = lane; q < wcnt; q += 32) load_record(p.segs, ws + q, sm.recs + 6 * q);
                for (int32_t q = lane; q <= wcnt; q += 32) sm.offs[q] = __ldg(p.offsets + ws + q);
                __syncwarp();
                const int64_t wend = sm.offs[wcnt];  // the first sample beyond the window
                // passes over the window, the lanes in step at the top of each: the
                // lanes that need a segment enter it together, then each walks the
                // rest of its segment part (a list run at most until its row is full)
#pragma unroll 1
                while (true) {
                    if (i < n_i && !in_seg && g0 + i < wend) {  // enter the segment of sample g0 + i
                        const int64_t r = g0 + i;
                        const int32_t jj = find_in_window64(sm.offs, wcnt, r);
                        const int64_t sb = sm.offs[jj];
                        const int32_t N = static_cast<int32_t>(sm.offs[jj + 1] - sb) - 1;
                        const int32_t k0 = static_cast<int32_t>(r - sb);
                        cur = ws + jj;
                        i_end = static_cast<int32_t>(min64(sm.offs[jj + 1] - g0, n_i));
                        const int32_t *rec = sm.recs + 6 * jj;
                        if (k0 == 0) {
                            st.enter_n(rec, N, 0, w, wh);
                            add = true;
                            // the segment's first voxel lands at the lane's next output
                            // position (a flush moves outp and f together)
                            if (kWrite && p.seg_off != nullptr) p.seg_off[cur] = outp + f;
                        } else {  // sample k0 adds a voxel when some axis moved from sample k0 - 1
                            st.enter_n(rec, N, k0 - 1, w, wh);
                            add = st.template step<kList, kMask>();
                        }
                        in_seg = true;
                    }
                    int32_t m = in_seg ? i_end - i : 0;  // samples left in this segment part
                    if constexpr (kList) m = min(m, kRow - f);  // one row entry per sample at most
                    // the next sample's flag comes from each step (a step past the
                    // segment's end is discarded: the next segment is entered afresh)
                    if constexpr (kMask) {
#pragma unroll 4
                        for (int32_t e = 0; e < m; ++e) {
                            if (add) {
                                if constexpr (kList) row[f++] = st.P;
                                const LinT word = st.L >> 5;
                                if (word != cur_word) {
                                    if (acc) red_or_keep(p.mask + cur_word, acc, keep_policy);
                                    cur_word = word;
                                    acc = 0;
                                }
                                acc |= 1u << (static_cast<uint32_t>(st.L) & 31u);
                            }
                            add = st.template step<kList, kMask>();
                        }
                    } else if constexpr (kList) {
                        // the slot at f is written every sample and kept when the
                        // sample adds (f < kRow throughout: m is capped by the room)
#pragma unroll 4
                        for (int32_t e = 0; e < m; ++e) {
                            row[f] = st.P;
                            f += add ? 1 : 0;
                            add = st.template step<kList, kMask>();
                        }
                    } else {
#pragma unroll 4
                        for (int32_t e = 0; e < m; ++e) {
                            cnt += add ? 1 : 0;
                            add = st.template step<kList, kMask>();
                        }
                    }
                    i += m;
                    if (in_seg && i == i_end) in_seg = false;  // the next sample starts the next segment
                    if constexpr (kList) {
                        if (__any_sync(0xffffffffu, f == kRow)) flush();
                    }
                    // another pass while some lane can go on in this window
                    const bool more = i < n_i && (in_seg || g0 + i < wend);
                    if (!__any_sync(0xffffffffu, more)) break;
                }
                // every lane is done or waits for a segment beyond this window
                if (!__any_sync(0xffffffffu, i < n_i)) break;
                ws += wcnt;
            }
            if constexpr (kList) flush();
            if (kMask && acc) red_or_keep(p.mask + cur_word, acc, keep_policy);
        }
        if (!kWrite && j < p.n_runs) p.run_count[j] = cnt;
    }
}

}  // namespace vox
