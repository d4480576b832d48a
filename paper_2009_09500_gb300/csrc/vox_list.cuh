// vox_list.cuh -- the packed voxel list by warp slices and TMA bulk stores (sm_103a).
//
// The list of Fig. 3 / Section 4 (every voxel of every segment, in segment order,
// at offsets[s] + k) is written by warps that own slices of kListSlice = 32 x 33
// consecutive global voxel ids. Lane l of a warp takes the run of kListRun = 33
// voxels starting at slice position 33 l and steps through it with the exact
// carry recurrence of Eq. (3) (vox_device.cuh), entering its first segment by one
// division per minor axis and the following ones at k = 0. The voxels go to a
// per-warp stage in shared memory in their final (linear) order: with an odd run
// length, lane l's u-th voxel sits at word 33 l + u, bank (l + u) mod 32, so the
// 32 lanes' stores never collide (64-bit voxels: two lanes per bank pair, the
// minimum for 256 bytes). The finished slice leaves with one TMA bulk copy from
// shared to global memory (cp.async.bulk), so the SM issues no load/store
// instructions for the write-out and no CTA-wide barrier: each warp runs on its
// own, taking chunks of slices from a global work counter (one atomic and one
// search in the offsets per chunk; 1 to 16 slices per chunk, about eight chunks
// per warp, so that short lists still spread evenly).
//
// A slice with few segment ends inside it (kListFlatMax at most, counted in the
// staged window) is walked by the lanes in step over their runs: four voxels at
// a time while no lane is within four voxels of its segment's or run's end (one
// vote per four voxels), else one voxel, a voxel that ends its segment being
// followed in place by the next segment's first voxel (entered at k = 0, no
// division); the few lanes that cross a segment end hold the others up only for
// that entry. A slice with many ends is walked part by part (one part per
// segment), so that the lanes' entries happen together instead of one after
// another.
//
// Segment records and offsets are staged per warp in windows of 32 segments
// (plain coalesced loads into the warp's shared memory) and kept for the next
// slice of the chunk while at least 16 of the window's segments lie ahead of
// it; a slice that spans more segments is processed in several windows, each
// lane keeping its stepping state across them.
#pragma once

#include <cstdint>
#include <type_traits>

#include "vox_bricks.cuh"
#include "vox_device.cuh"
#include "vox_kernels.cuh"

namespace vox {

constexpr int kListRun = 33;                   // voxels per lane run (odd)
constexpr int kListSlice = 32 * kListRun;      // voxels per warp slice (1056, a multiple of 4)
constexpr int kListWarps = 4;                  // warps per CTA
constexpr int kListThreads = 32 * kListWarps;
constexpr int kListWin = 32;                   // segments per staged window
constexpr int kListChunkMax = 16;              // slices per fetch from the work counter, at most
constexpr int kListChunksPerWarp = 8;          // chunks per warp aimed at (for balance)
constexpr int kListFlatMax = 12;                // segment ends per slice up to which runs cross them in place
static_assert(kListSlice % 4 == 0, "slices must keep 16-byte aligned list addresses");

struct ListParams {
    const int32_t *segs;     // [n][6]
    int64_t n;
    const int64_t *offsets;  // [n + 1] exclusive offsets (workspace), offsets[n] = V
    void *list;              // uint32 or uint64 list, 16-byte aligned
    int64_t capacity;
    int32_t *status;
    uint32_t *counter;       // chunk counter, zeroed before the launch
};

template <typename PackT>
struct ListWarpSmem {
    alignas(16) PackT stage[kListSlice];   // the slice's voxels in list order (bulk-copy source)
    int64_t offs[kListWin + 1];            // offsets of the window's segments (+ the next)
    int32_t recs[kListWin * 6];            // the window's segment records
};
static_assert(sizeof(ListWarpSmem<uint32_t>) % 16 == 0 && sizeof(ListWarpSmem<uint64_t>) % 16 == 0,
              "per-warp regions keep the stage 16-byte aligned");

// Largest s in [0, n) with offsets[s] <= g (offsets[0] <= g < offsets[n]): a
// 32-ary search in which every lane probes one position per round; called by
// the whole warp with the same arguments.
__device__ __forceinline__ int64_t warp_find_segment(const int64_t *offsets, int64_t n, int64_t g, int lane)
{
    int64_t lo = 0, hi = n;
    while (hi - lo > 1) {
        const int64_t stride = (hi - lo + 31) / 32;
        const int64_t pos = lo + static_cast<int64_t>(lane) * stride;
        const bool le = pos < hi && __ldg(offsets + pos) <= g;
        const int cnt = __popc(__ballot_sync(0xffffffffu, le));  // probes 0 .. cnt-1 hold (monotone)
        const int64_t base = lo;
        lo = base + static_cast<int64_t>(cnt - 1) * stride;
        hi = min(hi, base + static_cast<int64_t>(cnt) * stride);
    }
    return lo;
}

// Largest j in [0, cnt) with offs[j] <= r, given offs[0] <= r < offs[cnt], cnt <= 32.
__device__ __forceinline__ int32_t find_in_window32(const int64_t *offs, int32_t cnt, int64_t r)
{
    int32_t lo = 0;
#pragma unroll
    for (int32_t step = 16; step > 0; step >>= 1) {
        const int32_t m = lo + step;
        if (m < cnt && offs[m] <= r) lo = m;
    }
    return lo;
}

template <typename PackT>
__global__ void __launch_bounds__(kListThreads) k_list(ListParams p)
{
    extern __shared__ __align__(16) unsigned char list_smem_raw[];
    __shared__ int32_t s_go;
    __shared__ int64_t s_V;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    ListWarpSmem<PackT> &sm = reinterpret_cast<ListWarpSmem<PackT> *>(list_smem_raw)[warp];

    // prologue decided by one thread so that the whole CTA agrees
    if (threadIdx.x == 0) {
        int32_t go = ld_volatile_i32(p.status) == 0;  // an earlier error: write nothing
        const int64_t V = __ldg(p.offsets + p.n);
        if (go && V > p.capacity) {
            set_status(p.status, kStCapacity);
            go = 0;
        }
        s_go = go;
        s_V = V;
    }
    __syncthreads();
    if (!s_go) return;
    const int64_t V = s_V;
    PackT *const list = static_cast<PackT *>(p.list);
    const int64_t n_slices = (V + kListSlice - 1) / kListSlice;
    const int64_t n_warps = static_cast<int64_t>(gridDim.x) * kListWarps;
    const int64_t chunk_slices = max64(1, min64(kListChunkMax, n_slices / (n_warps * kListChunksPerWarp)));
    const int64_t kChunk = chunk_slices * kListSlice;
    bool pending = false;  // lane 0: a bulk store may still be reading this warp's stage

    while (true) {
        uint32_t c = 0;
        if (lane == 0) c = atomicAdd(p.counter, 1u);
        c = __shfl_sync(0xffffffffu, c, 0);
        const int64_t g_begin = static_cast<int64_t>(c) * kChunk;
        if (g_begin >= V) break;
        const int64_t g_end = min64(g_begin + kChunk, V);
        int64_t s = warp_find_segment(p.offsets, p.n, g_begin, lane);
        int64_t ws_keep = -1;   // the staged window of the previous slice
        int32_t wcnt_keep = 0;
        for (int64_t g = g_begin; g < g_end; g += kListSlice) {
            const int32_t len = static_cast<int32_t>(min64(kListSlice, g_end - g));
            const int32_t my0 = kListRun * lane;
            const int32_t rlen = max(0, min(kListRun, len - my0));
            if (lane == 0 && pending) bulk_wait_read_all();  // the stage is free again
            __syncwarp();

            Stepper<PackT, uint32_t> st;
            int32_t done = 0;
            int64_t cur = -1;   // the segment being walked (-1: not found yet)
            int32_t kin = 0;    // step at which to enter it
            bool live = false;  // stepping state valid for cur
            bool ended = false; // the last voxel written ended its segment
            // keep the previous slice's window while 16 of its segments lie ahead
            bool staged = ws_keep >= 0 && s >= ws_keep && s + kListWin / 2 <= ws_keep + wcnt_keep;
            int64_t ws = staged ? ws_keep : s;  // first segment of the window
            while (__any_sync(0xffffffffu, done < rlen)) {
                const int32_t wcnt = staged ? wcnt_keep : static_cast<int32_t>(min64(kListWin, p.n - ws));
                __syncwarp();  // every lane is done with the previous window
                if (!staged) {
                    const int64_t sj = ws + lane;
                    if (lane < wcnt) {
                        const int2 *r = reinterpret_cast<const int2 *>(p.segs + 6 * sj);
                        const int2 a = __ldg(r), b = __ldg(r + 1), e = __ldg(r + 2);
                        int32_t *d = sm.recs + 6 * lane;
                        d[0] = a.x; d[1] = a.y; d[2] = b.x; d[3] = b.y; d[4] = e.x; d[5] = e.y;
                    }
                    if (lane <= wcnt) sm.offs[lane] = __ldg(p.offsets + sj);
                    if (lane == 0 && wcnt == kListWin) sm.offs[kListWin] = __ldg(p.offsets + ws + kListWin);
                }
                __syncwarp();
                // segment ends inside the slice that this window holds: with few, the
                // lanes cross them in one loop over their runs (entering the next
                // segment in place); with many, a loop per segment part keeps the
                // entries together
                const bool flat = __popc(__ballot_sync(0xffffffffu, lane >= 1 && lane <= wcnt && sm.offs[lane] > g &&
                                                                         sm.offs[lane] < g + len)) <= kListFlatMax;
                if (done < rlen && cur < 0) {  // the segment of the run's first voxel, if in this window
                    const int64_t r = g + my0;
                    if (r < sm.offs[wcnt]) {
                        const int32_t j = find_in_window32(sm.offs, wcnt, r);
                        cur = ws + j;
                        kin = static_cast<int32_t>(r - sm.offs[j]);
                    }
                }
                // the flat walk's votes need every lane: flat is the same for the whole warp
                if (flat) {
                    // the lanes walk in step: four voxels at once while no walking
                    // lane is within four voxels of its segment's or run's end,
                    // else one voxel, a segment end crossed in place
                    bool go = cur >= 0 && done < rlen && cur < ws + wcnt;  // walks in this window
                    if (go && !live) {
                        st.enter(sm.recs + 6 * static_cast<int32_t>(cur - ws), kin, 0u, 0u);
                        live = true;
                    }
                    int32_t left = go ? st.left : 0;  // voxels after this one in its segment
                    int32_t u = done;
                    while (__any_sync(0xffffffffu, go)) {
                        if (__all_sync(0xffffffffu, !go || (left >= 4 && u + 4 <= rlen))) {
                            if (go) {
#pragma unroll
                                for (int v = 0; v < 4; ++v) {
                                    sm.stage[my0 + u + v] = st.P;
                                    st.template step<true, false>();
                                }
                                u += 4;
                                left -= 4;
                                ended = false;
                                go = u < rlen;
                            }
                            continue;
                        }
                        if (go) {
                            sm.stage[my0 + u] = st.P;
                            ended = (left == 0);
                            ++u;
                            if (!ended) {
                                --left;
                                st.template step<true, false>();
                                go = u < rlen;
                            } else if (u == rlen) {  // the run ends with its segment
                                go = false;
                            } else {                 // the run goes on in the next segment
                                ++cur;
                                kin = 0;
                                live = false;
                                if (cur >= ws + wcnt) {  // ... which a later window holds
                                    go = false;
                                } else {
                                    st.enter(sm.recs + 6 * static_cast<int32_t>(cur - ws), 0, 0u, 0u);
                                    live = true;
                                    left = st.left;
                                }
                            }
                        }
                    }
                    done = u;
                } else if (done < rlen) {
                    PackT *o = sm.stage + my0 + done;
                    while (cur >= 0 && done < rlen && cur < ws + wcnt) {
                        if (!live) {
                            st.enter(sm.recs + 6 * static_cast<int32_t>(cur - ws), kin, 0u, 0u);
                            live = true;
                        }
                        const int32_t m = min(st.left + 1, rlen - done);
                        ended = (m == st.left + 1);
                        int32_t e = 0;
                        for (; e + 4 <= m; e += 4) {
#pragma unroll
                            for (int v = 0; v < 4; ++v) {
                                o[v] = st.P;
                                st.template step<true, false>();
                            }
                            o += 4;
                        }
                        for (; e < m; ++e) {
                            *o++ = st.P;
                            st.template step<true, false>();
                        }
                        done += m;
                        if (done < rlen) {  // the run goes on in the next segment
                            ++cur;
                            kin = 0;
                            live = false;
                        }
                    }
                }
                ws_keep = ws;
                wcnt_keep = wcnt;
                staged = false;  // a further round stages the next window
                if (__any_sync(0xffffffffu, done < rlen)) {
                    ws += wcnt;
                    if (wcnt == 0) break;  // unreachable for a consistent scan; keeps the loop finite
                }
            }
            // the next slice starts in the segment of this slice's last voxel, or
            // the next one if that voxel ended its segment
            const int last = (len - 1) / kListRun;
            const int64_t cur_last = __shfl_sync(0xffffffffu, cur, last);
            const bool ended_last = __shfl_sync(0xffffffffu, ended ? 1 : 0, last) != 0;
            s = cur_last + (ended_last ? 1 : 0);

            // write-out: the 16-byte part by one bulk copy, a ragged end (only at
            // the end of the list) by plain stores
            fence_proxy_async_smem();  // this lane's stage writes, visible to the bulk-copy unit
            __syncwarp();
            const uint32_t bytes = (static_cast<uint32_t>(len) * sizeof(PackT)) & ~15u;
            if (lane == 0 && bytes) {
                bulk_store_1d(list + g, sm.stage, bytes);
                pending = true;
            }
            const int32_t tail0 = static_cast<int32_t>(bytes / sizeof(PackT));
            for (int32_t e = tail0 + lane; e < len; e += 32) list[g + e] = sm.stage[e];
        }
    }
    if (lane == 0 && pending) bulk_wait_all();  // copies complete before the CTA's memory goes
}

}  // namespace vox
