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
//   k_euclid_runs<false>  voxels added per run
//   k_scan<false>         exclusive scan of the run counts (output positions)
//   k_euclid_runs<true>   the voxels, written compacted at their run's position
//                         (and OR-ed into the volume, per-voxel atomics)
#pragma once

#include <cstdint>

#include "vox_device.cuh"
#include "vox_kernels.cuh"

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

// The list writer: like the write pass of k_euclid_runs, but a warp takes 32
// consecutive runs (one per lane) and walks them in lock step (every run has L
// samples, the last ones fewer), each lane appending its voxels to its own row
// of a shared-memory stage; whenever a row fills, the warp flushes every row,
// row by row, with coalesced stores at the rows' list positions. Segment offsets
// and (optionally) the volume's atomics are written on the way. Stage entries per
// lane: 32 for 32-bit lists (one store instruction per row when it is full), 16
// for 64-bit ones (the stage stays within 48 KB).
template <typename PackT>
__host__ __device__ constexpr int euclid_row() { return sizeof(PackT) == 4 ? 32 : 16; }

template <int OUT, bool LIN64>
__global__ void __launch_bounds__(256) k_euclid_list(EuclidParams p)
{
    using PackT = typename std::conditional<(OUT & kOutList64) != 0, uint64_t, uint32_t>::type;
    using LinT = typename std::conditional<LIN64, uint64_t, uint32_t>::type;
    constexpr bool kMask = (OUT & kOutMask) != 0;
    constexpr int kRow = euclid_row<PackT>();
    constexpr int kStride = kRow + 1;  // padded rows: lanes at equal fill hit different banks
    __shared__ PackT stage[8][32 * kStride];
    if (ld_volatile_i32(p.status) != 0) return;
    if (__ldg(p.run_off + p.n_runs) > p.capacity) {
        if (blockIdx.x == 0 && threadIdx.x == 0) set_status(p.status, kStCapacity);
        return;
    }
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    PackT *const rows = stage[wib];
    PackT *const row = rows + lane * kStride;
    const int64_t Vs = __ldg(p.offsets + p.n);
    const int64_t L = max(kEuclidMinRun, (Vs + p.n_runs - 1) / p.n_runs);
    uint64_t keep_policy = 0;
    if (kMask) asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(keep_policy));
    const LinT w = static_cast<LinT>(p.w);
    const LinT wh = static_cast<LinT>(p.w) * static_cast<LinT>(p.h);
    PackT *const list = static_cast<PackT *>(p.list);
    const int64_t warps = static_cast<int64_t>(gridDim.x) * (blockDim.x / 32);
    for (int64_t jw = (static_cast<int64_t>(blockIdx.x) * (blockDim.x / 32) + wib) * 32; jw < p.n_runs;
         jw += warps * 32) {
        const int64_t j = jw + lane;
        const int64_t g0 = j * L;
        const bool has = j < p.n_runs && g0 < Vs;
        const int64_t g1 = has ? min(g0 + L, Vs) : g0;
        int64_t s = 0, seg_end = 0, outp = 0;
        int32_t rec[6] = {0, 0, 0, 0, 0, 0};
        EuclidStepper<PackT, LinT> st;
        bool add = false, first = false;
        if (has) {
            int64_t lo = 0, hi = p.n;
            while (hi - lo > 1) {
                const int64_t mid = (lo + hi) >> 1;
                if (__ldg(p.offsets + mid) <= g0) lo = mid;
                else hi = mid;
            }
            s = lo;
            const int64_t seg_begin = __ldg(p.offsets + s);
            seg_end = __ldg(p.offsets + s + 1);
            load_record(p.segs, s, rec);
            const int32_t N = static_cast<int32_t>(seg_end - seg_begin - 1);
            const int32_t k0 = static_cast<int32_t>(g0 - seg_begin);
            if (k0 == 0) {
                st.enter_n(rec, N, 0, w, wh);
                add = first = true;
            } else {
                st.enter_n(rec, N, k0 - 1, w, wh);
                add = st.template step<true, kMask>();
            }
            outp = __ldg(p.run_off + j);
        }
        // samples g0 + i, i < n_i (below 2^31, as in k_euclid_runs)
        const int32_t n_i = static_cast<int32_t>(g1 - g0);
        int32_t i_end = static_cast<int32_t>(seg_end - g0);
        int f = 0;
        LinT cur_word = static_cast<LinT>(~LinT(0));
        uint32_t acc = 0;
        auto flush = [&]() {
#pragma unroll 1
            for (int l = 0; l < 32; ++l) {
                const int fl = __shfl_sync(0xffffffffu, f, l);
                const int64_t ol = __shfl_sync(0xffffffffu, outp, l);
                if (lane < fl) list[ol + lane] = rows[l * kStride + lane];
            }
            __syncwarp();
            outp += f;
            f = 0;
        };
        const int32_t n_it = static_cast<int32_t>(L);
#pragma unroll 1
        for (int32_t i = 0; i < n_it; ++i) {
            if (i < n_i) {
                if (i == i_end) {  // the next segment starts here
                    ++s;
                    const int64_t next_end = __ldg(p.offsets + s + 1);
                    const int32_t N = static_cast<int32_t>(next_end - seg_end) - 1;
                    seg_end = next_end;
                    i_end = static_cast<int32_t>(seg_end - g0);
                    load_record(p.segs, s, rec);
                    st.enter_n(rec, N, 0, w, wh);
                    add = first = true;
                }
                if (add) {
                    if (first && p.seg_off != nullptr) p.seg_off[s] = outp + f;
                    row[f++] = st.P;
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
                first = false;
                if (i + 1 < i_end) add = st.template step<true, kMask>();
            }
            __syncwarp();
            if (__any_sync(0xffffffffu, f == kRow)) flush();
        }
        __syncwarp();
        flush();
        if (kMask && acc) red_or_keep(p.mask + cur_word, acc, keep_policy);
    }
}

}  // namespace vox
