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


// Stepping state with the Euclidean N: no axis moves every step, so all three
// carry (remainder r_a = (2 k A_a + N) mod 2N, the offset growing when it wraps).
template <typename PackT, typename LinT>
struct EuclidStepper {
    int32_t twoN;
    int32_t A2[3], r[3];
    PackT P, dP[3];
    LinT L, dL[3];

    __device__ __forceinline__ void enter(const int32_t *rec, int32_t k, LinT w, LinT wh)
    {
        const int32_t N = euclid_steps(rec);
        twoN = 2 * N;
        int32_t v[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const int32_t d = rec[3 + a] - rec[a];
            const int32_t A = abs(d);
            int32_t q = 0, rr = N;
            if (k > 0) axis_entry(A, N, k, q, rr);
            r[a] = rr;
            A2[a] = 2 * A;
            v[a] = rec[a] + (d >= 0 ? q : -q);
            dP[a] = signed_step<PackT>(d, pack_unit<PackT>(a));
            dL[a] = signed_step<LinT>(d, a == 0 ? LinT(1) : (a == 1 ? w : wh));
        }
        P = static_cast<PackT>(v[0]) | (static_cast<PackT>(v[1]) * pack_unit<PackT>(1)) |
            (static_cast<PackT>(v[2]) * pack_unit<PackT>(2));
        L = static_cast<LinT>(v[0]) + static_cast<LinT>(v[1]) * w + static_cast<LinT>(v[2]) * wh;
    }

    // Advance one sample; true when the voxel changed (some axis moved).
    template <bool kP, bool kL>
    __device__ __forceinline__ bool step()
    {
        bool moved = false;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            r[a] += A2[a];
            if (r[a] >= twoN) {
                r[a] -= twoN;
                if (kP) P += dP[a];
                if (kL) L += dL[a];
                moved = true;
            }
        }
        return moved;
    }
};

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
        const int32_t k0 = static_cast<int32_t>(g0 - __ldg(p.offsets + s));
        EuclidStepper<PackT, LinT> st;
        bool add, first;
        if (k0 == 0) {
            st.enter(rec, 0, w, wh);
            add = first = true;
        } else {  // sample k0 adds a voxel when some axis moved from sample k0 - 1
            st.enter(rec, k0 - 1, w, wh);
            add = st.template step<kWrite && kList, kWrite && kMask>();
            first = false;
        }
        const int64_t base = kWrite ? __ldg(p.run_off + j) : 0;
        int32_t cnt = 0;
        LinT cur_word = static_cast<LinT>(~LinT(0));
        uint32_t acc = 0;
        for (int64_t g = g0; g < g1; ++g) {
            if (g == seg_end) {  // the next segment starts here
                ++s;
                seg_end = next_end;
                rec[0] = na.x; rec[1] = na.y; rec[2] = nb.x; rec[3] = nb.y; rec[4] = nc.x; rec[5] = nc.y;
                prefetch(s);
                st.enter(rec, 0, w, wh);
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
            if (g + 1 < seg_end) add = st.template step<kWrite && kList, kWrite && kMask>();
        }
        if (kWrite && kMask && acc) red_or_keep(p.mask + cur_word, acc, keep_policy);
        if (!kWrite) p.run_count[j] = cnt;
    }
}

}  // namespace vox
