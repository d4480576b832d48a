// vox.cu -- the C ABI of libvox (declared in include/vox.h): argument checks,
// workspace layout, kernel selection and launches. Host code only calls the
// CUDA runtime for launches, stream-ordered memsets/copies and device queries;
// it allocates no device memory.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdint>
#include <cstring>
#include <map>
#include <mutex>
#include <utility>

#include "vox.h"
#include "vox_bricks.cuh"
#include "vox_kernels.cuh"
#include "vox_euclid.cuh"
#include "vox_list.cuh"

namespace {

using namespace vox;

constexpr size_t kWsAlign = 256;
constexpr int64_t kMaxDim = int64_t(1) << 21;
constexpr int64_t kMinPerCta = 2048;          // smallest voxel range given to one CTA
constexpr int64_t kDefaultWaitNs = 500000000;  // 0.5 s bound on every in-kernel wait
constexpr size_t kListCounterOffset = 128;    // k_list's chunk counter, in the workspace's ticket region

std::atomic<int64_t> g_stall_tile{-1};
std::atomic<int64_t> g_wait_ns{kDefaultWaitNs};

std::mutex g_tuning_mu;
vox_tuning g_tuning{0, 0, 0, 0};

vox_tuning current_tuning()
{
    std::lock_guard<std::mutex> lock(g_tuning_mu);
    return g_tuning;
}

size_t align_up(size_t x) { return (x + kWsAlign - 1) & ~(kWsAlign - 1); }

struct WsLayout {
    int64_t n_tiles;
    size_t desc;     // uint64 [n_tiles]; the ticket sits at byte 0
    size_t offsets;  // int64 [n + 4]
    size_t total;
};

WsLayout ws_layout(int64_t n)
{
    WsLayout L;
    L.n_tiles = (n + kScanTile - 1) / kScanTile;
    L.desc = kWsAlign;
    L.offsets = L.desc + align_up(sizeof(uint64_t) * static_cast<size_t>(L.n_tiles > 0 ? L.n_tiles : 1));
    L.total = L.offsets + align_up(sizeof(int64_t) * static_cast<size_t>(n + 4));
    return L;
}

bool aligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0; }

vox_status check_dims(vox_dims dims)
{
    if (dims.w < 1 || dims.h < 1 || dims.d < 1) return VOX_ERR_INVALID_ARG;
    if (dims.w > kMaxDim || dims.h > kMaxDim || dims.d > kMaxDim) return VOX_ERR_INVALID_ARG;
    return VOX_OK;
}

uint64_t volume_bits(vox_dims d)
{
    return static_cast<uint64_t>(d.w) * static_cast<uint64_t>(d.h) * static_cast<uint64_t>(d.d);
}

int sm_count()
{
    static std::mutex mu;
    static std::map<int, int> cache;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find(dev);
    if (it != cache.end()) return it->second;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    cache[dev] = sms;
    return sms;
}

int blocks_per_sm(const void *kernel, int threads, size_t smem)
{
    static std::mutex mu;
    static std::map<std::pair<const void *, int>, int> cache;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    std::lock_guard<std::mutex> lock(mu);
    auto key = std::make_pair(kernel, dev);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, threads, smem) != cudaSuccess) return 0;
    cache[key] = b;
    return b;
}

// Opt a kernel in to `smem` bytes of dynamic shared memory (above the 48 KB
// default), once per kernel and device.
vox_status allow_smem(const void *kernel, size_t smem)
{
    static std::mutex mu;
    static std::map<std::pair<const void *, int>, bool> done;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return VOX_ERR_CUDA;
    std::lock_guard<std::mutex> lock(mu);
    auto key = std::make_pair(kernel, dev);
    if (done.count(key)) return VOX_OK;
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)) !=
        cudaSuccess)
        return VOX_ERR_CUDA;
    done[key] = true;
    return VOX_OK;
}

bool make_geom(vox_dims dims, BrickGeom *G);

// Host-side checks shared by the generation entry points.
vox_status check_generate_args(const vox_segment *segs, int64_t n, vox_dims dims, const void *list,
                               int64_t capacity, const uint32_t *mask, int flags, const void *ws,
                               size_t ws_bytes, const int32_t *status)
{
    if (n < 0 || status == nullptr) return VOX_ERR_INVALID_ARG;
    if (n > 0 && segs == nullptr) return VOX_ERR_INVALID_ARG;
    if (vox_status e = check_dims(dims)) return e;
    if (flags & ~(VOX_OUT_LIST32 | VOX_OUT_LIST64 | VOX_OUT_BITMASK | VOX_OUT_FRESH | VOX_OUT_BRICKED))
        return VOX_ERR_INVALID_ARG;
    const bool l32 = flags & VOX_OUT_LIST32, l64 = flags & VOX_OUT_LIST64, bm = flags & VOX_OUT_BITMASK;
    if (!(l32 || l64 || bm) || (l32 && l64)) return VOX_ERR_INVALID_ARG;
    if ((flags & (VOX_OUT_FRESH | VOX_OUT_BRICKED)) && !bm) return VOX_ERR_INVALID_ARG;
    if (flags & VOX_OUT_BRICKED) {  // the layout exists only with a brick geometry
        BrickGeom G;
        if (!make_geom(dims, &G)) return VOX_ERR_INVALID_ARG;
        if (mask != nullptr && !aligned(mask, 16)) return VOX_ERR_ALIGNMENT;
    }
    if (l32 && (dims.w > 1024 || dims.h > 1024 || dims.d > 1024)) return VOX_ERR_PACK_WIDTH;
    if ((l32 || l64) && (list == nullptr || capacity < 0)) return VOX_ERR_INVALID_ARG;
    if (bm && mask == nullptr) return VOX_ERR_INVALID_ARG;
    if (n > 0 && !aligned(segs, 16)) return VOX_ERR_ALIGNMENT;
    if ((l32 || l64) && !aligned(list, 16)) return VOX_ERR_ALIGNMENT;
    if (bm && !aligned(mask, 4)) return VOX_ERR_ALIGNMENT;
    if (ws == nullptr || !aligned(ws, kWsAlign) || ws_bytes < ws_layout(n).total) return VOX_ERR_WORKSPACE;
    return VOX_OK;
}

// ---- the volume by brick ownership ------------------------------------------

// The brick geometry of a single volume (brick_geom, with counter replicas).
bool make_geom(vox_dims dims, BrickGeom *G)
{
    if (check_dims(dims) != VOX_OK) return false;
    return brick_geom(dims.w, dims.h, dims.d, G, true);
}

// Tensor map of the volume as a 3-D array of 32-bit words (row_words x h x d)
// with brick-sized boxes, for the TMA reduce-OR merge. Needs 16-byte aligned
// rows and box rows (w and B0 multiples of 128) and a 16-byte aligned volume.
bool make_volume_tmap(const BrickGeom &G, uint32_t *mask, CUtensorMap *out, int32_t box_z = 0)
{
    if (G.bxw % 4 != 0 || G.row_words % 4 != 0 || !aligned(mask, 16)) return false;
    static std::mutex mu;
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    {
        std::lock_guard<std::mutex> lock(mu);
        if (encode == nullptr) {
            void *fn = nullptr;
            cudaDriverEntryPointQueryResult q;
            if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                    cudaSuccess ||
                q != cudaDriverEntryPointSuccess || fn == nullptr)
                return false;
            encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
        }
    }
    const cuuint64_t dims[3] = {static_cast<cuuint64_t>(G.row_words), static_cast<cuuint64_t>(G.dim[1]),
                                static_cast<cuuint64_t>(G.dim[2])};
    const cuuint64_t strides[2] = {4ull * G.row_words, 4ull * G.row_words * static_cast<cuuint64_t>(G.dim[1])};
    const cuuint32_t box[3] = {static_cast<cuuint32_t>(G.bxw), static_cast<cuuint32_t>(G.B[1]),
                               static_cast<cuuint32_t>(box_z > 0 ? box_z : G.B[2])};
    const cuuint32_t estr[3] = {1, 1, 1};
    if (box[1] > 256 || box[2] > 256) return false;
    return encode(out, CU_TENSOR_MAP_DATA_TYPE_UINT32, 3, mask, dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

struct VolLayout {
    int64_t n_tiles;  // scan tiles over the brick counts
    size_t hdr;       // scan ticket at +0, brick ticket at +128
    size_t count;     // int32 [n_slots]
    size_t desc;      // uint64 [n_tiles]
    size_t off;       // int64 [n_slots + 4]
    size_t cursor;    // int64 [n_slots + 1]
    size_t pieces;    // uint64 [capacity]
    size_t total;
};

// ---- the Euclidean-N variant ---------------------------------------------------
// Workspace: the count + scan layout of the samples, then the run arrays.
struct EuclidLayout {
    int64_t n_runs;   // run slots
    int64_t n_tiles;  // scan tiles over the run counts
    size_t hdr;       // ticket of the run scan
    size_t count;     // int32 [n_runs]
    size_t desc;      // uint64 [n_tiles]
    size_t off;       // int64 [n_runs + 4]
    size_t total;
};

EuclidLayout euclid_layout(int64_t n)
{
    EuclidLayout E;
    E.n_runs = std::max<int64_t>(n, kEuclidRunSlots);
    E.n_tiles = (E.n_runs + kScanTile - 1) / kScanTile;
    E.hdr = ws_layout(n).total;
    E.count = E.hdr + kWsAlign;
    E.desc = E.count + align_up(4 * static_cast<size_t>(E.n_runs));
    E.off = E.desc + align_up(8 * static_cast<size_t>(E.n_tiles));
    E.total = E.off + align_up(8 * static_cast<size_t>(E.n_runs + 4));
    return E;
}

// The volume path's workspace follows the base layout of ws_layout(n) (base 0),
// or another layout ending at `base` (the Euclidean variant's run arrays).
VolLayout vol_layout(int64_t n, const BrickGeom &G, int64_t capacity, size_t base = 0)
{
    VolLayout L;
    const size_t nb = static_cast<size_t>(G.n_slots);
    L.n_tiles = (G.n_slots + kScanTile - 1) / kScanTile;
    L.hdr = base != 0 ? base : ws_layout(n).total;
    L.count = L.hdr + kWsAlign;
    L.desc = L.count + align_up(4 * nb);
    L.off = L.desc + align_up(8 * static_cast<size_t>(L.n_tiles));
    L.cursor = L.off + align_up(8 * (nb + 4));
    L.pieces = L.cursor + align_up(8 * (nb + 1));
    L.total = L.pieces + align_up(8 * static_cast<size_t>(capacity));
    return L;
}

// Whether a call on n segments with this workspace builds the volume by brick
// ownership (the workspace holds the brick arrays and room for a piece).
// Pieces name their segment in 32 bits: beyond 2^32 segments the volume takes
// the atomics path.
bool uses_bricks(int64_t n, vox_dims dims, size_t ws_bytes, BrickGeom *G, size_t base = 0)
{
    return n > 0 && n < (int64_t(1) << 32) && make_geom(dims, G) && ws_bytes >= vol_layout(n, *G, 1, base).total;
}

int grid_ctas(const void *kernel, int threads, size_t smem);

// The binning passes: persistent grids (SMs x CTAs per SM, no more CTAs than
// the segments fill), warps taking batches of segments.
template <bool kEuclid, bool kBatched>
vox_status launch_bin_t(const BinParams &bp, bool scatter, int64_t n, cudaStream_t stream)
{
    const void *k = scatter ? reinterpret_cast<const void *>(k_bin_scatter<kEuclid, kBatched>)
                            : reinterpret_cast<const void *>(k_bin_count<kEuclid, kBatched>);
    int grid = grid_ctas(k, kBinThreads, 0);
    if (grid <= 0) return VOX_ERR_CUDA;
    grid = static_cast<int>(std::min<int64_t>(grid, (n + kBinWarps * kBinBatch - 1) / (kBinWarps * kBinBatch)));
    if (scatter) k_bin_scatter<kEuclid, kBatched><<<static_cast<unsigned>(grid), kBinThreads, 0, stream>>>(bp);
    else k_bin_count<kEuclid, kBatched><<<static_cast<unsigned>(grid), kBinThreads, 0, stream>>>(bp);
    return cudaGetLastError() == cudaSuccess ? VOX_OK : VOX_ERR_CUDA;
}

vox_status launch_bin(const BinParams &bp, bool euclid, bool batched, bool scatter, int64_t n, cudaStream_t stream)
{
    if (batched) return launch_bin_t<false, true>(bp, scatter, n, stream);
    if (euclid) return launch_bin_t<true, false>(bp, scatter, n, stream);
    return launch_bin_t<false, false>(bp, scatter, n, stream);
}

vox_status launch_bin_count(const BinParams &bp, bool euclid, bool batched, int64_t n, cudaStream_t stream)
{
    return launch_bin(bp, euclid, batched, false, n, stream);
}

vox_status launch_bin_scatter(const BinParams &bp, bool euclid, bool batched, int64_t n, cudaStream_t stream)
{
    return launch_bin(bp, euclid, batched, true, n, stream);
}

// Count + scan. With a brick workspace it also zeroes the brick arrays and
// counts every segment's pieces per brick (k_bin_count).
vox_status launch_count_scan(const vox_segment *segs, int64_t n, vox_dims dims, int32_t *counts,
                             int64_t *offsets_out, void *ws, size_t ws_bytes, int32_t *status, cudaStream_t stream,
                             const SceneDesc *scenes = nullptr, const int32_t *scene_of = nullptr,
                             int32_t n_scenes = 0, bool euclid = false)
{
    const WsLayout L = ws_layout(n);
    char *base = static_cast<char *>(ws);
    if (cudaMemsetAsync(base, 0, L.offsets, stream) != cudaSuccess) return VOX_ERR_CUDA;
    BrickGeom G;
    const size_t vbase = euclid ? euclid_layout(n).total : 0;
    const bool bins = scene_of == nullptr && uses_bricks(n, dims, ws_bytes, &G, vbase);
    VolLayout VL{};
    if (bins) {
        VL = vol_layout(n, G, 0, vbase);
        if (cudaMemsetAsync(base + VL.hdr, 0, VL.off - VL.hdr, stream) != cudaSuccess) return VOX_ERR_CUDA;
    }
    ScanParams p;
    p.segs = reinterpret_cast<const int32_t *>(segs);
    p.counts_in = nullptr;
    p.offsets_copy = nullptr;
    p.n = n;
    p.w = dims.w;
    p.h = dims.h;
    p.d = dims.d;
    p.counts = counts;
    p.offsets = reinterpret_cast<int64_t *>(base + L.offsets);
    p.offsets_out = offsets_out;
    p.desc = reinterpret_cast<uint64_t *>(base + L.desc);
    p.ticket = reinterpret_cast<uint32_t *>(base);
    p.status = status;
    p.n_tiles = L.n_tiles;
    p.stall_tile = g_stall_tile.load();
    p.wait_ns = static_cast<uint64_t>(g_wait_ns.load());
    p.scenes = scenes;
    p.scene_of = scene_of;
    p.n_scenes = n_scenes;
    if (euclid) k_scan<true, true><<<static_cast<unsigned>(L.n_tiles), kScanThreads, 0, stream>>>(p);
    else k_scan<true><<<static_cast<unsigned>(L.n_tiles), kScanThreads, 0, stream>>>(p);
    if (bins) {
        BinParams bp{};
        bp.segs = p.segs;
        bp.n = n;
        bp.G = G;
        bp.brick_count = reinterpret_cast<int32_t *>(base + VL.count);
        bp.status = status;
        if (vox_status e = launch_bin_count(bp, euclid, false, n, stream)) return e;
    }
    return cudaGetLastError() == cudaSuccess ? VOX_OK : VOX_ERR_CUDA;
}

// Persistent grid: SMs x CTAs per SM (occupancy maximum, or the tuned value
// when it is smaller).
int grid_ctas(const void *kernel, int threads, size_t smem)
{
    const int per_sm = blocks_per_sm(kernel, threads, smem);
    const int sms = sm_count();
    if (per_sm <= 0 || sms <= 0) return 0;
    const vox_tuning tu = current_tuning();
    const int use = (tu.ctas_per_sm > 0 && tu.ctas_per_sm < per_sm) ? tu.ctas_per_sm : per_sm;
    return use * sms;
}

template <int R, int OUT, bool LIN64>
vox_status launch_gen_r(const GenParams &p, cudaStream_t stream)
{
    auto kernel = k_generate<R, OUT, LIN64>;
    const size_t smem = sizeof(GenSmem<R, OUT>);
    if (vox_status e = allow_smem(reinterpret_cast<const void *>(kernel), smem)) return e;
    const int grid = grid_ctas(reinterpret_cast<const void *>(kernel), kGenThreads, smem);
    if (grid <= 0) return VOX_ERR_CUDA;
    kernel<<<static_cast<unsigned>(grid), kGenThreads, smem, stream>>>(p);
    return cudaGetLastError() == cudaSuccess ? VOX_OK : VOX_ERR_CUDA;
}

template <int OUT, bool LIN64>
vox_status launch_gen_t(const GenParams &p, cudaStream_t stream)
{
    // run length: 32 voxels per thread by default; the tuning may ask for 16 or
    // 64 (64-bit lists, whose staging is twice as large, stop at 32)
    if constexpr ((OUT & kOutList64) != 0) {
        if (current_tuning().run_len == 16) return launch_gen_r<16, OUT, LIN64>(p, stream);
        return launch_gen_r<32, OUT, LIN64>(p, stream);
    } else if constexpr (OUT == kOutList32) {
        // a 32-bit list alone may cut its runs at segment ends (list_runs = 1)
        const vox_tuning tu = current_tuning();
        if (tu.list_runs == 1 && p.scene_of == nullptr) {
            if (tu.run_len == 16) return launch_gen_r<16, OUT | kOutSegRuns, LIN64>(p, stream);
            if (tu.run_len == 64) return launch_gen_r<64, OUT | kOutSegRuns, LIN64>(p, stream);
            return launch_gen_r<32, OUT | kOutSegRuns, LIN64>(p, stream);
        }
        if (tu.run_len == 16) return launch_gen_r<16, OUT, LIN64>(p, stream);
        if (tu.run_len == 64) return launch_gen_r<64, OUT, LIN64>(p, stream);
        return launch_gen_r<32, OUT, LIN64>(p, stream);
    } else if constexpr (OUT == kOutMask) {
        // the volume alone: per-lane word runs, or merged across the warp too
        const vox_tuning tu = current_tuning();
        if (tu.volume_path == VOX_VOLUME_ATOMIC_WARP) {
            if (tu.run_len == 16) return launch_gen_r<16, OUT | kOutWarpDedup, LIN64>(p, stream);
            if (tu.run_len == 64) return launch_gen_r<64, OUT | kOutWarpDedup, LIN64>(p, stream);
            return launch_gen_r<32, OUT | kOutWarpDedup, LIN64>(p, stream);
        }
        if (tu.run_len == 16) return launch_gen_r<16, OUT, LIN64>(p, stream);
        if (tu.run_len == 64) return launch_gen_r<64, OUT, LIN64>(p, stream);
        return launch_gen_r<32, OUT, LIN64>(p, stream);
    } else {
        if (current_tuning().run_len == 16) return launch_gen_r<16, OUT, LIN64>(p, stream);
        if (current_tuning().run_len == 64) return launch_gen_r<64, OUT, LIN64>(p, stream);
        return launch_gen_r<32, OUT, LIN64>(p, stream);
    }
}

// The list alone by warp slices (k_list): persistent grid, the chunk counter in
// the workspace's ticket region reset first.
template <typename PackT>
vox_status launch_list(const vox_segment *segs, int64_t n, void *list, int64_t capacity, void *ws, int32_t *status,
                       cudaStream_t stream)
{
    const WsLayout L = ws_layout(n);
    char *base = static_cast<char *>(ws);
    ListParams p;
    p.segs = reinterpret_cast<const int32_t *>(segs);
    p.n = n;
    p.offsets = reinterpret_cast<const int64_t *>(base + L.offsets);
    p.list = list;
    p.capacity = capacity;
    p.status = status;
    p.counter = reinterpret_cast<uint32_t *>(base + kListCounterOffset);
    auto kernel = k_list<PackT>;
    const size_t smem = sizeof(ListWarpSmem<PackT>) * kListWarps;
    if (vox_status e = allow_smem(reinterpret_cast<const void *>(kernel), smem)) return e;
    const int grid = grid_ctas(reinterpret_cast<const void *>(kernel), kListThreads, smem);
    if (grid <= 0) return VOX_ERR_CUDA;
    if (cudaMemsetAsync(p.counter, 0, sizeof(uint32_t), stream) != cudaSuccess) return VOX_ERR_CUDA;
    kernel<<<static_cast<unsigned>(grid), kListThreads, smem, stream>>>(p);
    return cudaGetLastError() == cudaSuccess ? VOX_OK : VOX_ERR_CUDA;
}

vox_status launch_generate(const vox_segment *segs, int64_t n, vox_dims dims, void *list, int64_t capacity,
                           uint32_t *mask, int flags, void *ws, int32_t *status, cudaStream_t stream,
                           const int64_t *gate_total = nullptr, int64_t gate_cap = 0,
                           const SceneDesc *scenes = nullptr, const int32_t *scene_of = nullptr,
                           int32_t n_scenes = 0)
{
    if (n == 0) return VOX_OK;
    const WsLayout L = ws_layout(n);
    GenParams p;
    p.segs = reinterpret_cast<const int32_t *>(segs);
    p.n = n;
    p.offsets = reinterpret_cast<const int64_t *>(static_cast<char *>(ws) + L.offsets);
    p.w = dims.w;
    p.h = dims.h;
    p.d = dims.d;
    p.list = list;
    p.capacity = capacity;
    p.mask = mask;
    p.status = status;
    p.wait_ns = static_cast<uint64_t>(g_wait_ns.load());
    p.min_per_cta = kMinPerCta;
    p.gate_total = gate_total;
    p.gate_cap = gate_cap;
    p.scenes = scenes;
    p.scene_of = scene_of;
    p.n_scenes = n_scenes;
    p.interleave = scene_of != nullptr ? 1 : 0;
    // batched volumes may differ in size: 64-bit bit indices cover them all
    const bool lin64 = scene_of != nullptr || volume_bits(dims) > (uint64_t(1) << 32);
    const bool bm = flags & VOX_OUT_BITMASK;
    if (!bm && current_tuning().list_runs == 2) {  // a list alone by warp slices
        if (flags & VOX_OUT_LIST32) return launch_list<uint32_t>(segs, n, list, capacity, ws, status, stream);
        if (flags & VOX_OUT_LIST64) return launch_list<uint64_t>(segs, n, list, capacity, ws, status, stream);
    }
    if (flags & VOX_OUT_LIST32) {
        return bm ? launch_gen_t<kOutList32 | kOutMask, false>(p, stream) : launch_gen_t<kOutList32, false>(p, stream);
    }
    if (flags & VOX_OUT_LIST64) {
        if (!bm) return launch_gen_t<kOutList64, false>(p, stream);
        return lin64 ? launch_gen_t<kOutList64 | kOutMask, true>(p, stream)
                     : launch_gen_t<kOutList64 | kOutMask, false>(p, stream);
    }
    return lin64 ? launch_gen_t<kOutMask, true>(p, stream) : launch_gen_t<kOutMask, false>(p, stream);
}

// bin -> scan -> scatter -> per-brick volume, then the atomic kernel, which only
// runs if the pieces did not fit in the workspace
vox_status launch_bricks(const vox_segment *segs, int64_t n, const BrickGeom &G, vox_dims dims, uint32_t *mask,
                         void *ws, size_t ws_bytes, int32_t *status, cudaStream_t stream, bool count_only = false,
                         bool fresh = false, bool bricked = false, bool euclid = false)
{
    // the brick counts come from the count + scan (k_bin_count); the
    // tickets and look-back flags of this pass are reset here, so that the pass
    // can run again on the same counts
    const VolLayout VL = vol_layout(n, G, 0, euclid ? euclid_layout(n).total : 0);
    const int64_t capacity = static_cast<int64_t>((ws_bytes - VL.pieces) / 8);
    char *base = static_cast<char *>(ws);
    if (cudaMemsetAsync(base + VL.hdr, 0, kWsAlign, stream) != cudaSuccess) return VOX_ERR_CUDA;
    if (cudaMemsetAsync(base + VL.desc, 0, VL.off - VL.desc, stream) != cudaSuccess) return VOX_ERR_CUDA;
    BinParams bp;
    bp.segs = reinterpret_cast<const int32_t *>(segs);
    bp.n = n;
    bp.G = G;
    bp.brick_count = reinterpret_cast<int32_t *>(base + VL.count);
    bp.cursor = reinterpret_cast<int64_t *>(base + VL.cursor);
    bp.brick_off = reinterpret_cast<const int64_t *>(base + VL.off);
    bp.pieces = reinterpret_cast<uint64_t *>(base + VL.pieces);
    bp.capacity = capacity;
    bp.status = status;
    const int sms = sm_count();
    if (sms <= 0) return VOX_ERR_CUDA;
    ScanParams sp;
    sp.segs = nullptr;
    sp.counts_in = bp.brick_count;
    sp.offsets_copy = bp.cursor;
    sp.n = G.n_slots;
    sp.w = sp.h = sp.d = 0;
    sp.counts = nullptr;
    sp.offsets = reinterpret_cast<int64_t *>(base + VL.off);
    sp.offsets_out = nullptr;
    sp.desc = reinterpret_cast<uint64_t *>(base + VL.desc);
    sp.ticket = reinterpret_cast<uint32_t *>(base + VL.hdr);
    sp.status = status;
    sp.n_tiles = VL.n_tiles;
    sp.stall_tile = -1;
    sp.wait_ns = static_cast<uint64_t>(g_wait_ns.load());
    sp.scenes = nullptr;
    sp.scene_of = nullptr;
    sp.n_scenes = 0;
    k_scan<false><<<static_cast<unsigned>(VL.n_tiles), kScanThreads, 0, stream>>>(sp);
    if (count_only) return cudaGetLastError() == cudaSuccess ? VOX_OK : VOX_ERR_CUDA;
    if (vox_status e = launch_bin_scatter(bp, euclid, false, n, stream)) return e;
    BrickParams brp;
    brp.segs = bp.segs;
    brp.G = G;
    brp.brick_off = bp.brick_off;
    brp.pieces = bp.pieces;
    brp.capacity = capacity;
    brp.mask = mask;
    brp.status = status;
    brp.ticket = reinterpret_cast<uint32_t *>(base + VL.hdr + 128);
    CUtensorMap tmap;
    std::memset(&tmap, 0, sizeof(tmap));
    brp.use_tma = (!bricked && mask != nullptr && make_volume_tmap(G, mask, &tmap)) ? 1 : 0;
    brp.fresh = (fresh || bricked) ? 1 : 0;
    brp.bricked = bricked ? 1 : 0;
    const size_t bsmem = sizeof(BrickSmem);
    const void *bk = euclid ? reinterpret_cast<const void *>(k_brick_volume<true>)
                            : reinterpret_cast<const void *>(k_brick_volume<false>);
    if (vox_status e = allow_smem(bk, bsmem)) return e;
    const int bgrid = grid_ctas(bk, kBrickThreads, bsmem);
    if (bgrid <= 0) return VOX_ERR_CUDA;
    if (euclid) k_brick_volume<true><<<static_cast<unsigned>(bgrid), kBrickThreads, bsmem, stream>>>(brp, tmap);
    else k_brick_volume<false><<<static_cast<unsigned>(bgrid), kBrickThreads, bsmem, stream>>>(brp, tmap);
    if (cudaGetLastError() != cudaSuccess) return VOX_ERR_CUDA;
    if (bricked) return VOX_OK;  // no atomics fallback for the brick-major layout (pieces must fit)
    if (euclid) return VOX_OK;   // the variant's own atomics pass is the fallback (launched by the caller)
    return launch_generate(segs, n, dims, nullptr, 0, mask, VOX_OUT_BITMASK, ws, status, stream,
                           bp.brick_off + G.n_slots, capacity);
}

// All requested outputs of one scene, after the count + scan: the list by the
// voxel-parallel kernel; the volume by brick ownership when the workspace holds
// the brick arrays (vox_workspace_size_volume), else by per-voxel atomics.
vox_status launch_outputs(const vox_segment *segs, int64_t n, vox_dims dims, void *list, int64_t capacity,
                          uint32_t *mask, int flags, void *ws, size_t ws_bytes, int32_t *status, cudaStream_t stream)
{
    BrickGeom G;
    const bool bm = flags & VOX_OUT_BITMASK;
    const bool fresh = bm && (flags & VOX_OUT_FRESH);
    const bool bricked = bm && (flags & VOX_OUT_BRICKED);
    if (bricked) {  // brick-major volume: only the brick path writes it
        if (!make_geom(dims, &G)) return VOX_ERR_INVALID_ARG;
        if (n == 0) {
            if (cudaMemsetAsync(mask, 0, 4 * static_cast<size_t>(G.n_bricks) * static_cast<size_t>(G.words),
                                stream) != cudaSuccess)
                return VOX_ERR_CUDA;
            return VOX_OK;
        }
        if (!uses_bricks(n, dims, ws_bytes, &G)) return VOX_ERR_WORKSPACE;
        const int list_flags = flags & (VOX_OUT_LIST32 | VOX_OUT_LIST64);
        if (list_flags) {
            if (vox_status e = launch_generate(segs, n, dims, list, capacity, nullptr, list_flags, ws, status, stream))
                return e;
        }
        return launch_bricks(segs, n, G, dims, mask, ws, ws_bytes, status, stream, false, true, true);
    }
    const bool bricks =
        n > 0 && bm && current_tuning().volume_path == VOX_VOLUME_AUTO && uses_bricks(n, dims, ws_bytes, &G);
    if (!bricks) {
        // a fresh volume without the brick path: cleared first, then OR-ed into
        if (fresh && cudaMemsetAsync(mask, 0, 4 * static_cast<size_t>(vox_mask_words(dims)), stream) != cudaSuccess)
            return VOX_ERR_CUDA;
        if (n == 0) return VOX_OK;
        return launch_generate(segs, n, dims, list, capacity, mask, flags, ws, status, stream);
    }
    const int list_flags = flags & (VOX_OUT_LIST32 | VOX_OUT_LIST64);
    if (list_flags) {
        if (vox_status e = launch_generate(segs, n, dims, list, capacity, nullptr, list_flags, ws, status, stream))
            return e;
    }
    return launch_bricks(segs, n, G, dims, mask, ws, ws_bytes, status, stream, false, fresh);
}

// ---- batched scenes ----------------------------------------------------------
static_assert(sizeof(vox_scene) == sizeof(SceneDesc), "vox_scene and SceneDesc must match");
static_assert(offsetof(vox_scene, dims) == offsetof(SceneDesc, w) && offsetof(vox_scene, mask) == offsetof(SceneDesc, mask),
              "vox_scene and SceneDesc must match");

// Batched workspace: the single-scene layout for all segments, then the
// segment -> scene map and the per-scene voxel bases.
struct BatchLayout {
    size_t scene_of;  // int32 [n_total]
    size_t base;      // int64 [n_scenes + 1]
    size_t total;
};

BatchLayout batch_layout(int64_t n_total, int32_t n_scenes)
{
    BatchLayout B;
    B.scene_of = ws_layout(n_total).total;
    B.base = B.scene_of + align_up(4 * static_cast<size_t>(n_total > 0 ? n_total : 1));
    B.total = B.base + align_up(8 * static_cast<size_t>(n_scenes + 1));
    return B;
}

// Batched volumes by bricks: the batched layout, then every scene's brick
// numbering, then the brick arrays over all scenes' slots and the pieces.
struct BatchBrickLayout {
    size_t sb;           // SceneBricks [n_scenes]
    size_t brick_scene;  // int32 [total_bricks]
    VolLayout VL;        // slots = total_bricks * kPieceClasses
    BrickGeom tot;  // n_bricks and n_slots of the whole batch (the rest unused)
};

BatchBrickLayout batch_brick_layout(int64_t n_total, int32_t n_scenes, int64_t total_bricks, int64_t capacity)
{
    BatchBrickLayout L;
    std::memset(&L.tot, 0, sizeof(L.tot));
    L.tot.n_bricks = total_bricks;
    L.tot.n_slots = total_bricks * kPieceClasses;
    L.tot.reps = 1;
    L.sb = batch_layout(n_total, n_scenes).total;
    L.brick_scene = L.sb + align_up(sizeof(SceneBricks) * static_cast<size_t>(n_scenes));
    L.VL = vol_layout(n_total, L.tot, capacity, L.brick_scene + align_up(4 * static_cast<size_t>(total_bricks)));
    return L;
}

// The batched volumes by bricks: scene numbering, bin count, scan of the slot
// counts, scatter, one CTA per brick (plain-store merge into its scene's
// volume), then the batched atomics, run only if the pieces did not fit.
vox_status launch_batched_bricks(const vox_segment *segs, int64_t n_total, const SceneDesc *scenes,
                                 const int32_t *scene_of, int32_t n_scenes, int64_t total_bricks, bool fresh,
                                 void *ws, size_t ws_bytes, int32_t *status, cudaStream_t stream, bool count_only)
{
    const BatchBrickLayout BL = batch_brick_layout(n_total, n_scenes, total_bricks, 0);
    const VolLayout &VL = BL.VL;
    const int64_t capacity = static_cast<int64_t>((ws_bytes - VL.pieces) / 8);
    char *base = static_cast<char *>(ws);
    SceneBricks *sb = reinterpret_cast<SceneBricks *>(base + BL.sb);
    int32_t *brick_scene = reinterpret_cast<int32_t *>(base + BL.brick_scene);
    k_scene_bricks<<<1, kSceneBrickThreads, 0, stream>>>(scenes, n_scenes, sb, brick_scene, total_bricks, status);
    if (cudaGetLastError() != cudaSuccess) return VOX_ERR_CUDA;
    if (cudaMemsetAsync(base + VL.hdr, 0, VL.off - VL.hdr, stream) != cudaSuccess) return VOX_ERR_CUDA;
    BinParams bp{};
    bp.segs = reinterpret_cast<const int32_t *>(segs);
    bp.n = n_total;
    bp.G = BL.tot;
    bp.brick_count = reinterpret_cast<int32_t *>(base + VL.count);
    bp.cursor = reinterpret_cast<int64_t *>(base + VL.cursor);
    bp.brick_off = reinterpret_cast<const int64_t *>(base + VL.off);
    bp.pieces = reinterpret_cast<uint64_t *>(base + VL.pieces);
    bp.capacity = capacity;
    bp.status = status;
    bp.sb = sb;
    bp.scene_of = scene_of;
    bp.n_scenes = n_scenes;
    if (vox_status e = launch_bin_count(bp, false, true, n_total, stream)) return e;
    ScanParams sp{};
    sp.counts_in = bp.brick_count;
    sp.offsets_copy = bp.cursor;
    sp.n = BL.tot.n_slots;
    sp.offsets = reinterpret_cast<int64_t *>(base + VL.off);
    sp.desc = reinterpret_cast<uint64_t *>(base + VL.desc);
    sp.ticket = reinterpret_cast<uint32_t *>(base + VL.hdr);
    sp.status = status;
    sp.n_tiles = VL.n_tiles;
    sp.stall_tile = -1;
    sp.wait_ns = static_cast<uint64_t>(g_wait_ns.load());
    k_scan<false><<<static_cast<unsigned>(VL.n_tiles), kScanThreads, 0, stream>>>(sp);
    if (cudaGetLastError() != cudaSuccess) return VOX_ERR_CUDA;
    if (count_only) return VOX_OK;
    if (vox_status e = launch_bin_scatter(bp, false, true, n_total, stream)) return e;
    BrickParams brp{};
    brp.segs = bp.segs;
    brp.G = BL.tot;
    brp.brick_off = bp.brick_off;
    brp.pieces = bp.pieces;
    brp.capacity = capacity;
    brp.mask = nullptr;
    brp.status = status;
    brp.ticket = reinterpret_cast<uint32_t *>(base + VL.hdr + 128);
    brp.use_tma = 0;
    brp.fresh = fresh ? 1 : 0;
    brp.bricked = 0;
    brp.sb = sb;
    brp.n_scenes = n_scenes;
    brp.brick_scene = brick_scene;
    CUtensorMap tmap;
    std::memset(&tmap, 0, sizeof(tmap));
    const size_t bsmem = sizeof(BrickSmem);
    const void *bk = reinterpret_cast<const void *>(k_brick_volume<false, true>);
    if (vox_status e = allow_smem(bk, bsmem)) return e;
    const int bgrid = grid_ctas(bk, kBrickThreads, bsmem);
    if (bgrid <= 0) return VOX_ERR_CUDA;
    k_brick_volume<false, true><<<static_cast<unsigned>(bgrid), kBrickThreads, bsmem, stream>>>(brp, tmap);
    if (cudaGetLastError() != cudaSuccess) return VOX_ERR_CUDA;
    const vox_dims unused{1, 1, 1};
    return launch_generate(segs, n_total, unused, nullptr, 0, nullptr, VOX_OUT_BITMASK, ws, status, stream,
                           bp.brick_off + BL.tot.n_slots, capacity, scenes, scene_of, n_scenes);
}

// ---- measurement helper: red.or throughput ------------------------------------
// Each thread issues `per_thread` 32-bit OR reductions (the instruction the
// per-voxel atomic volume issues) at pseudo-random words of the buffer: a
// per-thread linear congruential sequence x <- 1664525 x + 1013904223 (mod 2^32),
// word = floor(x * words / 2^32), bit = x mod 32.
__global__ void __launch_bounds__(256) k_probe_red_or(uint32_t *buf, uint64_t words, int64_t per_thread, uint32_t seed)
{
    uint64_t policy;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(policy));
    uint32_t x = seed ^ ((blockIdx.x * blockDim.x + threadIdx.x) * 0x9E3779B9u);
    for (int64_t i = 0; i < per_thread; ++i) {
        x = x * 1664525u + 1013904223u;
        const uint64_t idx = (static_cast<uint64_t>(x) * words) >> 32;
        red_or_keep(buf + idx, 1u << (x & 31u), policy);
    }
}

// ---- allocation-free variant: scratch in a static device array -------------
// Same layout as ws_layout(VOX_NOALLOC_MAX_SEGMENTS): ticket region, tile
// descriptors, offsets; each region rounded up to 256 bytes.
constexpr int64_t kNoAllocMaxSegments = VOX_NOALLOC_MAX_SEGMENTS;
constexpr size_t round256(size_t x) { return (x + 255) / 256 * 256; }
constexpr size_t kNoAllocScratchBytes =
    256 + round256(8 * static_cast<size_t>((kNoAllocMaxSegments + kScanTile - 1) / kScanTile)) +
    round256(8 * static_cast<size_t>(kNoAllocMaxSegments + 4));
static_assert(kNoAllocScratchBytes == VOX_NOALLOC_SCRATCH_BYTES, "scratch size in vox.h is stale");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Unique id of the current device's current context (0 when none can be read):
// a context that replaces an earlier one (after cudaDeviceReset) gets a new id
// even if its handle value repeats.
unsigned long long current_context_id()
{
    static std::mutex mu;
    static PFN_cuCtxGetCurrent_v4000 get_current = nullptr;
    static PFN_cuCtxGetId_v12000 get_id = nullptr;
    {
        std::lock_guard<std::mutex> lock(mu);
        if (get_current == nullptr || get_id == nullptr) {
            void *f1 = nullptr, *f2 = nullptr;
            cudaDriverEntryPointQueryResult q1, q2;
            if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 4000, cudaEnableDefault, &q1) != cudaSuccess ||
                q1 != cudaDriverEntryPointSuccess ||
                cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) != cudaSuccess ||
                q2 != cudaDriverEntryPointSuccess || f1 == nullptr || f2 == nullptr)
                return 0;
            get_current = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(f1);
            get_id = reinterpret_cast<PFN_cuCtxGetId_v12000>(f2);
        }
    }
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (get_current(&ctx) != CUDA_SUCCESS || ctx == nullptr || get_id(ctx, &id) != CUDA_SUCCESS) return 0;
    return id;
}

// Device address of the static scratch on the current device, looked up once
// per device and context (host code must not use the symbol itself as a device
// pointer; a context that replaces the device's earlier one reloads the module,
// so its address is looked up again).
vox_status noalloc_scratch(void **out)
{
    static std::mutex mu;
    static std::map<std::pair<int, unsigned long long>, void *> cache;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return VOX_ERR_CUDA;
    // no context current yet (0): the lookup below creates it, and the next
    // call finds it and caches
    const unsigned long long ctx = current_context_id();
    std::lock_guard<std::mutex> lock(mu);
    const auto key = std::make_pair(dev, ctx);
    auto it = ctx != 0 ? cache.find(key) : cache.end();
    if (it != cache.end()) {
        *out = it->second;
        return VOX_OK;
    }
    void *ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || ptr == nullptr) return VOX_ERR_CUDA;
    if (ctx != 0) cache[key] = ptr;
    *out = ptr;
    return VOX_OK;
}

template <bool kWrite, int OUT, bool LIN64>
vox_status launch_euclid_runs(const EuclidParams &p, cudaStream_t stream)
{
    const int sms = sm_count();
    if (sms <= 0) return VOX_ERR_CUDA;
    const int64_t want = (p.n_runs + 255) / 256;
    const unsigned blocks = static_cast<unsigned>(std::min<int64_t>(want, static_cast<int64_t>(sms) * 8));
    k_euclid_runs<kWrite, OUT, LIN64><<<blocks, 256, 0, stream>>>(p);
    return cudaGetLastError() == cudaSuccess ? VOX_OK : VOX_ERR_CUDA;
}

// The warp walk over groups of 32 runs: a persistent grid (SMs x CTAs per SM,
// no more CTAs than the groups fill), warps striding over the groups.
template <bool kWrite, int OUT, bool LIN64>
vox_status launch_euclid_warp(const EuclidParams &p, cudaStream_t stream)
{
    const void *k = reinterpret_cast<const void *>(k_euclid_warp<kWrite, OUT, LIN64>);
    int grid = grid_ctas(k, 32 * kEuclidWarps, 0);
    if (grid <= 0) return VOX_ERR_CUDA;
    const int64_t groups = (p.n_runs + 31) / 32;
    grid = static_cast<int>(std::min<int64_t>(grid, (groups + kEuclidWarps - 1) / kEuclidWarps));
    k_euclid_warp<kWrite, OUT, LIN64><<<static_cast<unsigned>(grid), 32 * kEuclidWarps, 0, stream>>>(p);
    return cudaGetLastError() == cudaSuccess ? VOX_OK : VOX_ERR_CUDA;
}

template <int OUT, bool LIN64>
vox_status launch_euclid_list(const EuclidParams &p, cudaStream_t stream)
{
    return launch_euclid_warp<true, OUT, LIN64>(p, stream);
}

// Count + scan of the samples (and the brick binning's counts when the workspace
// holds brick arrays after the run arrays), voxels per run, scan of the run
// counts, and (unless count_only) the outputs: the compacted list by the run
// walk, the volume by bricks (then a gated atomics pass if the pieces did not
// fit) or by the run walk's atomics.
vox_status launch_euclid(const vox_segment *segs, int64_t n, vox_dims dims, void *list, int64_t capacity,
                         uint32_t *mask, int flags, int64_t *seg_off, void *ws, size_t ws_bytes, int32_t *status,
                         cudaStream_t stream, bool count_only)
{
    const EuclidLayout E = euclid_layout(n);
    char *base = static_cast<char *>(ws);
    BrickGeom G;
    const bool bricks = uses_bricks(n, dims, ws_bytes, &G, E.total);
    if (vox_status e = launch_count_scan(segs, n, dims, nullptr, nullptr, ws, ws_bytes, status, stream, nullptr,
                                         nullptr, 0, true))
        return e;
    if (cudaMemsetAsync(base + E.hdr, 0, kWsAlign, stream) != cudaSuccess) return VOX_ERR_CUDA;
    if (cudaMemsetAsync(base + E.desc, 0, E.off - E.desc, stream) != cudaSuccess) return VOX_ERR_CUDA;
    EuclidParams p;
    p.segs = reinterpret_cast<const int32_t *>(segs);
    p.n = n;
    p.offsets = reinterpret_cast<const int64_t *>(base + ws_layout(n).offsets);
    p.w = dims.w;
    p.h = dims.h;
    p.n_runs = E.n_runs;
    p.run_count = reinterpret_cast<int32_t *>(base + E.count);
    p.run_off = reinterpret_cast<const int64_t *>(base + E.off);
    p.list = list;
    p.capacity = capacity;
    p.mask = mask;
    p.seg_off = seg_off;
    p.status = status;
    p.gate_total = nullptr;
    p.gate_cap = 0;
    // output positions (the run counts and their scan) are needed for a list,
    // the segment offsets and the plan; a volume alone goes without them
    const bool positions = count_only || seg_off != nullptr || (flags & (VOX_OUT_LIST32 | VOX_OUT_LIST64));
    if (positions) {
        if (vox_status e = launch_euclid_warp<false, 0, false>(p, stream)) return e;
        ScanParams sp{};
        sp.counts_in = p.run_count;
        sp.n = E.n_runs;
        sp.offsets = reinterpret_cast<int64_t *>(base + E.off);
        sp.desc = reinterpret_cast<uint64_t *>(base + E.desc);
        sp.ticket = reinterpret_cast<uint32_t *>(base + E.hdr);
        sp.status = status;
        sp.n_tiles = E.n_tiles;
        sp.stall_tile = -1;
        sp.wait_ns = static_cast<uint64_t>(g_wait_ns.load());
        k_scan<false><<<static_cast<unsigned>(E.n_tiles), kScanThreads, 0, stream>>>(sp);
        if (cudaGetLastError() != cudaSuccess) return VOX_ERR_CUDA;
    }
    if (count_only) {
        if (bricks) return launch_bricks(segs, n, G, dims, nullptr, ws, ws_bytes, status, stream, true, false, false, true);
        return VOX_OK;
    }
    const bool bm = flags & VOX_OUT_BITMASK;
    const bool lin64 = volume_bits(dims) > (uint64_t(1) << 32);
    const bool vol_by_bricks = bm && bricks;
    const bool mask_in_walk = bm && !bricks;
    if (mask_in_walk && (flags & VOX_OUT_FRESH) &&
        cudaMemsetAsync(mask, 0, 4 * static_cast<size_t>(vox_mask_words(dims)), stream) != cudaSuccess)
        return VOX_ERR_CUDA;
    // the run walk's write pass first: a list capacity error found there keeps
    // every later kernel (the bricks too) from writing
    vox_status e = VOX_OK;
    if (flags & VOX_OUT_LIST32) {
        e = mask_in_walk ? launch_euclid_list<kOutList32 | kOutMask, false>(p, stream)
                         : launch_euclid_list<kOutList32, false>(p, stream);
    } else if (flags & VOX_OUT_LIST64) {
        e = !mask_in_walk ? launch_euclid_list<kOutList64, false>(p, stream)
                          : (lin64 ? launch_euclid_list<kOutList64 | kOutMask, true>(p, stream)
                                   : launch_euclid_list<kOutList64 | kOutMask, false>(p, stream));
    } else if (mask_in_walk) {
        e = lin64 ? launch_euclid_runs<true, kOutMask, true>(p, stream)
                  : launch_euclid_runs<true, kOutMask, false>(p, stream);
    } else if (seg_off != nullptr) {
        e = launch_euclid_runs<true, 0, false>(p, stream);  // the segment offsets alone
    }
    if (e) return e;
    if (vol_by_bricks) {
        const bool fresh = flags & VOX_OUT_FRESH;
        if ((e = launch_bricks(segs, n, G, dims, mask, ws, ws_bytes, status, stream, false, fresh, false, true)))
            return e;
        // per-voxel atomics, run only if the pieces did not fit the workspace
        const VolLayout VL = vol_layout(n, G, 0, E.total);
        EuclidParams g = p;
        g.list = nullptr;
        g.seg_off = nullptr;
        g.gate_total = reinterpret_cast<const int64_t *>(base + VL.off) + G.n_slots;
        g.gate_cap = static_cast<int64_t>((ws_bytes - VL.pieces) / 8);
        e = lin64 ? launch_euclid_runs<true, kOutMask, true>(g, stream)
                  : launch_euclid_runs<true, kOutMask, false>(g, stream);
    }
    if (e) return e;
    if (seg_off != nullptr && cudaMemcpyAsync(seg_off + n, base + E.off + 8 * static_cast<size_t>(E.n_runs),
                                              sizeof(int64_t), cudaMemcpyDeviceToDevice, stream) != cudaSuccess)
        return VOX_ERR_CUDA;
    return VOX_OK;
}

// Bytes of the host-call arena before its workspace: status, segments, list, volume.
size_t host_arena_prefix(int64_t n, vox_dims dims, int flags, int64_t list_capacity)
{
    const size_t elem = (flags & VOX_OUT_LIST64) ? 8 : ((flags & VOX_OUT_LIST32) ? 4 : 0);
    size_t total = align_up(sizeof(int32_t));                                   // status
    total += align_up(sizeof(vox_segment) * static_cast<size_t>(n));            // segments
    total += align_up(elem * static_cast<size_t>(list_capacity));               // list
    if (flags & VOX_OUT_BITMASK) total += align_up(4 * static_cast<size_t>(vox_mask_words(dims)));
    return total;
}

// A second stream per device for the host call's list copy, so that the copy
// overlaps the volume's kernels. Created on first use, kept for the process.
cudaStream_t copy_stream()
{
    static std::mutex mu;
    static std::map<int, cudaStream_t> streams;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    std::lock_guard<std::mutex> lock(mu);
    auto it = streams.find(dev);
    if (it != streams.end()) return it->second;
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return nullptr;
    streams[dev] = s;
    return s;
}

}  // namespace

extern "C" {

vox_status vox_generate_noalloc(const vox_segment *d_segs, int64_t n, vox_dims dims, void *d_list,
                                int64_t list_capacity, uint32_t *d_mask, int flags, int32_t *d_status, void *stream)
{
    if (n > kNoAllocMaxSegments) return VOX_ERR_WORKSPACE;
    if (n < 0) return VOX_ERR_INVALID_ARG;
    if (ws_layout(n).total > kNoAllocScratchBytes) return VOX_ERR_WORKSPACE;
    void *scratch = nullptr;
    if (vox_status e = noalloc_scratch(&scratch)) return e;
    // exactly the count/scan workspace of n segments: the same path as
    // vox_generate with vox_workspace_size(n) bytes (per-voxel atomic volume)
    return vox_generate(d_segs, n, dims, d_list, list_capacity, d_mask, flags, scratch, ws_layout(n).total, d_status,
                        stream);
}

vox_status vox_probe_red_or(uint32_t *d_buf, int64_t words, int64_t ops, uint32_t seed, void *stream)
{
    if (d_buf == nullptr || words < 1 || words > (int64_t(1) << 32) || ops < 0) return VOX_ERR_INVALID_ARG;
    if (!aligned(d_buf, 4)) return VOX_ERR_ALIGNMENT;
    const int sms = sm_count();
    if (sms <= 0) return VOX_ERR_CUDA;
    const int64_t threads = static_cast<int64_t>(sms) * 8 * 256;
    const int64_t per_thread = (ops + threads - 1) / threads;
    if (per_thread == 0) return VOX_OK;
    k_probe_red_or<<<static_cast<unsigned>(sms * 8), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        d_buf, static_cast<uint64_t>(words), per_thread, seed);
    return cudaGetLastError() == cudaSuccess ? VOX_OK : VOX_ERR_CUDA;
}

int64_t vox_probe_red_or_ops(int64_t ops)
{
    const int sms = sm_count();
    if (sms <= 0 || ops < 0) return 0;
    const int64_t threads = static_cast<int64_t>(sms) * 8 * 256;
    return (ops + threads - 1) / threads * threads;
}

size_t vox_workspace_size(int64_t n_segments)
{
    if (n_segments < 0) return 0;
    return ws_layout(n_segments).total;
}

int64_t vox_scan_tile_segments(void) { return kScanTile; }

int64_t vox_mask_words(vox_dims dims)
{
    if (check_dims(dims) != VOX_OK) return 0;
    return static_cast<int64_t>((volume_bits(dims) + 31) / 32);
}

vox_status vox_count(const vox_segment *d_segs, int64_t n, vox_dims dims, int32_t *d_counts, int64_t *d_offsets,
                     void *d_ws, size_t ws_bytes, int32_t *d_status, void *stream)
{
    if (n < 0 || d_status == nullptr || (n > 0 && d_segs == nullptr)) return VOX_ERR_INVALID_ARG;
    if (vox_status e = check_dims(dims)) return e;
    if (n > 0 && !aligned(d_segs, 16)) return VOX_ERR_ALIGNMENT;
    if (d_ws == nullptr || !aligned(d_ws, kWsAlign) || ws_bytes < ws_layout(n).total) return VOX_ERR_WORKSPACE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(d_status, 0, sizeof(int32_t), s) != cudaSuccess) return VOX_ERR_CUDA;
    if (n == 0) {
        const WsLayout L = ws_layout(0);
        if (cudaMemsetAsync(static_cast<char *>(d_ws) + L.offsets, 0, 4 * sizeof(int64_t), s) != cudaSuccess)
            return VOX_ERR_CUDA;
        if (d_offsets && cudaMemsetAsync(d_offsets, 0, sizeof(int64_t), s) != cudaSuccess) return VOX_ERR_CUDA;
        return VOX_OK;
    }
    return launch_count_scan(d_segs, n, dims, d_counts, d_offsets, d_ws, ws_bytes, d_status, s);
}

vox_status vox_count_bins(const vox_segment *d_segs, int64_t n, vox_dims dims, void *d_ws, size_t ws_bytes,
                          void *stream)
{
    if (n < 0 || (n > 0 && d_segs == nullptr)) return VOX_ERR_INVALID_ARG;
    if (vox_status e = check_dims(dims)) return e;
    if (n > 0 && !aligned(d_segs, 16)) return VOX_ERR_ALIGNMENT;
    if (d_ws == nullptr || !aligned(d_ws, kWsAlign)) return VOX_ERR_WORKSPACE;
    if (n == 0) return VOX_OK;
    BrickGeom G;
    if (!uses_bricks(n, dims, ws_bytes, &G)) return VOX_ERR_WORKSPACE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const VolLayout VL = vol_layout(n, G, 0);
    char *base = static_cast<char *>(d_ws);
    if (cudaMemsetAsync(base + VL.hdr, 0, VL.off - VL.hdr, s) != cudaSuccess) return VOX_ERR_CUDA;
    BinParams bp{};
    bp.segs = reinterpret_cast<const int32_t *>(d_segs);
    bp.n = n;
    bp.G = G;
    bp.brick_count = reinterpret_cast<int32_t *>(base + VL.count);
    return launch_bin_count(bp, false, false, n, s);
}

vox_status vox_generate(const vox_segment *d_segs, int64_t n, vox_dims dims, void *d_list, int64_t list_capacity,
                        uint32_t *d_mask, int flags, void *d_ws, size_t ws_bytes, int32_t *d_status, void *stream)
{
    if (vox_status e = check_generate_args(d_segs, n, dims, d_list, list_capacity, d_mask, flags, d_ws, ws_bytes,
                                           d_status))
        return e;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(d_status, 0, sizeof(int32_t), s) != cudaSuccess) return VOX_ERR_CUDA;
    if (n > 0) {
        if (vox_status e = launch_count_scan(d_segs, n, dims, nullptr, nullptr, d_ws, ws_bytes, d_status, s))
            return e;
    }
    return launch_outputs(d_segs, n, dims, d_list, list_capacity, d_mask, flags, d_ws, ws_bytes, d_status, s);
}

vox_status vox_generate_from_scan(const vox_segment *d_segs, int64_t n, vox_dims dims, void *d_list,
                                  int64_t list_capacity, uint32_t *d_mask, int flags, void *d_ws, size_t ws_bytes,
                                  int32_t *d_status, void *stream)
{
    if (vox_status e = check_generate_args(d_segs, n, dims, d_list, list_capacity, d_mask, flags, d_ws, ws_bytes,
                                           d_status))
        return e;
    return launch_outputs(d_segs, n, dims, d_list, list_capacity, d_mask, flags, d_ws, ws_bytes, d_status,
                          static_cast<cudaStream_t>(stream));
}

size_t vox_workspace_size_batched(int64_t n_total, int32_t n_scenes)
{
    if (n_total < 0 || n_scenes < 1) return 0;
    return batch_layout(n_total, n_scenes).total;
}

vox_status vox_generate_batched_ex(const vox_segment *d_segs, int64_t n_total, const vox_scene *d_scenes,
                                   int32_t n_scenes, int64_t total_bricks, void *d_list, int64_t list_capacity,
                                   int flags, int64_t *d_scene_base, void *d_ws, size_t ws_bytes, int32_t *d_status,
                                   void *stream)
{
    if (total_bricks < 0) return VOX_ERR_INVALID_ARG;
    if (n_total < 0 || n_scenes < 1 || d_scenes == nullptr || d_status == nullptr) return VOX_ERR_INVALID_ARG;
    if (n_total > 0 && d_segs == nullptr) return VOX_ERR_INVALID_ARG;
    if (flags & ~(VOX_OUT_LIST32 | VOX_OUT_LIST64 | VOX_OUT_BITMASK | VOX_OUT_FRESH)) return VOX_ERR_INVALID_ARG;
    const bool l32 = flags & VOX_OUT_LIST32, l64 = flags & VOX_OUT_LIST64, bm = flags & VOX_OUT_BITMASK;
    if (!(l32 || l64 || bm) || (l32 && l64)) return VOX_ERR_INVALID_ARG;
    if ((flags & VOX_OUT_FRESH) && !bm) return VOX_ERR_INVALID_ARG;
    if ((l32 || l64) && (d_list == nullptr || list_capacity < 0)) return VOX_ERR_INVALID_ARG;
    if (n_total > 0 && !aligned(d_segs, 16)) return VOX_ERR_ALIGNMENT;
    if ((l32 || l64) && !aligned(d_list, 16)) return VOX_ERR_ALIGNMENT;
    if (!aligned(d_scenes, 8)) return VOX_ERR_ALIGNMENT;
    const BatchLayout B = batch_layout(n_total, n_scenes);
    if (d_ws == nullptr || !aligned(d_ws, kWsAlign) || ws_bytes < B.total) return VOX_ERR_WORKSPACE;
    // the volumes by bricks when the caller gave the batch's brick count and the
    // workspace holds the brick arrays and a piece
    const bool bricks = bm && total_bricks > 0 && n_total > 0 && n_total < (int64_t(1) << 32) &&
                        current_tuning().volume_path == VOX_VOLUME_AUTO &&
                        ws_bytes >= batch_brick_layout(n_total, n_scenes, total_bricks, 1).VL.total;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    char *base = static_cast<char *>(d_ws);
    const SceneDesc *scenes = reinterpret_cast<const SceneDesc *>(d_scenes);
    int32_t *scene_of = reinterpret_cast<int32_t *>(base + B.scene_of);
    if (cudaMemsetAsync(d_status, 0, sizeof(int32_t), s) != cudaSuccess) return VOX_ERR_CUDA;
    k_scene_map<<<static_cast<unsigned>(n_scenes), 256, 0, s>>>(scenes, n_scenes, n_total, scene_of, d_status,
                                                                 l32 ? 1 : 0);
    if (cudaGetLastError() != cudaSuccess) return VOX_ERR_CUDA;
    if (bm && (flags & VOX_OUT_FRESH) && !bricks) {  // every scene's volume cleared (a valid table only)
        k_scene_clear<<<dim3(kSceneClearCtas, static_cast<unsigned>(n_scenes)), 256, 0, s>>>(scenes, d_status);
        if (cudaGetLastError() != cudaSuccess) return VOX_ERR_CUDA;
    }
    if (n_total > 0) {
        const vox_dims unused{1, 1, 1};
        if (vox_status e = launch_count_scan(d_segs, n_total, unused, nullptr, nullptr, d_ws, ws_bytes, d_status, s,
                                             scenes, scene_of, n_scenes))
            return e;
    } else {
        const WsLayout L = ws_layout(0);
        if (cudaMemsetAsync(base + L.offsets, 0, 4 * sizeof(int64_t), s) != cudaSuccess) return VOX_ERR_CUDA;
    }
    const WsLayout L = ws_layout(n_total);
    k_scene_base<<<static_cast<unsigned>((n_scenes + 1 + 255) / 256), 256, 0, s>>>(
        scenes, n_scenes, reinterpret_cast<const int64_t *>(base + L.offsets), n_total,
        reinterpret_cast<int64_t *>(base + B.base), d_scene_base, d_status);
    if (cudaGetLastError() != cudaSuccess) return VOX_ERR_CUDA;
    if (n_total == 0) return VOX_OK;
    const vox_dims unused{1, 1, 1};
    if (l32 || l64) {
        if (vox_status e = launch_generate(d_segs, n_total, unused, d_list, list_capacity, nullptr,
                                           flags & (VOX_OUT_LIST32 | VOX_OUT_LIST64), d_ws, d_status, s))
            return e;
    }
    if (bm && bricks)
        return launch_batched_bricks(d_segs, n_total, scenes, scene_of, n_scenes, total_bricks,
                                     (flags & VOX_OUT_FRESH) != 0, d_ws, ws_bytes, d_status, s, false);
    if (bm) {
        if (vox_status e = launch_generate(d_segs, n_total, unused, nullptr, 0, nullptr, VOX_OUT_BITMASK, d_ws, d_status,
                                           s, nullptr, 0, scenes, scene_of, n_scenes))
            return e;
    }
    return VOX_OK;
}

vox_status vox_generate_batched(const vox_segment *d_segs, int64_t n_total, const vox_scene *d_scenes,
                                int32_t n_scenes, void *d_list, int64_t list_capacity, int flags,
                                int64_t *d_scene_base, void *d_ws, size_t ws_bytes, int32_t *d_status, void *stream)
{
    return vox_generate_batched_ex(d_segs, n_total, d_scenes, n_scenes, 0, d_list, list_capacity, flags, d_scene_base,
                                   d_ws, ws_bytes, d_status, stream);
}

int64_t vox_scene_bricks(vox_dims dims)
{
    BrickGeom G;
    if (check_dims(dims) != VOX_OK || !brick_geom(dims.w, dims.h, dims.d, &G, false)) return 0;
    return G.n_bricks;
}

size_t vox_workspace_size_batched_volume(int64_t n_total, int32_t n_scenes, int64_t total_bricks,
                                         int64_t piece_capacity)
{
    if (n_total < 0 || n_scenes < 1 || total_bricks < 0 || piece_capacity < 0) return 0;
    if (total_bricks == 0) return batch_layout(n_total, n_scenes).total;
    return batch_brick_layout(n_total, n_scenes, total_bricks, piece_capacity > 0 ? piece_capacity : 1).VL.total;
}

vox_status vox_plan_batched(const vox_segment *d_segs, int64_t n_total, const vox_scene *d_scenes, int32_t n_scenes,
                            int64_t total_bricks, void *d_ws, size_t ws_bytes, int32_t *d_status, int64_t *h_voxels,
                            int64_t *h_pieces, void *stream)
{
    if (n_total < 0 || n_scenes < 1 || total_bricks < 0 || d_scenes == nullptr || d_status == nullptr)
        return VOX_ERR_INVALID_ARG;
    if (n_total > 0 && (d_segs == nullptr || !aligned(d_segs, 16))) return VOX_ERR_INVALID_ARG;
    if (!aligned(d_scenes, 8)) return VOX_ERR_ALIGNMENT;
    const bool bricks = total_bricks > 0 && n_total > 0 && n_total < (int64_t(1) << 32);
    const size_t need = bricks ? batch_brick_layout(n_total, n_scenes, total_bricks, 0).VL.total
                               : batch_layout(n_total, n_scenes).total;
    if (d_ws == nullptr || !aligned(d_ws, kWsAlign) || ws_bytes < need) return VOX_ERR_WORKSPACE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    char *base = static_cast<char *>(d_ws);
    const BatchLayout B = batch_layout(n_total, n_scenes);
    const SceneDesc *scenes = reinterpret_cast<const SceneDesc *>(d_scenes);
    int32_t *scene_of = reinterpret_cast<int32_t *>(base + B.scene_of);
    if (cudaMemsetAsync(d_status, 0, sizeof(int32_t), s) != cudaSuccess) return VOX_ERR_CUDA;
    k_scene_map<<<static_cast<unsigned>(n_scenes), 256, 0, s>>>(scenes, n_scenes, n_total, scene_of, d_status, 0);
    if (cudaGetLastError() != cudaSuccess) return VOX_ERR_CUDA;
    int64_t V = 0, pieces = 0;
    int32_t st = 0;
    if (n_total > 0) {
        const vox_dims unused{1, 1, 1};
        if (vox_status e = launch_count_scan(d_segs, n_total, unused, nullptr, nullptr, d_ws, ws_bytes, d_status, s,
                                             scenes, scene_of, n_scenes))
            return e;
        if (bricks) {
            if (vox_status e = launch_batched_bricks(d_segs, n_total, scenes, scene_of, n_scenes, total_bricks, false,
                                                     d_ws, ws_bytes, d_status, s, true))
                return e;
            const BatchBrickLayout BL = batch_brick_layout(n_total, n_scenes, total_bricks, 0);
            if (cudaMemcpyAsync(&pieces, base + BL.VL.off + 8 * static_cast<size_t>(BL.tot.n_slots), 8,
                                cudaMemcpyDeviceToHost, s) != cudaSuccess)
                return VOX_ERR_CUDA;
        }
        if (cudaMemcpyAsync(&V, base + ws_layout(n_total).offsets + 8 * static_cast<size_t>(n_total), 8,
                            cudaMemcpyDeviceToHost, s) != cudaSuccess)
            return VOX_ERR_CUDA;
    }
    if (cudaMemcpyAsync(&st, d_status, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return VOX_ERR_CUDA;
    if (h_voxels) *h_voxels = V;
    if (h_pieces) *h_pieces = pieces;
    return static_cast<vox_status>(st);
}

int64_t vox_mask_words_bricked(vox_dims dims)
{
    BrickGeom G;
    if (!make_geom(dims, &G)) return 0;
    return G.n_bricks * static_cast<int64_t>(G.words);
}

vox_status vox_brick_shape(vox_dims dims, int32_t *h_shape)
{
    BrickGeom G;
    if (h_shape == nullptr || !make_geom(dims, &G)) return VOX_ERR_INVALID_ARG;
    for (int a = 0; a < 3; ++a) {
        h_shape[a] = G.B[a];
        h_shape[3 + a] = G.nb[a];
    }
    return VOX_OK;
}

vox_status vox_unbrick(const uint32_t *d_bricked, vox_dims dims, uint32_t *d_mask, int32_t *d_status, void *stream)
{
    BrickGeom G;
    if (d_bricked == nullptr || d_mask == nullptr || !make_geom(dims, &G)) return VOX_ERR_INVALID_ARG;
    if (!aligned(d_bricked, 4) || !aligned(d_mask, 4)) return VOX_ERR_ALIGNMENT;
    const int sms = sm_count();
    if (sms <= 0) return VOX_ERR_CUDA;
    // half bricks through the bulk-copy unit when the volume takes brick-shaped
    // TMA boxes (w and B0 multiples of 128, 16-byte aligned buffers)
    CUtensorMap tmap;
    std::memset(&tmap, 0, sizeof(tmap));
    if (G.B[2] % kUnbrickSplit == 0 && aligned(d_bricked, 16) &&
        make_volume_tmap(G, d_mask, &tmap, G.B[2] / kUnbrickSplit)) {
        const size_t smem = 4 * static_cast<size_t>(G.words / kUnbrickSplit);
        if (vox_status e = allow_smem(reinterpret_cast<const void *>(k_unbrick_tma), smem)) return e;
        const int grid = grid_ctas(reinterpret_cast<const void *>(k_unbrick_tma), 32, smem);
        if (grid <= 0) return VOX_ERR_CUDA;
        k_unbrick_tma<<<static_cast<unsigned>(grid), 32, smem, static_cast<cudaStream_t>(stream)>>>(
            d_bricked, G, tmap, d_status, static_cast<uint64_t>(g_wait_ns.load()));
        return cudaGetLastError() == cudaSuccess ? VOX_OK : VOX_ERR_CUDA;
    }
    const int64_t rows = static_cast<int64_t>(dims.h) * dims.d;
    const int64_t blocks = std::min<int64_t>((rows + 7) / 8, static_cast<int64_t>(sms) * 16);
    k_unbrick<<<static_cast<unsigned>(blocks), 256, 0, static_cast<cudaStream_t>(stream)>>>(d_bricked, G, d_mask);
    return cudaGetLastError() == cudaSuccess ? VOX_OK : VOX_ERR_CUDA;
}

size_t vox_euclid_workspace_size(int64_t n)
{
    if (n < 0) return 0;
    return euclid_layout(n).total;
}

size_t vox_euclid_workspace_size_volume(int64_t n, vox_dims dims, int64_t piece_capacity)
{
    if (n < 0 || piece_capacity < 0) return 0;
    BrickGeom G;
    const size_t base = euclid_layout(n).total;
    if (!make_geom(dims, &G)) return base;
    return vol_layout(n, G, piece_capacity > 0 ? piece_capacity : 1, base).total;
}

vox_status vox_euclid_generate(const vox_segment *d_segs, int64_t n, vox_dims dims, void *d_list,
                               int64_t list_capacity, uint32_t *d_mask, int flags, int64_t *d_offsets, void *d_ws,
                               size_t ws_bytes, int32_t *d_status, void *stream)
{
    if (flags & VOX_OUT_BRICKED) return VOX_ERR_INVALID_ARG;
    if (vox_status e = check_generate_args(d_segs, n, dims, d_list, list_capacity, d_mask, flags, d_ws, ws_bytes,
                                           d_status))
        return e;
    if (n >= 0 && ws_bytes < euclid_layout(n).total) return VOX_ERR_WORKSPACE;
    if (d_offsets != nullptr && !aligned(d_offsets, 8)) return VOX_ERR_ALIGNMENT;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(d_status, 0, sizeof(int32_t), s) != cudaSuccess) return VOX_ERR_CUDA;
    if (n == 0) {
        if ((flags & VOX_OUT_BITMASK) && (flags & VOX_OUT_FRESH) &&
            cudaMemsetAsync(d_mask, 0, 4 * static_cast<size_t>(vox_mask_words(dims)), s) != cudaSuccess)
            return VOX_ERR_CUDA;
        if (d_offsets != nullptr && cudaMemsetAsync(d_offsets, 0, sizeof(int64_t), s) != cudaSuccess)
            return VOX_ERR_CUDA;
        return VOX_OK;
    }
    return launch_euclid(d_segs, n, dims, d_list, list_capacity, d_mask, flags, d_offsets, d_ws, ws_bytes, d_status, s,
                         false);
}

vox_status vox_euclid_plan(const vox_segment *d_segs, int64_t n, vox_dims dims, void *d_ws, size_t ws_bytes,
                           int32_t *d_status, int64_t *h_voxels, int64_t *h_samples, int64_t *h_pieces, void *stream)
{
    if (n < 0 || d_status == nullptr || (n > 0 && d_segs == nullptr)) return VOX_ERR_INVALID_ARG;
    if (vox_status e = check_dims(dims)) return e;
    if (n > 0 && !aligned(d_segs, 16)) return VOX_ERR_ALIGNMENT;
    if (d_ws == nullptr || !aligned(d_ws, kWsAlign) || ws_bytes < euclid_layout(n).total) return VOX_ERR_WORKSPACE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int64_t voxels = 0, samples = 0, pieces = 0;
    int32_t st = 0;
    if (n > 0) {
        if (cudaMemsetAsync(d_status, 0, sizeof(int32_t), s) != cudaSuccess) return VOX_ERR_CUDA;
        if (vox_status e = launch_euclid(d_segs, n, dims, nullptr, 0, nullptr, 0, nullptr, d_ws, ws_bytes, d_status, s,
                                         true))
            return e;
        const EuclidLayout E = euclid_layout(n);
        const char *base = static_cast<const char *>(d_ws);
        BrickGeom G;
        if (uses_bricks(n, dims, ws_bytes, &G, E.total)) {
            const VolLayout VL = vol_layout(n, G, 0, E.total);
            if (cudaMemcpyAsync(&pieces, base + VL.off + 8 * static_cast<size_t>(G.n_slots), 8,
                                cudaMemcpyDeviceToHost, s) != cudaSuccess)
                return VOX_ERR_CUDA;
        }
        if (cudaMemcpyAsync(&samples, base + ws_layout(n).offsets + 8 * static_cast<size_t>(n), 8,
                            cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaMemcpyAsync(&voxels, base + E.off + 8 * static_cast<size_t>(E.n_runs), 8, cudaMemcpyDeviceToHost,
                            s) != cudaSuccess ||
            cudaMemcpyAsync(&st, d_status, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return VOX_ERR_CUDA;
    }
    if (h_voxels) *h_voxels = voxels;
    if (h_samples) *h_samples = samples;
    if (h_pieces) *h_pieces = pieces;
    return static_cast<vox_status>(st);
}

size_t vox_workspace_size_volume(int64_t n, vox_dims dims, int64_t piece_capacity)
{
    if (n < 0 || piece_capacity < 0) return 0;
    BrickGeom G;
    if (!make_geom(dims, &G)) return ws_layout(n).total;
    return vol_layout(n, G, piece_capacity > 0 ? piece_capacity : 1).total;
}

vox_status vox_plan(const vox_segment *d_segs, int64_t n, vox_dims dims, void *d_ws, size_t ws_bytes,
                    int32_t *d_status, int64_t *h_voxels, int64_t *h_pieces, void *stream)
{
    if (n < 0 || d_status == nullptr || (n > 0 && d_segs == nullptr)) return VOX_ERR_INVALID_ARG;
    if (vox_status e = check_dims(dims)) return e;
    if (n > 0 && !aligned(d_segs, 16)) return VOX_ERR_ALIGNMENT;
    BrickGeom G;
    const bool brickable = make_geom(dims, &G);
    const size_t need = brickable ? vol_layout(n, G, 1).total : ws_layout(n).total;
    if (d_ws == nullptr || !aligned(d_ws, kWsAlign) || ws_bytes < need) return VOX_ERR_WORKSPACE;
    const bool bricks = n > 0 && brickable;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (vox_status e = vox_count(d_segs, n, dims, nullptr, nullptr, d_ws, ws_bytes, d_status, s)) return e;
    int64_t V = 0, pieces = 0;
    int32_t st = 0;
    if (n > 0 && bricks) {
        if (vox_status e = launch_bricks(d_segs, n, G, dims, nullptr, d_ws, ws_bytes, d_status, s, true)) return e;
        const VolLayout VL = vol_layout(n, G, 0);
        if (cudaMemcpyAsync(&pieces, static_cast<char *>(d_ws) + VL.off + 8 * static_cast<size_t>(G.n_slots),
                            sizeof(int64_t), cudaMemcpyDeviceToHost, s) != cudaSuccess)
            return VOX_ERR_CUDA;
    }
    const WsLayout L = ws_layout(n);
    if (cudaMemcpyAsync(&V, static_cast<char *>(d_ws) + L.offsets + sizeof(int64_t) * static_cast<size_t>(n),
                        sizeof(int64_t), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return VOX_ERR_CUDA;
    if (cudaMemcpyAsync(&st, d_status, sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess) return VOX_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return VOX_ERR_CUDA;
    if (h_voxels) *h_voxels = V;
    if (h_pieces) *h_pieces = pieces;
    return static_cast<vox_status>(st);
}

size_t vox_host_arena_size(int64_t n, vox_dims dims, int flags, int64_t list_capacity)
{
    if (n < 0 || list_capacity < 0 || check_dims(dims) != VOX_OK) return 0;
    return host_arena_prefix(n, dims, flags, list_capacity) + ws_layout(n).total;
}

size_t vox_host_arena_size_volume(int64_t n, vox_dims dims, int flags, int64_t list_capacity,
                                  int64_t piece_capacity)
{
    if (n < 0 || list_capacity < 0 || piece_capacity < 0 || check_dims(dims) != VOX_OK) return 0;
    return host_arena_prefix(n, dims, flags, list_capacity) + vox_workspace_size_volume(n, dims, piece_capacity);
}

vox_status vox_generate_host(const vox_segment *h_segs, int64_t n, vox_dims dims, void *h_list,
                             int64_t list_capacity, uint32_t *h_mask, int flags, void *d_arena, size_t arena_bytes,
                             int64_t *h_total, void *stream)
{
    if (n < 0 || (n > 0 && h_segs == nullptr)) return VOX_ERR_INVALID_ARG;
    if (flags & VOX_OUT_BRICKED) return VOX_ERR_INVALID_ARG;  // host volumes are row-major
    if (vox_status e = check_dims(dims)) return e;
    const bool has_list = flags & (VOX_OUT_LIST32 | VOX_OUT_LIST64);
    const bool bm = flags & VOX_OUT_BITMASK;
    if ((has_list && h_list == nullptr) || (bm && h_mask == nullptr)) return VOX_ERR_INVALID_ARG;
    const size_t need = vox_host_arena_size(n, dims, flags, list_capacity);
    if (d_arena == nullptr || !aligned(d_arena, kWsAlign) || need == 0 || arena_bytes < need) return VOX_ERR_WORKSPACE;
    const size_t elem = (flags & VOX_OUT_LIST64) ? 8 : ((flags & VOX_OUT_LIST32) ? 4 : 0);
    char *a = static_cast<char *>(d_arena);
    int32_t *d_status = reinterpret_cast<int32_t *>(a);
    a += align_up(sizeof(int32_t));
    vox_segment *d_segs = reinterpret_cast<vox_segment *>(a);
    a += align_up(sizeof(vox_segment) * static_cast<size_t>(n));
    void *d_list = has_list ? a : nullptr;
    a += align_up(elem * static_cast<size_t>(list_capacity));
    uint32_t *d_mask = nullptr;
    const int64_t words = vox_mask_words(dims);
    if (bm) {
        d_mask = reinterpret_cast<uint32_t *>(a);
        a += align_up(4 * static_cast<size_t>(words));
    }
    void *d_ws = a;
    // the workspace takes the rest of the arena: with room for the brick arrays
    // and pieces (vox_host_arena_size_volume) the volume is built by bricks
    const size_t ws_bytes = arena_bytes - static_cast<size_t>(a - static_cast<char *>(d_arena));
    if (vox_status e = check_generate_args(n > 0 ? d_segs : nullptr, n, dims, d_list, list_capacity, d_mask, flags,
                                           d_ws, ws_bytes, d_status))
        return e;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (n > 0 && cudaMemcpyAsync(d_segs, h_segs, sizeof(vox_segment) * static_cast<size_t>(n),
                                 cudaMemcpyHostToDevice, s) != cudaSuccess)
        return VOX_ERR_CUDA;
    if (vox_status e = vox_count(d_segs, n, dims, nullptr, nullptr, d_ws, ws_bytes, d_status, s)) return e;
    int64_t V = 0;
    int32_t st = 0;
    const WsLayout L = ws_layout(n);
    if (cudaMemcpyAsync(&V, static_cast<char *>(d_ws) + L.offsets + sizeof(int64_t) * static_cast<size_t>(n),
                        sizeof(int64_t), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return VOX_ERR_CUDA;
    if (cudaMemcpyAsync(&st, d_status, sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess) return VOX_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return VOX_ERR_CUDA;
    if (h_total) *h_total = V;
    if (st != VOX_OK) return static_cast<vox_status>(st);
    if (has_list && V > list_capacity) return VOX_ERR_CAPACITY;
    BrickGeom G;
    const bool bricks = bm && n > 0 && current_tuning().volume_path == VOX_VOLUME_AUTO &&
                        uses_bricks(n, dims, ws_bytes, &G);
    if (!bricks) {
        // one pass produces the list and the (cleared) volume together
        if (bm && cudaMemsetAsync(d_mask, 0, 4 * static_cast<size_t>(words), s) != cudaSuccess) return VOX_ERR_CUDA;
        if (vox_status e = launch_generate(d_segs, n, dims, d_list, list_capacity, d_mask, flags, d_ws, d_status, s))
            return e;
        if (has_list && V > 0 &&
            cudaMemcpyAsync(h_list, d_list, elem * static_cast<size_t>(V), cudaMemcpyDeviceToHost, s) != cudaSuccess)
            return VOX_ERR_CUDA;
        if (bm && cudaMemcpyAsync(h_mask, d_mask, 4 * static_cast<size_t>(words), cudaMemcpyDeviceToHost, s) !=
                      cudaSuccess)
            return VOX_ERR_CUDA;
    } else {
        // the list first; its copy to the host runs on a second stream while the
        // brick-built (fresh) volume is computed, then the volume's copy
        cudaStream_t s2 = has_list && V > 0 ? copy_stream() : nullptr;
        if (has_list && V > 0 && s2 == nullptr) return VOX_ERR_CUDA;
        cudaEvent_t listed = nullptr, copied = nullptr;
        auto cleanup = [&]() {
            if (listed) cudaEventDestroy(listed);
            if (copied) cudaEventDestroy(copied);
        };
        const int list_flags = flags & (VOX_OUT_LIST32 | VOX_OUT_LIST64);
        if (list_flags) {
            if (vox_status e = launch_generate(d_segs, n, dims, d_list, list_capacity, nullptr, list_flags, d_ws,
                                               d_status, s))
                return e;
        }
        if (s2 != nullptr) {
            if (cudaEventCreateWithFlags(&listed, cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreateWithFlags(&copied, cudaEventDisableTiming) != cudaSuccess ||
                cudaEventRecord(listed, s) != cudaSuccess || cudaStreamWaitEvent(s2, listed, 0) != cudaSuccess ||
                cudaMemcpyAsync(h_list, d_list, elem * static_cast<size_t>(V), cudaMemcpyDeviceToHost, s2) !=
                    cudaSuccess ||
                cudaEventRecord(copied, s2) != cudaSuccess) {
                cleanup();
                return VOX_ERR_CUDA;
            }
        }
        if (vox_status e = launch_bricks(d_segs, n, G, dims, d_mask, d_ws, ws_bytes, d_status, s, false, true)) {
            if (copied) cudaStreamWaitEvent(s, copied, 0);
            cudaStreamSynchronize(s);
            cleanup();
            return e;
        }
        const bool ok =
            cudaMemcpyAsync(h_mask, d_mask, 4 * static_cast<size_t>(words), cudaMemcpyDeviceToHost, s) == cudaSuccess &&
            (copied == nullptr || cudaStreamWaitEvent(s, copied, 0) == cudaSuccess);
        if (!ok) {
            cudaStreamSynchronize(s);
            if (s2) cudaStreamSynchronize(s2);
            cleanup();
            return VOX_ERR_CUDA;
        }
        cleanup();  // destroying a recorded event is allowed; the wait above holds
    }
    if (cudaMemcpyAsync(&st, d_status, sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess) return VOX_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return VOX_ERR_CUDA;
    return static_cast<vox_status>(st);
}

const char *vox_strerror(int status)
{
    switch (status) {
    case VOX_OK: return "ok";
    case VOX_ERR_INVALID_ARG: return "invalid argument";
    case VOX_ERR_OUT_OF_BOUNDS: return "segment endpoint outside the volume";
    case VOX_ERR_PACK_WIDTH: return "32-bit list needs every volume edge <= 1024";
    case VOX_ERR_CAPACITY: return "list capacity below the total voxel count";
    case VOX_ERR_TIMEOUT: return "bounded in-kernel wait expired";
    case VOX_ERR_CUDA: return "CUDA runtime error";
    case VOX_ERR_WORKSPACE: return "workspace missing, misaligned or too small";
    case VOX_ERR_ALIGNMENT: return "buffer misaligned (segments and lists need 16 bytes)";
    default: return "unknown status";
    }
}

void vox_set_tuning(const vox_tuning *t)
{
    std::lock_guard<std::mutex> lock(g_tuning_mu);
    if (t == nullptr) {
        g_tuning = vox_tuning{0, 0, 0, 0};
        return;
    }
    g_tuning = *t;
    if (g_tuning.run_len != 16 && g_tuning.run_len != 32 && g_tuning.run_len != 64) g_tuning.run_len = 0;
    if (g_tuning.volume_path < 0 || g_tuning.volume_path > VOX_VOLUME_ATOMIC_WARP) g_tuning.volume_path = 0;
    if (g_tuning.ctas_per_sm < 0) g_tuning.ctas_per_sm = 0;
    if (g_tuning.list_runs != 1 && g_tuning.list_runs != 2) g_tuning.list_runs = 0;
}

void vox_get_tuning(vox_tuning *t)
{
    if (t) *t = current_tuning();
}

void vox_debug_set_scan_stall(int64_t tile, int64_t wait_ns)
{
    g_stall_tile.store(tile < 0 ? -1 : tile);
    g_wait_ns.store(wait_ns > 0 ? wait_ns : kDefaultWaitNs);
}

}  // extern "C"
