// vox_bricks.cuh -- the occupancy volume by brick ownership (sm_103a).
//
// OR-ing each voxel into the volume with a global atomic costs one L2/DRAM
// read-modify-write of a 32-byte sector per voxel (the volume is far larger than
// L2 for big scenes), which makes the volume store DRAM-bound at a small fraction
// of the bandwidth. Instead the volume is cut into bricks of whole 32-bit words
// (B0 x B1 x B2 voxels, B0 a multiple of 32, at most 8192 words), every segment
// is cut into pieces that stay inside one brick, the pieces are counting-sorted
// by brick, and one CTA owns each brick: it ORs the brick's voxels into a
// shared-memory bitmap and merges the bitmap into the volume with one coalesced
// read-modify-write per touched word. Each volume sector then crosses DRAM at
// most twice (read + write), whatever the number of voxels in it.
//
//   k_bin_count    pieces per brick (one thread per segment, global atomics)
//   k_scan<false>  exclusive scan of the per-brick counts (decoupled look-back)
//   k_bin_scatter  pieces written into their brick's bucket
//   k_brick_volume one CTA per brick: voxels -> shared bitmap -> volume
//
// A piece is (segment, first step k, length). The steps at which a segment's
// coordinate on an axis enters the next brick follow from the same exact rounding
// as the voxels themselves (Eq. (3) with nearest-lattice rounding): the offset
// q(k) = floor((2 k A + N) / (2 N)) first reaches Q at k = ceil(N (2Q - 1) / (2A)).
#pragma once

#include <cstdint>

#include "vox_device.cuh"

namespace vox {

constexpr int kBrickThreads = 256;
constexpr int kBrickWordsMax = 8192;  // 32 KB shared bitmap per brick
constexpr int32_t kNoStep = 0x7fffffff;

struct BrickGeom {
    int32_t B[3];       // brick extent in voxels per axis (B[0] a multiple of 32)
    int32_t nb[3];      // bricks per axis
    int32_t bxw;        // words per brick row, B[0] / 32
    int32_t row_words;  // words per volume row, w / 32
    int32_t dim[3];     // volume extent
    int32_t words;      // words per brick, bxw * B[1] * B[2]
    int64_t n_bricks;
};

__device__ __forceinline__ int64_t brick_index(const BrickGeom &G, int32_t b0, int32_t b1, int32_t b2)
{
    return b0 + static_cast<int64_t>(G.nb[0]) * (b1 + static_cast<int64_t>(G.nb[1]) * b2);
}

// Smallest step k with floor((2 k A + N) / (2 N)) >= Q, for 1 <= Q <= A <= N:
// k = ceil(N (2Q - 1) / (2A)).
__device__ __forceinline__ int32_t first_step_reaching(int32_t A, int32_t N, int32_t Q)
{
    if (N <= 46340) {  // N (2Q - 1) + 2A - 1 < 2 N^2 + 2N < 2^32
        const uint32_t num = static_cast<uint32_t>(N) * static_cast<uint32_t>(2 * Q - 1);
        const uint32_t den = 2u * static_cast<uint32_t>(A);
        return static_cast<int32_t>((num + den - 1u) / den);
    }
    const uint64_t num = static_cast<uint64_t>(N) * static_cast<uint64_t>(2 * Q - 1);
    const uint64_t den = 2ull * static_cast<uint64_t>(A);
    return static_cast<int32_t>((num + den - 1ull) / den);
}

// Calls f(brick, k_lo, len) for every maximal run of consecutive steps of the
// segment that stays in one brick, in increasing k. Endpoints must be inside
// the volume.
template <typename F>
__device__ __forceinline__ void for_each_piece(const int32_t *rec, const BrickGeom &G, F &&f)
{
    int32_t S[3], A[3], b0[3], b[3], dir[3], left[3], j[3], nk[3];
    int32_t N = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        S[a] = rec[a];
        const int32_t d = rec[3 + a] - rec[a];
        A[a] = abs(d);
        N = max(N, A[a]);
        b0[a] = S[a] / G.B[a];
        const int32_t be = rec[3 + a] / G.B[a];
        b[a] = b0[a];
        dir[a] = be > b0[a] ? 1 : (be < b0[a] ? -1 : 0);
        left[a] = abs(be - b0[a]);
        j[a] = 1;
    }
    // step at which axis a enters its next brick (the j-th crossing)
    auto next_cross = [&](int a) -> int32_t {
        if (left[a] == 0) return kNoStep;
        const int32_t Q = dir[a] > 0 ? (b0[a] + j[a]) * G.B[a] - S[a] : S[a] - ((b0[a] - j[a] + 1) * G.B[a] - 1);
        return first_step_reaching(A[a], N, Q);
    };
#pragma unroll
    for (int a = 0; a < 3; ++a) nk[a] = next_cross(a);
    int32_t k = 0;
    while (true) {
        const int32_t kn = min(min(nk[0], nk[1]), min(nk[2], N + 1));
        f(brick_index(G, b[0], b[1], b[2]), k, kn - k);
        if (kn > N) break;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (nk[a] == kn) {
                b[a] += dir[a];
                --left[a];
                ++j[a];
                nk[a] = next_cross(a);
            }
        }
        k = kn;
    }
}

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
    int32_t *brick_count;     // [n_bricks], zeroed before k_bin_count
    int64_t *cursor;          // [n_bricks], exclusive offsets (k_bin_scatter bumps them)
    const int64_t *brick_off; // [n_bricks + 1]; brick_off[n_bricks] = number of pieces
    uint64_t *pieces;         // [capacity]
    int64_t capacity;
    const int32_t *status;
};

__device__ __forceinline__ void load_record(const int32_t *segs, int64_t s, int32_t *r)
{
    const int2 *p = reinterpret_cast<const int2 *>(segs + 6 * s);
    const int2 a = __ldg(p), b = __ldg(p + 1), c = __ldg(p + 2);
    r[0] = a.x; r[1] = a.y; r[2] = b.x; r[3] = b.y; r[4] = c.x; r[5] = c.y;
}

__global__ void __launch_bounds__(256) k_bin_count(BinParams p)
{
    if (ld_volatile_i32(p.status) != 0) return;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t s = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; s < p.n; s += stride) {
        int32_t r[6];
        load_record(p.segs, s, r);
        if (!endpoints_inside(r, p.G)) continue;  // reported by the count kernel
        for_each_piece(r, p.G, [&](int64_t b, int32_t, int32_t) { atomicAdd(p.brick_count + b, 1); });
    }
}

__global__ void __launch_bounds__(256) k_bin_scatter(BinParams p)
{
    if (ld_volatile_i32(p.status) != 0) return;
    if (__ldg(p.brick_off + p.G.n_bricks) > p.capacity) return;  // the volume falls back to atomics
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t s = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; s < p.n; s += stride) {
        int32_t r[6];
        load_record(p.segs, s, r);
        if (!endpoints_inside(r, p.G)) continue;
        for_each_piece(r, p.G, [&](int64_t b, int32_t k, int32_t len) {
            const unsigned long long pos =
                atomicAdd(reinterpret_cast<unsigned long long *>(p.cursor + b), 1ull);
            p.pieces[pos] = pack_piece(s, k, len);
        });
    }
}

struct BrickParams {
    const int32_t *segs;
    BrickGeom G;
    const int64_t *brick_off;  // [n_bricks + 1]
    const uint64_t *pieces;
    int64_t capacity;
    uint32_t *mask;
    const int32_t *status;
    uint32_t *ticket;  // zeroed before launch
};

__global__ void __launch_bounds__(kBrickThreads) k_brick_volume(BrickParams p)
{
    __shared__ __align__(16) uint32_t bits[kBrickWordsMax];
    __shared__ int64_t s_brick;
    const int t = threadIdx.x;
    if (ld_volatile_i32(p.status) != 0) return;
    if (__ldg(p.brick_off + p.G.n_bricks) > p.capacity) return;  // pieces did not fit: atomics path
    const BrickGeom &G = p.G;
    const uint32_t bw = static_cast<uint32_t>(G.B[0]);
    const uint32_t bwh = static_cast<uint32_t>(G.B[0]) * static_cast<uint32_t>(G.B[1]);
    while (true) {
        if (t == 0) s_brick = atomicAdd(p.ticket, 1u);
        __syncthreads();
        const int64_t b = s_brick;
        __syncthreads();  // s_brick is rewritten only after everyone has read it
        if (b >= G.n_bricks) break;
        const int64_t lo = __ldg(p.brick_off + b), hi = __ldg(p.brick_off + b + 1);
        if (lo == hi) continue;
        const int32_t i0 = static_cast<int32_t>(b % G.nb[0]);
        const int64_t rest = b / G.nb[0];
        const int32_t i1 = static_cast<int32_t>(rest % G.nb[1]);
        const int32_t i2 = static_cast<int32_t>(rest / G.nb[1]);
        const int32_t X0 = i0 * G.B[0], Y0 = i1 * G.B[1], Z0 = i2 * G.B[2];
        for (int q = t; q < G.words; q += kBrickThreads) bits[q] = 0u;
        __syncthreads();
        // brick-local bit index of (x, y, z): (x - X0) + B0 (y - Y0) + B0 B1 (z - Z0),
        // kept modulo 2^32 while stepping (only the local value is ever used)
        const uint32_t origin = static_cast<uint32_t>(X0) + static_cast<uint32_t>(Y0) * bw +
                                static_cast<uint32_t>(Z0) * bwh;
        for (int64_t pi = lo + t; pi < hi; pi += kBrickThreads) {
            const uint64_t pc = __ldg(p.pieces + pi);
            const int64_t seg = static_cast<int64_t>(pc & 0xffffffffull);
            const int32_t k_lo = static_cast<int32_t>((pc >> 32) & 0x3fffffull);
            const int32_t len = static_cast<int32_t>(pc >> 54) + 1;
            int32_t r[6];
            load_record(p.segs, seg, r);
            Stepper<uint32_t, uint32_t> st;
            st.enter(r, k_lo, bw, bwh);
            st.L -= origin;
            uint32_t cur = 0xffffffffu, acc = 0;
            for (int32_t e = 0; e < len; ++e) {
                const uint32_t word = st.L >> 5;
                if (word != cur) {
                    if (acc) atomicOr(bits + cur, acc);
                    cur = word;
                    acc = 0;
                }
                acc |= 1u << (st.L & 31u);
                st.template step<false, true>();
            }
            if (acc) atomicOr(bits + cur, acc);
        }
        __syncthreads();
        // merge into the volume: brick row (ly, lz) holds bxw words that are
        // contiguous in the volume; only touched words are read and written
        for (int q = t; q < G.words; q += kBrickThreads) {
            const uint32_t v = bits[q];
            if (v == 0) continue;
            const int32_t row = q / G.bxw, col = q - row * G.bxw;
            const int32_t y = Y0 + row % G.B[1], z = Z0 + row / G.B[1];
            if (y >= G.dim[1] || z >= G.dim[2] || X0 / 32 + col >= G.row_words) continue;
            const int64_t gw = X0 / 32 + col + static_cast<int64_t>(G.row_words) *
                                                    (y + static_cast<int64_t>(G.dim[1]) * z);
            p.mask[gw] |= v;  // the brick owns these words: no other writer
        }
        __syncthreads();
    }
}

}  // namespace vox
