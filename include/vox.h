/*
 * vox.h -- C ABI of libvox, a GB300 (sm_103a) library for parametric voxel
 * generation of 3D straight-line segments.
 *
 * The operation (Section 3 of "3D Primitives GPGPU Generation for Volume
 * Visualization in 3D Graphics Systems", Eq. (2)-(3) and Fig. 3):
 *   a segment from S = (x0, y0, z0) to E = (x1, y1, z1) (integer endpoints) has
 *   N = max(|x1 - x0|, |y1 - y0|, |z1 - z0|) steps and N + 1 voxels; voxel k
 *   (k = 0..N) is the lattice point nearest to G_k = S + (E - S) k / N on each
 *   axis, a coordinate exactly half-way between two integers going to the one
 *   farther from S. In integers, per axis a with d_a = E_a - S_a:
 *     q_a(k) = floor((2 k |d_a| + N) / (2 N)),  v_a(k) = S_a + sign(d_a) q_a(k).
 *   N = 0 gives the single voxel S. All arithmetic is exact.
 *
 * Outputs (all optional, any combination; OR the VOX_OUT_* flags):
 *   VOX_OUT_LIST32   uint32 per voxel: x | y << 10 | z << 20   (every dim <= 1024)
 *   VOX_OUT_LIST64   uint64 per voxel: x | y << 21 | z << 42
 *   VOX_OUT_BITMASK  occupancy volume, one bit per voxel: voxel (x, y, z) is bit
 *                    b = x + w*(y + h*z), i.e. bit (b % 32) of uint32 word b / 32;
 *                    ceil(w*h*d / 32) words. Bits are OR-ed in: the caller clears
 *                    the volume when it wants a fresh one, or adds VOX_OUT_FRESH.
 *   VOX_OUT_FRESH    (with VOX_OUT_BITMASK only) the call writes the whole volume:
 *                    afterwards it holds exactly these segments' voxels, whatever
 *                    it held before. The brick path stores each brick whole
 *                    (no read of the old volume); the other paths clear the volume
 *                    first. If the call fails on the device (*d_status != 0), the
 *                    volume is either unchanged or cleared.
 *   VOX_OUT_BRICKED  (with VOX_OUT_BITMASK only) the volume in brick-major layout,
 *                    written whole like VOX_OUT_FRESH: brick (bx, by, bz) of
 *                    vox_brick_shape's B0 x B1 x B2 voxels is the `words` =
 *                    B0*B1*B2/32 words at index (bx + nb0 (by + nb1 bz)) * words,
 *                    and inside it voxel (lx, ly, lz) is bit lx + B0 (ly + B1 lz)
 *                    (x fastest; edge bricks padded with zero bits);
 *                    vox_mask_words_bricked(dims) words, 16-byte aligned. Each
 *                    brick leaves the GPU as one contiguous bulk copy.
 *                    vox_unbrick converts to the row-major layout. Needs a width
 *                    that is a multiple of 32 and a brick workspace
 *                    (vox_workspace_size_volume; VOX_ERR_WORKSPACE otherwise, and
 *                    on the device when more pieces than its capacity arise);
 *                    not accepted by vox_generate_batched / vox_generate_host.
 *   The list holds the voxels of segment 0 (k = 0..N), then segment 1, and so on:
 *   voxel k of segment s sits at index offsets[s] + k, offsets being the exclusive
 *   prefix sum of the per-segment counts N + 1. Voxels shared by two segments
 *   appear twice in a list and once in the volume.
 *
 * Conventions for every call:
 *   - Pointers named d_* or documented as "device" are CUDA device pointers on
 *     the current device; h_* are host pointers. The caller allocates and owns
 *     every buffer; the library allocates nothing and keeps no state between
 *     calls except a per-device cache of launch limits.
 *   - Calls are asynchronous on `stream` (a cudaStream_t passed as void*; NULL
 *     means the legacy default stream) unless documented otherwise, and never
 *     synchronise the device.
 *   - Errors the host can see (bad pointer, size, flag, alignment, workspace too
 *     small) are returned at once and nothing is launched. Errors found on the
 *     device are written to *d_status (a device int32 that the call first sets
 *     to VOX_OK); the first error wins. Once *d_status holds an error, the
 *     generation kernels of that call write nothing at all (list and volume are
 *     left untouched). Read *d_status after synchronising the stream.
 *   - Segment arrays are vox_segment[n] (24 bytes each, int32), device memory,
 *     16-byte aligned. Every endpoint must lie in [0, dim) of its axis, and
 *     every dim in [1, 2^21].
 */
#ifndef VOX_H
#define VOX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum vox_status {
    VOX_OK = 0,
    VOX_ERR_INVALID_ARG = 1,   /* NULL pointer, n < 0, bad flags, dims outside [1, 2^21] */
    VOX_ERR_OUT_OF_BOUNDS = 2, /* (device) an endpoint lies outside [0, dim) */
    VOX_ERR_PACK_WIDTH = 3,    /* LIST32 requested with a dim above 1024 */
    VOX_ERR_CAPACITY = 4,      /* (device) list capacity below the total voxel count */
    VOX_ERR_TIMEOUT = 5,       /* (device) a bounded wait inside a kernel expired */
    VOX_ERR_CUDA = 6,          /* a CUDA runtime call or launch failed */
    VOX_ERR_WORKSPACE = 7,     /* workspace NULL, too small or not 256-byte aligned; (device)
                                  brick-major volume with more pieces than the workspace holds */
    VOX_ERR_ALIGNMENT = 8      /* segments not 16-byte aligned, list/volume misaligned */
} vox_status;

typedef struct vox_segment {
    int32_t x0, y0, z0; /* start point S */
    int32_t x1, y1, z1; /* end point E */
} vox_segment;

typedef struct vox_dims {
    int32_t w, h, d; /* volume extent along x, y, z, in voxels */
} vox_dims;

#define VOX_OUT_LIST32 1
#define VOX_OUT_LIST64 2
#define VOX_OUT_BITMASK 4
#define VOX_OUT_FRESH 8
#define VOX_OUT_BRICKED 16

/* Bytes of workspace a call on n segments needs (count, scan and generation of
 * one scene). The workspace is device memory, 256-byte aligned, caller-owned,
 * and may be reused by the next call on the same stream. */
size_t vox_workspace_size(int64_t n_segments);

/*
 * vox_count -- per-segment voxel counts N + 1 and their exclusive prefix sum
 * (the preprocessing of Section 4, step 1, and the lengths N_i of the
 * multi-segment case). Validates every endpoint against dims.
 *   d_segs     device vox_segment[n], 16-byte aligned
 *   n          number of segments (0 allowed)
 *   dims       volume extent (each in [1, 2^21])
 *   d_counts   device int32[n] receiving N + 1, or NULL
 *   d_offsets  device int64[n + 1] receiving the exclusive prefix sum, with the
 *              total voxel count V in d_offsets[n], or NULL
 *   d_ws       workspace of vox_workspace_size(n) bytes; it also keeps the
 *              offsets for a following vox_generate_from_scan
 *   d_status   device int32, set to VOX_OK then to the first device error
 *   stream     cudaStream_t as void*
 */
vox_status vox_count(const vox_segment *d_segs, int64_t n, vox_dims dims,
                     int32_t *d_counts, int64_t *d_offsets,
                     void *d_ws, size_t ws_bytes, int32_t *d_status, void *stream);

/*
 * vox_generate -- the whole method on one scene: counts, exclusive scan, then
 * every voxel of every segment (Fig. 3 for all segments at once, Section 4),
 * written to the requested outputs.
 *   d_segs, n, dims  as for vox_count
 *   d_list           device list (uint32 for LIST32, uint64 for LIST64; 16-byte
 *                    aligned) or NULL when no list flag is set
 *   list_capacity    elements available in d_list; V above it is
 *                    VOX_ERR_CAPACITY (device) and nothing is written
 *   d_mask           device uint32[ceil(w*h*d/32)], 4-byte aligned, OR-ed into
 *                    (overwritten with VOX_OUT_FRESH); NULL when
 *                    VOX_OUT_BITMASK is not set
 *   flags            VOX_OUT_LIST32 or VOX_OUT_LIST64 (not both), optionally
 *                    | VOX_OUT_BITMASK (| VOX_OUT_FRESH); at least one output
 *   d_ws, ws_bytes   workspace of at least vox_workspace_size(n) bytes
 *   d_status         as for vox_count
 */
vox_status vox_generate(const vox_segment *d_segs, int64_t n, vox_dims dims,
                        void *d_list, int64_t list_capacity, uint32_t *d_mask, int flags,
                        void *d_ws, size_t ws_bytes, int32_t *d_status, void *stream);

/*
 * vox_count_bins -- the brick binning's counting pass alone: pieces per brick
 * slot, the part of vox_count that runs when ws_bytes covers the brick arrays
 * (vox_workspace_size_volume). With vox_count given ws_bytes =
 * vox_workspace_size(n) (count + scan only) the two passes can run on two
 * streams: they read only the segments and write disjoint workspace parts. A
 * volume generated after both then needs the full ws_bytes and a stream ordered
 * after both. Asynchronous; does not touch the status word (segments with
 * endpoints outside the volume are skipped; vox_count reports them).
 * VOX_ERR_WORKSPACE when the workspace does not hold the brick arrays.
 */
vox_status vox_count_bins(const vox_segment *d_segs, int64_t n, vox_dims dims, void *d_ws, size_t ws_bytes,
                          void *stream);

/*
 * vox_generate_from_scan -- the generation step alone, reusing the counts and
 * offsets that a preceding vox_count left in d_ws for the same d_segs, n and
 * dims, on the same stream (or on a stream ordered after it). Does not reset
 * *d_status: an error found by that vox_count keeps this call from writing
 * anything. Arguments as for vox_generate.
 * After one vox_count, a list-only call (VOX_OUT_LIST32/64) and a volume-only
 * call (VOX_OUT_BITMASK) may run concurrently on two streams: the list reads
 * the scanned offsets, the volume reads them and writes only the brick arrays
 * that follow them in the workspace, and errors are recorded first-wins.
 */
vox_status vox_generate_from_scan(const vox_segment *d_segs, int64_t n, vox_dims dims,
                                  void *d_list, int64_t list_capacity, uint32_t *d_mask,
                                  int flags, void *d_ws, size_t ws_bytes, int32_t *d_status,
                                  void *stream);

/*
 * The Euclidean-N variant (Section 3, Eq. (1)-(2) read literally): N =
 * int(|E - S|), the integer part of the Euclidean length, instead of
 * max |d_a|; samples G_k = S + W k, W = (E - S) / N, k = 0..N, each mapped to
 * its nearest lattice point with the same rounding (ties away from S). Since N
 * can exceed max |d_a|, consecutive samples can share a voxel; a voxel equal to
 * the previous sample's is not added again (the voxel set of Fig. 3). The
 * output of a segment is therefore between max|d_a| + 1 and N + 1 voxels, not
 * known before the call: vox_euclid_plan returns the total for sizing.
 *   vox_euclid_workspace_size  workspace bytes for n segments (the sample scan
 *                              plus max(n, 2^20) run slots, 12 B each)
 *   vox_euclid_workspace_size_volume  the same followed by the brick arrays and
 *                              room for piece_capacity pieces (e.g. *h_pieces of
 *                              vox_euclid_plan): with it the volume is built by
 *                              bricks (falling back to atomics on the device when
 *                              the pieces do not fit)
 *   vox_euclid_generate        as vox_generate (same outputs and flags except
 *                              VOX_OUT_BRICKED; the volume by bricks when the
 *                              workspace holds them, else per-voxel atomics),
 *                              asynchronous; d_offsets: device int64[n + 1] that
 *                              receives each segment's first list position and
 *                              the total at [n], or NULL. A list capacity below
 *                              the total is VOX_ERR_CAPACITY (device), nothing
 *                              written.
 *   vox_euclid_plan            SYNCHRONOUS: the total voxel count (*h_voxels),
 *                              the total sample count (*h_samples) and the brick
 *                              pieces (*h_pieces, 0 unless the workspace holds the
 *                              brick arrays), each may be NULL; returns the
 *                              device status (e.g. VOX_ERR_OUT_OF_BOUNDS).
 */
size_t vox_euclid_workspace_size(int64_t n);
size_t vox_euclid_workspace_size_volume(int64_t n, vox_dims dims, int64_t piece_capacity);
vox_status vox_euclid_generate(const vox_segment *d_segs, int64_t n, vox_dims dims, void *d_list,
                               int64_t list_capacity, uint32_t *d_mask, int flags, int64_t *d_offsets, void *d_ws,
                               size_t ws_bytes, int32_t *d_status, void *stream);
vox_status vox_euclid_plan(const vox_segment *d_segs, int64_t n, vox_dims dims, void *d_ws, size_t ws_bytes,
                           int32_t *d_status, int64_t *h_voxels, int64_t *h_samples, int64_t *h_pieces,
                           void *stream);

/*
 * Brick-major volumes (VOX_OUT_BRICKED). The brick geometry depends on dims only:
 * B0 = the largest 32 * 2^k not above min(w, 256), then B1 x B2 power-of-two
 * rows (B1 = 2 B2 or B2) with B0/32 * B1 * B2 <= 32768 words; w % 32 == 0.
 *   vox_mask_words_bricked  words of the brick-major volume (0: no geometry)
 *   vox_brick_shape         h_shape[0..5] = B0, B1, B2, nb0, nb1, nb2 (host
 *                           int32[6]); VOX_ERR_INVALID_ARG when w % 32 != 0
 *   vox_unbrick             device brick-major volume -> device row-major volume
 *                           (vox_mask_words(dims) words), asynchronous on stream;
 *                           half bricks through TMA when w and B0 are multiples of
 *                           128 and both buffers 16-byte aligned (its bounded
 *                           waits report VOX_ERR_TIMEOUT to d_status, which may be
 *                           NULL), else one warp per volume row
 */
int64_t vox_mask_words_bricked(vox_dims dims);
vox_status vox_brick_shape(vox_dims dims, int32_t *h_shape);
vox_status vox_unbrick(const uint32_t *d_bricked, vox_dims dims, uint32_t *d_mask, int32_t *d_status, void *stream);

/*
 * The occupancy volume can be built two ways; vox_generate picks one from the
 * workspace it is given:
 *   - by brick ownership (volumes whose width w is a multiple of 32): the volume
 *     is cut into bricks of whole words, each segment into pieces that stay in
 *     one brick, the pieces are sorted by brick, and one CTA per brick ORs its
 *     voxels in shared memory and merges them into the volume, so that each
 *     volume sector is read and written once. Needs a workspace of at least
 *     vox_workspace_size_volume(n, dims, P) bytes with P >= the number of pieces
 *     (vox_plan reports it). If the pieces turn out not to fit, the same call
 *     falls back, on the device, to the per-voxel atomic path (same result).
 *   - by per-voxel atomic ORs of deduplicated words: any volume, any workspace
 *     of at least vox_workspace_size(n) bytes.
 * Both give the same bits. With the brick path the volume's words are written
 * with plain read-modify-writes: calls that write the same volume must not
 * overlap on the GPU.
 *
 * vox_workspace_size_volume -- workspace bytes for n segments in a volume of
 * `dims` with room for `piece_capacity` pieces (falls back to
 * vox_workspace_size(n) when the volume cannot use bricks).
 */
size_t vox_workspace_size_volume(int64_t n, vox_dims dims, int64_t piece_capacity);

/*
 * vox_plan -- SYNCHRONOUS sizing helper: runs the count, the scan and the
 * brick binning count on the device and returns the total voxel count V and
 * the number of brick pieces (0 when the volume cannot use bricks), so that
 * the caller can size the list and the workspace of a following vox_generate.
 *   d_ws   at least vox_workspace_size_volume(n, dims, 0) bytes
 *   returns VOX_OK or the first error (host or device)
 */
vox_status vox_plan(const vox_segment *d_segs, int64_t n, vox_dims dims, void *d_ws, size_t ws_bytes,
                    int32_t *d_status, int64_t *h_voxels, int64_t *h_pieces, void *stream);

/*
 * Batched scenes (many independent problems in one launch sequence, Section 5's
 * conclusion 3: few kernel calls, many segments per call).
 *
 * A batch is one segment array holding the scenes' segments back to back, and a
 * DEVICE table of n_scenes vox_scene entries: scene k covers segments
 * [seg_begin, seg_begin + n), seg_begin of scene 0 is 0, each scene starts where
 * the previous one ends, and the last ends at n_total (checked on the device:
 * VOX_ERR_INVALID_ARG in *d_status, nothing written).
 */
typedef struct vox_scene {
    int64_t seg_begin; /* first segment of the scene in the batch's segment array */
    int64_t n;         /* segments of the scene */
    vox_dims dims;     /* the scene's volume extent (each in [1, 2^21]) */
    int32_t reserved;  /* must be 0 */
    uint32_t *mask;    /* the scene's volume (ceil(w*h*d/32) words, OR-ed into), or NULL */
} vox_scene;           /* 40 bytes */

/* Workspace bytes for a batch of n_total segments in n_scenes scenes. */
size_t vox_workspace_size_batched(int64_t n_total, int32_t n_scenes);

/*
 * vox_generate_batched -- count, scan and generate every scene of a batch with
 * one launch per step (scene map, count + scan, scene bases, list, volumes),
 * whatever the number of scenes; suitable for capture in a CUDA graph.
 *   d_segs          device vox_segment[n_total], 16-byte aligned
 *   d_scenes        device vox_scene[n_scenes], 8-byte aligned
 *   d_list          ONE list for the whole batch (LIST32 or LIST64 in flags):
 *                   scene k's voxels are at [base[k], base[k+1]), in segment
 *                   order, k = 0..N per segment; list_capacity elements; every
 *                   scene must have edges <= 1024 for LIST32
 *   flags           list format and/or VOX_OUT_BITMASK (each scene's voxels are
 *                   OR-ed into that scene's mask; scenes with mask NULL skip it);
 *                   VOX_OUT_FRESH clears every scene's mask first
 *   d_scene_base    device int64[n_scenes + 1] receiving base[k] (first voxel of
 *                   scene k in the list) and base[n_scenes] = total V, or NULL
 *   d_ws, ws_bytes  at least vox_workspace_size_batched(n_total, n_scenes)
 *   d_status        as for vox_generate
 * The volumes are built by per-voxel deduplicated atomic ORs over voxel tiles
 * dealt round-robin to the CTAs, so that the scenes in flight at any moment are
 * few and their volumes stay in L2.
 */
vox_status vox_generate_batched(const vox_segment *d_segs, int64_t n_total, const vox_scene *d_scenes,
                                int32_t n_scenes, void *d_list, int64_t list_capacity, int flags,
                                int64_t *d_scene_base, void *d_ws, size_t ws_bytes, int32_t *d_status,
                                void *stream);

/*
 * Batched volumes by bricks (the brick path of the single-scene volume, over
 * all scenes at once; one counter replica, bricks merged by plain stores):
 *   vox_scene_bricks   bricks of one scene's volume (its width a multiple of
 *                      32), 0 when it cannot take bricks; host-only
 *   vox_workspace_size_batched_volume  the batched workspace followed by the
 *                      brick arrays of total_bricks bricks and piece_capacity
 *                      pieces (vox_plan_batched gives the count)
 *   vox_generate_batched_ex  vox_generate_batched with total_bricks = the sum of
 *                      vox_scene_bricks over the scenes (every scene must take
 *                      bricks; a different sum on the device is
 *                      VOX_ERR_INVALID_ARG): with such a workspace the volumes
 *                      are built by bricks, pieces beyond the capacity by the
 *                      batched atomics on the device; total_bricks = 0 or a
 *                      smaller workspace gives vox_generate_batched exactly
 *   vox_plan_batched   SYNCHRONOUS: total voxels and brick pieces of a batch
 *                      (pieces 0 when total_bricks is 0)
 */
int64_t vox_scene_bricks(vox_dims dims);
size_t vox_workspace_size_batched_volume(int64_t n_total, int32_t n_scenes, int64_t total_bricks,
                                         int64_t piece_capacity);
vox_status vox_generate_batched_ex(const vox_segment *d_segs, int64_t n_total, const vox_scene *d_scenes,
                                   int32_t n_scenes, int64_t total_bricks, void *d_list, int64_t list_capacity,
                                   int flags, int64_t *d_scene_base, void *d_ws, size_t ws_bytes, int32_t *d_status,
                                   void *stream);
vox_status vox_plan_batched(const vox_segment *d_segs, int64_t n_total, const vox_scene *d_scenes, int32_t n_scenes,
                            int64_t total_bricks, void *d_ws, size_t ws_bytes, int32_t *d_status, int64_t *h_voxels,
                            int64_t *h_pieces, void *stream);

/*
 * vox_generate_host -- vox_generate on host buffers, copies included (the
 * host-device pipeline of Fig. 4: input copy, kernels, result copy back).
 * SYNCHRONOUS: returns once the results are in host memory (it synchronises
 * `stream` twice: once to learn V, once at the end).
 *   h_segs          host vox_segment[n] (pinned memory for full copy speed)
 *   h_list          host list of list_capacity elements, or NULL
 *   h_mask          host uint32[ceil(w*h*d/32)], OVERWRITTEN with the volume of
 *                   these segments alone (not OR-ed; VOX_OUT_FRESH changes
 *                   nothing here), or NULL
 *   d_arena         device scratch of at least vox_host_arena_size(...) bytes,
 *                   256-byte aligned. With vox_host_arena_size_volume(...) bytes
 *                   (room for the brick arrays and piece_capacity pieces, e.g.
 *                   the count vox_plan returns) the volume is built by bricks and
 *                   the list's copy to the host overlaps the volume's kernels on
 *                   a second stream (created once per device by the library);
 *                   with fewer pieces than needed the volume falls back to
 *                   atomics on the device, same result.
 *   h_total         receives V (may be NULL)
 *   returns         VOX_OK or the first error, host or device
 */
size_t vox_host_arena_size(int64_t n, vox_dims dims, int flags, int64_t list_capacity);
size_t vox_host_arena_size_volume(int64_t n, vox_dims dims, int flags, int64_t list_capacity,
                                  int64_t piece_capacity);
vox_status vox_generate_host(const vox_segment *h_segs, int64_t n, vox_dims dims,
                             void *h_list, int64_t list_capacity, uint32_t *h_mask, int flags,
                             void *d_arena, size_t arena_bytes, int64_t *h_total, void *stream);

/*
 * vox_probe_red_or -- measurement helper; the paper has no counterpart. The
 * per-voxel atomic volume issues one 32-bit OR reduction (red.or, result not
 * returned, L2 asked to keep the line) per merged word; this call issues about
 * `ops` of them at pseudo-random words of d_buf (words 32-bit words, at most
 * 2^32; a per-thread linear congruential sequence from `seed` picks word and
 * bit), on SMs x 8 CTAs of 256 threads, asynchronously on `stream`, so that a
 * caller timing it with events gets the GPU's reduction throughput for a
 * buffer of that size (L2-resident or not). The buffer's bits are OR-ed into;
 * nothing else is written. vox_probe_red_or_ops(ops) is the exact number the
 * call issues (ops rounded up to a multiple of the thread count).
 * Errors: VOX_ERR_INVALID_ARG (null buffer, words out of range, ops < 0),
 * VOX_ERR_ALIGNMENT, VOX_ERR_CUDA.
 */
vox_status vox_probe_red_or(uint32_t *d_buf, int64_t words, int64_t ops, uint32_t seed, void *stream);
int64_t vox_probe_red_or_ops(int64_t ops);

/*
 * vox_generate_noalloc -- vox_generate without a caller-provided workspace.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory at the point where they voxelize, such as
 * plug-ins inside a host application that owns the whole device-memory budget
 * through its own pool (a cudaMalloc behind its back can fail or break its
 * accounting), or real-time loops that cannot pay for cudaMalloc/cudaFree
 * (cudaFree synchronises the device). The caller still provides the segments,
 * the outputs and the status word, as for vox_generate.
 *
 * Path: the call runs exactly what vox_generate runs with a workspace of
 * vox_workspace_size(n) bytes: count + scan, then the list and/or the volume
 * by per-voxel atomics (never the brick path, whose arrays do not fit the
 * scratch). So its outputs are those of that vox_generate call bit for bit,
 * and VOX_OUT_BRICKED, which needs the brick path, returns VOX_ERR_WORKSPACE.
 *
 * Scratch: the count/scan scratch (scan tile counter and flags, offsets) lives
 * in a static device array inside the library, VOX_NOALLOC_SCRATCH_BYTES bytes
 * (about 15.3 MiB), which every GPU that loads the library holds until the
 * process exits. It is sized for at most VOX_NOALLOC_MAX_SEGMENTS segments per
 * call; a larger n returns VOX_ERR_WORKSPACE at once and launches nothing. The
 * call allocates nothing (no cudaMalloc, cudaFree or allocating library
 * routine).
 *
 * Set-up: the first call on each device (and again after the device's context
 * is replaced, e.g. after cudaDeviceReset) looks up the device address of the
 * array with cudaGetSymbolAddress, with that device current; the address is
 * kept per device and context. Make that first call outside any stream
 * capture (for example once at start-up).
 *
 * Sharing: every call on a device uses the same array, which keeps the
 * contents of the last call. Each call clears, with a stream-ordered memset,
 * the part that must start at zero (the scan's tile counter and flags) and
 * overwrites the rest. Calls whose work overlaps on the GPU (issued on
 * different streams, or from several host threads without ordering) race on
 * the array and can corrupt each other's results: issue them on one stream or
 * order them with events.
 */
#define VOX_NOALLOC_MAX_SEGMENTS 2000000
#define VOX_NOALLOC_SCRATCH_BYTES 16008448
vox_status vox_generate_noalloc(const vox_segment *d_segs, int64_t n, vox_dims dims,
                                void *d_list, int64_t list_capacity, uint32_t *d_mask, int flags,
                                int32_t *d_status, void *stream);

/*
 * Launch tuning (process-wide, every device). The outputs do not depend on it:
 * only how the work is spread. Chosen by measurement (the Python autotuner).
 *   run_len       voxels per thread run in the list/atomic generation kernel:
 *                 16, 32 or 64 (0 = default: 32; 64-bit lists take 64 as 32);
 *                 longer runs pay the run's entry less often, shorter runs keep
 *                 more threads busy on small inputs
 *   volume_path   VOX_VOLUME_AUTO (bricks when the workspace allows; pieces
 *                 beyond the workspace by per-voxel atomics), VOX_VOLUME_ATOMIC
 *                 (always per-voxel atomics: each thread merges the bits of
 *                 consecutive voxels in one word into one reduction), or
 *                 VOX_VOLUME_ATOMIC_WARP (always per-voxel atomics, the volume
 *                 alone also merged across the warp: at every step the lanes
 *                 holding equal words (__match_any_sync) OR their bits together
 *                 (__reduce_or_sync) and one lane issues the reduction)
 *   ctas_per_sm   persistent CTAs per SM for the generation and brick kernels
 *                 (0 = the occupancy maximum; larger values are capped there)
 *   list_runs     a list alone (no volume in the same launch, or the volume
 *                 by bricks): 0 = a thread's run of run_len voxels continues
 *                 into the next segments (best when segments share one length
 *                 that run_len divides or that divides run_len); 1 = 32-bit
 *                 lists only: runs end at segment ends (best for short segments
 *                 of varying length); 2 = warp slices: each warp writes 1056
 *                 consecutive voxels (lanes' runs of 33) in list order into
 *                 shared memory and stores them with one TMA bulk copy, taking
 *                 slices from a global work counter (32- and 64-bit lists; best
 *                 for long segments); other values are 0
 * vox_set_tuning(NULL) restores the defaults. Not to be changed while calls
 * are being issued from other host threads.
 */
#define VOX_VOLUME_AUTO 0
#define VOX_VOLUME_ATOMIC 1
#define VOX_VOLUME_ATOMIC_WARP 2
typedef struct vox_tuning {
    int32_t run_len;
    int32_t volume_path;
    int32_t ctas_per_sm;
    int32_t list_runs;
} vox_tuning;
void vox_set_tuning(const vox_tuning *t);
void vox_get_tuning(vox_tuning *t);

/* Human-readable name of a status code. Never NULL. */
const char *vox_strerror(int status);

/* Number of 32-bit words of the occupancy volume for dims (ceil(w*h*d / 32)). */
int64_t vox_mask_words(vox_dims dims);

/*
 * Test hook for failure detection: when tile >= 0, the next count/scan launches
 * make scan tile `tile` skip publishing its prefix, so the tile after it meets
 * the bounded wait of the decoupled look-back, gives up after wait_ns
 * nanoseconds, and reports VOX_ERR_TIMEOUT in *d_status instead of hanging.
 * tile < 0 turns the hook off. wait_ns <= 0 restores the default limit.
 * Process-wide; not for production use.
 */
void vox_debug_set_scan_stall(int64_t tile, int64_t wait_ns);

/* Segments per scan tile of the count/scan kernel (for tests that aim the hook). */
int64_t vox_scan_tile_segments(void);

#ifdef __cplusplus
}
#endif

#endif /* VOX_H */
