/*
 * gsnfs.h -- C ABI of the GB300 (sm_103a) implementation of the GS-NFS
 * per-frame codec hot path (arxiv 2606.05650): octree geometry coding of
 * voxelised Gaussian positions and RAHT attribute coding with quantisation
 * and entropy coding, plus the matching decoder; beside the codec, a batched
 * frames x rungs ladder with per-stream distortion for rate-distortion
 * selection, level-of-detail decoding, SH colour decorrelation, the RAHT
 * transforms as standalone (FP32 and FP64) calls, and a splat rasteriser for
 * rendered-view quality of decoded frames.
 *
 * Conventions for every entry point
 *   - Pointers named d_* are DEVICE memory owned by the caller; h_* are host
 *     memory owned by the caller.  The library never frees caller memory.
 *   - `stream` is a cudaStream_t passed as void*; NULL means the legacy
 *     default stream.  Work is enqueued in stream order.  Calls that return
 *     host scalars (out_* pointers) synchronise `stream` once before
 *     returning; everything else returns after enqueueing.
 *   - A gsnfs_ctx owns the device scratch for one stream at a time; calls on
 *     one context must not overlap (use one context per concurrent stream).
 *   - No exception crosses the ABI.  Errors are negative gsnfs_status
 *     values; gsnfs_status_string() names them.  Decoders validate stream
 *     headers on the host and check every device read of a stream against
 *     its length; a malformed stream yields GSNFS_ERR_CORRUPT, never a trap.
 *   - Arrays of points are row-major: positions N x 3 float32, attributes
 *     N x C float32.  Decoded voxels are in ascending Morton order.
 *   - The bitstream layout is this library's own (the paper fixes only the
 *     octree header); it is described beside the implementation.
 */
#ifndef GSNFS_H
#define GSNFS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gsnfs_ctx gsnfs_ctx;
typedef struct gsnfs_raht_plan gsnfs_raht_plan;

typedef enum {
    GSNFS_OK = 0,
    GSNFS_ERR_INVALID_ARG = -1, /* bad argument: depth, sizes, steps, pointers */
    GSNFS_ERR_CAPACITY = -2,    /* output buffer too small; required size reported */
    GSNFS_ERR_CORRUPT = -3,     /* malformed bitstream */
    GSNFS_ERR_CUDA = -4,        /* a CUDA runtime call failed */
    GSNFS_ERR_TIMEOUT = -5,     /* a bounded device wait expired */
    GSNFS_ERR_OOM = -6,         /* device allocation failed */
    GSNFS_ERR_UNSUPPORTED = -7  /* valid request outside what this build supports */
} gsnfs_status;

/* Quantisation and entropy-coder parameters (Sec. 3.4).
 * Attribute channels are split into groups, one quantisation step per group
 * (coefficients of different attributes are quantised to different levels).
 * q = sign(y) floor(|y| / step + tau); tau = 0.5 is the uniform mid-tread
 * quantiser, smaller tau widens the dead zone.  Coefficients of a channel
 * are RLGR-coded in blocks of rlgr_block (Sec. 3.4, Table A.5). */
typedef struct {
    uint32_t num_channels;         /* C, 0..256 (0 = geometry only) */
    uint32_t num_groups;           /* G, 1..255 when C > 0 */
    const uint8_t *channel_group;  /* host, length C, values < G */
    const double *steps;           /* host, length G, each > 0 */
    double tau;                    /* rounding offset in (0, 0.5] */
    uint32_t rlgr_block;           /* B: power of two in [32, 65536] */
    uint32_t rans_chunk;           /* occupancy symbols per rANS chunk: multiple of 32 in [32, 1<<20] */
    uint32_t color;                /* 0, or 1: SH colour decorrelation of Sec. 4 before RAHT (C must be 56:
                                    * scale 0-2, rotation 3-6, opacity 7, SH DC RGB 8-10, SH AC 11-55 as
                                    * R[15] G[15] B[15]): BT.601 YUV on every SH function, then one KLT per
                                    * YUV channel over the 15 AC functions, its matrices in the header */
} gsnfs_quant;

/* Creates a context on CUDA device `cuda_device` (made current for the
 * call).  Returns GSNFS_OK and *out, or GSNFS_ERR_CUDA / GSNFS_ERR_OOM. */
gsnfs_status gsnfs_create(gsnfs_ctx **out, int cuda_device);

/* Frees the context and its scratch (synchronises the device first). */
void gsnfs_destroy(gsnfs_ctx *ctx);

/* Static description of a status code. */
const char *gsnfs_status_string(gsnfs_status s);

/* Grows the context's scratch so that frames of up to n points with C
 * channels at depth J encode and decode without further allocation (call
 * before capturing the codec into a CUDA graph). */
gsnfs_status gsnfs_reserve(gsnfs_ctx *ctx, uint64_t n, uint32_t C, uint32_t J, const gsnfs_quant *q);

/* CUDA graphs for the encoder (off by default).  When on, the device work of
 * gsnfs_encode_frame / gsnfs_encode_batch (from the parameter uploads to the
 * result read-back) is captured into a graph the first time a request shape
 * is seen and replayed afterwards.  The shape is: frame count, rungs, point
 * count and depth of every frame, channels, groups, RLGR block, rANS chunk,
 * tau, output buffer and capacity, reconstruction buffers, and the context's
 * scratch addresses; point and attribute pointers, steps and rung scales may
 * change between replays.  Up to 64 graphs are kept (least recently used
 * dropped); growing the scratch drops them all.  The graph runs on a stream
 * of the context ordered after the caller's stream and joined back to it.
 * A capture that fails falls back to running the work directly.  Replays
 * report the same per-stage times as direct calls while profiling is on (the
 * graph records its own stage events). */
gsnfs_status gsnfs_set_graphs(gsnfs_ctx *ctx, int enable);
/* out[0] replays, out[1] captures, out[2] failed captures, out[3] graphs cached. */
gsnfs_status gsnfs_graph_stats(gsnfs_ctx *ctx, uint64_t *out);

/* Launch-shape tunables of a context.  Bitstreams and decoded values do not
 * depend on them (each butterfly and each code is computed the same way
 * whatever the tiling); only the speed does.  Value 0 restores the built-in
 * default.  Changing one drops the context's captured graphs.
 *   GSNFS_TUNE_RAHT_TILE     RAHT tile size in voxels: power of two in
 *                            [256, 4096] (default: largest whose C rows fit
 *                            56 KB of shared memory, at least 256)
 *   GSNFS_TUNE_RAHT_GRID     CTAs per SM of the first transform pass, 1..32 (4)
 *   GSNFS_TUNE_PRELUDE_GRID  CTAs per SM of the prelude tile passes, 1..32 (8)
 *   GSNFS_TUNE_RAHT_PIPE     first pass of FP32 transforms, where its
 *                            buffers fit shared memory: 0 software-pipelined
 *                            metadata (three CTAs per SM), 1 plain, 2 deep
 *                            pipeline (one CTA per SM, rows of the next two
 *                            tiles in flight) */
enum { GSNFS_TUNE_RAHT_TILE = 0, GSNFS_TUNE_RAHT_GRID = 1, GSNFS_TUNE_PRELUDE_GRID = 2, GSNFS_TUNE_RAHT_PIPE = 3 };
gsnfs_status gsnfs_tune_set(gsnfs_ctx *ctx, int which, uint32_t value);
gsnfs_status gsnfs_tune_get(gsnfs_ctx *ctx, int which, uint32_t *value);

/* Upper bound of the encoded size of a frame of n points (host only). */
gsnfs_status gsnfs_max_bitstream_bytes(uint64_t n, uint32_t J, const gsnfs_quant *q, uint64_t *out);

/* Encodes one frame (Sec. 2, Sec. 3; Algorithm 1 for geometry, Algorithms
 * 4-6 and Sec. 3.4 for attributes):
 *   voxelise to a 2^J grid over the bounding cube, Morton-code, radix-sort,
 *   merge Gaussians sharing a voxel by averaging, emit the octree header and
 *   breadth-first occupancy bytes (rANS coded), RAHT-transform the merged
 *   attributes over all 3J binary levels, quantise per group and RLGR-code
 *   each channel in blocks.
 * d_pos: N x 3 float32; d_attr: N x C float32 (may be NULL when C == 0);
 * n may be 0 (valid empty stream); J in 1..21.
 * d_bitstream receives the stream; on GSNFS_ERR_CAPACITY *out_bytes holds
 * the required size and nothing beyond `capacity` is written.
 * Optional reconstruction (the decoder's output, computed inside the
 * encoder): d_recon_pos (N_v x 3) and d_recon_attr (N_v x C), each may be
 * NULL; they must hold N_v <= n rows.  *out_nv receives N_v. */
gsnfs_status gsnfs_encode_frame(gsnfs_ctx *ctx, void *stream, const float *d_pos, const float *d_attr,
                                uint64_t n, uint32_t J, const gsnfs_quant *q, uint8_t *d_bitstream,
                                uint64_t capacity, uint64_t *out_bytes, float *d_recon_pos,
                                float *d_recon_attr, uint64_t *out_nv);

/* Reads the fixed header of a stream (>= 96 bytes): number of voxels,
 * channels and depth.  `header` may point to host memory (pageable, pinned
 * or managed) or to device memory; from device memory the first 96 bytes
 * are copied to the host first (a synchronous copy: call it outside stream
 * capture).  Returns GSNFS_ERR_CORRUPT for fewer than 96 bytes or a bad
 * magic, version or depth, GSNFS_ERR_CUDA if that copy fails. */
gsnfs_status gsnfs_peek_frame(const uint8_t *header, uint64_t bytes, uint64_t *out_nv, uint32_t *out_C,
                              uint32_t *out_J);

/* Decodes one frame (Sec. 2.3, Algorithms 2-3; inverse of Algorithm 6):
 * occupancy rANS decode, level-synchronous octree expansion, voxel centres,
 * RLGR decode and dequantisation, inverse RAHT.  d_bitstream (device) holds
 * `bytes` bytes.  d_pos receives N_v x 3 float32 voxel centres, d_attr
 * N_v x C float32 attributes (either may be NULL); capacity_nv is the row
 * capacity of both.  *out_nv receives N_v. */
gsnfs_status gsnfs_decode_frame(gsnfs_ctx *ctx, void *stream, const uint8_t *d_bitstream, uint64_t bytes,
                                float *d_pos, float *d_attr, uint64_t capacity_nv, uint64_t *out_nv);

/* Level of detail: decodes the frame to the nodes of octree depth
 * `depth` <= J (Algorithm 2's depth shift read as J - depth).  Node k (in
 * Morton order) gets the centre of its cell at that depth in d_pos (x 3) and
 * the mean of its voxels' decoded attributes in d_attr (x C), which by Eq. (1)
 * is its RAHT low-pass coefficient divided by sqrt(voxel count): the geometry
 * and the coefficients are decoded in full, but the inverse RAHT runs over
 * the node sequence only (the butterflies inside nodes are never applied) and
 * no per-voxel output is formed.  *out_nodes receives the node count;
 * GSNFS_ERR_CAPACITY (outputs untouched) when it exceeds capacity_nodes.
 * depth = J gives the full decode.  d_pos and d_attr may each be NULL. */
gsnfs_status gsnfs_decode_frame_lod(gsnfs_ctx *ctx, void *stream, const uint8_t *d_bitstream, uint64_t bytes,
                                    uint32_t depth, float *d_pos, float *d_attr, uint64_t capacity_nodes,
                                    uint64_t *out_nodes);

/* Pinhole camera of the splat rasteriser.  view is the 3 x 4 world-to-camera
 * matrix [R | t] in row-major order (camera looks along +z, image x right,
 * y down); pixel (px, py) has its centre at (px + 0.5, py + 0.5); points with
 * camera depth <= znear (> 0) are culled; background is the RGB behind all
 * splats. */
typedef struct {
    double view[12];
    double fx, fy, cx, cy;
    uint32_t width, height;  /* 1 .. 16384 */
    double znear;
    double background[3];
} gsnfs_camera;

/* Splat rasteriser used to measure rendered-view quality of decoded frames
 * (Sec. 5.1 scores decoded frames by the PSNR of their renders against
 * renders of the uncompressed Gaussians).  Standard 3DGS forward pass: per Gaussian, the projected mean,
 * the EWA 2-D covariance J W Sigma W^T J^T + 0.3 I, a square footprint of
 * radius ceil(3 sqrt(largest eigenvalue)) over 16 x 16-pixel tiles, opacity
 * sigmoid(logit) and a degree-3 real-SH colour (+0.5, clamped at 0) seen
 * from the camera centre; per pixel, front-to-back alpha compositing over the
 * Gaussians whose footprint covers its tile, ordered by depth then index,
 * alpha = min(0.99, opacity exp(-d^T conic d / 2)), skipping alpha < 1/255
 * and stopping before transmittance falls below 1e-4.
 * d_pos (n x 3) and d_attr (n x 56: log-scales 0-2, rotation w x y z 3-6,
 * opacity logit 7, SH DC RGB 8-10, SH AC 11-55 as R[15] G[15] B[15]) are
 * device float32; d_image (device) receives height x width x 3 float32, row
 * major.  Work is FP32.  Scratch is owned by ctx and grown on demand; the call
 * synchronises the stream once (to size the tile lists).  Errors:
 * GSNFS_ERR_INVALID_ARG (null or misaligned pointers, image size or znear out
 * of range), GSNFS_ERR_CAPACITY (more than 2^32 - 1 tile entries),
 * GSNFS_ERR_OOM, GSNFS_ERR_CUDA. */
gsnfs_status gsnfs_render(gsnfs_ctx *ctx, void *stream, const float *d_pos, const float *d_attr, uint64_t n,
                          const gsnfs_camera *cam, float *d_image);

/* Batched bandwidth ladder (frames x rungs): encodes `frames` frames, frame f
 * with n[f] points at depth J[f] (16..19 supported together, any mix),
 * each at `rungs` quantisation rungs whose steps are q->steps scaled by
 * rung_scale[r].  Geometry and RAHT run once per frame; quantisation and
 * RLGR run per rung.  Stream (f, r) is written to
 * d_out[h_offsets[f*rungs + r] .. h_offsets[f*rungs + r + 1]).
 * h_pos/h_attr are host arrays of `frames` device pointers; h_n, h_J host
 * arrays of length `frames`; h_offsets (host) has frames*rungs + 1 entries.
 * frames <= 64, rungs <= 8, rungs x channels <= 1024. */
gsnfs_status gsnfs_encode_batch(gsnfs_ctx *ctx, void *stream, uint32_t frames, const float *const *h_pos,
                                const float *const *h_attr, const uint64_t *h_n, const uint32_t *h_J,
                                uint32_t rungs, const double *h_rung_scale, const gsnfs_quant *q,
                                uint8_t *d_out, uint64_t capacity, uint64_t *h_offsets);

/* gsnfs_encode_batch that also returns the distortion of every stream for
 * rate-distortion selection over the ladder: h_sq_err (host, frames x rungs x
 * C, in that order) receives, per frame, rung and channel, the sum over the
 * frame's voxels of the squared difference between each RAHT coefficient and
 * its dequantised value.  RAHT is orthonormal (Sec. 3.2), so this is also the
 * squared error of the decoded attributes against the voxel means (Parseval).
 * Coefficients are taken in FP32 as coded (the DC in FP64). */
gsnfs_status gsnfs_encode_batch_rd(gsnfs_ctx *ctx, void *stream, uint32_t frames, const float *const *h_pos,
                                   const float *const *h_attr, const uint64_t *h_n, const uint32_t *h_J,
                                   uint32_t rungs, const double *h_rung_scale, const gsnfs_quant *q,
                                   uint8_t *d_out, uint64_t capacity, uint64_t *h_offsets, double *h_sq_err);

/* Batched decoder: decodes `frames` streams; stream f lives at
 * d_in + h_in_offsets[f] with h_in_offsets[f+1] - h_in_offsets[f] bytes.
 * Voxels of frame f are written to rows h_out_rows[f] .. of d_pos / d_attr
 * (host array of frames + 1 row offsets, filled by this call; capacity_rows
 * bounds the total). */
gsnfs_status gsnfs_decode_batch(gsnfs_ctx *ctx, void *stream, uint32_t frames, const uint8_t *d_in,
                                const uint64_t *h_in_offsets, float *d_pos, float *d_attr,
                                uint64_t capacity_rows, uint64_t *h_out_rows);

/* Header records for the decoder: GSNFS_HEADER_RECORD_BYTES per stream, holding the stream's header tables
 * (bytes [0, header size) of the stream, at most 4096) at offset 0, the first 24 bytes of its occupancy section at
 * 4096 and the first 8 bytes of its attribute section at 4160 (zeros where a section is shorter). */
#define GSNFS_HEADER_RECORD_BYTES 4224u

/* gsnfs_encode_batch that also returns the header record of every stream in h_headers (host, frames x rungs
 * records, in stream order), read back together with the offsets.  A decoder given these records
 * (gsnfs_decode_batch_async) needs no read of the streams from the host. */
gsnfs_status gsnfs_encode_batch_headers(gsnfs_ctx *ctx, void *stream, uint32_t frames, const float *const *h_pos,
                                        const float *const *h_attr, const uint64_t *h_n, const uint32_t *h_J,
                                        uint32_t rungs, const double *h_rung_scale, const gsnfs_quant *q,
                                        uint8_t *d_out, uint64_t capacity, uint64_t *h_offsets,
                                        uint8_t *h_headers);

/* gsnfs_decode_batch without host synchronisation: with the streams' header records given (h_headers, host,
 * frames records in stream order, as gsnfs_encode_batch_headers returns them) nothing is read back from the
 * device; the call validates the records on the host, fills h_out_rows, enqueues the decode on `stream` and
 * returns.  The device's status (0, or 1 = corrupt stream, 2 = capacity, 4 = a bounded wait expired) is written
 * into *status (device memory, or pinned host memory the device can write) in stream order after the last
 * kernel; the outputs are valid once the stream has reached that point.  With h_headers NULL the headers are read
 * from d_in with host synchronisations first (the decode itself is still asynchronous).  Host-detected errors are
 * returned as usual.  The call stages its frame tables in a pinned buffer of its own (one of four, reused once
 * the decode that last used it has completed).  As for every call on a context, calls must not overlap: keep
 * the context's calls on one stream (or order them with events). */
gsnfs_status gsnfs_decode_batch_async(gsnfs_ctx *ctx, void *stream, uint32_t frames, const uint8_t *d_in,
                                      const uint64_t *h_in_offsets, const uint8_t *h_headers, float *d_pos,
                                      float *d_attr, uint64_t capacity_rows, uint64_t *h_out_rows,
                                      uint32_t *status);

/* ---- stage entry points (each is one step of the path above) ---------- */

/* Voxelisation and Morton coding (Sec. 2.1, Sec. 2.2): the distinct voxel
 * codes in ascending order (d_codes, n entries of capacity) and the grid
 * (h_grid[0..3] = lo_x, lo_y, lo_z, ext as float64).  *out_nv receives N_v. */
gsnfs_status gsnfs_voxelize(gsnfs_ctx *ctx, void *stream, const float *d_pos, uint64_t n, uint32_t J,
                            uint64_t *d_codes, double *h_grid, uint64_t *out_nv);

/* Octree occupancy bytes (Algorithm 1) of nv distinct ascending Morton codes
 * at depth J: d_occ receives sum_{d<J} |L_d| bytes in breadth-first order
 * (capacity occ_capacity), h_level_sizes (J+1 entries) the header. */
gsnfs_status gsnfs_octree_encode(gsnfs_ctx *ctx, void *stream, const uint64_t *d_codes, uint64_t nv,
                                 uint32_t J, uint8_t *d_occ, uint64_t occ_capacity, uint32_t *h_level_sizes,
                                 uint64_t *out_occ_bytes);

/* Octree decoding (Sec. 2.3, Algorithms 2-3): ascending leaf codes from
 * occupancy bytes and the header.  Returns GSNFS_ERR_CORRUPT when the bytes
 * contradict the level sizes. */
gsnfs_status gsnfs_octree_decode(gsnfs_ctx *ctx, void *stream, const uint8_t *d_occ, uint64_t occ_bytes,
                                 uint32_t J, const uint32_t *h_level_sizes, uint64_t *d_codes);

/* Occupancy entropy stage (Sec. 2.2 last paragraph; own rANS): codes n
 * bytes into an occupancy section (d_out, capacity) / decodes a section. */
gsnfs_status gsnfs_occupancy_section_encode(gsnfs_ctx *ctx, void *stream, const uint8_t *d_in, uint64_t n,
                                            uint32_t rans_chunk, uint8_t *d_out, uint64_t capacity,
                                            uint64_t *out_bytes);
gsnfs_status gsnfs_occupancy_section_decode(gsnfs_ctx *ctx, void *stream, const uint8_t *d_sec,
                                            uint64_t sec_bytes, uint8_t *d_out, uint64_t n);

/* RAHT plan (Sec. 3.2 prelude, Algorithms 4-5): the butterfly schedule of nv
 * distinct ascending Morton codes at depth J for C channels.  The plan owns
 * its device memory; it is bound to the context's device. */
gsnfs_status gsnfs_raht_plan_create(gsnfs_ctx *ctx, void *stream, const uint64_t *d_codes, uint64_t nv,
                                    uint32_t J, uint32_t C, gsnfs_raht_plan **out);
void gsnfs_raht_plan_destroy(gsnfs_raht_plan *plan);

/* RAHT forward (Eq. 1, Algorithm 6 bottom-up over all 3J levels):
 * d_in (nv x C, Morton order) -> d_out (nv x C coefficients in place
 * layout: DC at row 0, each high pass at its right sibling's first row).
 * d_in and d_out may alias. */
gsnfs_status gsnfs_raht_forward(gsnfs_raht_plan *plan, void *stream, const float *d_in, float *d_out);

/* RAHT inverse (Algorithm 6 top-down, transposed rotations).  When
 * q != NULL each coefficient is first quantised and dequantised with q
 * (the encoder's reconstruction).  d_in and d_out may alias. */
gsnfs_status gsnfs_raht_inverse(gsnfs_raht_plan *plan, void *stream, const float *d_in, float *d_out,
                                const gsnfs_quant *q);

/* The same two transforms evaluated in FP64 by the same kernels, with the
 * butterfly coefficients computed in FP64 from the plan's integer weights
 * (w0, w1): for gradient checks and reference-precision runs.  Layout,
 * aliasing and q as above; q's steps and tau are used in FP64.  The first
 * call allocates an FP64 survivor pool (about 8 x nv x C bytes) that the
 * plan keeps until it is destroyed (GSNFS_ERR_OOM if that fails). */
gsnfs_status gsnfs_raht_forward_f64(gsnfs_raht_plan *plan, void *stream, const double *d_in, double *d_out);
gsnfs_status gsnfs_raht_inverse_f64(gsnfs_raht_plan *plan, void *stream, const double *d_in, double *d_out,
                                    const gsnfs_quant *q);

/* Block RLGR of int32 quantisation indices (Sec. 3.4): d_q is nv x C
 * row-major; each channel is cut into blocks of B coefficients and block b of
 * channel c (nb = ceil(nv / B) blocks per channel) is one RLGR stream written
 * at d_slots + (b * C + c) * gsnfs_rlgr_slot_words(B); d_block_words[b*C+c]
 * receives its length in 32-bit words.  Decoding reads the same layout and
 * writes d_q (GSNFS_ERR_CORRUPT on a malformed block). */
uint32_t gsnfs_rlgr_slot_words(uint32_t B);
gsnfs_status gsnfs_rlgr_encode_indices(gsnfs_ctx *ctx, void *stream, const int32_t *d_q, uint64_t nv, uint32_t C,
                                       uint32_t B, uint32_t *d_slots, uint32_t *d_block_words);
gsnfs_status gsnfs_rlgr_decode_indices(gsnfs_ctx *ctx, void *stream, const uint32_t *d_slots,
                                       const uint32_t *d_block_words, uint64_t nv, uint32_t C, uint32_t B,
                                       int32_t *d_q);

/* ---- allocation-free occupancy encoder (no counterpart in the paper) ---- */

/* Largest voxel count gsnfs_octree_encode_static accepts. */
#define GSNFS_STATIC_MAX_VOXELS 1048576u

/* The occupancy bytes and level sizes of gsnfs_octree_encode, computed
 * without allocating anything: for callers that may not allocate device
 * memory while running (hosts that give all device memory to their own pool
 * at start-up, real-time loops that cannot take the synchronisation and
 * locks of cudaMalloc / cudaFree).  Needs no context.  Its scratch is one
 * fixed device array of about 1.3 MB that the library reserves on every GPU
 * that loads it, kept until the process exits.
 *   d_codes       nv distinct ascending Morton codes (device), nv <=
 *                 GSNFS_STATIC_MAX_VOXELS, else GSNFS_ERR_UNSUPPORTED
 *   d_occ         output bytes (device, 4-byte aligned); written in whole
 *                 32-bit words, so occ_capacity must cover the byte count
 *                 rounded up to 4 (else GSNFS_ERR_CAPACITY, with the byte
 *                 count in *out_occ_bytes)
 *   h_level_sizes J + 1 level sizes (host)
 * Runs on the current CUDA device and synchronises `stream` before it
 * returns.  The first call on a device looks up the array's device address;
 * make that first call before any stream capture.  All calls on a device
 * share the array: calls that overlap on the GPU race and must be
 * serialised by the caller. */
gsnfs_status gsnfs_octree_encode_static(void *stream, const uint64_t *d_codes, uint64_t nv, uint32_t J,
                                        uint8_t *d_occ, uint64_t occ_capacity, uint32_t *h_level_sizes,
                                        uint64_t *out_occ_bytes);

/* ---- instrumentation (no counterpart in the paper) --------------------- */

/* Number of kernels this library has enqueued since it was loaded. */
uint64_t gsnfs_launch_count(void);

/* Per-stage timing: when enabled, every stage of encode / decode records a
 * pair of CUDA events on the launching stream.  gsnfs_profile_read
 * synchronises on the recorded events, returns the accumulated milliseconds
 * and interval counts per stage (cap entries; names from
 * gsnfs_profile_stage_names, which returns the number of stages) and resets
 * the accumulators. */
gsnfs_status gsnfs_profile_enable(int enable);
int gsnfs_profile_stage_names(const char **names, int cap);
gsnfs_status gsnfs_profile_read(double *ms, uint64_t *count, int cap);

#ifdef __cplusplus
}
#endif
#endif /* GSNFS_H */
