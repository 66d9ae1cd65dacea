// Host-side launchers of the codec's kernels (one translation unit each).
#pragma once

#include <stdint.h>

#include "common.cuh"
#include "color.cuh"

namespace gsnfs {

// Every kernel launch of the library is counted (gsnfs_launch_count).
void count_launch();

// Optional per-stage timing with CUDA events on the launching stream.
enum StageId {
    kStVoxelize, kStSort, kStDedup, kStOccupancy, kStRans, kStPrelude, kStRahtFwd, kStRahtFwd0, kStRlgrEnc,
    kStContainer, kStRecon, kStOccDecode, kStOctreeDecode, kStRlgrDec, kStRahtInv, kStRahtInv0, kStCount
};
void stage_begin(cudaStream_t s, int id);
void stage_end(cudaStream_t s, int id);

// Device description of a batch of frames (F = 1 for the plain path).
struct FrameSet {
    uint32_t F;
    uint32_t frame_shift;        // key bit where the frame id starts (64 when F == 1)
    const float *const *pos;     // device array of F device pointers (N_f x 3)
    const float *const *attr;    // device array of F device pointers (N_f x C) or null
    const uint64_t *poff;        // device, F + 1 point offsets into the key arrays
    const uint32_t *J;           // device, F depths
    FrameGrid *grid;             // device, F grids
};

// ---- voxel.cu: bounding box, grid, Morton keys (Sec. 2.1, Sec. 2.2) ------
void launch_voxelize(const FrameSet &fs, DevState *st, uint64_t n_total, uint64_t n_max, uint64_t *keys,
                     uint32_t *vals, int num_sms, cudaStream_t s);

// ---- sort.cu: LSD radix sort of (key, value) over bits [0, nbits) -------
// Returns true when the result is in (keys_alt, vals_alt).
bool radix_sort(uint64_t *keys, uint32_t *vals, uint64_t *keys_alt, uint32_t *vals_alt, uint32_t *hist,
                uint64_t n, uint32_t nbits, int num_sms, cudaStream_t s);
// histogram words for n keys (room for `segments` extra CTAs of a segmented sort)
uint64_t radix_sort_hist_words(uint64_t n, int num_sms, uint32_t segments = 0);
// Segmented sort: segment f = elements [seg_lo[f], seg_lo[f + 1]) is sorted on its own (keys never leave it).
// Host table of the CTAs (cta_lo: ctas + 1 element offsets, cta_seg: 2 per CTA, first CTA of its segment and of
// the next), at most sort CTAs + segments entries; returns the CTA count.
uint32_t radix_sort_segment_table(const uint64_t *seg_lo, uint32_t segments, int num_sms, uint64_t *cta_lo,
                                  uint32_t *cta_seg);
bool radix_sort_segments(uint64_t *keys, uint32_t *vals, uint64_t *keys_alt, uint32_t *vals_alt, uint32_t *hist,
                         uint64_t n, uint32_t nbits, uint32_t ctas, const uint64_t *cta_lo, const uint32_t *cta_seg,
                         int num_sms, cudaStream_t s);
uint64_t radix_sort_max_ctas(uint64_t n, int num_sms);

// ---- geometry.cu ----------------------------------------------------------
// Dedup of sorted keys: codes[v], seg[v] (first sorted point of voxel v,
// seg[nv] = n), gap[v] (gap level to v-1, kInfLevel at frame starts and at
// gap[nv]), vstart[F+1] (voxel offset of each frame), nv -> st->nv_total.
// row0 (optional, with vals): input row of each voxel's first point, | kCarry when the voxel holds several.
void launch_dedup(const uint64_t *keys, uint64_t n, uint32_t frame_shift, uint32_t F, uint64_t *codes,
                  uint32_t *seg, uint8_t *gap, uint32_t *vstart, uint32_t *partials, DevState *st, int num_sms,
                  cudaStream_t s, const uint32_t *vals = nullptr, uint32_t *row0 = nullptr);
uint64_t dedup_partial_words(uint64_t n, int num_sms);

// Octree occupancy bytes of every frame, all levels at once (Algorithm 1).
// level_sizes[f * 22 + d], occ_off[F+1] (byte offset of each frame's bytes).
struct OccupancyOut {
    uint8_t *occ;            // capacity occ_capacity bytes
    uint64_t occ_capacity;
    uint32_t *level_sizes;   // F x 22
    uint64_t *occ_off;       // F + 1
    uint32_t *hoff;          // F x 22: byte offset of height h inside the frame
    uint32_t *partials;      // scratch
};
void launch_occupancy(const uint64_t *codes, const uint8_t *gap, const uint32_t *vstart, const uint32_t *J,
                      uint32_t F, uint32_t frame_shift, const OccupancyOut &o, DevState *st, int num_sms,
                      cudaStream_t s);
uint64_t occupancy_partial_words(uint32_t F, int num_sms);
// the same bound for one frame on a GPU with at most max_sms SMs
constexpr uint64_t occupancy_partial_words_one_frame(int max_sms) { return 8ull * max_sms * 22 + 2 * kMaxFrames + 8; }

// Octree decoding of one frame (Algorithms 2-3): level sizes known on host.
void launch_octree_decode(const uint8_t *occ, uint64_t n_occ, uint32_t J, const uint32_t *h_level_sizes,
                          uint64_t *nodes, uint32_t *pref, uint32_t *partials, uint64_t *leaves,
                          DevState *st, int num_sms, cudaStream_t s);
uint64_t octree_decode_node_words(const uint32_t *h_level_sizes, uint32_t J);

// gap levels of ascending codes (one frame), gap[0] = gap[nv] = kInfLevel
void launch_gap_levels(const uint64_t *codes, uint64_t nv, uint8_t *gap, cudaStream_t s);
// voxel centres of the codes of one frame (Sec. 2.1)
// ctab (3 x 2^J floats, or null): per-axis centre table used when 2^J <= nv
void launch_voxel_centres(const uint64_t *codes, uint64_t nv, uint32_t J, const FrameGrid *grid, float *pos,
                          cudaStream_t s, float *ctab = nullptr);
// voxel centres of a batch: codes carry frame ids above frame_shift
void launch_voxel_centres_batch(const uint64_t *codes, const DevState *st, uint64_t nv_bound,
                                uint32_t frame_shift, const uint32_t *J, const FrameGrid *grid, float *pos,
                                cudaStream_t s);

// ---- raht.cu: prelude and tile transforms (Sec. 3, Algorithms 4-6) -------
constexpr uint32_t kRahtCarrySlots = 128;  // survivors of a tile: at most 2 x 64 (strictly rising gap levels
                                           // from either tile edge)
constexpr int kRahtMultiPasses = 3;  // passes launched grid-wide; the rest run in one CTA
constexpr int kRahtMaxPasses = 40;

struct RahtPass {  // device-resident description of one pass
    uint32_t n;        // elements in this pass
    uint32_t ntiles;
    uint32_t seq_off;  // offset of pos/gap/dest arrays (elements)
    uint32_t tile_off; // first tile index in the schedule arrays
    uint32_t surv_off; // row offset of this pass's input rows in the survivor pool (pass >= 2)
    uint32_t pad[3];
};

struct RahtPlanDev {  // device pointers of a plan
    uint32_t T;            // tile size (elements)
    uint32_t xgrid_mult;   // transform pass 0: CTAs per SM (0 = default 4)
    uint32_t pgrid_mult;   // prelude tile passes: CTAs per SM (0 = default 8)
    uint32_t xpipe_off;    // first transform pass: 0 pipelined metadata, 1 plain, 2 deep pipeline
    uint32_t cap_elems;    // capacity of the pooled sequence arrays
    uint32_t cap_tiles;
    uint32_t cap_surv;     // rows in the survivor pool
    uint32_t *pos;         // pooled sequence arrays: first voxel of each element,
    uint32_t *endseq;      // one past its last voxel,
    uint32_t *send;        // (scratch) subtree end of each carried survivor,
    uint8_t *gapseq;       // gap level to the previous element
    uint32_t *dest;
    uint32_t *tile_nbf;    // per tile: number of butterflies
    uint32_t *tile_nr;     // per tile: number of rounds
    uint16_t *round_end;   // per tile x 64
    uint32_t *bf_idx;      // per tile x T: i0 | i1 << 16
    float2 *bf_ab;         // per tile x T: FP32 coefficients (a, b)
    uint2 *bf_w;           // per tile x T: integer weights (w0, w1), or null (not recorded)
    uint32_t *tile_carry;  // per tile carried count, then exclusive base
    uint16_t *carry_list;  // per tile x kRahtCarrySlots: in-tile index of each carried survivor, by rank
    RahtPass *passes;      // kRahtMaxPasses
    uint32_t *npasses;     // device counter
    // pass 0 elements: first voxel and one past the last voxel of element j, or null when element j is voxel j
    // (a coarser sequence: the nodes of an octree depth, each a run of voxels, for level-of-detail decoding)
    const uint32_t *pos0;
    const uint32_t *end0;
    uint32_t *pipe_ctr;    // 2 words: tiles claimed and CTAs finished in the pipelined first transform pass
                           // (zeroed by the prelude; the last CTA of every launch puts them back to zero)
};

uint32_t raht_tile_size(uint32_t C);
void raht_plan_sizes(uint64_t nv_cap, uint32_t T, uint64_t *elems, uint64_t *tiles, uint64_t *surv_rows);
void launch_raht_prelude(const RahtPlanDev &p, const uint8_t *gap, const DevState *st, const uint64_t *nv_host,
                         int num_sms, cudaStream_t s);

template <typename S>
struct RahtIOT {  // S = float (codec) or double (FP64 instantiation of the same kernels)
    uint32_t C;
    const S *in;            // forward: nv x C input rows (if gather == null)
    const uint32_t *seg;    // forward gather: first sorted point of each voxel
    const uint32_t *vals;   // forward gather: local point index of sorted points
    const uint32_t *row0;   // forward gather: input row of each voxel's first point, | kCarry if it holds
                            // several (or null)
    const uint64_t *codes;  // forward gather: voxel codes (frame id) for the attr pointer
    const S *const *attr;   // forward gather: per-frame attribute pointers
    const S *center;        // forward gather: per frame x C value subtracted from every voxel row, or null
    uint32_t frame_shift;
    S *Y;                   // coefficients nv x C
    S *out;                 // inverse output nv x C
    S *pool;                // survivor rows
    const S *inv_step;      // inverse with quantise->dequantise: per channel 1/step (device), or null
    const S *step;          // per channel step (device)
    S tau;
    // SH colour decorrelation (FP32 codec path only): per frame K (3 x 15 x 15), or null
    const float *klt;
    const uint32_t *frame_color;  // inverse: per frame 1 if colour-coded (null: every frame)
    const uint32_t *vstart;       // inverse: F + 1 voxel offsets (frame of a row)
    uint32_t F;
    YuvInv yuv_inv;
    // inverse over a coarse first pass (plan pos0/end0: level of detail): each output row is divided by
    // sqrt(its element's voxel count), a node's low pass becoming its voxels' mean (Eq. 1)
    uint32_t lod_mean;
};
typedef RahtIOT<float> RahtIO;
// FP64 transforms need a plan built with integer weights recorded (bf_w)
template <typename S>
void launch_raht_forward(const RahtPlanDev &p, const RahtIOT<S> &io, uint64_t nv_bound, int num_sms, cudaStream_t s);
template <typename S>
void launch_raht_inverse(const RahtPlanDev &p, const RahtIOT<S> &io, uint64_t nv_bound, int num_sms, cudaStream_t s);

// ---- batched decoding: one description per frame (device) -------------------
struct DecFrame {
    const uint8_t *occ_sec;     // occupancy section of the frame's stream
    uint64_t occ_bytes;         // its size
    const uint32_t *bw;         // block word counts (attribute section)
    const uint32_t *payload;    // attribute payload words
    uint64_t payload_words;
    uint64_t occ_off;           // first byte of the frame's occupancy bytes in the batch buffer
    uint64_t n_occ;
    uint64_t blk_off;           // first RLGR block of the frame (nb * C blocks)
    uint64_t chunk_off;         // first rANS chunk of the frame (among the batch's rANS chunks)
    uint32_t vstart, nv;        // first output row, voxels
    uint32_t J, mode, aux, chunk;
    uint32_t B, nb;
    FrameGrid grid;
    uint64_t ctab_off;          // first entry of the frame's centre table (3 x 2^J floats), or ~0: computed directly
    uint64_t noff[22];          // node-array offset of each level (level J lives in the voxel rows)
    uint64_t boff[22];          // offset of each level's bytes inside the frame's occupancy bytes
    uint64_t pbase[22];         // set bits of the batch occupancy bytes before each level's first byte
    uint32_t lsz[22];
};

// ---- rlgr.cu: quantiser + block RLGR (Sec. 3.4) ----------------------------
struct RlgrJob {
    uint32_t C;
    uint32_t B;
    uint32_t R;                 // rungs
    const float *Y;             // coefficients, rows = voxels of all frames
    const uint32_t *vstart;     // F + 1 voxel offsets
    uint32_t F;
    const float *inv_step;      // R x C (device)
    float tau;
    uint32_t *slots;            // word slots, one per (frame, rung, channel, block)
    uint32_t *block_words;      // per block: words needed
    const uint64_t *blk_off;    // F + 1: first block of each frame (R x C x nb_f blocks per frame)
    uint32_t slot_words;        // words per slot (a block needing more sets *overflow)
    uint32_t *overflow;
    const double *dc;           // per frame x C: each frame's DC in FP64, quantised in FP64 (or null: from Y)
    double *sq_err;             // per frame x rung x channel: sum of squared quantisation errors, or null
    const float *step;          // R x C FP32 steps (with sq_err)
    const double *steps_rg;     // R x G FP64 steps (with dc)
    const uint8_t *groups;      // C group ids (with dc)
    uint32_t G;
    double tau64;
};
// KLT matrices of the colour mode (color.cu): per frame from its first input
// points; the frame's centres are carried into the decorrelated domain.
void launch_color_klt(const float *const *attr, const uint64_t *poff, uint32_t F, float *klt, float *center,
                      double *partials, cudaStream_t s);
uint64_t color_klt_partial_words(uint32_t F);
// Per-frame channel centres: FP32 mean of the first (up to 1024) input rows
// of each frame, summed in a fixed order.
void launch_frame_centres(const float *const *attr, const uint64_t *poff, uint32_t F, uint32_t C, float *center,
                          cudaStream_t s);
// After a centred forward transform: each frame's DC in FP64 (centred DC +
// sqrt(N_v) x centre), and in Y the rung-0 dequantised DC.
void launch_frame_dc(float *Y, const uint32_t *vstart, uint32_t F, uint32_t C, const float *center,
                     const double *steps_rg, const uint8_t *groups, uint32_t G, double tau, double *dc, cudaStream_t s);
uint32_t rlgr_slot_words(uint32_t B, bool worst_case);
void launch_rlgr_offsets(const uint32_t *vstart, uint32_t F, uint32_t B, uint32_t R, uint32_t C, uint64_t *job_off,
                         uint64_t *blk_off, cudaStream_t s);
void launch_rlgr_encode(const RlgrJob &j, const uint64_t *job_off, uint64_t jobs_bound, cudaStream_t s);
void launch_rlgr_encode_indices(const int32_t *q, const uint32_t *vstart, uint32_t C, uint32_t B, uint32_t *slots,
                                uint32_t slot_words, uint32_t *bw, const uint64_t *job_off, const uint64_t *blk_off,
                                uint64_t jobs_bound, uint32_t *overflow, cudaStream_t s);
void launch_rlgr_decode(const uint32_t *payload, uint64_t payload_words, const uint32_t *block_words,
                        const uint64_t *block_off, uint64_t nv, uint32_t C, uint32_t B, const float *step, float *Y,
                        DevState *st, cudaStream_t s);
void launch_rlgr_decode_batch(const DecFrame *fr, uint32_t F, const uint64_t *job_off, uint64_t jobs_bound,
                              const uint32_t *bw_all, const uint64_t *boff_all, const float *steps_all, uint32_t C,
                              float *Y, DevState *st, cudaStream_t s);
void launch_rlgr_decode_indices(const uint32_t *words, uint64_t total_words, const uint32_t *bw, uint32_t stride,
                                uint64_t nv, uint32_t C, uint32_t B, int32_t *q, DevState *st, cudaStream_t s);

// ---- rans.cu: occupancy entropy stage ------------------------------------
struct RansFrames {
    uint32_t F;
    const uint8_t *occ;        // all frames' bytes
    const uint64_t *occ_off;   // F + 1
    uint32_t chunk;            // symbols per chunk
    uint64_t *chunk_off;       // F + 1 global chunk index (computed)
    uint16_t *freq;            // F x 256
    uint32_t *cum;             // F x 256
    uint32_t *mode;            // F: 0 raw, 1 rANS, 2 constant (decided after sizing)
    uint32_t *chunk_words;     // per global chunk: 16-bit words
    uint32_t *chunk_top;       // per global chunk: first used stack entry
    uint32_t *chunk_pos;       // per global chunk: byte offset inside the section
    uint8_t *chunk_slots;      // per global chunk: rans_chunk_slot_bytes(chunk)
    uint64_t *sec_bytes;       // F: occupancy section size
};
uint64_t rans_chunk_slot_bytes(uint32_t chunk);
void launch_rans_encode(const RansFrames &r, DevState *st, uint64_t max_chunks, int num_sms, cudaStream_t s);
uint64_t rans_table_words();
void launch_rans_decode(const uint8_t *sec, uint64_t sec_bytes, uint64_t n, uint32_t nch, uint32_t chunk,
                        uint8_t *out, uint32_t *tabs, DevState *st, int num_sms, cudaStream_t s);
void launch_fill(uint8_t *out, uint64_t n, uint8_t v, cudaStream_t s);

// ---- batchdec.cu: batch-wide decoding steps --------------------------------
void launch_batch_occ_bytes(const DecFrame *fr, uint32_t F, uint8_t *occ_all, uint64_t max_occ, int num_sms,
                            cudaStream_t s);
// cstart: one word per rANS chunk of the batch (frames' chunks from DecFrame::chunk_off): scratch for the
// chunks' byte offsets
void launch_batch_rans_decode(const DecFrame *fr, uint32_t F, uint32_t max_chunks_per_frame, uint32_t chunk_max,
                              uint8_t *occ_all, uint32_t *tabs, uint64_t *cstart, DevState *st, cudaStream_t s);
// Octree levels of every frame (Algorithm 3), one launch per level: tile popcounts of the batch occupancy
// bytes and their exclusive scan (tbase, tiles + 1 entries), then per level the CTAs of the tiles holding
// that level's bytes (tile_pref: F + 1 CTA offsets per frame; a frame's CTAs start at tile
// occ_tile_first(first byte of the level)).  A frame's last level writes voxel centres and gap levels, not
// codes.  The roots launch writes every frame's root and the gap sentinel gap[nv_total].
uint64_t occ_tiles(uint64_t n_occ);
uint64_t occ_tile_first(uint64_t byte);
void launch_occ_tile_bases(const uint8_t *occ, uint64_t n_occ, uint32_t *tsum, uint64_t *tbase, uint64_t *partials,
                           int num_sms, cudaStream_t s);
void launch_batch_roots(const DecFrame *fr, uint32_t F, uint64_t *nodes, uint8_t *gap, uint64_t nv_total,
                        cudaStream_t s);
void launch_batch_level(const DecFrame *fr, uint32_t F, uint32_t d, const uint32_t *tile_pref, uint32_t tiles,
                        const uint8_t *occ, uint64_t n_occ, const uint64_t *tbase, uint64_t *nodes, const float *ctab,
                        float *pos, uint8_t *gap, DevState *st, cudaStream_t s);
// Voxel-centre tables: a centre coordinate depends only on that axis' voxel
// coordinate, so frames with 2^J <= N_v evaluate the FP64 expression once per
// axis value (3 x 2^J) instead of once per voxel.
void launch_batch_centre_tables(const DecFrame *fr, uint32_t F, uint32_t Jmax, float *ctab, int num_sms,
                                cudaStream_t s);
void launch_batch_block_tables(const DecFrame *fr, uint32_t F, const uint64_t *blk_pref, uint64_t nblk,
                               uint32_t *bw_all, int num_sms, cudaStream_t s);

// ---- lod.cu: level of detail ------------------------------------------------
struct LodGrid {
    double lo[3];
    double cell;  // ext / 2^Jp
};
// node index of every voxel at depth Jp: flags, exclusive offsets (offs[nv] =
// node count) and the first voxel of each node (starts[n] = nv)
void launch_lod_index(const uint64_t *codes, uint64_t nv, uint32_t sh, uint32_t *flags, uint64_t *offs,
                      uint64_t *partials, uint64_t *starts, int num_sms, cudaStream_t s);
// The nodes of a depth as the first pass of a coarser RAHT sequence (pos0, end0, gap0 of n_nodes + 1 entries), and
// the nodes' cell centres (n_nodes: a bound for the launch shape; the count itself is read on the device).
void launch_lod_sequence(const uint64_t *starts, const uint64_t *n_nodes_dev, uint64_t nv, uint64_t n_nodes,
                         const uint8_t *gap, uint32_t *pos0, uint32_t *end0, uint8_t *gap0, int num_sms,
                         cudaStream_t s);
void launch_lod_centres(const uint64_t *codes, const uint64_t *starts, const uint64_t *n_nodes_dev, uint64_t n_nodes,
                        uint32_t sh, uint32_t Jp, const LodGrid &g, float *pos, int num_sms, cudaStream_t s);

// ---- render.cu: splat rasteriser ------------------------------------------------
struct RenderCam {  // camera in FP64: the per-Gaussian projection is evaluated in FP64
    double R[9], t[3], campos[3];
    double fx, fy, cx, cy, znear;
    int W, H, TX, TY;
    float bg[3];
};
size_t render_splat_bytes();
void launch_render_prepare(const float *pos, const float *attr, uint64_t n, const RenderCam &cam, void *splats,
                           float *depth, int4 *rect, uint32_t *count, uint64_t *offs, uint64_t *partials,
                           int num_sms, cudaStream_t s);
void launch_render_tiles(uint64_t n, const int4 *rect, const float *depth, const uint32_t *count,
                         const uint64_t *offs, uint64_t total, const RenderCam &cam, const void *splats,
                         uint64_t *keys, uint32_t *vals, uint64_t *keys_alt, uint32_t *vals_alt, uint32_t *hist,
                         uint2 *ranges, float *image, int num_sms, cudaStream_t s);

// ---- scan.cu / api.cu helpers -------------------------------------------
// exclusive scan of n u32 values into u64 offsets (out has n + 1 entries)
void launch_scan_u32_to_u64(const uint32_t *in, uint64_t n, uint64_t *out, uint64_t *partials, int num_sms,
                            cudaStream_t s);
uint64_t scan_partial_words(uint64_t n, int num_sms);
// stream-ordered device memset run as a kernel (arguments as cudaMemsetAsync)
cudaError_t dev_memset(void *p, int value, size_t bytes, cudaStream_t s);

}  // namespace gsnfs
