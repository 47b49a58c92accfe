/*
 * me.h -- C-ABI of libme: block-matching motion estimation on one GB300.
 *
 * The library computes, for every non-overlapping B x B block of an 8-bit
 * luma frame `cur`, the displacement (dx, dy) into the previous frame `ref`
 * that the chosen search returns (Jia & Zhang, "Directional Cross Diamond
 * Search Algorithm for Fast Block Motion Estimation", Sec. I: the block
 * matching problem; Sec. III-B: the DCDS algorithm).
 *
 * Conventions shared by every entry point:
 *   - Frames are row-major uint8, `pitch` bytes per row (the single-frame
 *     calls use pitch = w).  w and pitch are multiples of 16, w and h are
 *     multiples of the block size, frame pointers are 16-byte aligned.
 *   - The block whose top-left pixel is (x, y) in `cur` is compared with the
 *     block at (x + dx, y + dy) in `ref`.  A displacement is a candidate only
 *     if |dx| <= range, |dy| <= range and the reference block lies entirely
 *     inside the frame (no padding).
 *   - Distortion is the SAD (sum of absolute differences, uint32).  The paper
 *     uses MAD = SAD / B^2 (Sec. II-C, Sec. IV); every argmin is the same.
 *   - Outputs are indexed by block in raster order: k = by * (w / B) + bx.
 *     mv[2k] = dx, mv[2k+1] = dy (int16); sad[k] (uint32); nsp[k] (uint16)
 *     = the number of distinct candidates evaluated ("number of search
 *     points", Sec. III-C and Table IX).
 *   - Every frame and output pointer is DEVICE memory owned by the caller
 *     (e.g. torch tensors), except in me_estimate_host_batch, which takes
 *     host memory.  The library owns only its context: scratch, descriptor
 *     tables, captured graphs, tuning results and the host-batch staging.
 *   - Calls are asynchronous on `stream` (a cudaStream_t; NULL = the legacy
 *     default stream).  Outputs are valid once the stream has reached them.
 *   - Errors: every call returns an me_status; the reason is kept in
 *     me_last_error(ctx).  ME_ERR_ARG is returned before any launch when an
 *     argument is invalid.  There is no CPU fallback: without a usable
 *     sm_103a device me_init fails with ME_ERR_CUDA.
 *
 * Thread safety: one context per host thread.  Calls on one context that run
 * concurrently on different streams share its work-queue counters; at most
 * ME_MAX_INFLIGHT launches of one context may be in flight at once.
 */
#ifndef ME_H
#define ME_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct me_ctx me_ctx;

typedef enum me_status {
    ME_OK = 0,
    ME_ERR_ARG = 1,          /* invalid argument, nothing was launched */
    ME_ERR_CUDA = 2,         /* a CUDA runtime call failed */
    ME_ERR_UNSUPPORTED = 3,  /* valid but not provided (e.g. no weights loaded) */
    ME_ERR_TIMEOUT = 4,      /* a bounded device-side wait gave up */
    ME_ERR_NOMEM = 5         /* a library-owned allocation failed */
} me_status;

typedef enum me_algo {
    ME_ALGO_FS = 0,          /* full search, Sec. I; argmin of (SAD, |dx|+|dy|, dy, dx) */
    ME_ALGO_DCDS = 1,        /* DCDS, Sec. III-B steps 1-4 */
    ME_ALGO_DCDS_S = 2,      /* simplified DCDS^S, Sec. IV-C */
    ME_ALGO_DCDS_LEARNED = 3 /* DCDS from a learned start proposal (not in the paper) */
} me_algo;

enum { ME_MAX_RANGE = 32, ME_MAX_INFLIGHT = 64, ME_STATIC_MAX_FRAMES = 64 };

/* One frame pair of a batch.  All pointers are device memory. */
typedef struct me_frame_desc {
    const uint8_t* cur;
    const uint8_t* ref;
    int32_t w, h, pitch;     /* pixels, pixels, bytes */
    int32_t range;           /* search range R, 1..ME_MAX_RANGE */
    int16_t* mv;             /* [nb][2] */
    uint32_t* sad;           /* [nb] */
    uint16_t* nsp;           /* [nb], may be NULL */
} me_frame_desc;

/* me_init: create a context on `cuda_device`.  `tune_cache_path` (nullable)
 * names a text file where me_tune stores the launch shapes it picked; it is
 * read here if it exists.  Fails with ME_ERR_CUDA when the device is missing
 * or is not sm_103. */
int me_init(me_ctx** out, int cuda_device, const char* tune_cache_path);

/* me_free: release the context (waits for nothing; the caller must have
 * synchronised the streams it used).  NULL is accepted. */
void me_free(me_ctx* ctx);

/* me_last_error: text of the last failure on this context ("" if none).
 * The string is owned by the context and valid until the next call. */
const char* me_last_error(const me_ctx* ctx);

/* me_estimate: motion field of one frame pair (pitch = w).
 *   block: 8 or 16; range: 1..32; algo: an me_algo value.
 *   Full search: Sec. I and the FS rows of Table IX.
 *   DCDS: HCSP at the origin (step 1), then HDSP/VDSP by switching strategy
 *   one and two until the centre wins (steps 2-3), then the two middle points
 *   (step 4), Sec. III-B.  A point already evaluated is not evaluated or
 *   counted again; ties keep the earlier point in the fixed order
 *   HCSP: (0,0),(-1,0),(+1,0),(0,-1),(0,+1),(-2,0),(+2,0);
 *   HDSP: (0,-1),(0,+1),(-2,0),(+2,0); VDSP: (-1,0),(+1,0),(0,-2),(0,+2);
 *   middle points: HDSP (-1,0),(+1,0); VDSP (0,-1),(0,+1).
 *   DCDS^S (Sec. IV-C): step 4 checks only the middle point on the side of
 *   the distant point with the smaller SAD (negative side on a tie; both
 *   middle points when neither distant point is a candidate).
 *   DCDS from a learned start (not in the paper): runs
 *   me_estimate_learned_batch with the context's own proposal (loaded by
 *   me_proposal_load or _set_params with a NULL proposal, or trained by
 *   me_proposal_train); ME_ERR_ARG when the context has none.  That call
 *   synchronises `stream`.
 *   mv, sad: required; nsp: may be NULL. */
int me_estimate(me_ctx* ctx, const uint8_t* cur, const uint8_t* ref, int w, int h,
                int block, int range, int algo,
                int16_t* mv, uint32_t* sad, uint16_t* nsp, void* stream);

/* me_estimate_batch: many frame pairs (of any sizes and ranges) in one
 * persistent launch that pulls tiles of blocks from a global work queue.
 * `block` and `algo` apply to all descriptors.  Results are identical to
 * calling me_estimate on each pair.  `descs` is HOST memory, read before the
 * call returns.  algo ME_ALGO_DCDS_LEARNED runs me_estimate_learned_batch
 * with the context's own proposal, as me_estimate does. */
int me_estimate_batch(me_ctx* ctx, const me_frame_desc* descs, int n, int block, int algo,
                      void* stream);

/* me_estimate_batch_noalloc: the same DCDS / DCDS^S search as
 * me_estimate_batch, for callers that must not allocate device memory.
 * The paper has no counterpart; this is a deployment aid.
 *
 * It is for code that cannot call cudaMalloc at the time it searches: a
 * real-time video path that must not trigger the device-wide
 * synchronisation an allocation or free can cause, a host application or
 * plugin framework that owns all device memory through its own pool and
 * forbids libraries from allocating, or a process running so close to the
 * memory limit that a late allocation could fail in the middle of a stream.
 * No context is needed (me_init allocates) and nothing is allocated, on the
 * device or pinned on the host.
 *
 * The work-queue counter and descriptor table live in a fixed library-owned
 * device array sized for ME_STATIC_MAX_FRAMES descriptors; every device that
 * loads libme keeps it until the process exits.  n above that limit is
 * rejected with ME_ERR_ARG.  The first call on a device looks up the array's
 * device address (with that device current); make that first call before
 * any stream capture.  Every call reuses the same array: calls whose work
 * overlaps on the GPU (different streams, or different host threads on one
 * device) race and must be serialised by the caller.  Frames and outputs are
 * caller-owned device memory as for me_estimate_batch; `descs` is host
 * memory read before the call returns.  algo: ME_ALGO_DCDS or
 * ME_ALGO_DCDS_S (ME_ERR_UNSUPPORTED otherwise).  The launch shape is the
 * library default.  Results are identical to me_estimate_batch.
 * err (nullable) receives a message of at most err_len bytes on failure.
 *
 * The first call on a device also loads every kernel this path launches
 * (with CUDA's lazy module loading a kernel is otherwise loaded, which may
 * allocate, at its first launch), so after that first call no later call
 * allocates, whatever its block size or algo.
 *
 * A failure the search detects on the device (a bounded wait that gave up:
 * the tiles it had not reached keep their old output) is recorded in a
 * status word inside the same fixed array.  The word accumulates over calls
 * until me_noalloc_check_status reads and clears it; the call itself has
 * already returned ME_OK by then. */
int me_estimate_batch_noalloc(const me_frame_desc* descs, int n, int block, int algo, void* stream,
                              char* err, int err_len);

/* me_noalloc_check_status: the companion of me_estimate_batch_noalloc (no
 * counterpart in the paper).  Synchronises `stream`, reads the no-allocation
 * path's status word of the current device with one 4-byte device-to-host
 * copy, clears it, and returns ME_ERR_TIMEOUT if a bounded device-side wait
 * of any call since the last check gave up (ME_ERR_CUDA for a refused access
 * in the bounds-check build), else ME_OK.  Allocates nothing.  err (nullable)
 * receives a message of at most err_len bytes on failure. */
int me_noalloc_check_status(void* stream, char* err, int err_len);

/* A captured batch: the descriptor table is uploaded once and the launch
 * sequence (queue reset + search kernel) is captured in a CUDA graph that
 * me_graph_launch replays.  The frame and output buffers named by `descs`
 * must stay allocated while the graph exists.  Replays of one graph share its
 * work-queue counters, so they must not overlap on the GPU: replay it on one
 * stream, or order the streams (distinct graphs may run concurrently). */
typedef struct me_graph me_graph;
int me_graph_create(me_ctx* ctx, const me_frame_desc* descs, int n, int block, int algo,
                    me_graph** out);
int me_graph_launch(me_ctx* ctx, me_graph* g, void* stream);
void me_graph_free(me_graph* g);

/* me_fs_dual_batch: the full search of every frame for 16x16 AND 8x8 blocks
 * in one sweep (not in the paper; both block sizes of the CIF workload at
 * once).  The 16x16 accumulation keeps its four 8x8 quadrants apart, so each
 * 8x8 sub-block's SAD at every displacement of the +-range square comes out
 * of the same pass; each field is the argmin of its own candidates (the
 * 8x8 candidates limited by the 8x8 block's own frame borders) under the key
 * (SAD, |dx|+|dy|, dy, dx).  Results equal me_estimate_batch(FS) with block 16
 * on d16 and with block 8 on the 8x8 outputs.
 *   d16: as for me_estimate_batch (block 16; w, h multiples of 16).
 *   d8:  HOST array of n descriptors whose mv ([4 nb][2] int16), sad and nsp
 *        (nullable) receive the 8x8 field (raster order over the frame's
 *        2 nbx x 2 nby 8x8 blocks); its other fields are not used. */
int me_fs_dual_batch(me_ctx* ctx, const me_frame_desc* d16, const me_frame_desc* d8, int n, void* stream);

/* me_estimate_eval_batch: me_estimate_batch (DCDS or DCDS^S) with the
 * evaluation of Sec. IV fused into the search.  The search writes mv, sad
 * and nsp as me_estimate_batch does; in the same pass, from the tiles it has
 * already staged, it forms for every frame i exactly the ME_NSUMS sums that
 * me_eval_batch would compute for the resulting motion field with
 * mv = descs[i].mv, nsp = descs[i].nsp and mv_fs = mv_fs[i], so the frames are
 * read from memory once per step instead of twice.
 *   mv_fs: HOST array of n DEVICE pointers to full-search fields ([nb][2]
 *          int16, 4-byte aligned); the array or any entry may be NULL (then
 *          ME_SUM_EQUAL and ME_SUM_DIST_Q24 are 0 and ME_SUM_HAS_FS is 0).
 *   sums:  DEVICE uint64 [n][ME_NSUMS], 8-byte aligned, overwritten.
 * algo other than DCDS / DCDS^S: ME_ERR_UNSUPPORTED.  Argument errors as for
 * me_estimate_batch, plus a NULL or misaligned sums.  The tile-phase kernel
 * runs this path whatever launch shape the tuner chose. */
int me_estimate_eval_batch(me_ctx* ctx, const me_frame_desc* descs, const int16_t* const* mv_fs, int n,
                           int block, int algo, uint64_t* sums, void* stream);

/* me_graph_create_eval: me_graph_create for me_estimate_eval_batch (the
 * sums are reset and refilled by every replay).  The mv_fs array is read
 * before the call returns; the fields it points to and sums must stay
 * allocated while the graph exists. */
int me_graph_create_eval(me_ctx* ctx, const me_frame_desc* descs, const int16_t* const* mv_fs, int n,
                         int block, int algo, uint64_t* sums, me_graph** out);

/* me_estimate_host_batch: me_estimate_batch or, with `sums`, the fused
 * search and evaluation of me_estimate_eval_batch, on frames and outputs in
 * HOST memory.  Not in the paper: the upload of a batch, pipelined.  The
 * library stages the batch in device memory it owns: a copy stream of its own
 * uploads the frames of `chunk` pairs at a time, chunk k is searched on
 * `stream` while chunk k+1 uploads, and a second copy stream brings chunk k's
 * results back while later chunks upload and search.  A frame that several
 * descriptors name by the same pointer (a sequence passed as consecutive
 * pairs: ref of pair i+1 = cur of pair i) is uploaded once.  Copies of
 * buffers that are adjacent on both sides are merged.
 *   descs: HOST array; cur, ref, mv, sad and nsp (nullable) point to host
 *          memory, page-locked (cudaHostAlloc, torch pin_memory) for the
 *          copies to overlap; pageable memory gives the same results with the
 *          copies blocking the calling thread.  A frame needs
 *          (h - 1) * pitch + w readable bytes.  Device pointers also work
 *          (the copies then stay on the device).
 *   mv_fs: NULL, or a HOST array of n HOST pointers (entries may be NULL) to
 *          full-search fields ([nb][2] int16); read only when sums is set.
 *   sums:  NULL (search only, any algo but the learned one) or HOST uint64
 *          [n][ME_NSUMS] (DCDS or DCDS^S): the sums me_estimate_eval_batch
 *          writes.
 *   chunk: pairs per chunk; 0 picks ceil(n / 4); negative: ME_ERR_ARG.
 * Outputs are valid once `stream` has passed the call (for example after
 * cudaStreamSynchronize(stream)); the uploads wait until `stream` reaches the
 * call.  Two staging sets alternate between calls: a call's uploads also wait
 * for the result copies of the call before the previous one, so that calls
 * issued on two streams in turn overlap one call's uploads with the previous
 * call's last search.  The staging grows to the largest batch seen and lives
 * until me_free.  Results
 * are identical to me_estimate_batch / me_estimate_eval_batch on device
 * copies of the same data.  Argument errors as for those calls; ME_ERR_NOMEM
 * when the staging cannot be allocated. */
int me_estimate_host_batch(me_ctx* ctx, const me_frame_desc* descs, const int16_t* const* mv_fs, int n,
                           int block, int algo, uint64_t* sums, int chunk, void* stream);

/* ---------------------------------------------------------------------- */
/* Learned start proposal.  Not in the paper: libme adds a small CNN that    */
/* proposes a start point and a horizontal/vertical prior for DCDS, in the    */
/* spirit of the paper's directional conditional MVP model (Sec. II-C-2,      */
/* Sec. II-D).  One proposal per 16x16 region: a 16x16 block, or the four     */
/* 8x8 blocks of the region, which share it.                                  */
/*   features: the current region centred in a zero 32x32 canvas and the     */
/*   co-located 32x32 reference patch (clamped), both (p - 128) / 128; the    */
/*   final MVs of the left, top and top-right neighbours of the region's      */
/*   top-left block (in the grid of the search's block size) and their       */
/*   component-wise median (an absent neighbour counts as (0,0)), divided by */
/*   16: 8 scalars;                                                           */
/*   network: 4 conv 3x3 stride 2 (32 channels, ReLU) then a linear head to  */
/*   68 logits (dx in [-16,16], dy in [-16,16], H/V).  Convolutions run on    */
/*   the BF16 tensor cores with FP32 accumulation, weights rounded to bf16;  */
/*   inference carries each activation as two bf16 parts (hi + lo), so the   */
/*   logits follow the network with exact activations (to about 2e-4 for    */
/*   trained weights); training rounds each activation once to bf16.         */
/*   parameters (host float, this order): conv1.w [32][2][3][3], conv1.b      */
/*   [32], conv2.w [32][32][3][3], conv2.b, conv3.w, conv3.b, conv4.w,        */
/*   conv4.b, fc.w [68][136], fc.b [68]; fc inputs are the 128 conv-4         */
/*   outputs in (channel, y, x) order, then the 8 neighbour scalars.          */
/* Every me_proposal_* call that takes a proposal also accepts NULL: it then */
/* names the context's own proposal, which me_estimate and me_estimate_batch */
/* use for ME_ALGO_DCDS_LEARNED.  The calls that give it weights             */
/* (_set_params, _load, _train_step, _train) create it on first use; the     */
/* others return ME_ERR_ARG until it exists.  me_free releases it.           */
/* ---------------------------------------------------------------------- */
typedef struct me_proposal me_proposal;
enum { ME_PROPOSAL_NPARAMS = 37668, ME_PROPOSAL_NLOGITS = 68 };

/* Create (all parameters zero: the network then proposes the origin with a
 * horizontal prior, so the learned search starts from the better of the
 * origin and the neighbours' median) / free. */
int me_proposal_create(me_ctx* ctx, me_proposal** out);
void me_proposal_free(me_proposal* p);
/* Copy ME_PROPOSAL_NPARAMS floats in / out (HOST arrays).  Setting the
 * parameters resets the optimiser state.  Both synchronise the device. */
int me_proposal_set_params(me_ctx* ctx, me_proposal* p, const float* params);
int me_proposal_get_params(me_ctx* ctx, me_proposal* p, float* params);
/* Checkpoint and resume of training (not in the paper).  me_proposal_save
 * synchronises the device and writes the parameters, both Adam moment vectors
 * and the Adam step count to `path`: a 32-byte header (magic "MEPROP\0\1",
 * version 2, ME_PROPOSAL_NPARAMS, ME_PROPOSAL_NLOGITS, step, CRC-32 of the
 * payload, a reserved word; little-endian) followed by three float32 arrays of
 * ME_PROPOSAL_NPARAMS values in parameter order.  It writes `path`.tmp and
 * renames it over `path`, so a crash never leaves a half-written checkpoint.
 * me_proposal_load restores all of it (training then continues exactly where
 * the saved one stopped, up to the run-to-run rounding of the training
 * kernels' atomics); a file of the wrong size, magic, version or shape, or
 * whose CRC does not match, is rejected with ME_ERR_ARG and leaves `p`
 * unchanged. */
int me_proposal_save(me_ctx* ctx, me_proposal* p, const char* path);
int me_proposal_load(me_ctx* ctx, me_proposal* p, const char* path);
/* One training step over every 16x16 block of the n pairs: descs[i].mv (a
 * DEVICE motion field, e.g. the full-search field) gives the labels (dx, dy
 * clamped to +-16; H when |dx| >= |dy|) and the neighbour scalars.  The loss
 * is the mean over blocks of three softmax cross-entropies.  lr > 0 applies
 * one Adam step (beta 0.9 / 0.999); lr = 0 only computes.  *loss receives the
 * mean loss, grad (HOST, nullable) the gradient in parameter order.  At most
 * 65536 blocks per step.  Synchronises `stream`. */
int me_proposal_train_step(me_ctx* ctx, me_proposal* p, const me_frame_desc* descs, int n, float lr,
                           float* loss, float* grad, void* stream);

/* Training of the proposal, the loop in the library (not in the paper).
 * Each of `steps` steps draws pairs_per_step distinct pairs of descs (the
 * first places of a Fisher-Yates shuffle driven by SplitMix64 from `seed`, so
 * a seed repeats its sequence) and runs me_proposal_train_step on them with
 * learning rate lr.  descs: HOST array of n pairs whose mv fields are the
 * DEVICE label fields (e.g. full-search fields, 16x16 blocks).  losses: HOST
 * float [steps] receiving each step's mean loss, nullable.  Synchronises
 * `stream` at every step. */
typedef struct me_train_cfg {
    const me_frame_desc* descs;
    int32_t n;
    int32_t steps;
    int32_t pairs_per_step;  /* 1..n */
    float lr;                /* > 0 */
    uint64_t seed;
    float* losses;
    void* stream;
} me_train_cfg;
int me_proposal_train(me_ctx* ctx, me_proposal* p, const me_train_cfg* cfg);
/* Logits of every block of one pair (DEVICE float [nb][68]), the neighbour
 * scalars taken from desc->mv (a DEVICE motion field).  Synchronises
 * `stream`. */
int me_proposal_logits(me_ctx* ctx, me_proposal* p, const me_frame_desc* desc, float* logits, void* stream);
/* Learned-start DCDS over n pairs, blocks of `block` (8 or 16) pixels, w and
 * h multiples of 16.  Regions run in wavefront order so that the neighbours
 * their proposal reads are final first (16x16: t = bx + 2 by; 8x8: regions by
 * t = rx + ry, the four blocks of a region together).  The head turns those
 * MVs, their median and the region's conv features into a start (argmax of
 * the dx and dy heads, ties to the class nearest 0; the origin instead when
 * the network is not confident: the product of the two heads' softmax
 * maxima below 0.6) and a prior (V when its logit is larger).  For each block of the region the median and the start
 * are clamped to the block's window and frame; the origin, the median and
 * the start are evaluated in this order, the best one (the earliest on a
 * tie) centres the first pattern (HCSP, or its transpose for a V prior), then
 * DCDS steps 2-4 follow.  NSP counts every
 * distinct point.  Outputs go to descs[i].mv / sad / nsp; starts (DEVICE
 * int16 [total blocks][3] = sx, sy, prior per search block, clamped;
 * nullable) records the proposals.  p = NULL uses the context's own
 * proposal.  Waits between blocks are bounded (ME_ERR_TIMEOUT via
 * me_check_status).  Synchronises `stream`. */
int me_estimate_learned_batch(me_ctx* ctx, me_proposal* p, const me_frame_desc* descs, int n, int block,
                              int16_t* starts, void* stream);

/* me_estimate_median_batch: the non-learned control for the learned start
 * (not in the paper).  The same wavefront search as me_estimate_learned_batch
 * (the same block sizes, regions and neighbours), with the region's start at
 * the component-wise median of those three neighbours' final MVs (an absent
 * neighbour counts as (0,0)) and a vertical prior (the VCSP first) when the
 * median's |dy| > |dx|; each block clamps it to its window and frame.  The
 * origin and the start are evaluated, the better one (the origin on a tie)
 * centres the first pattern, then DCDS steps 2-4.  Arguments, outputs and
 * errors as for me_estimate_learned_batch; no proposal is needed.  The call
 * returns after the search (it waits on `stream`). */
int me_estimate_median_batch(me_ctx* ctx, const me_frame_desc* descs, int n, int block, int16_t* starts,
                             void* stream);

/* ---------------------------------------------------------------------- */
/* Evaluation: the six measures of Sec. IV (MAD, MSE, NSP, PSNR, distance  */
/* to the FS motion vector, probability of finding it).                    */
/* The device computes exact integer sums; me_stats_from_sums turns them   */
/* into the measures on the host.                                          */
/* ---------------------------------------------------------------------- */
enum {
    ME_SUM_ABS = 0,        /* sum over the frame of |cur - prediction| */
    ME_SUM_SQ = 1,         /* sum of (cur - prediction)^2 */
    ME_SUM_NSP = 2,        /* sum of nsp over blocks (0 if nsp is NULL) */
    ME_SUM_EQUAL = 3,      /* blocks whose MV equals the FS MV (0 if mv_fs is NULL) */
    ME_SUM_DIST_Q24 = 4,   /* sum over blocks of round(|mv - mv_fs| * 2^24) */
    ME_SUM_BLOCKS = 5,     /* number of blocks */
    ME_SUM_PIXELS = 6,     /* number of pixels */
    ME_SUM_HAS_FS = 7,     /* 1 if mv_fs was given */
    ME_NSUMS = 8
};

typedef struct me_eval_desc {
    const uint8_t* cur;
    const uint8_t* ref;
    int32_t w, h, pitch;
    const int16_t* mv;     /* [nb][2] */
    const int16_t* mv_fs;  /* [nb][2] or NULL */
    const uint16_t* nsp;   /* [nb] or NULL */
} me_eval_desc;

/* me_eval: motion-compensate `cur` from `ref` with `mv` (prediction of the
 * pixel (x, y) of block k is ref(x + dx_k, y + dy_k)) and write the
 * ME_NSUMS uint64 sums to the DEVICE array `sums` (overwritten). */
int me_eval(me_ctx* ctx, const uint8_t* cur, const uint8_t* ref, int w, int h, int block,
            const int16_t* mv, const int16_t* mv_fs, const uint16_t* nsp,
            uint64_t* sums, void* stream);

/* me_eval_batch: one launch over n frames; sums is DEVICE [n][ME_NSUMS]. */
int me_eval_batch(me_ctx* ctx, const me_eval_desc* descs, int n, int block,
                  uint64_t* sums, void* stream);

/* me_mvp_stats: the motion-vector probability statistics of Sec. II-C
 * (Tables II-V) over full-search fields, for 16x16 blocks.  descs[i].mv is
 * frame i's FS field (input, [nb][2] int16), descs[i].range its search range
 * (at most `range`); sad and nsp are not used.  out (DEVICE uint64,
 * 8-byte aligned, overwritten) receives, with Q = (2*range + 1)^2 and
 * q(dx, dy) = (dy + range) * (2*range + 1) + (dx + range):
 *   out[q]                 blocks whose FS MV (the global best-matched point,
 *                          eq. (5)) is (dx, dy)              -- Tables II, III
 *   out[Q + p*Q + q]       blocks whose current best-matched point (eq. (3))
 *                          in S1 is point p and whose FS MV is q: the prior
 *                          distribution D1 of eq. (4)        -- Table IV
 *   out[10*Q + q*25 + i]   blocks whose FS MV is q and whose current
 *                          best-matched point in S2 is point i: the
 *                          posterior distribution D2 of eq. (6) -- Table V
 * S1 = the first step of CDS as in the paper's example, in the order
 * (0,0), (-2,0), (-1,0), (1,0), (2,0), (0,2), (0,1), (0,-1), (0,-2);
 * S2 = the 5x5 square, point i = (i % 5 - 2, i / 5 - 2).  A set's current
 * best-matched point is the strict SAD minimum over its points inside the
 * window and the frame, compared with the centre first, then in the set's
 * order.  35 * Q values in all. */
int me_mvp_stats(me_ctx* ctx, const me_frame_desc* descs, int n, int range, uint64_t* out, void* stream);

typedef struct me_stats {
    double mad, mse, nsp, psnr, distance, probability;
} me_stats;

/* me_stats_from_sums: host-side arithmetic on one frame's sums (HOST array).
 * PSNR = 10 log10(255^2 / MSE), 100 dB when MSE = 0. */
int me_stats_from_sums(const uint64_t* sums, me_stats* out);

/* ---------------------------------------------------------------------- */
/* Launch shapes and the byte-absolute-difference peak.                    */
/* ---------------------------------------------------------------------- */

/* me_tune: time the candidate launch shapes for (w, h, block, range, algo)
 * on `stream` with the given frames and keep the fastest in the context
 * (and in the tune cache file, if one was named).  Outputs are overwritten.
 * Returns the chosen shape's index in *chosen (nullable). */
int me_tune(me_ctx* ctx, const uint8_t* cur, const uint8_t* ref, int w, int h, int block,
            int range, int algo, int16_t* mv, uint32_t* sad, uint16_t* nsp,
            int* chosen, void* stream);

/* me_tune_batch: the same for a batch of frame pairs (the shape is kept for
 * batches of the same block, algo, largest range and largest frame size). */
int me_tune_batch(me_ctx* ctx, const me_frame_desc* descs, int n, int block, int algo, int* chosen,
                  void* stream);

/* me_absdiff_peak: microbenchmark of the 4-byte SIMD absolute-difference
 * primitives.  Runs `iters` dependent-chain-free accumulations per thread on
 * every SM and returns the measured rate in byte-absolute-differences per
 * second for each variant (out[0..n_variants)), and which variant the
 * kernels use (*used).  Synchronises `stream`. */
int me_absdiff_peak(me_ctx* ctx, int iters, double* out, int n_variants, int* used, void* stream);

/* me_check_status: synchronise `stream` and report a device-side error that
 * a kernel recorded (ME_ERR_TIMEOUT for a bounded wait that gave up;
 * ME_ERR_CUDA for an access the bounds-check build, compiled with ME_CHECK,
 * refused); the recorded flags are cleared. */
int me_check_status(me_ctx* ctx, void* stream);

/* Tracing (not in the paper).  me_set_tracing(ctx, 1) makes every launching
 * call of this context (me_estimate, me_estimate_batch,
 * me_estimate_eval_batch, me_estimate_host_batch, me_fs_dual_batch,
 * me_graph_launch, me_eval_batch, me_mvp_stats, me_proposal_train_step,
 * me_proposal_logits, me_estimate_learned_batch, me_estimate_median_batch)
 * open an NVTX range named after the call around its host part (visible to
 * Nsight tools, free without one) and record CUDA events around its work on
 * its stream; a call that ends by synchronising its stream records the
 * closing event before that wait.  me_last_call_ms waits for the last traced
 * call's work and returns its device time in ms (ME_ERR_UNSUPPORTED before
 * any traced call).  Off by default. */
int me_set_tracing(me_ctx* ctx, int on);
int me_last_call_ms(me_ctx* ctx, float* ms);

/* me_inject_wait_timeout: failure-detection test hook (not in the paper).
 * While `on` is non-zero, every DCDS / DCDS^S launch of this context that
 * runs the tile kernel (me_estimate, me_estimate_batch, the fused and host
 * batches, graphs captured meanwhile) arms each CTA's first tile-copy barrier
 * for 16 bytes more than the copy delivers.  The copies land, the barrier
 * never completes, and each CTA's bounded wait (shortened to a few thousand
 * polls) gives up, records the time-out and exits: the launch writes no
 * output and the next me_check_status returns ME_ERR_TIMEOUT.  In the
 * wavefront searches (me_estimate_learned_batch, me_estimate_median_batch)
 * the blocks of the first region in wavefront order then never publish their
 * hand-off words:
 * the blocks that wait for it give up after a shortened wait (taking that
 * neighbour as absent), record the time-out and go on, so every block is
 * written and the next me_check_status returns ME_ERR_TIMEOUT.  Nothing faults,
 * traps or hangs, and the context stays usable: with `on` = 0 the next launch
 * is a normal one.  The no-allocation path has no context: ctx = NULL arms
 * the same hook for every later me_estimate_batch_noalloc call in the
 * process (its time-out is then reported by me_noalloc_check_status). */
int me_inject_wait_timeout(me_ctx* ctx, int on);

#ifdef __cplusplus
}
#endif

#endif /* ME_H */
