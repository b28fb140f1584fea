/*
 * wt.h -- C ABI of the warp-tiled image-pipeline library (GB300, sm_103a).
 *
 * The library executes a DAG of stencil, pointwise and down/up-sampling
 * stages over images as fused groups of warp-sized overlapped tiles, after
 * Jangda & Guha, "Model-Based Warp Overlapped Tiling for Image Processing
 * Programs on GPUs" (PACT'20).  Section numbers below refer to that paper.
 *
 * Conventions for every entry point:
 *   - Returns wt_status (WT_OK == 0); on failure wt_last_error() gives a
 *     thread-local message.  No entry point aborts the process.
 *   - Images are caller-owned.  Device images live in device memory of the
 *     current CUDA device; "host" images live in host memory.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default).
 *   - Pointers named *out are written only on success.
 */
#ifndef WT_H
#define WT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  WT_OK = 0,
  WT_EINVAL = -1,       /* malformed argument or DAG                         */
  WT_ENOMEM = -2,       /* host or device allocation failed                  */
  WT_ECUDA = -3,        /* a CUDA runtime/driver call failed                 */
  WT_EUNSUPPORTED = -4, /* valid request this build does not implement       */
  WT_ETIMEOUT = -5,     /* a device-side bounded wait gave up                */
  WT_EDEVICE = -6,      /* a device-side check raised the error word         */
  WT_ECOMPILE = -7      /* run-time compilation of a group kernel failed     */
} wt_status;

/* Storage types.  Arithmetic is always FP32; 16-bit types are storage only
 * (round to nearest even on store, exact widening on load).               */
typedef enum { WT_F32 = 0, WT_F16 = 1, WT_BF16 = 2 } wt_dtype;

/* ------------------------------------------------------------ stage DAG -- */

/* Postfix opcodes of a stage program (Sec. 2.2 Fig. 2: each stage is a
 * per-point function of producer values).                                 */
typedef enum {
  WT_OP_CONST = 1, /* push `value`                                           */
  WT_OP_TAP = 2,   /* push producer inputs[slot] at a constant offset        */
  WT_OP_ADD = 3, WT_OP_SUB = 4, WT_OP_MUL = 5, WT_OP_DIV = 6,
  WT_OP_MIN = 7, WT_OP_MAX = 8,
  WT_OP_NEG = 9, WT_OP_ABS = 10, WT_OP_SQRT = 11,
  WT_OP_XPAR = 12, /* push (x & 1) of the output point, as 0.0 or 1.0       */
  WT_OP_YPAR = 13, /* push (y & 1) of the output point                      */
  WT_OP_CHAN = 14, /* push the output point's channel index (0.0, 1.0, ...):
                      per-plane programs such as a histogram's bins         */
  /* 3-D tap (App. A, groups over volumes): a D x H x W volume is an image
   * of D planes; push producer inputs[slot] at (x + dx, y + dy) of plane
   * clamp(z + chan, 0, D - 1), z = the output point's plane.  `chan` holds
   * the plane offset dz (-16..16); mode must be WT_TAP_SAME; the producer
   * has the stage's plane count, or one plane (then plane 0 is read).     */
  WT_OP_TAPZ = 15
} wt_opcode;

/* How a tap maps the output point (x, y) to the producer point; these are
 * the constant dependence vectors after alignment and scaling (Sec. 2.3,
 * Sec. 5).  The producer coordinate is clamped to the producer's domain
 * (clamp-to-edge at every producer read).                                  */
typedef enum {
  WT_TAP_SAME = 0,  /* P(x + dx, y + dy)                        */
  WT_TAP_DOWN2 = 1, /* P(2x + dx, 2y + dy)   producer one level finer   */
  WT_TAP_UP2 = 2,   /* P(x/2 + dx, y/2 + dy) producer one level coarser */
  WT_TAP_DOWN4 = 3, /* P(4x + dx, 4y + dy)   two levels finer            */
  WT_TAP_UP4 = 4,   /* P(x/4 + dx, y/4 + dy) two levels coarser          */
  WT_TAP_DOWN8 = 5, /* P(8x + dx, 8y + dy)   three levels finer          */
  WT_TAP_UP8 = 6    /* P(x/8 + dx, y/8 + dy) three levels coarser        */
} wt_tapmode;       /* (divisions round down; odd modes scale down, even up) */

typedef struct {
  int32_t op;   /* wt_opcode                                                 */
  int32_t slot; /* TAP: index into the stage's `inputs`                      */
  int32_t dx, dy;
  int32_t chan; /* TAP: producer channel; -1 = the output point's channel
                   (channel 0 if the producer has one channel)              */
  int32_t mode; /* TAP: wt_tapmode                                           */
  float value;  /* CONST                                                     */
} wt_op;

typedef struct {
  int32_t channels;      /* planes of this stage's output (>= 1)            */
  int32_t n_inputs;
  const int32_t *inputs; /* producer ids: stage index < this stage's index,
                            or -(j+1) for pipeline input j                  */
  int32_t n_ops;
  const wt_op *ops;      /* postfix program, at most 256 ops, stack <= 32   */
} wt_stage;

/* An image: `channels` planes of height x width elements of `dtype`, rows
 * `pitch_bytes` apart, plane c starting at data + c * height * pitch_bytes.
 * pitch_bytes must be a multiple of 16 and data 16-byte aligned (TMA rule). */
typedef struct {
  void *data;
  int32_t width, height, channels;
  int32_t dtype; /* wt_dtype */
  int64_t pitch_bytes;
} wt_image;

typedef struct wt_pipeline wt_pipeline;

#define WT_BOUNDARY_CLAMP 0

/* Builds a pipeline from a stage DAG (Sec. 2.2-2.3; Fig. 4 "Create DAG").
 * stages are in topological order; input_channels[j] gives the planes of
 * pipeline input j; outputs are stage ids.  All inputs share one width and
 * height (level 0); a stage's level follows from its taps (DOWN2 +1, UP2
 * -1) and level l has width ceil(W / 2^l).  Copies everything it needs.
 * Errors: WT_EINVAL (cycle/forward reference, mixed levels, negative level,
 * bad program, bad channel), WT_EUNSUPPORTED (boundary other than clamp). */
wt_status wt_pipeline_create(const wt_stage *stages, int32_t n_stages,
                             const int32_t *input_channels, int32_t n_inputs,
                             const int32_t *outputs, int32_t n_outputs,
                             int32_t boundary, wt_pipeline **out);

wt_status wt_pipeline_destroy(wt_pipeline *p);

/* ------------------------------------------------------------- schedule -- */

/* Per-group execution parameters (Sec. 4 OTPW tile, Sec. 5 hybrid tiling). */
typedef struct {
  int32_t tile_h;          /* T_y: output rows per warp tile (>= 1; default
                              40).  Single-image runs too small to give the
                              resident warps about 1.5 tiles each use a
                              shorter height of the same parity.             */
  int32_t warps_per_block; /* 1..16 (default 1); warps are independent (no
                              block sync)                                   */
  float frac_reg;          /* fracReg in [0,1]: share of the group's
                              intermediate window bytes kept in registers;
                              the rest lives in the warp's shared memory    */
  int32_t vec;             /* pixels per lane along x: 4 or 8 (0 = auto)     */
  int32_t max_regs;        /* register cap per thread (0 = 255)             */
  int32_t chunk_rows;      /* TMA staging rows per chunk (0 = 8)             */
  int32_t n_buffers;       /* TMA staging buffers per input (0 = 2)          */
  int32_t flags;           /* WT_FLAG_* bits; 0 = all features on            */
  int32_t tile_o;          /* 3-D groups: points of the axis that is neither
                              x nor streamed (planes, or rows with
                              WT_FLAG_ZSTREAM) per warp tile, held in
                              registers (0 = 4)                              */
} wt_group_params;

#define WT_FLAG_NO_PAIRS 1      /* scalar FP32 instead of packed f32x2 pairs     */
#define WT_FLAG_NO_TILE_SPLIT 2 /* one tile height (no short last round)         */
#define WT_FLAG_PLAIN 4         /* the group's stages as per-stage kernels       */
/* One overlapped tile per thread block (Sec. 3, Fig. 3: the tiling of the
 * systems the paper compares with): each block computes a (32 vec) x tile_h
 * output tile, every stage of the group over its tile-plus-halo region in
 * shared memory, block barriers between stages; vec may be 1, 2, 4 or 8;
 * warps_per_block sets the block size; frac_reg, chunk_rows, n_buffers and
 * the other flags are ignored.  Groups that read other levels
 * (down/up-sampling taps into the group) return WT_EUNSUPPORTED at run. */
#define WT_FLAG_OTPTB 8
/* Shared-memory windows of intermediates (the share 1 - frac_reg) stored
 * in the group's 16-bit storage type (that of its first staged source) when
 * it is FP16 or BF16, halving their bytes; values are rounded to that type
 * (RNE) when stored, arithmetic stays FP32.  No effect on FP32 groups.     */
#define WT_FLAG_SMEM16 16
/* Groups with plane-offset taps (WT_OP_TAPZ) run as 3-D warp tiles (App. A
 * generalised hybrid tiling): lanes along x (vec = 1, 2 or 4 points each,
 * 0 = 2), tile_h points along the streamed (split) axis, tile_o points of
 * the third axis in registers.  The split axis is y (rows) by default; with
 * this flag it is z (planes) and tile_o counts rows.  frac_reg = 1 keeps
 * source rows in registers; below 1 they are staged in the warp's shared
 * memory by asynchronous copies; n_buffers (1..8) sets how many rows ahead
 * of their first use source rows are loaded.  chunk_rows and the other
 * flags are ignored for such groups; a group the
 * 3-D kernel cannot take (other levels, parity or channel ops, fixed-
 * channel taps, windows above 224 registers) runs per stage.              */
#define WT_FLAG_ZSTREAM 32
/* Test only (failure detection without a GPU fault): in warp-tile group
 * kernels the first staging chunk of every tile is armed for bytes that no
 * copy delivers (no copy is issued for it, so nothing is in flight) and
 * bounded waits give up after 256 polls.  Every warp's first wait times
 * out, raises the error word and the warp drains its other copies and
 * exits; the run writes no output and wt_check() returns WT_ETIMEOUT.
 * Other kernel kinds ignore the flag.                                      */
#define WT_FLAG_TEST_STALL 64
/* Warp-tile kernels of single-image runs launch one warp per tile (blocks
 * of warps_per_block warps, handed out by the hardware in tile order: the
 * edge columns' tiles first, tall tiles before a band of short ones).  With
 * this flag a persistent grid (the resident capacity) pulls tiles from a
 * device queue instead (the batched kernels always do).                  */
#define WT_FLAG_TILE_QUEUE 128
/* Set on any group of a schedule, a run issues all its launches in plan
 * order on the caller's stream.  Without it, launches that read nothing an
 * earlier launch of the run writes (another pyramid's down-sampling, an
 * independent stage) run concurrently on up to three side streams of the
 * pipeline, forked from the caller's stream at the run's first launch and
 * joined back into it after the last, so the run still begins and ends in
 * the caller's stream order (and a CUDA graph captured from that stream
 * holds the launches as parallel branches).                               */
#define WT_FLAG_ONE_STREAM 256
/* Warp-tile group kernels normally defer the constant factors of stage
 * programs (a filter's normalisation, a weight) to the stages that read
 * them: a value in registers may hold the stage's value divided by a
 * compile-time constant, the factor is merged into the next constant or
 * product and applied once where a value leaves the kernel (HBM stores,
 * 16-bit shared-memory windows).  Results differ from the undeferred
 * evaluation by rounding only.  This flag evaluates every stage as
 * written.                                                                 */
#define WT_FLAG_NO_FOLD 512

typedef enum {
  WT_EXEC_FUSED = 0, /* warp-tiled group kernels (OTPW + hybrid tiling)     */
  WT_EXEC_PLAIN = 1  /* one simple kernel per stage, every intermediate in
                        HBM: the unfused "plain method" baseline            */
} wt_exec;

typedef struct {
  int32_t exec;                  /* wt_exec                                  */
  int32_t n_groups;              /* FUSED: groups in topological order       */
  const int32_t *group_of_stage; /* FUSED: n_stages entries in [0, n_groups);
                                    every group a contiguous run of stages   */
  const wt_group_params *params; /* FUSED: n_groups entries (NULL: defaults) */
  int32_t intermediate_dtype;    /* storage of HBM intermediates (wt_dtype);
                                    -1: FP32 for WT_EXEC_PLAIN (the unfused
                                    baseline), else the first input's dtype */
} wt_schedule_desc;

/* Installs an explicit schedule.  Groups whose taps change level are run
 * with the per-stage kernel.  Kernels are compiled lazily (NVRTC, sm_103a)
 * on the first run of each group and cached per device.  WT_EINVAL if the
 * grouping is not contiguous or parameters are out of range.              */
wt_status wt_schedule(wt_pipeline *p, const wt_schedule_desc *desc);

/* Cost models used by wt_schedule_auto (Sec. 6).                           */
typedef enum {
  WT_MODEL_ANALYTIC = 0, /* Alg. 2 weighted cost, DP over groupings          */
  WT_MODEL_LEARNED = 1   /* 3-layer MLP trained on measured runtimes        */
} wt_model;

/* Picks grouping, tile heights and fracReg for images of the given size and
 * storage type by DP-Fusion over contiguous groupings with the chosen cost
 * model (Sec. 2.4, Sec. 6), then installs the schedule.                    */
wt_status wt_schedule_auto(wt_pipeline *p, int32_t width, int32_t height,
                           int32_t dtype, int32_t model);

/* Reads back the installed schedule: n_groups, group_of_stage (n_stages
 * entries, caller-allocated, may be NULL) and params (n_groups entries,
 * caller-allocated, may be NULL).                                          */
wt_status wt_schedule_get(const wt_pipeline *p, int32_t *exec, int32_t *n_groups,
                          int32_t *group_of_stage, wt_group_params *params);

/* --------------------------------------------------- cost model (Sec. 6) -- */

/* Sec. 6 preprocessing: runs each stage's body alone in a one-thread
 * micro-kernel on the current GPU and records its time per iteration
 * (ns_per_iter[s]) and register count (regs[s]); either array (n_stages
 * entries) may be null.  The pipeline keeps the results and the analytic
 * cost model, the learned model's features and the measured search use
 * them from then on (before, they use estimates from the stage programs).
 * WT_ECUDA without a GPU.                                                  */
wt_status wt_preprocess(wt_pipeline *p, double *ns_per_iter, int32_t *regs);

/* GPU quantities the cost function uses (Table 1).                         */
typedef struct {
  int32_t nsms, cores_per_sm;
  double glmem_bw_gbs;
  int32_t max_smem_per_block, smem_per_sm, max_warps_per_sm, max_blocks_per_sm;
  int32_t regs_per_sm, max_regs_per_thread, warp_size, max_threads_per_sm;
} wt_gpu_config;

/* Configuration of CUDA device `device`, or (device < 0) of a GB300 from
 * its published figures with the measured copy bandwidth of 6781 GB/s.   */
wt_status wt_gpu_config_get(int32_t device, wt_gpu_config *out);

/* Sec. 4: warp sizes of a thread block, W_x = min(B_x, WarpSize),
 * W_y = min(B_y, WarpSize / W_x), W_z = min(B_z, WarpSize / (W_x W_y)).    */
wt_status wt_otpw_warp_sizes(const int32_t block[3], int32_t warp_size, int32_t warp[3]);

/* Sec. 4: points of one stage's scratchpad per thread block,
 * prod_i ceil(B_i / W_i) * (T_i W_i + O_i).                               */
wt_status wt_otpw_scratchpad(const int32_t block[3], const int32_t warp[3], const int32_t tile[3],
                             const int32_t overlap[3], int64_t *points);

/* Alg. 2 theoretical occupancy from shared memory per block, warps per
 * block and registers per thread (fraction of MaxWarpPerSM).              */
wt_status wt_cost_occupancy(const wt_gpu_config *cfg, int64_t smem_per_block, int32_t warps_per_block,
                            int32_t regs_per_thread, double *occupancy, int32_t *blocks_per_sm);

/* Minimum number of txn_bytes-sized, txn_bytes-aligned transactions that
 * cover n accesses of access_bytes each (Alg. 2 MinGLTxs).               */
wt_status wt_min_transactions(const int64_t *byte_addresses, int32_t n, int32_t access_bytes,
                              int32_t txn_bytes, int64_t *txns);

/* Alg. 2 terms of one candidate group: [0] global traffic relative to the
 * pipeline's minimum bytes, [1] 1 - occupancy, [2] memTime / computeTime,
 * [3] unallocated shared memory, [4] unused registers, [5] fraction of
 * overlapped (redundant) computation, [6] idle fraction of the last wave. */
typedef struct {
  double terms[7];
  double cost;       /* weighted sum (wt_cost_weights)                     */
  int32_t feasible;  /* 0: the candidate exceeds shared memory/registers  */
  int32_t regs_per_thread;
  int32_t smem_per_block;
  double occupancy, waves, work;
} wt_cost_info;

/* Cost of running stages [first_stage, first_stage + n_stages) as one
 * fused group with parameters prm and txn_bytes (32 or 128) transactions
 * on width x height images of dtype; cfg NULL = GB300 defaults.          */
wt_status wt_cost_group(wt_pipeline *p, int32_t first_stage, int32_t n_stages, const wt_group_params *prm,
                        int32_t txn_bytes, int32_t width, int32_t height, int32_t dtype,
                        const wt_gpu_config *cfg, wt_cost_info *out);

/* Gets and/or sets the seven cost weights w1..w7 of Alg. 2 (either pointer
 * may be NULL).  Defaults: Table 3's Tesla V100 weights.                  */
wt_status wt_cost_weights(const double *set7, double *get7);

/* ------------------------------------------------------------------ run -- */

/* Runs the pipeline on device images, asynchronously on `stream`
 * (Fig. 4 "CUDA code generation" output, Sec. 4-5 execution).  inputs[j]
 * match input_channels[j]; outputs[k] must have the level/size/channels of
 * stage outputs[k].  Input and output dtypes may differ.  The first run for
 * a new image size allocates the library's device workspace and compiles
 * the group kernels; later runs allocate nothing and may be captured in a
 * CUDA graph.  Launches that read nothing an earlier launch of the run
 * writes run concurrently on the pipeline's side streams (WT_FLAG_ONE_STREAM
 * describes the fork and join); the run as a whole stays ordered on
 * `stream`.  The intermediates, the side streams and their events belong to
 * the pipeline, so runs of one pipeline must not overlap on the GPU (issue
 * them on one stream, or order their streams); separate pipelines may run
 * at the same time.  Device-side failures are reported by wt_check().
 * Size limits (WT_EUNSUPPORTED when exceeded, before any launch): a fused
 * warp-tile group at most 2^30 tiles (a batch: 2^30 over all its images);
 * a block-tile group at most 65535 rows of tiles; per-stage and
 * reduction-chain kernels at most 65535 rows of the image they write;
 * down-sampling and cascade kernels at most 65535 row blocks; block-tile,
 * per-stage, down-sampling and cascade kernels at most 65535 planes.      */
wt_status wt_run(wt_pipeline *p, const wt_image *inputs, int32_t n_inputs,
                 const wt_image *outputs, int32_t n_outputs, void *stream);

/* Same computation with host buffers: copies inputs to device (inside the
 * call), runs, copies outputs back; returns when the outputs are on the
 * host.  Work is ordered after earlier work on `stream`.  Host images use
 * the same layout rules; pinned memory makes the copies asynchronous.
 * Pipelines whose stages are all at level 0, with one-plane inputs of at
 * least 16 MiB, run in 2 to 8 row bands of at least 8 MiB of input (each
 * band's rows plus the pipeline's row halo, starting on an even row so
 * that WT_OP_YPAR reads the whole image's row parity; results identical to
 * the whole-image run) with the copy-in, the compute and the copy-out of
 * consecutive bands overlapped on the library's own streams.  The second call with the same host image descriptors
 * captures that work as a CUDA graph; later calls with them replay it (a
 * new schedule or larger staging discards the captured graphs).  Device
 * staging buffers are allocated on first use and kept.                    */
wt_status wt_run_host(wt_pipeline *p, const wt_image *inputs, int32_t n_inputs,
                      const wt_image *outputs, int32_t n_outputs, void *stream);

/* Batched serving: n_images independent runs (inputs[i*n_inputs + j],
 * outputs[i*n_outputs + k], with n_inputs/n_outputs the pipeline's counts)
 * of images of any sizes.  Each schedule group runs as ONE persistent
 * launch whose warps pull warp tiles of every image from one device work
 * queue (tile list: image, tile column, tile row, channel), so the batch
 * costs one launch per group.  Every group of the schedule must fuse
 * (WT_EUNSUPPORTED otherwise) and all images must share channels and
 * dtypes (WT_EINVAL).  The first call for a set of image descriptors
 * plans, compiles, allocates and uploads the tables (synchronizing
 * `stream`); later calls with the same descriptors only launch, so they may
 * be captured in a CUDA graph.  Intermediates between groups live in the
 * pipeline's workspace, one slice per image.                               */
wt_status wt_run_batch(wt_pipeline *p, const wt_image *inputs,
                       const wt_image *outputs, int32_t n_images, void *stream);

/* ------------------------------------------- measured schedule search -- */

/* Kernel time of the installed schedule on these images: 3 samples of
 * `reps` back-to-back runs on `stream`, the minimum of the sample means
 * (the timing protocol of Sec. 7), in *ms per run.  n_images = 0 times
 * wt_run(inputs, n_inputs, outputs, n_outputs); n_images >= 1 times
 * wt_run_batch over n_images images (n_inputs, n_outputs ignored).  The
 * first runs (planning, compilation) are not timed.  WT_EDEVICE if a timed
 * run raised the device error word.                                       */
wt_status wt_schedule_time(wt_pipeline *p, const wt_image *inputs, int32_t n_inputs,
                           const wt_image *outputs, int32_t n_outputs, int32_t n_images,
                           int32_t reps, void *stream, double *ms);

/* The schedule search with device timings in place of the cost model's
 * estimate (an autotuner), on the caller's images (same conventions as
 * wt_schedule_time).  Candidates: the DP-Fusion grouping of the analytic
 * model and, when it fuses, the whole pipeline as one group; then per group
 * the max_variants (0 = 12) kernel variants -- warps per block, pixels per
 * lane, register/shared placement, staging buffers -- that the analytic
 * cost ranks best, and tile heights for the two fastest.  Kernels are
 * compiled in parallel host threads first.  Installs the fastest schedule
 * timed and returns its time (*best_ms) and the number of schedules timed
 * (*n_timed; either may be null).  On failure the previous schedule stays
 * installed.  Writes the outputs (every candidate runs).                   */
wt_status wt_schedule_tune(wt_pipeline *p, const wt_image *inputs, int32_t n_inputs,
                           const wt_image *outputs, int32_t n_outputs, int32_t n_images,
                           int32_t max_variants, int32_t reps, void *stream, double *best_ms,
                           int32_t *n_timed);

/* Compiles (NVRTC, parallel host threads) the kernels that these n_descs
 * schedules would launch on these images (batched != 0: the persistent
 * batch kernels), filling the process and disk kernel caches; runs nothing
 * and installs nothing.  Schedules that do not plan are skipped.           */
wt_status wt_prepare(wt_pipeline *p, const wt_schedule_desc *descs, int32_t n_descs,
                     const wt_image *inputs, int32_t n_inputs, const wt_image *outputs,
                     int32_t n_outputs, int32_t batched);

/* Per-launch kernel times of one wt_run of the installed schedule on these
 * images: each launch repeated `reps` times on its own (it re-reads what the
 * earlier launches wrote), 3 samples, the minimum of the means.  ms[i] and
 * info[3i..3i+2] = (first stage, stage count, fused 1 / per-stage 0) for
 * launch i, in launch order; *n_launches gets the count (arrays of `cap`
 * entries; WT_EINVAL if too small).  Training data of the learned model.  */
wt_status wt_schedule_time_launches(wt_pipeline *p, const wt_image *inputs, int32_t n_inputs,
                                    const wt_image *outputs, int32_t n_outputs, int32_t reps,
                                    void *stream, double *ms, int32_t *info, int32_t cap,
                                    int32_t *n_launches);

/* ------------------------------------------------- learned cost model -- */

/* A 3-layer FP32 MLP, WT_COSTMODEL_FEATURES -> 64 -> 64 -> 1 with ReLU, that
 * predicts the natural log of one launch's kernel time in ms.  The paper's
 * cost function is a hand-weighted sum of Alg. 2's terms whose weights are
 * fitted per GPU (Sec. 6, Table 3); this model is trained instead on times
 * the library measures.  Training and inference run in hand-written CUDA
 * kernels; wt_schedule_auto(..., WT_MODEL_LEARNED) uses a trained or loaded
 * model and falls back to the analytic model without one.                 */
#define WT_COSTMODEL_FEATURES 18
#define WT_COSTMODEL_HIDDEN 64
/* parameters, in order: W1[64][18], b1[64], W2[64][64], b2[64], w3[64], b3 */
#define WT_MLP_PARAMS (64 * 18 + 64 + 64 * 64 + 64 + 64 + 1)

/* Features of one launch at image size width x height (level-0 pixels) and
 * storage dtype: stages [first_stage, first_stage + n_stages) as one fused
 * group with `params` (fused = 1), or stage first_stage's per-stage kernel
 * (fused = 0, n_stages = 1, params may be null).  features[18] = log2 of the
 * group's pixels, stages, computed nodes, operations per pixel, bytes read
 * and written per pixel, y and x footprint growth, log2 tile height,
 * pixels per lane, warps per block, fracReg, registers/255, shared bytes per
 * block/227 KB, Alg. 2 occupancy, redundant-compute fraction, tail
 * fraction, fused.  WT_EUNSUPPORTED if the launch is infeasible.           */
wt_status wt_costmodel_features(wt_pipeline *p, int32_t first_stage, int32_t n_stages,
                                const wt_group_params *params, int32_t fused, int32_t width,
                                int32_t height, int32_t dtype, float *features);

/* Training data of the learned model from one run of the installed
 * schedule on these images (single-image runs, Sec. 6's measured inputs of
 * the cost function): every launch of the run is timed as by
 * wt_schedule_time_launches (`reps` repetitions, 3 samples, the minimum of
 * the means) and described by its features as by wt_costmodel_features
 * (fused groups with their schedule parameters, per-stage kernels without).
 * features[i * WT_COSTMODEL_FEATURES ...] and log_ms[i] (natural log of
 * ms) for row i; stages[2i], stages[2i+1] (may be null) = the launch's
 * first stage and stage count.  Launches of other kinds (reduction chains,
 * down-sampling streams and cascades, 3-D groups, block tiles) have no
 * features and are skipped.  *n_rows gets the row count; arrays of `cap`
 * rows (null arrays with cap 0 size the call; WT_EINVAL if too small).
 * Writes the outputs (the run executes).                                   */
wt_status wt_costmodel_collect(wt_pipeline *p, const wt_image *inputs, int32_t n_inputs,
                               const wt_image *outputs, int32_t n_outputs, int32_t reps, void *stream,
                               float *features, float *log_ms, int32_t *stages, int32_t cap,
                               int32_t *n_rows);

/* The MLP training kernel: `steps` Adam steps (beta 0.9/0.999, eps 1e-8,
 * t0 steps taken before) on the mean squared error over mini-batches
 * idx[steps][batch] of rows of x[n][18] with targets y[n], decoupled L2
 * weight decay on the weight matrices.  params, adam_m, adam_v
 * (WT_MLP_PARAMS floats each, host memory) are read and updated; loss[k]
 * (may be null) = batch mean squared error before step k.  batch in
 * [1, 128].  Synchronizes `stream`.                                        */
wt_status wt_mlp_train_steps(float *params, float *adam_m, float *adam_v, int32_t t0,
                             const float *x, const float *y, int32_t n, const int32_t *idx,
                             int32_t steps, int32_t batch, float lr, float weight_decay,
                             float *loss, void *stream);
/* The MLP inference kernel: y[i] = MLP(params; x[i]) for n rows (host
 * arrays).  Synchronizes `stream`.                                          */
wt_status wt_mlp_forward(const float *params, const float *x, int32_t n, float *y, void *stream);

/* Trains the process-wide model on n (features, log ms) pairs: features and
 * targets standardised over the set, He-initialised weights and mini-batch
 * order from `seed`, `epochs` passes of Adam (learning rate lr, batch in
 * [1, 128]) on the GPU; installs it.  *final_loss (may be null) = mean
 * squared error of the last epoch, in standardised units.                 */
wt_status wt_costmodel_train(const float *features, const float *log_ms, int32_t n, int32_t epochs,
                             int32_t batch, float lr, uint64_t seed, float *final_loss);
/* Predicted log ms of n launches (features as wt_costmodel_features).
 * WT_EUNSUPPORTED without a model.                                          */
wt_status wt_costmodel_predict(const float *features, int32_t n, float *log_ms);
/* 1 if a model is trained or loaded.                                       */
int32_t wt_costmodel_ready(void);
/* Drops the model (the analytic model is used again).                      */
wt_status wt_costmodel_reset(void);
/* Writes / reads the model (standardisation and parameters) as text.       */
wt_status wt_costmodel_save(const char *path);
wt_status wt_costmodel_load(const char *path);

/* Runs like wt_run, but allocates no device memory.  The paper has no
 * counterpart: this is for callers that cannot let a library call
 * cudaMalloc -- processes whose device memory is handed to their own
 * allocator up front under a fixed budget, and latency-critical paths where
 * cudaMalloc/cudaFree may synchronize the device.  Intermediates between
 * groups, the device status word and the tile-queue counters live in one
 * file-scope static device array of 32 MiB, held by every GPU that loads
 * the library until exit: a 4 KiB control block, then at most
 * 32 MiB - 4 KiB of intermediates; runs needing more are rejected with
 * WT_EINVAL (single-group schedules need none).  The first call on a device
 * takes the array's address (cudaGetSymbolAddress).  It never compiles or
 * loads kernels, because loading code allocates device memory: run the same
 * schedule and image sizes/dtypes once with wt_run first, else
 * WT_EUNSUPPORTED.  Every call on a device shares the array and the array
 * keeps the last call's contents; each call clears the control block on
 * `stream`.  Calls whose work overlaps on the GPU (other streams, or before
 * an earlier call's kernels finished) race on the array.  Device-side
 * failures (bounded waits, device checks) are reported by wt_check() of the
 * pipeline, which reads the static status word once a wt_run_static call
 * has run it on the current device.                                       */
wt_status wt_run_static(wt_pipeline *p, const wt_image *inputs, int32_t n_inputs,
                        const wt_image *outputs, int32_t n_outputs, void *stream);

/* Synchronizes `stream` and reads the device error word of the pipeline
 * (and, after wt_run_static on the current device, the static scratch's
 * status word, which every wt_run_static call on the device shares):
 * WT_ETIMEOUT if a bounded mbarrier/queue wait gave up, WT_EDEVICE for any
 * other device-side check; clears the words.                               */
wt_status wt_check(wt_pipeline *p, void *stream);

/* Number of kernel launches one wt_run issues with the installed schedule. */
int32_t wt_launches_per_run(const wt_pipeline *p);

const char *wt_last_error(void);

/* Library version (major*10000 + minor*100 + patch). */
int32_t wt_version(void);

#ifdef __cplusplus
}
#endif
#endif
