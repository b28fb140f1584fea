/*
 * wt_debug.h -- introspection entry points of the warp-tiled pipeline
 * library, for tests and tools.  They never launch GPU work.
 */
#ifndef WT_DEBUG_H
#define WT_DEBUG_H

#include "wt.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Size in bytes of the argument block every generated kernel takes. */
int64_t wt_debug_args_size(void);

/* Describes launch `launch_index` of the run plan that wt_run would build
 * for these images with the installed schedule, without running it:
 *   src/src_cap/src_len: generated CUDA source (NUL-terminated, truncated to
 *                        src_cap-1 bytes; src_len gets the full length);
 *   args/args_cap:       the kernel's argument block (wt_debug_args_size()
 *                        bytes), with tensor maps left zero;
 *   launch[8]:           grid x, y, z, threads per block, dynamic shared
 *                        bytes, fused (1) or per-stage (0), launches in the
 *                        plan, unroll factor;
 *   kname:               the kernel's entry-point name.
 * Image pointers may be host pointers.  WT_EUNSUPPORTED if the launch reads
 * or writes the library workspace (intermediates between groups).          */
wt_status wt_debug_kernel(wt_pipeline *p, int32_t launch_index, const wt_image *inputs,
                          int32_t n_inputs, const wt_image *outputs, int32_t n_outputs, char *src,
                          int64_t src_cap, int64_t *src_len, void *args, int64_t args_cap,
                          int32_t *launch, char *kname, int64_t kname_cap);

/* Describes launch `launch_index` of the batched run wt_run_batch would
 * make for these n_images images (inputs[i*n_inputs + j], outputs[i*n_outputs
 * + k]), without running it: the persistent kernel's source, its top-level
 * argument block (tile count and image count set; table, queue and error
 * pointers left zero for the caller), the n_images per-image argument blocks
 * (wt_debug_args_size() bytes each, tensor maps in the introspection
 * encoding of wt_debug_kernel) and the tile list, 4 int32 per tile (image,
 * tile column, tile row, channel).  *n_tiles gets the tile count; null
 * buffers are skipped, so a first call with nulls sizes them.  launch[8] as
 * for wt_debug_kernel.  WT_EUNSUPPORTED if a group does not fuse.           */
wt_status wt_debug_batch(wt_pipeline *p, int32_t launch_index, const wt_image *inputs,
                         const wt_image *outputs, int32_t n_images, char *src, int64_t src_cap,
                         int64_t *src_len, void *args, void *img_tab, int64_t img_tab_cap,
                         int32_t *tiles, int64_t tiles_cap, int64_t *n_tiles, int32_t *launch,
                         char *kname, int64_t kname_cap);

/* wt_debug_kernel with the plan's workspace (intermediates between groups)
 * placed at `workspace` (ws_cap bytes; may be null, then launches that use
 * it fail as above).  *ws_bytes (may be null) gets the workspace size the
 * plan needs.                                                               */
wt_status wt_debug_kernel_ws(wt_pipeline *p, int32_t launch_index, const wt_image *inputs,
                             int32_t n_inputs, const wt_image *outputs, int32_t n_outputs,
                             void *workspace, int64_t ws_cap, char *src, int64_t src_cap,
                             int64_t *src_len, void *args, int64_t args_cap, int32_t *launch,
                             char *kname, int64_t kname_cap, int64_t *ws_bytes);

/* Compiles launch `launch_index` of that run plan with NVRTC for sm_103a
 * (no GPU needed) and returns the CUBIN size; WT_ECOMPILE with the NVRTC
 * log in wt_last_error() on failure.                                       */
wt_status wt_debug_compile(wt_pipeline *p, int32_t launch_index, const wt_image *inputs,
                           int32_t n_inputs, const wt_image *outputs, int32_t n_outputs,
                           int64_t *cubin_bytes);

/* Shared-memory layout of fused launch `launch_index` for these images:
 * out = [bytes per warp, mbarrier offset, chunk rows, buffers, pixels per
 * lane, output columns per warp tile, n_sources, then per source: staging
 * ring offset, bytes per buffer, TMA box width (elements), element bytes]. */
wt_status wt_debug_layout(wt_pipeline *p, int32_t launch_index, const wt_image *inputs,
                          int32_t n_inputs, const wt_image *outputs, int32_t n_outputs,
                          int32_t *out, int32_t cap, int32_t *n_out);

/* Stream lanes of the run plan for these images (the concurrent launches
 * of WT_FLAG_ONE_STREAM's description): out = [launches, lanes, then per
 * launch: its lane, the count and indices of the earlier launches on other
 * lanes it waits for, the count and indices of the stages it computes].
 * *n_out gets the full length; at most cap values are written.             */
wt_status wt_debug_lanes(wt_pipeline *p, const wt_image *inputs, int32_t n_inputs, const wt_image *outputs,
                         int32_t n_outputs, int32_t *out, int32_t cap, int32_t *n_out);

/* Row bands of wt_run_host for these images (planning only, no device
 * work): 4 values per band, (y0, y1, ys, ye): the band keeps output rows
 * [y0, y1) and runs the pipeline on input rows [ys, ye), ys even.
 * *n_bands = 0 when the call runs the whole image at once.  At most cap
 * bands are written; *n_bands gets the full count.                         */
wt_status wt_debug_host_bands(wt_pipeline *p, const wt_image *inputs, int32_t n_inputs, const wt_image *outputs,
                              int32_t n_outputs, int32_t *bands, int32_t cap, int32_t *n_bands);

/* The analytic model's cost of stages [first, first + n) as one group, as
 * wt_schedule_auto's DP-Fusion (Alg. 2) weighs it for a width x height
 * image of `dtype`: the best over the group's tile shapes and fracReg, or
 * the per-stage kernel for one stage.  *fused = 1 when a group kernel is
 * the choice.  WT_EINVAL for a range outside the pipeline or longer than
 * the longest group DP-Fusion forms (16 stages); *cost = +inf when no
 * kernel can run the range as one group.                                   */
wt_status wt_debug_segment_cost(wt_pipeline *p, int32_t first, int32_t n, int32_t width, int32_t height,
                                int32_t dtype, double *cost, int32_t *fused);

/* Halo/window analysis of schedule group `group` (Sec. 4 overlap, Sec. 5
 * parallelogram skew): out = [fusable, halo_l, halo_r, halo_t, halo_b,
 * unroll, n_nodes, then per node: id, src_chan, is_source, is_liveout, top,
 * bot, delay, window, xl*1000+xr, in_smem].  *n_out gets the length.        */
wt_status wt_debug_group_geometry(wt_pipeline *p, int32_t group, int32_t vec, float frac_reg,
                                  int32_t *out, int32_t cap, int32_t *n_out);

/* Failure injection for tests of the error paths (no GPU fault involved).
 * kind 0: host allocation points (pipeline creation, run planning), which
 * then fail as an out-of-memory condition; kind 1: the library's device
 * allocations (workspace, control block, host-run staging, batch tables,
 * cost-model and preprocessing buffers).  The allocation of that kind
 * after `after` successful ones fails once, with WT_ENOMEM at the entry
 * point; after < 0 disarms.  Process-wide, not thread-safe with respect to
 * concurrent library calls.                                                */
wt_status wt_debug_inject_alloc_failure(int32_t kind, int32_t after);

/* Live pipelines (created, not destroyed) and device bytes the library
 * holds in workspaces, staging buffers, batch tables and temporary
 * buffers; either pointer may be null.  For leak tests.                     */
wt_status wt_debug_live_objects(int64_t *pipelines, int64_t *device_bytes);

#ifdef __cplusplus
}
#endif
#endif
