/*
 * oracle.h -- plain, slow FP64 CPU oracle for image-pipeline DAGs.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / --impl reference legs of bench.py may load this library.
 * It shares no code, header, table or constant with the CUDA path.
 *
 * What it computes (Jangda & Guha, "Model-Based Warp Overlapped Tiling for
 * Image Processing Programs on GPUs", PACT'20):
 *   An image-processing program is a DAG of stages, each a per-pixel function
 *   of producer values at constant offsets (Sec. 1, Sec. 2.2 Fig. 2, Sec. 2.3
 *   dependence vectors).  Fusion and overlapped tiling are schedule
 *   transformations (Sec. 2.2 "liveouts"/"scratchpads", Sec. 4), so the value
 *   the method must reach is the UNFUSED definition: evaluate every stage in
 *   topological order into a full array over its domain.
 *
 * Readings taken where the paper is silent:
 *   - Boundary: every producer read is clamped to the producer's domain
 *     (clamp-to-edge at every stage, not only at the input).
 *   - Sampling: a tap in DOWN2 mode reads P(2x+dx, 2y+dy); in UP2 mode it
 *     reads P(floor(x/2)+dx, floor(y/2)+dy); DOWN4/UP4 and DOWN8/UP8 scale
 *     by 4 and 8 (two and three levels); XPAR/YPAR push x&1, y&1 of the
 *     consumer point (Sec. 5 "alignment and scaling" makes such dependences
 *     constant).  Domain of level l: W_l = ceil(W_{l-1}/2).
 *   - Channels are planar; a tap with chan < 0 reads the consumer's channel
 *     (channel 0 when the producer has one channel).
 *   - Volumes (App. A, 3-D groups): a D x H x W volume is an image of D
 *     planes; a TAPZ reads the producer at plane offset dz from the
 *     consumer's plane, clamped to [0, D-1] like x and y.
 *
 * Layout of every array: planar, data[(c*H + y)*W + x], FP64.
 */
#ifndef WT_ORACLE_H
#define WT_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum or_opcode {
  OR_CONST = 1, /* push value                                   */
  OR_TAP = 2,   /* push producer in[slot] at (dx,dy) per mode   */
  OR_ADD = 3, OR_SUB = 4, OR_MUL = 5, OR_DIV = 6,
  OR_MIN = 7, OR_MAX = 8,
  OR_NEG = 9, OR_ABS = 10, OR_SQRT = 11,
  OR_XPAR = 12, /* push (x & 1) of the consumer point           */
  OR_YPAR = 13, /* push (y & 1) of the consumer point           */
  OR_CHAN = 14, /* push the consumer point's channel index      */
  OR_TAPZ = 15  /* push producer in[slot] at (x+dx, y+dy) of plane
                   clamp(c + chan, 0, C_p - 1): a 3-D tap whose plane
                   offset dz is held in `chan` (mode must be same)    */
};
/* down by 2^s: mode 2s-1 (producer s levels finer); up by 2^s: mode 2s */
enum or_tapmode { OR_SAME = 0, OR_DOWN2 = 1, OR_UP2 = 2, OR_DOWN4 = 3, OR_UP4 = 4, OR_DOWN8 = 5, OR_UP8 = 6 };

typedef struct {
  int32_t op, slot, dx, dy, chan, mode;
  double value;
} or_op;

/* A stage: `in[k]` >= 0 names an earlier stage, -(j+1) names pipeline
 * input j.  `ops` is a postfix program evaluated per output point.      */
typedef struct {
  int32_t channels;
  int32_t n_in;
  const int32_t *in;
  int32_t n_ops;
  const or_op *ops;
} or_stage;

typedef struct {
  int32_t width, height, channels;
  const double *data;
} or_input;

/* Domain (level, width, height, channels) of every stage.  Returns 0, or a
 * negative code for a malformed DAG (-1 bad producer index / not
 * topological, -2 inconsistent level, -3 negative level, -4 bad program,
 * -5 inputs of different sizes).                                         */
int or_dag_shapes(const or_stage *st, int n_st, const or_input *in, int n_in,
                  int32_t *level, int32_t *W, int32_t *H, int32_t *C);

/* Full unfused evaluation.  out[k] receives stage out_ids[k] (caller-owned,
 * sized by or_dag_shapes).  Returns 0 or a negative code.               */
int or_dag_eval(const or_stage *st, int n_st, const or_input *in, int n_in,
                const int32_t *out_ids, int n_out, double *const *out);

/* Values of stage `sid` at n points (x[i], y[i], c[i]).  Each stage is
 * evaluated only over the bounding box its consumers need, with the same
 * per-point definition as or_dag_eval, so results are identical to it.   */
int or_dag_eval_points(const or_stage *st, int n_st, const or_input *in,
                       int n_in, int sid, int n, const int32_t *x,
                       const int32_t *y, const int32_t *c, double *val);

/* Memo-free recursive evaluation of one point straight from the expression
 * trees (a second, independent evaluator; exponential, tiny inputs only). */
double or_brute(const or_stage *st, int n_st, const or_input *in, int n_in,
                int sid, int x, int y, int c);

/* Direct transcriptions of the benchmark pipelines, without the DAG
 * machinery (clamp-to-edge at every producer read).                     */
/* 3-stage sharpen: bx = [1,4,6,4,1]/16 along x, by = same along y,
 * out = clamp(in + 1.5*(in - by), 0, 1).                                */
void or_sharpen(const double *in, int W, int H, double *out);
/* 11-stage corner response: Sobel Ix, Iy (correlation, x = column), Ixx,
 * Iyy, Ixy, 3x3 box of each, det, trace, R = det - k*trace^2.
 * normalized != 0 scales Sobel by 1/8 and box sums by 1/9.              */
void or_harris(const double *in, int W, int H, int normalized, double k,
               double *out);
/* Laplacian-pyramid blend with `levels` Gaussian levels (G_0..G_{L-1}):
 * 5x5 binomial downsample by 2, half-pixel bilinear upsample, per-level
 * mask blend, reconstruction.  A, B: C planes; M: one plane.            */
void or_blend(const double *A, const double *B, const double *M, int W, int H,
              int C, int levels, double *out);

int or_num_threads(void);
/* Threads of the parallel loops from now on (n >= 1; timing only). */
void or_set_num_threads(int n);

#ifdef __cplusplus
}
#endif
#endif
