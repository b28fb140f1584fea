/*
 * oracle.c -- plain FP64 CPU oracle (TEST INFRASTRUCTURE ONLY; see oracle.h).
 *
 * Every function follows the problem statement of Jangda & Guha (PACT'20):
 * stages are per-pixel functions of producer values at constant offsets
 * (Sec. 2.2, Fig. 2; Sec. 2.3 dependence vectors), evaluated here unfused,
 * stage by stage, over full arrays, with the clamp-to-edge boundary rule
 * applied at every producer read.  No blocking, fusion or reordering.
 */
#include "oracle.h"

#include <limits.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_STACK 64

int or_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Threads of the parallel loops from now on (n >= 1; timing only). */
void or_set_num_threads(int n) {
#ifdef _OPENMP
  if (n >= 1) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* Source coordinate of a tap along one axis (Sec. 2.3; Sec. 5 scaling). */
static int tap_coord(int mode, int p, int d) {
  /* modes 2s-1: down by 2^s (P(2^s p + d)); 2s: up by 2^s (P(floor(p / 2^s) + d)) */
  if (mode > 0) {
    const int s = (mode + 1) / 2;
    if (mode & 1) return (p << s) + d;
    return (p >> s) + d; /* p >= 0: floor(p / 2^s) */
  }
  return p + d;
}

static int half_up(int n) { return (n + 1) / 2; }

/* ---------------------------------------------------------------- shapes */

int or_dag_shapes(const or_stage *st, int n_st, const or_input *in, int n_in,
                  int32_t *level, int32_t *W, int32_t *H, int32_t *C) {
  if (n_in < 1) return -5;
  for (int j = 0; j < n_in; j++) {
    if (in[j].width < 1 || in[j].height < 1 || in[j].channels < 1) return -5;
    if (in[j].width != in[0].width || in[j].height != in[0].height) return -5;
  }
  for (int s = 0; s < n_st; s++) {
    const or_stage *S = &st[s];
    if (S->channels < 1 || S->n_ops < 1) return -4;
    int lv = INT_MIN, depth = 0;
    for (int i = 0; i < S->n_ops; i++) {
      const or_op *o = &S->ops[i];
      switch (o->op) {
        case OR_CONST: case OR_XPAR: case OR_YPAR: case OR_CHAN: depth++; break;
        case OR_TAP: case OR_TAPZ: {
          if (o->slot < 0 || o->slot >= S->n_in) return -4;
          int p = S->in[o->slot];
          if (p >= s || p < -n_in) return -1;
          int pl = p >= 0 ? level[p] : 0;
          int pc = p >= 0 ? C[p] : in[-p - 1].channels;
          if (o->op == OR_TAPZ) {
            /* a plane offset reads planes of the same depth (or the one
               plane of a one-plane producer), at the consumer's level */
            if (o->mode != OR_SAME || (pc != 1 && pc != S->channels)) return -4;
          } else {
            if (o->chan >= 0 && o->chan >= pc) return -4;
            if (o->chan < 0 && pc != 1 && pc != S->channels) return -4;
          }
          int implied;
          if (o->mode == OR_SAME) implied = pl;
          else if (o->mode >= OR_DOWN2 && o->mode <= OR_UP8)
            implied = (o->mode & 1) ? pl + (o->mode + 1) / 2 : pl - (o->mode + 1) / 2;
          else return -4;
          if (lv == INT_MIN) lv = implied;
          else if (lv != implied) return -2;
          depth++;
        } break;
        case OR_ADD: case OR_SUB: case OR_MUL: case OR_DIV: case OR_MIN: case OR_MAX:
          if (depth < 2) return -4;
          depth--;
          break;
        case OR_NEG: case OR_ABS: case OR_SQRT:
          if (depth < 1) return -4;
          break;
        default: return -4;
      }
      if (depth > OR_STACK) return -4;
    }
    if (depth != 1) return -4;
    if (lv == INT_MIN) lv = 0;
    if (lv < 0) return -3;
    level[s] = lv;
    int w = in[0].width, h = in[0].height;
    for (int l = 0; l < lv; l++) { w = half_up(w); h = half_up(h); }
    W[s] = w; H[s] = h; C[s] = S->channels;
  }
  return 0;
}

/* ------------------------------------------------------- point evaluation */

/* A producer as seen by a consumer: a box [x0, x0+bw) x [y0, y0+bh) of a
 * domain W x H, all C channels, stored planar inside the box.            */
typedef struct {
  const double *data;
  int x0, y0, bw, bh, W, H, C;
} src_box;

static double eval_point(const or_stage *S, const src_box *src, int x, int y, int c) {
  double stk[OR_STACK];
  int sp = 0;
  for (int i = 0; i < S->n_ops; i++) {
    const or_op *o = &S->ops[i];
    switch (o->op) {
      case OR_CONST: stk[sp++] = o->value; break;
      case OR_XPAR: stk[sp++] = (double)(x & 1); break;
      case OR_YPAR: stk[sp++] = (double)(y & 1); break;
      case OR_CHAN: stk[sp++] = (double)c; break;
      case OR_TAP: {
        const src_box *p = &src[o->slot];
        int px = clampi(tap_coord(o->mode, x, o->dx), 0, p->W - 1);
        int py = clampi(tap_coord(o->mode, y, o->dy), 0, p->H - 1);
        int pc = o->chan >= 0 ? o->chan : (p->C == 1 ? 0 : c);
        stk[sp++] = p->data[((size_t)pc * p->bh + (py - p->y0)) * p->bw + (px - p->x0)];
      } break;
      case OR_TAPZ: {
        const src_box *p = &src[o->slot];
        int px = clampi(x + o->dx, 0, p->W - 1);
        int py = clampi(y + o->dy, 0, p->H - 1);
        int pc = clampi(c + o->chan, 0, p->C - 1);
        stk[sp++] = p->data[((size_t)pc * p->bh + (py - p->y0)) * p->bw + (px - p->x0)];
      } break;
      case OR_ADD: sp--; stk[sp - 1] = stk[sp - 1] + stk[sp]; break;
      case OR_SUB: sp--; stk[sp - 1] = stk[sp - 1] - stk[sp]; break;
      case OR_MUL: sp--; stk[sp - 1] = stk[sp - 1] * stk[sp]; break;
      case OR_DIV: sp--; stk[sp - 1] = stk[sp - 1] / stk[sp]; break;
      case OR_MIN: sp--; stk[sp - 1] = fmin(stk[sp - 1], stk[sp]); break;
      case OR_MAX: sp--; stk[sp - 1] = fmax(stk[sp - 1], stk[sp]); break;
      case OR_NEG: stk[sp - 1] = -stk[sp - 1]; break;
      case OR_ABS: stk[sp - 1] = fabs(stk[sp - 1]); break;
      case OR_SQRT: stk[sp - 1] = sqrt(stk[sp - 1]); break;
      default: return NAN;
    }
  }
  return stk[0];
}

/* ------------------------------------------------------- box evaluation */

typedef struct { int x0, x1, y0, y1, used; } box;

static void box_union(box *b, int x0, int x1, int y0, int y1) {
  if (!b->used) { b->x0 = x0; b->x1 = x1; b->y0 = y0; b->y1 = y1; b->used = 1; return; }
  if (x0 < b->x0) b->x0 = x0;
  if (x1 > b->x1) b->x1 = x1;
  if (y0 < b->y0) b->y0 = y0;
  if (y1 > b->y1) b->y1 = y1;
}

/* Evaluates every stage s <= last over need[s] (inclusive boxes), freeing a
 * stage's box once no later needed stage reads it.  On success vals[s]
 * holds the box of stage s for every s with keep[s] != 0.                */
static int eval_boxes(const or_stage *st, int n_st, const or_input *in,
                      const int32_t *W, const int32_t *H, const int32_t *C,
                      const box *need, const int *keep, double **vals) {
  int last = n_st - 1;
  int *last_use = (int *)malloc(sizeof(int) * (size_t)(n_st > 0 ? n_st : 1));
  if (!last_use) return -6;
  for (int s = 0; s < n_st; s++) last_use[s] = -1;
  for (int s = 0; s <= last; s++) {
    if (!need[s].used) continue;
    for (int k = 0; k < st[s].n_in; k++)
      if (st[s].in[k] >= 0) last_use[st[s].in[k]] = s;
  }
  int rc = 0;
  for (int s = 0; s <= last && rc == 0; s++) {
    vals[s] = NULL;
    if (!need[s].used) continue;
    const or_stage *S = &st[s];
    src_box *src = (src_box *)malloc(sizeof(src_box) * (size_t)(S->n_in > 0 ? S->n_in : 1));
    if (!src) { rc = -6; break; }
    for (int k = 0; k < S->n_in; k++) {
      int p = S->in[k];
      if (p < 0) {
        const or_input *I = &in[-p - 1];
        src[k].data = I->data; src[k].x0 = 0; src[k].y0 = 0;
        src[k].bw = I->width; src[k].bh = I->height;
        src[k].W = I->width; src[k].H = I->height; src[k].C = I->channels;
      } else {
        src[k].data = vals[p];
        src[k].x0 = need[p].x0; src[k].y0 = need[p].y0;
        src[k].bw = need[p].x1 - need[p].x0 + 1; src[k].bh = need[p].y1 - need[p].y0 + 1;
        src[k].W = W[p]; src[k].H = H[p]; src[k].C = C[p];
        if (!src[k].data) rc = -7;
      }
    }
    if (rc != 0) { free(src); break; }
    int bw = need[s].x1 - need[s].x0 + 1, bh = need[s].y1 - need[s].y0 + 1, cs = C[s];
    double *out = (double *)malloc(sizeof(double) * (size_t)bw * (size_t)bh * (size_t)cs);
    if (!out) { free(src); rc = -6; break; }
    long rows = (long)cs * bh;
#pragma omp parallel for schedule(static)
    for (long r = 0; r < rows; r++) {
      int c = (int)(r / bh), yy = (int)(r % bh);
      for (int xx = 0; xx < bw; xx++)
        out[(size_t)r * bw + xx] = eval_point(S, src, need[s].x0 + xx, need[s].y0 + yy, c);
    }
    free(src);
    vals[s] = out;
    for (int k = 0; k < S->n_in; k++) {
      int p = S->in[k];
      if (p >= 0 && last_use[p] == s && !keep[p]) { free(vals[p]); vals[p] = NULL; }
    }
  }
  free(last_use);
  return rc;
}

/* Inclusive range of producer coordinates that consumer range [a, b] taps. */
static void tap_range(int mode, int a, int b, int d, int n, int *lo, int *hi) {
  *lo = clampi(tap_coord(mode, a, d), 0, n - 1);
  *hi = clampi(tap_coord(mode, b, d), 0, n - 1);
}

static void propagate_need(const or_stage *st, int last, const int32_t *W,
                           const int32_t *H, box *need) {
  for (int s = last; s >= 0; s--) {
    if (!need[s].used) continue;
    const or_stage *S = &st[s];
    for (int i = 0; i < S->n_ops; i++) {
      const or_op *o = &S->ops[i];
      if (o->op != OR_TAP && o->op != OR_TAPZ) continue;
      int p = S->in[o->slot];
      if (p < 0) continue;
      int x0, x1, y0, y1;
      tap_range(o->mode, need[s].x0, need[s].x1, o->dx, W[p], &x0, &x1);
      tap_range(o->mode, need[s].y0, need[s].y1, o->dy, H[p], &y0, &y1);
      box_union(&need[p], x0, x1, y0, y1);
    }
  }
}

typedef struct {
  int32_t *level, *W, *H, *C;
  box *need;
  int *keep;
  double **vals;
} work;

static int work_alloc(work *w, int n) {
  size_t m = (size_t)(n > 0 ? n : 1);
  w->level = (int32_t *)calloc(m, sizeof(int32_t));
  w->W = (int32_t *)calloc(m, sizeof(int32_t));
  w->H = (int32_t *)calloc(m, sizeof(int32_t));
  w->C = (int32_t *)calloc(m, sizeof(int32_t));
  w->need = (box *)calloc(m, sizeof(box));
  w->keep = (int *)calloc(m, sizeof(int));
  w->vals = (double **)calloc(m, sizeof(double *));
  return (w->level && w->W && w->H && w->C && w->need && w->keep && w->vals) ? 0 : -6;
}

static void work_free(work *w, int n) {
  if (w->vals)
    for (int s = 0; s < n; s++) free(w->vals[s]);
  free(w->level); free(w->W); free(w->H); free(w->C);
  free(w->need); free(w->keep); free(w->vals);
}

int or_dag_eval(const or_stage *st, int n_st, const or_input *in, int n_in,
                const int32_t *out_ids, int n_out, double *const *out) {
  work w;
  int rc = work_alloc(&w, n_st);
  if (rc == 0) rc = or_dag_shapes(st, n_st, in, n_in, w.level, w.W, w.H, w.C);
  if (rc == 0) {
    for (int k = 0; k < n_out; k++)
      if (out_ids[k] < 0 || out_ids[k] >= n_st) rc = -1;
  }
  if (rc == 0) {
    for (int s = 0; s < n_st; s++) {
      w.need[s].x0 = 0; w.need[s].x1 = w.W[s] - 1;
      w.need[s].y0 = 0; w.need[s].y1 = w.H[s] - 1;
      w.need[s].used = 1;
    }
    for (int k = 0; k < n_out; k++) w.keep[out_ids[k]] = 1;
    rc = eval_boxes(st, n_st, in, w.W, w.H, w.C, w.need, w.keep, w.vals);
  }
  if (rc == 0) {
    for (int k = 0; k < n_out; k++) {
      int s = out_ids[k];
      memcpy(out[k], w.vals[s], sizeof(double) * (size_t)w.W[s] * (size_t)w.H[s] * (size_t)w.C[s]);
    }
  }
  work_free(&w, n_st);
  return rc;
}

int or_dag_eval_points(const or_stage *st, int n_st, const or_input *in,
                       int n_in, int sid, int n, const int32_t *x,
                       const int32_t *y, const int32_t *c, double *val) {
  if (sid < 0 || sid >= n_st) return -1;
  if (n <= 0) return 0;
  work w;
  int rc = work_alloc(&w, n_st);
  if (rc == 0) rc = or_dag_shapes(st, n_st, in, n_in, w.level, w.W, w.H, w.C);
  if (rc == 0) {
    for (int i = 0; i < n; i++) {
      if (x[i] < 0 || x[i] >= w.W[sid] || y[i] < 0 || y[i] >= w.H[sid] ||
          c[i] < 0 || c[i] >= w.C[sid]) { rc = -8; break; }
      box_union(&w.need[sid], x[i], x[i], y[i], y[i]);
    }
  }
  if (rc == 0) {
    propagate_need(st, sid, w.W, w.H, w.need);
    w.keep[sid] = 1;
    rc = eval_boxes(st, sid + 1, in, w.W, w.H, w.C, w.need, w.keep, w.vals);
  }
  if (rc == 0) {
    const box *b = &w.need[sid];
    int bw = b->x1 - b->x0 + 1, bh = b->y1 - b->y0 + 1;
    for (int i = 0; i < n; i++)
      val[i] = w.vals[sid][((size_t)c[i] * bh + (y[i] - b->y0)) * bw + (x[i] - b->x0)];
  }
  work_free(&w, n_st);
  return rc;
}

/* ------------------------------------------------- recursive brute force */

static double brute_rec(const or_stage *st, const int32_t *W, const int32_t *H,
                        const int32_t *C, const or_input *in, int s, int x, int y, int c) {
  const or_stage *S = &st[s];
  double stk[OR_STACK];
  int sp = 0;
  for (int i = 0; i < S->n_ops; i++) {
    const or_op *o = &S->ops[i];
    switch (o->op) {
      case OR_CONST: stk[sp++] = o->value; break;
      case OR_XPAR: stk[sp++] = (double)(x & 1); break;
      case OR_YPAR: stk[sp++] = (double)(y & 1); break;
      case OR_CHAN: stk[sp++] = (double)c; break;
      case OR_TAP: {
        int p = S->in[o->slot];
        int pw, ph, pcn;
        if (p < 0) { pw = in[-p - 1].width; ph = in[-p - 1].height; pcn = in[-p - 1].channels; }
        else { pw = W[p]; ph = H[p]; pcn = C[p]; }
        int px = clampi(tap_coord(o->mode, x, o->dx), 0, pw - 1);
        int py = clampi(tap_coord(o->mode, y, o->dy), 0, ph - 1);
        int pc = o->chan >= 0 ? o->chan : (pcn == 1 ? 0 : c);
        if (p < 0) stk[sp++] = in[-p - 1].data[((size_t)pc * ph + py) * pw + px];
        else stk[sp++] = brute_rec(st, W, H, C, in, p, px, py, pc);
      } break;
      case OR_TAPZ: {
        int p = S->in[o->slot];
        int pw, ph, pcn;
        if (p < 0) { pw = in[-p - 1].width; ph = in[-p - 1].height; pcn = in[-p - 1].channels; }
        else { pw = W[p]; ph = H[p]; pcn = C[p]; }
        int px = clampi(x + o->dx, 0, pw - 1);
        int py = clampi(y + o->dy, 0, ph - 1);
        int pc = clampi(c + o->chan, 0, pcn - 1);
        if (p < 0) stk[sp++] = in[-p - 1].data[((size_t)pc * ph + py) * pw + px];
        else stk[sp++] = brute_rec(st, W, H, C, in, p, px, py, pc);
      } break;
      case OR_ADD: sp--; stk[sp - 1] += stk[sp]; break;
      case OR_SUB: sp--; stk[sp - 1] -= stk[sp]; break;
      case OR_MUL: sp--; stk[sp - 1] *= stk[sp]; break;
      case OR_DIV: sp--; stk[sp - 1] /= stk[sp]; break;
      case OR_MIN: sp--; stk[sp - 1] = stk[sp - 1] < stk[sp] ? stk[sp - 1] : stk[sp]; break;
      case OR_MAX: sp--; stk[sp - 1] = stk[sp - 1] > stk[sp] ? stk[sp - 1] : stk[sp]; break;
      case OR_NEG: stk[sp - 1] = -stk[sp - 1]; break;
      case OR_ABS: stk[sp - 1] = stk[sp - 1] < 0 ? -stk[sp - 1] : stk[sp - 1]; break;
      case OR_SQRT: stk[sp - 1] = sqrt(stk[sp - 1]); break;
      default: return NAN;
    }
  }
  return stk[0];
}

double or_brute(const or_stage *st, int n_st, const or_input *in, int n_in,
                int sid, int x, int y, int c) {
  work w;
  double v = NAN;
  if (work_alloc(&w, n_st) == 0 &&
      or_dag_shapes(st, n_st, in, n_in, w.level, w.W, w.H, w.C) == 0 &&
      sid >= 0 && sid < n_st)
    v = brute_rec(st, w.W, w.H, w.C, in, sid, x, y, c);
  work_free(&w, n_st);
  return v;
}

/* --------------------------------------------- direct benchmark pipelines */

#define AT(p, W, x, y) ((p)[(size_t)(y) * (W) + (x)])

void or_sharpen(const double *in, int W, int H, double *out) {
  static const double w[5] = {1.0 / 16, 4.0 / 16, 6.0 / 16, 4.0 / 16, 1.0 / 16};
  double *bx = (double *)malloc(sizeof(double) * (size_t)W * H);
  double *by = (double *)malloc(sizeof(double) * (size_t)W * H);
  if (!bx || !by) { free(bx); free(by); return; }
#pragma omp parallel for schedule(static)
  for (int y = 0; y < H; y++)
    for (int x = 0; x < W; x++) {
      double s = 0;
      for (int i = -2; i <= 2; i++) s += w[i + 2] * AT(in, W, clampi(x + i, 0, W - 1), y);
      AT(bx, W, x, y) = s;
    }
#pragma omp parallel for schedule(static)
  for (int y = 0; y < H; y++)
    for (int x = 0; x < W; x++) {
      double s = 0;
      for (int j = -2; j <= 2; j++) s += w[j + 2] * AT(bx, W, x, clampi(y + j, 0, H - 1));
      AT(by, W, x, y) = s;
    }
#pragma omp parallel for schedule(static)
  for (int y = 0; y < H; y++)
    for (int x = 0; x < W; x++) {
      double v = AT(in, W, x, y);
      double o = v + 1.5 * (v - AT(by, W, x, y));
      AT(out, W, x, y) = o < 0 ? 0 : (o > 1 ? 1 : o);
    }
  free(bx); free(by);
}

/* 3x3 correlation with clamp-to-edge: out(x,y) = s * sum K[j][i] P(x+i-1, y+j-1). */
static void corr3(const double *P, int W, int H, const double K[3][3], double s, double *out) {
#pragma omp parallel for schedule(static)
  for (int y = 0; y < H; y++)
    for (int x = 0; x < W; x++) {
      double acc = 0;
      for (int j = 0; j < 3; j++)
        for (int i = 0; i < 3; i++)
          acc += K[j][i] * AT(P, W, clampi(x + i - 1, 0, W - 1), clampi(y + j - 1, 0, H - 1));
      AT(out, W, x, y) = s * acc;
    }
}

void or_harris(const double *in, int W, int H, int normalized, double k, double *out) {
  static const double KX[3][3] = {{-1, 0, 1}, {-2, 0, 2}, {-1, 0, 1}};
  static const double KY[3][3] = {{-1, -2, -1}, {0, 0, 0}, {1, 2, 1}};
  static const double KB[3][3] = {{1, 1, 1}, {1, 1, 1}, {1, 1, 1}};
  double sx = normalized ? 1.0 / 8 : 1.0, sb = normalized ? 1.0 / 9 : 1.0;
  size_t n = (size_t)W * H;
  double *buf = (double *)malloc(sizeof(double) * n * 8);
  if (!buf) return;
  double *Ix = buf, *Iy = buf + n, *Ixx = buf + 2 * n, *Iyy = buf + 3 * n, *Ixy = buf + 4 * n;
  double *Sxx = buf + 5 * n, *Syy = buf + 6 * n, *Sxy = buf + 7 * n;
  corr3(in, W, H, KX, sx, Ix);
  corr3(in, W, H, KY, sx, Iy);
#pragma omp parallel for schedule(static)
  for (long i = 0; i < (long)n; i++) {
    Ixx[i] = Ix[i] * Ix[i];
    Iyy[i] = Iy[i] * Iy[i];
    Ixy[i] = Ix[i] * Iy[i];
  }
  corr3(Ixx, W, H, KB, sb, Sxx);
  corr3(Iyy, W, H, KB, sb, Syy);
  corr3(Ixy, W, H, KB, sb, Sxy);
#pragma omp parallel for schedule(static)
  for (long i = 0; i < (long)n; i++) {
    double det = Sxx[i] * Syy[i] - Sxy[i] * Sxy[i];
    double tr = Sxx[i] + Syy[i];
    out[i] = det - k * tr * tr;
  }
  free(buf);
}

/* G_{k+1}(x,y) = sum_{i,j=-2..2} b_i b_j G_k(2x+i, 2y+j), clamped. */
static void down2(const double *P, int Wp, int Hp, double *out, int Wc, int Hc) {
  static const double b[5] = {1.0 / 16, 4.0 / 16, 6.0 / 16, 4.0 / 16, 1.0 / 16};
#pragma omp parallel for schedule(static)
  for (int y = 0; y < Hc; y++)
    for (int x = 0; x < Wc; x++) {
      double acc = 0;
      for (int j = -2; j <= 2; j++)
        for (int i = -2; i <= 2; i++)
          acc += b[i + 2] * b[j + 2] *
                 AT(P, Wp, clampi(2 * x + i, 0, Wp - 1), clampi(2 * y + j, 0, Hp - 1));
      AT(out, Wc, x, y) = acc;
    }
}

/* Half-pixel-centred bilinear upsample of a coarse P (Wp x Hp) onto a fine
 * Wc x Hc grid: along each axis, even 2i -> 0.75 P(i) + 0.25 P(i-1), odd
 * 2i+1 -> 0.75 P(i) + 0.25 P(i+1), clamped.                              */
static void up2(const double *P, int Wp, int Hp, double *out, int Wc, int Hc) {
#pragma omp parallel for schedule(static)
  for (int y = 0; y < Hc; y++)
    for (int x = 0; x < Wc; x++) {
      double wx[3], wy[3];
      int px = x >> 1, py = y >> 1;
      wx[0] = (x & 1) ? 0.0 : 0.25; wx[1] = 0.75; wx[2] = (x & 1) ? 0.25 : 0.0;
      wy[0] = (y & 1) ? 0.0 : 0.25; wy[1] = 0.75; wy[2] = (y & 1) ? 0.25 : 0.0;
      double acc = 0;
      for (int j = 0; j < 3; j++)
        for (int i = 0; i < 3; i++)
          acc += wx[i] * wy[j] *
                 AT(P, Wp, clampi(px + i - 1, 0, Wp - 1), clampi(py + j - 1, 0, Hp - 1));
      AT(out, Wc, x, y) = acc;
    }
}

void or_blend(const double *A, const double *B, const double *M, int W, int H,
              int C, int levels, double *out) {
  if (levels < 1 || levels > 16) return;
  int lw[16], lh[16];
  size_t off[17];
  lw[0] = W; lh[0] = H; off[0] = 0;
  for (int l = 1; l < levels; l++) { lw[l] = half_up(lw[l - 1]); lh[l] = half_up(lh[l - 1]); }
  for (int l = 0; l < levels; l++) off[l + 1] = off[l] + (size_t)lw[l] * lh[l];
  size_t tot = off[levels];
  double *GM = (double *)malloc(sizeof(double) * tot);
  double *GA = (double *)malloc(sizeof(double) * tot);
  double *GB = (double *)malloc(sizeof(double) * tot);
  double *R = (double *)malloc(sizeof(double) * tot);
  double *U = (double *)malloc(sizeof(double) * off[1]);
  if (!GM || !GA || !GB || !R || !U) goto done;
  memcpy(GM, M, sizeof(double) * off[1]);
  for (int l = 0; l + 1 < levels; l++)
    down2(GM + off[l], lw[l], lh[l], GM + off[l + 1], lw[l + 1], lh[l + 1]);
  for (int c = 0; c < C; c++) {
    memcpy(GA, A + (size_t)c * off[1], sizeof(double) * off[1]);
    memcpy(GB, B + (size_t)c * off[1], sizeof(double) * off[1]);
    for (int l = 0; l + 1 < levels; l++) {
      down2(GA + off[l], lw[l], lh[l], GA + off[l + 1], lw[l + 1], lh[l + 1]);
      down2(GB + off[l], lw[l], lh[l], GB + off[l + 1], lw[l + 1], lh[l + 1]);
    }
    /* Laplacian levels L_l = G_l - up(G_{l+1}) (L_top = G_top) and the blend
     * BL_l = M_l L^A_l + (1 - M_l) L^B_l, kept in GA.                    */
    for (int l = 0; l < levels; l++) {
      size_t n = (size_t)lw[l] * lh[l];
      double *ga = GA + off[l], *gb = GB + off[l], *gm = GM + off[l];
      if (l + 1 < levels) {
        up2(GA + off[l + 1], lw[l + 1], lh[l + 1], U, lw[l], lh[l]);
        for (size_t i = 0; i < n; i++) R[off[l] + i] = ga[i] - U[i]; /* L^A_l */
        up2(GB + off[l + 1], lw[l + 1], lh[l + 1], U, lw[l], lh[l]);
        for (size_t i = 0; i < n; i++) {
          double la = R[off[l] + i], lb = gb[i] - U[i];
          R[off[l] + i] = gm[i] * la + (1.0 - gm[i]) * lb;
        }
      } else {
        for (size_t i = 0; i < n; i++) R[off[l] + i] = gm[i] * ga[i] + (1.0 - gm[i]) * gb[i];
      }
    }
    /* Reconstruction: R_top = BL_top; R_l = BL_l + up(R_{l+1}). */
    for (int l = levels - 2; l >= 0; l--) {
      size_t n = (size_t)lw[l] * lh[l];
      up2(R + off[l + 1], lw[l + 1], lh[l + 1], U, lw[l], lh[l]);
      for (size_t i = 0; i < n; i++) R[off[l] + i] += U[i];
    }
    memcpy(out + (size_t)c * off[1], R, sizeof(double) * off[1]);
  }
done:
  free(GM); free(GA); free(GB); free(R); free(U);
}
