/*
 * lr_oracle.c -- plain, slow CPU reference of the exact order-independent-transparency
 * rasteriser described in "LucidRaster: GPU Software Rasterizer for Exact
 * Order-Independent Transparency" (arXiv 2405.13364).
 *
 * TEST INFRASTRUCTURE ONLY. This file is the oracle that the CUDA path is checked
 * against. Only the test suite, the smoke check and the benchmark's CPU-baseline leg
 * may load it. It shares no code, header, table or helper with the CUDA library.
 *
 * What it computes (the plain definition of exact OIT, Sec. 1: identify every fragment
 * that contributes to a pixel, sort all of them, blend in order):
 *   for every pixel centre, gather every covering (quad, triangle) fragment, sort the
 *   fragments fully by interpolated depth with ties broken by quad index, and composite
 *   them back to front with the over operator in fp32.
 * The paper does not fix the fixed-point format, fill rule, per-sample depth or tie
 * order; the readings used here (each stated at the function that applies it) are:
 *   O.2 transform   c_r = ((M[r][0]x + M[r][1]y) + M[r][2]z) + M[r][3], fp32, each op
 *                   rounded to nearest, no fused multiply-add (build with
 *                   -ffp-contract=off).
 *   O.3 reject      whole quad culled if any vertex is non-finite, has w outside
 *                   [near, far], or lands outside the +-16384 px guard band; also if
 *                   both triangles are degenerate or the AABB holds no pixel centre.
 *   O.4 snap        sx = ((cx/w)+1)(W/2), sy = (1-(cy/w))(H/2); X = rint(256 sx) etc.
 *                   (8 fractional bits, round half to even); q = 1/w.
 *   O.5 triangles   T0 = (v0,v1,v2), T1 = (v0,v2,v3); int64 doubled area; negative
 *                   area -> swap v1,v2; zero area -> no coverage.
 *   O.6 coverage    centre (256px+128, 256py+128) (or another sample position of the
 *                   pixel, for multisampling); edge a->b value
 *                   E = (Xb-Xa)(Py-Ya) - (Yb-Ya)(Px-Xa); owned iff dy<0 || (dy==0 && dx>0);
 *                   covered iff every edge has E>0 or (E==0 and owned).
 *   O.8 depth key   inv = 1/(float)A; l1 = (float)E_20 * inv; l2 = (float)E_01 * inv;
 *                   key = q0 + ((l1*(q1-q0)) + (l2*(q2-q0))) (interpolated 1/w; larger
 *                   is nearer).
 *   O.9 order       back to front = ascending (key, quad, triangle).
 *   O.10 colour     flat per quad, or perspective-correct per-vertex
 *                   sum(l_k q_k c_k) / sum(l_k q_k).
 *   lit colour      (simple lighting: per-vertex normals, one directional light) the
 *                   perspective-correct base RGBA as above; the normal's direction
 *                   n = sum(l_k q_k n_k); RGB scaled by amb + (1 - amb) |n.L| / (|n| |L|)
 *                   (two-sided Lambert plus ambient, 0 for a zero normal); alpha unlit.
 *   O.11 composite  C = a c + (1-a) C, A = a + (1-a) A, from black transparent.
 *   O.12 8-bit      rint(clamp(v,0,1) * 255).
 *   O.13 backward   fp64 gradient of the composite w.r.t. flat per-quad RGBA.
 *   alpha threshold (opt-in, lossy; Sec. 2 "Sample blending", Sec. 3 "Alpha threshold"):
 *                   composite front to back (the paper's order), blending a fragment
 *                   only while the transmittance T = prod(1 - a) of the fragments in
 *                   front of it is above t_min (the paper stops at accumulated alpha
 *                   1 - 1/128, i.e. t_min = 1/128); T is the running fp32 product, one
 *                   rounding per operation, so the stop decision is taken in fp32.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#define OR_VISIBLE 0
#define OR_BAD_INDEX 1
#define OR_NONFINITE 2
#define OR_DEPTH 3
#define OR_GUARD 4
#define OR_DEGENERATE 5
#define OR_NO_PIXEL 6

#define OR_GUARD_PX 16384.0f

typedef struct {
  const float* positions;   /* [V][3] */
  int64_t num_vertices;
  const uint32_t* indices;  /* [Q][4] or NULL: quad q uses 4q..4q+3 */
  int64_t num_quads;
  const float* colors;      /* flat [Q][4] or per-vertex [V][4], straight RGBA */
  int32_t color_mode;       /* 0 flat, 1 per-vertex, 2 per-vertex lit: [V][8] = RGBA, normal
                               xyz, unused */
  const float* view_proj;   /* [16], row-major */
  float near_z, far_z;
  int32_t width, height;
  /* where in each pixel the sample lies, in 1/256 px from the pixel's top-left corner:
   * (128, 128) is the pixel centre of O.6; a multisampled image (MSAA) is the mean of
   * the images of several sample positions */
  int32_t sample_x, sample_y;
  /* lit colours: direction toward the light (world space, any length) and the ambient term */
  float light[4];
} or_scene;

typedef struct {
  int64_t quads_by_status[8];
  int64_t fragments;
  int64_t max_depth;        /* largest per-pixel fragment count */
  int64_t key_ties;         /* adjacent sorted fragments of different quads, equal key */
} or_stats;

/* ---- per-quad setup (O.2 - O.5) ----------------------------------------------- */

typedef struct {
  int32_t status;
  int32_t X[4], Y[4];
  float q[4];
  int64_t vid[4];
  int32_t px0, px1, py0, py1;   /* pixel-centre AABB clipped to the screen */
} or_quad;

static float transform_row(const float* M, int r, float x, float y, float z) {
  /* O.2: ((M[r][0]*x + M[r][1]*y) + M[r][2]*z) + M[r][3] */
  float a = M[r * 4 + 0] * x;
  float b = M[r * 4 + 1] * y;
  float s = a + b;
  float c = M[r * 4 + 2] * z;
  s = s + c;
  s = s + M[r * 4 + 3];
  return s;
}

static int32_t floor_div256(int64_t a) {
  int64_t d = a / 256;
  if ((a % 256 != 0) && (a < 0)) d -= 1;
  return (int32_t)d;
}

static int32_t ceil_div256(int64_t a) { return -floor_div256(-a); }

static int64_t area2(int32_t xa, int32_t ya, int32_t xb, int32_t yb, int32_t xc, int32_t yc) {
  return (int64_t)(xb - xa) * (int64_t)(yc - ya) - (int64_t)(yb - ya) * (int64_t)(xc - xa);
}

static void setup_quad(const or_scene* s, int64_t j, or_quad* out) {
  memset(out, 0, sizeof(*out));
  int worst = OR_VISIBLE;
  for (int k = 0; k < 4; ++k) {
    int64_t v = s->indices ? (int64_t)s->indices[j * 4 + k] : j * 4 + k;
    out->vid[k] = v;
    if (v < 0 || v >= s->num_vertices) { worst = OR_BAD_INDEX; continue; }
    float x = s->positions[v * 3 + 0], y = s->positions[v * 3 + 1], z = s->positions[v * 3 + 2];
    float cx = transform_row(s->view_proj, 0, x, y, z);
    float cy = transform_row(s->view_proj, 1, x, y, z);
    float w = transform_row(s->view_proj, 3, x, y, z);
    int why = OR_VISIBLE;
    if (!isfinite(cx) || !isfinite(cy) || !isfinite(w)) {
      why = OR_NONFINITE;
    } else if (!(w >= s->near_z && w <= s->far_z)) {
      why = OR_DEPTH;
    } else {
      float halfw = 0.5f * (float)s->width, halfh = 0.5f * (float)s->height;
      float ndx = cx / w, ndy = cy / w;
      float sx = (ndx + 1.0f) * halfw;
      float sy = (1.0f - ndy) * halfh;
      if (!(fabsf(sx) <= OR_GUARD_PX && fabsf(sy) <= OR_GUARD_PX)) {
        why = OR_GUARD;
      } else {
        out->X[k] = (int32_t)rintf(sx * 256.0f);
        out->Y[k] = (int32_t)rintf(sy * 256.0f);
        out->q[k] = 1.0f / w;
      }
    }
    /* precedence: bad index > non-finite > depth > guard band */
    if (why != OR_VISIBLE && (worst == OR_VISIBLE || why < worst)) worst = why;
  }
  if (worst != OR_VISIBLE) { out->status = worst; return; }
  int64_t a0 = area2(out->X[0], out->Y[0], out->X[1], out->Y[1], out->X[2], out->Y[2]);
  int64_t a1 = area2(out->X[0], out->Y[0], out->X[2], out->Y[2], out->X[3], out->Y[3]);
  if (a0 == 0 && a1 == 0) { out->status = OR_DEGENERATE; return; }
  int32_t xmin = out->X[0], xmax = out->X[0], ymin = out->Y[0], ymax = out->Y[0];
  for (int k = 1; k < 4; ++k) {
    if (out->X[k] < xmin) xmin = out->X[k];
    if (out->X[k] > xmax) xmax = out->X[k];
    if (out->Y[k] < ymin) ymin = out->Y[k];
    if (out->Y[k] > ymax) ymax = out->Y[k];
  }
  /* pixels whose sample position lies in the quad's box */
  int32_t px0 = ceil_div256((int64_t)xmin - s->sample_x), px1 = floor_div256((int64_t)xmax - s->sample_x);
  int32_t py0 = ceil_div256((int64_t)ymin - s->sample_y), py1 = floor_div256((int64_t)ymax - s->sample_y);
  if (px0 < 0) px0 = 0;
  if (py0 < 0) py0 = 0;
  if (px1 > s->width - 1) px1 = s->width - 1;
  if (py1 > s->height - 1) py1 = s->height - 1;
  if (px0 > px1 || py0 > py1) { out->status = OR_NO_PIXEL; return; }
  out->px0 = px0; out->px1 = px1; out->py0 = py0; out->py1 = py1;
  out->status = OR_VISIBLE;
}

/* ---- fragments (O.5 - O.10) ------------------------------------------------------- */

typedef struct {
  float key;
  uint32_t j;
  uint32_t t;
  int32_t pix;     /* pixel index within the current band / request */
  float rgba[4];
} or_frag;

typedef struct {
  int ok;              /* triangle has non-zero area */
  int32_t X[3], Y[3];
  float q[3];
  int64_t vid[3];
  int64_t A;
  float inv;
  int owned[3];        /* edges v1->v2, v2->v0, v0->v1 */
  int32_t px0, px1, py0, py1;
} or_tri;

static int edge_owned(int32_t xa, int32_t ya, int32_t xb, int32_t yb) {
  int64_t dx = (int64_t)xb - xa, dy = (int64_t)yb - ya;
  return dy < 0 || (dy == 0 && dx > 0);
}

static void make_tri(const or_quad* qd, int t, const or_scene* s, or_tri* tri) {
  static const int corner[2][3] = {{0, 1, 2}, {0, 2, 3}};
  int c0 = corner[t][0], c1 = corner[t][1], c2 = corner[t][2];
  int64_t A = area2(qd->X[c0], qd->Y[c0], qd->X[c1], qd->Y[c1], qd->X[c2], qd->Y[c2]);
  tri->ok = (A != 0);
  if (!tri->ok) return;
  if (A < 0) { int tmp = c1; c1 = c2; c2 = tmp; A = -A; }
  int c[3] = {c0, c1, c2};
  for (int k = 0; k < 3; ++k) {
    tri->X[k] = qd->X[c[k]];
    tri->Y[k] = qd->Y[c[k]];
    tri->q[k] = qd->q[c[k]];
    tri->vid[k] = qd->vid[c[k]];
  }
  tri->A = A;
  tri->inv = 1.0f / (float)A;
  tri->owned[0] = edge_owned(tri->X[1], tri->Y[1], tri->X[2], tri->Y[2]);
  tri->owned[1] = edge_owned(tri->X[2], tri->Y[2], tri->X[0], tri->Y[0]);
  tri->owned[2] = edge_owned(tri->X[0], tri->Y[0], tri->X[1], tri->Y[1]);
  int32_t xmin = tri->X[0], xmax = tri->X[0], ymin = tri->Y[0], ymax = tri->Y[0];
  for (int k = 1; k < 3; ++k) {
    if (tri->X[k] < xmin) xmin = tri->X[k];
    if (tri->X[k] > xmax) xmax = tri->X[k];
    if (tri->Y[k] < ymin) ymin = tri->Y[k];
    if (tri->Y[k] > ymax) ymax = tri->Y[k];
  }
  tri->px0 = ceil_div256((int64_t)xmin - s->sample_x);
  tri->px1 = floor_div256((int64_t)xmax - s->sample_x);
  tri->py0 = ceil_div256((int64_t)ymin - s->sample_y);
  tri->py1 = floor_div256((int64_t)ymax - s->sample_y);
  if (tri->px0 < 0) tri->px0 = 0;
  if (tri->py0 < 0) tri->py0 = 0;
  if (tri->px1 > s->width - 1) tri->px1 = s->width - 1;
  if (tri->py1 > s->height - 1) tri->py1 = s->height - 1;
}

static int64_t edge_value(int32_t xa, int32_t ya, int32_t xb, int32_t yb, int64_t px, int64_t py) {
  return (int64_t)(xb - xa) * (py - ya) - (int64_t)(yb - ya) * (px - xa);
}

/* Returns 1 and fills key / rgba if pixel (px, py) is covered by the triangle. */
static int shade(const or_scene* s, const or_tri* tri, int64_t j, int32_t px, int32_t py,
                 float* key, float rgba[4]) {
  int64_t Px = 256 * (int64_t)px + s->sample_x, Py = 256 * (int64_t)py + s->sample_y;
  int64_t e0 = edge_value(tri->X[1], tri->Y[1], tri->X[2], tri->Y[2], Px, Py);
  int64_t e1 = edge_value(tri->X[2], tri->Y[2], tri->X[0], tri->Y[0], Px, Py);
  int64_t e2 = edge_value(tri->X[0], tri->Y[0], tri->X[1], tri->Y[1], Px, Py);
  if (!(e0 > 0 || (e0 == 0 && tri->owned[0]))) return 0;
  if (!(e1 > 0 || (e1 == 0 && tri->owned[1]))) return 0;
  if (!(e2 > 0 || (e2 == 0 && tri->owned[2]))) return 0;
  float l1 = (float)e1 * tri->inv;
  float l2 = (float)e2 * tri->inv;
  float d1 = tri->q[1] - tri->q[0];
  float d2 = tri->q[2] - tri->q[0];
  float t1 = l1 * d1;
  float t2 = l2 * d2;
  float sum = t1 + t2;
  *key = tri->q[0] + sum;
  if (s->color_mode == 0) {
    for (int c = 0; c < 4; ++c) rgba[c] = s->colors[j * 4 + c];
  } else {
    /* perspective-correct: weights l_k q_k, evaluated in double and rounded */
    double l[3] = {(double)e0 / (double)tri->A, (double)e1 / (double)tri->A,
                   (double)e2 / (double)tri->A};
    const int stride = s->color_mode == 2 ? 8 : 4;
    double wsum = 0.0, acc[4] = {0, 0, 0, 0}, n[3] = {0, 0, 0};
    for (int k = 0; k < 3; ++k) {
      double wk = l[k] * (double)tri->q[k];
      wsum += wk;
      const float* ck = s->colors + tri->vid[k] * stride;
      for (int c = 0; c < 4; ++c) acc[c] += wk * (double)ck[c];
      if (s->color_mode == 2)
        for (int c = 0; c < 3; ++c) n[c] += wk * (double)ck[4 + c];
    }
    double shade_f = 1.0;
    if (s->color_mode == 2) {
      double L[3] = {s->light[0], s->light[1], s->light[2]};
      double nn = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
      double ll = sqrt(L[0] * L[0] + L[1] * L[1] + L[2] * L[2]);
      double lam = (nn > 0.0 && ll > 0.0) ? fabs(n[0] * L[0] + n[1] * L[1] + n[2] * L[2]) / (nn * ll) : 0.0;
      double amb = s->light[3];
      shade_f = amb + (1.0 - amb) * lam;
    }
    for (int c = 0; c < 3; ++c) rgba[c] = (float)(acc[c] / wsum * shade_f);
    rgba[3] = (float)(acc[3] / wsum);
  }
  return 1;
}

static uint64_t splitmix64(uint64_t x) {
  /* splitmix64 output function (Steele, Lea, Flood 2014; constants as published by Vigna) */
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

static int frag_cmp(const void* pa, const void* pb) {
  const or_frag* a = (const or_frag*)pa;
  const or_frag* b = (const or_frag*)pb;
  if (a->pix != b->pix) return a->pix < b->pix ? -1 : 1;
  if (a->key != b->key) return a->key < b->key ? -1 : 1;
  if (a->j != b->j) return a->j < b->j ? -1 : 1;
  if (a->t != b->t) return a->t < b->t ? -1 : 1;
  return 0;
}

/* ---- shared state for the threaded passes ------------------------------------------ */

typedef struct {
  const or_scene* s;
  or_quad* quads;
  /* band buckets: quads whose AABB meets each band of rows */
  int band_rows;
  int nbands;
  int64_t* band_start;
  int64_t* band_list;
  /* outputs */
  float* rgba;
  uint32_t* count;
  uint64_t* hash;
  uint8_t* rgba8;
  double* rgba64;
  /* backward / fp64 forward */
  const double* colors64;     /* flat [Q][4] used by the fp64 forward, NULL = s->colors */
  const double* grad_out;     /* [H][W][4] */
  double* grad_colors;        /* per-thread [nthreads][Q][4] */
  int mode;                   /* 0 forward fp32, 1 fp64 forward, 2 backward,
                                 3 alpha-threshold forward */
  /* alpha threshold */
  float t_min;                /* blend while T > t_min */
  uint32_t* nblend;           /* [H][W] fragments blended before the stop */
  float* margin;              /* [H][W] min |T - t_min| / t_min over the stop tests made */
  /* work distribution */
  pthread_mutex_t lock;
  int next_band;
  int64_t frags, max_depth, ties;
  int failed;
} or_job;

typedef struct { or_job* job; int tid; } or_worker;

static void composite_pixel(or_job* job, const or_frag* f, int64_t n, int64_t pixel_index,
                            int tid, int64_t* ties) {
  const or_scene* s = job->s;
  if (job->mode == 0) {
    float C[3] = {0.f, 0.f, 0.f}, Aout = 0.f;
    double C64[3] = {0, 0, 0}, A64 = 0;
    uint64_t h = 0;
    for (int64_t i = 0; i < n; ++i) {
      float a = f[i].rgba[3];
      float om = 1.0f - a;
      for (int c = 0; c < 3; ++c) {
        float ac = a * f[i].rgba[c];
        float keep = om * C[c];
        C[c] = ac + keep;
        C64[c] = (double)a * (double)f[i].rgba[c] + (1.0 - (double)a) * C64[c];
      }
      float keepa = om * Aout;
      Aout = a + keepa;
      A64 = (double)a + (1.0 - (double)a) * A64;
      h += splitmix64(2ull * f[i].j + f[i].t);
      if (i > 0 && f[i].key == f[i - 1].key && f[i].j != f[i - 1].j) (*ties)++;
    }
    float out[4] = {C[0], C[1], C[2], Aout};
    for (int c = 0; c < 4; ++c) {
      if (job->rgba) job->rgba[pixel_index * 4 + c] = out[c];
      if (job->rgba8) {
        float v = out[c];
        if (!(v > 0.0f)) v = 0.0f;   /* also maps NaN to 0 */
        if (v > 1.0f) v = 1.0f;
        job->rgba8[pixel_index * 4 + c] = (uint8_t)rintf(v * 255.0f);
      }
    }
    if (job->rgba64) {
      for (int c = 0; c < 3; ++c) job->rgba64[pixel_index * 4 + c] = C64[c];
      job->rgba64[pixel_index * 4 + 3] = A64;
    }
    if (job->count) job->count[pixel_index] = (uint32_t)n;
    if (job->hash) job->hash[pixel_index] = h;
    return;
  }
  if (job->mode == 3) {
    /* alpha threshold: f[] is ascending (back first), so walk it from the end */
    float C[3] = {0.f, 0.f, 0.f}, T = 1.0f, margin = INFINITY;
    uint32_t nb = 0;
    for (int64_t i = n - 1; i >= 0; --i) {
      if (job->t_min > 0.0f) {
        float d = fabsf(T - job->t_min) / job->t_min;
        if (d < margin) margin = d;
      }
      if (!(T > job->t_min)) break;   /* accumulated alpha 1 - T reached 1 - t_min */
      float a = f[i].rgba[3];
      float w = T * a;
      for (int c = 0; c < 3; ++c) {
        float wc = w * f[i].rgba[c];
        C[c] = C[c] + wc;
      }
      T = T * (1.0f - a);
      nb++;
    }
    float out[4] = {C[0], C[1], C[2], 1.0f - T};
    for (int c = 0; c < 4; ++c) job->rgba[pixel_index * 4 + c] = out[c];
    if (job->nblend) job->nblend[pixel_index] = nb;
    if (job->margin) job->margin[pixel_index] = margin;
    if (job->count) job->count[pixel_index] = (uint32_t)n;
    return;
  }
  /* fp64 colours for the fp64 forward and the backward */
  const double* col64 = job->colors64;
  double cc[4];
  if (job->mode == 1) {
    double C[3] = {0, 0, 0}, A = 0;
    for (int64_t i = 0; i < n; ++i) {
      for (int c = 0; c < 4; ++c) cc[c] = col64 ? col64[f[i].j * 4 + c] : (double)s->colors[f[i].j * 4 + c];
      for (int c = 0; c < 3; ++c) C[c] = cc[3] * cc[c] + (1.0 - cc[3]) * C[c];
      A = cc[3] + (1.0 - cc[3]) * A;
    }
    for (int c = 0; c < 3; ++c) job->rgba64[pixel_index * 4 + c] = C[c];
    job->rgba64[pixel_index * 4 + 3] = A;
    return;
  }
  /* O.13 backward, front to back: T_i = prod over nearer (1 - a_k); B_i, Abeta_i =
   * composite colour / alpha of the fragments behind i. f[] is ascending (back first). */
  const double* g = job->grad_out + pixel_index * 4;
  double* gc = job->grad_colors + (int64_t)tid * s->num_quads * 4;
  /* behind-composites: walk back to front and record the composite before fragment i */
  double Bc[3] = {0, 0, 0}, Ba = 0;
  double* behind = (double*)malloc(sizeof(double) * 4 * (size_t)(n > 0 ? n : 1));
  for (int64_t i = 0; i < n; ++i) {
    for (int c = 0; c < 3; ++c) behind[i * 4 + c] = Bc[c];
    behind[i * 4 + 3] = Ba;
    for (int c = 0; c < 4; ++c) cc[c] = col64 ? col64[f[i].j * 4 + c] : (double)s->colors[f[i].j * 4 + c];
    for (int c = 0; c < 3; ++c) Bc[c] = cc[3] * cc[c] + (1.0 - cc[3]) * Bc[c];
    Ba = cc[3] + (1.0 - cc[3]) * Ba;
  }
  double T = 1.0;
  for (int64_t i = n - 1; i >= 0; --i) {
    for (int c = 0; c < 4; ++c) cc[c] = col64 ? col64[f[i].j * 4 + c] : (double)s->colors[f[i].j * 4 + c];
    double a = cc[3];
    double* gq = gc + (int64_t)f[i].j * 4;
    double ga = 0.0;
    for (int c = 0; c < 3; ++c) {
      gq[c] += g[c] * T * a;
      ga += g[c] * T * (cc[c] - behind[i * 4 + c]);
    }
    ga += g[3] * T * (1.0 - behind[i * 4 + 3]);
    gq[3] += ga;
    T *= (1.0 - a);
  }
  free(behind);
}

static void* band_worker(void* arg) {
  or_worker* wk = (or_worker*)arg;
  or_job* job = wk->job;
  const or_scene* s = job->s;
  size_t cap = 1 << 16;
  or_frag* frags = (or_frag*)malloc(cap * sizeof(or_frag));
  int64_t ties = 0, nfr = 0, maxd = 0;
  for (;;) {
    pthread_mutex_lock(&job->lock);
    int b = job->next_band++;
    pthread_mutex_unlock(&job->lock);
    if (b >= job->nbands) break;
    int y0 = b * job->band_rows;
    int y1 = y0 + job->band_rows - 1;
    if (y1 > s->height - 1) y1 = s->height - 1;
    size_t n = 0;
    for (int64_t li = job->band_start[b]; li < job->band_start[b + 1]; ++li) {
      int64_t j = job->band_list[li];
      const or_quad* qd = &job->quads[j];
      for (int t = 0; t < 2; ++t) {
        or_tri tri;
        make_tri(qd, t, s, &tri);
        if (!tri.ok) continue;
        int ya = tri.py0 > y0 ? tri.py0 : y0;
        int yb = tri.py1 < y1 ? tri.py1 : y1;
        for (int py = ya; py <= yb; ++py) {
          for (int px = tri.px0; px <= tri.px1; ++px) {
            float key, rgba[4];
            if (!shade(s, &tri, j, px, py, &key, rgba)) continue;
            if (n == cap) {
              cap *= 2;
              or_frag* nf = (or_frag*)realloc(frags, cap * sizeof(or_frag));
              if (!nf) { job->failed = 1; free(frags); return NULL; }
              frags = nf;
            }
            or_frag* f = &frags[n++];
            f->key = key; f->j = (uint32_t)j; f->t = (uint32_t)t;
            f->pix = (py - y0) * s->width + px;
            memcpy(f->rgba, rgba, sizeof(rgba));
          }
        }
      }
    }
    qsort(frags, n, sizeof(or_frag), frag_cmp);
    /* every pixel of the band, including empty ones */
    size_t i = 0;
    for (int py = y0; py <= y1; ++py) {
      for (int px = 0; px < s->width; ++px) {
        int32_t pl = (py - y0) * s->width + px;
        size_t k = i;
        while (k < n && frags[k].pix == pl) ++k;
        int64_t cnt = (int64_t)(k - i);
        composite_pixel(job, frags + i, cnt, (int64_t)py * s->width + px, wk->tid, &ties);
        nfr += cnt;
        if (cnt > maxd) maxd = cnt;
        i = k;
      }
    }
  }
  free(frags);
  pthread_mutex_lock(&job->lock);
  job->ties += ties;
  job->frags += nfr;
  if (maxd > job->max_depth) job->max_depth = maxd;
  pthread_mutex_unlock(&job->lock);
  return NULL;
}

static int resolve_threads(int nthreads) {
  if (nthreads > 0) return nthreads;
  long n = sysconf(_SC_NPROCESSORS_ONLN);
  return n > 0 ? (int)n : 1;
}

static int run_job(or_job* job, int nthreads, or_stats* st) {
  const or_scene* s = job->s;
  int64_t Q = s->num_quads;
  job->quads = (or_quad*)malloc(sizeof(or_quad) * (size_t)(Q > 0 ? Q : 1));
  if (!job->quads) return -1;
  int64_t by_status[8] = {0};
  for (int64_t j = 0; j < Q; ++j) {
    setup_quad(s, j, &job->quads[j]);
    by_status[job->quads[j].status]++;
  }
  job->band_rows = 4;
  job->nbands = (s->height + job->band_rows - 1) / job->band_rows;
  job->band_start = (int64_t*)calloc((size_t)job->nbands + 1, sizeof(int64_t));
  for (int64_t j = 0; j < Q; ++j) {
    const or_quad* qd = &job->quads[j];
    if (qd->status != OR_VISIBLE) continue;
    for (int b = qd->py0 / job->band_rows; b <= qd->py1 / job->band_rows; ++b) job->band_start[b + 1]++;
  }
  for (int b = 0; b < job->nbands; ++b) job->band_start[b + 1] += job->band_start[b];
  job->band_list = (int64_t*)malloc(sizeof(int64_t) * (size_t)(job->band_start[job->nbands] + 1));
  int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)(job->nbands + 1));
  memcpy(fill, job->band_start, sizeof(int64_t) * (size_t)(job->nbands + 1));
  for (int64_t j = 0; j < Q; ++j) {
    const or_quad* qd = &job->quads[j];
    if (qd->status != OR_VISIBLE) continue;
    for (int b = qd->py0 / job->band_rows; b <= qd->py1 / job->band_rows; ++b) job->band_list[fill[b]++] = j;
  }
  free(fill);
  nthreads = resolve_threads(nthreads);
  pthread_mutex_init(&job->lock, NULL);
  job->next_band = 0;
  pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)nthreads);
  or_worker* wk = (or_worker*)malloc(sizeof(or_worker) * (size_t)nthreads);
  for (int i = 0; i < nthreads; ++i) {
    wk[i].job = job; wk[i].tid = i;
    pthread_create(&th[i], NULL, band_worker, &wk[i]);
  }
  for (int i = 0; i < nthreads; ++i) pthread_join(th[i], NULL);
  pthread_mutex_destroy(&job->lock);
  free(th); free(wk);
  if (st) {
    memset(st, 0, sizeof(*st));
    for (int k = 0; k < 8; ++k) st->quads_by_status[k] = by_status[k];
    st->fragments = job->frags;
    st->max_depth = job->max_depth;
    st->key_ties = job->ties;
  }
  free(job->band_start); free(job->band_list); free(job->quads);
  return job->failed ? -1 : 0;
}

/* ---- exported entry points ----------------------------------------------------------- */

int or_setup(const or_scene* s, int32_t* status, int32_t* X, int32_t* Y, float* q, int32_t* bbox) {
  for (int64_t j = 0; j < s->num_quads; ++j) {
    or_quad qd;
    setup_quad(s, j, &qd);
    status[j] = qd.status;
    for (int k = 0; k < 4; ++k) {
      X[j * 4 + k] = qd.X[k];
      Y[j * 4 + k] = qd.Y[k];
      q[j * 4 + k] = qd.q[k];
    }
    bbox[j * 4 + 0] = qd.px0; bbox[j * 4 + 1] = qd.px1;
    bbox[j * 4 + 2] = qd.py0; bbox[j * 4 + 3] = qd.py1;
  }
  return 0;
}

int or_render(const or_scene* s, int nthreads, float* rgba, uint32_t* count, uint64_t* hash,
              uint8_t* rgba8, double* rgba64, or_stats* st) {
  or_job job;
  memset(&job, 0, sizeof(job));
  job.s = s; job.rgba = rgba; job.count = count; job.hash = hash; job.rgba8 = rgba8;
  job.rgba64 = rgba64; job.mode = 0;
  return run_job(&job, nthreads, st);
}

/* Alpha-threshold composite (see the header): rgba [H][W][4], per-pixel number of
 * fragments blended, per-pixel fragment count, and how close T came to t_min at the stop
 * tests (relative; a pixel with a small margin may stop one fragment earlier or later
 * under another rounding of its alphas). */
int or_render_threshold(const or_scene* s, int nthreads, float t_min, float* rgba, uint32_t* nblend,
                        uint32_t* count, float* margin) {
  if (!(t_min >= 0.0f && t_min < 1.0f)) return -2;
  or_job job;
  memset(&job, 0, sizeof(job));
  job.s = s; job.rgba = rgba; job.count = count; job.mode = 3;
  job.t_min = t_min; job.nblend = nblend; job.margin = margin;
  return run_job(&job, nthreads, NULL);
}

int or_render64(const or_scene* s, int nthreads, const double* colors64, double* rgba64) {
  if (s->color_mode != 0) return -2;
  or_job job;
  memset(&job, 0, sizeof(job));
  job.s = s; job.rgba64 = rgba64; job.colors64 = colors64; job.mode = 1;
  return run_job(&job, nthreads, NULL);
}

int or_backward(const or_scene* s, int nthreads, const double* colors64, const double* grad_out,
                double* grad_colors) {
  if (s->color_mode != 0) return -2;
  nthreads = resolve_threads(nthreads);
  int64_t Q = s->num_quads;
  double* per = (double*)calloc((size_t)nthreads * (size_t)(Q > 0 ? Q : 1) * 4, sizeof(double));
  if (!per) return -1;
  or_job job;
  memset(&job, 0, sizeof(job));
  job.s = s; job.colors64 = colors64; job.grad_out = grad_out; job.grad_colors = per; job.mode = 2;
  int rc = run_job(&job, nthreads, NULL);
  for (int64_t i = 0; i < Q * 4; ++i) {
    double acc = 0.0;
    for (int t = 0; t < nthreads; ++t) acc += per[(int64_t)t * Q * 4 + i];
    grad_colors[i] = acc;
  }
  free(per);
  return rc;
}

/* Selected pixels only: scans every quad for each requested pixel (O(Q) per pixel). */
typedef struct {
  const or_scene* s;
  const or_quad* quads;
  int64_t n;
  const int32_t* px;
  const int32_t* py;
  float* rgba;
  uint32_t* count;
  uint64_t* hash;
  pthread_mutex_t lock;
  int64_t next;
} or_pix_job;

static void* pixel_worker(void* arg) {
  or_pix_job* job = (or_pix_job*)arg;
  const or_scene* s = job->s;
  size_t cap = 1024;
  or_frag* frags = (or_frag*)malloc(cap * sizeof(or_frag));
  for (;;) {
    pthread_mutex_lock(&job->lock);
    int64_t i = job->next;
    job->next += 16;
    pthread_mutex_unlock(&job->lock);
    if (i >= job->n) break;
    int64_t iend = i + 16 < job->n ? i + 16 : job->n;
    for (; i < iend; ++i) {
      int32_t px = job->px[i], py = job->py[i];
      size_t n = 0;
      for (int64_t j = 0; j < s->num_quads; ++j) {
        const or_quad* qd = &job->quads[j];
        if (qd->status != OR_VISIBLE) continue;
        if (px < qd->px0 || px > qd->px1 || py < qd->py0 || py > qd->py1) continue;
        for (int t = 0; t < 2; ++t) {
          or_tri tri;
          make_tri(qd, t, s, &tri);
          if (!tri.ok) continue;
          float key, rgba[4];
          if (!shade(s, &tri, j, px, py, &key, rgba)) continue;
          if (n == cap) { cap *= 2; frags = (or_frag*)realloc(frags, cap * sizeof(or_frag)); }
          or_frag* f = &frags[n++];
          f->key = key; f->j = (uint32_t)j; f->t = (uint32_t)t; f->pix = 0;
          memcpy(f->rgba, rgba, sizeof(rgba));
        }
      }
      qsort(frags, n, sizeof(or_frag), frag_cmp);
      float C[3] = {0.f, 0.f, 0.f}, Aout = 0.f;
      uint64_t h = 0;
      for (size_t k = 0; k < n; ++k) {
        float a = frags[k].rgba[3];
        float om = 1.0f - a;
        for (int c = 0; c < 3; ++c) {
          float ac = a * frags[k].rgba[c];
          float keep = om * C[c];
          C[c] = ac + keep;
        }
        float keepa = om * Aout;
        Aout = a + keepa;
        h += splitmix64(2ull * frags[k].j + frags[k].t);
      }
      if (job->rgba) {
        job->rgba[i * 4 + 0] = C[0]; job->rgba[i * 4 + 1] = C[1];
        job->rgba[i * 4 + 2] = C[2]; job->rgba[i * 4 + 3] = Aout;
      }
      if (job->count) job->count[i] = (uint32_t)n;
      if (job->hash) job->hash[i] = h;
    }
  }
  free(frags);
  return NULL;
}

int or_render_pixels(const or_scene* s, int nthreads, int64_t n, const int32_t* px, const int32_t* py,
                     float* rgba, uint32_t* count, uint64_t* hash) {
  int64_t Q = s->num_quads;
  or_quad* quads = (or_quad*)malloc(sizeof(or_quad) * (size_t)(Q > 0 ? Q : 1));
  if (!quads) return -1;
  for (int64_t j = 0; j < Q; ++j) setup_quad(s, j, &quads[j]);
  or_pix_job job;
  memset(&job, 0, sizeof(job));
  job.s = s; job.quads = quads; job.n = n; job.px = px; job.py = py;
  job.rgba = rgba; job.count = count; job.hash = hash;
  pthread_mutex_init(&job.lock, NULL);
  nthreads = resolve_threads(nthreads);
  pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)nthreads);
  for (int i = 0; i < nthreads; ++i) pthread_create(&th[i], NULL, pixel_worker, &job);
  for (int i = 0; i < nthreads; ++i) pthread_join(th[i], NULL);
  pthread_mutex_destroy(&job.lock);
  free(th); free(quads);
  return 0;
}

/* The fully sorted fragment list of one pixel (back to front), for inspection by tests.
 * Returns the number of fragments; at most cap are written. */
int64_t or_pixel_fragments(const or_scene* s, int32_t px, int32_t py, int64_t cap, float* key,
                           uint32_t* quad, uint32_t* tri, float* rgba) {
  int64_t Q = s->num_quads;
  size_t n = 0, fcap = 64;
  or_frag* frags = (or_frag*)malloc(fcap * sizeof(or_frag));
  for (int64_t j = 0; j < Q; ++j) {
    or_quad qd;
    setup_quad(s, j, &qd);
    if (qd.status != OR_VISIBLE) continue;
    if (px < qd.px0 || px > qd.px1 || py < qd.py0 || py > qd.py1) continue;
    for (int t = 0; t < 2; ++t) {
      or_tri tr;
      make_tri(&qd, t, s, &tr);
      if (!tr.ok) continue;
      float k, c[4];
      if (!shade(s, &tr, j, px, py, &k, c)) continue;
      if (n == fcap) { fcap *= 2; frags = (or_frag*)realloc(frags, fcap * sizeof(or_frag)); }
      frags[n].key = k; frags[n].j = (uint32_t)j; frags[n].t = (uint32_t)t; frags[n].pix = 0;
      memcpy(frags[n].rgba, c, sizeof(c));
      ++n;
    }
  }
  qsort(frags, n, sizeof(or_frag), frag_cmp);
  for (size_t i = 0; i < n && (int64_t)i < cap; ++i) {
    key[i] = frags[i].key; quad[i] = frags[i].j; tri[i] = frags[i].t;
    memcpy(rgba + 4 * i, frags[i].rgba, 4 * sizeof(float));
  }
  free(frags);
  return (int64_t)n;
}

int or_num_threads(int nthreads) { return resolve_threads(nthreads); }
